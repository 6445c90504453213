"""Seeded synthetic inputs: right-hand-side fields and wall-normal grids.

This module holds no arithmetic of the solver.  It turns a seed into the
bit-identical host arrays that both the CUDA library and the CPU reference
receive, so that the two never draw their own random numbers.

Generator: splitmix64 (Steele, Lea & Flood 2014) as a counter-based stream --
element i of stream ``seed`` is splitmix64's output for state
``seed + (i + 1) * 0x9E3779B97F4A7C15`` -- mapped to uniform doubles on [0, 1)
from the top 53 bits, and to N(0, 1) by the Box-Muller transform on consecutive
pairs.
"""

from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of the counter-based splitmix64 stream starting at ``offset``."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, n)).reshape(shape)


def normal(seed: int, shape) -> np.ndarray:
    """i.i.d. N(0,1) by Box-Muller on pairs (u1, u2) of the uniform stream."""
    n = int(np.prod(shape))
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
    t = 2.0 * np.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:n].reshape(shape)


def tanh_faces(nz: int, beta: float) -> np.ndarray:
    """Wall-clustered faces z_k = tanh(beta (2k/nz - 1)) / tanh(beta), k = 0..nz."""
    k = np.arange(nz + 1, dtype=np.float64)
    return np.tanh(beta * (2.0 * k / nz - 1.0)) / np.tanh(beta)


def tanh_dz(nz: int, beta: float) -> np.ndarray:
    """Cell widths of the tanh-stretched grid on [-1, 1] (they sum to 2)."""
    return np.diff(tanh_faces(nz, beta))


def uniform_dz(nz: int, lz: float = 2.0) -> np.ndarray:
    return np.full(nz, lz / nz)


def remove_weighted_mean(f: np.ndarray, dz: np.ndarray) -> np.ndarray:
    """Input conditioning for Neumann right-hand sides: subtract the
    cell-volume-weighted mean so that the field is compatible."""
    w = np.asarray(dz)[:, None, None]
    mean = float((f * w).sum() / (w.sum() * f.shape[1] * f.shape[2]))
    return f - mean


# --- the workloads ---------------------------------------------------------------
# 32^3 uniform Poisson (Lx = 2 pi, Ly = pi, Lz = 2), and the channel-shaped
# 512 x 384 x 384 step on the tanh(1.8) grid.  The channel box length and width
# follow the paper's channel runs (12.8 x 6.4 x 2).

SMALL = dict(name="poisson_uniform_32x32x32", nx=32, ny=32, nz=32, lx=2 * np.pi, ly=np.pi,
             beta=None, seed=20250206)
CHANNEL = dict(name="channel_512x384x384_tanh1.8", nx=512, ny=384, nz=384, lx=12.8, ly=6.4,
               beta=1.8, seed=2502063)
# The precision workload: the 32^3 physics (uniform grid, 2 pi x pi x 2,
# Neumann walls, uniform[-1, 1] right-hand side minus its mean) at 1024 x 768 x 512.
PRECISION = dict(name="poisson_uniform_1024x768x512", nx=1024, ny=768, nz=512, lx=2 * np.pi,
                 ly=np.pi, beta=None, seed=20250207)
# The paper's per-GPU machine of its weak-scaling runs (3456 x 3072 x 30), on one
# GPU: a thin wall-normal direction (tanh 1.8 grid), the channel's box lengths.
STRESS = dict(name="stress_3456x3072x30_tanh1.8", nx=3456, ny=3072, nz=30, lx=12.8, ly=6.4,
              beta=1.8, seed=2502066)
# Helmholtz coefficient of Eq. (11): alpha * nu * dt with alpha = 0.5, nu = 1/5200, dt = 1e-4.
CHANNEL_C = 0.5 * (1.0 / 5200.0) * 1e-4


# Batched ensemble: 48 boxes drawn from a seed (sizes from the menus below,
# tanh stretching in [1.2, 2.2], Helmholtz alpha nu dt log-uniform in [1e-6, 1e-4]).
ENSEMBLE = dict(name="ensemble_48_boxes", nbox=48, nx=(128, 192, 256, 384), ny=(96, 128, 192),
                nz=(64, 96, 128, 192), beta=(1.2, 2.2), c=(1e-6, 1e-4), seed=2502064,
                lx=12.8, ly=6.4)
# Serving stream: 20,000 requests, Poisson arrivals at 2,000 per second from 32
# runs with sizes drawn per axis from the menu, 1:3 Poisson:Helmholtz.
SERVING = dict(name="serving_20000_requests", nreq=20000, rate=2000.0, nruns=32,
               sizes=(64, 96, 128, 192, 256, 384, 512), beta=(1.2, 2.2), c=(1e-6, 1e-4),
               poisson_share=0.25, budget_gb=120, seed=2502065, lx=12.8, ly=6.4)


def _draw(seed: int, n: int, offset: int) -> np.ndarray:
    return uniform01(seed, n, offset)


def ensemble_boxes(cfg=ENSEMBLE):
    """[(nx, ny, nz, beta, c)] of the ensemble, from the counter stream."""
    nb = cfg["nbox"]
    u = _draw(cfg["seed"], 5 * nb, 0).reshape(nb, 5)
    out = []
    for b in range(nb):
        pick = lambda menu, x: menu[min(int(x * len(menu)), len(menu) - 1)]
        lo, hi = cfg["beta"]
        clo, chi = cfg["c"]
        out.append((pick(cfg["nx"], u[b, 0]), pick(cfg["ny"], u[b, 1]), pick(cfg["nz"], u[b, 2]),
                    lo + (hi - lo) * u[b, 3], clo * (chi / clo) ** u[b, 4]))
    return out


def serving_stream(cfg=SERVING):
    """Runs [(nx, ny, nz, beta, (c0, c1, c2))] and requests
    [(arrival_s, run, kind 0 Poisson / 1 Helmholtz, which c, loc)]."""
    nr, nq = cfg["nruns"], cfg["nreq"]
    u = _draw(cfg["seed"], 7 * nr, 0).reshape(nr, 7)
    menu = cfg["sizes"]
    pick = lambda x: menu[min(int(x * len(menu)), len(menu) - 1)]
    lo, hi = cfg["beta"]
    clo, chi = cfg["c"]
    runs = [(pick(u[r, 0]), pick(u[r, 1]), pick(u[r, 2]), lo + (hi - lo) * u[r, 3],
             tuple(clo * (chi / clo) ** u[r, 4 + k] for k in range(3))) for r in range(nr)]
    v = _draw(cfg["seed"], 5 * nq, 7 * nr).reshape(nq, 5)
    gaps = -np.log1p(-v[:, 0]) / cfg["rate"]  # exponential inter-arrival times
    t = np.cumsum(gaps)
    reqs = []
    for i in range(nq):
        kind = 0 if v[i, 2] < cfg["poisson_share"] else 1
        reqs.append((float(t[i]), min(int(v[i, 1] * nr), nr - 1), kind,
                     min(int(v[i, 3] * 3), 2), 0 if v[i, 4] < 2.0 / 3.0 else 1))
    return runs, reqs


def grid_dz(cfg) -> np.ndarray:
    return uniform_dz(cfg["nz"]) if cfg["beta"] is None else tanh_dz(cfg["nz"], cfg["beta"])


def small_rhs(cfg=SMALL) -> np.ndarray:
    """Uniform[-1, 1] with its mean removed (uniform grid: plain mean)."""
    f = uniform(cfg["seed"], (cfg["nz"], cfg["ny"], cfg["nx"]))
    return f - f.mean()


def channel_fields(cfg=CHANNEL):
    """Poisson RHS (N(0,1), zero weighted mean) and three Helmholtz RHS fields."""
    shape = (cfg["nz"], cfg["ny"], cfg["nx"])
    dz = grid_dz(cfg)
    f = remove_weighted_mean(normal(cfg["seed"], shape), dz)
    rhs = [normal(cfg["seed"] + 1 + i, shape) for i in range(3)]
    return f, rhs


def precision_rhs(cfg=PRECISION) -> np.ndarray:
    """Uniform[-1, 1] with its mean removed, as for the 32^3 workload."""
    f = uniform(cfg["seed"], (cfg["nz"], cfg["ny"], cfg["nx"]))
    f -= f.mean()
    return f
