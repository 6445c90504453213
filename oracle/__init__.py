"""Oracle: plain single-threaded FP64 reference for the channel-flow Poisson and
z-implicit Helmholtz solves of Diez, Peeters & Costa (arXiv 2502.06296).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package never
imports this module and shares no code with it.

The arithmetic lives in ``chanfs_oracle.c`` (compiled with ``-O2
-ffp-contract=off``); this module only compiles it on demand and marshals numpy
arrays through ctypes.  Every C function cites the passage of the paper it
follows.
"""

from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chanfs_oracle.c")
_HDR = os.path.join(_HERE, "chanfs_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libchanfs_oracle.so")

NEUMANN, DIRICHLET = 0, 1
CENTER, FACE = 0, 1
THOMAS, ALG2, ALG1 = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C11) if it is stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    lock = _LIB + ".lock"
    with open(lock, "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "or_dft_naive": [i, dp, dp, i],
            "or_fft": [i, dp, dp, i],
            "or_rfft_packed": [i, dp, dp],
            "or_irfft_packed": [i, dp, dp],
            "or_packed_wavenumber": [i, i],
            "or_eig_periodic": [i, d, dp],
            "or_eig_packed": [i, d, dp],
            "or_dzc": [i, dp, dp],
            "or_lz_coefficients": [i, dp, i, i, dp, dp, dp],
            "or_thomas": [i, dp, dp, dp, dp, dp],
            "or_alg1_solve": [i, i, dp, dp, dp, dp, dp],
            "or_alg2_prepare": [i, dp, dp, dp, dp, dp, dp],
            "or_alg2_runtime": [i, dp, dp, dp, dp],
            "or_alg2_reconstruct": [i, dp, dp, dp, d, d, dp],
            "or_alg2_solve": [i, i, dp, dp, dp, dp, dp],
            "or_apply_poisson": [i, i, i, d, d, dp, i, dp, dp],
            "or_apply_helmholtz": [i, i, i, dp, d, i, dp, dp],
            "or_poisson_solve": [i, i, i, d, d, dp, i, dp, dp],
            "or_helmholtz_solve": [i, i, i, dp, d, i, i, i, dp, dp],
            "or_apply_helmholtz3d": [i, i, i, d, d, dp, d, i, dp, dp],
            "or_dct2": [i, dp, dp],
            "or_idct2": [i, dp, dp],
            "or_dst2": [i, dp, dp],
            "or_idst2": [i, dp, dp],
            "or_eig_wall": [i, d, i, dp],
            "or_apply_poisson_walls": [i, i, i, d, d, dp, i, i, dp, dp],
            "or_poisson_solve_walls": [i, i, i, d, d, dp, i, i, dp, dp],
            "or_helmholtz3d_solve": [i, i, i, d, d, dp, d, i, dp, dp],
            "or_apply_helmholtz3d_walls": [i, i, i, d, d, dp, d, i, i, dp, dp],
            "or_helmholtz3d_solve_walls": [i, i, i, d, d, dp, d, i, i, dp, dp],
            "or_spectral_forward": [i, i, i, dp, dp],
            "or_spectral_inverse": [i, i, i, dp, dp],
            "or_dense_solve": [i, dp, dp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, name: str) -> int:
    if rc < 0:
        raise ValueError(f"oracle {name} rejected its arguments (rc={rc})")
    return rc


# --- transforms -------------------------------------------------------------

def dft_naive(x, sign: int = -1) -> np.ndarray:
    x = _c128(x)
    out = np.empty_like(x)
    _check(_load().or_dft_naive(x.size, _p(x.view(np.float64)), _p(out.view(np.float64)), sign), "dft")
    return out


def fft(x, sign: int = -1) -> np.ndarray:
    x = _c128(x)
    out = np.empty_like(x)
    _check(_load().or_fft(x.size, _p(x.view(np.float64)), _p(out.view(np.float64)), sign), "fft")
    return out


def rfft_packed(x) -> np.ndarray:
    x = _f64(x)
    out = np.empty_like(x)
    _check(_load().or_rfft_packed(x.size, _p(x), _p(out)), "rfft_packed")
    return out


def irfft_packed(packed) -> np.ndarray:
    packed = _f64(packed)
    out = np.empty_like(packed)
    _check(_load().or_irfft_packed(packed.size, _p(packed), _p(out)), "irfft_packed")
    return out


def packed_wavenumber(n: int, slot: int) -> int:
    return _check(_load().or_packed_wavenumber(n, slot), "packed_wavenumber")


def eig_periodic(n: int, h: float) -> np.ndarray:
    out = np.empty(n)
    _check(_load().or_eig_periodic(n, h, _p(out)), "eig_periodic")
    return out


def eig_packed(n: int, h: float) -> np.ndarray:
    out = np.empty(n)
    _check(_load().or_eig_packed(n, h, _p(out)), "eig_packed")
    return out


# --- z stencil and 1-D solvers ------------------------------------------------

def dzc(dzf) -> np.ndarray:
    dzf = _f64(dzf)
    out = np.empty(dzf.size - 1)
    _check(_load().or_dzc(dzf.size, _p(dzf), _p(out)), "dzc")
    return out


def lz_coefficients(dzf, bc: int, loc: int):
    """(A, B, C) of the z stencil; length Nz (centred) or Nz-1 (face)."""
    dzf = _f64(dzf)
    nz = dzf.size
    A, B, C = np.zeros(nz), np.zeros(nz), np.zeros(nz)
    n = _check(_load().or_lz_coefficients(nz, _p(dzf), bc, loc, _p(A), _p(B), _p(C)), "lz")
    return A[:n].copy(), B[:n].copy(), C[:n].copy()


def thomas(a, b, c, d) -> np.ndarray:
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    _check(_load().or_thomas(d.size, _p(a), _p(b), _p(c), _p(d), _p(x)), "thomas")
    return x


def alg1_solve(a, b, c, d, p: int) -> np.ndarray:
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    _check(_load().or_alg1_solve(d.size, p, _p(a), _p(b), _p(c), _p(d), _p(x)), "alg1")
    return x


def alg2_solve(A, B, C, d, p: int) -> np.ndarray:
    A, B, C, d = map(_f64, (A, B, C, d))
    x = np.empty_like(d)
    _check(_load().or_alg2_solve(d.size, p, _p(A), _p(B), _p(C), _p(d), _p(x)), "alg2")
    return x


def alg2_prepare(A, B, C):
    A, B, C = map(_f64, (A, B, C))
    a, b, c = np.empty_like(A), np.empty_like(A), np.empty_like(A)
    _check(_load().or_alg2_prepare(A.size, _p(A), _p(B), _p(C), _p(a), _p(b), _p(c)), "alg2_prepare")
    return a, b, c


def alg2_runtime(A, C, b, d) -> np.ndarray:
    A, C, b = map(_f64, (A, C, b))
    d = _f64(d).copy()
    _check(_load().or_alg2_runtime(d.size, _p(A), _p(C), _p(b), _p(d)), "alg2_runtime")
    return d


def alg2_reconstruct(a, b, c, d, x0: float, xm1: float) -> np.ndarray:
    a, b, c = map(_f64, (a, b, c))
    d = _f64(d).copy()
    _check(_load().or_alg2_reconstruct(d.size, _p(a), _p(b), _p(c), x0, xm1, _p(d)), "alg2_rec")
    return d


def dense_solve(A, b) -> np.ndarray:
    A = _f64(A).copy()
    b = _f64(b).copy()
    _check(_load().or_dense_solve(b.size, _p(A), _p(b)), "dense_solve")
    return b


# --- 3-D operators and solvers (fields shaped (Nz, Ny, Nx), x fastest) -------

def _shape(f):
    if f.ndim != 3:
        raise ValueError("fields are (Nz, Ny, Nx) arrays")
    nz, ny, nx = f.shape
    return nx, ny, nz


def apply_poisson(p, lx: float, ly: float, dzf, bc: int) -> np.ndarray:
    p, dzf = _f64(p), _f64(dzf)
    nx, ny, nz = _shape(p)
    out = np.empty_like(p)
    _check(_load().or_apply_poisson(nx, ny, nz, lx, ly, _p(dzf), bc, _p(p), _p(out)), "apply_poisson")
    return out


def apply_helmholtz(u, dzf, c: float, loc: int) -> np.ndarray:
    u, dzf = _f64(u), _f64(dzf)
    nx, ny, nz = _shape(u)
    out = np.empty_like(u)
    _check(_load().or_apply_helmholtz(nx, ny, nz, _p(dzf), c, loc, _p(u), _p(out)), "apply_helmholtz")
    return out


def poisson_solve(f, lx: float, ly: float, dzf, bc: int) -> np.ndarray:
    f, dzf = _f64(f), _f64(dzf)
    nx, ny, nz = _shape(f)
    out = np.empty_like(f)
    _check(_load().or_poisson_solve(nx, ny, nz, lx, ly, _p(dzf), bc, _p(f), _p(out)), "poisson")
    return out


def helmholtz_solve(rhs, dzf, c: float, loc: int, method: int = THOMAS, nparts: int = 1) -> np.ndarray:
    rhs, dzf = _f64(rhs), _f64(dzf)
    nx, ny, nz = _shape(rhs)
    out = np.empty_like(rhs)
    _check(_load().or_helmholtz_solve(nx, ny, nz, _p(dzf), c, loc, method, nparts, _p(rhs), _p(out)),
           "helmholtz")
    return out


Y_PERIODIC, Y_NEUMANN, Y_DIRICHLET = 0, 1, 2


def _r2r(name, x):
    x = _f64(x)
    out = np.empty_like(x)
    _check(getattr(_load(), name)(x.size, _p(x), _p(out)), name)
    return out


def dct2(x):
    """DCT-II by its definition: X_k = sum_j x_j cos(pi k (j + 1/2) / n)."""
    return _r2r("or_dct2", x)


def idct2(X):
    return _r2r("or_idct2", X)


def dst2(x):
    """DST-II by its definition: X_k = sum_j x_j sin(pi (k + 1)(j + 1/2) / n)."""
    return _r2r("or_dst2", x)


def idst2(X):
    return _r2r("or_idst2", X)


def eig_wall(n: int, h: float, ybc: int) -> np.ndarray:
    out = np.empty(n)
    _check(_load().or_eig_wall(n, h, ybc, _p(out)), "eig_wall")
    return out


def apply_poisson_walls(p, lx: float, ly: float, dzf, bc: int, ybc: int) -> np.ndarray:
    p, dzf = _f64(p), _f64(dzf)
    nx, ny, nz = _shape(p)
    out = np.empty_like(p)
    _check(_load().or_apply_poisson_walls(nx, ny, nz, lx, ly, _p(dzf), bc, ybc, _p(p), _p(out)),
           "apply_poisson_walls")
    return out


def poisson_solve_walls(f, lx: float, ly: float, dzf, bc: int, ybc: int) -> np.ndarray:
    f, dzf = _f64(f), _f64(dzf)
    nx, ny, nz = _shape(f)
    out = np.empty_like(f)
    _check(_load().or_poisson_solve_walls(nx, ny, nz, lx, ly, _p(dzf), bc, ybc, _p(f), _p(out)),
           "poisson_solve_walls")
    return out


def apply_helmholtz3d(u, lx: float, ly: float, dzf, c: float, loc: int, ybc: int = 0) -> np.ndarray:
    """(I - c L) u, the full 3-D operator of Eq. 8 with Dirichlet z walls."""
    u, dzf = _f64(u), _f64(dzf)
    nx, ny, nz = _shape(u)
    out = np.empty_like(u)
    _check(_load().or_apply_helmholtz3d_walls(nx, ny, nz, lx, ly, _p(dzf), c, loc, ybc, _p(u),
                                              _p(out)), "apply_helmholtz3d")
    return out


def helmholtz3d_solve(rhs, lx: float, ly: float, dzf, c: float, loc: int, ybc: int = 0) -> np.ndarray:
    """u with (I - c L) u = rhs (Eq. 8) by eigenfunction expansion."""
    rhs, dzf = _f64(rhs), _f64(dzf)
    nx, ny, nz = _shape(rhs)
    out = np.empty_like(rhs)
    _check(_load().or_helmholtz3d_solve_walls(nx, ny, nz, lx, ly, _p(dzf), c, loc, ybc, _p(rhs),
                                              _p(out)), "helmholtz3d")
    return out


def spectral_forward(f) -> np.ndarray:
    """Packed-x / complex-y spectrum, returned as complex (Nz, Ny, Nx/2)."""
    f = _f64(f)
    nx, ny, nz = _shape(f)
    out = np.empty((nz, ny, nx // 2), dtype=np.complex128)
    _check(_load().or_spectral_forward(nx, ny, nz, _p(f), _p(out.view(np.float64))), "spectral_fwd")
    return out


def spectral_inverse(s) -> np.ndarray:
    s = _c128(s)
    nz, ny, m = s.shape
    out = np.empty((nz, ny, 2 * m))
    _check(_load().or_spectral_inverse(2 * m, ny, nz, _p(s.view(np.float64)), _p(out)), "spectral_inv")
    return out
