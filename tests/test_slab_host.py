"""The z-slab decomposition's exchange (Sec. 2.2.3, P-TDMA) among 2 and 4
gloo ranks on the CPU, no GPU involved.

Each rank takes the planes the library assigns it (cfs_slab_partition),
runs Step 2 of Algorithm 2 on them with the oracle's routines (standing in
for the library's device kernels), and exchanges its two boundary values per
column through the library's own gather (paper_2502_06296_gb300.slab, the
call the multi-GPU solve uses, here over gloo).  Each rank then assembles the
2p reduced system of every column from the gathered rows in the library's
layout (rank-major; rank r's first and last rows are rows 2r and 2r + 1),
solves it, and reconstructs its planes.  The gathered result must equal the
oracle's direct solves: Thomas and Algorithm 2 for the Helmholtz columns of
Eq. 11, and the Poisson solve of Eq. 12 with Dirichlet walls (the x and y
transforms of each rank's planes by numpy's FFT).
"""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import chanfs, synth

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _partitions(nz, world, n):
    """Row ranges of every rank: the library's planes, a face field's last
    one ending below the top wall (n rows in all)."""
    parts = [list(chanfs.slab_partition(nz, world, r)) for r in range(world)]
    parts[-1][1] = n
    return parts


def _reduced_solve(parts, A, B, C, bnd_all, rank):
    """Every column's reduced system from the gathered boundary rows; returns
    this rank's (x_0, x_{m-1}) per column, shapes (ncols,)."""
    world = len(parts)
    ra, rb, rc = np.zeros(2 * world), np.zeros(2 * world), np.zeros(2 * world)
    for q, (s, e) in enumerate(parts):
        a, b, c = oracle.alg2_prepare(A[s:e], B[s:e], C[s:e])
        ra[2 * q], rb[2 * q], rc[2 * q] = a[0], b[0], c[0]
        ra[2 * q + 1], rb[2 * q + 1], rc[2 * q + 1] = a[-1], b[-1], c[-1]
    rd = bnd_all.reshape(world * 2, -1)  # row 2q + t: rank q's boundary t
    x = np.stack([oracle.thomas(ra, rb, rc, rd[:, k]) for k in range(rd.shape[1])], axis=1)
    return x[2 * rank], x[2 * rank + 1]


def _helmholtz_rank(rank, world, nz, loc, c):
    from paper_2502_06296_gb300 import slab
    import torch.distributed as dist
    dz = synth.tanh_dz(nz, 1.6)
    A, B, C = oracle.lz_coefficients(dz, oracle.DIRICHLET, loc)
    A, B, C = -c * A, 1.0 - c * B, -c * C  # I - c L_z (Eq. 11)
    n = B.size
    ncols = 6
    rhs = synth.normal(40 + nz + loc, (n, ncols))  # the same seeded field on every rank
    parts = _partitions(nz, world, n)
    s, e = parts[rank]
    a, b, cc = oracle.alg2_prepare(A[s:e], B[s:e], C[s:e])
    dp = np.stack([oracle.alg2_runtime(A[s:e], C[s:e], b, rhs[s:e, k]) for k in range(ncols)], 1)
    bnd = torch.from_numpy(np.concatenate([dp[0], dp[-1]]))  # [2][ncols]
    bnd_all = slab.gather_boundaries(bnd).numpy()
    assert bnd_all.size == world * 2 * ncols
    x0, xm = _reduced_solve(parts, A, B, C, bnd_all, rank)
    mine = np.stack([oracle.alg2_reconstruct(a, b, cc, dp[:, k], x0[k], xm[k])
                     for k in range(ncols)], 1)
    pieces = [None] * world
    dist.all_gather_object(pieces, mine)
    x = np.concatenate(pieces)
    ref = np.stack([oracle.thomas(A, B, C, rhs[:, k]) for k in range(ncols)], 1)
    ref2 = np.stack([oracle.alg2_solve(A, B, C, rhs[:, k], world) for k in range(ncols)], 1)
    return (float(np.max(np.abs(x - ref)) / np.max(np.abs(ref))),
            float(np.max(np.abs(x - ref2)) / np.max(np.abs(ref2))))


def _poisson_rank(rank, world, nx, ny, nz):
    from paper_2502_06296_gb300 import slab
    import torch.distributed as dist
    lx, ly = 2.0, 1.5
    dz = synth.tanh_dz(nz, 1.7)
    f = synth.normal(77, (nz, ny, nx))
    A, B, C = oracle.lz_coefficients(dz, oracle.DIRICHLET, oracle.CENTER)
    lamx = oracle.eig_periodic(nx, lx / nx)
    lamy = oracle.eig_periodic(ny, ly / ny)
    parts = _partitions(nz, world, nz)
    s, e = parts[rank]
    F = np.fft.fft2(f[s:e])  # the rank's planes, transformed along y and x
    dp = np.empty_like(F)
    shifted = {}
    for ky in range(ny):
        for kx in range(nx):
            Bk = B + lamx[kx] + lamy[ky]
            a, b, cc = oracle.alg2_prepare(A[s:e], Bk[s:e], C[s:e])
            shifted[ky, kx] = (Bk, a, b, cc)
            dp[:, ky, kx] = (oracle.alg2_runtime(A[s:e], C[s:e], b, F[:, ky, kx].real) +
                             1j * oracle.alg2_runtime(A[s:e], C[s:e], b, F[:, ky, kx].imag))
    bnd = torch.from_numpy(np.stack([dp[0], dp[-1]]).view(np.float64).ravel())
    bnd_all = slab.gather_boundaries(bnd).numpy().view(np.complex128).reshape(world, 2, ny, nx)
    out = np.empty_like(F)
    for ky in range(ny):
        for kx in range(nx):
            Bk, a, b, cc = shifted[ky, kx]
            col = bnd_all[:, :, ky, kx].reshape(-1)
            re = _reduced_solve(parts, A, Bk, C, col.real.copy(), rank)
            im = _reduced_solve(parts, A, Bk, C, col.imag.copy(), rank)
            out[:, ky, kx] = (oracle.alg2_reconstruct(a, b, cc, dp[:, ky, kx].real, re[0][0], re[1][0])
                              + 1j * oracle.alg2_reconstruct(a, b, cc, dp[:, ky, kx].imag,
                                                             im[0][0], im[1][0]))
    mine = np.fft.ifft2(out).real
    pieces = [None] * world
    dist.all_gather_object(pieces, mine)
    p = np.concatenate(pieces)
    ref = oracle.poisson_solve(f, lx, ly, dz, oracle.DIRICHLET)
    return float(np.max(np.abs(p - ref)) / np.max(np.abs(ref)))


def _rank_main(rank, world, port, queue, job):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        kind, args = job
        res = _helmholtz_rank(rank, world, *args) if kind == "helmholtz" else \
            _poisson_rank(rank, world, *args)
        queue.put((rank, res))
    finally:
        dist.destroy_process_group()


def _run(world, job):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, job)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == list(range(world))
    return [o[1] for o in out]


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("nz,loc,c", [(24, 0, 1e-3), (25, 1, 2e-4), (41, 0, 9.6e-9)])
def test_slab_exchange_helmholtz(world, nz, loc, c):
    for thomas_err, alg2_err in _run(world, ("helmholtz", (nz, loc, c))):
        assert thomas_err < 1e-12 and alg2_err < 1e-12


@pytest.mark.parametrize("world", [2, 4])
def test_slab_exchange_poisson(world):
    for err in _run(world, ("poisson", (8, 6, 19))):
        assert err < 1e-12


def test_slab_partition_rule():
    """Every plane in exactly one slab, in rank order, the library's rule."""
    for nz, world in ((384, 2), (41, 3), (30, 8), (16, 4)):
        parts = [chanfs.slab_partition(nz, world, r) for r in range(world)]
        assert parts[0][0] == 0 and parts[-1][1] == nz
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        assert all(e - s in (nz // world, nz // world + 1) for s, e in parts)
    with pytest.raises(chanfs.ChanfsError):
        chanfs.slab_partition(40, 2, 2)
