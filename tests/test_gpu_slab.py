"""GPU: the z-slab solves (Sec. 2.2.3, P-TDMA) through the C ABI, against the
oracle.

One GPU holds every rank's slab here, in one process: each slab's reduce
call runs, the boundary buffers are concatenated rank-major (what the
all-gather of a multi-GPU run delivers), and each slab's finish call runs.
No kernel waits for another.  The stacked planes must match the oracle's
whole-field solve element by element at 1e-12 (relative max-norm): Poisson
with Neumann (the singular (0, 0) column's projections from every rank's
partial sums) and Dirichlet walls, Helmholtz for cell-centred and
face-located fields, even and uneven slabs, 1 to 4 ranks.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def chanfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_06296_gb300 import build as libbuild
    libbuild.build()
    from paper_2502_06296_gb300 import chanfs as c
    c.lib()
    return c


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def slabs(chanfs, nx, ny, nz, lx, ly, dz, bc, R):
    return [chanfs.Slab(nx, ny, nz, lx, ly, dz, bc, R, r) for r in range(R)]


@pytest.mark.parametrize("R", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [0, 1])
def test_slab_poisson_matches_oracle(chanfs, R, bc):
    nx, ny, nz, lx, ly = 32, 24, 41, 2.0, 1.5
    dz = synth.tanh_dz(nz, 1.7)
    f = synth.normal(300 + R + bc, (nz, ny, nx))
    if bc == chanfs.NEUMANN:
        f = synth.remove_weighted_mean(f, dz)
    ref = oracle.poisson_solve(f, lx, ly, dz, bc)
    ss = slabs(chanfs, nx, ny, nz, lx, ly, dz, bc, R)
    fl = [dev(f[s.z0:s.z1]) for s in ss]
    work = [torch.empty_like(x) for x in fl]
    bnd = [torch.empty(s.boundary_doubles(chanfs.REQ_POISSON), dtype=torch.float64, device="cuda")
           for s in ss]
    for s, x, w, b in zip(ss, fl, work, bnd):
        s.poisson_reduce(x, w, b)
    bnd_all = torch.cat(bnd)
    outs = [torch.empty_like(x) for x in fl]
    for s, w, o in zip(ss, work, outs):
        s.poisson_finish(bnd_all, w, o)
    torch.cuda.synchronize()
    p = np.concatenate([o.cpu().numpy() for o in outs])
    assert rel(p, ref) < TOL, rel(p, ref)
    # the single-GPU plan agrees too
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc) as plan:
        assert rel(p, plan.poisson_solve(dev(f)).cpu().numpy()) < TOL
    for s in ss:
        s.close()


@pytest.mark.parametrize("R", [1, 2, 4])
@pytest.mark.parametrize("loc,c", [(0, 9.615e-9), (1, 1e-4), (0, 1e-2)])
def test_slab_helmholtz_matches_oracle(chanfs, R, loc, c):
    nx, ny, nz = 16, 12, 48
    dz = synth.tanh_dz(nz, 1.8)
    rhs = synth.normal(400 + R + loc, (nz, ny, nx))
    ref = oracle.helmholtz_solve(rhs, dz, c, loc)
    ss = slabs(chanfs, nx, ny, nz, 1.0, 1.0, dz, 0, R)
    rl = [dev(rhs[s.z0:s.z1]) for s in ss]
    work = [torch.empty_like(x) for x in rl]
    bnd = [torch.empty(s.boundary_doubles(chanfs.REQ_HELMHOLTZ), dtype=torch.float64,
                       device="cuda") for s in ss]
    for s, x, w, b in zip(ss, rl, work, bnd):
        s.helmholtz_reduce(c, loc, x, w, b)
    bnd_all = torch.cat(bnd)
    outs = [torch.full_like(x, np.nan) for x in rl]
    for s, w, o in zip(ss, work, outs):
        s.helmholtz_finish(c, loc, bnd_all, w, o)
    torch.cuda.synchronize()
    u = np.concatenate([o.cpu().numpy() for o in outs])
    assert rel(u, ref) < TOL, rel(u, ref)
    if loc == 1:
        assert np.all(u[-1] == 0.0)
    for s in ss:
        s.close()


def test_slab_solver_single_rank_and_argument_checks(chanfs):
    from paper_2502_06296_gb300 import slab
    nx, ny, nz = 16, 12, 20
    dz = synth.tanh_dz(nz, 1.5)
    f = synth.remove_weighted_mean(synth.normal(9, (nz, ny, nx)), dz)
    solver = slab.SlabSolver(nx, ny, nz, 2.0, 1.0, dz)  # no process group: one rank
    p = solver.poisson_solve(dev(f)).cpu().numpy()
    assert rel(p, oracle.poisson_solve(f, 2.0, 1.0, dz, 0)) < TOL
    u = solver.helmholtz_solve(1e-4, dev(f), chanfs.FACE).cpu().numpy()
    assert rel(u, oracle.helmholtz_solve(f, dz, 1e-4, 1)) < TOL
    solver.close()
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.Slab(nx, ny, 12, 2.0, 1.0, np.full(12, 0.1), 0, 4, 0)  # 3 planes per slab
    assert err.value.status == chanfs.EUNSUPPORTED
    with pytest.raises(chanfs.ChanfsError):
        chanfs.Slab(nx, ny, nz, 2.0, 1.0, dz, 0, 2, 2)  # rank outside
