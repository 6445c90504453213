"""GPU: walls in y (DCT-II for Neumann, DST-II for Dirichlet walls, each by
one complex FFT of length Ny), against the FP64 CPU oracle, which sums the
transforms by their definitions.

Tolerance: 1e-12 relative max-norm for FP64 plans, 1e-10 for refined plans.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rhs_for(nx, ny, nz, dz, bc, ybc, seed):
    f = synth.normal(seed, (nz, ny, nx))
    if bc == 0 and ybc == 1:  # the constants are the null space: compatible rhs
        f = synth.remove_weighted_mean(f, dz)
    return f


# even and odd Ny, Ny = 1, two TMA boxes along y (Ny > 256), ragged y tiles
WALL_CASES = [
    ((32, 24, 20), 1.8, 0, 1), ((32, 24, 20), 1.8, 1, 1), ((32, 24, 20), 1.8, 0, 2),
    ((32, 24, 20), 1.8, 1, 2), ((6, 9, 5), 1.2, 0, 1), ((6, 27, 5), 1.2, 1, 2),
    ((24, 288, 6), 1.5, 0, 1), ((24, 288, 6), 1.5, 0, 2), ((8, 1, 16), 1.4, 0, 2),
    ((48, 36, 12), None, 0, 1),
]


@pytest.mark.parametrize("dims,beta,bc,ybc", WALL_CASES)
def test_poisson_with_y_walls_matches_oracle(chanfs, dims, beta, bc, ybc):
    nx, ny, nz = dims
    lx, ly = 2 * np.pi, 1.7
    dz = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    f = rhs_for(nx, ny, nz, dz, bc, ybc, 17 * nx + ny + nz + 3 * ybc + bc)
    ref = oracle.poisson_solve_walls(f, lx, ly, dz, bc, ybc)
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc, chanfs.F64, ybc) as plan:
        p = host(plan.poisson_solve(dev(f)))
        assert rel(p, ref) < 1e-12, rel(p, ref)
        t = dev(f)
        plan.poisson_solve(t, out=t)
        assert np.array_equal(host(t), p)
        # the z-implicit Helmholtz does not see y
        u = host(plan.helmholtz_solve(1e-4, dev(f), chanfs.FACE))
        assert rel(u, oracle.helmholtz_solve(f, dz, 1e-4, 1)) < 1e-12
        # the fully implicit Helmholtz (Eq. 8) with the same y transforms
        for loc, c in ((chanfs.CENTER, 1e-3), (chanfs.FACE, 0.2)):
            u3 = host(plan.helmholtz3d_solve(c, dev(f), loc))
            ref3 = oracle.helmholtz3d_solve(f, lx, ly, dz, c, loc, ybc)
            assert rel(u3, ref3) < 1e-12, (loc, rel(u3, ref3))
        assert plan.check() == 0


@pytest.mark.parametrize("dims,beta,bc,ybc", [((32, 24, 20), 1.8, 0, 1), ((64, 48, 40), 1.8, 1, 2),
                                              ((48, 36, 12), 1.5, 0, 2), ((16, 288, 8), 1.5, 0, 1)])
def test_refined_poisson_with_y_walls(chanfs, dims, beta, bc, ybc):
    nx, ny, nz = dims
    lx, ly = 12.8, 6.4
    dz = synth.tanh_dz(nz, beta)
    f = rhs_for(nx, ny, nz, dz, bc, ybc, 23 * nx + nz + ybc)
    ref = oracle.poisson_solve_walls(f, lx, ly, dz, bc, ybc)
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc, chanfs.F32_REFINED, ybc) as plan:
        p = host(plan.poisson_solve(dev(f)))
        iters, rho = plan.last_info()
        assert rho <= 1e-10 and iters <= 4, (iters, rho)
        assert rel(p, ref) < 1e-10, rel(p, ref)
        # grouped with a periodic box: the same bits as alone
        with chanfs.Plan(32, 24, 10, 1.0, 1.0, synth.tanh_dz(10, 1.3), 0, chanfs.F32_REFINED) as other:
            g_rhs = synth.remove_weighted_mean(synth.normal(5, (10, 24, 32)), synth.tanh_dz(10, 1.3))
            alone_other = host(other.poisson_solve(dev(g_rhs)))
            with chanfs.Group([plan, other]) as g:
                got = [host(o) for o in g.poisson_solve([dev(f), dev(g_rhs)])]
            assert np.array_equal(got[0], p)
            assert np.array_equal(got[1], alone_other)
        assert plan.check() == 0


def test_walls_reject_bad_condition(chanfs):
    import ctypes
    h = ctypes.c_void_p()
    dz = np.full(5, 0.4)
    rc = chanfs.lib().cfs_plan_create_walls(ctypes.byref(h), 8, 6, 5, 1.0, 1.0,
                                            dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            0, 3, 0)
    assert rc == chanfs.EINVAL and not h.value
