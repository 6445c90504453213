"""GPU: FP32 solves with FP64 iterative refinement (plans created with
CFS_F32_REFINED), against the FP64 CPU oracle.

Accuracy bar: relative max-norm error <= 1e-10 against the oracle's FP64
solution, and the reported relative residual <= 1e-10, within at most four
FP32 solves.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


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


POISSON = [
    ((32, 32, 32), None, 0, "uniform"),
    ((64, 48, 64), 1.8, 0, "normal"),
    ((64, 48, 64), 1.8, 1, "normal"),
    ((48, 36, 40), 2.0, 0, "uniform"),
    ((12, 9, 5), 1.2, 0, "normal"),     # odd complex length along y
    ((128, 96, 96), 1.8, 0, "normal"),
    ((96, 384, 24), 1.5, 0, "normal"),   # two TMA boxes along y
]


@pytest.mark.parametrize("dims,beta,bc,dist", POISSON)
def test_refined_poisson_matches_fp64_oracle(chanfs, dims, beta, bc, dist):
    nx, ny, nz = dims
    lx, ly = 12.8, 6.4
    dz = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    seed = 100 + nx + nz
    f = synth.uniform(seed, (nz, ny, nx)) if dist == "uniform" else synth.normal(seed, (nz, ny, nx))
    if bc == 0:
        f = synth.remove_weighted_mean(f, dz)
    ref = oracle.poisson_solve(f, lx, ly, dz, bc)
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc, chanfs.F32_REFINED) as plan:
        p = host(plan.poisson_solve(dev(f)))
        iters, rho = plan.last_info()
        assert rho <= TOL and 1 <= iters <= 4, (iters, rho)
        assert rel(p, ref) < TOL, rel(p, ref)
        if bc == 0:  # the solution's zero dz-weighted mean (kept by the correction passes)
            m = (np.repeat(dz, nx * ny) @ p.ravel()) / (dz.sum() * nx * ny)
            assert abs(m) <= 1e-13 * np.max(np.abs(p)), m
        # the residual as the oracle computes it
        r = f - oracle.apply_poisson(p, lx, ly, dz, bc)
        if bc == 0:
            r -= (np.repeat(dz, nx * ny) @ r.ravel()) / (dz.sum() * nx * ny)
        assert np.max(np.abs(r)) / np.max(np.abs(f)) < 2 * TOL
        # in place
        t = dev(f)
        plan.poisson_solve(t, out=t)
        assert np.array_equal(host(t), p)
        assert plan.check() == 0


# Right-hand sides that make the first residual's cancellation hard: a field
# with most of its energy at mid wavenumbers (p is then far from smooth on
# the grid), on a strongly stretched grid, with both wall conditions.
HARD = [
    (0, 2.6, "mid"), (1, 2.6, "mid"), (0, 2.6, "noise"), (1, 0.0, "mid"),
]


@pytest.mark.parametrize("bc,beta,kind", HARD)
def test_refined_residual_is_evaluated_to_fp64_accuracy(chanfs, bc, beta, kind):
    """The library's residual norm against the oracle's FP64 residual of the
    returned solution, at a tolerance ten times below the default."""
    nx, ny, nz = 64, 48, 96
    lx, ly = 6.4, 3.2
    dz = synth.uniform_dz(nz) if beta == 0.0 else synth.tanh_dz(nz, beta)
    f = synth.normal(77 + bc, (nz, ny, nx))
    if kind == "mid":  # modes kx = nx/4, ky = ny/4 and a z wave of 12 cells
        x = np.arange(nx) / nx
        y = np.arange(ny) / ny
        zc = np.cumsum(dz) - 0.5 * dz
        f = f * 1e-3 + (np.sin(2 * np.pi * 16 * x)[None, None, :]
                        * np.cos(2 * np.pi * 12 * y)[None, :, None]
                        * np.cos(np.pi * 8 * zc)[:, None, None])
    if bc == 0:
        f = synth.remove_weighted_mean(f, dz)
    tol = 1e-11
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc, chanfs.F32_REFINED) as plan:
        plan.set_refinement(tol, 8)
        p = host(plan.poisson_solve(dev(f)))
        iters, rho = plan.last_info()
        assert rho <= tol, (iters, rho)
        r = f - oracle.apply_poisson(p, lx, ly, dz, bc)
        if bc == 0:
            r -= (np.repeat(dz, nx * ny) @ r.ravel()) / (dz.sum() * nx * ny)
        true_rho = np.max(np.abs(r)) / np.max(np.abs(f))
        assert true_rho < 2 * tol, (true_rho, rho)
        ref = oracle.poisson_solve(f, lx, ly, dz, bc)
        assert rel(p, ref) < 10 * tol, rel(p, ref)


@pytest.mark.parametrize("tw", [-1, 1, 8, 16])
def test_refined_poisson_thomas_shapes(chanfs, tw):
    nx, ny, nz = 64, 48, 300   # two TMA boxes along z, near-singular FP64 columns
    dz = synth.tanh_dz(nz, 1.8)
    f = synth.remove_weighted_mean(synth.normal(17, (nz, ny, nx)), dz)
    ref = oracle.poisson_solve(f, 12.8, 6.4, dz, 0)
    with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, 0, chanfs.F32_REFINED) as plan:
        plan.set_option(chanfs.OPT_THOMAS_TILE, tw)
        p = host(plan.poisson_solve(dev(f)))
        iters, rho = plan.last_info()
        assert rho <= TOL and iters <= 4, (iters, rho)
        assert rel(p, ref) < TOL, rel(p, ref)
        assert plan.check() == 0


# The partitioned FP32 z solve (CFS_OPT_THOMAS_TILE 1: Algorithm 2 over
# z-partitions of 8 rows in registers, coefficients formed on the fly, the
# reduced system by cyclic reduction): one partition, ragged last partitions
# (nz = 97: one real row and seven identity rows), the largest reduced system
# (nz = 512: 64 partitions, 4 column pairs per tile), both z walls, both kinds
# of y walls (one slot per thread), odd Ny (no self-paired slot Ny/2).
ZPART = [
    ((32, 24, 5), 1.2, 0, 0),
    ((48, 36, 97), 2.0, 1, 0),
    ((64, 48, 300), 1.8, 0, 0),
    ((128, 96, 512), 1.8, 0, 0),
    ((16, 12, 512), 1.8, 0, 0),
    ((32, 27, 41), 1.6, 0, 0),
    ((64, 48, 64), 1.5, 0, 1),
    ((64, 48, 66), 1.5, 1, 2),
]


@pytest.mark.parametrize("dims,beta,bc,ybc", ZPART)
def test_refined_poisson_partitioned_z_solve(chanfs, dims, beta, bc, ybc):
    nx, ny, nz = dims
    lx, ly = 12.8, 6.4
    dz = synth.tanh_dz(nz, beta)
    f = synth.normal(31 * nz + bc + ybc, (nz, ny, nx))
    if bc == 0 and ybc != 2:
        f = synth.remove_weighted_mean(f, dz)
    ref = (oracle.poisson_solve(f, lx, ly, dz, bc) if ybc == 0
           else oracle.poisson_solve_walls(f, lx, ly, dz, bc, ybc))
    out = {}
    for tw in (-1, 1):
        with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc, chanfs.F32_REFINED, ybc) as plan:
            plan.set_option(chanfs.OPT_THOMAS_TILE, tw)
            assert plan.get_option(chanfs.OPT_THOMAS_TILE) == tw
            p = host(plan.poisson_solve(dev(f)))
            iters, rho = plan.last_info()
            assert rho <= TOL and iters <= 4, (tw, iters, rho)
            assert rel(p, ref) < TOL, (tw, rel(p, ref))
            assert plan.check() == 0
            out[tw] = iters
    # the partitioned inner solve is as good a preconditioner as the sweep
    assert out[1] <= out[-1] + 1, out


def test_partitioned_z_solve_grouped_bits_match_alone(chanfs):
    """Boxes that take the partitioned z solve run it in a group too: the
    same bits as alone, beside a box on the streaming sweep."""
    dims = [(64, 48, 97), (32, 24, 300), (48, 36, 40)]
    tws = [1, 1, -1]
    plans, rhs, alone = [], [], []
    try:
        for (nx, ny, nz), tw in zip(dims, tws):
            dz = synth.tanh_dz(nz, 1.7)
            pl = chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, 0, chanfs.F32_REFINED)
            pl.set_option(chanfs.OPT_THOMAS_TILE, tw)
            f = synth.remove_weighted_mean(synth.normal(nz + nx, (nz, ny, nx)), dz)
            plans.append(pl)
            rhs.append(dev(f))
            alone.append(host(pl.poisson_solve(rhs[-1])))
        with chanfs.Group(plans) as g:
            for _ in range(3):  # direct launches, graph capture, graph replay
                got = [host(o) for o in g.poisson_solve(rhs)]
                for a, b in zip(got, alone):
                    assert np.array_equal(a, b)
    finally:
        for pl in plans:
            pl.close()


def test_partitioned_z_solve_option_rules(chanfs):
    dz = synth.tanh_dz(40, 1.5)
    with chanfs.Plan(32, 24, 40, 1.0, 1.0, dz, 0) as p64:  # FP64 plans: no partitioned solve
        with pytest.raises(chanfs.ChanfsError) as err:
            p64.set_option(chanfs.OPT_THOMAS_TILE, 1)
        assert err.value.status == chanfs.EUNSUPPORTED
    dz = synth.tanh_dz(520, 1.5)   # more than 64 partitions of 8 rows
    with chanfs.Plan(16, 12, 520, 1.0, 1.0, dz, 0, chanfs.F32_REFINED) as p:
        with pytest.raises(chanfs.ChanfsError) as err:
            p.set_option(chanfs.OPT_THOMAS_TILE, 1)
        assert err.value.status == chanfs.EUNSUPPORTED


def test_refined_poisson_reports_nonconvergence(chanfs):
    nx, ny, nz = 64, 48, 64
    dz = synth.tanh_dz(nz, 1.8)
    f = synth.remove_weighted_mean(synth.normal(5, (nz, ny, nx)), dz)
    with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, 0, chanfs.F32_REFINED) as plan:
        plan.set_refinement(1e-14, 1)
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.poisson_solve(dev(f))
        assert err.value.status == chanfs.ENOTCONVERGED
        iters, rho = plan.last_info()
        assert iters == 1 and 1e-14 < rho < 1e-2
        plan.set_refinement(1e-10, 4)
        plan.poisson_solve(dev(f))
        assert plan.last_info()[1] <= 1e-10


def test_refined_plan_needs_nx_multiple_of_4(chanfs):
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.Plan(6, 9, 5, 1.0, 1.0, np.full(5, 0.4), 0, chanfs.F32_REFINED)
    assert err.value.status == chanfs.EUNSUPPORTED


def test_refined_zero_rhs_gives_zero(chanfs):
    with chanfs.Plan(16, 12, 10, 1.0, 1.0, np.full(10, 0.2), 0, chanfs.F32_REFINED) as plan:
        p = host(plan.poisson_solve(torch.zeros(10, 12, 16, dtype=torch.float64, device="cuda")))
        assert np.all(p == 0.0)


HELM = [
    (16, 12, 48, 1.8, 0, 9.615e-5),
    (16, 12, 48, 1.8, 1, 9.615e-5),
    (32, 24, 384, 1.8, 0, 9.615e-9),
    (32, 24, 384, 1.8, 1, 9.615e-9),
    (12, 9, 100, 1.5, 0, 1e-2),   # far from the identity
]


@pytest.mark.parametrize("nx,ny,nz,beta,loc,c", HELM)
def test_refined_helmholtz_matches_fp64_oracle(chanfs, nx, ny, nz, beta, loc, c):
    dz = synth.tanh_dz(nz, beta)
    rhs = synth.normal(nx + nz + loc, (nz, ny, nx))
    ref = oracle.helmholtz_solve(rhs, dz, c, loc)
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, dz, 0, chanfs.F32_REFINED) as plan:
        u = host(plan.helmholtz_solve(c, dev(rhs), loc))
        iters, rho = plan.last_info()
        assert rho <= TOL and 1 <= iters <= 4, (iters, rho)
        assert rel(u, ref) < TOL, rel(u, ref)
        if loc == 1:
            assert np.all(u[-1] == 0.0)
        t = dev(rhs)
        plan.helmholtz_solve(c, t, loc, out=t)
        assert np.array_equal(host(t), u)


# The refined Helmholtz solve runs in one pass (FP32 Algorithm 2 and
# double-float residuals on tiles in shared memory) where a tile fits, else
# as the loop of FP32 solves and FP64 residual passes (long columns, or FP32
# Thomas inner solves).  Both against the oracle, with partition counts,
# ragged tiles, both locations, a coefficient far from the identity, and
# the outcome reported when the target is missed.
ONE_PASS = [
    (12, 9, 64, 2.2, 0, 1e-4, 0),     # ragged last tile (108 columns), c/h^2 large
    (16, 12, 192, 1.2, 1, 1e-6, 6),
    (32, 24, 384, 1.8, 0, 9.615e-9, 16),
    (8, 4, 600, 1.8, 1, 3e-5, 24),
    (12, 9, 100, 1.5, 0, 1e-2, 3),    # far from the identity: several FP32 solves
    (8, 6, 900, 1.8, 0, 1e-5, 0),     # too long for one pass: the loop
]


@pytest.mark.parametrize("nx,ny,nz,beta,loc,c,nparts", ONE_PASS)
def test_refined_helmholtz_one_pass_matches_oracle(chanfs, nx, ny, nz, beta, loc, c, nparts):
    dz = synth.tanh_dz(nz, beta)
    rhs = synth.normal(3 * nz + loc, (nz, ny, nx))
    ref = oracle.helmholtz_solve(rhs, dz, c, loc)
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, dz, 0, chanfs.F32_REFINED) as plan:
        plan.set_option(chanfs.OPT_PCR_PARTS, nparts)
        u = host(plan.helmholtz_solve(c, dev(rhs), loc))
        iters, rho = plan.last_info()
        assert rho <= TOL and 1 <= iters <= 4, (iters, rho)
        assert rel(u, ref) < TOL, rel(u, ref)
        # the reported residual against the oracle's operator
        r = rhs - oracle.apply_helmholtz(u, dz, c, loc)
        if loc == 1:
            r[-1] = 0.0
            assert np.all(u[-1] == 0.0)
        assert np.max(np.abs(r)) / np.max(np.abs(rhs)) < 2 * TOL
        # zero right-hand side, and a tolerance one FP32 solve cannot meet
        z = host(plan.helmholtz_solve(c, torch.zeros_like(dev(rhs)), loc))
        assert np.all(z == 0.0) and plan.last_info()[1] == 0.0
        plan.set_refinement(1e-14, 1)
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.helmholtz_solve(c, dev(rhs), loc)
        assert err.value.status == chanfs.ENOTCONVERGED
        iters, rho = plan.last_info()
        assert iters == 1 and 1e-14 < rho < 1e-3
        assert plan.check() == 0


@pytest.mark.slow
def test_refined_precision_workload_full_size(chanfs):
    """The 1024 x 768 x 512 uniform precision workload in the launch
    configuration the benchmark times (shapes from the autotuner): the
    refined solve meets the residual target and matches the oracle's FP64
    solution element by element."""
    cfg = synth.PRECISION
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    dz = synth.grid_dz(cfg)
    f = synth.precision_rhs(cfg)
    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, 0, chanfs.F32_REFINED) as plan:
        plan.autotune()
        p = host(plan.poisson_solve(dev(f)))
        iters, rho = plan.last_info()
        assert rho <= TOL and iters <= 4, (iters, rho)
        assert plan.check() == 0
    ref = oracle.poisson_solve(f, cfg["lx"], cfg["ly"], dz, 0)
    assert rel(p, ref) < TOL, rel(p, ref)
    del ref
    r = f - oracle.apply_poisson(p, cfg["lx"], cfg["ly"], dz, 0)
    assert np.max(np.abs(r)) / np.max(np.abs(f)) < 2 * TOL


def test_integer_unit_conversions_match_the_hardware(chanfs):
    """The refinement's FP32 <-> FP64 conversions, done on the integer units,
    give the hardware conversion's bits for every sampled operand."""
    assert chanfs.selfcheck_conversions(1 << 24) == 0
