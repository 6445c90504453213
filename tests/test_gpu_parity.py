"""GPU parity: every stage of the CUDA path, called through the C ABI, against
the CPU oracle on the same seeded inputs, element by element.

Tolerance: 1e-12 in the relative max-norm, max|gpu - oracle| / max|oracle|,
the figure the FP64 path is specified to meet.  Both sides compute in FP64;
they differ only in rounding order (and FMA use on the GPU).
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
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make_dz(nz, beta):
    return synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)


# sizes span several y tiles and a ragged tail (M not a multiple of the tile
# width), odd complex lengths along x and y, ny = 1 and ny > 256 (two TMA boxes)
SPECTRAL_SIZES = [(32, 32, 4), (48, 36, 3), (6, 9, 3), (18, 27, 3), (2, 1, 3), (8, 1, 5),
                  (24, 384, 3), (64, 288, 3), (54, 12, 3), (512, 8, 3), (16, 486, 3)]


@pytest.mark.parametrize("dims", SPECTRAL_SIZES)
def test_spectral_forward_and_inverse(chanfs, dims):
    nx, ny, nz = dims
    f = synth.normal(100 + nx + ny, (nz, ny, nx))
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, np.full(nz, 1.0)) as plan:
        s = host(plan.spectral_forward(dev(f)))
        ref = oracle.spectral_forward(f)  # complex (nz, ny, nx/2)
        got = s.view(np.complex128).reshape(ref.shape)
        assert rel(got, ref) < TOL
        back = host(plan.spectral_inverse(dev(s)))
        assert rel(back, f) < TOL
        assert rel(back, oracle.spectral_inverse(ref)) < TOL
        # in place
        t = dev(f)
        plan.spectral_forward(t, out=t)
        assert rel(host(t).view(np.complex128).reshape(ref.shape), ref) < TOL
        assert plan.check() == 0


def _oracle_x_packed(f):
    nz, ny, nx = f.shape
    out = np.empty_like(f)
    for z in range(nz):
        for y in range(ny):
            out[z, y] = oracle.rfft_packed(f[z, y])
    return out


def _oracle_y(c, sign):
    """Oracle FFT along axis 1 of a complex (nz, ny, m) array."""
    out = np.empty_like(c)
    for z in range(c.shape[0]):
        for j in range(c.shape[2]):
            out[z, :, j] = oracle.fft(c[z, :, j], sign)
    return out


STAGE_SIZES = [(24, 384, 3), (32, 32, 4), (16, 486, 3), (64, 288, 3), (8, 48, 3)]


@pytest.mark.parametrize("dims", STAGE_SIZES)
def test_each_transform_stage(chanfs, dims):
    """x and y transforms one kernel at a time, forward and inverse."""
    nx, ny, nz = dims
    m = nx // 2
    f = synth.normal(11 + nx + ny, (nz, ny, nx))
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, np.full(nz, 1.0)) as plan:
        x = host(plan.poisson_stage(chanfs.X_FORWARD, dev(f)))
        xref = _oracle_x_packed(f)
        assert rel(x, xref) < TOL, ("x forward", rel(x, xref))
        # y forward of the packed x spectrum gives the solver's spectral layout
        y = host(plan.poisson_stage(chanfs.Y_FORWARD, dev(xref)))
        sref = oracle.spectral_forward(f)
        assert rel(y.view(np.complex128).reshape(nz, ny, m), sref) < TOL, "y forward"
        # columns kx >= 1 are plain DFTs along y
        yref = _oracle_y(xref.view(np.complex128).reshape(nz, ny, m), -1)
        assert rel(y.view(np.complex128).reshape(nz, ny, m)[:, :, 1:], yref[:, :, 1:]) < TOL
        # y inverse (unnormalised) of the layout gives Ny times the x spectrum
        sl = np.ascontiguousarray(sref).view(np.float64).reshape(nz, ny, nx)
        yi = host(plan.poisson_stage(chanfs.Y_INVERSE, dev(sl)))
        assert rel(yi, ny * xref) < TOL, "y inverse"
        xi = host(plan.poisson_stage(chanfs.X_INVERSE, dev(xref)))
        assert rel(xi, f * m) < TOL, ("x inverse", rel(xi, f * m))
        assert plan.check() == 0


POISSON_CASES = [
    ((32, 32, 32), None, 0),      # the small uniform workload
    ((32, 32, 32), None, 1),
    ((48, 36, 20), 1.8, 0),       # stretched, ragged y tiles
    ((48, 36, 20), 1.8, 1),
    ((6, 9, 5), 1.2, 0),          # odd complex lengths
    ((6, 27, 5), 1.2, 1),         # odd y pass count: the result tile in the second buffer
    ((2, 1, 3), None, 0),         # degenerate: one x pair, ny = 1, nz = 3
    ((8, 1, 16), 1.5, 1),
    ((64, 384, 12), 1.8, 0),      # two TMA boxes along y
    ((96, 54, 33), 2.0, 0),
]


@pytest.mark.parametrize("dims,beta,bc", POISSON_CASES)
def test_poisson_matches_oracle(chanfs, dims, beta, bc):
    nx, ny, nz = dims
    lx, ly = 2 * np.pi, np.pi
    dz = make_dz(nz, beta)
    f = synth.normal(7 * nx + ny + nz, (nz, ny, nx))
    if bc == chanfs.NEUMANN:
        f = synth.remove_weighted_mean(f, dz)
    ref = oracle.poisson_solve(f, lx, ly, dz, bc)
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc) as plan:
        p = host(plan.poisson_solve(dev(f)))
        assert rel(p, ref) < TOL, rel(p, ref)
        # in place gives the same bits
        t = dev(f)
        plan.poisson_solve(t, out=t)
        assert np.array_equal(host(t), p)
        assert plan.check() == 0


# Shapes of the z sweeps of Eq. 12: shared-memory tiles of 16 and 8 columns
# and the streaming kernel.  Ragged last tiles (M not a multiple of the tile
# width), nz in one and in several TMA boxes (nz > 256, odd), ny = 1.
THOMAS_CASES = [
    ((48, 36, 20), 1.8, 0),
    ((48, 36, 20), 1.8, 1),
    ((6, 9, 5), 1.2, 0),
    ((24, 12, 300), 1.8, 0),
    ((48, 12, 301), 1.8, 1),
    ((8, 1, 16), 1.5, 0),
]


@pytest.mark.parametrize("dims,beta,bc", THOMAS_CASES)
def test_thomas_shapes_match_oracle(chanfs, dims, beta, bc):
    nx, ny, nz = dims
    lx, ly = 2 * np.pi, np.pi
    dz = make_dz(nz, beta)
    f = synth.normal(11 * nx + ny + nz, (nz, ny, nx))
    if bc == chanfs.NEUMANN:
        f = synth.remove_weighted_mean(f, dz)
    ref = oracle.poisson_solve(f, lx, ly, dz, bc)
    got = {}
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, bc) as plan:
        for tw in (-1, 8, 16):
            plan.set_option(chanfs.OPT_THOMAS_TILE, tw)
            assert plan.get_option(chanfs.OPT_THOMAS_TILE) == tw
            got[tw] = host(plan.poisson_solve(dev(f)))
            assert rel(got[tw], ref) < TOL, (tw, rel(got[tw], ref))
        plan.set_option(chanfs.OPT_THOMAS_TILE, 0)
        assert plan.get_option(chanfs.OPT_THOMAS_TILE) in (-1, 8, 16)
        assert plan.check() == 0
    # the sweeps do the same arithmetic in every shape; only the singular
    # Neumann column sums its weighted means in another order
    for tw in (8, 16):
        if bc == chanfs.DIRICHLET:
            assert np.array_equal(got[tw], got[-1])
        else:
            assert rel(got[tw], got[-1]) < 1e-14


def test_thomas_option_rejects_bad_values(chanfs):
    with chanfs.Plan(16, 12, 10, 1.0, 1.0, np.full(10, 0.2)) as plan:
        for bad in (2, 4, 32, -2):
            with pytest.raises(chanfs.ChanfsError) as err:
                plan.set_option(chanfs.OPT_THOMAS_TILE, bad)
            assert err.value.status == chanfs.EINVAL
        with pytest.raises(chanfs.ChanfsError) as err:  # the partitioned solve is FP32 only
            plan.set_option(chanfs.OPT_THOMAS_TILE, 1)
        assert err.value.status == chanfs.EUNSUPPORTED
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.set_option(99, 0)
        assert err.value.status == chanfs.EINVAL
    # a tile of 16 FP64 columns x 16000 rows does not fit in shared memory
    with chanfs.Plan(16, 2, 16000, 1.0, 1.0, np.full(16000, 1e-4)) as plan:
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.set_option(chanfs.OPT_THOMAS_TILE, 16)
        assert err.value.status == chanfs.EUNSUPPORTED
        assert plan.get_option(chanfs.OPT_THOMAS_TILE) == -1


def test_poisson_neumann_removes_incompatible_mean(chanfs):
    nx, ny, nz = 16, 12, 10
    dz = synth.tanh_dz(nz, 1.4)
    f = synth.normal(3, (nz, ny, nx)) + 0.25  # not compatible
    ref = oracle.poisson_solve(f, 1.0, 2.0, dz, 0)
    with chanfs.Plan(nx, ny, nz, 1.0, 2.0, dz, 0) as plan:
        p = host(plan.poisson_solve(dev(f)))
    assert rel(p, ref) < TOL
    w = np.repeat(dz, nx * ny)
    assert abs(w @ p.ravel()) < 1e-13 * w.sum() * np.max(np.abs(p))


def test_poisson_small_workload_residual(chanfs):
    cfg = synth.SMALL
    f = synth.small_rhs(cfg)
    dz = synth.grid_dz(cfg)
    with chanfs.Plan(cfg["nx"], cfg["ny"], cfg["nz"], cfg["lx"], cfg["ly"], dz, 0) as plan:
        p = host(plan.poisson_solve(dev(f)))
    r = f - oracle.apply_poisson(p, cfg["lx"], cfg["ly"], dz, 0)
    assert np.max(np.abs(r)) / np.max(np.abs(f)) < 1e-12
    assert abs(p.mean()) < 1e-14 * np.max(np.abs(p))


HELM_CASES = [
    # (nx, ny, nz, beta, loc, nparts)
    (16, 12, 48, 1.8, 0, 0),
    (16, 12, 48, 1.8, 1, 0),
    (12, 9, 100, 1.5, 0, 7),      # uneven partitions, ragged column tile
    (12, 9, 100, 1.5, 1, 11),
    (8, 8, 384, 1.8, 0, 12),      # 32-row partitions
    (8, 8, 384, 1.8, 1, 12),
    (8, 8, 384, 1.8, 0, 24),
    (4, 3, 3, None, 0, 1),        # smallest column
    (6, 4, 4, None, 1, 1),        # face: 3 unknowns
    (48, 36, 512, 2.0, 0, 32),    # 512 unknowns, 32 partitions
    (16, 12, 1024, 1.8, 0, 0),    # largest column, 4 TMA boxes
    (16, 12, 700, 1.6, 1, 64),    # 64 partitions, ragged boxes
    (6, 3, 40, 1.2, 0, 1),        # one partition: Algorithm 2 degenerates to Thomas
]


@pytest.mark.parametrize("nx,ny,nz,beta,loc,nparts", HELM_CASES)
def test_helmholtz_matches_oracle(chanfs, nx, ny, nz, beta, loc, nparts):
    dz = make_dz(nz, beta)
    rhs = synth.normal(nx * nz + loc, (nz, ny, nx))
    c = 9.615e-5
    ref = oracle.helmholtz_solve(rhs, dz, c, loc, oracle.THOMAS)
    n = nz if loc == 0 else nz - 1
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, dz) as plan:
        plan.helmholtz_prepare(c, loc, nparts)
        u = host(plan.helmholtz_solve(c, dev(rhs), loc))
        assert rel(u, ref) < TOL, rel(u, ref)
        if nparts and n >= 3 * nparts:
            ref2 = oracle.helmholtz_solve(rhs, dz, c, loc, oracle.ALG2, nparts)
            assert rel(u, ref2) < TOL
        t = dev(rhs)
        plan.helmholtz_solve(c, t, loc, out=t)
        assert np.array_equal(host(t), u)
        assert plan.check() == 0


def test_helmholtz_identity_and_strong_coefficient(chanfs):
    nx, ny, nz = 12, 8, 64
    dz = synth.tanh_dz(nz, 1.8)
    rhs = synth.normal(5, (nz, ny, nx))
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, dz) as plan:
        for loc in (0, 1):
            u = host(plan.helmholtz_solve(0.0, dev(rhs), loc))
            ref = rhs.copy()
            if loc == 1:
                ref[-1] = 0.0
            assert np.array_equal(u, ref)
            c = 1e-2  # far from the identity: c / dz^2 ~ 1e4
            u = host(plan.helmholtz_solve(c, dev(rhs), loc))
            assert rel(u, oracle.helmholtz_solve(rhs, dz, c, loc)) < TOL


def test_helmholtz_rejects_unsupported_partitions(chanfs):
    with chanfs.Plan(8, 8, 40, 1.0, 1.0, np.full(40, 0.05)) as plan:
        with pytest.raises(chanfs.ChanfsError):
            plan.helmholtz_prepare(1e-3, 0, 20)   # 2 rows per partition
        plan.helmholtz_prepare(1e-3, 0, 1)        # one partition of 40 rows is fine
        with pytest.raises(chanfs.ChanfsError):
            plan.helmholtz_prepare(-1.0, 0, 0)
    with chanfs.Plan(8, 8, 1100, 1.0, 1.0, np.full(1100, 2 / 1100)) as plan:
        with pytest.raises(chanfs.ChanfsError):
            plan.helmholtz_prepare(1e-3, 0, 0)    # 1100 unknowns > 1024
        with pytest.raises(chanfs.ChanfsError):
            plan.helmholtz_prepare(1e-3, 0, 65)   # more than 64 partitions


def test_host_buffer_entry_points_match_device_path(chanfs):
    nx, ny, nz = 32, 24, 16
    dz = synth.tanh_dz(nz, 1.6)
    f = synth.remove_weighted_mean(synth.normal(9, (nz, ny, nx)), dz)
    with chanfs.Plan(nx, ny, nz, 3.0, 2.0, dz) as plan:
        p_dev = host(plan.poisson_solve(dev(f)))
        out = np.empty_like(f)
        plan.poisson_solve_host(f, out)
        assert np.array_equal(out, p_dev)
        pinned_in = torch.from_numpy(f).pin_memory()
        pinned_out = torch.empty_like(pinned_in).pin_memory()
        plan.poisson_solve_host(pinned_in, pinned_out)
        assert np.array_equal(pinned_out.numpy(), p_dev)
        u_dev = host(plan.helmholtz_solve(1e-3, dev(f), 1))
        plan.helmholtz_solve_host(1e-3, f, out, 1)
        assert np.array_equal(out, u_dev)


@pytest.fixture(scope="module")
def channel_reference():
    """The 512 x 384 x 384 channel workload's inputs and the oracle's FP64
    solutions (Poisson, and Helmholtz for u, v centred and w face)."""
    cfg = synth.CHANNEL
    dz = synth.grid_dz(cfg)
    f, rhs = synth.channel_fields(cfg)
    c = synth.CHANNEL_C
    p = oracle.poisson_solve(f, cfg["lx"], cfg["ly"], dz, 0)
    us = [oracle.helmholtz_solve(r, dz, c, loc) for r, loc in zip(rhs, CHANNEL_LOCS)]
    return cfg, dz, f, rhs, p, us


CHANNEL_LOCS = (0, 0, 1)  # u, v cell-centred; w face-located


def _channel_solve_and_check(plan, f_d, rhs_d, p_ref, u_refs, what, poisson=True,
                             helmholtz=True):
    p = None
    if poisson:
        p = host(plan.poisson_solve(f_d))
        assert rel(p, p_ref) < TOL, (what, rel(p, p_ref))
    if helmholtz:
        for r, loc, uref in zip(rhs_d, CHANNEL_LOCS, u_refs):
            u = host(plan.helmholtz_solve(synth.CHANNEL_C, r, loc))
            assert rel(u, uref) < TOL, (what, loc, rel(u, uref))
    assert plan.check() == 0
    return p


@pytest.mark.slow
def test_channel_workload_full_size(chanfs, channel_reference):
    """The benchmark's 512 x 384 x 384 channel step in the launch
    configuration the benchmark times: shapes chosen by the autotuner, the
    Helmholtz solves by Algorithm 2 with the tuned partition count, the
    Poisson solve both whole and stage by stage; every element against the
    oracle."""
    cfg, dz, f, rhs, p_ref, u_refs = channel_reference
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    c = synth.CHANNEL_C
    f_d = dev(f)
    rhs_d = [dev(r) for r in rhs]
    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN) as plan:
        shapes = plan.autotune()
        plan.set_option(chanfs.OPT_HELM_THOMAS, 0)
        for loc in (chanfs.CENTER, chanfs.FACE):
            plan.helmholtz_prepare(c, loc, 0)
        p = _channel_solve_and_check(plan, f_d, rhs_d, p_ref, u_refs, shapes)
        # the benchmark launches the five Poisson kernels one by one
        s = torch.empty_like(f_d)
        plan.poisson_stage(chanfs.X_FORWARD, f_d, out=s)
        for stage in (chanfs.Y_FORWARD, chanfs.Z_SOLVE, chanfs.Y_INVERSE, chanfs.X_INVERSE):
            plan.poisson_stage(stage, s, out=s)
        assert np.array_equal(host(s), p)
        assert plan.check() == 0
    res = f - oracle.apply_poisson(p, cfg["lx"], cfg["ly"], dz, 0)
    assert np.max(np.abs(res)) / np.max(np.abs(f)) < 1e-12


# The candidates the autotuner times for each option (csrc/tune.cu), and
# whether the option shapes the Poisson or the Helmholtz kernels; a candidate
# that cannot run at this size is rejected by set_option.
TUNER_CANDIDATES = [
    ("OPT_FFT_RADIX", (8, 4), "poisson"),
    ("OPT_X_LINES", (1, 2, 4, 8, 16, 32, 64), "poisson"),
    ("OPT_Y_TILE", (1, 2, 4, 8, 16, 32), "poisson"),
    ("OPT_THOMAS_TILE", (-1, 8, 16), "poisson"),
    ("OPT_PCR_PARTS", (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64), "helmholtz"),
    ("OPT_HELM_THOMAS", (0, 1), "helmholtz"),
]


@pytest.mark.slow
def test_channel_workload_every_tuner_candidate(chanfs, channel_reference):
    """Whatever shape the autotuner picks for the benchmark's channel step,
    the result meets the oracle: every candidate of every option, one option
    at a time from the defaults, every element at full size."""
    cfg, dz, f, rhs, p_ref, u_refs = channel_reference
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    f_d = dev(f)
    rhs_d = [dev(r) for r in rhs]
    ran = 0
    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN) as plan:
        for name, values, kind in TUNER_CANDIDATES:
            opt = getattr(chanfs, name)
            for v in values:
                try:
                    plan.set_option(opt, v)
                except chanfs.ChanfsError as err:
                    assert err.status == chanfs.EUNSUPPORTED, (name, v)
                    continue
                _channel_solve_and_check(plan, f_d, rhs_d, p_ref, u_refs, (name, v),
                                         poisson=kind == "poisson",
                                         helmholtz=kind == "helmholtz")
                ran += 1
            plan.set_option(opt, 0)  # back to the automatic choice
    assert ran >= 20


@pytest.mark.parametrize("dtype", [0, 1])
def test_options_and_autotune_keep_results(chanfs, dtype):
    """Every kernel shape the options allow computes the same solution."""
    nx, ny, nz = 64, 48, 40
    dz = make_dz(nz, 1.7)
    f = synth.remove_weighted_mean(synth.normal(77, (nz, ny, nx)), dz)
    rhs = synth.normal(78, (nz, ny, nx))
    c = 2e-5
    ref = oracle.poisson_solve(f, 2.0, 1.0, dz, 0)
    href = oracle.helmholtz_solve(rhs, dz, c, 0)
    tol = 1e-10 if dtype == 1 else TOL
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, dtype) as plan:
        for opt, vals in ((chanfs.OPT_X_LINES, (1, 4, 16)), (chanfs.OPT_Y_TILE, (2, 4, 16)),
                          (chanfs.OPT_PCR_PARTS, (1, 3, 8)), (chanfs.OPT_FFT_RADIX, (4, 8))):
            for v in vals:
                plan.set_option(opt, v)
                assert plan.get_option(opt) == v
                p = host(plan.poisson_solve(dev(f)))
                u = host(plan.helmholtz_solve(c, dev(rhs)))
                assert rel(p, ref) < tol and rel(u, href) < tol, (opt, v)
            plan.set_option(opt, 0)
        thomas_opt = chanfs.OPT_HELM_THOMAS32 if dtype == 1 else chanfs.OPT_HELM_THOMAS
        for v in (1, 0):  # Thomas sweeps or Algorithm 2 for the Helmholtz systems
            plan.set_option(thomas_opt, v)
            assert plan.get_option(thomas_opt) == v
            u = host(plan.helmholtz_solve(c, dev(rhs)))
            assert rel(u, href) < tol, (thomas_opt, v)
        if dtype == 0:
            with pytest.raises(chanfs.ChanfsError) as err:
                plan.set_option(chanfs.OPT_HELM_THOMAS32, 1)  # FP64 plans have no FP32 solves
            assert err.value.status == chanfs.EUNSUPPORTED
        for opt, bad in ((chanfs.OPT_X_LINES, 65), (chanfs.OPT_Y_TILE, 33), (chanfs.OPT_PCR_PARTS, 65),
                         (chanfs.OPT_HELM_THOMAS, 2), (chanfs.OPT_HELM_THOMAS32, -1),
                         (chanfs.OPT_FFT_RADIX, 2)):
            with pytest.raises(chanfs.ChanfsError):
                plan.set_option(opt, bad)
        with pytest.raises(chanfs.ChanfsError) as err:
            plan.set_option(chanfs.OPT_PCR_PARTS, 20)  # 39 / 20 < 3 rows
        assert err.value.status == chanfs.EUNSUPPORTED
        chosen = plan.autotune()
        assert chosen["x_lines"] >= 1 and chosen["y_tile"] >= 1 and chosen["pcr_parts"] >= 1
        p = host(plan.poisson_solve(dev(f)))
        u = host(plan.helmholtz_solve(c, dev(rhs)))
        assert rel(p, ref) < tol and rel(u, href) < tol
        assert plan.check() == 0
    # a second plan of the same size takes the remembered choice
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, dtype) as plan2:
        assert plan2.autotune() == chosen


# The z-implicit Helmholtz systems by Thomas sweeps (the tuner's alternative
# to Algorithm 2): column counts that leave a partial block, columns shorter
# than the in-thread prefetch, centred and face fields
HTH_CASES = [
    ((64, 48, 40), 1.7, 0, 2e-5), ((64, 48, 40), 1.7, 1, 2e-5), ((24, 9, 5), 1.3, 0, 1e-2),
    ((24, 9, 4), 1.3, 1, 1e-2), ((12, 6, 33), None, 1, 0.3), ((36, 27, 19), 2.2, 0, 0.0),
]


@pytest.mark.parametrize("dims,beta,loc,c", HTH_CASES)
@pytest.mark.parametrize("dtype", [0, 1])
def test_helmholtz_thomas_matches_oracle(chanfs, dims, beta, loc, c, dtype):
    nx, ny, nz = dims
    if dtype == 1 and nx % 4:
        pytest.skip("refined plans need nx % 4 == 0")
    dz = make_dz(nz, beta)
    rhs = synth.normal(31 * nx + nz + loc, (nz, ny, nx))
    ref = oracle.helmholtz_solve(rhs, dz, c, loc)
    tol = 1e-10 if dtype == 1 else TOL
    with chanfs.Plan(nx, ny, nz, 1.0, 1.0, dz, 0, dtype) as plan:
        plan.set_option(chanfs.OPT_HELM_THOMAS32 if dtype == 1 else chanfs.OPT_HELM_THOMAS, 1)
        u = host(plan.helmholtz_solve(c, dev(rhs), loc))
        assert rel(u, ref) < tol, rel(u, ref)
        if loc == 1:
            assert np.all(u[-1] == 0.0)
        t = dev(rhs)  # in place
        plan.helmholtz_solve(c, t, loc, out=t)
        assert np.array_equal(host(t), u)
        if dtype == 1:  # FP64 direct solve by Thomas sweeps
            plan.set_option(chanfs.OPT_HELM_FP64, 1)
            plan.set_option(chanfs.OPT_HELM_THOMAS, 1)
            u64 = host(plan.helmholtz_solve(c, dev(rhs), loc))
            assert rel(u64, ref) < TOL, rel(u64, ref)
        assert plan.check() == 0


# Fully implicit 3-D Helmholtz (Eq. 8) on the Poisson machinery
HELM3_CASES = [
    ((32, 24, 20), 1.8, 0, 1e-3), ((32, 24, 20), 1.8, 1, 1e-3), ((48, 36, 33), 2.0, 0, 0.5),
    ((6, 9, 5), 1.2, 1, 1e-2), ((64, 288, 12), 1.5, 0, 1e-4), ((8, 1, 16), None, 1, 3.0),
    ((16, 12, 10), 1.4, 0, 0.0),
]


@pytest.mark.parametrize("dims,beta,loc,c", HELM3_CASES)
@pytest.mark.parametrize("dtype", [0, 1])
def test_helmholtz3d_matches_oracle(chanfs, dims, beta, loc, c, dtype):
    nx, ny, nz = dims
    if dtype == 1 and nx % 4:
        pytest.skip("refined plans need nx % 4 == 0")
    lx, ly = 2 * np.pi, np.pi
    dz = make_dz(nz, beta)
    f = synth.normal(13 * nx + ny + nz + loc, (nz, ny, nx))
    ref = oracle.helmholtz3d_solve(f, lx, ly, dz, c, loc)
    with chanfs.Plan(nx, ny, nz, lx, ly, dz, 0, dtype) as plan:
        u = host(plan.helmholtz3d_solve(c, dev(f), loc))
        assert rel(u, ref) < TOL, rel(u, ref)
        if loc == 1:
            assert np.all(u[-1] == 0.0)
        t = dev(f)
        plan.helmholtz3d_solve(c, t, loc, out=t)
        assert np.array_equal(host(t), u)
        # a second coefficient, then the first again (cached set)
        plan.helmholtz3d_solve(2 * c + 1e-3, dev(f), loc)
        assert np.array_equal(host(plan.helmholtz3d_solve(c, dev(f), loc)), u)
        assert plan.check() == 0


def sampled_residual(f, p, lx, ly, dz, bc, c=None, loc=0, samples=20000, seed=5):
    """max |f - L p| (Poisson) or |f - (p - c L_z p)| (Helmholtz, c given) at
    seeded sample points, with the oracle's z stencil, relative to max |f|."""
    nz, ny, nx = f.shape
    A, B, C = oracle.lz_coefficients(dz, bc, loc)
    n = len(A)
    rng = np.random.default_rng(seed)
    k = rng.integers(0, n, samples)
    j = rng.integers(0, ny, samples)
    i = rng.integers(0, nx, samples)
    P = p[k, j, i]
    Lz = B[k] * P
    Lz += np.where(k > 0, A[k] * p[np.maximum(k - 1, 0), j, i], 0.0)
    Lz += np.where(k < n - 1, C[k] * p[np.minimum(k + 1, n - 1), j, i], 0.0)
    if c is None:
        dx2, dy2 = (lx / nx) ** 2, (ly / ny) ** 2
        L = (p[k, j, (i + 1) % nx] - 2 * P + p[k, j, (i - 1) % nx]) / dx2
        L += (p[k, (j + 1) % ny, i] - 2 * P + p[k, (j - 1) % ny, i]) / dy2
        r = f[k, j, i] - (L + Lz)
    else:
        r = f[k, j, i] - (P - c * Lz)
    return float(np.max(np.abs(r)) / np.max(np.abs(f)))


@pytest.mark.slow
def test_stress_box_full_size(chanfs):
    """The 3456 x 3072 x 30 box of the benchmark (tuned shapes, both
    Helmholtz methods): the residual of the Eq. 12 / Eq. 11 operators at
    sampled points, and the zero weighted mean of the Poisson solution."""
    cfg = synth.STRESS
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    dz = synth.grid_dz(cfg)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg["seed"])
    f = torch.randn(nz, ny, nx, dtype=torch.float64, device="cuda", generator=gen)
    w = torch.from_numpy(dz).cuda()
    f -= (f.sum(dim=(1, 2)) * w).sum() / (w.sum() * nx * ny)
    fh = host(f)
    with chanfs.Plan(nx, ny, nz, cfg["lx"], cfg["ly"], dz, chanfs.NEUMANN) as plan:
        plan.autotune()
        p = host(plan.poisson_solve(f))
        assert sampled_residual(fh, p, cfg["lx"], cfg["ly"], dz, 0) < 1e-12
        mean = float(np.tensordot(p.sum(axis=(1, 2)), dz, 1) / (dz.sum() * nx * ny))
        assert abs(mean) < 1e-12 * np.max(np.abs(p))
        del p
        for thomas in (0, 1):
            plan.set_option(chanfs.OPT_HELM_THOMAS, thomas)
            for loc in (chanfs.CENTER, chanfs.FACE):
                u = host(plan.helmholtz_solve(synth.CHANNEL_C, f, loc))
                assert sampled_residual(fh, u, 0, 0, dz, 1, synth.CHANNEL_C, loc) < 1e-12
        assert plan.check() == 0


@pytest.mark.parametrize("dtype", [0, 1])
def test_thin_box_matches_oracle(chanfs, dtype):
    """A reduced box of the stress shape (x and y lengths with factors of 3,
    a thin z) against the oracle, Helmholtz by both methods."""
    nx, ny, nz = 432, 384, 30
    dz = make_dz(nz, 1.8)
    f = synth.remove_weighted_mean(synth.normal(91, (nz, ny, nx)), dz)
    tol = 1e-10 if dtype == 1 else TOL
    ref = oracle.poisson_solve(f, 12.8, 6.4, dz, 0)
    href = oracle.helmholtz_solve(f, dz, 1e-4, 1)
    with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz, 0, dtype) as plan:
        plan.autotune()
        assert rel(host(plan.poisson_solve(dev(f))), ref) < tol
        opt = chanfs.OPT_HELM_THOMAS32 if dtype == 1 else chanfs.OPT_HELM_THOMAS
        for v in (0, 1):
            plan.set_option(opt, v)
            assert rel(host(plan.helmholtz_solve(1e-4, dev(f), 1)), href) < tol
        assert plan.check() == 0


def test_tuning_choices_survive_a_file_round_trip(chanfs, tmp_path):
    """Choices saved to a file and loaded in a clean tuner are applied to new
    plans of the same size without timing; lines of another GPU are skipped
    and a malformed line is rejected."""
    nx, ny, nz = 64, 48, 40
    dz = make_dz(nz, 1.5)
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, chanfs.F32_REFINED) as plan:
        chosen = plan.autotune()
    path = tmp_path / "tune.txt"
    chanfs.autotune_save(path)
    text = path.read_text().splitlines()
    assert any(f" {nx} {ny} {nz} 1 " in line for line in text)
    chanfs.autotune_clear()
    other = tmp_path / "other.txt"
    other.write_text("chanfs-tune-1 Some_Other_GPU 8 8 8 0 1 1 -1 0 0 0 0 8\n"
                     + path.read_text())
    assert chanfs.autotune_load(other) >= 1
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, chanfs.F32_REFINED) as plan2:
        assert plan2.autotune() == chosen
    bad = tmp_path / "bad.txt"
    bad.write_text("not a tuning line\n")
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.autotune_load(bad)
    assert err.value.status == chanfs.EINVAL


@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_of_host_solves_matches_single_solves(chanfs, dtype):
    """A channel-like step through cfs_solve_batch_host (Poisson + three
    Helmholtz, copies overlapped with the solves) gives the bits of the
    device solves one by one; a second batch reuses the plan's slots."""
    nx, ny, nz = 64, 48, 40
    dz = make_dz(nz, 1.8)
    f = synth.remove_weighted_mean(synth.normal(61, (nz, ny, nx)), dz)
    rhs = [synth.normal(62 + i, (nz, ny, nx)) for i in range(3)]
    c = 2e-5
    locs = (chanfs.CENTER, chanfs.CENTER, chanfs.FACE)
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, dtype) as plan:
        want = [host(plan.poisson_solve(dev(f)))]
        want += [host(plan.helmholtz_solve(c, dev(r), loc)) for r, loc in zip(rhs, locs)]
        ins = [torch.from_numpy(x).pin_memory() for x in [f] + rhs]
        for _ in range(2):
            outs = [torch.full_like(x, float("nan")).pin_memory() for x in ins]
            jobs = [(chanfs.REQ_POISSON, 0.0, 0, ins[0], outs[0])]
            jobs += [(chanfs.REQ_HELMHOLTZ, c, loc, ins[1 + i], outs[1 + i])
                     for i, loc in enumerate(locs)]
            plan.solve_batch_host(jobs)
            for got, w in zip(outs, want):
                assert np.array_equal(got.numpy(), w)
        assert plan.check() == 0


@pytest.mark.parametrize("dims,chunks,ybc,thomas", [
    ((64, 48, 40), 2, 0, 0), ((64, 48, 40), 3, 0, 0), ((64, 48, 40), 8, 0, 0),
    ((96, 36, 27), 5, 0, 0), ((32, 6, 17), 8, 0, 0), ((64, 48, 40), 3, 1, 0),
    ((64, 48, 40), 3, 0, 1), ((48, 2, 9), 4, 2, 0),
])
def test_streamed_batch_matches_single_solves(chanfs, dims, chunks, ybc, thomas):
    """FP64 batches streamed in chunks (CFS_OPT_STREAM_CHUNKS: z-plane ranges
    of Poisson fields, y-row ranges of Helmholtz fields, more chunks than y
    rows or z planes, y walls, Thomas Helmholtz solves taking whole fields)
    give the bits of the device solves, for job orders that move the first
    Helmholtz solve ahead and batches larger than the plan's four slots."""
    nx, ny, nz = dims
    dz = make_dz(nz, 1.5)
    f = [synth.normal(71 + i, (nz, ny, nx)) for i in range(2)]
    if ybc != 2:
        f = [synth.remove_weighted_mean(x, dz) for x in f]
    rhs = [synth.normal(75 + i, (nz, ny, nx)) for i in range(4)]
    c = 3e-5
    with chanfs.Plan(nx, ny, nz, 2.0, 1.0, dz, 0, 0, ybc) as plan:
        plan.set_option(chanfs.OPT_HELM_THOMAS, thomas)
        plan.set_option(chanfs.OPT_STREAM_CHUNKS, chunks)
        assert plan.get_option(chanfs.OPT_STREAM_CHUNKS) == min(chunks, nz)
        P = lambda k: (chanfs.REQ_POISSON, 0.0, 0, f[k])
        H = lambda k, loc: (chanfs.REQ_HELMHOLTZ, c, loc, rhs[k])
        for order in ([P(0), H(0, 0), H(1, 0), H(2, 1)],
                      [H(0, 1), P(0), P(1), H(1, 0), H(2, 0), H(3, 1)],
                      [P(1), P(0)], [H(3, 0)]):
            want = []
            for kind, cc, loc, x in order:
                d = dev(x)
                want.append(host(plan.poisson_solve(d) if kind == chanfs.REQ_POISSON
                                 else plan.helmholtz_solve(cc, d, loc)))
            ins = [torch.from_numpy(x).pin_memory() for *_, x in order]
            outs = [torch.full_like(x, float("nan")).pin_memory() for x in ins]
            plan.solve_batch_host([(k, cc, loc, a, b) for (k, cc, loc, _), a, b
                                   in zip(order, ins, outs)])
            for got, w in zip(outs, want):
                assert np.array_equal(got.numpy(), w)
        assert plan.check() == 0
