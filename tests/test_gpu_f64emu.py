"""GPU: the FP64 transforms with part of their butterfly additions on the
integer units (CFS_OPT_F64_ADDS_X / _Y).

Those additions are exact IEEE-754 binary64 round-to-nearest-even additions
done in integer arithmetic, so every level must give the FP64 pipe's bits:
the device self-check compares them with the hardware's over hashed operand
pairs, and whole solves at every level are compared bit for bit with level 0
(plus the oracle at 1e-12 on one emulated plan).  Sizes cover radix-8, 4, 2
and 3 passes along x and y, Ny = 1, odd Nz, the radix-4 option and two TMA
boxes along y.
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


def test_integer_unit_additions_match_the_fp64_pipe(chanfs):
    assert chanfs.selfcheck_f64_addsub(1 << 24, on_device=True) == 0


LEVELS = [(1, 1), (2, 2), (3, 3), (4, 4), (4, 0), (0, 4), (2, 3)]
CASES = [  # (nx, ny, nz, stretching, radix)
    (512, 384, 24, 1.8, 8), (96, 48, 40, 1.5, 8), (24, 36, 17, 1.2, 8), (64, 1, 8, None, 8),
    (128, 96, 33, 1.8, 4), (48, 288, 6, 1.4, 8), (2048, 6, 4, None, 8),
]


@pytest.mark.parametrize("nx,ny,nz,beta,radix", CASES)
def test_every_level_gives_the_fp64_bits(chanfs, nx, ny, nz, beta, radix):
    dz = synth.tanh_dz(nz, beta) if beta else np.full(nz, 2.0 / nz)
    f_h = synth.remove_weighted_mean(synth.normal(nx + ny + nz, (nz, ny, nx)), dz)
    f = torch.from_numpy(f_h).cuda()
    with chanfs.Plan(nx, ny, nz, 2 * np.pi, np.pi, dz) as plan:
        plan.set_option(chanfs.OPT_FFT_RADIX, radix)
        plan.set_option(chanfs.OPT_F64_ADDS_X, 0)
        plan.set_option(chanfs.OPT_F64_ADDS_Y, 0)
        ref_p = plan.poisson_solve(f).clone()
        ref_s = plan.spectral_forward(f).clone()
        ref_h = plan.helmholtz3d_solve(1e-3, f).clone()
        ref_i = plan.spectral_inverse(ref_s).clone()
        for lx, ly in LEVELS:
            plan.set_option(chanfs.OPT_F64_ADDS_X, lx)
            plan.set_option(chanfs.OPT_F64_ADDS_Y, ly)
            assert plan.get_option(chanfs.OPT_F64_ADDS_X) == lx
            assert plan.get_option(chanfs.OPT_F64_ADDS_Y) == ly
            assert torch.equal(plan.spectral_forward(f), ref_s), (lx, ly)
            assert torch.equal(plan.poisson_solve(f), ref_p), (lx, ly)
            assert torch.equal(plan.helmholtz3d_solve(1e-3, f), ref_h), (lx, ly)
            assert torch.equal(plan.spectral_inverse(ref_s), ref_i), (lx, ly)
        assert plan.check() == 0


def test_emulated_plan_matches_oracle(chanfs):
    nx, ny, nz = 96, 72, 30
    dz = synth.tanh_dz(nz, 1.8)
    f_h = synth.remove_weighted_mean(synth.normal(5, (nz, ny, nx)), dz)
    ref = oracle.poisson_solve(f_h, 2 * np.pi, np.pi, dz, 0)
    with chanfs.Plan(nx, ny, nz, 2 * np.pi, np.pi, dz) as plan:
        plan.set_option(chanfs.OPT_F64_ADDS_X, 4)
        plan.set_option(chanfs.OPT_F64_ADDS_Y, 4)
        p = plan.poisson_solve(torch.from_numpy(f_h).cuda()).cpu().numpy()
    assert float(np.max(np.abs(p - ref)) / np.max(np.abs(ref))) < TOL


@pytest.mark.parametrize("ybc", [1, 2])
def test_every_level_gives_the_fp64_bits_with_y_walls(chanfs, ybc):
    nx, ny, nz = 64, 24, 12
    dz = synth.tanh_dz(nz, 1.5)
    f_h = synth.normal(ybc, (nz, ny, nx))
    if ybc == 1:
        f_h = synth.remove_weighted_mean(f_h, dz)
    f = torch.from_numpy(f_h).cuda()
    with chanfs.Plan(nx, ny, nz, 2 * np.pi, np.pi, dz, ybc=ybc) as plan:
        plan.set_option(chanfs.OPT_F64_ADDS_X, 0)
        plan.set_option(chanfs.OPT_F64_ADDS_Y, 0)
        ref = plan.poisson_solve(f).clone()
        plan.set_option(chanfs.OPT_F64_ADDS_X, 4)
        plan.set_option(chanfs.OPT_F64_ADDS_Y, 4)
        assert torch.equal(plan.poisson_solve(f), ref)


def test_level_is_checked(chanfs):
    with chanfs.Plan(16, 8, 8, 1.0, 1.0, np.full(8, 0.25)) as plan:
        for opt in (chanfs.OPT_F64_ADDS_X, chanfs.OPT_F64_ADDS_Y):
            for bad in (-1, 5):
                with pytest.raises(chanfs.ChanfsError) as err:
                    plan.set_option(opt, bad)
                assert err.value.status == chanfs.EINVAL
