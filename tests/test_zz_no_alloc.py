"""GPU: the allocation-free Helmholtz entry point against the regular one and
against the oracle.

cfs_helmholtz_solve_noalloc serves callers that cannot allocate device memory
where they solve (cudaMalloc/cudaFree synchronise the device; some
applications reserve all device memory for their own pool).  It computes its
coefficients on the GPU into a fixed array inside the library instead of
plan memory.  Two calls in a row, each compared with cfs_helmholtz_solve on
the same input and with the CPU oracle, at the tolerance of the other GPU
tests; the caller's status word must come back 0.  This file runs last on
purpose.
"""

import ctypes

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
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_matches_plan_entry_point_and_oracle_twice(chanfs):
    nx, ny, nz = 48, 36, 384
    dz = synth.tanh_dz(nz, 1.8)
    dz_ptr = np.ascontiguousarray(dz).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    calls = [(9.615e-9, chanfs.CENTER, 0, 11), (1e-3, chanfs.FACE, 12, 12)]
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    with chanfs.Plan(nx, ny, nz, 12.8, 6.4, dz) as plan:
        for c, loc, nparts, seed in calls:
            rhs_h = synth.normal(seed, (nz, ny, nx))
            ref_oracle = torch.from_numpy(oracle.helmholtz_solve(rhs_h, dz, c, loc))
            rhs = torch.from_numpy(rhs_h).cuda()
            plan.helmholtz_prepare(c, loc, nparts)
            plan.set_option(chanfs.OPT_PCR_PARTS, nparts)
            ref = plan.helmholtz_solve(c, rhs, loc)
            # the C ABI directly, then the binding
            out = torch.empty_like(rhs)
            rc = chanfs.lib().cfs_helmholtz_solve_noalloc(
                nx, ny, nz, dz_ptr, c, loc, nparts, ctypes.c_void_p(rhs.data_ptr()),
                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == chanfs.OK
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert rel(out, ref) < TOL
            assert rel(out.cpu(), ref_oracle) < TOL
            out2, st2 = chanfs.helmholtz_solve_noalloc(dz, c, rhs, loc, nparts)
            torch.cuda.synchronize()
            assert int(st2.item()) == 0
            assert rel(out2, ref) < TOL
            assert rel(out2.cpu(), ref_oracle) < TOL
            if loc == chanfs.FACE:
                assert bool((out[-1] == 0).all())
        assert plan.check() == 0


def test_noalloc_rejects_sizes_beyond_its_array(chanfs):
    dz = np.full(1100, 2.0 / 1100)
    rhs = torch.zeros(1100, 2, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.helmholtz_solve_noalloc(dz, 1e-3, rhs)
    assert err.value.status == chanfs.EUNSUPPORTED
    with pytest.raises(chanfs.ChanfsError) as err:
        chanfs.helmholtz_solve_noalloc(np.full(40, 0.05), 1e-3,
                                       torch.zeros(40, 2, 4, dtype=torch.float64, device="cuda"),
                                       nparts=65)
    assert err.value.status == chanfs.EUNSUPPORTED
    # a missing status word is an argument error, caught before anything is queued
    rhs = torch.zeros(40, 2, 4, dtype=torch.float64, device="cuda")
    d = np.full(40, 0.05)
    rc = chanfs.lib().cfs_helmholtz_solve_noalloc(
        4, 2, 40, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1e-3, 0, 0,
        ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(rhs.data_ptr()), None, None)
    assert rc == chanfs.EINVAL
