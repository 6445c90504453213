"""The C-ABI library builds, loads and exports every entry point that
include/chanfs.h declares; host-side argument checks work without a GPU."""

import ctypes
import re

import numpy as np
import pytest

from paper_2502_06296_gb300 import build as libbuild
from paper_2502_06296_gb300 import chanfs


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return chanfs.lib()


def test_header_declares_the_boundary():
    names = chanfs.exported_symbols()
    for required in ["cfs_plan_create", "cfs_plan_destroy", "cfs_poisson_solve",
                     "cfs_helmholtz_prepare", "cfs_helmholtz_solve", "cfs_spectral_forward",
                     "cfs_spectral_inverse", "cfs_poisson_solve_host", "cfs_helmholtz_solve_host",
                     "cfs_plan_check", "cfs_status_string", "cfs_version", "cfs_plan_device_bytes"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in chanfs.exported_symbols():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert lib.cfs_version() == 100
    for s in range(-8, 1):
        assert chanfs.status_string(s) not in ("", "unknown status")
    assert chanfs.status_string(-99) == "unknown status"


def _create(lib, nx, ny, nz, lx=1.0, ly=1.0, dz=None, bc=0, dtype=0):
    dz = np.full(nz, 2.0 / max(nz, 1)) if dz is None else np.asarray(dz, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = lib.cfs_plan_create(ctypes.byref(h), nx, ny, nz, lx, ly,
                             dz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), bc, dtype)
    return rc, h


@pytest.mark.parametrize("args,expect", [
    (dict(nx=7, ny=8, nz=8), chanfs.EUNSUPPORTED),      # odd nx
    (dict(nx=10, ny=8, nz=8), chanfs.EUNSUPPORTED),     # nx/2 = 5 not 2^a 3^b
    (dict(nx=8, ny=5, nz=8), chanfs.EUNSUPPORTED),      # ny = 5
    (dict(nx=8, ny=8192, nz=8), chanfs.EUNSUPPORTED),   # ny too large
    (dict(nx=8192, ny=8, nz=8), chanfs.EUNSUPPORTED),   # nx too large
    (dict(nx=8, ny=8, nz=2), chanfs.EINVAL),            # nz < 3
    (dict(nx=0, ny=8, nz=8), chanfs.EINVAL),
    (dict(nx=8, ny=8, nz=8, lx=0.0), chanfs.EINVAL),
    (dict(nx=8, ny=8, nz=8, ly=float("nan")), chanfs.EINVAL),
    (dict(nx=8, ny=8, nz=8, bc=5), chanfs.EINVAL),
    (dict(nx=8, ny=8, nz=8, dtype=3), chanfs.EUNSUPPORTED),
    (dict(nx=8, ny=8, nz=4, dz=[0.5, 0.5, -0.5, 0.5]), chanfs.EINVAL),
    (dict(nx=8, ny=8, nz=4, dz=[0.5, 0.5, float("inf"), 0.5]), chanfs.EINVAL),
])
def test_plan_create_rejects_bad_arguments_on_the_host(lib, args, expect):
    rc, h = _create(lib, **args)
    assert rc == expect
    assert not h.value


def test_null_handles_are_rejected(lib):
    assert lib.cfs_plan_create(None, 8, 8, 8, 1.0, 1.0, None, 0, 0) == chanfs.EINVAL
    assert lib.cfs_plan_destroy(None) == chanfs.EINVAL
    assert lib.cfs_poisson_solve(None, None, None, None) == chanfs.EINVAL
    assert lib.cfs_helmholtz_solve(None, 0.0, 0, None, None, None) == chanfs.EINVAL
    assert lib.cfs_helmholtz_prepare(None, 0.0, 0, 0) == chanfs.EINVAL
    assert lib.cfs_plan_check(None, None) == chanfs.EINVAL
    assert lib.cfs_spectral_forward(None, None, None, None) == chanfs.EINVAL
    assert lib.cfs_poisson_solve_host(None, None, None, None) == chanfs.EINVAL
    assert lib.cfs_plan_check_guards(None, None) == chanfs.EINVAL
    assert lib.cfs_plan_debug_guard_poke(None, 0, 0) == chanfs.EINVAL
    assert lib.cfs_group_set_trace(None, 1) == chanfs.EINVAL
    assert lib.cfs_group_trace(None, None, 0, None) == chanfs.EINVAL


def test_product_package_does_not_import_the_oracle():
    import os
    pkg = os.path.dirname(chanfs.__file__)
    for root, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                src = open(os.path.join(root, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), fn
                assert "chanfs_oracle" not in src, fn


def test_tuning_file_entry_points_check_their_arguments(lib, tmp_path):
    assert lib.cfs_autotune_save(None) == chanfs.EINVAL
    assert lib.cfs_autotune_load(None, None) == chanfs.EINVAL
    missing = str(tmp_path / "no_such_file").encode()
    n = ctypes.c_int(7)
    assert lib.cfs_autotune_load(missing, ctypes.byref(n)) == chanfs.EINVAL
    assert n.value == 0
    assert lib.cfs_autotune_clear() == chanfs.OK


def test_batch_host_entry_point_checks_its_arguments(lib):
    i3 = (ctypes.c_int * 1)(5)  # not a request kind
    p = (ctypes.c_void_p * 1)(None)
    assert lib.cfs_solve_batch_host(None, 1, i3, None, None, p, p, None) == chanfs.EINVAL
    assert lib.cfs_solve_batch_host(None, -1, None, None, None, None, None, None) == chanfs.EINVAL


def test_server_and_selftest_entry_points_check_their_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.cfs_server_create(None, 1 << 30, 1, 1, 1, 0) == chanfs.EINVAL
    assert lib.cfs_server_create(ctypes.byref(h), 1 << 30, 0, 1, 1, 0) == chanfs.EINVAL
    assert lib.cfs_server_create(ctypes.byref(h), 1 << 30, 1, 1, 0, 0) == chanfs.EINVAL
    assert lib.cfs_server_create(ctypes.byref(h), 1 << 30, 1, 1, 17, 0) == chanfs.EINVAL
    assert lib.cfs_server_cancel(None, 1) == chanfs.EINVAL
    assert lib.cfs_server_pause(None, 1) == chanfs.EINVAL
    assert lib.cfs_server_inject_fault(None, chanfs.FAULT_PLAN_ALLOC, 1) == chanfs.EINVAL
    assert lib.cfs_server_inject_fault(None, chanfs.FAULT_WORKER_START, -1) == chanfs.EINVAL
    # exactly one of plan and device_status; polls within range
    assert lib.cfs_selftest_wait_timeout(None, None, 100, None) == chanfs.EINVAL
    assert lib.cfs_selftest_wait_timeout(None, ctypes.c_void_p(16), 0, None) == chanfs.EINVAL
    assert lib.cfs_selftest_wait_timeout(None, ctypes.c_void_p(16), (1 << 20) + 1, None) == chanfs.EINVAL


def test_probe_checks_its_arguments(lib):
    rate = ctypes.c_double(0.0)
    assert lib.cfs_probe_fma(16, 100, ctypes.byref(rate), None) == chanfs.EINVAL
    assert lib.cfs_probe_fma(64, 0, ctypes.byref(rate), None) == chanfs.EINVAL
    assert lib.cfs_probe_fma(64, 100, None, None) == chanfs.EINVAL
