"""CPU: the integer-unit FP64 additions of the transforms, run on the host.

cfs_selfcheck_f64_addsub(on_device=0) executes the same host/device
functions the FP64 transforms call on the GPU, here on the CPU, and compares
each sum and difference bit for bit with the CPU's own IEEE-754 binary64
arithmetic (round to nearest, ties to even) over hashed operand pairs of
eight kinds (any bit patterns, close and distant exponents, cancellation,
exact ties, the ends of the integer range, equal magnitudes, FFT-sized
values).  No GPU is needed.
"""

import ctypes

import pytest

from paper_2502_06296_gb300 import chanfs


def test_host_additions_are_ieee_exact():
    assert chanfs.selfcheck_f64_addsub(1 << 23, on_device=False) == 0


def test_selfcheck_arguments():
    lib = chanfs.lib()
    bad = ctypes.c_ulonglong(0)
    assert lib.cfs_selfcheck_f64_addsub(0, 0, ctypes.byref(bad)) == chanfs.EINVAL
    assert lib.cfs_selfcheck_f64_addsub(16, 2, ctypes.byref(bad)) == chanfs.EINVAL
    assert lib.cfs_selfcheck_f64_addsub(16, 0, None) == chanfs.EINVAL
    rate = ctypes.c_double(0.0)
    assert lib.cfs_probe_addsub(2, 100, ctypes.byref(rate), None) == chanfs.EINVAL
    assert lib.cfs_probe_addsub(1, 0, ctypes.byref(rate), None) == chanfs.EINVAL
    assert lib.cfs_probe_addsub(1, 100, None, None) == chanfs.EINVAL


@pytest.mark.parametrize("samples", [1, 7, 1000])
def test_small_sample_counts(samples):
    assert chanfs.selfcheck_f64_addsub(samples, on_device=False) == 0
