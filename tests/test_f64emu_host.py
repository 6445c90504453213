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

import numpy as np
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


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)


def _same(x, y):
    return (_bits(x) == _bits(y)) | (np.isnan(x) & np.isnan(y))


def _structured_operands():
    """Operand pairs built to hit every branch of the integer path and its
    limits: exponent differences 0..70 (alignment shifts, the sticky bit,
    operands shifted out entirely) for significands with few, many and
    alternating bits; cancellation of equal and nearly equal magnitudes;
    exact ties at the rounding position with odd and even kept parts;
    carries of the rounding into the next binade; the ends of the integer
    path's exponent range and the values just outside it (zeros,
    subnormals, tiny and huge numbers, infinities, NaN)."""
    fracs = np.array([0, 1, 2, 3, (1 << 52) - 1, (1 << 51), (1 << 51) + 1, 0x5555555555555,
                      0xAAAAAAAAAAAAA, 0x8000000000001, (1 << 52) - 2, 0x0000000000400],
                     dtype=np.uint64)
    a, b = [], []
    for ea in (64, 65, 500, 1023, 1024, 2000, 2044, 2045):
        for d in range(0, 71):
            eb = ea - d
            if eb < 1:
                continue
            for fa in fracs:
                for fb in fracs[::3]:
                    for sa in (0, 1):
                        for sb in (0, 1):
                            a.append((sa << 63) | (ea << 52) | int(fa))
                            b.append((sb << 63) | (eb << 52) | int(fb))
    a = np.array(a, dtype=np.uint64).view(np.float64)
    b = np.array(b, dtype=np.uint64).view(np.float64)
    # nearly equal magnitudes: b = a with its last bits changed, both signs
    rng = np.random.default_rng(7)
    base = rng.standard_normal(4000) * np.exp2(rng.integers(-900, 900, 4000))
    near = (_bits(base) ^ rng.integers(0, 1 << 16, 4000).astype(np.uint64)).view(np.float64)
    # ties: b is half a unit in the last place of a (and 3/2, 5/2 units) at several scales
    t = rng.standard_normal(2000)
    ulp = np.spacing(np.abs(t))
    specials = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300,
                         2.0 ** -959, 2.0 ** -960, 2.0 ** 1022, 2.0 ** 1023, 1.7976931348623157e308,
                         np.inf, -np.inf, np.nan, 1.0, -1.0, 3.0])
    sa, sb = np.meshgrid(specials, specials)
    return (np.concatenate([a, base, base, t, t, t, sa.ravel()]),
            np.concatenate([b, near, -near, ulp / 2, 3 * ulp / 2, -5 * ulp / 2, sb.ravel()]))


def test_structured_operands_match_numpy_ieee_arithmetic():
    a, b = _structured_operands()
    assert a.size > 100000
    s, d = chanfs.f64_addsub_host(a, b)
    with np.errstate(all="ignore"):
        want_s, want_d = a + b, a - b
    assert _same(s, want_s).all()
    assert _same(d, want_d).all()


def test_host_entry_point_arguments():
    lib = chanfs.lib()
    assert lib.cfs_f64_addsub_host(-1, None, None, None, None) == chanfs.EINVAL
    assert lib.cfs_f64_addsub_host(3, None, None, None, None) == chanfs.EINVAL
    assert lib.cfs_f64_addsub_host(0, None, None, None, None) == chanfs.OK
    with pytest.raises(ValueError):
        chanfs.f64_addsub_host(np.zeros(3), np.zeros(4))
