"""Host-side checks of the index arithmetic behind the kernels' shared-memory
and scratch layouts, restated in Python (no GPU).

* The compile-time Stockham plans (radix 8, then 4, 2, 3) with the padded
  layout between passes (element e at e + e/16): every pass writes each
  element exactly once, inside the buffer the launch sizes, and a warp's
  8-byte accesses put at most X_WORST lanes on one bank pair (2, the
  minimum, for x lengths from 256 up and for the y tiles).
* The refined start pass's partition of each z plane into chunks covers the
  plane exactly, and its partial sums fit the plan's scratch.
* The order-preserving keys of the start pass's extremes.
"""

from collections import Counter

import numpy as np
import pytest

X_LENGTHS = [32, 48, 64, 96, 128, 192, 256, 384, 512, 1024]
Y_LENGTHS = [64, 96, 128, 192, 256, 384, 512, 768]
MAX_START_CHUNKS = 16


def fixed_radix(n, p):
    rest, q = n, 0
    for r in (8, 4):
        while rest % r == 0:
            if q == p:
                return r
            rest //= r
            q += 1
    if rest % 2 == 0:
        if q == p:
            return 2
        rest //= 2
        q += 1
    while rest % 3 == 0:
        if q == p:
            return 3
        rest //= 3
        q += 1
    return 0


def npass(n):
    p = 0
    while fixed_radix(n, p):
        p += 1
    return p


def span(n, p):
    out = 1
    for i in range(p):
        out *= fixed_radix(n, i)
    return out


def pad16(e):
    return e + (e >> 4)


def padded(n):
    return n + n // 16


def xbuf_elems(lines, m):  # FP32 buffers
    e = lines * padded(m)
    return (e + 1) & ~1


def y_buf_elems(tk, n):  # FP32 tiles, 8-byte elements, rounded to 128 bytes
    e = tk * n + tk * n // 16
    return (e * 8 + 127) // 128 * 128 // 8


def passes(n):
    for p in range(npass(n)):
        r, L = fixed_radix(n, p), span(n, p)
        yield p, r, L, n // r, p > 0, p + 1 < npass(n)


@pytest.mark.parametrize("n", X_LENGTHS)
def test_fixed_plans_factor_the_length(n):
    prod = 1
    for p in range(npass(n)):
        prod *= fixed_radix(n, p)
    assert prod == n


@pytest.mark.parametrize("n", X_LENGTHS)
@pytest.mark.parametrize("lines", [1, 2, 3, 4, 7, 16])
def test_x_line_passes_write_every_element_once_in_bounds(n, lines):
    cap = xbuf_elems(lines, n)
    for _, r, L, q, pin, pout in passes(n):
        sin, sout = (padded(n) if pin else n), (padded(n) if pout else n)
        reads, writes = [], []
        for bat in range(lines):
            for j in range(q):
                k = j % L
                o = (j - k) * r + k
                for rr in range(r):
                    e = j + rr * q
                    reads.append(bat * sin + (pad16(e) if pin else e))
                    w = o + rr * L
                    writes.append(bat * sout + (pad16(w) if pout else w))
        assert max(reads) < cap and max(writes) < cap
        assert len(set(reads)) == len(reads) == lines * n
        assert len(set(writes)) == len(writes) == lines * n


def lanes_per_bank_pair(addrs):
    return max(Counter(a % 16 for a in addrs).values())


def worst_x_lanes(n, lines, pad):
    """Most lanes of one warp on one bank pair over every access of every
    pass: thread t takes butterfly t % Q of line t / Q, as the kernel does."""
    worst = 0
    for _, r, L, q, pin, pout in passes(n):
        sin = padded(n) if (pin and pad) else n
        sout = padded(n) if (pout and pad) else n
        total = q * lines
        for w0 in range(0, total, 32):
            ts = range(w0, min(w0 + 32, total))
            for rr in range(r):
                rd, wr = [], []
                for t in ts:
                    bat, j = t // q, t % q
                    e = j + rr * q
                    rd.append(bat * sin + (pad16(e) if (pin and pad) else e))
                    k = j % L
                    o = (j - k) * r + k + rr * L
                    wr.append(bat * sout + (pad16(o) if (pout and pad) else o))
                worst = max(worst, lanes_per_bank_pair(rd), lanes_per_bank_pair(wr))
    return worst


# the minimum is 2 (32 lanes x 8 bytes = two 128-byte wavefronts)
X_WORST = {32: 4, 48: 4, 64: 4, 96: 4, 128: 2, 192: 3, 256: 2, 384: 2, 512: 2, 1024: 2}


@pytest.mark.parametrize("n", X_LENGTHS)
def test_x_line_passes_bank_conflicts(n):
    padded_worst = worst_x_lanes(n, 4, True)
    assert padded_worst <= X_WORST[n]
    assert padded_worst < worst_x_lanes(n, 4, False)  # unpadded: up to 16 lanes


@pytest.mark.parametrize("n", Y_LENGTHS)
@pytest.mark.parametrize("tk", [2, 4, 8, 16, 32])
def test_y_tile_passes_in_bounds_and_conflict_free(n, tk):
    cap = y_buf_elems(tk, n)
    threads = 256
    for _, r, L, q, pin, pout in passes(n):
        writes = set()
        for t in range(q * tk):
            c, j = t % tk, t // tk
            k = j % L
            for rr in range(r):
                i = (j + rr * q) * tk + c
                assert (pad16(i) if pin else i) < cap
                o = ((j - k) * r + k + rr * L) * tk + c
                writes.add(pad16(o) if pout else o)
        assert len(writes) == q * tk * r == n * tk
        assert max(writes) < cap
        for w0 in range(0, min(q * tk, threads), 32):
            ts = [t for t in range(w0, w0 + 32) if t < q * tk]
            for rr in range(r):
                rd, wr = [], []
                for t in ts:
                    c, j = t % tk, t // tk
                    k = j % L
                    i = (j + rr * q) * tk + c
                    o = ((j - k) * r + k + rr * L) * tk + c
                    rd.append(pad16(i) if pin else i)
                    wr.append(pad16(o) if pout else o)
                assert lanes_per_bank_pair(rd) <= 2
                assert lanes_per_bank_pair(wr) <= 2


def start_chunks(nz):
    c = (2432 + nz - 1) // nz
    return max(1, min(MAX_START_CHUNKS, c))


@pytest.mark.parametrize("nz", [1, 3, 30, 64, 152, 512, 2432, 5000])
@pytest.mark.parametrize("n2", [1, 7, 1000, 196608])
def test_start_pass_chunks_cover_each_plane(nz, n2):
    nch = start_chunks(nz)
    covered = []
    for c in range(nch):
        lo, hi = n2 * c // nch, n2 * (c + 1) // nch
        covered.extend(range(lo, hi))
    assert covered == list(range(n2))
    # partials at d_red + 3 .. + 3 + nz * nch within nz * nch + 8 doubles
    assert 3 + nz * nch <= nz * nch + 8


def float_key(v):
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000).astype(np.uint64)


def key_float(k):
    k = np.asarray(k, dtype=np.uint64)
    u = np.where(k & 0x80000000, k & 0x7FFFFFFF, (~k) & 0xFFFFFFFF).astype(np.uint32)
    return u.view(np.float32)


def test_extreme_keys_preserve_order():
    rng = np.random.default_rng(2502)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.17549435e-38,
                        -3.4028235e38, 3.4028235e38], dtype=np.float32)
    v = np.concatenate([special, rng.standard_normal(4000).astype(np.float32) *
                        np.float32(10.0) ** rng.integers(-40, 38, 4000).astype(np.float32)])
    v = v[np.isfinite(v) | np.isinf(v)]
    order = np.lexsort((~np.signbit(v), v))  # by value, -0 before +0 (the keys' order)
    keys = float_key(v)
    sv, sk = v[order], keys[order]
    # keys are non-decreasing along increasing values, strictly where values differ
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)
    differ = np.diff(sv) > 0
    assert np.all(np.diff(sk.astype(np.int64))[differ] > 0)
    assert np.array_equal(key_float(keys).view(np.uint32), v.view(np.uint32))
    assert np.all(keys > 0)  # a zeroed word is below every key
