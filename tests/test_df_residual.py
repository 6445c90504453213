"""The refinement's first Poisson residual in double-float arithmetic with the
stencil written in differences, emulated operation by operation in numpy
float32 (no GPU), against the exact residual (rational arithmetic) of the same
FP64 operator, beside a plain double-float evaluation of the direct form and
a direct FP64 evaluation.

What it pins (the analysis behind the kernel): the difference form's error is
within 2^-44 of sum c|d_n - d| + |f| (a few roundings of 2^-48 each); it
stays within the factor 16 h |grad d| / |d| <= 2^5 of a direct FP64
evaluation's; and for a smooth correction (what the first FP32 solve of a
Poisson problem returns) it is several times below the plain double-float
evaluation's (whose error scales with sum |c d|, the size of the terms that
cancel) and far below the refinement's tolerance (1e-10 of max |f|).
"""

from fractions import Fraction

import numpy as np
import pytest

from paper_2502_06296_gb300 import synth

f32 = np.float32


def split(v):
    hi = np.float32(v)
    return hi, np.float32(np.float64(v) - np.float64(hi))


def fma(a, b, c):  # a * b exact in FP64 (24 + 24 bits); one rounding to FP32 after the add
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def df_acc(acc, ch, cl, d, init=False):
    p = f32(ch * d)
    e = fma(ch, d, -p)
    e = fma(cl, d, e)
    if init:
        return [p, e]
    s, t = two_sum(acc[0], p)
    return [s, f32(acc[1] + f32(t + e))]


def diff_acc(acc, ch, cl, a, b, init=False):
    dh, dl = two_sum(a, -b)
    q = f32(ch * dh)
    e = fma(ch, dh, -q)
    e = fma(ch, dl, e)
    e = fma(cl, dh, e)
    if init:
        return [q, e]
    s, t = two_sum(acc[0], q)
    return [s, f32(acc[1] + f32(t + e))]


def operator(nz, dz, nx, ny, lx, ly):
    """Rows A_k | B'_k | C_k of the Neumann z operator (flux form on the
    staggered grid) and 1/dx^2, 1/dy^2, all as FP64 values."""
    zc = np.cumsum(dz) - 0.5 * dz
    dzc = np.diff(zc)  # centre spacings
    A = np.zeros(nz)
    C = np.zeros(nz)
    A[1:] = 1.0 / (dz[1:] * dzc)
    C[:-1] = 1.0 / (dz[:-1] * dzc)
    idx2, idy2 = 1.0 / (lx / nx) ** 2, 1.0 / (ly / ny) ** 2
    Bp = -(A + C) - 2.0 * idx2 - 2.0 * idy2
    return A, Bp, C, idx2, idy2


def residuals(f, d, A, Bp, C, idx2, idy2):
    """(exact, difference-form double-float, direct FP64) residuals
    f - L d at every point (periodic x, y; Neumann z)."""
    nz, ny, nx = d.shape
    D = []
    for k in range(nz):  # D_k summed exactly, split as the library does
        s = Fraction(A[k]) + Fraction(Bp[k]) + Fraction(C[k]) + 2 * Fraction(idx2) + \
            2 * Fraction(idy2)
        D.append(float(s))
    ex = np.zeros_like(f)
    dfv = np.zeros_like(f)
    dir64 = np.zeros_like(f)
    ax = split(idx2)
    ay = split(idy2)
    for k in range(nz):
        ac, cc, dd = split(A[k]), split(C[k]), split(D[k])
        for j in range(ny):
            for i in range(nx):
                dk = d[k, j, i]
                dm = d[k - 1, j, i] if k > 0 else f32(0)
                dp = d[k + 1, j, i] if k + 1 < nz else f32(0)
                xp, xm = d[k, j, (i + 1) % nx], d[k, j, i - 1]
                yp, ym = d[k, (j + 1) % ny, i], d[k, j - 1, i]
                terms = [(A[k], dm), (Bp[k], dk), (C[k], dp), (idx2, xp), (idx2, xm),
                         (idy2, yp), (idy2, ym)]
                ex[k, j, i] = float(Fraction(f[k, j, i]) -
                                    sum(Fraction(c) * Fraction(float(v)) for c, v in terms))
                t = np.float64(Bp[k]) * np.float64(dk)
                t = np.fma(idx2, np.float64(xp) + np.float64(xm), t) if hasattr(np, "fma") \
                    else t + idx2 * (np.float64(xp) + np.float64(xm))
                t = t + idy2 * (np.float64(yp) + np.float64(ym))
                t = t + A[k] * np.float64(dm) + C[k] * np.float64(dp)
                dir64[k, j, i] = f[k, j, i] - t
                acc = diff_acc(None, ac[0], ac[1], dm, dk, init=True)
                acc = diff_acc(acc, cc[0], cc[1], dp, dk)
                acc = diff_acc(acc, ax[0], ax[1], xp, dk)
                acc = diff_acc(acc, ax[0], ax[1], xm, dk)
                acc = diff_acc(acc, ay[0], ay[1], yp, dk)
                acc = diff_acc(acc, ay[0], ay[1], ym, dk)
                acc = df_acc(acc, dd[0], dd[1], dk)
                fh, fl = split(f[k, j, i])
                sh, se = two_sum(fh, -acc[0])
                se = f32(se + f32(fl - acc[1]))
                hi, lo = two_sum(sh, se)
                dfv[k, j, i] = np.float64(hi) + np.float64(lo)
    return ex, dfv, dir64


def scale_terms(d, A, Bp, C, idx2, idy2):
    """sum |c d| (direct form) and sum c |d_n - d| (difference form) per point."""
    nz = d.shape[0]
    d64 = d.astype(np.float64)
    dm = np.concatenate([np.zeros_like(d64[:1]), d64[:-1]])
    dp = np.concatenate([d64[1:], np.zeros_like(d64[:1])])
    xs = [np.roll(d64, -1, 2), np.roll(d64, 1, 2)]
    ys = [np.roll(d64, -1, 1), np.roll(d64, 1, 1)]
    a, b, c = A[:, None, None], Bp[:, None, None], C[:, None, None]
    direct = (np.abs(a * dm) + np.abs(b * d64) + np.abs(c * dp) +
              idx2 * sum(np.abs(x) for x in xs) + idy2 * sum(np.abs(y) for y in ys))
    diff = (a * np.abs(dm - d64) + c * np.abs(dp - d64) +
            idx2 * sum(np.abs(x - d64) for x in xs) + idy2 * sum(np.abs(y - d64) for y in ys))
    return direct, diff


def direct_double_float(f, d, A, Bp, C, idx2, idy2):
    """f - L d with the direct stencil in double-float (each c split hi + lo,
    TwoProd / TwoSum), the form the later residual updates use."""
    nz, ny, nx = d.shape
    out = np.zeros_like(f)
    ax, ay = split(idx2), split(idy2)
    for k in range(nz):
        a, b, c = split(A[k]), split(Bp[k]), split(C[k])
        for j in range(ny):
            for i in range(nx):
                dk = d[k, j, i]
                dm = d[k - 1, j, i] if k > 0 else f32(0)
                dp = d[k + 1, j, i] if k + 1 < nz else f32(0)
                acc = df_acc(None, b[0], b[1], dk, init=True)
                for (ch, cl), v in [(ax, d[k, j, (i + 1) % nx]), (ax, d[k, j, i - 1]),
                                    (ay, d[k, (j + 1) % ny, i]), (ay, d[k, j - 1, i]),
                                    (a, dm), (c, dp)]:
                    acc = df_acc(acc, ch, cl, v)
                fh, fl = split(f[k, j, i])
                sh, se = two_sum(fh, -acc[0])
                se = f32(se + f32(fl - acc[1]))
                hi, lo = two_sum(sh, se)
                out[k, j, i] = np.float64(hi) + np.float64(lo)
    return out


@pytest.mark.parametrize("kind", ["smooth", "grid_scale"])
def test_difference_form_first_residual(kind):
    nx, ny, nz, lx, ly = 8, 6, 64, 1.0, 0.75
    dz = synth.tanh_dz(nz, 2.4)  # strongly stretched: large cancellation near the walls
    A, Bp, C, idx2, idy2 = operator(nz, dz, nx, ny, lx, ly)
    rng = np.random.default_rng(7)
    z = np.cumsum(dz) - 0.5 * dz
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    if kind == "smooth":  # the lowest mode in each direction
        d = (np.cos(np.pi * (z + 1) / 2)[:, None, None] * np.cos(2 * np.pi * x)[None, None, :]
             * (1 + 0.5 * np.sin(2 * np.pi * y))[None, :, None])
    else:  # grid-scale oscillation: the worst case for the difference form
        d = rng.standard_normal((nz, ny, nx))
    d = d.astype(np.float32)
    f = rng.standard_normal((nz, ny, nx))
    ex, dfv, dir64 = residuals(f, d, A, Bp, C, idx2, idy2)
    plain = direct_double_float(f, d, A, Bp, C, idx2, idy2)
    direct, diff = scale_terms(d, A, Bp, C, idx2, idy2)
    err_df = np.abs(dfv - ex)
    err_plain = np.abs(plain - ex)
    err_64 = np.abs(dir64 - ex)
    assert np.all(err_df <= 2.0 ** -44 * (diff + np.abs(f)))
    assert np.max(err_df) <= 2.0 ** 5 * max(np.max(err_64), 2.0 ** -52 * np.max(np.abs(f)))
    if kind == "smooth":
        assert np.max(err_df) * 4 < np.max(err_plain)
        assert np.max(err_df) < 1e-11 * np.max(np.abs(f))  # vs the 1e-10 target


def test_residual_update_for_a_small_correction():
    """r_new = r_old - L delta in the direct double-float form (the later
    iterations): for a correction of 1e-6 of the solution's size its error,
    2^-44 of sum |c delta| at most, is far below the FP64 rounding of the
    first residual's terms."""
    nx, ny, nz, lx, ly = 8, 6, 64, 1.0, 0.75
    dz = synth.tanh_dz(nz, 2.4)
    A, Bp, C, idx2, idy2 = operator(nz, dz, nx, ny, lx, ly)
    rng = np.random.default_rng(11)
    delta = (1e-6 * rng.standard_normal((nz, ny, nx))).astype(np.float32)
    r_old = 1e-6 * rng.standard_normal((nz, ny, nx))  # a residual after one FP32 solve
    # r_old carried as the pair (hi, lo); the update subtracts L delta from it
    exact, _, _ = residuals(r_old, delta, A, Bp, C, idx2, idy2)
    upd = direct_double_float(r_old, delta, A, Bp, C, idx2, idy2)
    direct, _ = scale_terms(delta, A, Bp, C, idx2, idy2)
    err = np.abs(upd - exact)
    assert np.all(err <= 2.0 ** -44 * direct + 2.0 ** -46 * np.abs(r_old))
    # against the scale of the solution (|p| ~ 1, |f| ~ 1 here): far below 1e-10
    assert np.max(err) < 1e-14


def test_running_mean_removal_leaves_the_last_corrections_rounding():
    """Each correction pass after the first subtracts the running dz-weighted
    mean of p (rounded to FP32) from its FP32 correction before adding it in
    FP64: the mean left in p is the mean of the last correction plus roundings,
    far below its size.  Emulated with corrections whose own means are those
    an FP32 solve leaves (2^-24 of their size)."""
    rng = np.random.default_rng(3)
    nz, nxy = 48, 512
    dz = synth.tanh_dz(nz, 1.8)
    w = np.repeat(dz, nxy) / (dz.sum() * nxy)  # weights of the dz-weighted mean
    p = np.zeros(nz * nxy)
    sizes = [1.0, 1e-6, 1e-12]
    for it, size in enumerate(sizes):
        delta = size * rng.standard_normal(nz * nxy)
        delta -= w @ delta                      # the solve's own mean removal ...
        delta += size * 2.0 ** -24 * rng.standard_normal()  # ... up to FP32 rounding
        delta = delta.astype(np.float32)
        if it > 0:
            m = np.float32(w @ p)               # running mean, rounded to FP32
            delta = (delta - m).astype(np.float32)
        p = p + delta.astype(np.float64)
        if it == 0:
            first_mean = abs(w @ p)
    assert first_mean > 1e-9                    # the first solve's mean is visible ...
    assert abs(w @ p) < 1e-15 * np.max(np.abs(p))  # ... and gone after the next passes
