"""CPU: the library's Algorithm 2 pre-processing (csrc/chanfs_alg2.cuh, used on
the host by plan.cu and on the GPU by noalloc.cu), compiled with g++ as plain
C++, against numpy.

The factors it stores are applied by a numpy restatement of the run-time
Steps 2-4 (what pcr_kernel does per column), and the result must solve the
tridiagonal system: against numpy.linalg.solve on random diagonally dominant
systems and on the rows of I - c L_z of stretched grids, for even, uneven and
minimal (3-row) partitions.  The z-operator rows are checked against the
flux-form definition on unit vectors.
"""

import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2502_06296_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2502_06296_gb300", "csrc")

HARNESS = r"""
#define __host__
#define __device__
#include "chanfs_alg2.cuh"
using namespace chanfs;
extern "C" {
int factor(int n, int np, const double* A, const double* B, const double* C, double* rows,
           double* red) {
  double ra[128], rb[128], rc[128];
  for (int q = 0; q < np; ++q) {
    const int o = alg2_part_start(q, n, np), m = alg2_part_start(q + 1, n, np) - o;
    if (m < 3) return -1;
    auto row = [&](int i, double* lo, double* d, double* hi) {
      *lo = A[o + i]; *d = B[o + i]; *hi = C[o + i];
    };
    double f[3], l[3];
    alg2_factor_partition(m, row, rows + o, rows + n + o, rows + 2 * n + o, rows + 3 * n + o,
                          rows + 4 * n + o, f, l);
    ra[2 * q] = f[0]; rb[2 * q] = f[1]; rc[2 * q] = f[2];
    ra[2 * q + 1] = l[0]; rb[2 * q + 1] = l[1]; rc[2 * q + 1] = l[2];
  }
  alg2_reduced_factor(2 * np, ra, rb, rc, red, red + 2 * np, red + 4 * np);
  return 0;
}
void zrow(int k, int nz, const double* dzf, int bc, int loc, double* out) {
  z_operator_row(k, nz, dzf, bc, loc, out, out + 1, out + 2);
}
void hrow(int k, int nz, const double* dzf, int loc, double c, double* out) {
  helm_row(k, nz, dzf, loc, c, out, out + 1, out + 2);
}
int unknowns(int nz, int loc) { return helm_unknowns(nz, loc); }
int auto_parts(int n, int maxp) { return alg2_auto_parts(n, maxp); }
}
"""


@pytest.fixture(scope="module")
def h(tmp_path_factory):
    d = tmp_path_factory.mktemp("alg2")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libalg2.so"
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, "-o", str(so),
                    str(src)], check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.factor.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
    lib.zrow.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp]
    lib.hrow.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def factor(h, A, B, C, np_):
    n = len(B)
    rows = np.zeros(5 * n)
    red = np.zeros(6 * np_)
    A, B, C = (np.ascontiguousarray(x, dtype=np.float64) for x in (A, B, C))
    assert h.factor(n, np_, _p(A), _p(B), _p(C), _p(rows), _p(red)) == 0
    return rows, red


def runtime(rows, red, d, np_):
    """Steps 2-4 with the stored factors, as the run-time kernel applies them."""
    n = len(d)
    alpha, beta, ib, ap, cp = rows.reshape(5, n)
    J = 2 * np_
    rl, rip, ripc = red.reshape(3, J)
    d = d.astype(np.float64).copy()
    ends = []
    for q in range(np_):
        s, e = q * n // np_, (q + 1) * n // np_
        m = e - s
        for i in range(2, m):
            d[s + i] -= alpha[s + i] * d[s + i - 1]
        for i in range(m - 3, -1, -1):
            d[s + i] -= beta[s + i] * d[s + i + 1]
        ends += [d[s], d[s + m - 1]]
    y = np.array(ends)
    for j in range(1, J):
        y[j] -= rl[j] * y[j - 1]
    x = np.empty(J)
    x[J - 1] = rip[J - 1] * y[J - 1]
    for j in range(J - 2, -1, -1):
        x[j] = rip[j] * y[j] - ripc[j] * x[j + 1]
    out = np.empty(n)
    for q in range(np_):
        s, e = q * n // np_, (q + 1) * n // np_
        m = e - s
        x0, xm = x[2 * q], x[2 * q + 1]
        out[s], out[e - 1] = x0, xm
        for i in range(1, m - 1):
            out[s + i] = ib[s + i] * d[s + i] - ap[s + i] * x0 - cp[s + i] * xm
    return out


def dense(A, B, C):
    n = len(B)
    M = np.diag(B)
    M[np.arange(1, n), np.arange(n - 1)] = A[1:]
    M[np.arange(n - 1), np.arange(1, n)] = C[:-1]
    return M


@pytest.mark.parametrize("n,np_", [(3, 1), (7, 2), (12, 4), (40, 3), (97, 8), (256, 16),
                                   (1024, 64), (65, 21)])
def test_factors_solve_random_dominant_systems(h, n, np_):
    rng = np.random.default_rng(n * 100 + np_)
    A = rng.uniform(-1, 1, n)
    C = rng.uniform(-1, 1, n)
    A[0] = C[-1] = 0.0
    B = (np.abs(A) + np.abs(C) + rng.uniform(0.1, 1.0, n)) * rng.choice([-1, 1], n)
    d = rng.normal(size=n)
    rows, red = factor(h, A, B, C, np_)
    x = runtime(rows, red, d, np_)
    ref = np.linalg.solve(dense(A, B, C), d)
    assert np.max(np.abs(x - ref)) / np.max(np.abs(ref)) < 1e-13


@pytest.mark.parametrize("nz,beta,loc,c,np_", [(384, 1.8, 0, 9.615e-9, 12), (384, 1.8, 1, 9.615e-9, 16),
                                               (64, 2.2, 0, 1e-4, 4), (31, 1.2, 1, 1e-3, 10),
                                               (1024, 1.8, 0, 1e-5, 32)])
def test_factors_solve_the_helmholtz_rows(h, nz, beta, loc, c, np_):
    dz = synth.tanh_dz(nz, beta)
    n = h.unknowns(nz, loc)
    rows3 = np.zeros((n, 3))
    for k in range(n):
        out = np.zeros(3)
        h.hrow(k, nz, _p(dz), loc, c, _p(out))
        rows3[k] = out
    A, B, C = rows3.T
    assert A[0] == 0.0 and C[-1] == 0.0
    d = np.random.default_rng(nz).normal(size=n)
    rows, red = factor(h, A, B, C, np_)
    x = runtime(rows, red, d, np_)
    ref = np.linalg.solve(dense(A, B, C), d)
    assert np.max(np.abs(x - ref)) / np.max(np.abs(ref)) < 1e-13


@pytest.mark.parametrize("bc,loc", [(0, 0), (1, 0), (1, 1)])
def test_z_operator_rows_match_the_flux_form(h, bc, loc):
    """Row k applied to unit vectors equals the staggered flux-form operator
    with the wall ghosts (mirror for cell centres, zero on the walls for
    faces) evaluated directly."""
    nz = 9
    dzf = synth.tanh_dz(nz, 1.7)
    zf = np.concatenate([[0.0], np.cumsum(dzf)])
    zc = 0.5 * (zf[1:] + zf[:-1])
    n = nz if loc == 0 else nz - 1
    for j in range(n):
        q = np.zeros(n)
        q[j] = 1.0
        if loc == 0:  # cell centres, ghosts one cell width beyond each wall
            sgn = 1.0 if bc == 0 else -1.0
            qq = np.concatenate([[sgn * q[0]], q, [sgn * q[-1]]])
            zz = np.concatenate([[zc[0] - dzf[0]], zc, [zc[-1] + dzf[-1]]])
            flux = np.diff(qq) / np.diff(zz)
            Lq = np.diff(flux) / dzf
        else:  # interior faces, zero on both walls
            qq = np.concatenate([[0.0], q, [0.0]])
            flux = np.diff(qq) / dzf
            Lq = np.diff(flux) / np.diff(zc)
        for k in range(n):
            out = np.zeros(3)
            h.zrow(k, nz, _p(dzf), bc, loc, _p(out))
            lo, dg, hi = out
            got = dg * q[k] + (lo * q[k - 1] if k > 0 else 0.0) + (hi * q[k + 1] if k < n - 1 else 0.0)
            assert abs(got - Lq[k]) <= 1e-9 * max(1.0, abs(Lq[k])), (bc, loc, j, k)


def test_auto_partitions(h):
    for n in (3, 5, 31, 32, 33, 383, 384, 1024):
        p = h.auto_parts(n, 64)
        assert 1 <= p <= 64
        assert all((q + 1) * n // p - q * n // p >= 3 for q in range(p))
        assert p == max(1, min(64, (n + 31) // 32)) or n // ((n + 31) // 32) < 3


# ---------------------------------------------------------------------------
# The partitioned z solve of FP32 spectra (thomas.cu, zpart_kernel), restated
# in numpy: 8-row partitions with identity rows past the last row, the
# normalised downward elimination with x_0 a parameter, the upward
# elimination into row 0, cyclic reduction of the 2P-row reduced system, and
# back substitution in the downward form.  The restatement must solve the
# system (against numpy.linalg.solve): this checks the derivation the kernel
# implements; the kernel itself is checked against the oracle on the GPU.
# ---------------------------------------------------------------------------

def _zpart_solve(A, D, C, d, mm=8):
    n = D.size
    P = (n + mm - 1) // mm
    N = P * mm
    A_, D_, C_ = np.zeros(N), np.ones(N), np.zeros(N)
    A_[:n], D_[:n], C_[:n] = A, D, C
    A_[0] = 0.0
    C_[n - 1] = 0.0
    rhs = np.zeros(N, dtype=d.dtype)
    rhs[:n] = d
    red = np.zeros((2 * P, 3))
    ry = np.zeros(2 * P, dtype=d.dtype)
    keep = []
    for q in range(P):
        o = q * mm
        a, b, c, u = A_[o:o + mm], D_[o:o + mm], C_[o:o + mm], rhs[o:o + mm].copy()
        cq, gq = np.zeros(mm), np.zeros(mm)
        ib = 1.0 / b[1]
        cq[1], gq[1], u[1] = c[1] * ib, a[1] * ib, u[1] * ib
        for i in range(2, mm):
            ib = 1.0 / (b[i] - a[i] * cq[i - 1])
            cq[i] = c[i] * ib
            gq[i] = -a[i] * ib * gq[i - 1]
            u[i] = (u[i] - a[i] * u[i - 1]) * ib
        uu, vv, ww = u[mm - 2], gq[mm - 2], cq[mm - 2]
        for i in range(mm - 3, 0, -1):
            uu, vv, ww = u[i] - cq[i] * uu, gq[i] - cq[i] * vv, -cq[i] * ww
        red[2 * q] = (a[0], b[0] - c[0] * vv, -c[0] * ww)
        ry[2 * q] = u[0] - c[0] * uu
        red[2 * q + 1] = (gq[mm - 1], 1.0, cq[mm - 1])
        ry[2 * q + 1] = u[mm - 1]
        keep.append((cq, gq, u))
    # cyclic reduction: at stride s the rows k = -1 mod 2s take away k -+ s
    J = 2 * P
    s = 1
    while 2 * s <= J:
        for k in range(2 * s - 1, J, 2 * s):
            sub, dia, sup = red[k]
            y = ry[k]
            lo = red[k - s]
            e1 = sub / lo[1]
            dia -= e1 * lo[2]
            y -= e1 * ry[k - s]
            sub = -e1 * lo[0]
            new_sup = 0.0
            if k + s < J:
                hi = red[k + s]
                e2 = sup / hi[1]
                dia -= e2 * hi[0]
                y -= e2 * ry[k + s]
                new_sup = -e2 * hi[2]
            red[k] = (sub, dia, new_sup)
            ry[k] = y
        s *= 2
    x = np.zeros(J, dtype=d.dtype)
    top = s - 1
    x[top] = ry[top] / red[top][1]
    h = s // 2
    while h >= 1:
        for k in range(h - 1, J, 2 * h):
            if k == top:
                continue
            y = ry[k]
            if k - h >= 0:
                y = y - red[k][0] * x[k - h]
            if k + h < J:
                y = y - red[k][2] * x[k + h]
            x[k] = y / red[k][1]
        h //= 2
    out = np.zeros(N, dtype=d.dtype)
    for q in range(P):
        cq, gq, u = keep[q]
        o = q * mm
        xs = np.zeros(mm, dtype=d.dtype)
        xs[0], xs[mm - 1] = x[2 * q], x[2 * q + 1]
        for i in range(mm - 2, 0, -1):
            xs[i] = u[i] - cq[i] * xs[i + 1] - gq[i] * xs[0]
        out[o:o + mm] = xs
    return out[:n]


@pytest.mark.parametrize("n", [3, 5, 8, 9, 17, 40, 97, 128, 300, 512])
@pytest.mark.parametrize("lam", [-1e-3, -5.0])
def test_partitioned_z_solve_algebra(n, lam):
    """Eq. 12 rows (the z operator of a stretched grid shifted by an
    eigenvalue), complex right-hand side, against a dense solve."""
    dz = synth.tanh_dz(n, 1.8)
    zf = np.concatenate(([0.0], np.cumsum(dz)))
    zc = 0.5 * (zf[:-1] + zf[1:])
    h = np.diff(zc)
    A, C = np.zeros(n), np.zeros(n)
    A[1:] = 1.0 / (dz[1:] * h)
    C[:-1] = 1.0 / (dz[:-1] * h)
    B = -(A + C)  # Neumann walls: the wall couplings fold into the diagonal
    D = B + lam
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    T = np.diag(D) + np.diag(A[1:], -1) + np.diag(C[:-1], 1)
    ref = np.linalg.solve(T, d)
    got = _zpart_solve(A, D, C, d)
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
