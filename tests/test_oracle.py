"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: the
O(n^2) DFT definition, a library routine (numpy.fft, numpy.linalg), closed-form
eigenpairs of the second-difference operators, conservation and symmetry
invariants of the staggered stencil, second-order convergence to calculus,
dense-LU brute force on tiny 3-D grids, and the residual of the discrete
equations.  They are chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""

import numpy as np
import pytest

import oracle
from paper_2502_06296_gb300 import synth

RNG = np.random.default_rng(12345)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------------------------------
# Fourier transforms (Sec. 2.2.1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 18, 24, 27, 32, 48, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_dft_definition(n, sign):
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    # naive DFT written from the definition in the test as well
    k = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    ref = W @ x
    assert _rel(oracle.dft_naive(x, sign), ref) < 1e-13
    assert _rel(oracle.fft(x, sign), ref) < 1e-13


@pytest.mark.parametrize("n", [96, 128, 192, 256, 384, 512, 768, 1024])
def test_fft_matches_numpy(n):
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    assert _rel(oracle.fft(x, -1), np.fft.fft(x)) < 1e-13
    assert _rel(oracle.fft(x, 1), np.fft.ifft(x) * n) < 1e-13


def test_fft_impulse_constant_and_parseval():
    n = 384
    e = np.zeros(n, complex)
    e[0] = 1.0
    assert np.max(np.abs(oracle.fft(e) - 1.0)) < 1e-15
    x = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    X = oracle.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    # inverse with 1/n is the identity
    assert _rel(oracle.fft(X, 1) / n, x) < 1e-14


# ----------------------------------------------------------------------------
# Appendix A packed format
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 9, 16, 27, 32, 96, 384, 512])
def test_packed_layout_and_roundtrip(n):
    x = RNG.standard_normal(n)
    p = oracle.rfft_packed(x)
    R = np.fft.rfft(x)  # floor(n/2)+1 coefficients
    last = n // 2
    assert abs(p[0] - R[0].real) < 1e-12 * n
    if n % 2 == 0:
        assert abs(p[1] - R[last].real) < 1e-12 * n
    else:
        assert abs(p[1] - R[last].imag) < 1e-12 * n
        assert abs(p[n - 1] - R[last].real) < 1e-12 * n
    for k in range(1, (n - 1) // 2 + (1 if n % 2 == 0 else 0)):
        if 2 * k + 1 < n and k < last:
            assert abs(p[2 * k] - R[k].real) < 1e-12 * n
            assert abs(p[2 * k + 1] - R[k].imag) < 1e-12 * n
    assert _rel(oracle.irfft_packed(p), x) < 1e-13
    # n reals in, n reals out, no information lost (App. A)
    assert p.size == n


@pytest.mark.parametrize("n", [6, 7, 8, 9, 12])
def test_packed_wavenumbers_cover_each_mode_once(n):
    slots = [oracle.packed_wavenumber(n, s) for s in range(n)]
    # every wavenumber 0..n//2 appears, interior ones twice (re, im)
    for k in range(n // 2 + 1):
        expect = 1 if (k == 0 or (n % 2 == 0 and k == n // 2)) else 2
        assert slots.count(k) == expect


@pytest.mark.parametrize("n", [8, 9, 12])
def test_packed_eigenvalue_follows_single_mode(n):
    """A single cosine of wavenumber k lands in the slots whose packed
    eigenvalue is the eigenvalue of k."""
    h = 0.3
    lam_nat = oracle.eig_periodic(n, h)
    lam_p = oracle.eig_packed(n, h)
    j = np.arange(n)
    for k in range(n // 2 + 1):
        p = oracle.rfft_packed(np.cos(2 * np.pi * k * j / n) + 0.5 * np.sin(2 * np.pi * k * j / n))
        hot = np.abs(p) > 1e-9
        assert hot.any()
        assert np.allclose(lam_p[hot], lam_nat[k], rtol=1e-14, atol=1e-12)


# ----------------------------------------------------------------------------
# Modified wavenumbers (Eq. 12)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n,h", [(8, 0.5), (32, 2 * np.pi / 32), (384, 6.4 / 384)])
def test_eigenvalues_are_those_of_the_periodic_second_difference(n, h):
    lam = oracle.eig_periodic(n, h)
    j = np.arange(n)
    for k in [0, 1, n // 3, n // 2, n - 1]:
        v = np.exp(2j * np.pi * ((k * j) % n) / n)  # exact angle reduction
        lv = (np.roll(v, -1) - 2 * v + np.roll(v, 1)) / h**2
        assert np.max(np.abs(lv - lam[k] * v)) < 1e-9 * max(1.0, abs(lam[k]))
    assert np.all(lam <= 0) and lam[0] == 0.0


# ----------------------------------------------------------------------------
# z stencil (Sec. 2.1 staggered grid; eta of Eq. 12)
# ----------------------------------------------------------------------------

def _dense_lz(A, B, C):
    n = len(B)
    T = np.diag(B)
    T += np.diag(A[1:], -1) + np.diag(C[:-1], 1)
    return T


@pytest.mark.parametrize("N", [8, 17, 32])
def test_lz_uniform_closed_form_eigenpairs(N):
    dz = 2.0 / N
    dzf = np.full(N, dz)
    zc = (np.arange(N) + 0.5) * dz  # centres measured from the bottom wall
    zf = (np.arange(N - 1) + 1) * dz  # interior faces
    # Neumann centred: cos modes, l = 0..N-1
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.NEUMANN, oracle.CENTER))
    for l in range(N):
        v = np.cos(np.pi * l * zc / 2.0)
        mu = 2 * (np.cos(np.pi * l / N) - 1) / dz**2
        assert np.max(np.abs(T @ v - mu * v)) < 1e-9 / dz**2
    # Dirichlet centred: sin modes, l = 1..N
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.DIRICHLET, oracle.CENTER))
    for l in range(1, N + 1):
        v = np.sin(np.pi * l * zc / 2.0)
        mu = 2 * (np.cos(np.pi * l / N) - 1) / dz**2
        assert np.max(np.abs(T @ v - mu * v)) < 1e-9 / dz**2
    # Dirichlet face: sin modes on the N-1 interior faces, l = 1..N-1
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.DIRICHLET, oracle.FACE))
    assert T.shape == (N - 1, N - 1)
    for l in range(1, N):
        v = np.sin(np.pi * l * zf / 2.0)
        mu = 2 * (np.cos(np.pi * l / N) - 1) / dz**2
        assert np.max(np.abs(T @ v - mu * v)) < 1e-9 / dz**2


def test_lz_stretched_invariants():
    N = 24
    dzf = synth.tanh_dz(N, 1.8)
    dzc = oracle.dzc(dzf)
    assert np.allclose(dzc, 0.5 * (dzf[:-1] + dzf[1:]))
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.NEUMANN, oracle.CENTER))
    # conservation: volume-weighted column sums vanish (flux form, no wall flux)
    assert np.max(np.abs(dzf @ T)) < 1e-9 * np.max(np.abs(T))
    # constants are in the null space
    assert np.max(np.abs(T @ np.ones(N))) < 1e-9 * np.max(np.abs(T))
    # symmetric in the volume-weighted inner product
    for bc in (oracle.NEUMANN, oracle.DIRICHLET):
        T = _dense_lz(*oracle.lz_coefficients(dzf, bc, oracle.CENTER))
        S = np.diag(dzf) @ T
        assert np.max(np.abs(S - S.T)) < 1e-10 * np.max(np.abs(S))
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.DIRICHLET, oracle.FACE))
    S = np.diag(dzc) @ T
    assert np.max(np.abs(S - S.T)) < 1e-10 * np.max(np.abs(S))
    # Dirichlet operators are negative definite
    T = _dense_lz(*oracle.lz_coefficients(dzf, oracle.DIRICHLET, oracle.CENTER))
    assert np.all(np.linalg.eigvals(np.diag(dzf) @ T).real < 0)


@pytest.mark.parametrize("bc,loc", [(0, 0), (1, 0), (1, 1)])
def test_lz_converges_to_calculus_on_stretched_grid(bc, loc):
    """Against calculus, not a retyped formula: on a smoothly stretched grid the
    stencil's truncation error is first order pointwise, and the solution of
    (L_z - 1) u = u'' - u converges to the exact u at second order
    (supraconvergence of the staggered scheme); on a uniform grid the truncation
    error is second order as well."""
    def case(faces):
        dzf = np.diff(faces)
        zc = 0.5 * (faces[:-1] + faces[1:])
        z = zc if loc == 0 else faces[1:-1]
        if bc == 0:
            u, d2 = np.cos(np.pi * (z + 1)), -np.pi**2 * np.cos(np.pi * (z + 1))
        else:
            u, d2 = np.sin(np.pi * (z + 1) / 2), -(np.pi / 2) ** 2 * np.sin(np.pi * (z + 1) / 2)
        T = _dense_lz(*oracle.lz_coefficients(dzf, bc, loc))
        trunc = np.max(np.abs(T @ u - d2))
        sol = np.linalg.solve(T - np.eye(len(u)), d2 - u)
        return trunc, np.max(np.abs(sol - u))

    Ns = (32, 64, 128, 256)
    st = np.array([case(synth.tanh_faces(N, 1.4)) for N in Ns])
    un = np.array([case(np.linspace(-1, 1, N + 1)) for N in Ns])
    rate = lambda e: np.log2(e[:-1] / e[1:])
    assert rate(st[:, 0]).min() > 0.9, st
    assert rate(st[:, 1]).min() > 1.8, st
    assert rate(un[:, 0]).min() > 1.9, un
    assert rate(un[:, 1]).min() > 1.9, un


def test_apply_operators_agree_with_stencil_coefficients():
    """or_apply_* (flux form) and or_lz_coefficients are separate code paths;
    on unit vectors they must give the same matrix."""
    nx, ny, nz = 1, 1, 9
    dzf = synth.tanh_dz(nz, 1.3)
    for bc in (0, 1):
        A, B, C = oracle.lz_coefficients(dzf, bc, 0)
        T = _dense_lz(A, B, C)
        M = np.zeros((nz, nz))
        for k in range(nz):
            e = np.zeros((nz, ny, nx))
            e[k] = 1.0
            M[:, k] = oracle.apply_poisson(e, 1.0, 1.0, dzf, bc).ravel()
        assert np.max(np.abs(M - T)) < 1e-9 * np.max(np.abs(T))
    for loc in (0, 1):
        A, B, C = oracle.lz_coefficients(dzf, 1, loc)
        n = len(B)
        T = np.eye(n) - 0.01 * _dense_lz(A, B, C)
        M = np.zeros((n, n))
        for k in range(n):
            e = np.zeros((nz, ny, nx))
            e[k] = 1.0
            M[:, k] = oracle.apply_helmholtz(e, dzf, 0.01, loc).ravel()[:n]
        assert np.max(np.abs(M - T)) < 1e-12 * np.max(np.abs(T))


# ----------------------------------------------------------------------------
# Tridiagonal solvers: Thomas, Algorithm 1, Algorithm 2 (Sec. 2.2.4)
# ----------------------------------------------------------------------------

def _random_dd_system(n, rng):
    a = rng.uniform(-1, 1, n)
    c = rng.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.5, 2.0, n)
    b *= rng.choice([-1, 1], n)
    a[0] = 0.0
    c[-1] = 0.0
    d = rng.standard_normal(n)
    return a, b, c, d


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 383])
def test_thomas_matches_dense_solvers(n):
    rng = np.random.default_rng(n)
    a, b, c, d = _random_dd_system(n, rng)
    T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x = oracle.thomas(a, b, c, d)
    assert _rel(x, np.linalg.solve(T, d)) < 1e-12
    assert _rel(x, oracle.dense_solve(T, d)) < 1e-12


@pytest.mark.parametrize("n,p", [(3, 1), (9, 3), (10, 3), (64, 4), (383, 16), (384, 32), (384, 128), (100, 7)])
def test_alg1_and_alg2_match_thomas(n, p):
    rng = np.random.default_rng(1000 + n + p)
    a, b, c, d = _random_dd_system(n, rng)
    x = oracle.thomas(a, b, c, d)
    assert _rel(oracle.alg2_solve(a, b, c, d, p), x) < 1e-12
    assert _rel(oracle.alg1_solve(a, b, c, d, p), x) < 1e-12


def test_alg2_rejects_partitions_below_three_rows():
    a, b, c, d = _random_dd_system(10, np.random.default_rng(0))
    with pytest.raises(ValueError):
        oracle.alg2_solve(a, b, c, d, 4)  # m = 2 or 3 rows


@pytest.mark.parametrize("m", [3, 4, 5, 12, 24])
def test_alg2_reduced_rows_hold_for_the_true_solution(m):
    """After Step 2 every row is expressed through the partition's boundary
    values only (Eq. 14): a_i x_0 + b_i x_i + c_i x_{m-1} = d_i for interior i,
    and rows 0 / m-1 couple to the neighbouring partitions' boundaries."""
    rng = np.random.default_rng(m)
    n = m + 2  # one extra unknown either side of the partition
    a, b, c, _ = _random_dd_system(n, rng)
    xs = rng.standard_normal(n)
    T = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    d = T @ xs
    A, B, C, D = a[1:-1], b[1:-1], c[1:-1], d[1:-1]
    xp, x, xn = xs[0], xs[1:-1], xs[-1]
    aa, bb, cc = oracle.alg2_prepare(A, B, C)
    dd = oracle.alg2_runtime(A, C, bb, D)
    scale = np.max(np.abs(d))
    for i in range(1, m - 1):
        assert abs(aa[i] * x[0] + bb[i] * x[i] + cc[i] * x[m - 1] - dd[i]) < 1e-12 * scale
    assert abs(aa[0] * xp + bb[0] * x[0] + cc[0] * x[m - 1] - dd[0]) < 1e-12 * scale
    assert abs(aa[m - 1] * x[0] + bb[m - 1] * x[m - 1] + cc[m - 1] * xn - dd[m - 1]) < 1e-12 * scale
    rec = oracle.alg2_reconstruct(aa, bb, cc, dd, x[0], x[m - 1])
    assert _rel(rec, x) < 1e-12


# ----------------------------------------------------------------------------
# 3-D Poisson (Eq. 12 route) and Helmholtz (Eq. 11)
# ----------------------------------------------------------------------------

def _dense_poisson(nx, ny, nz, lx, ly, dzf, bc):
    n = nx * ny * nz
    L = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        L[:, i] = oracle.apply_poisson(e.reshape(nz, ny, nx), lx, ly, dzf, bc).ravel()
    return L


@pytest.mark.parametrize("dims,beta,bc", [((4, 4, 4), None, 0), ((6, 4, 5), 1.5, 0),
                                          ((4, 6, 5), 1.5, 1), ((8, 8, 8), 1.8, 0),
                                          ((8, 8, 8), None, 1), ((2, 3, 4), 1.2, 0)])
def test_poisson_matches_dense_lu_bruteforce(dims, beta, bc):
    nx, ny, nz = dims
    lx, ly = 2 * np.pi, np.pi
    dzf = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    f = rng.standard_normal((nz, ny, nx))
    p = oracle.poisson_solve(f, lx, ly, dzf, bc)
    L = _dense_poisson(nx, ny, nz, lx, ly, dzf, bc)
    n = nx * ny * nz
    w = np.repeat(dzf, nx * ny)
    if bc == 0:
        # bordered system [L 1; w^T 0][p; mu] = [f; 0]: L p = f - mu,  w.p = 0
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = L
        K[:n, n] = 1.0
        K[n, :n] = w
        sol = oracle.dense_solve(K, np.concatenate([f.ravel(), [0.0]]))
        ref = sol[:n]
        assert abs(w @ p.ravel()) < 1e-12 * np.sum(w) * np.max(np.abs(p))
    else:
        ref = oracle.dense_solve(L, f.ravel())
    assert _rel(p.ravel(), ref) < 1e-11
    assert _rel(p.ravel(), np.linalg.lstsq(K if bc == 0 else L,
                                           np.concatenate([f.ravel(), [0.0]]) if bc == 0 else f.ravel(),
                                           rcond=None)[0][:n]) < 1e-10


@pytest.mark.parametrize("bc", [0, 1])
def test_poisson_single_mode_closed_form_uniform(bc):
    nx, ny, nz = 16, 12, 10
    lx, ly, lz = 2 * np.pi, np.pi, 2.0
    dx, dy, dz = lx / nx, ly / ny, lz / nz
    xc = np.arange(nx) * dx  # periodic directions: only the index matters
    yc = np.arange(ny) * dy
    zc = (np.arange(nz) + 0.5) * dz
    for (m, q, l) in [(1, 1, 1), (3, 2, 4), (8, 6, 2), (0, 5, 3), (2, 0, 0 if bc == 0 else 1)]:
        zmode = np.cos(np.pi * l * zc / lz) if bc == 0 else np.sin(np.pi * l * zc / lz)
        f = (np.cos(2 * np.pi * m * xc / lx)[None, None, :]
             * np.cos(2 * np.pi * q * yc / ly)[None, :, None]
             * zmode[:, None, None])
        lam = (2 * (np.cos(2 * np.pi * m / nx) - 1) / dx**2 + 2 * (np.cos(2 * np.pi * q / ny) - 1) / dy**2
               + 2 * (np.cos(np.pi * l / nz) - 1) / dz**2)
        p = oracle.poisson_solve(f, lx, ly, synth.uniform_dz(nz, lz), bc)
        assert _rel(p, f / lam) < 1e-12


def test_poisson_single_xy_mode_on_stretched_grid():
    """A single x-y Fourier mode times g(z) gives the same mode times h(z), with
    h the solution of the 1-D system (lx + ly + L_z) h = g (numpy.linalg)."""
    nx, ny, nz = 12, 8, 24
    lx, ly = 12.8, 6.4
    dzf = synth.tanh_dz(nz, 1.8)
    g = np.random.default_rng(5).standard_normal(nz)
    m, q = 2, 3
    xc = (np.arange(nx) + 0.5) * lx / nx
    yc = (np.arange(ny) + 0.5) * ly / ny
    mode = np.cos(2 * np.pi * m * xc / lx)[None, :] * np.sin(2 * np.pi * q * yc / ly)[:, None]
    f = g[:, None, None] * mode[None]
    shift = 2 * (np.cos(2 * np.pi * m / nx) - 1) / (lx / nx) ** 2 + 2 * (np.cos(2 * np.pi * q / ny) - 1) / (ly / ny) ** 2
    A, B, C = oracle.lz_coefficients(dzf, 0, 0)
    h = np.linalg.solve(_dense_lz(A, B, C) + shift * np.eye(nz), g)
    p = oracle.poisson_solve(f, lx, ly, dzf, 0)
    assert _rel(p, h[:, None, None] * mode[None]) < 1e-12


def test_poisson_small_config_residual_and_invariants():
    cfg = synth.SMALL
    f = synth.small_rhs(cfg)
    dzf = synth.grid_dz(cfg)
    p = oracle.poisson_solve(f, cfg["lx"], cfg["ly"], dzf, 0)
    r = f - oracle.apply_poisson(p, cfg["lx"], cfg["ly"], dzf, 0)
    assert np.max(np.abs(r)) / np.max(np.abs(f)) < 1e-12
    assert abs(np.mean(p)) < 1e-14 * np.max(np.abs(p))
    # cyclic shift in x and y commutes with the solve
    ps = oracle.poisson_solve(np.roll(f, (3, 5), axis=(1, 2)), cfg["lx"], cfg["ly"], dzf, 0)
    assert _rel(ps, np.roll(p, (3, 5), axis=(1, 2))) < 1e-12
    # linearity
    g = synth.uniform(7, f.shape)
    g -= g.mean()
    pg = oracle.poisson_solve(g, cfg["lx"], cfg["ly"], dzf, 0)
    pfg = oracle.poisson_solve(2.0 * f - 3.0 * g, cfg["lx"], cfg["ly"], dzf, 0)
    assert _rel(pfg, 2.0 * p - 3.0 * pg) < 1e-12


def test_poisson_neumann_projects_incompatible_rhs():
    """A constant added to f is removed by the projection: same solution."""
    nx, ny, nz = 8, 6, 12
    dzf = synth.tanh_dz(nz, 1.6)
    f = np.random.default_rng(3).standard_normal((nz, ny, nx))
    p1 = oracle.poisson_solve(f, 1.0, 2.0, dzf, 0)
    p2 = oracle.poisson_solve(f + 5.0, 1.0, 2.0, dzf, 0)
    # removing a mean of 5 from O(1) data costs ~3 bits of f, and |p| ~ 0.02 |f|
    assert _rel(p1, p2) < 1e-10
    w = np.repeat(dzf, nx * ny)
    assert abs(w @ p1.ravel()) < 1e-13 * np.max(np.abs(p1)) * w.sum()


@pytest.mark.parametrize("loc", [0, 1])
def test_helmholtz_closed_form_uniform(loc):
    nx, ny, nz = 3, 2, 16
    dz = 2.0 / nz
    c = 1e-3
    zc = (np.arange(nz) + 0.5) * dz
    zf = (np.arange(nz) + 1) * dz
    for l in [1, 2, 7, nz - 1]:
        z = zc if loc == 0 else zf
        col = np.sin(np.pi * l * z / 2.0)
        if loc == 1:
            col[-1] = 0.0  # wall slot
        rhs = np.broadcast_to(col[:, None, None], (nz, ny, nx)).copy()
        mu = 2 * (np.cos(np.pi * l / nz) - 1) / dz**2
        for method, parts in [(0, 1), (1, 3), (2, 3), (1, 5)]:
            u = oracle.helmholtz_solve(rhs, synth.uniform_dz(nz), c, loc, method, parts)
            assert _rel(u, rhs / (1 - c * mu)) < 1e-13


@pytest.mark.parametrize("loc", [0, 1])
def test_helmholtz_stretched_methods_agree_and_residual(loc):
    nx, ny, nz = 5, 4, 48
    dzf = synth.tanh_dz(nz, 1.8)
    rhs = synth.normal(11, (nz, ny, nx))
    c = 9.615e-5
    u = oracle.helmholtz_solve(rhs, dzf, c, loc, oracle.THOMAS)
    for method, parts in [(oracle.ALG2, 4), (oracle.ALG2, 15), (oracle.ALG1, 8), (oracle.ALG2, 1)]:
        v = oracle.helmholtz_solve(rhs, dzf, c, loc, method, parts)
        assert _rel(v, u) < 1e-13
    r = oracle.apply_helmholtz(u, dzf, c, loc) - rhs
    if loc == 1:
        r[-1] = 0.0
        assert np.all(u[-1] == 0.0)
    assert np.max(np.abs(r)) / np.max(np.abs(rhs)) < 1e-13
    # c = 0 is the identity
    u0 = oracle.helmholtz_solve(rhs, dzf, 0.0, loc, oracle.ALG2, 4)
    ref = rhs.copy()
    if loc == 1:
        ref[-1] = 0.0
    assert np.array_equal(u0, ref)


# ----------------------------------------------------------------------------
# Spectral layout (App. A along x, complex along y)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(8, 6, 3), (16, 9, 2), (12, 12, 4), (4, 1, 2), (6, 2, 3)])
def test_spectral_layout_against_numpy_fft2(dims):
    nx, ny, nz = dims
    f = np.random.default_rng(nx + ny).standard_normal((nz, ny, nx))
    S = oracle.spectral_forward(f)
    F = np.fft.fft2(f, axes=(1, 2))  # (z, ky, kx)
    M = nx // 2
    assert _rel(S[:, :, 1:], F[:, :, 1:M]) < 1e-12
    for ky in range(ny):
        if ky == 0 or 2 * ky == ny:   # two real columns packed together
            ref = F[:, ky, 0] + 1j * F[:, ky, M]
        elif 2 * ky < ny:              # F(0, ky)
            ref = F[:, ky, 0]
        else:                          # F(Nx/2, Ny - ky)
            ref = F[:, ny - ky, M]
        assert _rel(S[:, ky, 0], ref) < 1e-12
    assert _rel(oracle.spectral_inverse(S), f) < 1e-13


def test_oracle_reproduces_its_stored_fixture():
    """tests/golden/poisson_small_oracle.json was written by
    tests/golden/make_golden.py (oracle only): the oracle still gives it."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "poisson_small_oracle.json")
    g = json.load(open(path))
    cfg = synth.SMALL
    p = oracle.poisson_solve(synth.small_rhs(cfg), cfg["lx"], cfg["ly"], synth.grid_dz(cfg), 0)
    scale = g["max_abs_p"]
    for s in g["samples"]:
        assert abs(p[tuple(s["zyx"])] - s["p"]) < 1e-13 * scale
    assert abs(np.max(np.abs(p)) - scale) < 1e-13 * scale


# ----------------------------------------------------------------------------
# Fully implicit 3-D Helmholtz (Eq. 8): (I - c L) u = rhs, Dirichlet z walls
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dims,beta,loc,c,ybc", [((4, 3, 5), 1.5, 0, 0.05, 0), ((4, 3, 5), 1.5, 1, 0.05, 0),
                                                 ((6, 4, 6), None, 0, 1.0, 0), ((5, 6, 4), 1.8, 1, 3e-3, 0),
                                                 ((2, 1, 7), 1.2, 0, 0.2, 0), ((4, 5, 4), 1.5, 0, 0.1, 1),
                                                 ((4, 3, 5), 1.4, 1, 0.3, 2), ((3, 6, 4), None, 1, 2.0, 1)])
def test_helmholtz3d_matches_dense_bruteforce(dims, beta, loc, c, ybc):
    """The eigenfunction-expansion solve against the assembled 3-D operator
    (a separate, point-by-point stencil apply) solved densely; y periodic or
    with Neumann / Dirichlet walls."""
    nx, ny, nz = dims
    lx, ly = 2.0, 1.5
    dzf = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    f = synth.normal(31 + nx + nz + loc, (nz, ny, nx))
    if loc == 1:
        f[-1] = 0.0  # the wall slot of a face field
    n = nx * ny * nz
    K = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        K[:, i] = oracle.apply_helmholtz3d(e.reshape(nz, ny, nx), lx, ly, dzf, c, loc, ybc).ravel()
    ref = np.linalg.solve(K, f.ravel()).reshape(nz, ny, nx)
    u = oracle.helmholtz3d_solve(f, lx, ly, dzf, c, loc, ybc)
    assert _rel(u, ref) < 1e-12
    if loc == 1:
        assert np.all(u[-1] == 0.0)


@pytest.mark.parametrize("loc", [0, 1])
def test_helmholtz3d_single_mode_closed_form_uniform(loc):
    nx, ny, nz = 8, 6, 12
    lx, ly = 2 * np.pi, np.pi
    dx, dy, dz = lx / nx, ly / ny, 2.0 / nz
    c = 2e-2
    x = np.arange(nx) * dx
    y = np.arange(ny) * dy
    z = (np.arange(nz) + 0.5) * dz if loc == 0 else (np.arange(nz) + 1) * dz
    for m, q, l in [(1, 0, 1), (2, 1, 3), (3, 2, 11 if loc == 0 else 10), (0, 0, 2)]:
        col = np.sin(np.pi * l * z / 2.0)
        if loc == 1:
            col[-1] = 0.0
        f = col[:, None, None] * np.cos(2 * np.pi * q * y / ly)[None, :, None] * \
            np.cos(2 * np.pi * m * x / lx)[None, None, :]
        lam = 2 * (np.cos(2 * np.pi * m / nx) - 1) / dx**2 + 2 * (np.cos(2 * np.pi * q / ny) - 1) / dy**2
        mu = 2 * (np.cos(np.pi * l / nz) - 1) / dz**2
        u = oracle.helmholtz3d_solve(f, lx, ly, synth.uniform_dz(nz), c, loc)
        assert _rel(u, f / (1 - c * (lam + mu))) < 1e-13


@pytest.mark.parametrize("loc", [0, 1])
def test_helmholtz3d_reduces_to_z_implicit_and_identity(loc):
    """A right-hand side constant in x and y has only the (0, 0) mode, where
    Eq. 8 is Eq. 11; c = 0 is the identity."""
    nx, ny, nz = 4, 6, 20
    dzf = synth.tanh_dz(nz, 1.6)
    col = synth.normal(5, (nz, 1, 1))
    f = np.broadcast_to(col, (nz, ny, nx)).copy()
    if loc == 1:
        f[-1] = 0.0
    c = 4e-3
    u3 = oracle.helmholtz3d_solve(f, 1.0, 1.0, dzf, c, loc)
    u1 = oracle.helmholtz_solve(f, dzf, c, loc)
    assert _rel(u3, u1) < 1e-13
    g = synth.normal(6, (nz, ny, nx))
    if loc == 1:
        g[-1] = 0.0
    assert _rel(oracle.helmholtz3d_solve(g, 1.0, 1.0, dzf, 0.0, loc), g) < 1e-15


# ----------------------------------------------------------------------------
# Walls in y: DCT-II / DST-II (Sec. 2.2.1) and the Poisson solve with them
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 27])
def test_dct_dst_match_scipy_and_invert(n):
    scipy_fft = pytest.importorskip("scipy.fft")
    x = synth.normal(n, (n,))
    # scipy's unnormalised type-2 transforms are twice the plain sums
    assert np.max(np.abs(oracle.dct2(x) - scipy_fft.dct(x, type=2) / 2)) < 1e-13 * n
    assert np.max(np.abs(oracle.dst2(x) - scipy_fft.dst(x, type=2) / 2)) < 1e-13 * n
    assert np.max(np.abs(oracle.idct2(oracle.dct2(x)) - x)) < 1e-13 * n
    assert np.max(np.abs(oracle.idst2(oracle.dst2(x)) - x)) < 1e-13 * n


@pytest.mark.parametrize("ybc", [1, 2])
def test_wall_eigenpairs_of_the_y_stencil(ybc):
    """cos / sin modes of the cell-centred wall stencil have the tabulated
    eigenvalues (the operator is applied point by point)."""
    ny, nz, ly = 12, 4, 3.0
    dy = ly / ny
    lam = oracle.eig_wall(ny, dy, ybc)
    j = np.arange(ny) + 0.5
    for k in range(ny):
        mode = np.cos(np.pi * k * j / ny) if ybc == 1 else np.sin(np.pi * (k + 1) * j / ny)
        p = np.broadcast_to(mode[None, :, None], (nz, ny, 3)).copy()
        # Neumann z walls: a z-constant field has no z contribution
        lp = oracle.apply_poisson_walls(p, 1.0, ly, synth.uniform_dz(nz), 0, ybc)
        assert np.max(np.abs(lp - lam[k] * p)) < 1e-10 * max(1.0, abs(lam[k]))


@pytest.mark.parametrize("dims,beta,bc,ybc", [((4, 4, 4), 1.5, 0, 1), ((4, 5, 4), 1.5, 1, 1),
                                              ((3, 4, 5), None, 0, 2), ((4, 3, 5), 1.8, 1, 2),
                                              ((2, 6, 4), 1.2, 0, 1), ((6, 4, 6), 1.6, 0, 2)])
def test_poisson_walls_match_dense_bruteforce(dims, beta, bc, ybc):
    nx, ny, nz = dims
    lx, ly = 2.0, 1.5
    dzf = synth.uniform_dz(nz) if beta is None else synth.tanh_dz(nz, beta)
    f = synth.normal(41 + nx + ny + nz + bc + ybc, (nz, ny, nx))
    n = nx * ny * nz
    L = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        L[:, i] = oracle.apply_poisson_walls(e.reshape(nz, ny, nx), lx, ly, dzf, bc, ybc).ravel()
    p = oracle.poisson_solve_walls(f, lx, ly, dzf, bc, ybc)
    w = np.repeat(dzf, nx * ny)
    if bc == 0 and ybc == 1:  # null space: the constants (bordered system)
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = L
        K[:n, n] = 1.0
        K[n, :n] = w
        ref = np.linalg.solve(K, np.concatenate([f.ravel(), [0.0]]))[:n]
        assert abs(w @ p.ravel()) < 1e-12 * np.sum(w) * np.max(np.abs(p))
    else:
        ref = np.linalg.solve(L, f.ravel())
    assert _rel(p.ravel(), ref) < 1e-11


@pytest.mark.parametrize("bc,ybc", [(0, 1), (1, 1), (0, 2), (1, 2)])
def test_poisson_walls_single_mode_closed_form(bc, ybc):
    nx, ny, nz = 8, 12, 10
    lx, ly = 2 * np.pi, 3.0
    dx, dy, dz = lx / nx, ly / ny, 2.0 / nz
    x = np.arange(nx) * dx
    jj = np.arange(ny) + 0.5
    zc = (np.arange(nz) + 0.5) * dz
    for m, k, l in [(1, 2, 1), (3, 0, 2), (0, 5, 3), (2, 11, 4)]:
        gy = np.cos(np.pi * k * jj / ny) if ybc == 1 else np.sin(np.pi * (k + 1) * jj / ny)
        gz = np.cos(np.pi * l * zc / 2.0) if bc == 0 else np.sin(np.pi * l * zc / 2.0)
        f = gz[:, None, None] * gy[None, :, None] * np.cos(2 * np.pi * m * x / lx)[None, None, :]
        kk = k if ybc == 1 else k + 1
        lam = 2 * (np.cos(2 * np.pi * m / nx) - 1) / dx**2 + 2 * (np.cos(np.pi * kk / ny) - 1) / dy**2 \
            + 2 * (np.cos(np.pi * l / nz) - 1) / dz**2
        p = oracle.poisson_solve_walls(f, lx, ly, synth.uniform_dz(nz), bc, ybc)
        assert _rel(p, f / lam) < 1e-12
