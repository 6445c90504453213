/*
 * chanfs_oracle.c -- plain, slow, single-threaded FP64 reference ("oracle")
 * for the Poisson / z-implicit Helmholtz solves of Diez, Peeters & Costa
 * (arXiv 2502.06296).  See chanfs_oracle.h for the conventions.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path.  It shares no code with
 * the CUDA library.  Built with -O2 -ffp-contract=off (no FMA contraction),
 * round-to-nearest-even throughout.
 *
 * Every function states the passage of the paper it follows.  Where the paper
 * is silent the reading taken is stated next to the code.
 */
#include "chanfs_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { BC_NEUMANN = 0, BC_DIRICHLET = 1 };
enum { LOC_CENTER = 0, LOC_FACE = 1 };
enum { HM_THOMAS = 0, HM_ALG2 = 1, HM_ALG1 = 2 };

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms.                                              */
/* Sec. 2.2.1: the x and y directions are diagonalised by discrete Fourier   */
/* transforms; any FFT library is allowed (Sec. 2.3.1).  Here: the O(n^2)    */
/* definition and a recursive mixed-radix Cooley-Tukey FFT checked against   */
/* it.                                                                       */
/* ------------------------------------------------------------------------ */

/* exp(sign * 2 pi i * e / n) with the exponent reduced modulo n first. */
static cplx unit_root(int n, long long e, int sign) {
  long long r = e % n;
  if (r < 0) r += n;
  double ang = TWO_PI * (double)r / (double)n;
  return cos(ang) + (double)sign * sin(ang) * I;
}

/* X_k = sum_j x_j exp(sign 2 pi i j k / n), straight from the definition. */
int or_dft_naive(int n, const double* in, double* out, int sign) {
  if (n < 1 || (sign != 1 && sign != -1)) return -1;
  const cplx* x = (const cplx*)in;
  cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int k = 0; k < n; ++k) {
    cplx acc = 0;
    for (int j = 0; j < n; ++j) acc += x[j] * unit_root(n, (long long)j * k, sign);
    X[k] = acc;
  }
  memcpy(out, X, sizeof(cplx) * (size_t)n);
  free(X);
  return 0;
}

static int smallest_factor(int n) {
  for (int r = 2; r * r <= n; ++r)
    if (n % r == 0) return r;
  return n;
}

/* Recursive decimation in time.  The length-n transform of x[0], x[s],
 * x[2s], ... is split into r interleaved sub-sequences (r = smallest prime
 * factor of n), each transformed recursively, and recombined as
 *   X[k] = sum_j W_n^{j k} Y_j[k mod n/r].
 * tw[e] = W_N^e for the top-level length N; W_n^e = tw[e * N/n]. */
static void fft_rec(int n, const cplx* x, int s, cplx* out, const cplx* tw,
                    int N) {
  if (n == 1) {
    out[0] = x[0];
    return;
  }
  int r = smallest_factor(n);
  int step = N / n;
  if (r == n) {
    for (int k = 0; k < n; ++k) {
      cplx acc = 0;
      for (int j = 0; j < n; ++j)
        acc += x[(size_t)j * s] * tw[(((long long)j * k) % n) * step];
      out[k] = acc;
    }
    return;
  }
  int m = n / r;
  cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int j = 0; j < r; ++j) fft_rec(m, x + (size_t)j * s, s * r, y + (size_t)j * m, tw, N);
  for (int k = 0; k < n; ++k) {
    cplx acc = 0;
    for (int j = 0; j < r; ++j)
      acc += y[(size_t)j * m + k % m] * tw[(((long long)j * k) % n) * step];
    out[k] = acc;
  }
  free(y);
}

static cplx* make_roots(int n, int sign) {
  cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int e = 0; e < n; ++e) tw[e] = unit_root(n, e, sign);
  return tw;
}

int or_fft(int n, const double* in, double* out, int sign) {
  if (n < 1 || (sign != 1 && sign != -1)) return -1;
  cplx* tw = make_roots(n, sign);
  cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  fft_rec(n, (const cplx*)in, 1, X, tw, n);
  memcpy(out, X, sizeof(cplx) * (size_t)n);
  free(X);
  free(tw);
  return 0;
}

/* Transform every line of a 3-D complex array along one axis.
 * dims = {n0, n1, n2} with axis 0 fastest; unnormalised. */
static void fft_axis(cplx* a, const int dims[3], int axis, int sign) {
  int n = dims[axis];
  size_t stride = 1;
  for (int d = 0; d < axis; ++d) stride *= (size_t)dims[d];
  size_t total = (size_t)dims[0] * dims[1] * dims[2];
  cplx* tw = make_roots(n, sign);
  cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (size_t base = 0; base < total; ++base) {
    /* base enumerates line starts: index with coordinate 0 along axis */
    if ((base / stride) % (size_t)n != 0) continue;
    for (int i = 0; i < n; ++i) line[i] = a[base + (size_t)i * stride];
    fft_rec(n, line, 1, res, tw, n);
    for (int i = 0; i < n; ++i) a[base + (size_t)i * stride] = res[i];
  }
  free(res);
  free(line);
  free(tw);
}

/* ------------------------------------------------------------------------ */
/* Appendix A: packed real-to-complex format.                                */
/* A real signal of n samples has floor(n/2)+1 DFT coefficients; X_0 is real, */
/* and for even n so is X_{n/2}.  The paper stores the n independent reals    */
/* in place of the 2(floor(n/2)+1) by moving one component of the last        */
/* coefficient into the (always zero) imaginary slot of X_0 (Eq. A.3).        */
/* Reading of the garbled subscripts: the last coefficient is X_{floor(n/2)}. */
/*   even n: [X0r, X_{n/2}r, X1r, X1i, ..., X_{n/2-1}r, X_{n/2-1}i]           */
/*   odd n : [X0r, X_{(n-1)/2}i, X1r, X1i, ..., X_{(n-1)/2}r]                 */
/* ------------------------------------------------------------------------ */

int or_rfft_packed(int n, const double* x, double* packed) {
  if (n < 2) return -1;
  cplx* z = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  for (int i = 0; i < n; ++i) z[i] = x[i];
  or_fft(n, (const double*)z, (double*)X, -1);
  int last = n / 2;
  for (int k = 1; k < last; ++k) {
    packed[2 * k] = creal(X[k]);
    packed[2 * k + 1] = cimag(X[k]);
  }
  packed[0] = creal(X[0]);
  if (n % 2 == 0) {
    packed[1] = creal(X[last]);
  } else {
    packed[2 * last] = creal(X[last]);
    packed[1] = cimag(X[last]);
  }
  free(X);
  free(z);
  return 0;
}

/* Inverse of or_rfft_packed: rebuild the Hermitian spectrum, inverse DFT
 * with 1/n, keep the real part. */
int or_irfft_packed(int n, const double* packed, double* x) {
  if (n < 2) return -1;
  cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cplx* z = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  int last = n / 2;
  X[0] = packed[0];
  for (int k = 1; k < last; ++k) X[k] = packed[2 * k] + packed[2 * k + 1] * I;
  if (n % 2 == 0)
    X[last] = packed[1];
  else
    X[last] = packed[2 * last] + packed[1] * I;
  for (int k = last + 1; k < n; ++k) X[k] = conj(X[n - k]);
  or_fft(n, (const double*)X, (double*)z, 1);
  for (int i = 0; i < n; ++i) x[i] = creal(z[i]) / (double)n;
  free(z);
  free(X);
  return 0;
}

/* Wavenumber held by a slot of the packed format (App. A: the eigenvalues
 * are re-ordered at initialisation to follow the packing). */
int or_packed_wavenumber(int n, int slot) {
  if (n < 2 || slot < 0 || slot >= n) return -1;
  if (slot == 0) return 0;
  if (slot == 1) return n / 2;
  if (n % 2 == 1 && slot == n - 1) return n / 2;
  return slot / 2;
}

/* ------------------------------------------------------------------------ */
/* Modified wavenumbers (Eq. 12, "second-order accurate eigenvalues", the     */
/* periodic case): lambda_k / h^2 = 2 (cos(2 pi k / n) - 1) / h^2.            */
/* ------------------------------------------------------------------------ */

int or_eig_periodic(int n, double h, double* lam) {
  if (n < 1 || !(h > 0)) return -1;
  for (int k = 0; k < n; ++k) lam[k] = 2.0 * (cos(TWO_PI * (double)k / (double)n) - 1.0) / (h * h);
  return 0;
}

int or_eig_packed(int n, double h, double* lam) {
  if (n < 2 || !(h > 0)) return -1;
  double* nat = (double*)malloc(sizeof(double) * (size_t)n);
  or_eig_periodic(n, h, nat);
  for (int s = 0; s < n; ++s) lam[s] = nat[or_packed_wavenumber(n, s)];
  free(nat);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* z metrics and stencil (Sec. 2.1: MAC staggered grid, second-order FD,     */
/* non-uniform z; eta of Eq. 12).                                            */
/* dzc[k] = distance between cell centres k and k+1 = (dzf[k]+dzf[k+1])/2.   */
/* Cell-centred operator (flux form):                                        */
/*   (L_z p)_k = [ (p_{k+1}-p_k)/dzc[k] - (p_k-p_{k-1})/dzc[k-1] ] / dzf[k]   */
/* so A_k = 1/(dzf[k] dzc[k-1]), C_k = 1/(dzf[k] dzc[k]), B_k = -(A_k+C_k).  */
/* Walls (reading; the paper does not spell them out, these are the standard */
/* MAC choices):                                                             */
/*   Neumann, centred:  ghost p_{-1} = p_0, so the wall flux vanishes.        */
/*   Dirichlet, centred: ghost u_{-1} = -u_0 at distance dzf[0].             */
/*   Dirichlet, face:   unknowns on the Nz-1 interior faces, w = 0 on walls; */
/*     (L_z w) at face k+1 = [ (w_{k+1}-w_k)/dzf[k+1] - (w_k-w_{k-1})/dzf[k] ] */
/*                           / dzc[k].                                       */
/* Returns the number of unknowns n (Nz or Nz-1).                            */
/* ------------------------------------------------------------------------ */

int or_dzc(int nz, const double* dzf, double* dzc) {
  if (nz < 2) return -1;
  for (int k = 0; k + 1 < nz; ++k) dzc[k] = 0.5 * (dzf[k] + dzf[k + 1]);
  return 0;
}

int or_lz_coefficients(int nz, const double* dzf, int bc, int loc, double* A,
                       double* B, double* C) {
  if (nz < 3) return -1;
  if (bc != BC_NEUMANN && bc != BC_DIRICHLET) return -1;
  if (loc != LOC_CENTER && loc != LOC_FACE) return -1;
  if (loc == LOC_FACE && bc != BC_DIRICHLET) return -1;
  double* dzc = (double*)malloc(sizeof(double) * (size_t)nz);
  or_dzc(nz, dzf, dzc);
  int n;
  if (loc == LOC_CENTER) {
    n = nz;
    for (int k = 0; k < nz; ++k) {
      double a = (k > 0) ? 1.0 / (dzf[k] * dzc[k - 1]) : 1.0 / (dzf[0] * dzf[0]);
      double c = (k < nz - 1) ? 1.0 / (dzf[k] * dzc[k]) : 1.0 / (dzf[nz - 1] * dzf[nz - 1]);
      A[k] = a;
      C[k] = c;
      B[k] = -(a + c);
    }
    /* fold the ghost cells */
    if (bc == BC_NEUMANN) {
      B[0] += A[0];
      B[nz - 1] += C[nz - 1];
    } else {
      B[0] -= A[0];
      B[nz - 1] -= C[nz - 1];
    }
    A[0] = 0.0;
    C[nz - 1] = 0.0;
  } else {
    n = nz - 1;
    for (int j = 0; j < n; ++j) {
      double a = 1.0 / (dzc[j] * dzf[j]);
      double c = 1.0 / (dzc[j] * dzf[j + 1]);
      A[j] = a;
      C[j] = c;
      B[j] = -(a + c);
    }
    A[0] = 0.0;     /* w = 0 on the bottom wall */
    C[n - 1] = 0.0; /* w = 0 on the top wall */
  }
  free(dzc);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal solvers.                                                      */
/* ------------------------------------------------------------------------ */

/* Thomas algorithm (Gaussian elimination without pivoting) for Eq. 13 --   */
/* the serial TDMA that the full-transpose method runs per (i,j) column      */
/* (Sec. 2.2.2, step 4).  a[0] and c[n-1] are ignored. */
int or_thomas(int n, const double* a, const double* b, const double* c,
              const double* d, double* x) {
  if (n < 1) return -1;
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  cp[0] = (n > 1) ? c[0] / b[0] : 0.0;
  dp[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    double piv = b[k] - a[k] * cp[k - 1];
    cp[k] = (k < n - 1) ? c[k] / piv : 0.0;
    dp[k] = (d[k] - a[k] * dp[k - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
  free(dp);
  free(cp);
  return 0;
}

/* Same, complex right-hand side, real matrix. */
static void thomas_complex(int n, const double* a, const double* b,
                           const double* c, const cplx* d, cplx* x) {
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  cplx* dp = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  cp[0] = (n > 1) ? c[0] / b[0] : 0.0;
  dp[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    double piv = b[k] - a[k] * cp[k - 1];
    cp[k] = (k < n - 1) ? c[k] / piv : 0.0;
    dp[k] = (d[k] - a[k] * dp[k - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
  free(dp);
  free(cp);
}

/* Partition q of p covers rows [q n / p, (q+1) n / p). */
static int part_begin(int n, int p, int q) { return (int)(((long long)q * n) / p); }

/* Algorithm 1 (Sec. 2.2.4, after Laszlo et al.): cyclic-reduction step per
 * partition, Thomas on the reduced 2p system (Step 2, unspecified in the
 * paper: reading = serial Thomas), in-place reconstruction (Step 3).
 * Works on copies because Algorithm 1 overwrites a, c and d. */
int or_alg1_solve(int n, int p, const double* a_in, const double* b_in,
                  const double* c_in, const double* d_in, double* x) {
  if (p < 1 || n < 3 * p) return -1;
  double* a = (double*)malloc(sizeof(double) * (size_t)n);
  double* b = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(a, a_in, sizeof(double) * (size_t)n);
  memcpy(b, b_in, sizeof(double) * (size_t)n);
  memcpy(c, c_in, sizeof(double) * (size_t)n);
  memcpy(d, d_in, sizeof(double) * (size_t)n);
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int m = part_begin(n, p, q + 1) - o;
    double *A = a + o, *B = b + o, *Cc = c + o, *D = d + o;
    /* Step 1: normalise rows 0 and 1 */
    A[0] /= B[0]; Cc[0] /= B[0]; D[0] /= B[0];
    A[1] /= B[1]; Cc[1] /= B[1]; D[1] /= B[1];
    /* forward elimination: express rows in terms of x_0 */
    for (int i = 2; i < m; ++i) {
      double r = 1.0 / (B[i] - A[i] * Cc[i - 1]);
      D[i] = r * (D[i] - A[i] * D[i - 1]);
      Cc[i] = r * Cc[i];
      A[i] = -r * A[i] * A[i - 1];
    }
    /* backward elimination: express rows in terms of x_{m-1} */
    for (int i = m - 3; i >= 1; --i) {
      D[i] = D[i] - Cc[i] * D[i + 1];
      A[i] = A[i] - Cc[i] * A[i + 1];
      Cc[i] = -Cc[i] * Cc[i + 1];
    }
    /* close row 0 */
    {
      double r = 1.0 / (1.0 - A[1] * Cc[0]);
      D[0] = r * (D[0] - Cc[0] * D[1]);
      A[0] = r * A[0];
      Cc[0] = -r * Cc[0] * Cc[1];
    }
    for (int i = 0; i < m; ++i) B[i] = 1.0;
  }
  /* Step 2: reduced system in [x_0^0, x_{m-1}^0, x_0^1, ...] */
  int nr = 2 * p;
  double* ra = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rb = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rc = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rd = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rx = (double*)malloc(sizeof(double) * (size_t)nr);
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int e = part_begin(n, p, q + 1) - 1;
    ra[2 * q] = a[o]; rb[2 * q] = 1.0; rc[2 * q] = c[o]; rd[2 * q] = d[o];
    ra[2 * q + 1] = a[e]; rb[2 * q + 1] = 1.0; rc[2 * q + 1] = c[e]; rd[2 * q + 1] = d[e];
  }
  or_thomas(nr, ra, rb, rc, rd, rx);
  /* Step 3: reconstruct */
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int m = part_begin(n, p, q + 1) - o;
    double x0 = rx[2 * q], xm = rx[2 * q + 1];
    x[o] = x0;
    x[o + m - 1] = xm;
    for (int i = 1; i <= m - 2; ++i) x[o + i] = d[o + i] - a[o + i] * x0 - c[o + i] * xm;
  }
  free(rx); free(rd); free(rc); free(rb); free(ra);
  free(d); free(c); free(b); free(a);
  return 0;
}

/* Algorithm 2 (Sec. 2.2.4), Step 1 -- initialisation from the original
 * coefficients (A, B, C) of one partition of m rows; only (a, b, c) are
 * produced, the right-hand side is not touched. */
int or_alg2_prepare(int m, const double* A, const double* B, const double* C,
                    double* a, double* b, double* c) {
  if (m < 3) return -1;
  a[1] = A[1];
  b[1] = B[1];
  for (int i = 2; i <= m - 1; ++i) {
    b[i] = B[i] - A[i] * C[i - 1] / b[i - 1];
    a[i] = -A[i] * a[i - 1] / b[i - 1];
  }
  c[m - 1] = C[m - 1];
  c[m - 2] = C[m - 2];
  for (int i = m - 3; i >= 1; --i) {
    a[i] = a[i] - C[i] * a[i + 1] / b[i + 1];
    c[i] = -C[i] * c[i + 1] / b[i + 1];
  }
  a[0] = A[0];
  b[0] = B[0] - C[0] * a[1] / B[1];
  c[0] = -C[0] * c[1] / B[1];
  return 0;
}

/* Algorithm 2, Step 2 -- runtime reduction: only d changes, in place. */
int or_alg2_runtime(int m, const double* A, const double* C, const double* b,
                    double* d) {
  if (m < 3) return -1;
  for (int i = 2; i <= m - 1; ++i) d[i] = d[i] - A[i] * d[i - 1] / b[i - 1];
  for (int i = m - 3; i >= 0; --i) d[i] = d[i] - C[i] * d[i + 1] / b[i + 1];
  return 0;
}

/* Algorithm 2, Step 4 -- reconstruct the interior in place from the two
 * boundary values of the partition. */
int or_alg2_reconstruct(int m, const double* a, const double* b,
                        const double* c, double x0, double xm1, double* d) {
  if (m < 3) return -1;
  d[0] = x0;
  d[m - 1] = xm1;
  for (int i = 1; i <= m - 2; ++i) d[i] = (d[i] - a[i] * x0 - c[i] * xm1) / b[i];
  return 0;
}

/* Algorithm 2 end to end on p partitions.  Step 3 (the reduced system of
 * the 2p boundary unknowns) is not given in the paper; reading: partition
 * q contributes
 *   a_0 x_{m-1}^{q-1} + b_0 x_0^q + c_0 x_{m-1}^q = d_0          (row 0)
 *   a_{m-1} x_0^q + b_{m-1} x_{m-1}^q + c_{m-1} x_0^{q+1} = d_{m-1} (row m-1)
 * which is tridiagonal in [x_0^0, x_{m-1}^0, x_0^1, ...]; solved by Thomas. */
int or_alg2_solve(int n, int p, const double* A, const double* B,
                  const double* C, const double* d_in, double* x) {
  if (p < 1 || n < 3 * p) return -1;
  double* a = (double*)malloc(sizeof(double) * (size_t)n);
  double* b = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(d, d_in, sizeof(double) * (size_t)n);
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int m = part_begin(n, p, q + 1) - o;
    or_alg2_prepare(m, A + o, B + o, C + o, a + o, b + o, c + o);
    or_alg2_runtime(m, A + o, C + o, b + o, d + o);
  }
  int nr = 2 * p;
  double* ra = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rb = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rc = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rd = (double*)malloc(sizeof(double) * (size_t)nr);
  double* rx = (double*)malloc(sizeof(double) * (size_t)nr);
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int e = part_begin(n, p, q + 1) - 1;
    ra[2 * q] = a[o]; rb[2 * q] = b[o]; rc[2 * q] = c[o]; rd[2 * q] = d[o];
    ra[2 * q + 1] = a[e]; rb[2 * q + 1] = b[e]; rc[2 * q + 1] = c[e]; rd[2 * q + 1] = d[e];
  }
  or_thomas(nr, ra, rb, rc, rd, rx);
  for (int q = 0; q < p; ++q) {
    int o = part_begin(n, p, q);
    int m = part_begin(n, p, q + 1) - o;
    or_alg2_reconstruct(m, a + o, b + o, c + o, rx[2 * q], rx[2 * q + 1], d + o);
  }
  memcpy(x, d, sizeof(double) * (size_t)n);
  free(rx); free(rd); free(rc); free(rb); free(ra);
  free(d); free(c); free(b); free(a);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 3-D operators, written directly in flux form from the staggered stencil   */
/* (Sec. 2.1), independently of or_lz_coefficients.                          */
/* ------------------------------------------------------------------------ */

/* Second difference along z of one centred column, with the wall ghosts. */
static double lz_centre(int nz, const double* dzf, const double* dzc, int bc,
                        const double* col, size_t st, int k) {
  double pk = col[(size_t)k * st];
  double up, dn;
  if (k < nz - 1)
    up = (col[(size_t)(k + 1) * st] - pk) / dzc[k];
  else
    up = (bc == BC_NEUMANN) ? 0.0 : (-pk - pk) / dzf[nz - 1];
  if (k > 0)
    dn = (pk - col[(size_t)(k - 1) * st]) / dzc[k - 1];
  else
    dn = (bc == BC_NEUMANN) ? 0.0 : (pk - (-pk)) / dzf[0];
  return (up - dn) / dzf[k];
}

/* Second difference along z at face slot j (face z_f[j+1]), w = 0 on walls. */
static double lz_face(int nz, const double* dzf, const double* dzc,
                      const double* col, size_t st, int j) {
  double wj = col[(size_t)j * st];
  double wu = (j + 1 <= nz - 2) ? col[(size_t)(j + 1) * st] : 0.0;
  double wd = (j - 1 >= 0) ? col[(size_t)(j - 1) * st] : 0.0;
  double up = (wu - wj) / dzf[j + 1];
  double dn = (wj - wd) / dzf[j];
  return (up - dn) / dzc[j];
}

/* (L p) = d2p/dx2 + d2p/dy2 (periodic, uniform) + L_z p, the operator of
 * Eq. 4 / Eq. 12 before the Fourier synthesis. */
int or_apply_poisson(int nx, int ny, int nz, double lx, double ly,
                     const double* dzf, int bc, const double* p, double* out) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0)) return -1;
  if (bc != BC_NEUMANN && bc != BC_DIRICHLET) return -1;
  double dx = lx / nx, dy = ly / ny;
  double* dzc = (double*)malloc(sizeof(double) * (size_t)nz);
  or_dzc(nz, dzf, dzc);
  size_t sxy = (size_t)nx * ny;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t i = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
        int xp = (x + 1) % nx, xm = (x + nx - 1) % nx;
        int yp = (y + 1) % ny, ym = (y + ny - 1) % ny;
        size_t row = (size_t)nx * ((size_t)y + (size_t)ny * z);
        double lxx = (p[row + xp] - 2.0 * p[i] + p[row + xm]) / (dx * dx);
        size_t pl = (size_t)nx * ((size_t)ny * z);
        double lyy = (p[pl + (size_t)nx * yp + x] - 2.0 * p[i] + p[pl + (size_t)nx * ym + x]) / (dy * dy);
        double lzz = lz_centre(nz, dzf, dzc, bc, p + (size_t)x + (size_t)nx * y, sxy, z);
        out[i] = lxx + lyy + lzz;
      }
  free(dzc);
  return 0;
}

/* (I - c L_z) u per column, homogeneous Dirichlet walls (Eq. 11 left-hand
 * side with c = gamma_k nu dt / 2).  For face fields the wall slot Nz-1 is
 * passed through unchanged. */
int or_apply_helmholtz(int nx, int ny, int nz, const double* dzf, double c,
                       int loc, const double* u, double* out) {
  if (nx < 1 || ny < 1 || nz < 3) return -1;
  if (loc != LOC_CENTER && loc != LOC_FACE) return -1;
  double* dzc = (double*)malloc(sizeof(double) * (size_t)nz);
  or_dzc(nz, dzf, dzc);
  size_t sxy = (size_t)nx * ny;
  for (size_t col = 0; col < sxy; ++col)
    for (int k = 0; k < nz; ++k) {
      size_t i = col + sxy * (size_t)k;
      if (loc == LOC_CENTER)
        out[i] = u[i] - c * lz_centre(nz, dzf, dzc, BC_DIRICHLET, u + col, sxy, k);
      else if (k < nz - 1)
        out[i] = u[i] - c * lz_face(nz, dzf, dzc, u + col, sxy, k);
      else
        out[i] = u[i];
    }
  free(dzc);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Poisson solve by eigenfunction expansion (Sec. 2.2.1, Eq. 12):           */
/*  1. Neumann only: project f onto the range of L by removing its           */
/*     dzf-weighted mean (reading: the compatibility condition of the        */
/*     conservative operator; w_k = dzf[k]).                                 */
/*  2. forward DFT along x, then along y.                                    */
/*  3. per (kx,ky): Thomas on A_k, B_k + lx[kx] + ly[ky], C_k.               */
/*     Neumann (0,0) column is singular: row 0 is replaced by phi_0 = 0, and */
/*     the dzf-weighted mean is removed afterwards (zero-mean convention).   */
/*  4. inverse DFT along y, then x, with 1/(Nx Ny); keep the real part.      */
/* ------------------------------------------------------------------------ */

int or_poisson_solve(int nx, int ny, int nz, double lx, double ly,
                     const double* dzf, int bc, const double* f, double* p) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0)) return -1;
  if (bc != BC_NEUMANN && bc != BC_DIRICHLET) return -1;
  size_t n = (size_t)nx * ny * nz, sxy = (size_t)nx * ny;
  cplx* F = (cplx*)malloc(sizeof(cplx) * n);
  double wmean = 0.0;
  if (bc == BC_NEUMANN) {
    double sw = 0.0, swf = 0.0;
    for (int z = 0; z < nz; ++z)
      for (size_t c = 0; c < sxy; ++c) {
        swf += dzf[z] * f[c + sxy * (size_t)z];
        sw += dzf[z];
      }
    wmean = swf / sw;
  }
  for (size_t i = 0; i < n; ++i) F[i] = f[i] - wmean;
  int dims[3] = {nx, ny, nz};
  fft_axis(F, dims, 0, -1);
  fft_axis(F, dims, 1, -1);

  double* lamx = (double*)malloc(sizeof(double) * (size_t)nx);
  double* lamy = (double*)malloc(sizeof(double) * (size_t)ny);
  or_eig_periodic(nx, lx / nx, lamx);
  or_eig_periodic(ny, ly / ny, lamy);
  double* A = (double*)malloc(sizeof(double) * (size_t)nz);
  double* B = (double*)malloc(sizeof(double) * (size_t)nz);
  double* C = (double*)malloc(sizeof(double) * (size_t)nz);
  double* b = (double*)malloc(sizeof(double) * (size_t)nz);
  double* a = (double*)malloc(sizeof(double) * (size_t)nz);
  double* c = (double*)malloc(sizeof(double) * (size_t)nz);
  cplx* d = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  or_lz_coefficients(nz, dzf, bc, LOC_CENTER, A, B, C);
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nx; ++kx) {
      double lam = lamx[kx] + lamy[ky];
      for (int k = 0; k < nz; ++k) {
        a[k] = A[k];
        b[k] = B[k] + lam;
        c[k] = C[k];
        d[k] = F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k];
      }
      int singular = (bc == BC_NEUMANN && kx == 0 && ky == 0);
      if (singular) {
        b[0] = 1.0;
        c[0] = 0.0;
        d[0] = 0.0;
      }
      thomas_complex(nz, a, b, c, d, x);
      if (singular) {
        cplx sw = 0.0, swx = 0.0;
        for (int k = 0; k < nz; ++k) {
          swx += dzf[k] * x[k];
          sw += dzf[k];
        }
        cplx mean = swx / sw;
        for (int k = 0; k < nz; ++k) x[k] -= mean;
      }
      for (int k = 0; k < nz; ++k) F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k] = x[k];
    }
  fft_axis(F, dims, 1, 1);
  fft_axis(F, dims, 0, 1);
  double scale = 1.0 / ((double)nx * (double)ny);
  for (size_t i = 0; i < n; ++i) p[i] = creal(F[i]) * scale;
  free(x); free(d); free(c); free(a); free(b); free(C); free(B); free(A);
  free(lamy); free(lamx); free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* z-implicit Helmholtz (Eq. 11): (I - c L_z) u = rhs per (x,y) column with   */
/* homogeneous Dirichlet walls; A' = -c A, B' = 1 - c B, C' = -c C.           */
/* method 0: Thomas (the plain definition); 1: Algorithm 2 on nparts           */
/* partitions; 2: Algorithm 1 on nparts partitions.                            */
/* ------------------------------------------------------------------------ */

int or_helmholtz_solve(int nx, int ny, int nz, const double* dzf, double c,
                       int loc, int method, int nparts, const double* rhs,
                       double* u) {
  if (nx < 1 || ny < 1 || nz < 3) return -1;
  if (loc != LOC_CENTER && loc != LOC_FACE) return -1;
  if (method != HM_THOMAS && method != HM_ALG2 && method != HM_ALG1) return -1;
  double* A = (double*)malloc(sizeof(double) * (size_t)nz);
  double* B = (double*)malloc(sizeof(double) * (size_t)nz);
  double* C = (double*)malloc(sizeof(double) * (size_t)nz);
  int n = or_lz_coefficients(nz, dzf, BC_DIRICHLET, loc, A, B, C);
  if (method != HM_THOMAS && (nparts < 1 || n < 3 * nparts)) {
    free(C); free(B); free(A);
    return -1;
  }
  for (int k = 0; k < n; ++k) {
    A[k] = -c * A[k];
    B[k] = 1.0 - c * B[k];
    C[k] = -c * C[k];
  }
  size_t sxy = (size_t)nx * ny;
  double* d = (double*)malloc(sizeof(double) * (size_t)nz);
  double* x = (double*)malloc(sizeof(double) * (size_t)nz);
  for (size_t col = 0; col < sxy; ++col) {
    for (int k = 0; k < n; ++k) d[k] = rhs[col + sxy * (size_t)k];
    if (method == HM_THOMAS)
      or_thomas(n, A, B, C, d, x);
    else if (method == HM_ALG2)
      or_alg2_solve(n, nparts, A, B, C, d, x);
    else
      or_alg1_solve(n, nparts, A, B, C, d, x);
    for (int k = 0; k < n; ++k) u[col + sxy * (size_t)k] = x[k];
    if (loc == LOC_FACE) u[col + sxy * (size_t)(nz - 1)] = 0.0;
  }
  free(x); free(d); free(C); free(B); free(A);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Fully implicit 3-D Helmholtz (Eq. 8): (I - c L) u = rhs with L the full    */
/* staggered Laplacian, periodic in x and y, homogeneous Dirichlet z walls   */
/* (cell-centred u, v or face-located w as in the z-implicit solve).         */
/* Apply: the stencil written out point by point (face fields: the wall slot */
/* Nz-1 is passed through unchanged).                                        */
/* ------------------------------------------------------------------------ */

int or_apply_helmholtz3d_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc, const double* u,
                               double* out);

int or_apply_helmholtz3d(int nx, int ny, int nz, double lx, double ly,
                         const double* dzf, double c, int loc, const double* u,
                         double* out) {
  return or_apply_helmholtz3d_walls(nx, ny, nz, lx, ly, dzf, c, loc, 0, u, out);
}

int or_apply_helmholtz3d_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc, const double* u,
                               double* out) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0)) return -1;
  if (loc != LOC_CENTER && loc != LOC_FACE) return -1;
  if (ybc < 0 || ybc > 2) return -1;
  const double g = (ybc == 1) ? 1.0 : -1.0;  /* wall ghost = g * boundary value */
  double dx = lx / nx, dy = ly / ny;
  double* dzc = (double*)malloc(sizeof(double) * (size_t)nz);
  or_dzc(nz, dzf, dzc);
  size_t sxy = (size_t)nx * ny;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t i = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
        if (loc == LOC_FACE && z == nz - 1) {
          out[i] = u[i];
          continue;
        }
        int xp = (x + 1) % nx, xm = (x + nx - 1) % nx;
        int yp = (y + 1) % ny, ym = (y + ny - 1) % ny;
        size_t row = (size_t)nx * ((size_t)y + (size_t)ny * z);
        size_t pl = (size_t)nx * ((size_t)ny * z);
        double lxx = (u[row + xp] - 2.0 * u[i] + u[row + xm]) / (dx * dx);
        double up = u[pl + (size_t)nx * yp + x], dn = u[pl + (size_t)nx * ym + x];
        if (ybc != 0) {
          up = (y + 1 < ny) ? u[pl + (size_t)nx * (y + 1) + x] : g * u[i];
          dn = (y > 0) ? u[pl + (size_t)nx * (y - 1) + x] : g * u[i];
        }
        double lyy = (up - 2.0 * u[i] + dn) / (dy * dy);
        const double* colp = u + (size_t)x + (size_t)nx * y;
        double lzz = (loc == LOC_CENTER) ? lz_centre(nz, dzf, dzc, BC_DIRICHLET, colp, sxy, z)
                                         : lz_face(nz, dzf, dzc, colp, sxy, z);
        out[i] = u[i] - c * (lxx + lyy + lzz);
      }
  free(dzc);
  return 0;
}

/* Solve by eigenfunction expansion, as the Poisson solve: DFT along x and y,  */
/* per (kx,ky) the tridiagonal system with A' = -c A_k,                        */
/* B' = 1 - c (B_k + lx[kx] + ly[ky]), C' = -c C_k (Dirichlet rows of the      */
/* field's location; nonsingular for c >= 0), inverse DFTs with 1/(Nx Ny).     */
int or_helmholtz3d_solve_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc,
                               const double* rhs, double* u);
static void y_walls_axis(cplx* F, int nx, int ny, int nz, int ybc, int inverse);

int or_helmholtz3d_solve(int nx, int ny, int nz, double lx, double ly,
                         const double* dzf, double c, int loc, const double* rhs,
                         double* u) {
  return or_helmholtz3d_solve_walls(nx, ny, nz, lx, ly, dzf, c, loc, 0, rhs, u);
}

/* ybc as for the Poisson solve with walls: DFT, DCT-II or DST-II along y. */
int or_helmholtz3d_solve_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc,
                               const double* rhs, double* u) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0) || !(c >= 0)) return -1;
  if (loc != LOC_CENTER && loc != LOC_FACE) return -1;
  if (ybc < 0 || ybc > 2) return -1;
  size_t n3 = (size_t)nx * ny * nz, sxy = (size_t)nx * ny;
  cplx* F = (cplx*)malloc(sizeof(cplx) * n3);
  for (size_t i = 0; i < n3; ++i) F[i] = rhs[i];
  int dims[3] = {nx, ny, nz};
  fft_axis(F, dims, 0, -1);
  if (ybc == 0) fft_axis(F, dims, 1, -1);
  else y_walls_axis(F, nx, ny, nz, ybc, 0);
  double* lamx = (double*)malloc(sizeof(double) * (size_t)nx);
  double* lamy = (double*)malloc(sizeof(double) * (size_t)ny);
  or_eig_periodic(nx, lx / nx, lamx);
  if (ybc == 0) or_eig_periodic(ny, ly / ny, lamy);
  else or_eig_wall(ny, ly / ny, ybc, lamy);
  double* A = (double*)malloc(sizeof(double) * (size_t)nz);
  double* B = (double*)malloc(sizeof(double) * (size_t)nz);
  double* C = (double*)malloc(sizeof(double) * (size_t)nz);
  double* a = (double*)malloc(sizeof(double) * (size_t)nz);
  double* b = (double*)malloc(sizeof(double) * (size_t)nz);
  double* cc = (double*)malloc(sizeof(double) * (size_t)nz);
  cplx* d = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  int n = or_lz_coefficients(nz, dzf, BC_DIRICHLET, loc, A, B, C);
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nx; ++kx) {
      double lam = lamx[kx] + lamy[ky];
      for (int k = 0; k < n; ++k) {
        a[k] = -c * A[k];
        b[k] = 1.0 - c * (B[k] + lam);
        cc[k] = -c * C[k];
        d[k] = F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k];
      }
      thomas_complex(n, a, b, cc, d, x);
      for (int k = 0; k < n; ++k) F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k] = x[k];
      for (int k = n; k < nz; ++k) F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k] = 0.0;
    }
  if (ybc == 0) fft_axis(F, dims, 1, 1);
  else y_walls_axis(F, nx, ny, nz, ybc, 1);
  fft_axis(F, dims, 0, 1);
  /* the inverse wall transforms include their 1/Ny */
  double scale = 1.0 / ((double)nx * (ybc == 0 ? (double)ny : 1.0));
  for (size_t i = 0; i < n3; ++i) u[i] = creal(F[i]) * scale;
  free(x); free(d); free(cc); free(b); free(a); free(C); free(B); free(A);
  free(lamy); free(lamx); free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Walls in y (Sec. 2.2.1 names DCT/DST for non-periodic directions).        */
/* Cell-centred unknowns, ghost p_{-1} = +-p_0 and p_{Ny} = +-p_{Ny-1}:      */
/*   Neumann   (+): eigenvectors cos(pi k (j+1/2)/N), k = 0..N-1 (DCT-II);   */
/*   Dirichlet (-): eigenvectors sin(pi (k+1)(j+1/2)/N), k = 0..N-1 (DST-II); */
/* eigenvalues 2(cos(pi k/N) - 1)/h^2 and 2(cos(pi (k+1)/N) - 1)/h^2.        */
/* The transforms below are their definitions, summed directly.             */
/* ybc: 0 periodic, 1 Neumann walls, 2 Dirichlet walls.                      */
/* ------------------------------------------------------------------------ */
enum { Y_PERIODIC = 0, Y_NEUMANN = 1, Y_DIRICHLET = 2 };
static const double PI_HALF_TURN = 3.141592653589793238462643383279502884;

int or_dct2(int n, const double* x, double* X) {
  if (n < 1) return -1;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += x[j] * cos(PI_HALF_TURN * k * (j + 0.5) / n);
    X[k] = s;
  }
  return 0;
}

int or_idct2(int n, const double* X, double* x) {
  if (n < 1) return -1;
  for (int j = 0; j < n; ++j) {
    double s = X[0];
    for (int k = 1; k < n; ++k) s += 2.0 * X[k] * cos(PI_HALF_TURN * k * (j + 0.5) / n);
    x[j] = s / n;
  }
  return 0;
}

int or_dst2(int n, const double* x, double* X) {
  if (n < 1) return -1;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += x[j] * sin(PI_HALF_TURN * (k + 1) * (j + 0.5) / n);
    X[k] = s;
  }
  return 0;
}

int or_idst2(int n, const double* X, double* x) {
  if (n < 1) return -1;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      const double w = (k == n - 1) ? 1.0 : 2.0;
      s += w * X[k] * sin(PI_HALF_TURN * (k + 1) * (j + 0.5) / n);
    }
    x[j] = s / n;
  }
  return 0;
}

int or_eig_wall(int n, double h, int ybc, double* lam) {
  if (n < 1 || !(h > 0) || (ybc != Y_NEUMANN && ybc != Y_DIRICHLET)) return -1;
  for (int k = 0; k < n; ++k) {
    const int m = (ybc == Y_NEUMANN) ? k : k + 1;
    lam[k] = 2.0 * (cos(PI_HALF_TURN * m / n) - 1.0) / (h * h);
  }
  return 0;
}

/* L p with walls in y: the 7-point stencil written out point by point. */
int or_apply_poisson_walls(int nx, int ny, int nz, double lx, double ly, const double* dzf,
                           int bc, int ybc, const double* p, double* out) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0)) return -1;
  if (bc != BC_NEUMANN && bc != BC_DIRICHLET) return -1;
  if (ybc != Y_PERIODIC && ybc != Y_NEUMANN && ybc != Y_DIRICHLET) return -1;
  double dx = lx / nx, dy = ly / ny;
  double* dzc = (double*)malloc(sizeof(double) * (size_t)nz);
  or_dzc(nz, dzf, dzc);
  size_t sxy = (size_t)nx * ny;
  const double g = (ybc == Y_NEUMANN) ? 1.0 : -1.0;  /* ghost = g * boundary value */
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t pl = sxy * (size_t)z;
        size_t i = pl + (size_t)nx * y + x;
        int xp = (x + 1) % nx, xm = (x + nx - 1) % nx;
        double lxx = (p[pl + (size_t)nx * y + xp] - 2.0 * p[i] + p[pl + (size_t)nx * y + xm]) / (dx * dx);
        double up, dn;
        if (ybc == Y_PERIODIC) {
          up = p[pl + (size_t)nx * ((y + 1) % ny) + x];
          dn = p[pl + (size_t)nx * ((y + ny - 1) % ny) + x];
        } else {
          up = (y + 1 < ny) ? p[pl + (size_t)nx * (y + 1) + x] : g * p[i];
          dn = (y > 0) ? p[pl + (size_t)nx * (y - 1) + x] : g * p[i];
        }
        double lyy = (up - 2.0 * p[i] + dn) / (dy * dy);
        double lzz = lz_centre(nz, dzf, dzc, bc, p + (size_t)x + (size_t)nx * y, sxy, z);
        out[i] = lxx + lyy + lzz;
      }
  free(dzc);
  return 0;
}

/* Transform along y of every (x, z) line of a complex field: DFT, or the
 * DCT-II / DST-II of real and imaginary parts (inverse: the inverse sums). */
static void y_walls_axis(cplx* F, int nx, int ny, int nz, int ybc, int inverse) {
  double* re = (double*)malloc(sizeof(double) * (size_t)ny);
  double* im = (double*)malloc(sizeof(double) * (size_t)ny);
  double* ro = (double*)malloc(sizeof(double) * (size_t)ny);
  double* io = (double*)malloc(sizeof(double) * (size_t)ny);
  for (int z = 0; z < nz; ++z)
    for (int x = 0; x < nx; ++x) {
      cplx* base = F + (size_t)x + (size_t)nx * (size_t)ny * z;
      for (int y = 0; y < ny; ++y) {
        re[y] = creal(base[(size_t)nx * y]);
        im[y] = cimag(base[(size_t)nx * y]);
      }
      if (ybc == Y_NEUMANN) {
        if (inverse) { or_idct2(ny, re, ro); or_idct2(ny, im, io); }
        else { or_dct2(ny, re, ro); or_dct2(ny, im, io); }
      } else {
        if (inverse) { or_idst2(ny, re, ro); or_idst2(ny, im, io); }
        else { or_dst2(ny, re, ro); or_dst2(ny, im, io); }
      }
      for (int y = 0; y < ny; ++y) base[(size_t)nx * y] = ro[y] + I * io[y];
    }
  free(io); free(ro); free(im); free(re);
}

/* Poisson solve with walls in y: DFT along x, DCT-II / DST-II (or DFT)
 * along y, one tridiagonal system per (kx, ky) with lx[kx] + ly[ky], inverse
 * transforms.  The (0,0) system is singular when both y and z walls are
 * Neumann (or y periodic and z Neumann): pinned, then the dz-weighted mean
 * removed, as in or_poisson_solve; the rhs is projected first. */
int or_poisson_solve_walls(int nx, int ny, int nz, double lx, double ly, const double* dzf,
                           int bc, int ybc, const double* f, double* p) {
  if (nx < 1 || ny < 1 || nz < 3 || !(lx > 0) || !(ly > 0)) return -1;
  if (bc != BC_NEUMANN && bc != BC_DIRICHLET) return -1;
  if (ybc != Y_PERIODIC && ybc != Y_NEUMANN && ybc != Y_DIRICHLET) return -1;
  if (ybc == Y_PERIODIC) return or_poisson_solve(nx, ny, nz, lx, ly, dzf, bc, f, p);
  const int has_null = (bc == BC_NEUMANN && ybc == Y_NEUMANN);
  size_t n = (size_t)nx * ny * nz, sxy = (size_t)nx * ny;
  cplx* F = (cplx*)malloc(sizeof(cplx) * n);
  double wmean = 0.0;
  if (has_null) {
    double sw = 0.0, swf = 0.0;
    for (int z = 0; z < nz; ++z)
      for (size_t c = 0; c < sxy; ++c) {
        swf += dzf[z] * f[c + sxy * (size_t)z];
        sw += dzf[z];
      }
    wmean = swf / sw;
  }
  for (size_t i = 0; i < n; ++i) F[i] = f[i] - wmean;
  int dims[3] = {nx, ny, nz};
  fft_axis(F, dims, 0, -1);
  y_walls_axis(F, nx, ny, nz, ybc, 0);
  double* lamx = (double*)malloc(sizeof(double) * (size_t)nx);
  double* lamy = (double*)malloc(sizeof(double) * (size_t)ny);
  or_eig_periodic(nx, lx / nx, lamx);
  or_eig_wall(ny, ly / ny, ybc, lamy);
  double* A = (double*)malloc(sizeof(double) * (size_t)nz);
  double* B = (double*)malloc(sizeof(double) * (size_t)nz);
  double* C = (double*)malloc(sizeof(double) * (size_t)nz);
  double* a = (double*)malloc(sizeof(double) * (size_t)nz);
  double* b = (double*)malloc(sizeof(double) * (size_t)nz);
  double* c = (double*)malloc(sizeof(double) * (size_t)nz);
  cplx* d = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)nz);
  or_lz_coefficients(nz, dzf, bc, LOC_CENTER, A, B, C);
  for (int ky = 0; ky < ny; ++ky)
    for (int kx = 0; kx < nx; ++kx) {
      double lam = lamx[kx] + lamy[ky];
      for (int k = 0; k < nz; ++k) {
        a[k] = A[k];
        b[k] = B[k] + lam;
        c[k] = C[k];
        d[k] = F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k];
      }
      int singular = (has_null && kx == 0 && ky == 0);
      if (singular) {
        b[0] = 1.0;
        c[0] = 0.0;
        d[0] = 0.0;
      }
      thomas_complex(nz, a, b, c, d, x);
      if (singular) {
        cplx sw = 0.0, swx = 0.0;
        for (int k = 0; k < nz; ++k) {
          swx += dzf[k] * x[k];
          sw += dzf[k];
        }
        cplx mean = swx / sw;
        for (int k = 0; k < nz; ++k) x[k] -= mean;
      }
      for (int k = 0; k < nz; ++k) F[(size_t)kx + (size_t)nx * ky + sxy * (size_t)k] = x[k];
    }
  y_walls_axis(F, nx, ny, nz, ybc, 1);
  fft_axis(F, dims, 0, 1);
  double scale = 1.0 / (double)nx;
  for (size_t i = 0; i < n; ++i) p[i] = creal(F[i]) * scale;
  free(x); free(d); free(c); free(b); free(a); free(C); free(B); free(A);
  free(lamy); free(lamx); free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Spectral layout of the solver: App. A packing along x (even Nx: pair j of */
/* a line is X_j for j >= 1 and X_0 + i X_{Nx/2} for j = 0), complex DFT     */
/* along y of each pair, and for pair j = 0 the same packing idea once more  */
/* along y (both F(0,ky) and F(Nx/2,ky) are DFTs of real sequences, so each  */
/* is fixed by ky = 0..Ny/2):                                                */
/*   slot ky, ky = 0 or 2ky = Ny:  F(0,ky) + i F(Nx/2,ky)  (both real)      */
/*   slot ky, 0 < 2ky < Ny:        F(0,ky)                                  */
/*   slot ky, 2ky > Ny:            F(Nx/2, Ny-ky)                           */
/* Built here from the full 2-D DFT, i.e. the definition of the layout.     */
/* ------------------------------------------------------------------------ */

int or_spectral_forward(int nx, int ny, int nz, const double* f, double* s) {
  if (nx < 2 || nx % 2 != 0 || ny < 1 || nz < 1) return -1;
  size_t n = (size_t)nx * ny * nz;
  int M = nx / 2;
  cplx* F = (cplx*)malloc(sizeof(cplx) * n);
  for (size_t i = 0; i < n; ++i) F[i] = f[i];
  int dims[3] = {nx, ny, nz};
  fft_axis(F, dims, 0, -1);
  fft_axis(F, dims, 1, -1);
  cplx* S = (cplx*)s; /* M complex pairs per (ky, z) line */
  for (int z = 0; z < nz; ++z)
    for (int ky = 0; ky < ny; ++ky) {
      const cplx* row = F + (size_t)nx * ((size_t)ky + (size_t)ny * z);
      cplx* out = S + (size_t)M * ((size_t)ky + (size_t)ny * z);
      if (ky == 0 || 2 * ky == ny) {
        out[0] = row[0] + I * row[M];
      } else if (2 * ky < ny) {
        out[0] = row[0];
      } else {
        const cplx* mirror = F + (size_t)nx * ((size_t)(ny - ky) + (size_t)ny * z);
        out[0] = mirror[M];
      }
      for (int j = 1; j < M; ++j) out[j] = row[j];
    }
  free(F);
  return 0;
}

int or_spectral_inverse(int nx, int ny, int nz, const double* s, double* f) {
  if (nx < 2 || nx % 2 != 0 || ny < 1 || nz < 1) return -1;
  size_t n = (size_t)nx * ny * nz;
  int M = nx / 2;
  const cplx* S = (const cplx*)s;
  cplx* F = (cplx*)malloc(sizeof(cplx) * n);
  for (int z = 0; z < nz; ++z)
    for (int ky = 0; ky < ny; ++ky) {
      int kym = (ny - ky) % ny;
      const cplx* in = S + (size_t)M * ((size_t)ky + (size_t)ny * z);
      const cplx* inm = S + (size_t)M * ((size_t)kym + (size_t)ny * z);
      cplx* row = F + (size_t)nx * ((size_t)ky + (size_t)ny * z);
      /* kx = 0 and kx = Nx/2 from the packed slots and Hermitian symmetry */
      if (ky == 0 || 2 * ky == ny) {
        row[0] = creal(in[0]);
        row[M] = cimag(in[0]);
      } else if (2 * ky < ny) {
        row[0] = in[0];           /* slot ky holds F(0, ky) */
        row[M] = inm[0];          /* slot Ny-ky holds F(M, ky) */
      } else {
        row[0] = conj(inm[0]);    /* F(0, ky) = conj F(0, Ny-ky) */
        row[M] = conj(in[0]);     /* slot ky holds F(M, Ny-ky) */
      }
      for (int j = 1; j < M; ++j) row[j] = in[j];
      /* Hermitian symmetry F(-kx,-ky) = conj F(kx,ky) for the other half */
      for (int j = 1; j < M; ++j) row[nx - j] = conj(inm[j]);
    }
  int dims[3] = {nx, ny, nz};
  fft_axis(F, dims, 1, 1);
  fft_axis(F, dims, 0, 1);
  double scale = 1.0 / ((double)nx * (double)ny);
  for (size_t i = 0; i < n; ++i) f[i] = creal(F[i]) * scale;
  free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting (brute-force check).    */
/* ------------------------------------------------------------------------ */

int or_dense_solve(int n, double* A, double* b) {
  if (n < 1) return -1;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
    if (A[(size_t)piv * n + k] == 0.0) return -2;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)piv * n + j];
        A[(size_t)piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      if (l == 0.0) continue;
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * b[j];
    b[k] = s / A[(size_t)k * n + k];
  }
  return 0;
}
