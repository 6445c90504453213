// chanfs_alg2.cuh -- the z operator's rows and the pre-processing of
// Algorithm 2 (Sec. 2.2.4, Step 1), as plain arithmetic shared by the host
// (plan.cu: cached coefficient sets) and the device (noalloc.cu: the
// allocation-free solve computes its own set on the GPU).  No CUDA API calls.
#ifndef CHANFS_ALG2_CUH
#define CHANFS_ALG2_CUH

#include "../../include/chanfs.h"

namespace chanfs {

// Row k of the staggered second-order z operator L_z (Sec. 2.1), flux form
//   [(q_{k+1} - q_k)/dzc_k - (q_k - q_{k-1})/dzc_{k-1}] / dz_k,
// dzc_k = (dz_k + dz_{k+1})/2, as (lo, diag, hi): the coefficients of q_{k-1},
// q_k and q_{k+1}.  Cell-centred unknowns (nz of them) use mirror ghosts at
// the walls, q_{-1} = +-q_0 (Neumann +, Dirichlet -) one cell width away;
// face-located unknowns (the nz - 1 interior faces) vanish on the walls.
// Couplings through a wall come back as lo = 0 or hi = 0.
__host__ __device__ inline void z_operator_row(int k, int nz, const double* dzf, int bc, int loc,
                                               double* lo, double* diag, double* hi) {
  if (loc == CFS_LOC_CENTER) {
    const double l = (k > 0) ? 1.0 / (dzf[k] * (0.5 * (dzf[k - 1] + dzf[k])))
                             : 1.0 / (dzf[0] * dzf[0]);
    const double h = (k < nz - 1) ? 1.0 / (dzf[k] * (0.5 * (dzf[k] + dzf[k + 1])))
                                  : 1.0 / (dzf[k] * dzf[k]);
    double d = -(l + h);
    if (k == 0) d += (bc == CFS_BC_NEUMANN) ? l : -l;
    if (k == nz - 1) d += (bc == CFS_BC_NEUMANN) ? h : -h;
    *lo = (k > 0) ? l : 0.0;
    *hi = (k < nz - 1) ? h : 0.0;
    *diag = d;
  } else {
    const int n = nz - 1;
    const double dzc = 0.5 * (dzf[k] + dzf[k + 1]);
    const double l = 1.0 / (dzc * dzf[k]);
    const double h = 1.0 / (dzc * dzf[k + 1]);
    *lo = (k > 0) ? l : 0.0;
    *hi = (k < n - 1) ? h : 0.0;
    *diag = -(l + h);
  }
}

// Unknowns of one column of the z-implicit Helmholtz system at location loc.
__host__ __device__ inline int helm_unknowns(int nz, int loc) {
  return loc == CFS_LOC_CENTER ? nz : nz - 1;
}

// Row k of I - c L_z with homogeneous Dirichlet walls (Eq. 11).
__host__ __device__ inline void helm_row(int k, int nz, const double* dzf, int loc, double c,
                                         double* lo, double* diag, double* hi) {
  double l, d, h;
  z_operator_row(k, nz, dzf, CFS_BC_DIRICHLET, loc, &l, &d, &h);
  *lo = -c * l;
  *diag = 1.0 - c * d;
  *hi = -c * h;
}

// The rows of a partition starting at row o, from arrays of the operator's
// (sub, diag, super) coefficients: a row function for alg2_factor_partition.
struct ArrayRows {
  const double* lo;
  const double* diag;
  const double* hi;
  int o;
  __host__ __device__ void operator()(int i, double* l, double* d, double* h) const {
    *l = lo[o + i];
    *d = diag[o + i];
    *h = hi[o + i];
  }
};

// Partition q of p over n rows: [start(q), start(q + 1)).
__host__ __device__ inline int alg2_part_start(int q, int n, int p) {
  return (int)(((long long)q * n) / p);
}

// The automatic partition count: about 32 rows per partition, at most
// max_parts, and every partition at least 3 rows.
__host__ __device__ inline int alg2_auto_parts(int n, int max_parts) {
  int p = (n + 31) / 32;
  if (p > max_parts) p = max_parts;
  if (p < 1) p = 1;
  while (p > 1 && n / p < 3) --p;
  return p;
}

// Step 1 of Algorithm 2 for one partition of m >= 3 rows, derived as two
// eliminations that keep the partition's end unknowns as parameters.
// Row i reads  L_i x_{i-1} + D_i x_i + U_i x_{i+1} = d_i  (x_{-1} and x_m
// belong to the neighbouring partitions); row(i, &L, &D, &U) returns it.
//  * Downward, with x_0 a parameter: row 1 keeps pivot D_1 and x_0 weight L_1;
//    row i >= 2 subtracts f_i = L_i / piv_{i-1} times row i-1, leaving pivot
//    piv_i = D_i - f_i U_{i-1} and x_0 weight g_i = -f_i g_{i-1}.
//  * Upward, with x_{m-1} a parameter: row m-2 couples x_{m-1} with weight
//    h_{m-2} = U_{m-2}; row i = m-3 .. 1 subtracts e_i = U_i / piv_{i+1}
//    times row i+1: g_i -= e_i g_{i+1}, h_i = -e_i h_{i+1}.  Row 0 does the
//    same with row 1: pivot piv_0 = D_0 - e_0 g_1, x_{m-1} weight -e_0 h_1.
// Interior unknowns then follow from the end ones,
//   x_i = (d''_i - g_i x_0 - h_i x_{m-1}) / piv_i,
// and rows 0 and m-1 are the partition's two rows of the reduced system:
//   L_0 x_{-1} + piv_0 x_0 + h_0 x_{m-1}           = d''_0
//   g_{m-1} x_0 + piv_{m-1} x_{m-1} + U_{m-1} x_m  = d'_{m-1}.
// Only the right-hand side changes at run time, so what is stored are the
// multipliers of its two sweeps (alpha_i = f_i for i >= 2, beta_i = e_i for
// i <= m-3, zero elsewhere) and the reconstruction factors ib_i = 1/piv_i,
// ap_i = g_i/piv_i, cp_i = h_i/piv_i (ap_0 = cp_{m-1} = 0: unused).  The
// arrays are the partition's slices; ib, ap and cp hold piv, g and h until
// the last loop.  red_first / red_last receive (sub, diag, super) of the two
// reduced rows.
template <class RowFn>
__host__ __device__ inline void alg2_factor_partition(int m, RowFn row, double* alpha,
                                                      double* beta, double* ib, double* ap,
                                                      double* cp, double red_first[3],
                                                      double red_last[3]) {
  double* piv = ib;
  double* g = ap;
  double* h = cp;
  double L, D, U, U_prev;
  row(1, &L, &D, &U);
  piv[1] = D;
  g[1] = L;
  U_prev = U;
  alpha[0] = alpha[1] = 0.0;
  for (int i = 2; i < m; ++i) {
    row(i, &L, &D, &U);
    const double f = L / piv[i - 1];
    alpha[i] = f;
    piv[i] = D - f * U_prev;
    g[i] = -f * g[i - 1];
    U_prev = U;
  }
  const double U_last = U_prev;  // row m-1's coupling to the next partition
  beta[m - 1] = beta[m - 2] = 0.0;
  row(m - 2, &L, &D, &U);
  h[m - 2] = U;
  h[m - 1] = 0.0;
  for (int i = m - 3; i >= 1; --i) {
    row(i, &L, &D, &U);
    const double e = U / piv[i + 1];
    beta[i] = e;
    g[i] -= e * g[i + 1];
    h[i] = -e * h[i + 1];
  }
  row(0, &L, &D, &U);
  const double e0 = U / piv[1];
  beta[0] = e0;
  piv[0] = D - e0 * g[1];
  g[0] = 0.0;
  h[0] = -e0 * h[1];
  red_first[0] = L;
  red_first[1] = piv[0];
  red_first[2] = h[0];
  red_last[0] = g[m - 1];
  red_last[1] = piv[m - 1];
  red_last[2] = U_last;
  for (int i = 0; i < m; ++i) {
    const double r = 1.0 / piv[i];
    ib[i] = r;
    ap[i] = (i == 0) ? 0.0 : g[i] * r;
    cp[i] = (i == m - 1) ? 0.0 : h[i] * r;
  }
}

// LU without pivoting of the reduced tridiagonal system of size J (Step 3;
// diagonally dominant): sub[j], diag[j], sup[j] of row j.  Stored for the
// run-time solve y_j = b_j - rl_j y_{j-1}, x_j = rip_j y_j - ripc_j x_{j+1}:
// rl_j = sub_j / u_{j-1} (rl_0 = 0), rip_j = 1/u_j, ripc_j = sup_j/u_j with
// the pivots u_0 = diag_0, u_j = diag_j - rl_j sup_{j-1}.
__host__ __device__ inline void alg2_reduced_factor(int J, const double* sub, const double* diag,
                                                    const double* sup, double* rl, double* rip,
                                                    double* ripc) {
  double u = diag[0];
  rl[0] = 0.0;
  rip[0] = 1.0 / u;
  ripc[0] = sup[0] / u;
  for (int j = 1; j < J; ++j) {
    rl[j] = sub[j] / u;
    u = diag[j] - rl[j] * sup[j - 1];
    rip[j] = 1.0 / u;
    ripc[j] = sup[j] / u;
  }
}

// The reduced system solved in parallel instead (Step 3 again): parallel
// cyclic reduction.  At level l (stride s = 2^l) row j takes away s-away rows
// j - s and j + s with the multipliers k1_j = sub_j / diag_{j-s} and
// k2_j = sup_j / diag_{j+s} (zero where the neighbour lies outside), which
// leaves it coupled to rows j -+ 2s only:
//   sub'_j = -k1_j sub_{j-s},  sup'_j = -k2_j sup_{j+s},
//   diag'_j = diag_j - k1_j sup_{j-s} - k2_j sub_{j+s};
// after ceil(log2 J) levels every row is decoupled.  The multipliers depend
// on the matrix only, so they are computed once: k1 at K1[l*J + j], k2 at
// K2[l*J + j], and the final 1/diag_j at ib[j].  At run time a level is
//   y_j <- y_j - k1_j y_{j-s} - k2_j y_{j+s}   (all j at once),
// and x_j = ib_j y_j.  sub, diag, sup are overwritten.
__host__ __device__ inline int alg2_pcr_levels(int J) {
  int l = 0;
  while ((1 << l) < J) ++l;
  return l;
}

__host__ __device__ inline void alg2_reduced_pcr(int J, double* sub, double* diag, double* sup,
                                                 double* na, double* nb, double* nc, double* K1,
                                                 double* K2, double* ib) {
  const int L = alg2_pcr_levels(J);
  for (int l = 0, st = 1; l < L; ++l, st <<= 1) {
    for (int j = 0; j < J; ++j) {
      const bool lo = j - st >= 0, hi = j + st < J;
      const double k1 = lo ? sub[j] / diag[j - st] : 0.0;
      const double k2 = hi ? sup[j] / diag[j + st] : 0.0;
      K1[l * J + j] = k1;
      K2[l * J + j] = k2;
      na[j] = lo ? -k1 * sub[j - st] : 0.0;
      nc[j] = hi ? -k2 * sup[j + st] : 0.0;
      nb[j] = diag[j] - (lo ? k1 * sup[j - st] : 0.0) - (hi ? k2 * sub[j + st] : 0.0);
    }
    for (int j = 0; j < J; ++j) {
      sub[j] = na[j];
      diag[j] = nb[j];
      sup[j] = nc[j];
    }
  }
  for (int j = 0; j < J; ++j) ib[j] = 1.0 / diag[j];
}

}  // namespace chanfs

#endif  // CHANFS_ALG2_CUH
