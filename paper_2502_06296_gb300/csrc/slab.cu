// slab.cu -- the z-slab decomposition of the paper's parallel tridiagonal
// solver (P-TDMA, Sec. 2.2.3) for several GPUs, one slab per rank.
//
// Each rank holds whole x-y planes [z0, z1) of one field, so the x and y
// transforms stay local.  Along z every (kx, ky) column (Poisson, Eq. 12) or
// every (x, y) column (Helmholtz, Eq. 11) is one tridiagonal system split
// over the ranks, each rank's planes one partition of Algorithm 2
// (Sec. 2.2.4):
//   reduce  Step 2 on the rank's rows: the two boundary values of every
//           column (and, for the singular Neumann column, two partial sums)
//           into a small buffer -- the only data that leaves the GPU;
//   (the caller gathers every rank's buffer, rank-major, e.g. by an NCCL
//    all-gather: 2 values per column per rank, as in the paper's exchange)
//   finish  Step 3 -- the reduced system of the 2 x nranks boundary unknowns
//           of each column, solved redundantly by every rank with LU factors
//           prepared at set-up -- and Step 4, the reconstruction of the
//           rank's rows; then the inverse transforms.
// The reduced systems' coefficients depend on the operator only, so every
// rank computes those of all ranks itself at set-up instead of receiving them
// (the paper does the same for the implicit diffusion; for the Poisson
// equation they are time-invariant, Sec. 2.2.4).  The set-up runs on the host
// in FP64 with the elimination of chanfs_alg2.cuh that the plans use.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "chanfs_alg2.cuh"
#include "chanfs_internal.cuh"

namespace chanfs {

constexpr int kSlabBlock = 128;

struct SlabHelm {
  double c;
  int loc;
  int nloc;        // rows of this rank (face fields: the top wall excluded)
  double* d_rows;  // alpha | beta | ib | ap | cp of the rank's rows (5 nloc)
  double* d_lu;    // rl | rip | ripc of the reduced system (3 * 2 nranks)
};

}  // namespace chanfs

using namespace chanfs;

struct cfs_slab {
  int rank, nranks, z0, z1, nzl, nz, nx, ny, M, nky, bc, has_null;
  cfs_plan_t plan = nullptr;   // the local planes' x and y transforms
  double* d_pf = nullptr;      // Poisson factors [5][nzl][nky][M+1], ib scaled by s
  double* d_plu = nullptr;     // reduced LU [3][J][nky][M+1], rip scaled by s
  double* d_sing = nullptr;    // Neumann (0,0): wn | gn | hs over the rank's rows
  double sing_cg = 0.0, sing_sc = 0.0;
  std::vector<double> dz;       // the global cell widths
  std::vector<SlabHelm> helm;
  size_t device_bytes = 0;
};

namespace {

template <typename T>
int upload(T** dst, const std::vector<T>& src, size_t* acc) {
  if (cudaMalloc(dst, sizeof(T) * src.size()) != cudaSuccess) return CFS_ENOMEM;
  *acc += sizeof(T) * src.size();
  if (cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return CFS_ECUDA;
  return CFS_OK;
}

// Thomas algorithm on the host (FP64): a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k.
void thomas_solve(const std::vector<double>& a, const std::vector<double>& b,
                  const std::vector<double>& c, const std::vector<double>& d,
                  std::vector<double>& x) {
  const int n = (int)b.size();
  std::vector<double> cp(n), dp(n);
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    const double piv = b[k] - a[k] * cp[k - 1];
    cp[k] = c[k] / piv;
    dp[k] = (d[k] - a[k] * dp[k - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
}

// Algorithm 2 Step 1 for every partition of one system (rows[k] = (L, D, U)
// of global row k, n rows, partition q = rows [start[q], start[q+1])): the
// factors of partition `own` into own_rows (5 m, alpha | beta | ib | ap | cp)
// and the LU of the reduced system into lu (rl | rip | ripc, 3 J).
void slab_factors(int n, const double* L, const double* D, const double* U, const int* start,
                  int nparts, int own, double* own_rows, double* lu) {
  const int J = 2 * nparts;
  std::vector<double> ra(J), rb(J), rc(J), tmp;
  for (int q = 0; q < nparts; ++q) {
    const int o = start[q], m = start[q + 1] - o;
    tmp.assign(5 * (size_t)m, 0.0);
    double* dst = (q == own) ? own_rows : tmp.data();
    const ArrayRows row{L, D, U, o};
    double first[3], last[3];
    alg2_factor_partition(m, row, dst, dst + m, dst + 2 * m, dst + 3 * m, dst + 4 * m, first, last);
    ra[2 * q] = first[0];
    rb[2 * q] = first[1];
    rc[2 * q] = first[2];
    ra[2 * q + 1] = last[0];
    rb[2 * q + 1] = last[1];
    rc[2 * q + 1] = last[2];
  }
  (void)n;
  alg2_reduced_factor(J, ra.data(), rb.data(), rc.data(), lu, lu + J, lu + 2 * J);
}

// Partition starts of nz rows over nranks (the plans' rule).
std::vector<int> starts_of(int n, int nranks) {
  std::vector<int> s(nranks + 1);
  for (int q = 0; q <= nranks; ++q) s[q] = alg2_part_start(q, n, nranks);
  return s;
}

}  // namespace

namespace chanfs {

// Factor sets of the real and imaginary parts of spectrum slot (ky, j) of a
// periodic-y spectrum (App. A packing; column j = 0 untangled along y): the
// offsets kyp * (M + 1) + kx of their wavenumbers in the factor tables.
__device__ __forceinline__ void slot_sets(int ky, int j, int M, int ny, int* ox, int* oy) {
  int kx_x = j, kx_y = j, kp;
  if (j > 0) {
    kp = min(ky, ny - ky);
  } else if (2 * ky == 0 || 2 * ky == ny) {  // real pair F(0, ky) + i F(M, ky)
    kp = ky;
    kx_y = M;
  } else if (2 * ky < ny) {  // F(0, ky)
    kp = ky;
  } else {  // F(M, Ny - ky)
    kx_x = kx_y = M;
    kp = ny - ky;
  }
  *ox = kp * (M + 1) + kx_x;
  *oy = kp * (M + 1) + kx_y;
}

struct SlabArgs {
  double2* S;            // local spectrum, (nzl, ny, M) complex
  const double* pf;      // [5][nzl][ncp]
  const double* plu;     // [3][J][ncp]
  const double* sing;    // wn | gn | hs over the local rows
  double sing_cg, sing_sc;
  int M, ny, nzl, ncp, J, rank, neumann, z0;
};

// Step 2 on the rank's rows of every spectrum column; boundary values to bnd
// ([2][ny][M] complex), the singular column's partial sums to bnd's tail.
__global__ void __launch_bounds__(kSlabBlock) slab_poisson_reduce_kernel(SlabArgs a, double2* bnd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  if (j >= a.M) return;
  int ox, oy;
  slot_sets(ky, j, a.M, a.ny, &ox, &oy);
  const long long rs = (long long)a.ny * a.M;
  double2* col = a.S + (long long)ky * a.M + j;
  const double* alpha = a.pf;
  const double* beta = a.pf + (long long)a.nzl * a.ncp;
  const int m = a.nzl;
  const bool sing = a.neumann && j == 0 && ky == 0;
  if (sing) {  // the Neumann (0, 0) column, real part: partial sums, pinned row
    double mu = 0.0, gam = 0.0;
    for (int i = 0; i < m; ++i) {
      const double e = col[i * rs].x;
      mu = fma(a.sing[i], e, mu);
      if (a.z0 + i > 0) gam = fma(a.sing[m + i], e, gam);
    }
    double* tail = reinterpret_cast<double*>(bnd + 2LL * a.ny * a.M);
    tail[0] = mu;
    tail[1] = gam;
    if (a.z0 == 0) col[0].x = 0.0;  // global row 0 is pinned (F_0 = 0)
  }
  double2 prev = col[rs];
  for (int i = 2; i < m; ++i) {
    const long long t = (long long)i * a.ncp;
    double2 v = col[i * rs];
    v.x = fma(-alpha[t + ox], prev.x, v.x);
    v.y = fma(-alpha[t + oy], prev.y, v.y);
    col[i * rs] = v;
    prev = v;
  }
  double2 next = col[(m - 2) * rs];
  for (int i = m - 3; i >= 0; --i) {
    const long long t = (long long)i * a.ncp;
    double2 v = col[i * rs];
    v.x = fma(-beta[t + ox], next.x, v.x);
    v.y = fma(-beta[t + oy], next.y, v.y);
    col[i * rs] = v;
    next = v;
  }
  bnd[(long long)ky * a.M + j] = col[0];
  bnd[(long long)(a.ny + ky) * a.M + j] = col[(m - 1) * rs];
}

// One part (x or y) of a column's reduced system: rhs from every rank's
// boundary buffer, LU factors at offset o; returns this rank's two values.
__device__ __forceinline__ void slab_reduced_part(const SlabArgs& a, const double2* bnd_all,
                                                  long long per_rank, long long slot, int o,
                                                  bool imag, double* x0, double* xm) {
  const double* rl = a.plu;
  const double* rip = a.plu + (long long)a.J * a.ncp;
  const double* ripc = a.plu + 2LL * a.J * a.ncp;
  double y[2 * 64];  // the reduced system has 2 nranks <= 128 rows
  for (int jj = 0; jj < a.J; ++jj) {
    const int r = jj >> 1, t = jj & 1;
    const double2 v = bnd_all[r * per_rank + (long long)t * a.ny * a.M + slot];
    const double b = imag ? v.y : v.x;
    y[jj] = jj == 0 ? b : fma(-rl[(long long)jj * a.ncp + o], y[jj - 1], b);
  }
  double x = rip[(long long)(a.J - 1) * a.ncp + o] * y[a.J - 1];
  y[a.J - 1] = x;
  for (int jj = a.J - 2; jj >= 0; --jj) {
    x = fma(-ripc[(long long)jj * a.ncp + o], x, rip[(long long)jj * a.ncp + o] * y[jj]);
    y[jj] = x;
  }
  *x0 = y[2 * a.rank];
  *xm = y[2 * a.rank + 1];
}

// Steps 3 and 4 for every spectrum column of the rank, scaled by s (folded
// into the factors), the singular column's projections applied.
__global__ void __launch_bounds__(kSlabBlock) slab_poisson_finish_kernel(SlabArgs a,
                                                                         const double2* bnd_all,
                                                                         long long per_rank) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, ky = blockIdx.y;
  if (j >= a.M) return;
  int ox, oy;
  slot_sets(ky, j, a.M, a.ny, &ox, &oy);
  const long long slot = (long long)ky * a.M + j;
  double x0x, xmx, x0y, xmy;
  slab_reduced_part(a, bnd_all, per_rank, slot, ox, false, &x0x, &xmx);
  slab_reduced_part(a, bnd_all, per_rank, slot, oy, true, &x0y, &xmy);
  const long long rs = (long long)a.ny * a.M;
  double2* col = a.S + slot;
  const int m = a.nzl;
  const double* ib = a.pf + 2LL * m * a.ncp;
  const double* ap = a.pf + 3LL * m * a.ncp;
  const double* cp = a.pf + 4LL * m * a.ncp;
  col[0] = make_double2(x0x, x0y);
  col[(m - 1) * rs] = make_double2(xmx, xmy);
  for (int i = 1; i < m - 1; ++i) {
    const long long t = (long long)i * a.ncp;
    const double2 v = col[i * rs];
    col[i * rs] = make_double2(
        fma(-cp[t + ox], xmx, fma(-ap[t + ox], x0x, ib[t + ox] * v.x)),
        fma(-cp[t + oy], xmy, fma(-ap[t + oy], x0y, ib[t + oy] * v.y)));
  }
  if (a.neumann && j == 0 && ky == 0) {  // x - mu h - nu, from every rank's partial sums
    double mu = 0.0, gam = 0.0;
    for (int r = 0; r < a.J / 2; ++r) {
      const double* tail = reinterpret_cast<const double*>(bnd_all + r * per_rank +
                                                           2LL * a.ny * a.M);
      mu += tail[0];
      gam += tail[1];
    }
    const double nu = a.sing_sc * (gam - mu * a.sing_cg);
    for (int i = 0; i < m; ++i) col[i * rs].x -= fma(mu, a.sing[2 * m + i], nu);
  }
}

struct SlabHelmArgs {
  double* W;            // local field (nloc rows of ncols)
  const double* rows;   // alpha | beta | ib | ap | cp (5 nloc)
  const double* lu;     // rl | rip | ripc (3 J)
  long long ncols;
  int nloc, J, rank;
};

__global__ void __launch_bounds__(kSlabBlock) slab_helm_reduce_kernel(SlabHelmArgs a,
                                                                      const double* rhs,
                                                                      double* bnd) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.ncols) return;
  const int m = a.nloc;
  const double* alpha = a.rows;
  const double* beta = a.rows + m;
  double prev = rhs[a.ncols + col];
  a.W[col] = rhs[col];
  a.W[a.ncols + col] = prev;
  for (int i = 2; i < m; ++i) {
    prev = fma(-alpha[i], prev, rhs[i * a.ncols + col]);
    a.W[i * a.ncols + col] = prev;
  }
  double next = a.W[(m - 2) * a.ncols + col];
  for (int i = m - 3; i >= 0; --i) {
    next = fma(-beta[i], next, a.W[i * a.ncols + col]);
    a.W[i * a.ncols + col] = next;
  }
  bnd[col] = a.W[col];
  bnd[a.ncols + col] = a.W[(m - 1) * a.ncols + col];
}

__global__ void __launch_bounds__(kSlabBlock) slab_helm_finish_kernel(SlabHelmArgs a,
                                                                      const double* bnd_all,
                                                                      long long per_rank,
                                                                      double* u, int zero_top,
                                                                      int nzl) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.ncols) return;
  const double* rl = a.lu;
  const double* rip = a.lu + a.J;
  const double* ripc = a.lu + 2 * a.J;
  double y[2 * 64];
  for (int jj = 0; jj < a.J; ++jj) {
    const double b = bnd_all[(jj >> 1) * per_rank + (long long)(jj & 1) * a.ncols + col];
    y[jj] = jj == 0 ? b : fma(-rl[jj], y[jj - 1], b);
  }
  double x = rip[a.J - 1] * y[a.J - 1];
  y[a.J - 1] = x;
  for (int jj = a.J - 2; jj >= 0; --jj) {
    x = fma(-ripc[jj], x, rip[jj] * y[jj]);
    y[jj] = x;
  }
  const double x0 = y[2 * a.rank], xm = y[2 * a.rank + 1];
  const int m = a.nloc;
  const double* ib = a.rows + 2 * m;
  const double* ap = a.rows + 3 * m;
  const double* cp = a.rows + 4 * m;
  u[col] = x0;
  for (int i = 1; i < m - 1; ++i)
    u[i * a.ncols + col] = fma(-cp[i], xm, fma(-ap[i], x0, ib[i] * a.W[i * a.ncols + col]));
  u[(m - 1) * a.ncols + col] = xm;
  if (zero_top) u[(long long)(nzl - 1) * a.ncols + col] = 0.0;  // the top wall of a face field
}

}  // namespace chanfs

// ----------------------------------------------------------------------------
// Public ABI
// ----------------------------------------------------------------------------
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
static int cuda_rc(cudaError_t e) {
  return e == cudaSuccess ? CFS_OK : (e == cudaErrorInvalidValue ? CFS_EINVAL : CFS_ECUDA);
}

extern "C" int cfs_slab_partition(int nz, int nranks, int rank, int* z0, int* z1) {
  if (!z0 || !z1 || nranks < 1 || nranks > 64 || rank < 0 || rank >= nranks || nz < 3)
    return CFS_EINVAL;
  *z0 = alg2_part_start(rank, nz, nranks);
  *z1 = alg2_part_start(rank + 1, nz, nranks);
  return CFS_OK;
}

static void slab_free(cfs_slab* S) {
  if (!S) return;
  if (S->plan) cfs_plan_destroy(S->plan);
  cudaFree(S->d_pf);
  cudaFree(S->d_plu);
  cudaFree(S->d_sing);
  for (SlabHelm& h : S->helm) {
    cudaFree(h.d_rows);
    cudaFree(h.d_lu);
  }
  delete S;
}

extern "C" int cfs_slab_create(cfs_slab_t* out, int nx, int ny, int nz, double lx, double ly,
                               const double* dz, int poisson_bc, int nranks, int rank) {
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (!dz || nz < 3 || nranks < 1 || nranks > 64 || rank < 0 || rank >= nranks) return CFS_EINVAL;
  if (poisson_bc != CFS_BC_NEUMANN && poisson_bc != CFS_BC_DIRICHLET) return CFS_EINVAL;
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !isfinite(dz[k])) return CFS_EINVAL;
  const std::vector<int> st = starts_of(nz, nranks);
  for (int q = 0; q < nranks; ++q)  // every partition 3 rows at least (the face fields' 4)
    if (st[q + 1] - st[q] < 4) return CFS_EUNSUPPORTED;
  cfs_slab* S = new (std::nothrow) cfs_slab();
  if (!S) return CFS_ENOMEM;
  S->rank = rank;
  S->nranks = nranks;
  S->nz = nz;
  S->nx = nx;
  S->ny = ny;
  S->z0 = st[rank];
  S->z1 = st[rank + 1];
  S->nzl = S->z1 - S->z0;
  S->bc = poisson_bc;
  S->dz.assign(dz, dz + nz);
  std::vector<double> dzl(dz + S->z0, dz + S->z1);
  int rc = cfs_plan_create(&S->plan, nx, ny, S->nzl, lx, ly, dzl.data(), poisson_bc, CFS_F64);
  if (rc) {
    slab_free(S);
    return rc;
  }
  if (S->plan->ybc != CFS_Y_PERIODIC) {
    slab_free(S);
    return CFS_EUNSUPPORTED;
  }
  S->M = S->plan->M;
  S->nky = S->plan->nky;
  S->has_null = (poisson_bc == CFS_BC_NEUMANN);
  const int M = S->M, nky = S->nky, m = S->nzl, J = 2 * nranks;
  const size_t ncp = (size_t)(M + 1) * nky;
  // the global z operator (Eq. 12 without the wavenumbers)
  std::vector<double> A(nz), B(nz), C(nz);
  for (int k = 0; k < nz; ++k) z_operator_row(k, nz, dz, poisson_bc, CFS_LOC_CENTER, &A[k], &B[k], &C[k]);
  const double s = 2.0 / ((double)nx * (double)ny);
  // per wavenumber pair: Step 1 over every partition, this rank's factors
  // kept, the reduced LU (s folded into ib and rip)
  std::vector<double> pf(5 * (size_t)m * ncp), plu(3 * (size_t)J * ncp);
  std::vector<double> Dk(nz), own(5 * (size_t)m), lu(3 * (size_t)J), L0(A), U0(C);
  for (int kyp = 0; kyp < nky; ++kyp)
    for (int kx = 0; kx <= M; ++kx) {
      const double lam = S->plan->lamx_h[kx] + S->plan->lamy_h[kyp];
      for (int k = 0; k < nz; ++k) Dk[k] = B[k] + lam;
      const bool pin = S->has_null && kx == 0 && kyp == 0;
      L0[0] = A[0];
      U0[0] = C[0];
      if (pin) {  // row 0 -> F_0 = 0
        Dk[0] = 1.0;
        U0[0] = 0.0;
      }
      slab_factors(nz, L0.data(), Dk.data(), U0.data(), st.data(), nranks, rank, own.data(),
                   lu.data());
      const size_t o = (size_t)kyp * (M + 1) + kx;
      for (int f = 0; f < 5; ++f)
        for (int i = 0; i < m; ++i)
          pf[((size_t)f * m + i) * ncp + o] = own[(size_t)f * m + i] * (f == 2 ? s : 1.0);
      for (int f = 0; f < 3; ++f)
        for (int jj = 0; jj < J; ++jj)
          plu[((size_t)f * J + jj) * ncp + o] = lu[(size_t)f * J + jj] * (f == 1 ? s : 1.0);
    }
  // Neumann (0,0): h = T'^{-1} (0,1,..,1), g = T'^{-T} w over the whole column
  std::vector<double> sing(3 * (size_t)m, 0.0);
  S->sing_sc = s;
  if (S->has_null) {
    std::vector<double> a(A), b(B), c(C), rhs(nz, 1.0), h(nz), g(nz), w(dz, dz + nz);
    b[0] = 1.0;
    c[0] = 0.0;
    rhs[0] = 0.0;
    thomas_solve(a, b, c, rhs, h);
    std::vector<double> at(nz, 0.0), ct(nz, 0.0);
    for (int k = 1; k < nz; ++k) at[k] = c[k - 1];
    for (int k = 0; k + 1 < nz; ++k) ct[k] = a[k + 1];
    thomas_solve(at, b, ct, w, g);
    double sw = 0.0;
    for (int k = 0; k < nz; ++k) sw += dz[k];
    for (int i = 0; i < m; ++i) {
      sing[i] = dz[S->z0 + i] / sw;
      sing[m + i] = g[S->z0 + i] / sw;
      sing[2 * m + i] = s * h[S->z0 + i];
    }
    for (int k = 1; k < nz; ++k) S->sing_cg += g[k];
    S->sing_cg /= sw;
  }
  rc = upload(&S->d_pf, pf, &S->device_bytes);
  if (!rc) rc = upload(&S->d_plu, plu, &S->device_bytes);
  if (!rc) rc = upload(&S->d_sing, sing, &S->device_bytes);
  if (rc) {
    slab_free(S);
    return rc;
  }
  *out = S;
  return CFS_OK;
}

extern "C" int cfs_slab_destroy(cfs_slab_t S) {
  if (!S) return CFS_EINVAL;
  cudaDeviceSynchronize();
  slab_free(S);
  return CFS_OK;
}

extern "C" int cfs_slab_extent(cfs_slab_t S, int* z0, int* z1) {
  if (!S || !z0 || !z1) return CFS_EINVAL;
  *z0 = S->z0;
  *z1 = S->z1;
  return CFS_OK;
}

extern "C" int cfs_slab_boundary_doubles(cfs_slab_t S, int kind, size_t* count) {
  if (!S || !count) return CFS_EINVAL;
  if (kind == CFS_REQ_POISSON) *count = 4 * (size_t)S->ny * S->M + 2;
  else if (kind == CFS_REQ_HELMHOLTZ) *count = 2 * (size_t)S->nx * S->ny;
  else return CFS_EINVAL;
  return CFS_OK;
}

static SlabArgs slab_args(const cfs_slab* S, double* work) {
  SlabArgs a;
  a.S = reinterpret_cast<double2*>(work);
  a.pf = S->d_pf;
  a.plu = S->d_plu;
  a.sing = S->d_sing;
  a.sing_cg = S->sing_cg;
  a.sing_sc = S->sing_sc;
  a.M = S->M;
  a.ny = S->ny;
  a.nzl = S->nzl;
  a.ncp = (S->M + 1) * S->nky;
  a.J = 2 * S->nranks;
  a.rank = S->rank;
  a.neumann = S->has_null;
  a.z0 = S->z0;
  return a;
}

extern "C" int cfs_slab_poisson_reduce(cfs_slab_t S, const double* f, double* work, double* bnd,
                                       void* stream) {
  if (!S || !f || !work || !bnd || !aligned16(f) || !aligned16(work) || !aligned16(bnd))
    return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_rfft_x(S->plan, f, work, false, 1.0, st);
  if (e == cudaSuccess) e = launch_fft_y(S->plan, work, false, st);
  if (e == cudaSuccess) {
    dim3 grid((S->M + kSlabBlock - 1) / kSlabBlock, S->ny);
    slab_poisson_reduce_kernel<<<grid, kSlabBlock, 0, st>>>(slab_args(S, work),
                                                            reinterpret_cast<double2*>(bnd));
    e = cudaGetLastError();
  }
  return cuda_rc(e);
}

extern "C" int cfs_slab_poisson_finish(cfs_slab_t S, const double* bnd_all, double* work,
                                       double* p, void* stream) {
  if (!S || !bnd_all || !work || !p || !aligned16(bnd_all) || !aligned16(work) || !aligned16(p))
    return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  size_t per = 0;
  cfs_slab_boundary_doubles(S, CFS_REQ_POISSON, &per);
  dim3 grid((S->M + kSlabBlock - 1) / kSlabBlock, S->ny);
  slab_poisson_finish_kernel<<<grid, kSlabBlock, 0, st>>>(
      slab_args(S, work), reinterpret_cast<const double2*>(bnd_all), (long long)(per / 2));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_fft_y(S->plan, work, true, st);
  if (e == cudaSuccess) e = launch_rfft_x(S->plan, work, p, true, 1.0, st);
  return cuda_rc(e);
}

// The Helmholtz set (c, loc) of the rank: Step 1 of every partition of the
// global I - c L_z, computed on the host and cached.
static int slab_helm(cfs_slab* S, double c, int loc, SlabHelm** out) {
  if (!(c >= 0) || !isfinite(c) || (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE))
    return CFS_EINVAL;
  for (SlabHelm& h : S->helm)
    if (h.c == c && h.loc == loc) {
      *out = &h;
      return CFS_OK;
    }
  const int n = helm_unknowns(S->nz, loc), R = S->nranks, J = 2 * R;
  std::vector<int> st = starts_of(S->nz, R);
  st[R] = n;  // a face field's last partition ends below the top wall
  if (st[R] - st[R - 1] < 3) return CFS_EUNSUPPORTED;
  std::vector<double> L(n), D(n), U(n);
  for (int k = 0; k < n; ++k) helm_row(k, S->nz, S->dz.data(), loc, c, &L[k], &D[k], &U[k]);
  const int m = st[S->rank + 1] - st[S->rank];
  std::vector<double> own(5 * (size_t)m), lu(3 * (size_t)J);
  slab_factors(n, L.data(), D.data(), U.data(), st.data(), R, S->rank, own.data(), lu.data());
  SlabHelm h;
  h.c = c;
  h.loc = loc;
  h.nloc = m;
  h.d_rows = nullptr;
  h.d_lu = nullptr;
  int rc = upload(&h.d_rows, own, &S->device_bytes);
  if (!rc) rc = upload(&h.d_lu, lu, &S->device_bytes);
  if (rc) {
    cudaFree(h.d_rows);
    cudaFree(h.d_lu);
    return rc;
  }
  S->helm.push_back(h);
  *out = &S->helm.back();
  return CFS_OK;
}

static SlabHelmArgs helm_args(const cfs_slab* S, const SlabHelm& h, double* work) {
  SlabHelmArgs a;
  a.W = work;
  a.rows = h.d_rows;
  a.lu = h.d_lu;
  a.ncols = (long long)S->nx * S->ny;
  a.nloc = h.nloc;
  a.J = 2 * S->nranks;
  a.rank = S->rank;
  return a;
}

extern "C" int cfs_slab_helmholtz_reduce(cfs_slab_t S, double c, int loc, const double* rhs,
                                         double* work, double* bnd, void* stream) {
  if (!S || !rhs || !work || !bnd || rhs == work) return CFS_EINVAL;
  SlabHelm* h = nullptr;
  int rc = slab_helm(S, c, loc, &h);
  if (rc) return rc;
  const SlabHelmArgs a = helm_args(S, *h, work);
  const unsigned grid = (unsigned)((a.ncols + kSlabBlock - 1) / kSlabBlock);
  slab_helm_reduce_kernel<<<grid, kSlabBlock, 0, (cudaStream_t)stream>>>(a, rhs, bnd);
  return cuda_rc(cudaGetLastError());
}

extern "C" int cfs_slab_helmholtz_finish(cfs_slab_t S, double c, int loc, const double* bnd_all,
                                         const double* work, double* u, void* stream) {
  if (!S || !bnd_all || !work || !u || work == u) return CFS_EINVAL;
  SlabHelm* h = nullptr;
  int rc = slab_helm(S, c, loc, &h);
  if (rc) return rc;
  const SlabHelmArgs a = helm_args(S, *h, const_cast<double*>(work));
  const unsigned grid = (unsigned)((a.ncols + kSlabBlock - 1) / kSlabBlock);
  const int zero_top = (loc == CFS_LOC_FACE && S->rank == S->nranks - 1);
  slab_helm_finish_kernel<<<grid, kSlabBlock, 0, (cudaStream_t)stream>>>(
      a, bnd_all, 2 * a.ncols, u, zero_top, S->nzl);
  return cuda_rc(cudaGetLastError());
}
