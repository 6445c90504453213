// noalloc.cu -- the z-implicit Helmholtz solve of Eq. 11 without any device
// allocation: cfs_helmholtz_solve_noalloc.
//
// cfs_helmholtz_solve keeps its Algorithm 2 coefficients in memory that a
// plan allocates.  Some callers cannot allocate device memory where they
// solve: cudaMalloc and cudaFree synchronise the whole device (stalling every
// other stream in flight), and applications that reserve the device's memory
// up front for their own pool or budget have none left to give.  This entry
// point needs no plan and allocates nothing: the coefficients (5n + 6p
// doubles for n unknowns and p partitions) are computed on the host in FP64
// and copied into a fixed file-scope device array, and the same Algorithm 2
// kernel runs on them.  The array holds at most kNoAllocRows = 1024 unknowns
// and kNoAllocParts = 64 partitions (about 44 KB, kept by every GPU that loads
// the library until the process exits).  The host staging buffer is a fixed
// file-scope array too.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "chanfs_internal.cuh"

namespace chanfs {

constexpr int kNoAllocRows = 1024;
constexpr int kNoAllocParts = 64;
// 5n row coefficients + 6p reduced factors, then one status word
constexpr int kNoAllocDoubles = 5 * kNoAllocRows + 6 * kNoAllocParts + 2;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

static double* g_scratch_addr[256];            // device address of the array, per device
static double g_host_coefs[kNoAllocDoubles];  // host staging of the coefficients

// Device address of the scratch array on the current device; the first call
// on a device looks it up (cudaGetSymbolAddress), later calls reuse it.
static int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return CFS_ECUDA;
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return CFS_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return CFS_OK;
}

// Rows of I - c L_z (Sec. 2.1 stencil, homogeneous Dirichlet walls) and
// Algorithm 2 Step 1 for each partition, written into g_host_coefs in the
// layout the kernel reads: alpha | beta | ib | ap | cp (n each) then
// rl | rip | ripc (2p each).  Fixed-size arrays only.
static int noalloc_coefficients(int nz, const double* dzf, double c, int loc, int np, int* n_out) {
  static double A[kNoAllocRows + 1], B[kNoAllocRows + 1], C[kNoAllocRows + 1];
  static double a[kNoAllocRows], b[kNoAllocRows], cc[kNoAllocRows];
  static double ra[2 * kNoAllocParts], rb[2 * kNoAllocParts], rc[2 * kNoAllocParts];
  const int n = (loc == CFS_LOC_CENTER) ? nz : nz - 1;
  if (n < 3 || n > kNoAllocRows) return CFS_EUNSUPPORTED;
  if (np > kNoAllocParts) return CFS_EUNSUPPORTED;
  if (np == 0) {  // the plan's automatic choice: about 32 rows per partition
    np = std::max(1, std::min(kNoAllocParts, (n + 31) / 32));
    while (np > 1 && n / np < 3) --np;
  }
  for (int q = 0; q < np; ++q)
    if ((int)(((long long)(q + 1) * n) / np) - (int)(((long long)q * n) / np) < 3)
      return CFS_EUNSUPPORTED;
  auto dzc = [&](int k) { return 0.5 * (dzf[k] + dzf[k + 1]); };
  for (int k = 0; k < n; ++k) {
    double lo, hi, diag;
    if (loc == CFS_LOC_CENTER) {
      lo = (k > 0) ? 1.0 / (dzf[k] * dzc(k - 1)) : 1.0 / (dzf[0] * dzf[0]);
      hi = (k < nz - 1) ? 1.0 / (dzf[k] * dzc(k)) : 1.0 / (dzf[k] * dzf[k]);
      diag = -(lo + hi);
      if (k == 0) diag -= lo;           // ghost u_{-1} = -u_0
      if (k == nz - 1) diag -= hi;      // ghost u_{nz} = -u_{nz-1}
      if (k == 0) lo = 0.0;
      if (k == nz - 1) hi = 0.0;
    } else {
      lo = 1.0 / (dzc(k) * dzf[k]);
      hi = 1.0 / (dzc(k) * dzf[k + 1]);
      diag = -(lo + hi);
      if (k == 0) lo = 0.0;             // w = 0 on the walls
      if (k == n - 1) hi = 0.0;
    }
    A[k] = -c * lo;
    B[k] = 1.0 - c * diag;
    C[k] = -c * hi;
  }
  double* rows = g_host_coefs;
  double* alpha = rows;
  double* beta = rows + n;
  double* ib = rows + 2 * n;
  double* ap = rows + 3 * n;
  double* cp = rows + 4 * n;
  for (int q = 0; q < np; ++q) {
    const int o = (int)(((long long)q * n) / np);
    const int m = (int)(((long long)(q + 1) * n) / np) - o;
    const double *Aq = A + o, *Bq = B + o, *Cq = C + o;
    double *aq = a + o, *bq = b + o, *cq = cc + o;
    aq[1] = Aq[1];
    bq[1] = Bq[1];
    for (int i = 2; i <= m - 1; ++i) {
      bq[i] = Bq[i] - Aq[i] * Cq[i - 1] / bq[i - 1];
      aq[i] = -Aq[i] * aq[i - 1] / bq[i - 1];
    }
    cq[m - 1] = Cq[m - 1];
    cq[m - 2] = Cq[m - 2];
    for (int i = m - 3; i >= 1; --i) {
      aq[i] = aq[i] - Cq[i] * aq[i + 1] / bq[i + 1];
      cq[i] = -Cq[i] * cq[i + 1] / bq[i + 1];
    }
    aq[0] = Aq[0];
    bq[0] = Bq[0] - Cq[0] * aq[1] / Bq[1];
    cq[0] = -Cq[0] * cq[1] / Bq[1];
    for (int i = 0; i < m; ++i) {
      alpha[o + i] = (i >= 2) ? Aq[i] / bq[i - 1] : 0.0;
      beta[o + i] = (i <= m - 3) ? Cq[i] / bq[i + 1] : 0.0;
      ib[o + i] = 1.0 / bq[i];
      ap[o + i] = aq[i] / bq[i];
      cp[o + i] = cq[i] / bq[i];
    }
    ra[2 * q] = aq[0];
    rb[2 * q] = bq[0];
    rc[2 * q] = cq[0];
    ra[2 * q + 1] = aq[m - 1];
    rb[2 * q + 1] = bq[m - 1];
    rc[2 * q + 1] = cq[m - 1];
  }
  const int J = 2 * np;
  double* rl = rows + 5 * n;
  double* rip = rl + J;
  double* ripc = rip + J;
  double piv = rb[0];
  rl[0] = 0.0;
  rip[0] = 1.0 / piv;
  ripc[0] = rc[0] / piv;
  for (int j = 1; j < J; ++j) {
    rl[j] = ra[j] / piv;
    piv = rb[j] - rl[j] * rc[j - 1];
    rip[j] = 1.0 / piv;
    ripc[j] = rc[j] / piv;
  }
  *n_out = n;
  return np;
}

}  // namespace chanfs

using namespace chanfs;

extern "C" int cfs_helmholtz_solve_noalloc(int nx, int ny, int nz, const double* dz, double c,
                                           int loc, int nparts, const double* rhs, double* u,
                                           void* stream) {
  if (!dz || !rhs || !u || nx < 1 || ny < 1 || nz < 3) return CFS_EINVAL;
  if ((((uintptr_t)rhs) & 15u) || (((uintptr_t)u) & 15u)) return CFS_EINVAL;
  if (!(c >= 0) || !isfinite(c) || (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE)) return CFS_EINVAL;
  if (nparts < 0) return CFS_EINVAL;
  if (((long long)nx * ny) % 2 != 0) return CFS_EUNSUPPORTED;  // 16-byte TMA rows
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !isfinite(dz[k])) return CFS_EINVAL;
  if (nz - (loc == CFS_LOC_FACE ? 1 : 0) > kNoAllocRows) return CFS_EUNSUPPORTED;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  int n = 0;
  const int np = noalloc_coefficients(nz, dz, c, loc, nparts, &n);
  if (np < 0) return np;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ncoef = 5 * (size_t)n + 6 * (size_t)np;
  int* status = reinterpret_cast<int*>(scratch + kNoAllocDoubles - 1);
  // the coefficients are overwritten whole; only the status word starts at 0
  cudaError_t e = cudaMemcpyAsync(scratch, g_host_coefs, sizeof(double) * ncoef,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  // the host staging array is reused by the next call: finish the copy first
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess)
    e = launch_pcr_raw((long long)nx * ny, nz, n, np, loc, scratch, scratch + 5 * n, rhs, u, status,
                       st);
  if (e == cudaErrorInvalidValue) return CFS_EINVAL;
  return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
}
