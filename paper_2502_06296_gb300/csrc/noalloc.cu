// noalloc.cu -- the z-implicit Helmholtz solve of Eq. 11 without any device
// allocation: cfs_helmholtz_solve_noalloc.
//
// cfs_helmholtz_solve keeps its Algorithm 2 coefficients in memory that a
// plan allocates.  Some callers cannot allocate device memory where they
// solve: cudaMalloc and cudaFree synchronise the whole device (stalling every
// other stream in flight), and applications that reserve the device's memory
// up front for their own pool or budget have none left to give.  This entry
// point needs no plan and allocates nothing.  A one-block kernel computes the
// coefficients (Step 1 of Algorithm 2 for every partition, then the LU of the
// reduced system: 5n + 6p doubles for n unknowns and p partitions) on the GPU
// in FP64 from the cell widths, which travel in its kernel parameters, into a
// fixed file-scope device array; the Algorithm 2 kernel of cfs_helmholtz_solve
// then runs on them.  The array holds at most kNoAllocRows = 1024 unknowns and
// kNoAllocParts = 64 partitions (about 44 KB, kept by every GPU that loads the
// library until the process exits).  Nothing is staged on the host, so the
// call queues its work and returns without waiting for the device.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "chanfs_alg2.cuh"
#include "chanfs_internal.cuh"

namespace chanfs {

constexpr int kNoAllocRows = 1024;
constexpr int kNoAllocParts = 64;
// 5n row coefficients + 6p reduced factors
constexpr int kNoAllocDoubles = 5 * kNoAllocRows + 6 * kNoAllocParts;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of the array per device, looked up once per device.
static double* g_scratch_addr[256];
static std::mutex g_scratch_mu;

static int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return CFS_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return CFS_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return CFS_OK;
}

// The cell widths as a kernel parameter (8 KB; copied at launch, so the
// caller's host array is free again when the call returns).
struct NoallocGrid {
  double dzf[kNoAllocRows + 1];
};

// Step 1 of Algorithm 2 (Sec. 2.2.4) for the np partitions of I - c L_z,
// thread q taking partition q, then the LU of the reduced 2np system by
// thread 0: the layout pcr_kernel reads, alpha | beta | ib | ap | cp (n each)
// at rows, then rl | rip | ripc (2np each) at red.
__global__ void __launch_bounds__(kNoAllocParts)
    noalloc_prepare_kernel(const __grid_constant__ NoallocGrid grid, int nz, int n, int np,
                           int loc, double c, double* rows, double* red) {
  __shared__ double ra[2 * kNoAllocParts], rb[2 * kNoAllocParts], rc[2 * kNoAllocParts];
  const int q = threadIdx.x;
  if (q < np) {
    const int o = alg2_part_start(q, n, np);
    const int m = alg2_part_start(q + 1, n, np) - o;
    auto row = [&](int i, double* lo, double* diag, double* hi) {
      helm_row(o + i, nz, grid.dzf, loc, c, lo, diag, hi);
    };
    double first[3], last[3];
    alg2_factor_partition(m, row, rows + o, rows + n + o, rows + 2 * n + o, rows + 3 * n + o,
                          rows + 4 * n + o, first, last);
    ra[2 * q] = first[0];
    rb[2 * q] = first[1];
    rc[2 * q] = first[2];
    ra[2 * q + 1] = last[0];
    rb[2 * q + 1] = last[1];
    rc[2 * q + 1] = last[2];
  }
  __syncthreads();
  if (q == 0) {
    const int J = 2 * np;
    alg2_reduced_factor(J, ra, rb, rc, red, red + J, red + 2 * J);
  }
}

}  // namespace chanfs

using namespace chanfs;

extern "C" int cfs_helmholtz_solve_noalloc(int nx, int ny, int nz, const double* dz, double c,
                                           int loc, int nparts, const double* rhs, double* u,
                                           int* device_status, void* stream) {
  if (!dz || !rhs || !u || !device_status || nx < 1 || ny < 1 || nz < 3) return CFS_EINVAL;
  if ((((uintptr_t)rhs) & 15u) || (((uintptr_t)u) & 15u) || (((uintptr_t)device_status) & 3u))
    return CFS_EINVAL;
  if (!(c >= 0) || !isfinite(c) || (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE)) return CFS_EINVAL;
  if (nparts < 0) return CFS_EINVAL;
  if (((long long)nx * ny) % 2 != 0) return CFS_EUNSUPPORTED;  // 16-byte TMA rows
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !isfinite(dz[k])) return CFS_EINVAL;
  const int n = helm_unknowns(nz, loc);
  if (n > kNoAllocRows || nparts > kNoAllocParts) return CFS_EUNSUPPORTED;
  const int np = nparts ? nparts : alg2_auto_parts(n, kNoAllocParts);
  for (int q = 0; q < np; ++q)
    if (alg2_part_start(q + 1, n, np) - alg2_part_start(q, n, np) < 3) return CFS_EUNSUPPORTED;
  if (pcr_smem_bytes(n, np) > 227 * 1024) return CFS_EUNSUPPORTED;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  NoallocGrid grid;
  for (int k = 0; k < nz; ++k) grid.dzf[k] = dz[k];
  for (int k = nz; k <= kNoAllocRows; ++k) grid.dzf[k] = 0.0;
  double* rows = scratch;
  double* red = scratch + 5 * n;
  // the failure bits start at zero; every coefficient is overwritten below
  cudaError_t e = cudaMemsetAsync(device_status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    noalloc_prepare_kernel<<<1, kNoAllocParts, 0, st>>>(grid, nz, n, np, loc, c, rows, red);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_pcr_raw((long long)nx * ny, nz, n, np, loc, rows, red, rhs, u, device_status, st);
  if (e == cudaErrorInvalidValue) return CFS_EINVAL;
  return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
}
