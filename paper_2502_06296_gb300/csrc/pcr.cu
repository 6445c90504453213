// pcr.cu -- z-implicit Helmholtz solve (I - c L_z) u = rhs (Eq. 11) by the
// reworked parallel cyclic reduction of Algorithm 2, Steps 2-4.
//
// A CTA works on tiles of 16 consecutive (x, y) columns x all n rows.  The
// Tensor Memory Accelerator copies a tile into shared memory (boxes of 16
// doubles x <= 256 rows, 128-byte rows) and writes the result back, so the
// kernel never stages data through registers.  Threads: one half-warp per
// z-partition, one lane per column; each thread runs its partition's
// recurrences in shared memory (conflict-free: a half-warp touches one
// 128-byte row).
//   Step 2: forward  d_i -= alpha_i d_{i-1}  (i = 2..m-1),
//           backward d_i -= beta_i  d_{i+1}  (i = m-3..0),
//   Step 3: the 2p boundary unknowns of each column go to a small array;
//           16 lanes of warp 0 solve the reduced tridiagonal systems with the
//           LU factors prepared on the host,
//   Step 4: d_i = ib_i d_i - ap_i x_0 - cp_i x_{m-1}.
// Only the right-hand side changes at run time (the point of Algorithm 2):
// 5 FP64 instructions per unknown, no division.  The coefficients, identical
// for every column, are staged once per CTA and read as broadcasts.  CTAs are
// persistent over tiles; several CTAs per SM overlap one CTA's serial phases
// (copies, the reduced solve) with another's arithmetic.
#include "chanfs_tma.cuh"
#include "chanfs_group.cuh"

namespace chanfs {

constexpr int kPcrCols = 16;  // columns per tile (one half-warp)


// Tiles tile0, tile0 + tstride, ... of one field.  Threads beyond the
// field's 16 * nparts (a grouped launch sized for its widest box) only take
// part in the barriers.
template <class R>
__device__ __forceinline__ void pcr_body(const CUtensorMap* in_map, const CUtensorMap* out_map,
                                         const PcrArgs<R>& a, int* status, long long tile0,
                                         long long tstride) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = a.n, J = 2 * a.nparts;
  const int rows_alloc = a.nbox * a.by;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  R* T = reinterpret_cast<R*>(smem_raw + 128);  // tile [rows_alloc][16]
  R* s_rows = T + rows_alloc * kPcrCols;               // 5n
  R* s_red = s_rows + 5 * n;                           // 3J
  R* s_x = s_red + 3 * J;                              // J x 16

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  for (int e = threadIdx.x; e < 5 * n; e += blockDim.x) s_rows[e] = a.rows[e];
  for (int e = threadIdx.x; e < 3 * J; e += blockDim.x) s_red[e] = a.red[e];
  __syncthreads();
  const R* alpha = s_rows;
  const R* beta = s_rows + n;
  const R* ib = s_rows + 2 * n;
  const R* ap = s_rows + 3 * n;
  const R* cp = s_rows + 4 * n;
  const R* rl = s_red;
  const R* rip = s_red + J;
  const R* ripc = s_red + 2 * J;

  const int c = threadIdx.x % kPcrCols;  // column within the tile
  const int q = threadIdx.x / kPcrCols;  // partition
  const bool part = q < a.nparts;
  // partition q covers rows [q n / p, (q+1) n / p) (the rule the host used)
  const int s = (int)(((long long)q * n) / a.nparts);
  const int m = (int)(((long long)(q + 1) * n) / a.nparts) - s;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  const uint32_t tile_bytes = (uint32_t)(a.nbox * a.by * kPcrCols * sizeof(R));
  uint32_t phase = 0;

  for (long long tile = tile0; tile < ntiles; tile += tstride) {
    const int col0 = (int)(tile * kPcrCols);
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, tile_bytes);
      for (int b = 0; b < a.nbox; ++b)
        tma_load_2d(T + b * a.by * kPcrCols, in_map, bar, col0, b * a.by);
    }
    const int ok = __syncthreads_and(mbar_wait(bar, phase) ? 1 : 0);
    phase ^= 1u;
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, kErrTmaTimeout);
      return;
    }
    R* col = T + c;  // element (row r) at col[r * 16]
    // Step 2: forward then backward reduction of d only
    if (part) {
      R prev = col[(s + 1) * kPcrCols];
      for (int i = 2; i < m; ++i) {
        const int r = s + i;
        prev = fma(-alpha[r], prev, col[r * kPcrCols]);
        col[r * kPcrCols] = prev;
      }
      R next = col[(s + m - 2) * kPcrCols];
      for (int i = m - 3; i >= 0; --i) {
        const int r = s + i;
        next = fma(-beta[r], next, col[r * kPcrCols]);
        col[r * kPcrCols] = next;
      }
      s_x[(2 * q) * kPcrCols + c] = col[s * kPcrCols];
      s_x[(2 * q + 1) * kPcrCols + c] = col[(s + m - 1) * kPcrCols];
    }
    __syncthreads();
    // Step 3: reduced system [x_0^0, x_{m-1}^0, x_0^1, ...], one lane per column
    if (threadIdx.x < kPcrCols) {
      R y = s_x[c];
      for (int jj = 1; jj < J; ++jj) {
        y = fma(-rl[jj], y, s_x[jj * kPcrCols + c]);
        s_x[jj * kPcrCols + c] = y;
      }
      R x = rip[J - 1] * y;
      s_x[(J - 1) * kPcrCols + c] = x;
      for (int jj = J - 2; jj >= 0; --jj) {
        x = fma(-ripc[jj], x, rip[jj] * s_x[jj * kPcrCols + c]);
        s_x[jj * kPcrCols + c] = x;
      }
    }
    __syncthreads();
    // Step 4: reconstruction in place
    if (part) {
      const R x0 = s_x[(2 * q) * kPcrCols + c];
      const R xm = s_x[(2 * q + 1) * kPcrCols + c];
      col[s * kPcrCols] = x0;
      col[(s + m - 1) * kPcrCols] = xm;
      for (int i = 1; i <= m - 2; ++i) {
        const int r = s + i;
        col[r * kPcrCols] = fma(-cp[r], xm, fma(-ap[r], x0, ib[r] * col[r * kPcrCols]));
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int b = 0; b < a.nbox; ++b)
        tma_store_2d(out_map, T + b * a.by * kPcrCols, col0, b * a.by);
      tma_store_commit_and_wait_read();  // the tile may be reused
    }
    if (a.face && threadIdx.x < kPcrCols && col0 + c < a.ncols)
      a.u[(long long)(a.nz - 1) * a.ncols + col0 + c] = R(0);
    __syncthreads();
  }
}

template <class R>
__global__ void __launch_bounds__(1024) pcr_kernel(const __grid_constant__ CUtensorMap in_map,
                                                   const __grid_constant__ CUtensorMap out_map,
                                                   PcrArgs<R> a, int* status) {
  pcr_body<R>(&in_map, &out_map, a, status, blockIdx.x, gridDim.x);
}

// One launch for several boxes (FP32 inner solves of grouped refinement): the
// blocks of box b stride over its tiles.
template <class R>
__global__ void __launch_bounds__(1024) pcr_group_kernel(const PcrBoxT<R>* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const PcrBoxT<R>& x = boxes[b];
  if (threadIdx.x == 0) {  // thread 0 issues the TMA copies
    tensormap_acquire(&x.in_map);
    tensormap_acquire(&x.out_map);
  }
  pcr_body<R>(&x.in_map, &x.out_map, x.a, x.status, blk, x.blocks);
}

// 2-D map over the first n rows of a field: ncols reals per row.
template <class R>
static bool pcr_map(CUtensorMap* map, const void* base, long long ncols, int n, int by) {
  const cuuint64_t gdim[2] = {(cuuint64_t)ncols, (cuuint64_t)n};
  const cuuint64_t gstride[1] = {(cuuint64_t)ncols * sizeof(R)};
  const cuuint32_t box[2] = {(cuuint32_t)kPcrCols, (cuuint32_t)by};
  return encode_map(map, sizeof(R), 2, base, gdim, gstride, box);
}

// Rows per TMA box: at most 256; even for FP32 so that every box starts on a
// 128-byte boundary of the shared tile (16 floats = 64 bytes per row).
static void pcr_boxes(int n, size_t rsize, int* nbox, int* by) {
  *nbox = (n + 255) / 256;
  *by = (n + *nbox - 1) / *nbox;
  if (rsize == 4 && (*by % 2)) ++*by;
}

template <class R>
static size_t pcr_smem_t(int n, int nparts) {
  int nbox, by;
  pcr_boxes(n, sizeof(R), &nbox, &by);
  return 128 + sizeof(R) * ((size_t)nbox * by * kPcrCols + 5 * (size_t)n + 6 * (size_t)nparts +
                            2 * (size_t)nparts * kPcrCols);
}

size_t pcr_smem_bytes(int n, int nparts) { return pcr_smem_t<double>(n, nparts); }

template <class R>
static cudaError_t launch_pcr_t(const cfs_plan* P, const HelmCoef& h, const R* rows, const R* red,
                                const R* rhs, R* u, cudaStream_t st) {
  PcrArgs<R> a;
  a.u = u;
  a.ncols = (long long)P->nx * P->ny;
  a.n = h.n;
  a.nparts = h.nparts;
  a.face = (h.loc == CFS_LOC_FACE);
  a.nz = P->nz;
  pcr_boxes(h.n, sizeof(R), &a.nbox, &a.by);
  a.rows = rows;
  a.red = red;
  CUtensorMap in_map, out_map;
  if (!pcr_map<R>(&in_map, rhs, a.ncols, h.n, a.by) || !pcr_map<R>(&out_map, u, a.ncols, h.n, a.by))
    return cudaErrorInvalidValue;
  const size_t smem = pcr_smem_t<R>(h.n, h.nparts);
  const int threads = kPcrCols * h.nparts;
  auto kern = pcr_kernel<R>;
  allow_max_smem(kern);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  kern<<<(unsigned)grid, threads, smem, st>>>(in_map, out_map, a, P->d_status);
  return cudaGetLastError();
}

cudaError_t launch_pcr(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       cudaStream_t st) {
  return launch_pcr_t<double>(P, h, h.d_rows, h.d_red, rhs, u, st);
}

cudaError_t launch_pcr32(const cfs_plan* P, const HelmCoef& h, const float* rhs, float* u,
                         cudaStream_t st) {
  if (!h.d_rows32) return cudaErrorInvalidValue;
  return launch_pcr_t<float>(P, h, h.d_rows32, h.d_red32, rhs, u, st);
}

// Tiles per block of a grouped launch: enough to amortise the staging of the
// coefficients, few enough to spread a small box over many SMs.
constexpr int kPcrGroupTiles = 8;

template <class R>
static size_t pcr_group_box_t(const cfs_plan* P, const HelmCoef& h, const R* rows, const R* red,
                              const R* rhs, R* u, PcrBoxT<R>* box, int* blocks, int* threads) {
  PcrArgs<R>& a = box->a;
  a.u = u;
  a.ncols = (long long)P->nx * P->ny;
  a.n = h.n;
  a.nparts = h.nparts;
  a.face = (h.loc == CFS_LOC_FACE);
  a.nz = P->nz;
  pcr_boxes(h.n, sizeof(R), &a.nbox, &a.by);
  a.rows = rows;
  a.red = red;
  if (!pcr_map<R>(&box->in_map, rhs, a.ncols, h.n, a.by) ||
      !pcr_map<R>(&box->out_map, u, a.ncols, h.n, a.by))
    return 0;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  box->blocks = (int)((ntiles + kPcrGroupTiles - 1) / kPcrGroupTiles);
  box->status = P->d_status;
  *blocks = box->blocks;
  *threads = kPcrCols * h.nparts;
  return pcr_smem_t<R>(h.n, h.nparts);
}

size_t pcr_group_box(const cfs_plan* P, const HelmCoef& h, PcrBox* box, int* blocks,
                     int* threads) {
  return pcr_group_box_t<float>(P, h, h.d_rows32, h.d_red32, P->d_r32, P->d_r32, box, blocks,
                                threads);
}

size_t pcr_group_box64(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       PcrBox64* box, int* blocks, int* threads) {
  return pcr_group_box_t<double>(P, h, h.d_rows, h.d_red, rhs, u, box, blocks, threads);
}

template <class R>
static cudaError_t launch_pcr_group_t(const PcrBoxT<R>* boxes, GroupMap g, int total,
                                      int threads, size_t smem, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  auto kern = pcr_group_kernel<R>;
  allow_max_smem(kern);
  kern<<<total, threads, smem, st>>>(boxes, g);
  return cudaGetLastError();
}

cudaError_t launch_pcr_group32(const PcrBox* boxes, GroupMap g, int total, int threads,
                               size_t smem, cudaStream_t st) {
  return launch_pcr_group_t<float>(boxes, g, total, threads, smem, st);
}

cudaError_t launch_pcr_group64(const PcrBox64* boxes, GroupMap g, int total, int threads,
                               size_t smem, cudaStream_t st) {
  return launch_pcr_group_t<double>(boxes, g, total, threads, smem, st);
}

}  // namespace chanfs

namespace chanfs {

// Launches the FP64 Algorithm 2 kernel on coefficient arrays given by raw
// device pointers (used by the allocation-free entry point).
cudaError_t launch_pcr_raw(long long ncols, int nz, int n, int nparts, int loc, const double* rows,
                           const double* red, const double* rhs, double* u, int* status,
                           cudaStream_t st) {
  PcrArgs<double> a;
  a.u = u;
  a.ncols = ncols;
  a.n = n;
  a.nparts = nparts;
  a.face = (loc == CFS_LOC_FACE);
  a.nz = nz;
  pcr_boxes(n, sizeof(double), &a.nbox, &a.by);
  a.rows = rows;
  a.red = red;
  CUtensorMap in_map, out_map;
  if (!pcr_map<double>(&in_map, rhs, ncols, n, a.by) ||
      !pcr_map<double>(&out_map, u, ncols, n, a.by))
    return cudaErrorInvalidValue;
  const size_t smem = pcr_smem_t<double>(n, nparts);
  const int threads = kPcrCols * nparts;
  auto kern = pcr_kernel<double>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = (ncols + kPcrCols - 1) / kPcrCols;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  kern<<<(unsigned)grid, threads, smem, st>>>(in_map, out_map, a, status);
  return cudaGetLastError();
}

}  // namespace chanfs
