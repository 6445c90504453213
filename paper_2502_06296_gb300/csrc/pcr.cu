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


// Steps 2-4 of Algorithm 2 on a tile T [rows][16] in shared memory, in place:
// the thread of column threadIdx.x % 16 and partition q (rows s .. s+m-1;
// `part` false for threads beyond the partitions) reduces its right-hand
// side, 16 lanes solve the reduced systems, and every partition is
// reconstructed.  s_x holds the 2p boundary values of each column.  Every
// thread of the CTA calls it (it contains the CTA barriers).
template <class R>
__device__ __forceinline__ void pcr_steps(R* T, R* s_x, const R* s_rows, const R* s_red, int n,
                                          int J, int q, bool part, int s, int m) {
  const R* alpha = s_rows;
  const R* beta = s_rows + n;
  const R* ib = s_rows + 2 * n;
  const R* ap = s_rows + 3 * n;
  const R* cp = s_rows + 4 * n;
  const R* rl = s_red;
  const R* rip = s_red + J;
  const R* ripc = s_red + 2 * J;
  const int c = threadIdx.x % kPcrCols;
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
}

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
    if (!cta_wait(bar, phase, status)) return;
    phase ^= 1u;
    pcr_steps<R>(T, s_x, s_rows, s_red, n, J, q, part, s, m);
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

// ----------------------------------------------------------------------------
// The refined Helmholtz solve in one pass over the field.  The z-implicit
// operator couples only the rows of one (x, y) column, and a tile holds whole
// columns, so iterative refinement runs entirely in shared memory: per tile
//   W = fl32(rhs);  repeat { W = FP32 Algorithm 2 solve of W;  u += W;
//                            r = r - (I - c L_z) W;  W = fl32(r) }
// with r (initially rhs) and u kept as double-float pairs and the operator's
// FP64 rows split into hi + lo, until max|r| <= tol max|rhs| over the tile
// (a bound at least as strict as the same test over the whole field) or
// maxit FP32 solves.  HBM traffic is one FP64 read and one FP64 write per
// point; the only FP64 instruction is the final hi + lo of each u.
// ----------------------------------------------------------------------------

// *slot = max(*slot, v) over the CTA (v >= 0; floats order like their bits).
__device__ __forceinline__ void cta_max_to(float v, unsigned int* slot) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(v));
}

// (bh + bl) - acc as a normalised pair.
__device__ __forceinline__ float2 df_sub(float bh, float bl, const DoubleFloat& acc) {
  float s, t;
  two_sum(bh, -acc.s, s, t);
  const float e = __fadd_rn(t, __fsub_rn(bl, acc.e));
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ void pcr_refine_body(const CUtensorMap* in_map,
                                                const CUtensorMap* out_map,
                                                const PcrRefineArgs& a, int* status,
                                                long long tile0, long long tstride) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int n = a.n, J = 2 * a.nparts;
  const int rows_alloc = a.nbox * a.by;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  // [0] max|rhs|, [1 + (it & 1)] max|r| of pass it (alternating, so that a
  // slot is cleared only after every thread has read it)
  unsigned int* s_max = reinterpret_cast<unsigned int*>(smem_raw + 16);
  double* Rt = reinterpret_cast<double*>(smem_raw + 128);  // [rows_alloc][16]: rhs, r, u
  float2* U = reinterpret_cast<float2*>(Rt + rows_alloc * kPcrCols);  // [n][16] u (hi, lo)
  float* W = reinterpret_cast<float*>(U + n * kPcrCols);             // [n][16] FP32 work
  float* s_rows = W + n * kPcrCols;                                  // 5n
  float* s_red = s_rows + 5 * n;                                     // 3J
  float* s_op = s_red + 3 * J;                                       // 6n: A', B', C' hi, lo
  float* s_x = s_op + 6 * n;                                         // J x 16

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  for (int e = threadIdx.x; e < 5 * n; e += blockDim.x) s_rows[e] = a.rows[e];
  for (int e = threadIdx.x; e < 3 * J; e += blockDim.x) s_red[e] = a.red[e];
  for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
    float hi, lo;
    f64_split(a.abc[e], &hi, &lo);
    s_op[2 * e] = hi;
    s_op[2 * e + 1] = lo;
  }
  __syncthreads();
  const float* opA = s_op;
  const float* opB = s_op + 2 * n;
  const float* opC = s_op + 4 * n;

  const int c = threadIdx.x % kPcrCols;
  const int q = threadIdx.x / kPcrCols;
  const bool part = q < a.nparts;
  const int s = (int)(((long long)q * n) / a.nparts);
  const int m = (int)(((long long)(q + 1) * n) / a.nparts) - s;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  const uint32_t tile_bytes = (uint32_t)(a.nbox * a.by * kPcrCols * sizeof(double));
  uint32_t phase = 0;

  for (long long tile = tile0; tile < ntiles; tile += tstride) {
    const int col0 = (int)(tile * kPcrCols);
    if (threadIdx.x == 0) {
      s_max[0] = s_max[1] = s_max[2] = 0u;
      mbar_expect_tx(bar, tile_bytes);
      for (int b = 0; b < a.nbox; ++b)
        tma_load_2d(Rt + b * a.by * kPcrCols, in_map, bar, col0, b * a.by);
    }
    if (!cta_wait(bar, phase, status)) return;
    phase ^= 1u;
    // the first FP32 right-hand side and the tile's max|rhs|
    float amax = 0.0f;
    if (part)
      for (int i = 0; i < m; ++i) {
        const int e = (s + i) * kPcrCols + c;
        const float h = f64_to_f32(Rt[e]);
        W[e] = h;
        amax = fmaxf(amax, fabsf(h));
      }
    cta_max_to(amax, s_max);
    int it = 0;
    for (;;) {
      pcr_steps<float>(W, s_x, s_rows, s_red, n, J, q, part, s, m);
      __syncthreads();  // every correction of the tile is in W
      // u += delta and r -= (I - c L_z) delta in double-float (on the first
      // pass u = delta and r = rhs - (I - c L_z) delta, rhs split from FP64)
      float rmax = 0.0f;
      if (part)
        for (int i = 0; i < m; ++i) {
          const int r = s + i, e = r * kPcrCols + c;
          const float d = W[e];
          DoubleFloat acc;
          df_acc<true>(acc, opB[2 * r], opB[2 * r + 1], d);
          if (r > 0) df_acc(acc, opA[2 * r], opA[2 * r + 1], W[e - kPcrCols]);
          if (r < n - 1) df_acc(acc, opC[2 * r], opC[2 * r + 1], W[e + kPcrCols]);
          float bh, bl;
          if (it == 0) {
            f64_split(Rt[e], &bh, &bl);
          } else {
            const float2 rb = reinterpret_cast<const float2*>(Rt)[e];
            bh = rb.x;
            bl = rb.y;
          }
          const float2 rn = df_sub(bh, bl, acc);
          reinterpret_cast<float2*>(Rt)[e] = rn;
          rmax = fmaxf(rmax, fabsf(rn.x));
          if (it == 0) {
            U[e] = make_float2(d, 0.0f);
          } else {
            const float2 uo = U[e];
            float us, ut;
            two_sum(uo.x, d, us, ut);
            const float ue = __fadd_rn(uo.y, ut);
            const float uh = __fadd_rn(us, ue);
            U[e] = make_float2(uh, __fsub_rn(ue, __fsub_rn(uh, us)));
          }
        }
      unsigned int* slot = s_max + 1 + (it & 1);
      cta_max_to(rmax, slot);
      __syncthreads();  // the residual is complete; W is free
      ++it;
      const float rm = __uint_as_float(*slot), am = __uint_as_float(s_max[0]);
      if (rm <= a.tol * am || it >= a.maxit) break;  // the same outcome on every thread
      if (part)
        for (int i = 0; i < m; ++i) {
          const int e = (s + i) * kPcrCols + c;
          W[e] = reinterpret_cast<const float2*>(Rt)[e].x;
        }
      // the next pass's slot was last read before this pass's barriers
      if (threadIdx.x == 0) s_max[1 + (it & 1)] = 0u;
      __syncthreads();
    }
    // u = hi + lo in FP64, written over the tile for the store
    if (part)
      for (int i = 0; i < m; ++i) {
        const int e = (s + i) * kPcrCols + c;
        const float2 uo = U[e];
        Rt[e] = f32_to_f64(uo.x) + f32_to_f64(uo.y);
      }
    if (threadIdx.x == 0) {
      atomicMax(a.words, s_max[1 + ((it - 1) & 1)]);
      atomicMax(a.words + 1, s_max[0]);
      atomicMax(a.words + 2, (unsigned int)it);
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int b = 0; b < a.nbox; ++b)
        tma_store_2d(out_map, Rt + b * a.by * kPcrCols, col0, b * a.by);
      tma_store_commit_and_wait_read();  // the tile may be reused
    }
    if (a.face && threadIdx.x < kPcrCols && col0 + c < a.ncols)
      a.u[(long long)(a.nz - 1) * a.ncols + col0 + c] = 0.0;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024)
    pcr_refine_kernel(const __grid_constant__ CUtensorMap in_map,
                      const __grid_constant__ CUtensorMap out_map, PcrRefineArgs a, int* status) {
  pcr_refine_body(&in_map, &out_map, a, status, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024) pcr_refine_group_kernel(const PcrRefineBox* boxes,
                                                                GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const PcrRefineBox& x = boxes[b];
  if (threadIdx.x == 0) {
    tensormap_acquire(&x.in_map);
    tensormap_acquire(&x.out_map);
  }
  pcr_refine_body(&x.in_map, &x.out_map, x.a, x.status, blk, x.blocks);
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

// ---- the refined Helmholtz solve in one pass: host side ---------------------

size_t pcr_refine_smem(int n, int nparts) {
  int nbox, by;
  pcr_boxes(n, sizeof(double), &nbox, &by);
  const size_t J = 2 * (size_t)nparts;
  return 128 + sizeof(double) * (size_t)nbox * by * kPcrCols   // rhs, r, u tile
         + sizeof(float2) * (size_t)n * kPcrCols               // u as (hi, lo)
         + sizeof(float) * (size_t)n * kPcrCols                // FP32 work
         + sizeof(float) * (5 * (size_t)n + 3 * J + 6 * (size_t)n + J * kPcrCols);
}

bool pcr_refine_fits(const cfs_plan* P, const HelmCoef& h) {
  return h.d_rows32 && h.d_abc && !P->helm_thomas32 && pcr_refine_smem(h.n, h.nparts) <= 227 * 1024;
}

static PcrRefineArgs refine_args(const cfs_plan* P, const HelmCoef& h, double* u,
                                 unsigned int* words) {
  PcrRefineArgs a;
  a.u = u;
  a.ncols = (long long)P->nx * P->ny;
  a.n = h.n;
  a.nparts = h.nparts;
  a.nz = P->nz;
  a.face = (h.loc == CFS_LOC_FACE);
  pcr_boxes(h.n, sizeof(double), &a.nbox, &a.by);
  a.maxit = P->maxit;
  a.tol = (float)P->tol;
  a.rows = h.d_rows32;
  a.red = h.d_red32;
  a.abc = h.d_abc;
  a.words = words;
  return a;
}

cudaError_t launch_pcr_refine(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                              unsigned int* words, cudaStream_t st) {
  const PcrRefineArgs a = refine_args(P, h, u, words);
  CUtensorMap in_map, out_map;
  if (!pcr_map<double>(&in_map, rhs, a.ncols, h.n, a.by) ||
      !pcr_map<double>(&out_map, u, a.ncols, h.n, a.by))
    return cudaErrorInvalidValue;
  const size_t smem = pcr_refine_smem(h.n, h.nparts);
  const int threads = kPcrCols * h.nparts;
  cudaError_t e = allow_max_smem(pcr_refine_kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcr_refine_kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  pcr_refine_kernel<<<(unsigned)grid, threads, smem, st>>>(in_map, out_map, a, P->d_status);
  return cudaGetLastError();
}

size_t pcr_refine_group_box(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                            unsigned int* words, PcrRefineBox* box, int* blocks, int* threads) {
  box->a = refine_args(P, h, u, words);
  if (!pcr_map<double>(&box->in_map, rhs, box->a.ncols, h.n, box->a.by) ||
      !pcr_map<double>(&box->out_map, u, box->a.ncols, h.n, box->a.by))
    return 0;
  const long long ntiles = (box->a.ncols + kPcrCols - 1) / kPcrCols;
  box->blocks = (int)((ntiles + kPcrGroupTiles - 1) / kPcrGroupTiles);
  box->status = P->d_status;
  *blocks = box->blocks;
  *threads = kPcrCols * h.nparts;
  return pcr_refine_smem(h.n, h.nparts);
}

cudaError_t launch_pcr_refine_group(const PcrRefineBox* boxes, GroupMap g, int total, int threads,
                                    size_t smem, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  cudaError_t e = allow_max_smem(pcr_refine_group_kernel);
  if (e != cudaSuccess) return e;
  pcr_refine_group_kernel<<<total, threads, smem, st>>>(boxes, g);
  return cudaGetLastError();
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
