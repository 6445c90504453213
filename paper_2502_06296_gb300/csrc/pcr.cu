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
#include "chanfs_alg2.cuh"
#include "chanfs_tma.cuh"
#include "chanfs_group.cuh"

namespace chanfs {

constexpr int kPcrCols = kPcrTileColumns;  // columns per tile (one half-warp)


// Steps 2-4 of Algorithm 2 on a tile T [rows][16] in shared memory, in place:
// the thread of column threadIdx.x % 16 and partition q (rows s .. s+m-1;
// `part` false for threads beyond the partitions) reduces its right-hand
// side (Step 2), 16 lanes solve the reduced systems (Step 3), and every
// partition is reconstructed (Step 4).  s_x holds the 2p boundary values of
// each column, [2p][16].
template <class R>
__device__ __forceinline__ void pcr_step2(R* T, R* s_x, const R* s_rows, int n, int q, bool part,
                                          int s, int m) {
  const R* alpha = s_rows;
  const R* beta = s_rows + n;
  const int c = threadIdx.x % kPcrCols;
  R* col = T + c;  // element (row r) at col[r * 16]
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
}

// Step 3 by the LU factors of the reduced system, one lane per column.
template <class R>
__device__ __forceinline__ void pcr_step3_lu(R* s_x, const R* s_red, int J) {
  const R* rl = s_red;
  const R* rip = s_red + J;
  const R* ripc = s_red + 2 * J;
  const int c = threadIdx.x % kPcrCols;
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
}

template <class R>
__device__ __forceinline__ void pcr_step4(R* T, const R* s_x, const R* s_rows, int n, int q,
                                          bool part, int s, int m) {
  const R* ib = s_rows + 2 * n;
  const R* ap = s_rows + 3 * n;
  const R* cp = s_rows + 4 * n;
  const int c = threadIdx.x % kPcrCols;
  R* col = T + c;
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

// Every thread of the CTA calls it (it contains the CTA barriers).
template <class R>
__device__ __forceinline__ void pcr_steps(R* T, R* s_x, const R* s_rows, const R* s_red, int n,
                                          int J, int q, bool part, int s, int m) {
  pcr_step2<R>(T, s_x, s_rows, n, q, part, s, m);
  __syncthreads();
  pcr_step3_lu<R>(s_x, s_red, J);
  __syncthreads();
  pcr_step4<R>(T, s_x, s_rows, n, q, part, s, m);
}

// Step 3 by parallel cyclic reduction with the precomputed multipliers
// (K1 | K2 | 1/diag, see alg2_reduced_pcr), every thread of the CTA taking
// (row, column) items of the 2p x 16 boundary values; ping-pong between s_x
// and s_y.  The solution ends in s_x.  Contains CTA barriers.
__device__ __forceinline__ void pcr_step3_pcr(float* s_x, float* s_y, const float* s_lv, int J,
                                              int L) {
  const float* K1 = s_lv;
  const float* K2 = s_lv + L * J;
  const float* ib = s_lv + 2 * L * J;
  const int items = J * kPcrCols;
  float* a = s_x;
  float* b = s_y;
  for (int l = 0, st = 1; l < L; ++l, st <<= 1) {
    for (int e = threadIdx.x; e < items; e += blockDim.x) {
      const int j = e / kPcrCols, c = e % kPcrCols;
      float y = a[e];
      if (j - st >= 0) y = fmaf(-K1[l * J + j], a[(j - st) * kPcrCols + c], y);
      if (j + st < J) y = fmaf(-K2[l * J + j], a[(j + st) * kPcrCols + c], y);
      b[e] = y;
    }
    __syncthreads();
    float* t = a;
    a = b;
    b = t;
  }
  for (int e = threadIdx.x; e < items; e += blockDim.x) s_x[e] = ib[e / kPcrCols] * a[e];
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
      a.u[(long long)(a.nz - 1) * a.zstride + col0 + c] = R(0);
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
// columns, so iterative refinement runs entirely on chip: per tile
//   w = fl32(rhs);  repeat { w = FP32 Algorithm 2 solve of w;  u += w;
//                            r = r - (I - c L_z) w;  w = fl32(r) }
// with r (initially rhs) and u kept as double-float pairs and the operator's
// FP64 rows split into hi + lo, until max|r| <= tol max|rhs| over the tile
// (a bound at least as strict as the same test over the whole field) or
// maxit FP32 solves.  The thread of column c and partition q keeps its
// partition's rows of w and u in registers (at most MM rows), so the
// recurrences of Algorithm 2 run without shared-memory latency; r lives in
// the FP64 tile the copies use (as a float pair per element), the reduced
// system is solved by parallel cyclic reduction over the whole CTA, and the
// residual's neighbours across a partition end are the reduced system's
// solution itself.  HBM traffic is one FP64 read and one FP64 write per point;
// the only FP64 instruction is the final hi + lo of each u.
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

// Threads per CTA of the one-pass kernel holding at most MM rows per thread
// (three registers per row: the correction and u as a pair).
template <int MM> struct refine_threads { static constexpr int value = MM <= 16 ? 512 : 256; };

template <int MM>
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
  float2* Rp = reinterpret_cast<float2*>(Rt);               // the same slots as (hi, lo)
  float* s_rows = reinterpret_cast<float*>(Rt + rows_alloc * kPcrCols);  // 5n
  float* s_op = s_rows + 5 * n;                 // 6n: A', B', C' as (hi, lo)
  float* s_x = s_op + 6 * n;                    // J x 16
  float* s_y = s_x + J * kPcrCols;              // J x 16
  float* s_lv = s_y + J * kPcrCols;             // (2L + 1) J

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  for (int e = threadIdx.x; e < 5 * n; e += blockDim.x) s_rows[e] = a.rows[e];
  for (int e = threadIdx.x; e < (2 * a.nlv + 1) * J; e += blockDim.x) s_lv[e] = a.lv[e];
  for (int e = threadIdx.x; e < 3 * n; e += blockDim.x) {
    float hi, lo;
    f64_split(a.abc[e], &hi, &lo);
    s_op[2 * e] = hi;
    s_op[2 * e + 1] = lo;
  }
  __syncthreads();
  const float* alpha = s_rows;
  const float* beta = s_rows + n;
  const float* ib = s_rows + 2 * n;
  const float* ap = s_rows + 3 * n;
  const float* cp = s_rows + 4 * n;
  const float* opA = s_op;
  const float* opB = s_op + 2 * n;
  const float* opC = s_op + 4 * n;

  const int c = threadIdx.x % kPcrCols;
  const int q = threadIdx.x / kPcrCols;
  const bool part = q < a.nparts;
  const int s = (int)(((long long)q * n) / a.nparts);
  const int m = part ? (int)(((long long)(q + 1) * n) / a.nparts) - s : 0;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  const uint32_t tile_bytes = (uint32_t)(a.nbox * a.by * kPcrCols * sizeof(double));
  uint32_t phase = 0;
  float w[MM], uh[MM], ul[MM];

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
#pragma unroll
    for (int i = 0; i < MM; ++i)
      if (i < m) {
        w[i] = f64_to_f32(Rt[(s + i) * kPcrCols + c]);
        amax = fmaxf(amax, fabsf(w[i]));
      }
    cta_max_to(amax, s_max);
    int it = 0;
    for (;;) {
      // Step 2 in registers: the partition's two boundary values to s_x
      if (m > 0) {
        // (the last row's value is kept on the way: a select of w[m - 1] by
        // a run-time index would move w to local memory)
        float wl = w[0];
#pragma unroll
        for (int i = 2; i < MM; ++i)
          if (i < m) {
            w[i] = fmaf(-alpha[s + i], w[i - 1], w[i]);
            wl = w[i];
          }
#pragma unroll
        for (int i = MM - 3; i >= 0; --i)
          if (i <= m - 3) w[i] = fmaf(-beta[s + i], w[i + 1], w[i]);
        s_x[(2 * q) * kPcrCols + c] = w[0];
        s_x[(2 * q + 1) * kPcrCols + c] = wl;
      }
      __syncthreads();
      pcr_step3_pcr(s_x, s_y, s_lv, J, a.nlv);  // Step 3, the whole CTA
      __syncthreads();
      // Step 4 in registers, then u += w and r -= (I - c L_z) w in
      // double-float; the neighbours beyond the partition's ends are the
      // neighbouring partitions' end values, solved in Step 3
      float rmax = 0.0f;
      if (m > 0) {
        const float x0 = s_x[(2 * q) * kPcrCols + c], xm = s_x[(2 * q + 1) * kPcrCols + c];
        const float below = q > 0 ? s_x[(2 * q - 1) * kPcrCols + c] : 0.0f;
        const float above = q + 1 < a.nparts ? s_x[(2 * q + 2) * kPcrCols + c] : 0.0f;
#pragma unroll
        for (int i = 0; i < MM; ++i)
          if (i < m) {
            const int r = s + i;
            w[i] = (i == 0) ? x0
                 : (i == m - 1) ? xm
                 : fmaf(-cp[r], xm, fmaf(-ap[r], x0, ib[r] * w[i]));
          }
        float dprev = below;
#pragma unroll
        for (int i = 0; i < MM; ++i)
          if (i < m) {
            const int r = s + i, e = r * kPcrCols + c;
            const float d = w[i];
            const float dnext = (i + 1 < m) ? w[i + 1 < MM ? i + 1 : MM - 1] : above;
            DoubleFloat acc;
            df_acc<true>(acc, opB[2 * r], opB[2 * r + 1], d);
            df_acc(acc, opA[2 * r], opA[2 * r + 1], dprev);
            df_acc(acc, opC[2 * r], opC[2 * r + 1], dnext);
            float bh, bl;
            if (it == 0) {
              f64_split(Rt[e], &bh, &bl);
            } else {
              const float2 rb = Rp[e];
              bh = rb.x;
              bl = rb.y;
            }
            const float2 rn = df_sub(bh, bl, acc);
            Rp[e] = rn;
            rmax = fmaxf(rmax, fabsf(rn.x));
            if (it == 0) {
              uh[i] = d;
              ul[i] = 0.0f;
            } else {
              float us, ut;
              two_sum(uh[i], d, us, ut);
              const float ue = __fadd_rn(ul[i], ut);
              uh[i] = __fadd_rn(us, ue);
              ul[i] = __fsub_rn(ue, __fsub_rn(uh[i], us));
            }
            dprev = d;
            w[i] = rn.x;  // the next FP32 right-hand side
          }
      }
      unsigned int* slot = s_max + 1 + (it & 1);
      cta_max_to(rmax, slot);
      __syncthreads();  // the residual is complete; s_x may be rewritten
      ++it;
      const float rm = __uint_as_float(*slot), am = __uint_as_float(s_max[0]);
      if (rm <= a.tol * am || it >= a.maxit) break;  // the same outcome on every thread
      // the next pass's slot was last read before this pass's barriers
      if (threadIdx.x == 0) s_max[1 + (it & 1)] = 0u;
    }
    // u = hi + lo in FP64, written over the tile for the store
#pragma unroll
    for (int i = 0; i < MM; ++i)
      if (i < m) Rt[(s + i) * kPcrCols + c] = f32_to_f64(uh[i]) + f32_to_f64(ul[i]);
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

template <int MM>
__global__ void __launch_bounds__(refine_threads<MM>::value)
    pcr_refine_kernel(const __grid_constant__ CUtensorMap in_map,
                      const __grid_constant__ CUtensorMap out_map, PcrRefineArgs a, int* status) {
  pcr_refine_body<MM>(&in_map, &out_map, a, status, blockIdx.x, gridDim.x);
}

template <int MM>
__global__ void __launch_bounds__(refine_threads<MM>::value)
    pcr_refine_group_kernel(const PcrRefineBox* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const PcrRefineBox& x = boxes[b];
  if (threadIdx.x == 0) {
    tensormap_acquire(&x.in_map);
    tensormap_acquire(&x.out_map);
  }
  pcr_refine_body<MM>(&x.in_map, &x.out_map, x.a, x.status, blk, x.blocks);
}

// 2-D map over the first n rows of a field: ncols reals per row, rows
// zstride reals apart (0: ncols).
template <class R>
static bool pcr_map(CUtensorMap* map, const void* base, long long ncols, int n, int by,
                    long long zstride = 0) {
  const cuuint64_t gdim[2] = {(cuuint64_t)ncols, (cuuint64_t)n};
  const cuuint64_t gstride[1] = {(cuuint64_t)(zstride ? zstride : ncols) * sizeof(R)};
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

// Columns [col0, col0 + ncols) of the field (ncols < 0: all of them).
template <class R>
static cudaError_t launch_pcr_t(const cfs_plan* P, const HelmCoef& h, const R* rows, const R* red,
                                const R* rhs, R* u, cudaStream_t st, long long col0 = 0,
                                long long ncols = -1) {
  const long long plane = (long long)P->nx * P->ny;
  if (ncols < 0) ncols = plane;
  if (ncols == 0) return cudaSuccess;
  rhs += col0;
  u += col0;
  PcrArgs<R> a;
  a.u = u;
  a.ncols = ncols;
  a.zstride = plane;
  a.n = h.n;
  a.nparts = h.nparts;
  a.face = (h.loc == CFS_LOC_FACE);
  a.nz = P->nz;
  pcr_boxes(h.n, sizeof(R), &a.nbox, &a.by);
  a.rows = rows;
  a.red = red;
  CUtensorMap in_map, out_map;
  if (!pcr_map<R>(&in_map, rhs, a.ncols, h.n, a.by, plane) ||
      !pcr_map<R>(&out_map, u, a.ncols, h.n, a.by, plane))
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

cudaError_t launch_pcr_cols(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                            long long col0, long long ncols, cudaStream_t st) {
  if (col0 < 0 || (col0 & 1) || ncols < 0 || col0 + ncols > (long long)P->nx * P->ny)
    return cudaErrorInvalidValue;  // (16-byte aligned TMA bases)
  return launch_pcr_t<double>(P, h, h.d_rows, h.d_red, rhs, u, st, col0, ncols);
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
  a.zstride = a.ncols;
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
  const size_t J = 2 * (size_t)nparts, L = (size_t)alg2_pcr_levels((int)J);
  return 128 + sizeof(double) * (size_t)nbox * by * kPcrCols   // rhs, r, u tile
         + sizeof(float) * (11 * (size_t)n + 2 * J * kPcrCols + (2 * L + 1) * J);
}

int pcr_refine_thread_limit(int rows) {
  return rows <= 16 ? refine_threads<16>::value : refine_threads<32>::value;
}

// Rows per thread the one-pass kernel is compiled for (8, 16, 24 or 32) for
// the largest partition of set h, or 0 if it has more rows or too many
// partitions for the kernel's CTA.
int pcr_refine_rows(const HelmCoef& h) {
  const int mm = h.mmax <= 8 ? 8 : h.mmax <= 16 ? 16 : h.mmax <= 24 ? 24 : h.mmax <= 32 ? 32 : 0;
  return (mm && kPcrCols * h.nparts <= pcr_refine_thread_limit(mm)) ? mm : 0;
}
static int refine_rows(const HelmCoef& h) { return pcr_refine_rows(h); }

bool pcr_refine_fits(const cfs_plan* P, const HelmCoef& h) {
  return h.d_rows32 && h.d_abc && h.d_lv32 && !P->helm_thomas32 && refine_rows(h) &&
         pcr_refine_smem(h.n, h.nparts) <= 227 * 1024;
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
  a.lv = h.d_lv32;
  a.nlv = alg2_pcr_levels(2 * h.nparts);
  a.words = words;
  return a;
}

template <int MM>
static cudaError_t launch_refine_mm(const CUtensorMap& in_map, const CUtensorMap& out_map,
                                    const PcrRefineArgs& a, int* status, size_t smem,
                                    int threads, cudaStream_t st) {
  auto kern = pcr_refine_kernel<MM>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = (a.ncols + kPcrCols - 1) / kPcrCols;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  kern<<<(unsigned)grid, threads, smem, st>>>(in_map, out_map, a, status);
  return cudaGetLastError();
}

cudaError_t launch_pcr_refine(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                              unsigned int* words, cudaStream_t st) {
  const int mm = refine_rows(h);
  if (!mm) return cudaErrorInvalidValue;
  const PcrRefineArgs a = refine_args(P, h, u, words);
  CUtensorMap in_map, out_map;
  if (!pcr_map<double>(&in_map, rhs, a.ncols, h.n, a.by) ||
      !pcr_map<double>(&out_map, u, a.ncols, h.n, a.by))
    return cudaErrorInvalidValue;
  const size_t smem = pcr_refine_smem(h.n, h.nparts);
  const int threads = kPcrCols * h.nparts;
  switch (mm) {
    case 8: return launch_refine_mm<8>(in_map, out_map, a, P->d_status, smem, threads, st);
    case 16: return launch_refine_mm<16>(in_map, out_map, a, P->d_status, smem, threads, st);
    case 24: return launch_refine_mm<24>(in_map, out_map, a, P->d_status, smem, threads, st);
    default: return launch_refine_mm<32>(in_map, out_map, a, P->d_status, smem, threads, st);
  }
}

size_t pcr_refine_group_box(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                            unsigned int* words, PcrRefineBox* box, int* blocks, int* threads,
                            int* rows) {
  *rows = refine_rows(h);
  if (!*rows) return 0;
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

template <int MM>
static cudaError_t launch_refine_group_mm(const PcrRefineBox* boxes, GroupMap g, int total,
                                          int threads, size_t smem, cudaStream_t st) {
  auto kern = pcr_refine_group_kernel<MM>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<total, threads, smem, st>>>(boxes, g);
  return cudaGetLastError();
}

cudaError_t launch_pcr_refine_group(const PcrRefineBox* boxes, GroupMap g, int total, int threads,
                                    size_t smem, int rows, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  switch (rows) {
    case 8: return launch_refine_group_mm<8>(boxes, g, total, threads, smem, st);
    case 16: return launch_refine_group_mm<16>(boxes, g, total, threads, smem, st);
    case 24: return launch_refine_group_mm<24>(boxes, g, total, threads, smem, st);
    case 32: return launch_refine_group_mm<32>(boxes, g, total, threads, smem, st);
    default: return cudaErrorInvalidValue;
  }
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
  a.zstride = ncols;
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
