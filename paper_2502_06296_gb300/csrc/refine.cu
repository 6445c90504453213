// refine.cu -- FP32 solves with FP64 iterative refinement.
//
// The FP32 transforms and sweeps are memory-bound on GB300, where FP64 runs
// at 1/64 of the FP32 rate.  Accuracy is won back by classical iterative
// refinement: p_0 = 0, r_0 = f; repeat { delta = solve32(r); p += delta (FP64);
// r = f - L p (FP64, the staggered 7-point operator) } until
// ||r||_inf <= tol ||f||_inf or the iteration budget is spent.  FP64 is used
// only for the residual, the accumulation, the near-singular low-wavenumber
// columns of the z sweep and the pre-processing of the coefficients.
//
// The correction p += delta is fused into the FP32 inverse x transform
// (fft_x.cu, OUT_ADD); the residual kernels write the next FP32 right-hand
// side and the max-norm of the residual in one pass.
#include <math.h>
#include <string.h>

#include "chanfs_group.cuh"

namespace chanfs {

constexpr int kResBlock = 128;

__device__ __forceinline__ void block_max_to(float v, unsigned int* out) {
  // non-negative floats order like their bit patterns
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ float wmax[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wmax[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? wmax[lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomicMax(out, __float_as_uint(v));
  }
}

// The block's sum of v in a fixed order (shuffle tree per warp, then the
// warps in order), written to *slot by thread 0.  Every thread calls it.
__device__ __forceinline__ void block_sum_to(double v, double* slot) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wsum[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += wsum[i];
    *slot = t;
  }
}

// ----------------------------------------------------------------------------
// Start of a refined Poisson solve, one pass over f: r_0 = f as FP32 (the
// right-hand side of the first FP32 solve), the dz-weighted plane sums of f
// for the Neumann compatibility mean (partial may be null), and the largest
// and smallest r_0 (the reference norm max |f - mean| follows from them and
// the mean).  The first solve does not need f - mean: its (0, 0) column
// removes the mean of its right-hand side, as the FP64 solve's does.
// Block b takes chunk b % nch of plane b / nch (16-byte loads, four
// accumulators), and the sums are reduced in a fixed order (per block, then
// per plane, then over the planes), so results are bit-reproducible.
// ----------------------------------------------------------------------------
// Order-preserving key of a float (larger float, larger key; 0 below all).
__device__ __forceinline__ unsigned int float_key(float v) {
  const unsigned int u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ inline float key_float(unsigned int k) {
  const unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  float v;
  memcpy(&v, &u, sizeof(v));
  return v;
}

// words[0] = max key(r), words[1] = max key(-r) over the block (atomics).
__device__ __forceinline__ void block_extremes_to(float hi, float lo, unsigned int* words) {
  unsigned int a = float_key(hi), b = float_key(-lo);
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_down_sync(0xffffffffu, a, o));
    b = max(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(words, a);
    atomicMax(words + 1, b);
  }
}

__device__ __forceinline__ void start_body(const double* __restrict__ f, long long nxy,
                                           const double* __restrict__ dzf, double* partial,
                                           float* __restrict__ r32, unsigned int* words,
                                           long long blk, int nch) {
  __shared__ double sh[256];
  const int k = (int)(blk / nch), c = (int)(blk % nch);
  const long long n2 = nxy >> 1;  // nx is even
  const long long lo = n2 * c / nch, hi = n2 * (c + 1) / nch;
  const double2* f2 = reinterpret_cast<const double2*>(f + (long long)k * nxy);
  float2* r2 = reinterpret_cast<float2*>(r32 + (long long)k * nxy);
  const long long B = blockDim.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  float vmax = -INFINITY, vmin = INFINITY;
  long long i = lo + threadIdx.x;
  for (; i + 3 * B < hi; i += 4 * B) {
    const double2 v0 = f2[i], v1 = f2[i + B], v2 = f2[i + 2 * B], v3 = f2[i + 3 * B];
    const float2 a = make_float2(f64_to_f32(v0.x), f64_to_f32(v0.y));
    const float2 b = make_float2(f64_to_f32(v1.x), f64_to_f32(v1.y));
    const float2 cc = make_float2(f64_to_f32(v2.x), f64_to_f32(v2.y));
    const float2 d = make_float2(f64_to_f32(v3.x), f64_to_f32(v3.y));
    r2[i] = a;
    r2[i + B] = b;
    r2[i + 2 * B] = cc;
    r2[i + 3 * B] = d;
    vmax = fmaxf(fmaxf(fmaxf(vmax, fmaxf(a.x, a.y)), fmaxf(b.x, b.y)),
                 fmaxf(fmaxf(cc.x, cc.y), fmaxf(d.x, d.y)));
    vmin = fminf(fminf(fminf(vmin, fminf(a.x, a.y)), fminf(b.x, b.y)),
                 fminf(fminf(cc.x, cc.y), fminf(d.x, d.y)));
    if (partial) {
      s0 += v0.x + v2.x;
      s1 += v0.y + v2.y;
      s2 += v1.x + v3.x;
      s3 += v1.y + v3.y;
    }
  }
  for (; i < hi; i += B) {
    const double2 v = f2[i];
    const float2 a = make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
    r2[i] = a;
    vmax = fmaxf(vmax, fmaxf(a.x, a.y));
    vmin = fminf(vmin, fminf(a.x, a.y));
    if (partial) {
      s0 += v.x;
      s1 += v.y;
    }
  }
  block_extremes_to(vmax, vmin, words);
  if (!partial) return;
  sh[threadIdx.x] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blk] = dzf[k] * sh[0];
}

__global__ void __launch_bounds__(256) start_kernel(const double* __restrict__ f, long long nxy,
                                                    const double* __restrict__ dzf,
                                                    double* partial, float* __restrict__ r32,
                                                    unsigned int* words, int nch) {
  start_body(f, nxy, dzf, partial, r32, words, blockIdx.x, nch);
}

// mean = (sum of the nz * nch partials) / (sum_k dz_k * Nx * Ny), fixed order.
__device__ __forceinline__ void mean_final_body(const double* partial, int nz, int nch,
                                                const double* dzf, long long nxy, double* mean) {
  __shared__ double sh[256], shw[256];
  double s = 0.0, w = 0.0;
  for (int i = threadIdx.x; i < nz * nch; i += blockDim.x) s += partial[i];
  for (int k = threadIdx.x; k < nz; k += blockDim.x) w += dzf[k];
  sh[threadIdx.x] = s;
  shw[threadIdx.x] = w;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[threadIdx.x] += sh[threadIdx.x + o];
      shw[threadIdx.x] += shw[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *mean = sh[0] / (shw[0] * (double)nxy);
}

__global__ void mean_final_kernel(const double* partial, int nz, int nch, const double* dzf,
                                  long long nxy, double* mean) {
  mean_final_body(partial, nz, nch, dzf, nxy, mean);
}

// The reference norm max |r_0 - mean| from the extremes of r_0 (mean 0
// without a null space).
__host__ __device__ inline double start_norm(const unsigned int* words, double mean) {
  const double hi = (double)key_float(words[0]), lo = -(double)key_float(words[1]);
  const double a = hi - mean, b = mean - lo;
  return a > b ? a : b;
}

// ----------------------------------------------------------------------------
// Residual update of the later iterations: r_new = r_old - L delta for the FP32
// correction delta (exact FP32 values) just added to p.  L delta is formed in
// double-float arithmetic on the FP32 units: each coefficient c is split as
// hi + lo (hi = fl32(c), lo = fl32(c - hi)); hi * d is taken exactly as
// p + e by TwoProd (an FMA gives e), lo * d is added to e, the p parts are
// summed exactly by TwoSum and the small parts plainly.  The result holds
// L delta to about 2^-48 of sum |c d|, and after the first correction
// |delta| is small, so r_new is as accurate as a direct FP64 evaluation
// (whose error is about 2^-53 ||L|| |p|).  The residual itself is kept as a
// double-float pair too, so the update runs without FP64 instructions.
// The first residual of a solve (|delta| ~ |p|) takes the stencil in
// differences (below).
// ----------------------------------------------------------------------------
// zk: the per-plane coefficients split hi + lo, packed so that a plane's are
// two 16-byte loads: zk[3k] = (A_k, C_k), zk[3k+1] = (B'_k, dz_k),
// zk[3k+2] = (D_k, dz_k) (first residual, below), zk[3nz] = (1/dx^2, 1/dy^2),
// each pair as (hi, lo).
template <class I>
__device__ __forceinline__ void poisson_update_body(const float* __restrict__ dlt,
                                                    float* __restrict__ rhi,
                                                    float* __restrict__ rlo,
                                                    const float4* __restrict__ zk,
                                                    unsigned int* rmax, int nx, int ny, int nz,
                                                    int ybc, double* mpart, long long blk) {
  const I nxy = (I)nx * ny;
  const I col = (I)(blk * blockDim.x + threadIdx.x);
  float vmax = 0.0f;
  DoubleFloat macc{0.0f, 0.0f};  // sum_k dz_k delta_k of the column
  if (col < nxy) {
    const int i = (int)(col % nx), j = (int)(col / nx);
    const I ip = (i + 1 == nx) ? col - i : col + 1;
    const I im = (i == 0) ? col + nx - 1 : col - 1;
    I jp, jm;
    bool np_ = false, nm_ = false;
    if (ybc == CFS_Y_PERIODIC) {
      jp = (j + 1 == ny) ? col - (I)j * nx : col + nx;
      jm = (j == 0) ? col + (I)(ny - 1) * nx : col - nx;
    } else {
      jp = (j + 1 == ny) ? col : col + nx;
      jm = (j == 0) ? col : col - nx;
      np_ = (ybc == CFS_Y_DIRICHLET) && (j + 1 == ny);
      nm_ = (ybc == CFS_Y_DIRICHLET) && (j == 0);
    }
    const float4 axy = zk[3 * nz];
    // the loads of plane k + 1 are issued one iteration ahead, so that they
    // are in flight while plane k is combined
    float dkm = 0.0f, dk = dlt[col];
    float dkp = (nz > 1) ? dlt[nxy + col] : 0.0f;
    float xp = dlt[ip], xm = dlt[im], yp = dlt[jp], ym = dlt[jm];
    float2 rp = make_float2(rhi[col], rlo[col]);
    for (int k = 0; k < nz; ++k) {
      const I o = (I)k * nxy;
      const bool more = k + 1 < nz;
      const I on = more ? o + nxy : o;  // plane k + 1 (clamped)
      const float dkp2 = (k + 2 < nz) ? dlt[on + nxy + col] : 0.0f;
      const float xpn = dlt[on + ip], xmn = dlt[on + im], ypn = dlt[on + jp], ymn = dlt[on + jm];
      const float2 rpn = make_float2(rhi[on + col], rlo[on + col]);
      const float4 ac = zk[3 * k], bw = zk[3 * k + 1];
      DoubleFloat acc;
      df_acc<true>(acc, bw.x, bw.y, dk);
      df_acc<false>(acc, axy.x, axy.y, xp);
      df_acc<false>(acc, axy.x, axy.y, xm);
      df_acc<false>(acc, axy.z, axy.w, np_ ? -yp : yp);
      df_acc<false>(acc, axy.z, axy.w, nm_ ? -ym : ym);
      df_acc<false>(acc, ac.x, ac.y, dkm);
      df_acc<false>(acc, ac.z, ac.w, dkp);
      // (hi, lo) - (s + e) in double-float: TwoSum of the leading parts, the
      // rest added to the error term, renormalised by a second TwoSum
      float sh, se, hi, lo;
      two_sum(rp.x, -acc.s, sh, se);
      se = __fadd_rn(se, __fsub_rn(rp.y, acc.e));
      two_sum(sh, se, hi, lo);
      rhi[o + col] = hi;  // also the next FP32 right-hand side
      rlo[o + col] = lo;
      vmax = fmaxf(vmax, fabsf(hi));
      if (mpart) df_acc<false>(macc, bw.z, bw.w, dk);
      dkm = dk;
      dk = dkp;
      dkp = dkp2;
      xp = xpn;
      xm = xmn;
      yp = ypn;
      ym = ymn;
      rp = rpn;
    }
  }
  if (mpart) block_sum_to(f32_to_f64(macc.s) + f32_to_f64(macc.e), mpart + blk);
  block_max_to(vmax, rmax);
}

// Index type of a residual kernel: 32-bit offsets where every index of the
// field (and the look-ahead two planes on) fits, which saves the 64-bit
// address arithmetic of the six loads and three stores per point.
inline __host__ __device__ bool res_idx32(int nx, int ny, int nz) {
  return (long long)nx * ny * (nz + 2) + kResBlock < (1LL << 31);
}

template <class I>
__global__ void __launch_bounds__(kResBlock) poisson_update_kernel(
    const float* __restrict__ dlt, float* __restrict__ rhi, float* __restrict__ rlo,
    const float4* __restrict__ zk, unsigned int* rmax, int nx, int ny, int nz, int ybc,
    double* mpart) {
  poisson_update_body<I>(dlt, rhi, rlo, zk, rmax, nx, ny, nz, ybc, mpart, blockIdx.x);
}

// ----------------------------------------------------------------------------
// First residual of a solve: r_1 = (f - mean) - L delta for the first FP32
// correction delta (= p).  Here |delta| ~ |p|, and the stencil's terms, of
// size |p|/h^2, cancel down to the size of f: the update's double-float
// error, 2^-48 of sum |c d|, would then exceed a direct FP64 evaluation's
// 2^-53 of the same sum by 2^5.  So L is taken in differences,
//   L d = A_k (d_{k-1} - d_k) + C_k (d_{k+1} - d_k)
//       + (1/dx^2) [(d_{i+1} - d) + (d_{i-1} - d)]
//       + (1/dy^2) [(d_{j+1} - d) + (d_{j-1} - d)] + D_k d,
//   D_k = A_k + B'_k + C_k + 2/dx^2 + 2/dy^2   (B'_k the zop centre row),
// the same sum regrouped (the ghost values of the walls enter as they do in
// the direct form).  D_k is summed exactly on the host; it is the rounding
// residue of zero in the interior and carries the wall terms of Dirichlet
// walls.  The difference of two FP32 values is exact as a TwoSum pair, so
// each term has the size of c |d_n - d|, and the error is 2^-48 of sum
// c |d_n - d| ~ 6 * 2^-48 |grad p| / h, against the direct FP64 evaluation's
// 12 * 2^-53 |p| / h^2: 16 h |grad p| / |p| times that, below it where the
// field is resolved by more than about 100 points per wavelength and never
// above it by more than 2^5.  The solution of the Poisson equation (Eq. 4) is
// smooth (its grid-scale part is O(h^2 |f|)).  f - mean is one FP64
// subtraction; its split into hi + lo runs on the integer units.
// ----------------------------------------------------------------------------
// acc (+)= c * (a - b), the difference exact (TwoSum), c = ch + cl.
template <bool INIT>
__device__ __forceinline__ void diff_acc(DoubleFloat& acc, float ch, float cl, float a, float b) {
  float dh, dl;
  two_sum(a, -b, dh, dl);
  const float q = __fmul_rn(ch, dh);
  float e = __fmaf_rn(ch, dh, -q);  // ch * dh - q, exact
  e = __fmaf_rn(ch, dl, e);
  e = __fmaf_rn(cl, dh, e);
  if (INIT) {
    acc.s = q;
    acc.e = e;
  } else {
    float s, t;
    two_sum(acc.s, q, s, t);
    acc.s = s;
    acc.e = __fadd_rn(acc.e, __fadd_rn(t, e));
  }
}

// zk as for the update.  r32 must not alias dlt (the neighbours of a column
// are read from dlt).
template <class I>
__device__ __forceinline__ void poisson_first_body(
    const double* __restrict__ f, const double* __restrict__ mean, const float* __restrict__ dlt,
    float* __restrict__ rhi, float* __restrict__ rlo, const float4* __restrict__ zk,
    unsigned int* rmax, int nx, int ny, int nz, int ybc, double* mpart, long long blk,
    float* __restrict__ dcopy) {
  const I nxy = (I)nx * ny;
  const I col = (I)(blk * blockDim.x + threadIdx.x);
  float vmax = 0.0f;
  DoubleFloat macc{0.0f, 0.0f};  // sum_k dz_k delta_k of the column
  if (col < nxy) {
    const double mu = mean ? *mean : 0.0;
    const int i = (int)(col % nx), j = (int)(col / nx);
    const I ip = (i + 1 == nx) ? col - i : col + 1;
    const I im = (i == 0) ? col + nx - 1 : col - 1;
    // y neighbours: periodic, or the mirror ghost of a wall (+d Neumann, -d Dirichlet)
    I jp, jm;
    bool np_ = false, nm_ = false;  // negate the ghost
    if (ybc == CFS_Y_PERIODIC) {
      jp = (j + 1 == ny) ? col - (I)j * nx : col + nx;
      jm = (j == 0) ? col + (I)(ny - 1) * nx : col - nx;
    } else {
      jp = (j + 1 == ny) ? col : col + nx;
      jm = (j == 0) ? col : col - nx;
      np_ = (ybc == CFS_Y_DIRICHLET) && (j + 1 == ny);
      nm_ = (ybc == CFS_Y_DIRICHLET) && (j == 0);
    }
    const float4 axy = zk[3 * nz];
    // the loads of plane k + 1 are issued one iteration ahead
    float dkm = 0.0f, dk = dlt[col];
    float dkp = (nz > 1) ? dlt[nxy + col] : 0.0f;
    float xp = dlt[ip], xm = dlt[im], yp = dlt[jp], ym = dlt[jm];
    double fk = f[col];
    for (int k = 0; k < nz; ++k) {
      const I o = (I)k * nxy;
      const I on = (k + 1 < nz) ? o + nxy : o;  // plane k + 1 (clamped)
      const float dkp2 = (k + 2 < nz) ? dlt[on + nxy + col] : 0.0f;
      const float xpn = dlt[on + ip], xmn = dlt[on + im], ypn = dlt[on + jp], ymn = dlt[on + jm];
      const double fkn = f[on + col];
      const float4 ac = zk[3 * k], dw = zk[3 * k + 2];
      DoubleFloat acc;
      diff_acc<true>(acc, ac.x, ac.y, dkm, dk);  // dkm = 0 below the first row
      diff_acc<false>(acc, ac.z, ac.w, dkp, dk);
      diff_acc<false>(acc, axy.x, axy.y, xp, dk);
      diff_acc<false>(acc, axy.x, axy.y, xm, dk);
      diff_acc<false>(acc, axy.z, axy.w, np_ ? -yp : yp, dk);
      diff_acc<false>(acc, axy.z, axy.w, nm_ ? -ym : ym, dk);
      df_acc<false>(acc, dw.x, dw.y, dk);
      // ((f - mean) split) - (s + e), renormalised as in the update
      float fh, fl, sh, se, hi, lo;
      f64_split(fk - mu, &fh, &fl);
      two_sum(fh, -acc.s, sh, se);
      se = __fadd_rn(se, __fsub_rn(fl, acc.e));
      two_sum(sh, se, hi, lo);
      rhi[o + col] = hi;  // also the next FP32 right-hand side
      rlo[o + col] = lo;
      if (dcopy) dcopy[o + col] = dk;  // the correction, for the pass that writes p
      vmax = fmaxf(vmax, fabsf(hi));
      if (mpart) df_acc<false>(macc, dw.z, dw.w, dk);
      dkm = dk;
      dk = dkp;
      dkp = dkp2;
      xp = xpn;
      xm = xmn;
      yp = ypn;
      ym = ymn;
      fk = fkn;
    }
  }
  if (mpart) block_sum_to(f32_to_f64(macc.s) + f32_to_f64(macc.e), mpart + blk);
  block_max_to(vmax, rmax);
}

template <class I>
__global__ void __launch_bounds__(kResBlock) poisson_first_kernel(
    const double* __restrict__ f, const double* __restrict__ mean, const float* __restrict__ dlt,
    float* __restrict__ rhi, float* __restrict__ rlo, const float4* __restrict__ zk,
    unsigned int* rmax, int nx, int ny, int nz, int ybc, double* mpart, float* __restrict__ dcopy) {
  poisson_first_body<I>(f, mean, dlt, rhi, rlo, zk, rmax, nx, ny, nz, ybc, mpart, blockIdx.x,
                        dcopy);
}

// The dz-weighted sum of a correction, from the per-block sums of the
// residual kernels, added in a fixed order to the running sum *num (the
// numerator of the weighted mean of the solution).
__device__ __forceinline__ void mean_acc_body(const double* __restrict__ mpart, int nparts,
                                              double* num) {
  double t = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += mpart[i];
  __shared__ double tot;
  block_sum_to(t, &tot);
  __syncthreads();
  if (threadIdx.x == 0) *num += tot;
}

__global__ void mean_acc_kernel(const double* __restrict__ mpart, int nparts, double* num) {
  mean_acc_body(mpart, nparts, num);
}

// mean = num * inv (inv = 1 / (sum of the cell widths * Nx * Ny)).
__global__ void mean_from_num_kernel(const double* num, double inv, double* mean) {
  if (threadIdx.x == 0) *mean = *num * inv;
}

// Helmholtz: u (+)= delta, then r = rhs - (I - c L_z) u, as FP32, and max |r|.
// mode 0: u is not read (r = rhs); 1: u = delta; 2: u += delta.  delta is read
// from r32 and overwritten by the new residual.  One thread per column,
// marching up in z one row behind the update so that u_{k+1} is final when
// row k is evaluated.  abc = [A' | B' | C'] of I - c L_z (n rows); the wall
// row of a face field (n < nz) keeps r = 0.  FP64: 5 instructions per point.
__device__ __forceinline__ void helm_residual_body(const double* __restrict__ rhs,
                                                   double* __restrict__ u, float* __restrict__ r32,
                                                   const double* __restrict__ abc,
                                                   unsigned int* rmax, long long ncols, int n,
                                                   int nz, int mode, long long blk) {
  const long long col = blk * blockDim.x + threadIdx.x;
  float vmax = 0.0f;
  if (col < ncols && mode == 0) {  // r = rhs: (I - c L_z) 0 vanishes exactly
    for (int k = 0; k < n; ++k) {
      const long long o = (long long)k * ncols + col;
      const float rf = f64_to_f32(rhs[o]);
      r32[o] = rf;
      vmax = fmaxf(vmax, fabsf(rf));
    }
    if (n < nz) r32[(long long)(nz - 1) * ncols + col] = 0.0f;
  } else if (col < ncols) {
    auto update = [&](int k) -> double {
      const long long o = (long long)k * ncols + col;
      if (mode == 0) return 0.0;
      const double d = f32_to_f64(r32[o]);
      const double v = (mode == 1) ? d : u[o] + d;
      u[o] = v;
      return v;
    };
    double um = 0.0, uk = update(0);
    for (int k = 0; k < n; ++k) {
      const double up = (k + 1 < n) ? update(k + 1) : 0.0;
      const long long o = (long long)k * ncols + col;
      double t = abc[n + k] * uk;
      t = fma(abc[k], um, t);
      t = fma(abc[2 * n + k], up, t);
      const float rf = f64_to_f32(rhs[o] - t);
      r32[o] = rf;
      vmax = fmaxf(vmax, fabsf(rf));
      um = uk;
      uk = up;
    }
    if (n < nz) {
      const long long o = (long long)(nz - 1) * ncols + col;
      r32[o] = 0.0f;
      if (mode == 1) u[o] = 0.0;
    }
  }
  block_max_to(vmax, rmax);
}

__global__ void __launch_bounds__(kResBlock) helm_residual_kernel(
    const double* __restrict__ rhs, double* __restrict__ u, float* __restrict__ r32,
    const double* __restrict__ abc, unsigned int* rmax, long long ncols, int n, int nz, int mode) {
  helm_residual_body(rhs, u, r32, abc, rmax, ncols, n, nz, mode, blockIdx.x);
}

// A solve that stopped after its first FP32 solve: p is that correction (the
// passes keep it in FP32 until a second one is added), less the solution's
// dz-weighted mean (mean may be null: no null space).
__device__ __forceinline__ void first_only_body(double* __restrict__ p,
                                                const float* __restrict__ delta, long long n,
                                                const double* __restrict__ mean, long long blk,
                                                long long nblk) {
  const double mu = mean ? *mean : 0.0;
  for (long long i = blk * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x)
    p[i] = f32_to_f64(delta[i]) - mu;
}

__global__ void first_only_kernel(double* __restrict__ p, const float* __restrict__ delta,
                                  long long n, const double* __restrict__ mean) {
  first_only_body(p, delta, n, mean, blockIdx.x, gridDim.x);
}

// ----------------------------------------------------------------------------
// Grouped forms: one launch per stage for every box of a group (the same
// per-box arithmetic and block partition as the single-plan kernels).
// ----------------------------------------------------------------------------

// Start pass: nz * start_chunks(nz) blocks per box.
__global__ void __launch_bounds__(256) start_group_kernel(const ResBox* boxes, GroupMap g,
                                                          const GroupIo* io) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  start_body(io[b].f, (long long)r.nx * r.ny, r.dzf, r.neumann ? r.partial : nullptr, r.r32,
             r.rmax, blk, start_chunks(r.nz));
}

__global__ void mean_final_group_kernel(const ResBox* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  mean_final_body(r.partial, r.nz, start_chunks(r.nz), r.dzf, (long long)r.nx * r.ny, r.mean);
}

__global__ void __launch_bounds__(kResBlock) poisson_first_group_kernel(const ResBox* boxes,
                                                                        GroupMap g,
                                                                        const GroupIo* io) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  const double* mean = r.neumann ? r.mean : nullptr;
  double* mpart = r.neumann ? r.mpart : nullptr;
  if (res_idx32(r.nx, r.ny, r.nz))
    poisson_first_body<int>(io[b].f, mean, r.r32, r.r32b, r.rlo, r.zk, r.rmax, r.nx, r.ny, r.nz,
                            r.ybc, mpart, blk, r.dcopy);
  else
    poisson_first_body<long long>(io[b].f, mean, r.r32, r.r32b, r.rlo, r.zk, r.rmax, r.nx, r.ny,
                                  r.nz, r.ybc, mpart, blk, r.dcopy);
}

// One block per box (Neumann boxes; the others have nothing to sum).
__global__ void mean_acc_group_kernel(const ResBox* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  if (!r.neumann) return;
  const long long nxy = (long long)r.nx * r.ny;
  mean_acc_body(r.mpart, (int)((nxy + kResBlock - 1) / kResBlock), r.mnum);
}

__global__ void mean_from_num_group_kernel(const ResBox* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  if (threadIdx.x == 0) *r.mean = *r.mnum * r.inv_wn;
}

__global__ void __launch_bounds__(kResBlock) helm_residual_group_kernel(const ResBox* boxes,
                                                                        GroupMap g,
                                                                        const GroupIo* io,
                                                                        int mode) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  helm_residual_body(io[b].f, io[b].p, r.r32, r.abc, r.rmax, (long long)r.nx * r.ny, r.n, r.nz,
                     mode, blk);
}

__global__ void __launch_bounds__(kResBlock) poisson_update_group_kernel(const ResBox* boxes,
                                                                         GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  double* mpart = r.neumann ? r.mpart : nullptr;
  if (res_idx32(r.nx, r.ny, r.nz))
    poisson_update_body<int>(r.r32, r.r32b, r.rlo, r.zk, r.rmax, r.nx, r.ny, r.nz, r.ybc, mpart,
                             blk);
  else
    poisson_update_body<long long>(r.r32, r.r32b, r.rlo, r.zk, r.rmax, r.nx, r.ny, r.nz, r.ybc,
                                   mpart, blk);
}

__global__ void first_only_group_kernel(const ResBox* boxes, GroupMap g, const GroupIo* io) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  const long long n = (long long)r.nx * r.ny * r.nz;
  first_only_body(io[b].p, r.r32, n, r.neumann ? r.mean : nullptr, blk, group_sub_blocks(n));
}

// Zero solution of the boxes whose right-hand side is zero.
__global__ void zero_fill_group_kernel(const ResBox* boxes, GroupMap g, const GroupIo* io) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const ResBox& r = boxes[b];
  const long long n = (long long)r.nx * r.ny * r.nz;
  const long long nblk = group_sub_blocks(n);
  double* p = io[b].p;
  for (long long i = blk * blockDim.x + threadIdx.x; i < n; i += nblk * blockDim.x) p[i] = 0.0;
}

// After the start: each box's reference norm and its starting state.  keys:
// the Poisson start pass left the extreme keys of r_0 = f (the norm is
// max |f - mean|, the mean of Neumann boxes); otherwise the norm word holds
// max |r_0| (Helmholtz).  A box iterates if it is eligible (null: every box)
// and the norm is not zero; an eligible box with a zero norm has the zero
// solution (zero[b]).  mean_on (may be null) marks the iterating boxes whose
// solution mean is removed at the end.  Every box starts at 0 iterations.
__global__ void group_start_kernel(const ResBox* boxes, int nbox, int keys, double* fmax,
                                   const int* eligible, int* active, int* mean_on, int* zero,
                                   int* iters, double* rho, GroupCtl* ctl, int* one) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    ctl->it = 0;
    ctl->nactive = 0;
  }
  if (b >= nbox) return;
  unsigned int* w = boxes[b].rmax;
  const double f = keys ? start_norm(w, boxes[b].neumann ? *boxes[b].mean : 0.0)
                        : (double)__uint_as_float(w[0]);
  w[0] = 0u;
  fmax[b] = f;
  const int elig = eligible ? eligible[b] : 1;
  const int on = elig && f != 0.0;
  active[b] = on;
  if (mean_on) mean_on[b] = on && boxes[b].neumann;
  if (one) one[b] = on;
  if (boxes[b].mnum) *boxes[b].mnum = 0.0;
  zero[b] = elig && !on;
  iters[b] = 0;
  rho[b] = 0.0;
}

// After a residual of iteration ctl->it: each active box takes its relative
// residual and leaves the iteration once it meets its tolerance or has used
// its FP32 solves.  One block; ctl->nactive counts the boxes still
// iterating, ctl->it advances, and inside a graph the loop's condition is
// set to (nactive > 0).  mean_on (may be null): a box that leaves after
// more than one FP32 solve needs no final mean removal (its correction
// passes kept the mean at zero; see refine_poisson).
__global__ void __launch_bounds__(1024) group_iter_end_kernel(
    const ResBox* boxes, int nbox, const double* fmax, const double* tol, const int* maxit,
    int* active, int* mean_on, int* iters, double* rho, GroupCtl* ctl,
    cudaGraphConditionalHandle cond, int set_cond, int* one) {
  __shared__ int count;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  const int it = ctl->it;
  int mine = 0;
  for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
    if (!active[b]) continue;
    unsigned int* w = boxes[b].rmax;
    const float rmax = __uint_as_float(*w);
    *w = 0u;
    const double r = (double)rmax / fmax[b];
    rho[b] = r;
    iters[b] = it + 1;
    if (r <= tol[b] || it + 1 >= maxit[b]) {
      active[b] = 0;
      if (mean_on && it >= 1) mean_on[b] = 0;
      if (one && it >= 1) one[b] = 0;  // more than one correction: p was written
    } else {
      ++mine;
    }
  }
  if (mine) atomicAdd(&count, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->it = it + 1;
    ctl->nactive = count;
    // (a refined solve takes at most 64 FP32 solves: a second bound on the loop)
    if (set_cond) cudaGraphSetConditional(cond, (count > 0 && it + 1 < 64) ? 1u : 0u);
  }
}

// Clears every box's max-norm word before the first residual (a plan's word
// holds whatever its last solve, or its allocation, left there).
__global__ void group_zero_max_kernel(const ResBox* boxes, int nbox) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) {  // the norm word and the start pass's second key
    boxes[b].rmax[0] = 0u;
    boxes[b].rmax[1] = 0u;
  }
}

cudaError_t launch_group_refine_stage(int stage, const ResBox* boxes, GroupMap g, int total,
                                      const GroupIo* io, int flag, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  switch (stage) {
    case GSTAGE_MEAN_FINAL:
      mean_final_group_kernel<<<total, 256, 0, st>>>(boxes, g);
      break;
    case GSTAGE_RESIDUAL:
      poisson_first_group_kernel<<<total, kResBlock, 0, st>>>(boxes, g, io);
      break;
    case GSTAGE_UPDATE:
      poisson_update_group_kernel<<<total, kResBlock, 0, st>>>(boxes, g);
      break;
    case GSTAGE_HELM_RESIDUAL:
      helm_residual_group_kernel<<<total, kResBlock, 0, st>>>(boxes, g, io, flag);
      break;
    case GSTAGE_ZERO:
      zero_fill_group_kernel<<<total, 256, 0, st>>>(boxes, g, io);
      break;
    case GSTAGE_START:
      start_group_kernel<<<total, 256, 0, st>>>(boxes, g, io);
      break;
    case GSTAGE_MEAN_ACC:
      mean_acc_group_kernel<<<total, 256, 0, st>>>(boxes, g);
      break;
    case GSTAGE_MEAN_FROM_NUM:
      mean_from_num_group_kernel<<<total, 32, 0, st>>>(boxes, g);
      break;
    default:  // GSTAGE_FIRST_ONLY
      first_only_group_kernel<<<total, 256, 0, st>>>(boxes, g, io);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_group_start(const ResBox* boxes, int nbox, int keys, double* fmax,
                               const int* eligible, int* active, int* mean_on, int* zero,
                               int* iters, double* rho, GroupCtl* ctl, cudaStream_t st, int* one) {
  group_start_kernel<<<(nbox + 127) / 128, 128, 0, st>>>(boxes, nbox, keys, fmax, eligible,
                                                         active, mean_on, zero, iters, rho, ctl,
                                                         one);
  return cudaGetLastError();
}

cudaError_t launch_group_iter_end(const ResBox* boxes, int nbox, const double* fmax,
                                  const double* tol, const int* maxit, int* active,
                                  int* mean_on, int* iters, double* rho, GroupCtl* ctl,
                                  cudaGraphConditionalHandle cond, int set_cond, cudaStream_t st,
                                  int* one) {
  group_iter_end_kernel<<<1, 1024, 0, st>>>(boxes, nbox, fmax, tol, maxit, active, mean_on,
                                            iters, rho, ctl, cond, set_cond, one);
  return cudaGetLastError();
}

cudaError_t launch_group_zero_max(const ResBox* boxes, int nbox, cudaStream_t st) {
  group_zero_max_kernel<<<(nbox + 127) / 128, 128, 0, st>>>(boxes, nbox);
  return cudaGetLastError();
}


// ----------------------------------------------------------------------------
// Self-check of the integer-unit conversions against the hardware's: sample
// i is a hashed 64-bit pattern (any double: every exponent, the special
// values), the same with its 29 dropped mantissa bits set to an exact tie
// inside the binary32 range, and its low 32 bits as a float.
// ----------------------------------------------------------------------------
// Equal encodings, or both NaN (the NaN payload is not specified).
__device__ __forceinline__ bool same_f32(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
}
__device__ __forceinline__ bool same_f64(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}

__global__ void conversion_check_kernel(unsigned long long n, unsigned long long* bad) {
  unsigned long long local = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull;  // splitmix64 of the counter
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double x = __longlong_as_double((long long)z);
    local += !same_f32(f64_to_f32(x), __double2float_rn(x));
    const unsigned long long e = 897ull + ((z >> 52) % 254ull);  // a binary32 exponent
    const unsigned long long t =
        (z & 0x800FFFFFE0000000ull) | (e << 52) | 0x10000000ull;  // exact tie
    const double xt = __longlong_as_double((long long)t);
    local += !same_f32(f64_to_f32(xt), __double2float_rn(xt));
    // binary32 subnormal results and their ties: exponents 870..896
    const unsigned long long es = 870ull + ((z >> 40) % 27ull);
    const double xs = __longlong_as_double((long long)((z & 0x800FFFFFFFFFFFFFull) | (es << 52)));
    local += !same_f32(f64_to_f32(xs), __double2float_rn(xs));
    // a tie at the rounding position (exponents 874..896: the tie bit is in
    // the stored mantissa)
    const unsigned long long et = 874ull + ((z >> 40) % 23ull);
    const unsigned long long sh = 926ull - et;  // 30..52
    const unsigned long long mt =
        ((z & 0x000FFFFFFFFFFFFFull) & ~((1ull << sh) - 1ull)) | (1ull << (sh - 1));
    const double xst =
        __longlong_as_double((long long)((z & 0x8000000000000000ull) | (et << 52) | mt));
    local += !same_f32(f64_to_f32(xst), __double2float_rn(xst));
    const float f = __uint_as_float((unsigned)z);
    local += !same_f64(f32_to_f64(f), (double)f);
    // the double-float split, for values in the normal binary32 range (and
    // lo counted only where the hardware's lo is normal or zero)
    const unsigned long long en = 897ull + ((z >> 45) % 254ull);
    const double xn = __longlong_as_double((long long)((z & 0x800FFFFFFFFFFFFFull) | (en << 52)));
    float split_hi, split_lo;
    f64_split(xn, &split_hi, &split_lo);
    const float hh = __double2float_rn(xn);
    const float hl = __double2float_rn(xn - (double)hh);
    const bool tiny = hl != 0.0f && fabsf(hl) < 1.17549435e-38f;
    local += !same_f32(split_hi, hh) || (!tiny && !same_f32(split_lo, hl));
    const float fs = __uint_as_float((unsigned)(z >> 32) & 0x807FFFFFu);  // subnormal or zero
    local += !same_f64(f32_to_f64(fs), (double)fs);
  }
  if (local) atomicAdd(bad, local);
}

static int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CFS_OK : CFS_ECUDA; }

// Reads back the max-norm word (one synchronisation of st).
static int read_max(cfs_plan* P, cudaStream_t st, float* out) {
  unsigned int bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, P->d_red, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CFS_ECUDA;
  memcpy(out, &bits, sizeof(float));
  return CFS_OK;
}

static unsigned int* max_word(cfs_plan* P) { return reinterpret_cast<unsigned int*>(P->d_red); }

// The running dz-weighted sum of the solution (after the plane partials).
static double* mean_num(cfs_plan* P) { return P->d_red + 2; }

int refine_poisson(cfs_plan* P, const double* f, double* p, cudaStream_t st) {
  const long long nxy = (long long)P->nx * P->ny;
  const unsigned grid = (unsigned)((nxy + kResBlock - 1) / kResBlock);
  const bool idx32 = res_idx32(P->nx, P->ny, P->nz);
  double* mean = nullptr;
  // one pass over f: r_0 = f as FP32, the extremes of r_0 and (Neumann) the
  // plane sums of the compatibility mean; then the reference norm
  // ||f - mean||_inf from the extremes and the mean
  const int nch = start_chunks(P->nz);
  cudaError_t e = cudaMemsetAsync(P->d_red, 0, 2 * sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    start_kernel<<<(unsigned)(P->nz * nch), 256, 0, st>>>(
        f, nxy, P->d_dzf, P->has_null ? P->d_red + 3 : nullptr, P->d_r32, max_word(P), nch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && P->has_null) {  // the dz-weighted mean of f (compatibility)
    mean = P->d_red + 1;
    mean_final_kernel<<<1, 256, 0, st>>>(P->d_red + 3, P->nz, nch, P->d_dzf, nxy, mean);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(mean_num(P), 0, sizeof(double), st);
  }
  double head[2] = {0.0, 0.0};  // the key words, the mean
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(head, P->d_red, sizeof(head), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int rc = cuda_rc(e);
  if (rc) return rc;
  unsigned int keys[2];
  memcpy(keys, &head[0], sizeof(keys));
  const double fmax = start_norm(keys, P->has_null ? head[1] : 0.0);
  P->last_iters = 0;
  P->last_rho = 0.0;
  if (fmax == 0.0) {  // zero right-hand side: zero solution
    return cuda_rc(cudaMemsetAsync(p, 0, sizeof(double) * (size_t)nxy * P->nz, st));
  }
  for (int it = 0; it < P->maxit; ++it) {
    // delta = solve32(r) in the workspace W (the right-hand side of the later
    // iterations comes from r32b); p (+)= delta fused into the last pass,
    // which also leaves delta in W for the residual update.  The second
    // solve works in w2, so that the first correction stays in r32 for the
    // pass that writes p = both corrections once.
    float* const W = (it == 1) ? P->d_w2 : P->d_r32;
    e = launch_rfft_x32(P, it >= 1 ? P->d_r32b : P->d_r32, W, false, st);
    if (e == cudaSuccess) e = launch_fft_y32(P, W, false, st);
    if (e == cudaSuccess) e = launch_thomas32(P, W, st);
    if (e == cudaSuccess) e = launch_fft_y32(P, W, true, st);
    // the first correction stays in FP32; the second pass writes p = both
    // once, later passes add to p
    const double* msum = P->has_null ? mean_num(P) : nullptr;
    if (e == cudaSuccess) {
      if (it == 0) e = launch_rfft_x32(P, W, W, true, st);
      else if (it == 1) e = launch_rfft_x32_sum(P, W, p, P->d_r32, st, msum);
      else e = launch_rfft_x32_to64(P, W, p, true, st, msum);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_red, 0, sizeof(unsigned int), st);
    // (Neumann: each kernel also sums its correction, dz-weighted, per block)
    double* mpart = P->has_null ? P->d_mpart : nullptr;
    if (e == cudaSuccess && it == 0) {  // r = (f - mean) - L delta, by differences
      auto k = idx32 ? poisson_first_kernel<int> : poisson_first_kernel<long long>;
      k<<<grid, kResBlock, 0, st>>>(f, mean, W, P->d_r32b, P->d_rlo, P->d_zk, max_word(P),
                                    P->nx, P->ny, P->nz, P->ybc, mpart, nullptr);
      e = cudaGetLastError();
    } else if (e == cudaSuccess) {  // r -= L delta
      auto k = idx32 ? poisson_update_kernel<int> : poisson_update_kernel<long long>;
      k<<<grid, kResBlock, 0, st>>>(W, P->d_r32b, P->d_rlo, P->d_zk, max_word(P), P->nx, P->ny,
                                    P->nz, P->ybc, mpart);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && mpart) {  // the weighted sum of p, correction by correction
      mean_acc_kernel<<<1, 256, 0, st>>>(mpart, (int)grid, mean_num(P));
      e = cudaGetLastError();
    }
    float rmax = 0.0f;
    rc = cuda_rc(e);
    if (!rc) rc = read_max(P, st, &rmax);
    if (rc) return rc;
    P->last_iters = it + 1;
    P->last_rho = (double)rmax / (double)fmax;
    if (P->last_rho <= P->tol) break;
  }
  if (P->last_iters == 1) {
    // p is still the first correction, in FP32: written here.  The residual
    // cannot see a constant, so the FP32 rounding of each correction's mean
    // would accumulate unchecked.  p is the sum of the corrections (each
    // added in FP64), so its dz-weighted sum is the sum of theirs,
    // accumulated by the residual kernels that read every correction
    // (double-float per column, FP64 across columns, in a fixed order).  Each
    // correction pass after the first subtracts the mean so far from its
    // correction; what is left is the mean of the last correction, at the
    // FP32 rounding of a correction that is itself small.  A solve that
    // stopped after its first FP32 solve has the mean of that solve left:
    // it is removed here (Neumann).
    if (P->has_null) mean_from_num_kernel<<<1, 32, 0, st>>>(mean_num(P), P->inv_wn, P->d_red + 1);
    first_only_kernel<<<1216, 256, 0, st>>>(p, P->d_r32, nxy * P->nz,
                                            P->has_null ? P->d_red + 1 : nullptr);
    rc = cuda_rc(cudaGetLastError());
    if (rc) return rc;
  }
  return (P->last_rho <= P->tol) ? CFS_OK : CFS_ENOTCONVERGED;
}

// The refined Helmholtz solve in one pass over the field (pcr.cu): one
// launch, then one read of the three result words (one synchronisation).
static int refine_helmholtz_fused(cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                                  cudaStream_t st) {
  unsigned int* words = max_word(P);  // three words at the start of the plan's scratch
  cudaError_t e = cudaMemsetAsync(words, 0, 3 * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = launch_pcr_refine(P, h, rhs, u, words, st);
  unsigned int w[3] = {0u, 0u, 0u};
  if (e == cudaSuccess) e = cudaMemcpyAsync(w, words, sizeof(w), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaErrorInvalidValue) return CFS_EINVAL;
  if (e != cudaSuccess) return CFS_ECUDA;
  float rmax, amax;
  memcpy(&rmax, &w[0], sizeof(float));
  memcpy(&amax, &w[1], sizeof(float));
  P->last_iters = (int)w[2];
  P->last_rho = amax > 0.0f ? (double)rmax / (double)amax : 0.0;
  return (P->last_rho <= P->tol) ? CFS_OK : CFS_ENOTCONVERGED;
}

int refine_helmholtz(cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                     cudaStream_t st) {
  if (pcr_refine_fits(P, h)) return refine_helmholtz_fused(P, h, rhs, u, st);
  const long long ncols = (long long)P->nx * P->ny;
  const unsigned grid = (unsigned)((ncols + kResBlock - 1) / kResBlock);
  auto residual = [&](int mode) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(P->d_red, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    helm_residual_kernel<<<grid, kResBlock, 0, st>>>(rhs, u, P->d_r32, h.d_abc, max_word(P), ncols,
                                                     h.n, P->nz, mode);
    return cudaGetLastError();
  };
  float fmax = 0.0f;
  int rc = cuda_rc(residual(0));  // r_0 = rhs
  if (!rc) rc = read_max(P, st, &fmax);
  if (rc) return rc;
  P->last_iters = 0;
  P->last_rho = 0.0;
  if (fmax == 0.0f)
    return cuda_rc(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)ncols * P->nz, st));
  for (int it = 0; it < P->maxit; ++it) {
    cudaError_t e = launch_helm32(P, h, P->d_r32, P->d_r32, st);
    if (e == cudaSuccess) e = residual(it == 0 ? 1 : 2);
    float rmax = 0.0f;
    rc = cuda_rc(e);
    if (!rc) rc = read_max(P, st, &rmax);
    if (rc) return rc;
    P->last_iters = it + 1;
    P->last_rho = (double)rmax / (double)fmax;
    if (P->last_rho <= P->tol) return CFS_OK;
  }
  return CFS_ENOTCONVERGED;
}

}  // namespace chanfs

extern "C" int cfs_selfcheck_conversions(unsigned long long samples,
                                         unsigned long long* mismatches) {
  chanfs::CaptureLock lock(chanfs::capture_mutex());
  if (!mismatches || samples == 0) return CFS_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    chanfs::conversion_check_kernel<<<1216, 256>>>(samples, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(mismatches, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
}
