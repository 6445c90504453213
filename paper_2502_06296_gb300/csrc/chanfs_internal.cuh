// chanfs_internal.cuh -- types and device helpers shared by the CUDA
// translation units of libchanfs (not part of the public ABI).
#pragma once

#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/chanfs.h"

namespace chanfs {

// Serialises CUDA graph captures with the library calls that synchronise the
// whole device or allocate and free device memory (plan creation and
// destruction, coefficient caches, tuning, group set-up): such a call from
// one thread while another thread captures a graph would invalidate the
// capture.  Recursive: those calls nest.
std::recursive_mutex& capture_mutex();
using CaptureLock = std::lock_guard<std::recursive_mutex>;

// ----------------------------------------------------------------------------
// Limits
// ----------------------------------------------------------------------------
constexpr int kMaxPasses = 16;     // radix passes of one FFT
constexpr int kMaxNx = 4096;       // x cells (complex length nx/2 <= 2048)
constexpr int kMaxNy = 4096;       // y cells (a y tile of one FP64 column fits in shared memory)
constexpr int kMaxNz = 16384;      // z cells
constexpr int kPcrMaxParts = 64;   // z-partitions (half-warps) of the PCR kernel
constexpr int kPcrMaxUnknowns = 1024;  // rows of a PCR tile in shared memory

constexpr int kMaxGroup = 4096;     // plans of one grouped solve
constexpr int kBatchSlots = 4;      // device slots of a batch of host-buffer solves
constexpr int kMaxStreamChunks = 8; // chunks a field of a streamed batch moves in
// Default levels of CFS_OPT_F64_ADDS_X / _Y (FP64 butterfly additions on the
// integer units).
constexpr int kEmuDefaultX = 0;
constexpr int kEmuDefaultY = 0;

// Device status bits (plan->d_status)
constexpr int kErrTmaTimeout = 1;

// ----------------------------------------------------------------------------
// FFT description: a length-n complex FFT as Stockham radix passes.
// Pass p has radix radix[p] and span span[p] (product of the radices of the
// passes before it); its twiddles W_{span*radix}^{r k}, k < span, 1 <= r < radix,
// are at tw[twoff[p] + k*(radix-1) + r-1] (forward sign; the inverse uses the
// conjugate).
// ----------------------------------------------------------------------------
struct FftDesc {
  int n;
  int npass;
  int ntw;  // complex entries in the twiddle table
  int radix[kMaxPasses];
  int span[kMaxPasses];
  int twoff[kMaxPasses];
};

// Builds the radix plan and its FP64 twiddle table on the host.
// Passes of radix 8 (max_radix 8) or 4 first, then at most one 2, then 3s.
bool make_fft_desc(int n, FftDesc* d, std::vector<double2>* tw, int max_radix);

// ----------------------------------------------------------------------------
// Helmholtz coefficient set for Algorithm 2 (one (c, loc, nparts) entry).
// Device arrays (n = rows): alpha[i] = A_i / b_{i-1}, beta[i] = C_i / b_{i+1},
// ib[i] = 1/b_i, ap[i] = a_i/b_i, cp[i] = c_i/b_i (partition-local recurrences
// of Algorithm 2, indexed by global row), and the LU factors of the reduced
// 2*nparts system: rl[j] (sub-diagonal multipliers), rip[j] (inverse pivots),
// ripc[j] (super-diagonal times inverse pivot).
// ----------------------------------------------------------------------------
struct HelmCoef {
  double c;
  int loc;
  int nparts;
  int n;       // unknowns per column (nz or nz-1)
  int mmax;    // largest partition
  int start[kPcrMaxParts + 1];
  double* d_rows;  // 5*n doubles: alpha | beta | ib | ap | cp
  double* d_red;   // 3*(2*nparts) doubles: rl | rip | ripc
  float* d_rows32; // FP32 copies (refined plans)
  float* d_red32;
  double* d_abc;   // 3*n doubles: A' | B' | C' of I - c L_z (refinement residual)
  double* d_th;    // 3*n doubles: Thomas factors fs | fa | fc of I - c L_z
  float* d_th32;   // FP32 copies (refined plans)
  float* d_lv32;   // refined plans: parallel reduction of the reduced system,
                   // K1 (L x 2p) | K2 (L x 2p) | 1/diag (2p), L = ceil(log2 2p)
  unsigned long long stamp;
};

// LU factors of the fully implicit Helmholtz systems of Eq. 8 for one
// (c, loc): per (kx, ky pair, k) the same layout as the Poisson factors, over
// the n = nz (centred) or nz - 1 (face) Dirichlet rows.
struct Helm3Coef {
  double c;
  int loc;
  int n;
  double2* d_fwd;
  double* d_bwd;
  unsigned long long stamp;
};

// Chunks per z plane of the refined Poisson start pass (refine.cu): about
// 2432 blocks (16 per SM) over the nz planes, at most kMaxStartChunks.
constexpr int kMaxStartChunks = 16;
// Rows appended to the FP32 z-operator table for the partitioned z solve (its
// partitions have 8 or 16 rows; the last one may extend past nz).
constexpr int kZPartRowPad = 16;
inline __host__ __device__ int start_chunks(int nz) {
  const int c = (2432 + nz - 1) / nz;
  return c < 1 ? 1 : (c > kMaxStartChunks ? kMaxStartChunks : c);
}

}  // namespace chanfs

// ----------------------------------------------------------------------------
// The plan (opaque in the public header).
// ----------------------------------------------------------------------------
struct cfs_plan {
  int device;
  int nx, ny, nz, M;  // M = nx/2 complex points per packed x-line
  int nky;            // ky rows of the factor tables: ny/2 + 1 pairs (periodic y), else ny
  double lx, ly;
  int bc;
  int ybc;            // y: CFS_Y_PERIODIC, CFS_Y_NEUMANN or CFS_Y_DIRICHLET
  int has_null;       // Neumann z walls with Neumann or periodic y: constants are the null space
  double2* d_wy;      // y walls: exp(-i pi k / 2 Ny), k < Ny (FP32 copy d_wy32)
  float2* d_wy32;
  std::vector<double> dzf;  // host copy of the cell widths
  // FFT plans and tables
  chanfs::FftDesc fx, fy;
  double2* d_twx;    // fx twiddles
  double2* d_twy;    // fy twiddles
  double2* d_post;   // 0.5 * W_nx^k, k = 0..M/2 (real-FFT post-processing)
  // y-tile geometry
  int tk;            // complex columns per y tile
  int by, nbox;      // rows per TMA box, boxes per tile
  // Thomas factors of Eq. 12, per (kx in [0,M], kyp in [0,nky), k):
  double2* d_fwd;    // (s/piv_k, A_k/piv_k)
  double* d_bwd;     // C_k/piv_k
  int thomas_tw;     // columns per shared-memory Thomas tile: 0 automatic,
                     // 8 or 16 forced, -1 the streaming kernel, 1 the partitioned
                     // FP32 solve (Algorithm 2 in registers)
  int x_lines;       // x-lines per CTA of the x transforms (0: about 16 KB of data)
  int tk_auto, tk32_auto;  // y tile widths chosen at creation
  int pcr_parts;     // partitions of Helmholtz sets prepared without a count (0: auto)
  int helm_fp64;     // refined plans: Helmholtz by FP64 Algorithm 2 directly, no refinement
  int helm_thomas;   // FP64 Helmholtz solves by Thomas sweeps instead of Algorithm 2
  int helm_thomas32; // FP32 inner Helmholtz solves of refinement by Thomas sweeps
  int fft_radix;     // largest radix of the x and y FFT passes (8 or 4)
  int emu_x, emu_y;  // FP64 x / y transforms: levels 0..4 of butterfly additions
                     // on the integer units (CFS_OPT_F64_ADDS_X / _Y)
  double* d_dzf;     // cell widths (weights of the Neumann mean)
  // Neumann (0,0) column: wn = w/sum(w), gn = g/sum(w) with g = T'^{-T} w,
  // hs = sc * T'^{-1} (0,1,..,1), T' the pinned operator; 3*nz doubles
  double* d_sing;
  double sing_cg, sing_sc;
  // ---- FP32 + FP64 iterative refinement (dtype CFS_F32_REFINED) ----
  int dtype;
  float2* d_twx32;   // FP32 copies of the twiddle tables
  float2* d_twy32;
  float2* d_post32;
  int tk32;          // complex columns per FP32 y tile (even: 16-byte TMA boxes)
  float2* d_fwd32;   // FP32 copies of the Thomas factors
  float* d_bwd32;
  int kx64, ky64;    // columns kx < kx64, min(ky, Ny-ky) < ky64 stay FP64
  float4* d_zrow32;  // (A_k, B_k, C_k, 1) of the z operator in FP32, then kZPartRowPad
                     // identity rows (0, 1, 0, 0) (partitioned z solve, thomas.cu)
  float* d_lam32;    // lx[0..M] then ly[0..nky) in FP32
  float* d_r32;      // FP32 residual / correction field (in-place inner solve)
  float* d_r32b;     // the residual kept between iterations, high part (FP32 input of the
                     // next solve)
  float* d_rlo;      // its low part: the double-float residual is (d_r32b, d_rlo)
  float* d_w2;       // single solves: the second FP32 solve's workspace (the first correction
                     // stays in d_r32); grouped solves: a copy of the first correction
  float4* d_zk;      // per plane k, split hi + lo: (A_k, C_k), (B'_k, dz_k), (D_k, dz_k); then
                     // (1/dx^2, 1/dy^2).  D_k = A_k + B'_k + C_k + 2/dx^2 + 2/dy^2 (exact sum)
  double* d_mpart;   // per-block dz-weighted sums of a correction (residual grid blocks)
  double inv_wn;     // 1 / (sum of the cell widths * Nx * Ny)
  double* d_red;     // reduction scratch: [0] two 32-bit words (max |r| as float bits; the
                     // start pass's extreme keys), [1] mean, [2] running weighted sum of
                     // the solution, [3..) nz * start_chunks(nz) plane partials
  double tol;        // relative residual target
  int maxit;         // at most this many corrections
  int last_iters;
  double last_rho;
  // Helmholtz cache
  std::vector<chanfs::HelmCoef> helm;
  std::vector<chanfs::Helm3Coef> helm3;  // fully implicit 3-D sets (LRU, small)
  std::vector<double> lamx_h, lamy_h;     // eigenvalues per kx in [0, M], ky pair
  unsigned long long helm_clock;
  // host-buffer staging
  double* d_stage;
  // batched host-buffer solves: up to kBatchSlots slots of (input, output)
  // device fields (as many as the largest batch so far), a copy-in stream,
  // a second compute stream and a copy-out stream per compute stream, and
  // their events (created at the first batch)
  double* d_batch;
  int batch_slots;
  cudaStream_t copy_in, copy_out, copy_out2, compute2;
  cudaEvent_t ev_entry, ev_done[chanfs::kBatchSlots], ev_free[chanfs::kBatchSlots];
  // streamed FP64 batches: per slot, a chunk's input landed / its result is ready
  cudaEvent_t ev_cin[chanfs::kBatchSlots][chanfs::kMaxStreamChunks];
  cudaEvent_t ev_cdone[chanfs::kBatchSlots][chanfs::kMaxStreamChunks];
  int stream_chunks;  // CFS_OPT_STREAM_CHUNKS (0 automatic)
  // device status word
  int* d_status;
  // work buffers allocated with guard words: (allocation base, payload bytes)
  std::vector<std::pair<unsigned char*, size_t>> guarded;
  size_t device_bytes;
};

namespace chanfs {

// ----------------------------------------------------------------------------
// Kernel launchers (one per translation unit)
// ----------------------------------------------------------------------------
// nlines >= 0: only the first nlines x lines of in / out (a range of z planes
// when in and out point at its first plane); -1: every line of the field.
cudaError_t launch_rfft_x(const cfs_plan* P, const double* in, double* out, bool inverse,
                          double scale, cudaStream_t st, long long nlines = -1);
cudaError_t launch_fft_y(const cfs_plan* P, double* data, bool inverse, cudaStream_t st);
cudaError_t launch_thomas(const cfs_plan* P, double* data, cudaStream_t st);
cudaError_t launch_rfft_x32(const cfs_plan* P, const float* in, float* out, bool inverse,
                            cudaStream_t st);
// add: p += delta (less msum * inv_wn when msum is not null), else p = delta
cudaError_t launch_rfft_x32_to64(const cfs_plan* P, const float* in, double* out, bool add,
                                 cudaStream_t st, const double* msum = nullptr);
// the second correction pass: p = first + delta (less msum * inv_wn when msum
// is not null), with delta left in `in`; p is not read
cudaError_t launch_rfft_x32_sum(const cfs_plan* P, const float* in, double* out,
                                const float* first, cudaStream_t st,
                                const double* msum = nullptr);
cudaError_t launch_fft_y32(const cfs_plan* P, float* data, bool inverse, cudaStream_t st);
cudaError_t launch_thomas32(const cfs_plan* P, float* data, cudaStream_t st);
// x-lines per CTA of the x transforms of complex element size csize.
int x_lines_per_cta(const cfs_plan* P, size_t csize);
size_t x_smem_bytes(const cfs_plan* P, int lines, size_t csize);
// Whether tk columns per y tile can run (alignment, shared memory).
bool y_tile_ok(const cfs_plan* P, int tk, bool fp32);
// Thomas tile width the plan's solves use (8, 16, or -1 for the streaming
// kernel), for the FP64 or the FP32 spectrum; 0 if `tw` cannot run.
int thomas_tile_width(const cfs_plan* P, bool fp32, int tw);
// Factors of n-row systems with diagonal B_k + lx[kx] + ly[kyp] (no pinned
// column) into fwd/bwd; s = 2 / (Nx Ny) folded in as for the Poisson set.
cudaError_t launch_thomas_factor_set(const cfs_plan* P, double2* fwd, double* bwd, int n,
                                     const double* dA, const double* dB, const double* dC,
                                     const double* dlx, const double* dly, cudaStream_t st);
// The FP64 z sweeps with another factor set over n rows (no pinned column).
cudaError_t launch_thomas_set(const cfs_plan* P, double* data, const double2* fwd,
                              const double* bwd, int n, cudaStream_t st);
cudaError_t launch_thomas_factor(cfs_plan* P, const double* dA, const double* dB,
                                 const double* dC, const double* dlamx, const double* dlamy,
                                 cudaStream_t st);
cudaError_t launch_pcr(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       cudaStream_t st);
// The columns [col0, col0 + ncols) of the (x, y) plane only (col0 even).
cudaError_t launch_pcr_cols(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                            long long col0, long long ncols, cudaStream_t st);
size_t pcr_smem_bytes(int n, int nparts);
cudaError_t launch_pcr_raw(long long ncols, int nz, int n, int nparts, int loc, const double* rows,
                           const double* red, const double* rhs, double* u, int* status,
                           cudaStream_t st);
// The Helmholtz systems by a Thomas sweep per column (helm_thomas.cu).
int plan_set_radix(cfs_plan* P, int max_radix);
cudaError_t launch_helm_thomas(const cfs_plan* P, const HelmCoef& h, const double* rhs,
                               double* u, cudaStream_t st);
cudaError_t launch_helm_thomas32(const cfs_plan* P, const HelmCoef& h, const float* rhs,
                                 float* u, cudaStream_t st);
// The plan's choice between them and Algorithm 2 (CFS_OPT_HELM_THOMAS for FP64
// solves, CFS_OPT_HELM_THOMAS32 for the FP32 inner solves of refinement).
cudaError_t launch_helm64(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                          cudaStream_t st);
cudaError_t launch_helm32(const cfs_plan* P, const HelmCoef& h, const float* rhs, float* u,
                          cudaStream_t st);
cudaError_t launch_pcr32(const cfs_plan* P, const HelmCoef& h, const float* rhs, float* u,
                         cudaStream_t st);
// Algorithm 2, Step 1 for (c, loc) on the plan, from its cache or computed
// and cached (plan.cu); nparts = 0 takes a cached set of any partition count.
int plan_helm_prepare(cfs_plan* P, double c, int loc, int nparts, HelmCoef** out);
void plan_helm_forget(cfs_plan* P, double c);
// Allocates the plan's FP64 staging field if it has none yet.
int plan_ensure_stage(cfs_plan* P);
// Iterative refinement drivers (refine.cu): FP32 inner solves, residuals in
// double-float (Poisson) or FP64 (Helmholtz), FP64 accumulation.  They
// synchronise `st` once per iteration.
int refine_poisson(cfs_plan* P, const double* f, double* p, cudaStream_t st);
int refine_helmholtz(cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                     cudaStream_t st);

// ----------------------------------------------------------------------------
// Device helpers (the FFT engine is in chanfs_fft.cuh)
// ----------------------------------------------------------------------------
#ifdef __CUDACC__

// Lets `kernel` launch with up to the per-block maximum of dynamic shared
// memory.  Always the same value: plans solved concurrently from several
// host threads must not lower the limit under one another's launches.
constexpr int kMaxDynSmem = 227 * 1024;
template <class K>
inline cudaError_t allow_max_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

// Conversions between FP32 and FP64 on the integer units.  On GB300 the
// hardware conversion instructions share the FP64 pipe (2 lanes per SM per
// clock), which the refinement kernels already saturate; these produce the
// values of IEEE 754 binary32 <-> binary64 conversion (round to nearest,
// ties to even) from the fields of the encodings alone, subnormals, infinities
// and out-of-range values included, so that no operand falls back to the
// hardware instruction (a fallback branch the compiler may turn into a select
// that runs the hardware conversion on every operand).  NaN maps to a quiet
// NaN of the same sign.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  unsigned hi = 0u, lo = 0u;
  if (a >= 0x00800000u) {  // normal, infinity or NaN: bias 127 -> 1023
    const unsigned e = a >> 23;
    hi = (e == 0xffu ? 0x7ff00000u : (e + 896u) << 20) | ((a >> 3) & 0xfffffu);
    lo = a << 29;
  } else if (a != 0u) {  // subnormal a * 2^-149: the leading bit moves to bit 23
    const unsigned sh = (unsigned)__clz((int)a) - 8u;
    const unsigned m = a << sh;
    hi = ((897u - sh) << 20) | ((m >> 3) & 0xfffffu);
    lo = m << 29;
  }
  return __hiloint2double((int)((u & 0x80000000u) | hi), (int)lo);
}

__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  unsigned bits;
  if (e >= 897u && e <= 1150u) {  // a normal binary32 (or its rounding overflows)
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the top 23 mantissa bits
    const unsigned rest = lo & 0x1fffffffu;                  // the 29 dropped bits
    bits = ((e - 896u) << 23) | m;
    // a carry out of the mantissa raises the exponent (to infinity past the
    // largest binary32)
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  } else if (e > 1150u) {  // too large, infinity or NaN
    bits = (e == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
  } else if (e == 0u) {  // binary64 zero or subnormal: rounds to zero
    bits = 0u;
  } else {  // a binary32 subnormal: significand * 2^(e - 1075) in units of 2^-149
    const unsigned sh = 926u - e;  // >= 30
    if (sh > 63u) {
      bits = 0u;  // below half the smallest subnormal
    } else {
      const unsigned long long M =
          (1ull << 52) | ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
      const unsigned long long q = M >> sh, r = M & ((1ull << sh) - 1ull);
      const unsigned long long half = 1ull << (sh - 1u);
      bits = (unsigned)(q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull));
    }
  }
  return __uint_as_float((hi & 0x80000000u) | bits);
}

// x as a double-float pair: hi = fl32(x) and lo = fl32(x - hi) (x - hi is
// exact in binary64), from the fields of x alone.  For x inside the normal
// binary32 range, x - hi is the 29 bits dropped by the rounding of hi, less
// 2^29 units if hi rounded up, so lo is that signed integer d times
// 2^(e - 1075), rounded to nearest even.  Outside that range lo is +0 (hi
// then carries x to binary32 precision, or x is below it); a lo below the
// normal binary32 range is a zero of its sign.
__device__ __forceinline__ void f64_split(double x, float* hi, float* lo) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned e = (hw >> 20) & 0x7ffu;
  *hi = f64_to_f32(x);
  unsigned lbits = 0u;
  if (e >= 897u && e <= 1150u) {
    const unsigned m = ((hw & 0xfffffu) << 3) | (lw >> 29);
    const unsigned rest = lw & 0x1fffffffu;
    const bool up = rest > 0x10000000u || (rest == 0x10000000u && (m & 1u));
    const int d = up ? (int)rest - 0x20000000 : (int)rest;  // |d| <= 2^28
    if (d != 0) {
      const unsigned a = d < 0 ? (unsigned)(-d) : (unsigned)d;
      const int lz = __clz((int)a);          // leading bit at 31 - lz
      const int ef = (int)e - 917 - lz;      // binary32 exponent field of a * 2^(e-1075)
      const unsigned neg = ((hw >> 31) ^ (d < 0 ? 1u : 0u)) & 1u;
      lbits = neg << 31;
      if (ef >= 1) {
        unsigned frac;
        if (lz >= 8) {  // at most 24 significant bits: exact
          frac = a << (lz - 8);
        } else {        // round the low 8 - lz bits away, ties to even
          const int sh = 8 - lz;
          const unsigned q = a >> sh, r = a & ((1u << sh) - 1u), half = 1u << (sh - 1);
          frac = q + ((r > half || (r == half && (q & 1u))) ? 1u : 0u);
        }
        // frac holds the significand with its leading bit at 23 (or 24
        // after a carry, which the exponent field below absorbs)
        lbits |= ((unsigned)ef << 23) + (frac - 0x800000u);
      }
    }
  }
  *lo = __uint_as_float(lbits);
}

// Double-float accumulation on the FP32 units (the refinement residuals).
struct DoubleFloat {
  float s, e;
};

// s + t = a + b exactly (Knuth's TwoSum); the _rn intrinsics keep the
// compiler from contracting or reassociating the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc (+)= (chi + clo) * d; INIT: acc = the product.
template <bool INIT = false>
__device__ __forceinline__ void df_acc(DoubleFloat& acc, float chi, float clo, float d) {
  const float p = __fmul_rn(chi, d);
  float e = __fmaf_rn(chi, d, -p);  // chi * d - p, exact
  e = __fmaf_rn(clo, d, e);
  if (INIT) {
    acc.s = p;
    acc.e = e;
  } else {
    float s, t;
    two_sum(acc.s, p, s, t);
    acc.s = s;
    acc.e = __fadd_rn(acc.e, __fadd_rn(t, e));
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

#endif  // __CUDACC__

}  // namespace chanfs
