// chanfs_internal.cuh -- types and device helpers shared by the CUDA
// translation units of libchanfs (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/chanfs.h"

namespace chanfs {

// ----------------------------------------------------------------------------
// Limits
// ----------------------------------------------------------------------------
constexpr int kMaxPasses = 16;     // radix passes of one FFT
constexpr int kMaxNx = 4096;       // x cells (complex length nx/2 <= 2048)
constexpr int kMaxNy = 1024;       // y cells
constexpr int kMaxNz = 16384;      // z cells
constexpr int kPcrMaxParts = 64;   // z-partitions (half-warps) of the PCR kernel
constexpr int kPcrMaxUnknowns = 1024;  // rows of a PCR tile in shared memory

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
bool make_fft_desc(int n, FftDesc* d, std::vector<double2>* tw);

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
  unsigned long long stamp;
};

}  // namespace chanfs

// ----------------------------------------------------------------------------
// The plan (opaque in the public header).
// ----------------------------------------------------------------------------
struct cfs_plan {
  int device;
  int nx, ny, nz, M;  // M = nx/2 complex points per packed x-line
  int nky;            // ky pairs handled by the Thomas kernel: ny/2 + 1
  double lx, ly;
  int bc;
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
  double* d_dzf;     // cell widths (weights of the Neumann mean)
  // Neumann (0,0) column: wn = w/sum(w), gn = g/sum(w) with g = T'^{-T} w,
  // hs = sc * T'^{-1} (0,1,..,1), T' the pinned operator; 3*nz doubles
  double* d_sing;
  double sing_cg, sing_sc;
  // Helmholtz cache
  std::vector<chanfs::HelmCoef> helm;
  unsigned long long helm_clock;
  // host-buffer staging
  double* d_stage;
  // device status word
  int* d_status;
  size_t device_bytes;
};

namespace chanfs {

// ----------------------------------------------------------------------------
// Kernel launchers (one per translation unit)
// ----------------------------------------------------------------------------
cudaError_t launch_rfft_x(const cfs_plan* P, const double* in, double* out, bool inverse,
                          double scale, cudaStream_t st);
cudaError_t launch_fft_y(const cfs_plan* P, double* data, bool inverse, cudaStream_t st);
cudaError_t launch_thomas(const cfs_plan* P, double* data, cudaStream_t st);
cudaError_t launch_thomas_factor(cfs_plan* P, const double* dA, const double* dB,
                                 const double* dC, const double* dlamx, const double* dlamy,
                                 cudaStream_t st);
cudaError_t launch_pcr(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       cudaStream_t st);
size_t pcr_smem_bytes(int n, int nparts);

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// a * w (4 FP64 instructions) and a * conj(w).
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
// Multiply by -i (forward) or +i (inverse): a swap and a sign, no arithmetic.
template <bool INV>
__device__ __forceinline__ double2 mul_mi(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// a + w x with fused multiply-adds (4 FP64 instructions); w is conjugated for
// the inverse transform.
template <bool INV>
__device__ __forceinline__ double2 cfma(double2 w, double2 x, double2 a) {
  if (INV)
    return make_double2(fma(w.x, x.x, fma(w.y, x.y, a.x)), fma(w.x, x.y, fma(-w.y, x.x, a.y)));
  return make_double2(fma(w.x, x.x, fma(-w.y, x.y, a.x)), fma(w.x, x.y, fma(w.y, x.x, a.y)));
}
template <bool INV>
__device__ __forceinline__ double2 ctw(double2 x, double2 w) {
  return INV ? cmulc(x, w) : cmul(x, w);
}
// 2a - s (2 FP64 instructions): the difference partner of s = a + t.
__device__ __forceinline__ double2 ctwice_minus(double2 a, double2 s) {
  return make_double2(fma(2.0, a.x, -s.x), fma(2.0, a.y, -s.y));
}

// Small DFTs in registers.  Forward kernel e^{-2 pi i / R}, inverse e^{+}.
// The *_tw variants take the inputs before their Stockham twiddles w[r-1]
// (r >= 1) and fold each twiddle product into the first butterfly level:
//   (a + w x, a - w x) = (s, 2a - s) with s = a + w x by four FMAs,
// 6 FP64 instructions per pair instead of 8.
template <bool INV>
__device__ __forceinline__ void dft2(double2& a, double2& b) {
  double2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft2_tw(double2* v, const double2* w) {
  double2 s = cfma<INV>(w[0], v[1], v[0]);
  v[1] = ctwice_minus(v[0], s);
  v[0] = s;
}

// y0 = a + s, y1,2 = (a - s/2) -/+ i (sqrt3/2) d  with s = b + c, d = b - c.
template <bool INV>
__device__ __forceinline__ void dft3_core(double2& a, double2& b, double2& c, double2 s, double2 d) {
  const double h = 0.8660254037844386467637231707529362;  // sqrt(3)/2
  double2 t = make_double2(fma(-0.5, s.x, a.x), fma(-0.5, s.y, a.y));
  a = cadd(a, s);
  const double sx = INV ? -h : h;
  b = make_double2(fma(sx, d.y, t.x), fma(-sx, d.x, t.y));
  c = make_double2(fma(-sx, d.y, t.x), fma(sx, d.x, t.y));
}

template <bool INV>
__device__ __forceinline__ void dft3(double2& a, double2& b, double2& c) {
  dft3_core<INV>(a, b, c, cadd(b, c), csub(b, c));
}

template <bool INV>
__device__ __forceinline__ void dft3_tw(double2* v, const double2* w) {
  double2 b = ctw<INV>(v[1], w[0]);
  double2 s = cfma<INV>(w[1], v[2], b);
  double2 d = ctwice_minus(b, s);
  dft3_core<INV>(v[0], v[1], v[2], s, d);
}

// Radix-4 second level from t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3,
// d = a1 - a3.
template <bool INV>
__device__ __forceinline__ void dft4_core(double2* y, double2 t0, double2 t1, double2 t2, double2 d) {
  double2 t3 = mul_mi<INV>(d);
  y[0] = cadd(t0, t2);
  y[2] = csub(t0, t2);
  y[1] = cadd(t1, t3);
  y[3] = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(double2& a0, double2& a1, double2& a2, double2& a3) {
  double2 y[4];
  dft4_core<INV>(y, cadd(a0, a2), csub(a0, a2), cadd(a1, a3), csub(a1, a3));
  a0 = y[0]; a1 = y[1]; a2 = y[2]; a3 = y[3];
}

// DFT4 of (x0, w1 x1, w2 x2, w3 x3) given x0..x3 and w1..w3 (x0 untwiddled).
template <bool INV>
__device__ __forceinline__ void dft4_tw4(double2* y, double2 x0, double2 x1, double2 x2, double2 x3,
                                         double2 w1, double2 w2, double2 w3) {
  double2 t0 = cfma<INV>(w2, x2, x0);
  double2 t1 = ctwice_minus(x0, t0);
  double2 u = ctw<INV>(x1, w1);
  double2 t2 = cfma<INV>(w3, x3, u);
  dft4_core<INV>(y, t0, t1, t2, ctwice_minus(u, t2));
}

template <bool INV>
__device__ __forceinline__ void dft4_tw(double2* v, const double2* w) {
  double2 y[4];
  dft4_tw4<INV>(y, v[0], v[1], v[2], v[3], w[0], w[1], w[2]);
  v[0] = y[0]; v[1] = y[1]; v[2] = y[2]; v[3] = y[3];
}

// Radix-2 combination of the even (E) and odd (O) half-DFTs of a DFT8, with
// the W8 factors folded into fused multiply-adds.
template <bool INV>
__device__ __forceinline__ void dft8_combine(double2* v, const double2* E, const double2* O) {
  const double r = 0.7071067811865475244008443621048490;  // 1/sqrt(2)
  v[0] = cadd(E[0], O[0]);
  v[4] = csub(E[0], O[0]);
  double2 m2 = mul_mi<INV>(O[2]);
  v[2] = cadd(E[2], m2);
  v[6] = csub(E[2], m2);
  if (!INV) {
    // W8 O = r (O.x + O.y, O.y - O.x);  W8^3 O = r (O.y - O.x, -(O.x + O.y))
    double p1 = O[1].x + O[1].y, q1 = O[1].y - O[1].x;
    v[1] = make_double2(fma(r, p1, E[1].x), fma(r, q1, E[1].y));
    v[5] = make_double2(fma(-r, p1, E[1].x), fma(-r, q1, E[1].y));
    double p3 = O[3].y - O[3].x, q3 = O[3].x + O[3].y;
    v[3] = make_double2(fma(r, p3, E[3].x), fma(-r, q3, E[3].y));
    v[7] = make_double2(fma(-r, p3, E[3].x), fma(r, q3, E[3].y));
  } else {
    // W8^-1 O = r (O.x - O.y, O.x + O.y);  W8^-3 O = r (-(O.x + O.y), O.x - O.y)
    double p1 = O[1].x - O[1].y, q1 = O[1].x + O[1].y;
    v[1] = make_double2(fma(r, p1, E[1].x), fma(r, q1, E[1].y));
    v[5] = make_double2(fma(-r, p1, E[1].x), fma(-r, q1, E[1].y));
    double q3 = O[3].x + O[3].y, p3 = O[3].x - O[3].y;
    v[3] = make_double2(fma(-r, q3, E[3].x), fma(r, p3, E[3].y));
    v[7] = make_double2(fma(r, q3, E[3].x), fma(-r, p3, E[3].y));
  }
}

template <bool INV>
__device__ __forceinline__ void dft8(double2* v) {
  double2 E[4], O[4];
  dft4_core<INV>(E, cadd(v[0], v[4]), csub(v[0], v[4]), cadd(v[2], v[6]), csub(v[2], v[6]));
  dft4_core<INV>(O, cadd(v[1], v[5]), csub(v[1], v[5]), cadd(v[3], v[7]), csub(v[3], v[7]));
  dft8_combine<INV>(v, E, O);
}

template <bool INV>
__device__ __forceinline__ void dft8_tw(double2* v, const double2* w) {
  double2 E[4], O[4];
  // even half: (v0, w2 v2, w4 v4, w6 v6)
  dft4_tw4<INV>(E, v[0], v[2], v[4], v[6], w[1], w[3], w[5]);
  // odd half: all four twiddled
  double2 a = ctw<INV>(v[1], w[0]);
  double2 t0 = cfma<INV>(w[4], v[5], a);
  double2 t1 = ctwice_minus(a, t0);
  double2 b = ctw<INV>(v[3], w[2]);
  double2 t2 = cfma<INV>(w[6], v[7], b);
  dft4_core<INV>(O, t0, t1, t2, ctwice_minus(b, t2));
  dft8_combine<INV>(v, E, O);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(double2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_tw(double2* v, const double2* w) {
  if constexpr (R == 2) dft2_tw<INV>(v, w);
  else if constexpr (R == 3) dft3_tw<INV>(v, w);
  else if constexpr (R == 4) dft4_tw<INV>(v, w);
  else if constexpr (R == 8) dft8_tw<INV>(v, w);
}

// One Stockham radix-R butterfly: reads R points j + r*n/R of one batch from
// `in`, applies the twiddles of pass (L, R), transforms, and writes them to
// positions (j - k)*R + k + r*L of `out` (k = j mod L).  es = element stride.
template <int R, bool INV>
__device__ __forceinline__ void stockham_bfly(const double2* __restrict__ in,
                                              double2* __restrict__ out, int j, int L,
                                              int n, int es, const double2* __restrict__ tw) {
  double2 v[R];
  const int q = n / R;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[(j + r * q) * es];
  const int k = j % L;
  if (L > 1) {
    double2 w[R - 1];
#pragma unroll
    for (int r = 0; r < R - 1; ++r) w[r] = tw[k * (R - 1) + r];
    dft_tw<R, INV>(v, w);
  } else {
    dft<R, INV>(v);
  }
  const int o = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[(o + r * L) * es] = v[r];
}

// All passes of an FFT over `nb` batches held in shared memory.  Element e of
// batch b lives at buf[b*bs + e*es].  Ping-pongs between a and b; returns the
// buffer holding the result.  BATCH_FAST: consecutive threads take consecutive
// batches (columns of a y tile) instead of consecutive butterflies.
template <bool INV, bool BATCH_FAST>
__device__ double2* stockham_smem(double2* a, double2* b, const FftDesc& d, int nb, int es,
                                  int bs, const double2* __restrict__ tw) {
  const int n = d.n;
  for (int p = 0; p < d.npass; ++p) {
    const int R = d.radix[p], L = d.span[p];
    const double2* twp = tw + d.twoff[p];
    const int nbf = n / R;
    const int total = nbf * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      int bat, j;
      if (BATCH_FAST) {
        bat = t % nb;
        j = t / nb;
      } else {
        j = t % nbf;
        bat = t / nbf;
      }
      const double2* in = a + bat * bs;
      double2* out = b + bat * bs;
      switch (R) {
        case 8: stockham_bfly<8, INV>(in, out, j, L, n, es, twp); break;
        case 4: stockham_bfly<4, INV>(in, out, j, L, n, es, twp); break;
        case 3: stockham_bfly<3, INV>(in, out, j, L, n, es, twp); break;
        default: stockham_bfly<2, INV>(in, out, j, L, n, es, twp); break;
      }
    }
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
  }
  return a;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

#endif  // __CUDACC__

}  // namespace chanfs
