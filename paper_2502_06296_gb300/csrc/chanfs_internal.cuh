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
constexpr int kPcrMaxParts = 32;   // warps of the PCR kernel
constexpr int kPcrMaxRows = 32;    // rows held in registers per partition
constexpr int kPcrMaxPartsWide = 12;  // warps when a partition has 17..32 rows

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

// Small DFTs in registers.  Forward kernel e^{-2 pi i / R}, inverse e^{+}.
template <bool INV>
__device__ __forceinline__ void dft2(double2& a, double2& b) {
  double2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(double2& a, double2& b, double2& c) {
  const double h = 0.8660254037844386467637231707529362;  // sqrt(3)/2
  double2 s = cadd(b, c);
  double2 d = csub(b, c);
  double2 t = make_double2(fma(-0.5, s.x, a.x), fma(-0.5, s.y, a.y));
  a = cadd(a, s);
  // forward: y1 = t - i h d, y2 = t + i h d
  double sx = INV ? -h : h;
  b = make_double2(fma(sx, d.y, t.x), fma(-sx, d.x, t.y));
  c = make_double2(fma(-sx, d.y, t.x), fma(sx, d.x, t.y));
}

template <bool INV>
__device__ __forceinline__ void dft4(double2& a0, double2& a1, double2& a2, double2& a3) {
  double2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  double2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft8(double2* v) {
  const double r = 0.7071067811865475244008443621048490;  // 1/sqrt(2)
  double2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  double2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o1 *= W8^1, o2 *= W8^2 = -i, o3 *= W8^3 (forward); conjugates for inverse
  double2 w1, w3;
  if (!INV) {
    w1 = make_double2((o1.x + o1.y) * r, (o1.y - o1.x) * r);
    w3 = make_double2((o3.y - o3.x) * r, -(o3.x + o3.y) * r);
  } else {
    w1 = make_double2((o1.x - o1.y) * r, (o1.y + o1.x) * r);
    w3 = make_double2(-(o3.x + o3.y) * r, (o3.x - o3.y) * r);
  }
  double2 w2 = mul_mi<INV>(o2);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1);
  v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2);
  v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3);
  v[7] = csub(e3, w3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(double2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
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
    const double2* w = tw + k * (R - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = INV ? cmulc(v[r], w[r - 1]) : cmul(v[r], w[r - 1]);
  }
  dft<R, INV>(v);
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
