// fft_x.cu -- real FFT along the contiguous x direction, packed output
// (App. A of the paper: n reals in, n reals out, X_{nx/2} stored in the
// imaginary slot of X_0).
//
// A line of nx = 2M reals is read as M complex numbers z_n = x_{2n} + i x_{2n+1}
// with 128-bit loads, transformed by an M-point complex Stockham FFT in shared
// memory, and untangled into the half spectrum:
//   X_k = E/2 - i (W^k/2) O,  X_{M-k} = conj(E/2 + i (W^k/2) O) ... (forward)
// with E = Z_k + conj Z_{M-k}, O = Z_k - conj Z_{M-k}, W = exp(-2 pi i/nx).
// The inverse runs the same steps backwards.  Consecutive lines (y, z) are
// contiguous, so a CTA's block of `lb` lines is one contiguous span.
// in and out may alias (the inverse runs in place): no __restrict__ on them.
#include "chanfs_internal.cuh"

namespace chanfs {

template <bool INV>
__global__ void __launch_bounds__(128) rfft_x_kernel(const double2* in,
                                                     double2* out, long long nlines,
                                                     FftDesc d, const double2* __restrict__ twg,
                                                     const double2* __restrict__ postg, int lb,
                                                     double scale, int scaled) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = d.n;
  const int bs = M;  // batch stride (complex)
  double2* buf0 = reinterpret_cast<double2*>(smem_raw);
  double2* buf1 = buf0 + lb * bs;
  double2* tw = buf1 + lb * bs;
  double2* post = tw + d.ntw;
  const int npost = M / 2 + 1;

  for (int e = threadIdx.x; e < d.ntw; e += blockDim.x) tw[e] = twg[e];
  for (int e = threadIdx.x; e < npost; e += blockDim.x) post[e] = postg[e];

  const long long line0 = (long long)blockIdx.x * lb;
  const double2 zero = make_double2(0.0, 0.0);

  if (!INV) {
    // contiguous span of lb*M complex values
    const double2* src = in + line0 * M;
    for (int e = threadIdx.x; e < lb * M; e += blockDim.x) {
      int l = e / M;
      buf0[e] = (line0 + l < nlines) ? src[e] : zero;
    }
    __syncthreads();
    double2* Z = stockham_smem<false, false>(buf0, buf1, d, lb, 1, bs, tw);
    // untangle the half-length spectrum into the packed real spectrum
    for (int e = threadIdx.x; e < lb * npost; e += blockDim.x) {
      int l = e / npost, k = e % npost;
      long long line = line0 + l;
      if (line >= nlines) continue;
      const double2* z = Z + l * bs;
      double2* o = out + line * M;
      if (k == 0) {
        double2 z0 = z[0];
        o[0] = make_double2(z0.x + z0.y, z0.x - z0.y);  // (X_0, X_M)
        continue;
      }
      double2 zk = z[k], zm = z[M - k];
      double2 E = make_double2(zk.x + zm.x, zk.y - zm.y);
      double2 O = make_double2(zk.x - zm.x, zk.y + zm.y);
      double2 u = cmul(O, post[k]);           // (W^k/2) O
      double2 t = make_double2(u.y, -u.x);    // -i (W^k/2) O
      o[k] = make_double2(fma(0.5, E.x, t.x), fma(0.5, E.y, t.y));
      if (M - k != k) o[M - k] = make_double2(fma(0.5, E.x, -t.x), fma(-0.5, E.y, t.y));
    }
  } else {
    __syncthreads();  // the untangling factors are read right away
    // re-tangle: Z_k = E/2 + i conj(W^k/2) T,  T = X_k - conj X_{M-k}
    for (int e = threadIdx.x; e < lb * npost; e += blockDim.x) {
      int l = e / npost, k = e % npost;
      long long line = line0 + l;
      double2* z = buf0 + l * bs;
      if (line >= nlines) {
        z[k] = zero;
        if (k > 0) z[M - k] = zero;
        continue;
      }
      const double2* x = in + line * M;
      double2 zk, zm;
      if (k == 0) {
        double2 x0 = x[0];  // (X_0, X_M)
        zk = make_double2(0.5 * (x0.x + x0.y), 0.5 * (x0.x - x0.y));
        zm = zk;
      } else {
        double2 xk = x[k], xm = x[M - k];
        double2 E = make_double2(xk.x + xm.x, xk.y - xm.y);
        double2 T = make_double2(xk.x - xm.x, xk.y + xm.y);
        double2 u = cmulc(T, post[k]);  // conj(W^k/2) T
        zk = make_double2(fma(0.5, E.x, -u.y), fma(0.5, E.y, u.x));
        zm = make_double2(fma(0.5, E.x, u.y), fma(-0.5, E.y, u.x));
      }
      if (scaled) {
        zk.x *= scale; zk.y *= scale;
        zm.x *= scale; zm.y *= scale;
      }
      z[k] = zk;
      if (k > 0 && M - k != k) z[M - k] = zm;
    }
    __syncthreads();
    double2* res = stockham_smem<true, false>(buf0, buf1, d, lb, 1, bs, tw);
    double2* dst = out + line0 * M;
    for (int e = threadIdx.x; e < lb * M; e += blockDim.x) {
      int l = e / M;
      if (line0 + l < nlines) dst[e] = res[e];
    }
  }
}

static int x_lines_per_cta(int M) { return M >= 1024 ? 1 : 1024 / M; }

static size_t x_smem_bytes(const cfs_plan* P, int lb) {
  return sizeof(double2) * (size_t)(2 * lb * P->M + P->fx.ntw + P->M / 2 + 1);
}

cudaError_t launch_rfft_x(const cfs_plan* P, const double* in, double* out, bool inverse,
                          double scale, cudaStream_t st) {
  const long long nlines = (long long)P->ny * P->nz;
  const int lb = x_lines_per_cta(P->M);
  const long long grid = (nlines + lb - 1) / lb;
  const size_t smem = x_smem_bytes(P, lb);
  const int scaled = (scale != 1.0);
  if (!inverse) {
    cudaFuncSetAttribute(rfft_x_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rfft_x_kernel<false><<<(unsigned)grid, 128, smem, st>>>(
        reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out), nlines, P->fx,
        P->d_twx, P->d_post, lb, scale, scaled);
  } else {
    cudaFuncSetAttribute(rfft_x_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rfft_x_kernel<true><<<(unsigned)grid, 128, smem, st>>>(
        reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out), nlines, P->fx,
        P->d_twx, P->d_post, lb, scale, scaled);
  }
  return cudaGetLastError();
}

}  // namespace chanfs
