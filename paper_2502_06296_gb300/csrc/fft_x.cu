// fft_x.cu -- real FFT along the contiguous x direction, packed output
// (App. A of the paper: n reals in, n reals out, X_{nx/2} stored in the
// imaginary slot of X_0).
//
// A line of nx = 2M reals is read as M complex numbers z_n = x_{2n} + i x_{2n+1}
// with 128-bit (FP64) or 64-bit (FP32) loads, transformed by an M-point complex
// Stockham FFT in shared memory, and untangled into the half spectrum:
//   X_k = E/2 - i (W^k/2) O,  X_{M-k} = conj(E/2 + i (W^k/2) O) ... (forward)
// with E = Z_k + conj Z_{M-k}, O = Z_k - conj Z_{M-k}, W = exp(-2 pi i/nx).
// The inverse runs the same steps backwards.  Consecutive lines (y, z) are
// contiguous, so a CTA's block of `lb` lines is one contiguous span.
// in and out may alias (the inverse runs in place): no __restrict__ on them.
// EMU (FP64 only) chooses the butterfly additions that run on the integer
// units instead of the FP64 pipe (kEmu* in chanfs_fft.cuh): the results are
// the same bits, the FP64 pipe that bounds these kernels does less.
//
// C = double2 is the FP64 solve.  C = float2 is the inner solve of iterative
// refinement; its inverse can write the FP64 result directly (OUT_SET) or add
// it to an FP64 field (OUT_ADD), the correction step p += delta; both leave
// the FP32 correction in place too, for the residual kernels.
#include "chanfs_fft.cuh"
#include "chanfs_group.cuh"
#include "chanfs_tma.cuh"

namespace chanfs {

// Block `blk` of the transform: lines [blk * lb, blk * lb + lb).  The lines
// of a block are one contiguous span: a bulk copy brings it into shared
// memory and another writes the result back, so the global traffic is two
// large asynchronous transfers per block and no thread computes an address
// per element.
template <bool INV, class C, int OUT, int EMU = 0>
__device__ __forceinline__ void rfft_x_body(const C* in, void* outv, long long nlines,
                                            const FftDesc& d, const C* __restrict__ twg,
                                            const C* __restrict__ postg, int lb, double scale,
                                            int scaled, int* status, long long blk,
                                            const double* msum = nullptr, double minv = 0.0,
                                            const C* add_src = nullptr) {
  using T = typename cscal<C>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int M = d.n;
  const int bs = M;  // batch stride (complex)
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  const int cap = xbuf_elems(lb, M, sizeof(C) == sizeof(float2));  // elements per buffer
  C* buf1 = buf0 + cap;
  C* tw = buf1 + cap;
  C* post = tw + d.ntw;
  const int npost = M / 2 + 1;
  const long long line0 = blk * lb;
  const int valid = (int)min((long long)lb, nlines - line0);  // lines of this block
  const uint32_t span = (uint32_t)((size_t)valid * M * sizeof(C));
  const C zero = mkc<C>(T(0), T(0));
  const T h = T(0.5);

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, span);
    bulk_load(INV ? buf1 : buf0, in + line0 * M, span, bar);
  }
  for (int e = threadIdx.x; e < d.ntw; e += blockDim.x) tw[e] = twg[e];
  for (int e = threadIdx.x; e < npost; e += blockDim.x) post[e] = postg[e];
  if (!INV)  // the lines past the end of the field transform zeros
    for (int e = valid * M + threadIdx.x; e < lb * M; e += blockDim.x) buf0[e] = zero;
  if (!cta_wait(bar, 0, status)) return;  // nothing is stored
  // work item e of a line-major loop over (line l, index k < npost), stepped
  // by blockDim.x without a division per item
  const int sk = blockDim.x % npost, sl = blockDim.x / npost;

  if (!INV) {
    C* Z = stockham_lines<false, C, EMU>(buf0, buf1, d, lb, tw);
    C* ob = (Z == buf0) ? buf1 : buf0;
    // untangle the half-length spectrum into the packed real spectrum
    int l = threadIdx.x / npost, k = threadIdx.x % npost;
    for (int e = threadIdx.x; e < valid * npost; e += blockDim.x) {
      const C* z = Z + l * bs;
      C* o = ob + l * bs;
      if (k == 0) {
        const C z0 = z[0];
        o[0] = mkc<C>(z0.x + z0.y, z0.x - z0.y);  // (X_0, X_M)
      } else {
        const C zk = z[k], zm = z[M - k];
        C p, m;
        cpair<(EMU & kEmuPost) != 0>(zk, zm, p, m);
        const C E = mkc<C>(p.x, m.y);  // (zk.x + zm.x, zk.y - zm.y)
        const C O = mkc<C>(m.x, p.y);  // (zk.x - zm.x, zk.y + zm.y)
        const C u = cmul(O, post[k]);  // (W^k/2) O
        const C t = mkc<C>(u.y, -u.x);  // -i (W^k/2) O
        o[k] = mkc<C>(fma(h, E.x, t.x), fma(h, E.y, t.y));
        if (M - k != k) o[M - k] = mkc<C>(fma(h, E.x, -t.x), fma(-h, E.y, t.y));
      }
      k += sk;
      l += sl;
      if (k >= npost) {
        k -= npost;
        ++l;
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      bulk_store(reinterpret_cast<C*>(outv) + line0 * M, ob, span);
      tma_store_commit_and_wait_read();
    }
  } else {
    // re-tangle: Z_k = E/2 + i conj(W^k/2) T,  T = X_k - conj X_{M-k}
    int l = threadIdx.x / npost, k = threadIdx.x % npost;
    for (int e = threadIdx.x; e < lb * npost; e += blockDim.x) {
      C* z = buf0 + l * bs;
      C zk, zm;
      if (l >= valid) {
        zk = zm = zero;
      } else if (k == 0) {
        const C x0 = buf1[l * bs];  // (X_0, X_M)
        zk = mkc<C>(h * (x0.x + x0.y), h * (x0.x - x0.y));
        zm = zk;
      } else {
        const C* x = buf1 + l * bs;
        const C xk = x[k], xm = x[M - k];
        C p, m;
        cpair<(EMU & kEmuPost) != 0>(xk, xm, p, m);
        const C E = mkc<C>(p.x, m.y);   // (xk.x + xm.x, xk.y - xm.y)
        const C Tt = mkc<C>(m.x, p.y);  // (xk.x - xm.x, xk.y + xm.y)
        const C u = cmulc(Tt, post[k]);  // conj(W^k/2) T
        zk = mkc<C>(fma(h, E.x, -u.y), fma(h, E.y, u.x));
        zm = mkc<C>(fma(h, E.x, u.y), fma(-h, E.y, u.x));
      }
      if (scaled) {
        const T sc = T(scale);
        zk.x *= sc;
        zk.y *= sc;
        zm.x *= sc;
        zm.y *= sc;
      }
      z[k] = zk;
      if (k > 0 && M - k != k) z[M - k] = zm;
      k += sk;
      l += sl;
      if (k >= npost) {
        k -= npost;
        ++l;
      }
    }
    __syncthreads();
    C* res = stockham_lines<true, C, EMU>(buf0, buf1, d, lb, tw);
    if (OUT == OUT_SAME) {
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        bulk_store(reinterpret_cast<C*>(outv) + line0 * M, res, span);
        tma_store_commit_and_wait_read();
      }
    } else {
      if ((OUT == OUT_ADD || OUT == OUT_SUM) && msum) {
        // the correction less the solution's current weighted mean (msum *
        // minv), so that p keeps a zero mean without a pass of its own; the
        // correction stored for the residual update is this one
        const T m = T(*msum * minv);
        for (int e = threadIdx.x; e < valid * M; e += blockDim.x) {
          res[e].x -= m;
          res[e].y -= m;
        }
        __syncthreads();
      }
      {  // the correction also stays behind (FP32, in place) for the residual kernels
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
          bulk_store(const_cast<C*>(in) + line0 * M, res, span);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      double2* dst = reinterpret_cast<double2*>(outv) + line0 * M;
      const C* first = add_src ? add_src + line0 * M : nullptr;
      for (int e = threadIdx.x; e < valid * M; e += blockDim.x) {
        const C r = res[e];
        if (OUT == OUT_SET) {
          dst[e] = make_double2(f32_to_f64(r.x), f32_to_f64(r.y));
        } else if (OUT == OUT_SUM) {  // p = the first correction + this one, written once
          const C a = first[e];
          dst[e] = make_double2(f32_to_f64(a.x) + f32_to_f64(r.x),
                                f32_to_f64(a.y) + f32_to_f64(r.y));
        } else {
          const double2 p = dst[e];
          dst[e] = make_double2(p.x + f32_to_f64(r.x), p.y + f32_to_f64(r.y));
        }
      }
      if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
}

template <bool INV, class C, int OUT, int EMU = 0>
__global__ void __launch_bounds__(128) rfft_x_kernel(const C* in, void* outv, long long nlines,
                                                     FftDesc d, const C* __restrict__ twg,
                                                     const C* __restrict__ postg, int lb,
                                                     double scale, int scaled, int* status,
                                                     const double* msum, double minv,
                                                     const C* add_src) {
  rfft_x_body<INV, C, OUT, EMU>(in, outv, nlines, d, twg, postg, lb, scale, scaled, status,
                                blockIdx.x, msum, minv, add_src);
}

// One launch for several boxes (FP32 inner solves of grouped refinement):
// the inverse's FP64 output goes to each box's solution in `io`.
template <bool INV, int OUT>
__global__ void __launch_bounds__(128) rfft_x_group_kernel(const XBox* boxes, GroupMap g,
                                                           const GroupIo* io, int alt_in) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const XBox& x = boxes[b];
  void* out = (OUT == OUT_SAME) ? x.out : static_cast<void*>(io[b].p);
  const float2* in = static_cast<const float2*>(alt_in ? x.in2 : x.in);
  rfft_x_body<INV, float2, OUT>(in, out, x.nlines, x.d,
                                static_cast<const float2*>(x.tw),
                                static_cast<const float2*>(x.post), x.lb, 1.0, 0, x.status, blk,
                                x.msum, x.minv, static_cast<const float2*>(x.add_src));
}

int x_lines_per_cta(const cfs_plan* P, size_t csize) {
  if (P->x_lines > 0) return P->x_lines;
  // about 16 KB of complex data per buffer
  const int target = (int)(16384 / csize);
  return P->M >= target ? 1 : target / P->M;
}

size_t x_smem_bytes(const cfs_plan* P, int lines, size_t csize) {
  const size_t cap = (size_t)xbuf_elems(lines, P->M, csize == sizeof(float2));
  return 128 + csize * (2 * cap + (size_t)P->fx.ntw + P->M / 2 + 1);
}

template <class C, int OUT, int EMU = 0>
static cudaError_t launch_x(const cfs_plan* P, const void* in, void* out, bool inverse,
                            double scale, const C* tw, const C* post, cudaStream_t st,
                            const double* msum = nullptr, const void* add_src = nullptr,
                            long long nlines = -1) {
  if (nlines < 0) nlines = (long long)P->ny * P->nz;
  if (nlines == 0) return cudaSuccess;
  const int lb = x_lines_per_cta(P, sizeof(C));
  const long long grid = (nlines + lb - 1) / lb;
  const size_t smem = x_smem_bytes(P, lb, sizeof(C));
  const int scaled = (scale != 1.0);
  const C* cin = reinterpret_cast<const C*>(in);
  if (!inverse) {
    auto k = rfft_x_kernel<false, C, OUT_SAME, EMU>;
    allow_max_smem(k);
    k<<<(unsigned)grid, 128, smem, st>>>(cin, out, nlines, P->fx, tw, post, lb, scale, scaled,
                                         P->d_status, nullptr, 0.0, nullptr);
  } else {
    auto k = rfft_x_kernel<true, C, OUT, EMU>;
    allow_max_smem(k);
    k<<<(unsigned)grid, 128, smem, st>>>(cin, out, nlines, P->fx, tw, post, lb, scale, scaled,
                                         P->d_status, msum, P->inv_wn,
                                         reinterpret_cast<const C*>(add_src));
  }
  return cudaGetLastError();
}

cudaError_t launch_rfft_x(const cfs_plan* P, const double* in, double* out, bool inverse,
                          double scale, cudaStream_t st, long long nlines) {
  const double2* tw = P->d_twx;
  const double2* post = P->d_post;
  // the plan's level L of integer-unit additions: kEmu* bits 0 .. L-1
  switch (P->emu_x) {
    case 1:
      return launch_x<double2, OUT_SAME, 1>(P, in, out, inverse, scale, tw, post, st, nullptr,
                                            nullptr, nlines);
    case 2:
      return launch_x<double2, OUT_SAME, 3>(P, in, out, inverse, scale, tw, post, st, nullptr,
                                            nullptr, nlines);
    case 3:
      return launch_x<double2, OUT_SAME, 7>(P, in, out, inverse, scale, tw, post, st, nullptr,
                                            nullptr, nlines);
    case 4:
      return launch_x<double2, OUT_SAME, 15>(P, in, out, inverse, scale, tw, post, st, nullptr,
                                             nullptr, nlines);
    default:
      return launch_x<double2, OUT_SAME, 0>(P, in, out, inverse, scale, tw, post, st, nullptr,
                                            nullptr, nlines);
  }
}

cudaError_t launch_rfft_x32(const cfs_plan* P, const float* in, float* out, bool inverse,
                            cudaStream_t st) {
  return launch_x<float2, OUT_SAME>(P, in, out, inverse, 1.0, P->d_twx32, P->d_post32, st);
}

cudaError_t launch_rfft_x32_to64(const cfs_plan* P, const float* in, double* out, bool add,
                                 cudaStream_t st, const double* msum) {
  if (add)
    return launch_x<float2, OUT_ADD>(P, in, out, true, 1.0, P->d_twx32, P->d_post32, st, msum);
  return launch_x<float2, OUT_SET>(P, in, out, true, 1.0, P->d_twx32, P->d_post32, st);
}

cudaError_t launch_rfft_x32_sum(const cfs_plan* P, const float* in, double* out,
                                const float* first, cudaStream_t st, const double* msum) {
  return launch_x<float2, OUT_SUM>(P, in, out, true, 1.0, P->d_twx32, P->d_post32, st, msum,
                                   first);
}

size_t x_group_box(const cfs_plan* P, bool inverse, XBox* box, int* blocks) {
  const int lb = x_lines_per_cta(P, sizeof(float2));
  box->d = P->fx;
  box->in = P->d_r32;
  box->in2 = P->d_r32b;
  box->out = P->d_r32;  // the FP32 result (forward, and the first inverse of refinement)
  box->add_src = P->d_w2;
  box->tw = P->d_twx32;
  box->post = P->d_post32;
  box->nlines = (long long)P->ny * P->nz;
  box->lb = lb;
  box->status = P->d_status;
  // the correction pass of refinement keeps the solution's mean at zero
  // (Neumann plans: the running weighted sum of p, see refine.cu)
  box->msum = (inverse && P->has_null) ? P->d_red + 2 : nullptr;
  box->minv = P->inv_wn;
  *blocks = (int)((box->nlines + lb - 1) / lb);
  return x_smem_bytes(P, lb, sizeof(float2));
}

cudaError_t launch_rfft_x_group32(const XBox* boxes, GroupMap g, int total, size_t smem,
                                  bool inverse, int out_mode, const GroupIo* io, int alt_in,
                                  cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  if (!inverse) {
    auto k = rfft_x_group_kernel<false, OUT_SAME>;
    allow_max_smem(k);
    k<<<total, 128, smem, st>>>(boxes, g, io, alt_in);
  } else if (out_mode == OUT_ADD) {
    auto k = rfft_x_group_kernel<true, OUT_ADD>;
    allow_max_smem(k);
    k<<<total, 128, smem, st>>>(boxes, g, io, alt_in);
  } else if (out_mode == OUT_SUM) {
    auto k = rfft_x_group_kernel<true, OUT_SUM>;
    allow_max_smem(k);
    k<<<total, 128, smem, st>>>(boxes, g, io, alt_in);
  } else if (out_mode == OUT_SAME) {
    auto k = rfft_x_group_kernel<true, OUT_SAME>;
    allow_max_smem(k);
    k<<<total, 128, smem, st>>>(boxes, g, io, alt_in);
  } else {
    auto k = rfft_x_group_kernel<true, OUT_SET>;
    allow_max_smem(k);
    k<<<total, 128, smem, st>>>(boxes, g, io, alt_in);
  }
  return cudaGetLastError();
}

}  // namespace chanfs
