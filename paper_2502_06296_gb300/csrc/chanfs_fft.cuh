// chanfs_fft.cuh -- the in-register small DFTs and the shared-memory Stockham
// engine shared by the x and y transforms, for complex types C = double2
// (the FP64 path) and float2 (the FP32 inner solves of iterative refinement).
#pragma once

#include "chanfs_internal.cuh"

namespace chanfs {

template <class C> struct cscal;
template <> struct cscal<double2> { using T = double; };
template <> struct cscal<float2> { using T = float; };

template <class C>
__device__ __forceinline__ C mkc(typename cscal<C>::T x, typename cscal<C>::T y);
template <>
__device__ __forceinline__ double2 mkc<double2>(double x, double y) { return make_double2(x, y); }
template <>
__device__ __forceinline__ float2 mkc<float2>(float x, float y) { return make_float2(x, y); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }

// a * w (2 MUL + 2 FMA) and a * conj(w).
template <class C> __device__ __forceinline__ C cmul(C a, C w) {
  return mkc<C>(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
template <class C> __device__ __forceinline__ C cmulc(C a, C w) {
  return mkc<C>(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
// Multiply by -i (forward) or +i (inverse): a swap and a sign, no arithmetic.
template <bool INV, class C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x);
}

// a + w x with fused multiply-adds (4 instructions); w is conjugated for the
// inverse transform.
template <bool INV, class C> __device__ __forceinline__ C cfma(C w, C x, C a) {
  if (INV)
    return mkc<C>(fma(w.x, x.x, fma(w.y, x.y, a.x)), fma(w.x, x.y, fma(-w.y, x.x, a.y)));
  return mkc<C>(fma(w.x, x.x, fma(-w.y, x.y, a.x)), fma(w.x, x.y, fma(w.y, x.x, a.y)));
}
template <bool INV, class C> __device__ __forceinline__ C ctw(C x, C w) {
  return INV ? cmulc(x, w) : cmul(x, w);
}
// 2a - s (2 instructions): the difference partner of s = a + t.
template <class C> __device__ __forceinline__ C ctwice_minus(C a, C s) {
  using T = typename cscal<C>::T;
  return mkc<C>(fma(T(2), a.x, -s.x), fma(T(2), a.y, -s.y));
}

// Small DFTs in registers.  Forward kernel e^{-2 pi i / R}, inverse e^{+}.
// The *_tw variants take the inputs before their Stockham twiddles w[r-1]
// (r >= 1) and fold each twiddle product into the first butterfly level:
//   (a + w x, a - w x) = (s, 2a - s) with s = a + w x by four FMAs,
// 6 instructions per pair instead of 8.
template <bool INV, class C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, class C> __device__ __forceinline__ void dft2_tw(C* v, const C* w) {
  C s = cfma<INV>(w[0], v[1], v[0]);
  v[1] = ctwice_minus(v[0], s);
  v[0] = s;
}

// y0 = a + s, y1,2 = (a - s/2) -/+ i (sqrt3/2) d  with s = b + c, d = b - c.
template <bool INV, class C>
__device__ __forceinline__ void dft3_core(C& a, C& b, C& c, C s, C d) {
  using T = typename cscal<C>::T;
  const T h = T(0.8660254037844386467637231707529362);  // sqrt(3)/2
  C t = mkc<C>(fma(T(-0.5), s.x, a.x), fma(T(-0.5), s.y, a.y));
  a = cadd(a, s);
  const T sx = INV ? -h : h;
  b = mkc<C>(fma(sx, d.y, t.x), fma(-sx, d.x, t.y));
  c = mkc<C>(fma(-sx, d.y, t.x), fma(sx, d.x, t.y));
}

template <bool INV, class C> __device__ __forceinline__ void dft3(C& a, C& b, C& c) {
  dft3_core<INV>(a, b, c, cadd(b, c), csub(b, c));
}

template <bool INV, class C> __device__ __forceinline__ void dft3_tw(C* v, const C* w) {
  C b = ctw<INV>(v[1], w[0]);
  C s = cfma<INV>(w[1], v[2], b);
  C d = ctwice_minus(b, s);
  dft3_core<INV>(v[0], v[1], v[2], s, d);
}

// Radix-4 second level from t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3,
// d = a1 - a3.
template <bool INV, class C>
__device__ __forceinline__ void dft4_core(C* y, C t0, C t1, C t2, C d) {
  C t3 = mul_mi<INV>(d);
  y[0] = cadd(t0, t2);
  y[2] = csub(t0, t2);
  y[1] = cadd(t1, t3);
  y[3] = csub(t1, t3);
}

template <bool INV, class C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C y[4];
  dft4_core<INV>(y, cadd(a0, a2), csub(a0, a2), cadd(a1, a3), csub(a1, a3));
  a0 = y[0]; a1 = y[1]; a2 = y[2]; a3 = y[3];
}

// DFT4 of (x0, w1 x1, w2 x2, w3 x3) given x0..x3 and w1..w3 (x0 untwiddled).
template <bool INV, class C>
__device__ __forceinline__ void dft4_tw4(C* y, C x0, C x1, C x2, C x3, C w1, C w2, C w3) {
  C t0 = cfma<INV>(w2, x2, x0);
  C t1 = ctwice_minus(x0, t0);
  C u = ctw<INV>(x1, w1);
  C t2 = cfma<INV>(w3, x3, u);
  dft4_core<INV>(y, t0, t1, t2, ctwice_minus(u, t2));
}

template <bool INV, class C> __device__ __forceinline__ void dft4_tw(C* v, const C* w) {
  C y[4];
  dft4_tw4<INV>(y, v[0], v[1], v[2], v[3], w[0], w[1], w[2]);
  v[0] = y[0]; v[1] = y[1]; v[2] = y[2]; v[3] = y[3];
}

// Radix-2 combination of the even (E) and odd (O) half-DFTs of a DFT8, with
// the W8 factors folded into fused multiply-adds.
template <bool INV, class C>
__device__ __forceinline__ void dft8_combine(C* v, const C* E, const C* O) {
  using T = typename cscal<C>::T;
  const T r = T(0.7071067811865475244008443621048490);  // 1/sqrt(2)
  v[0] = cadd(E[0], O[0]);
  v[4] = csub(E[0], O[0]);
  C m2 = mul_mi<INV>(O[2]);
  v[2] = cadd(E[2], m2);
  v[6] = csub(E[2], m2);
  if (!INV) {
    // W8 O = r (O.x + O.y, O.y - O.x);  W8^3 O = r (O.y - O.x, -(O.x + O.y))
    T p1 = O[1].x + O[1].y, q1 = O[1].y - O[1].x;
    v[1] = mkc<C>(fma(r, p1, E[1].x), fma(r, q1, E[1].y));
    v[5] = mkc<C>(fma(-r, p1, E[1].x), fma(-r, q1, E[1].y));
    T p3 = O[3].y - O[3].x, q3 = O[3].x + O[3].y;
    v[3] = mkc<C>(fma(r, p3, E[3].x), fma(-r, q3, E[3].y));
    v[7] = mkc<C>(fma(-r, p3, E[3].x), fma(r, q3, E[3].y));
  } else {
    // W8^-1 O = r (O.x - O.y, O.x + O.y);  W8^-3 O = r (-(O.x + O.y), O.x - O.y)
    T p1 = O[1].x - O[1].y, q1 = O[1].x + O[1].y;
    v[1] = mkc<C>(fma(r, p1, E[1].x), fma(r, q1, E[1].y));
    v[5] = mkc<C>(fma(-r, p1, E[1].x), fma(-r, q1, E[1].y));
    T q3 = O[3].x + O[3].y, p3 = O[3].x - O[3].y;
    v[3] = mkc<C>(fma(-r, q3, E[3].x), fma(r, p3, E[3].y));
    v[7] = mkc<C>(fma(r, q3, E[3].x), fma(-r, p3, E[3].y));
  }
}

template <bool INV, class C> __device__ __forceinline__ void dft8(C* v) {
  C E[4], O[4];
  dft4_core<INV>(E, cadd(v[0], v[4]), csub(v[0], v[4]), cadd(v[2], v[6]), csub(v[2], v[6]));
  dft4_core<INV>(O, cadd(v[1], v[5]), csub(v[1], v[5]), cadd(v[3], v[7]), csub(v[3], v[7]));
  dft8_combine<INV>(v, E, O);
}

template <bool INV, class C> __device__ __forceinline__ void dft8_tw(C* v, const C* w) {
  C E[4], O[4];
  // even half: (v0, w2 v2, w4 v4, w6 v6)
  dft4_tw4<INV>(E, v[0], v[2], v[4], v[6], w[1], w[3], w[5]);
  // odd half: all four twiddled
  C a = ctw<INV>(v[1], w[0]);
  C t0 = cfma<INV>(w[4], v[5], a);
  C t1 = ctwice_minus(a, t0);
  C b = ctw<INV>(v[3], w[2]);
  C t2 = cfma<INV>(w[6], v[7], b);
  dft4_core<INV>(O, t0, t1, t2, ctwice_minus(b, t2));
  dft8_combine<INV>(v, E, O);
}

template <int R, bool INV, class C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
}

template <int R, bool INV, class C> __device__ __forceinline__ void dft_tw(C* v, const C* w) {
  if constexpr (R == 2) dft2_tw<INV>(v, w);
  else if constexpr (R == 3) dft3_tw<INV>(v, w);
  else if constexpr (R == 4) dft4_tw<INV>(v, w);
  else if constexpr (R == 8) dft8_tw<INV>(v, w);
}

// One Stockham radix-R butterfly: reads R points j + r*n/R of one batch from
// `in`, applies the twiddles of pass (L, R), transforms, and writes them to
// positions (j - k)*R + k + r*L of `out` (k = j mod L, by a mask when L is a
// power of two: lmask = L - 1, else -1).  es = element stride.
template <int R, bool INV, class C>
__device__ __forceinline__ void stockham_bfly(const C* __restrict__ in, C* __restrict__ out, int j,
                                              int L, int lmask, int n, int es,
                                              const C* __restrict__ tw) {
  C v[R];
  const int q = n / R;
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[(j + r * q) * es];
  const int k = lmask >= 0 ? (j & lmask) : j % L;
  if (L > 1) {
    C w[R - 1];
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
template <bool INV, bool BATCH_FAST, class C>
__device__ C* stockham_smem(C* a, C* b, const FftDesc& d, int nb, int es, int bs,
                            const C* __restrict__ tw) {
  const int n = d.n;
  for (int p = 0; p < d.npass; ++p) {
    const int R = d.radix[p], L = d.span[p];
    const int lmask = (L & (L - 1)) == 0 ? L - 1 : -1;
    const C* twp = tw + d.twoff[p];
    const int nbf = n / R;
    const int total = nbf * nb;
    // (fast, slow) index of work item t, stepped by blockDim.x without a
    // division per item: the fast index runs over batches (BATCH_FAST) or
    // butterflies
    const int nfast = BATCH_FAST ? nb : nbf;
    const int sfast = blockDim.x % nfast, sslow = blockDim.x / nfast;
    int fi = threadIdx.x % nfast, si = threadIdx.x / nfast;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int bat = BATCH_FAST ? fi : si;
      const int j = BATCH_FAST ? si : fi;
      fi += sfast;
      si += sslow;
      if (fi >= nfast) {
        fi -= nfast;
        ++si;
      }
      const C* in = a + bat * bs;
      C* out = b + bat * bs;
      switch (R) {
        case 8: stockham_bfly<8, INV>(in, out, j, L, lmask, n, es, twp); break;
        case 4: stockham_bfly<4, INV>(in, out, j, L, lmask, n, es, twp); break;
        case 3: stockham_bfly<3, INV>(in, out, j, L, lmask, n, es, twp); break;
        default: stockham_bfly<2, INV>(in, out, j, L, lmask, n, es, twp); break;
      }
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace chanfs
