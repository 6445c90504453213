// chanfs_fft.cuh -- the in-register small DFTs and the shared-memory Stockham
// engine shared by the x and y transforms, for complex types C = double2
// (the FP64 path) and float2 (the FP32 inner solves of iterative refinement).
#pragma once

#include "chanfs_f64emu.cuh"
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
// Which butterfly additions of the FP64 transforms run on the integer units
// (f64_addsub, bit for bit the FP64 pipe's results), as a mask of template
// parameter EMU; FP32 transforms ignore it.
constexpr int kEmuCore = 1;   // the second level of every radix-4 core (t0 +- t2, t1 +- t3)
constexpr int kEmuComb = 2;   // the radix-2 combination of a DFT8 (E0 +- O0, E2 +- i O2)
constexpr int kEmuFirst = 4;  // the first level of untwiddled DFT8/4/2 and DFT3's b +- c
constexpr int kEmuPost = 8;   // the real-FFT untangle of the x transform

// (a + b, a - b); EMU: the FP64 additions by f64_addsub.
template <bool EMU, class C> __device__ __forceinline__ void cpair(C a, C b, C& p, C& m) {
  if constexpr (EMU && sizeof(C) == sizeof(double2)) {
    f64_addsub(a.x, b.x, p.x, m.x);
    f64_addsub(a.y, b.y, p.y, m.y);
  } else {
    p = cadd(a, b);
    m = csub(a, b);
  }
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
template <bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft2(C& a, C& b) {
  cpair<(EMU & kEmuFirst) != 0>(C(a), C(b), a, b);
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

template <bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft3(C& a, C& b, C& c) {
  C s, d;
  cpair<(EMU & kEmuFirst) != 0>(b, c, s, d);
  dft3_core<INV>(a, b, c, s, d);
}

template <bool INV, class C> __device__ __forceinline__ void dft3_tw(C* v, const C* w) {
  C b = ctw<INV>(v[1], w[0]);
  C s = cfma<INV>(w[1], v[2], b);
  C d = ctwice_minus(b, s);
  dft3_core<INV>(v[0], v[1], v[2], s, d);
}

// Radix-4 second level from t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3,
// d = a1 - a3.
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ void dft4_core(C* y, C t0, C t1, C t2, C d) {
  C t3 = mul_mi<INV>(d);
  cpair<(EMU & kEmuCore) != 0>(t0, t2, y[0], y[2]);
  cpair<(EMU & kEmuCore) != 0>(t1, t3, y[1], y[3]);
}

template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C y[4], t0, t1, t2, d;
  cpair<(EMU & kEmuFirst) != 0>(a0, a2, t0, t1);
  cpair<(EMU & kEmuFirst) != 0>(a1, a3, t2, d);
  dft4_core<INV, C, EMU>(y, t0, t1, t2, d);
  a0 = y[0]; a1 = y[1]; a2 = y[2]; a3 = y[3];
}

// DFT4 of (x0, w1 x1, w2 x2, w3 x3) given x0..x3 and w1..w3 (x0 untwiddled).
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ void dft4_tw4(C* y, C x0, C x1, C x2, C x3, C w1, C w2, C w3) {
  C t0 = cfma<INV>(w2, x2, x0);
  C t1 = ctwice_minus(x0, t0);
  C u = ctw<INV>(x1, w1);
  C t2 = cfma<INV>(w3, x3, u);
  dft4_core<INV, C, EMU>(y, t0, t1, t2, ctwice_minus(u, t2));
}

template <bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft4_tw(C* v, const C* w) {
  C y[4];
  dft4_tw4<INV, C, EMU>(y, v[0], v[1], v[2], v[3], w[0], w[1], w[2]);
  v[0] = y[0]; v[1] = y[1]; v[2] = y[2]; v[3] = y[3];
}

// Radix-2 combination of the even (E) and odd (O) half-DFTs of a DFT8, with
// the W8 factors folded into fused multiply-adds.
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ void dft8_combine(C* v, const C* E, const C* O) {
  using T = typename cscal<C>::T;
  const T r = T(0.7071067811865475244008443621048490);  // 1/sqrt(2)
  cpair<(EMU & kEmuComb) != 0>(E[0], O[0], v[0], v[4]);
  C m2 = mul_mi<INV>(O[2]);
  cpair<(EMU & kEmuComb) != 0>(E[2], m2, v[2], v[6]);
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

template <bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft8(C* v) {
  constexpr bool F = (EMU & kEmuFirst) != 0;
  C E[4], O[4], p[8];
  cpair<F>(v[0], v[4], p[0], p[1]);
  cpair<F>(v[2], v[6], p[2], p[3]);
  cpair<F>(v[1], v[5], p[4], p[5]);
  cpair<F>(v[3], v[7], p[6], p[7]);
  dft4_core<INV, C, EMU>(E, p[0], p[1], p[2], p[3]);
  dft4_core<INV, C, EMU>(O, p[4], p[5], p[6], p[7]);
  dft8_combine<INV, C, EMU>(v, E, O);
}

template <bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft8_tw(C* v, const C* w) {
  C E[4], O[4];
  // even half: (v0, w2 v2, w4 v4, w6 v6)
  dft4_tw4<INV, C, EMU>(E, v[0], v[2], v[4], v[6], w[1], w[3], w[5]);
  // odd half: all four twiddled
  C a = ctw<INV>(v[1], w[0]);
  C t0 = cfma<INV>(w[4], v[5], a);
  C t1 = ctwice_minus(a, t0);
  C b = ctw<INV>(v[3], w[2]);
  C t2 = cfma<INV>(w[6], v[7], b);
  dft4_core<INV, C, EMU>(O, t0, t1, t2, ctwice_minus(b, t2));
  dft8_combine<INV, C, EMU>(v, E, O);
}

template <int R, bool INV, class C, int EMU = 0> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2<INV, C, EMU>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV, C, EMU>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV, C, EMU>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV, C, EMU>(v);
}

template <int R, bool INV, class C, int EMU = 0>
__device__ __forceinline__ void dft_tw(C* v, const C* w) {
  if constexpr (R == 2) dft2_tw<INV>(v, w);
  else if constexpr (R == 3) dft3_tw<INV>(v, w);
  else if constexpr (R == 4) dft4_tw<INV, C, EMU>(v, w);
  else if constexpr (R == 8) dft8_tw<INV, C, EMU>(v, w);
}

// One Stockham radix-R butterfly: reads R points j + r*n/R of one batch from
// `in`, applies the twiddles of pass (L, R), transforms, and writes them to
// positions (j - k)*R + k + r*L of `out` (k = j mod L, by a mask when L is a
// power of two: lmask = L - 1, else -1).  es = element stride.
template <int R, bool INV, class C, int EMU = 0>
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
    dft_tw<R, INV, C, EMU>(v, w);
  } else {
    dft<R, INV, C, EMU>(v);
  }
  const int o = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) out[(o + r * L) * es] = v[r];
}

// All passes of an FFT over `nb` batches held in shared memory.  Element e of
// batch b lives at buf[b*bs + e*es].  Ping-pongs between a and b; returns the
// buffer holding the result.  BATCH_FAST: consecutive threads take consecutive
// batches (columns of a y tile) instead of consecutive butterflies.
template <bool INV, bool BATCH_FAST, class C, int EMU = 0>
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
        case 8: stockham_bfly<8, INV, C, EMU>(in, out, j, L, lmask, n, es, twp); break;
        case 4: stockham_bfly<4, INV, C, EMU>(in, out, j, L, lmask, n, es, twp); break;
        case 3: stockham_bfly<3, INV, C, EMU>(in, out, j, L, lmask, n, es, twp); break;
        default: stockham_bfly<2, INV, C, EMU>(in, out, j, L, lmask, n, es, twp); break;
      }
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
  }
  return a;
}

// The radix plan of make_fft_desc (largest radix 8) as compile-time
// functions of the length: pass p's radix (0 past the last pass), span and
// twiddle offset.
__host__ __device__ constexpr int fixed_radix(int n, int p) {
  int rest = n, q = 0;
  while (rest % 8 == 0) {
    if (q == p) return 8;
    rest /= 8;
    ++q;
  }
  while (rest % 4 == 0) {
    if (q == p) return 4;
    rest /= 4;
    ++q;
  }
  if (rest % 2 == 0) {
    if (q == p) return 2;
    rest /= 2;
    ++q;
  }
  while (rest % 3 == 0) {
    if (q == p) return 3;
    rest /= 3;
    ++q;
  }
  return 0;
}
__host__ __device__ constexpr int fixed_npass(int n) {
  int p = 0;
  while (fixed_radix(n, p)) ++p;
  return p;
}
__host__ __device__ constexpr int fixed_span(int n, int p) {
  int L = 1;
  for (int i = 0; i < p; ++i) L *= fixed_radix(n, i);
  return L;
}
__host__ __device__ constexpr int fixed_twoff(int n, int p) {
  int o = 0;
  for (int i = 0; i < p; ++i) o += fixed_span(n, i) * (fixed_radix(n, i) - 1);
  return o;
}

// Whether descriptor d is the compile-time plan of length N.
template <int N>
__device__ __forceinline__ bool is_fixed_plan(const FftDesc& d) {
  constexpr int np = fixed_npass(N), r0 = fixed_radix(N, 0);
  return d.n == N && d.npass == np && d.radix[0] == r0;
}

// Shared-memory layout of the intermediate passes of stockham_fixed:
// element e of a batch at e + e/16 (batch stride N + N/16).  In the
// unpadded layout the writes of the passes with span L < 16 (and the reads
// that follow) put a warp's 8-byte accesses on a few banks -- 16-way for the
// first pass's stride-R writes; with one pad element per 16 every such
// warp access takes the minimum two wavefronts.  The input of the first pass
// and the output of the last keep the contiguous layout that the bulk copies
// load and store.
__host__ __device__ constexpr int fixed_padded(int n) { return n + n / 16; }
__device__ __forceinline__ int pad16(int e) { return e + (e >> 4); }

// Elements of one x-transform buffer of `lines` lines of m complex points:
// FP32 buffers have room for the padded layout, rounded to an even count
// (the next buffer starts on a 16-byte boundary).
__host__ __device__ inline int xbuf_elems(int lines, int m, bool fp32) {
  if (!fp32) return lines * m;
  const int e = lines * fixed_padded(m);
  return (e + 1) & ~1;
}

// The Stockham passes of a compile-time length N over `nb` batches (element
// stride 1; batch stride N in the first pass's input and the last pass's
// output, fixed_padded(N) between passes): the same butterflies and twiddles
// as stockham_smem with every radix, span, stride and offset a constant.
// Returns the buffer holding the result.
template <bool INV, int N, int P, class C, int EMU = 0>
__device__ __forceinline__ C* stockham_fixed(C* a, C* b, int nb, const C* __restrict__ tw) {
  if constexpr (fixed_radix(N, P) == 0) {
    return a;
  } else {
    constexpr int R = fixed_radix(N, P), L = fixed_span(N, P), TO = fixed_twoff(N, P);
    constexpr int Q = N / R;  // butterflies per batch, and the input stride
    constexpr bool PIN = P > 0, POUT = P + 1 < fixed_npass(N);
    constexpr int SIN = PIN ? fixed_padded(N) : N, SOUT = POUT ? fixed_padded(N) : N;
    const int total = Q * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int bat = t / Q;
      const int j = t - bat * Q;
      const C* in = a + bat * SIN;
      C* out = b + bat * SOUT;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in[PIN ? pad16(j + r * Q) : j + r * Q];
      const int k = j % L;
      if constexpr (L > 1) {
        C w[R - 1];
#pragma unroll
        for (int r = 0; r < R - 1; ++r) w[r] = tw[TO + k * (R - 1) + r];
        dft_tw<R, INV, C, EMU>(v, w);
      } else {
        dft<R, INV, C, EMU>(v);
      }
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) out[POUT ? pad16(o + r * L) : o + r * L] = v[r];
    }
    __syncthreads();
    return stockham_fixed<INV, N, P + 1, C, EMU>(b, a, nb, tw);
  }
}

// The same for the y transform's tile: `tk` interleaved columns (element e
// of column c at e*tk + c), consecutive threads on consecutive columns.  The
// intermediate passes use the padded layout (flat index i at i + i/16; see
// stockham_fixed): for narrow tiles (tk < 16) the first pass's writes were
// bank conflicts of up to 8 ways.
template <bool INV, int N, int P, class C>
__device__ __forceinline__ C* stockham_fixed_cols(C* a, C* b, int tk, const C* __restrict__ tw) {
  if constexpr (fixed_radix(N, P) == 0) {
    return a;
  } else {
    constexpr int R = fixed_radix(N, P), L = fixed_span(N, P), TO = fixed_twoff(N, P);
    constexpr int Q = N / R;
    constexpr bool PIN = P > 0, POUT = P + 1 < fixed_npass(N);
    const int total = Q * tk;
    const int sfast = blockDim.x % tk, sslow = blockDim.x / tk;
    int c = threadIdx.x % tk, j = threadIdx.x / tk;  // column (fast), butterfly (slow)
    const int qs = Q * tk, ls = L * tk;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int i0 = j * tk + c;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = a[PIN ? pad16(i0 + r * qs) : i0 + r * qs];
      const int k = j % L;
      if constexpr (L > 1) {
        C w[R - 1];
#pragma unroll
        for (int r = 0; r < R - 1; ++r) w[r] = tw[TO + k * (R - 1) + r];
        dft_tw<R, INV>(v, w);
      } else {
        dft<R, INV>(v);
      }
      const int o0 = ((j - k) * R + k) * tk + c;
#pragma unroll
      for (int r = 0; r < R; ++r) b[POUT ? pad16(o0 + r * ls) : o0 + r * ls] = v[r];
      c += sfast;
      j += sslow;
      if (c >= tk) {
        c -= tk;
        ++j;
      }
    }
    __syncthreads();
    return stockham_fixed_cols<INV, N, P + 1>(b, a, tk, tw);
  }
}

// Whether an FP32 y tile of length d.n takes the compile-time path below.
__host__ __device__ inline bool tile_fixed_len(const FftDesc& d) {
  switch (d.n) {
    case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768:
      return d.npass == fixed_npass(d.n) && d.radix[0] == fixed_radix(d.n, 0);
    default:
      return false;
  }
}

// All passes of a y tile (FP32: the compile-time path for common lengths).
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ C* stockham_tile(C* a, C* b, const FftDesc& d, int tk,
                                            const C* __restrict__ tw) {
  if constexpr (sizeof(C) == sizeof(float2)) {
    switch (d.n) {
      case 64:
        if (is_fixed_plan<64>(d)) return stockham_fixed_cols<INV, 64, 0>(a, b, tk, tw);
        break;
      case 96:
        if (is_fixed_plan<96>(d)) return stockham_fixed_cols<INV, 96, 0>(a, b, tk, tw);
        break;
      case 128:
        if (is_fixed_plan<128>(d)) return stockham_fixed_cols<INV, 128, 0>(a, b, tk, tw);
        break;
      case 192:
        if (is_fixed_plan<192>(d)) return stockham_fixed_cols<INV, 192, 0>(a, b, tk, tw);
        break;
      case 256:
        if (is_fixed_plan<256>(d)) return stockham_fixed_cols<INV, 256, 0>(a, b, tk, tw);
        break;
      case 384:
        if (is_fixed_plan<384>(d)) return stockham_fixed_cols<INV, 384, 0>(a, b, tk, tw);
        break;
      case 512:
        if (is_fixed_plan<512>(d)) return stockham_fixed_cols<INV, 512, 0>(a, b, tk, tw);
        break;
      case 768:
        if (is_fixed_plan<768>(d)) return stockham_fixed_cols<INV, 768, 0>(a, b, tk, tw);
        break;
      default:
        break;
    }
  }
  return stockham_smem<INV, true, C, EMU>(a, b, d, tk, tk, 1, tw);
}

// All passes over `nb` contiguous batches of length d.n (the x transform's
// layout).  FP32 transforms are bound by instruction issue, and for the
// common lengths take a compile-time path (about a third fewer instructions
// at n = 512); FP64 transforms are bound by the FP64 pipe and keep the
// general one.
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ C* stockham_lines(C* a, C* b, const FftDesc& d, int nb,
                                             const C* __restrict__ tw) {
  if constexpr (sizeof(C) == sizeof(float2)) {
    switch (d.n) {
      case 32:
        if (is_fixed_plan<32>(d)) return stockham_fixed<INV, 32, 0>(a, b, nb, tw);
        break;
      case 48:
        if (is_fixed_plan<48>(d)) return stockham_fixed<INV, 48, 0>(a, b, nb, tw);
        break;
      case 64:
        if (is_fixed_plan<64>(d)) return stockham_fixed<INV, 64, 0>(a, b, nb, tw);
        break;
      case 96:
        if (is_fixed_plan<96>(d)) return stockham_fixed<INV, 96, 0>(a, b, nb, tw);
        break;
      case 128:
        if (is_fixed_plan<128>(d)) return stockham_fixed<INV, 128, 0>(a, b, nb, tw);
        break;
      case 192:
        if (is_fixed_plan<192>(d)) return stockham_fixed<INV, 192, 0>(a, b, nb, tw);
        break;
      case 256:
        if (is_fixed_plan<256>(d)) return stockham_fixed<INV, 256, 0>(a, b, nb, tw);
        break;
      case 384:
        if (is_fixed_plan<384>(d)) return stockham_fixed<INV, 384, 0>(a, b, nb, tw);
        break;
      case 512:
        if (is_fixed_plan<512>(d)) return stockham_fixed<INV, 512, 0>(a, b, nb, tw);
        break;
      case 1024:
        if (is_fixed_plan<1024>(d)) return stockham_fixed<INV, 1024, 0>(a, b, nb, tw);
        break;
      default:
        break;
    }
  }
  return stockham_smem<INV, false, C, EMU>(a, b, d, nb, 1, d.n, tw);
}

}  // namespace chanfs
