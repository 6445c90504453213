// thomas.cu -- the per-(kx, ky) tridiagonal solves along z of Eq. 12, and
// the plan-time factorisation of those systems.
//
// After the x and y transforms, column (kx, ky) solves
//   A_k F_{k-1} + (B_k + lx[kx] + ly[ky]) F_k + C_k F_{k+1} = f_k.
// The matrices depend on (kx, ky) but not on time, so the plan factors them
// once (the paper keeps the time-invariant Poisson coefficients for the whole
// run, Sec. 2.2.4), folding the inverse-FFT normalisation s into the factors:
//   forward  g_k = (s/piv_k) f_k - (A_k/piv_k) g_{k-1}
//   backward x_k = g_k - (C_k/piv_k) x_{k+1}
// i.e. 3 FP64 instructions per real unknown, no division at run time.
//
// One thread per column of the spectrum; consecutive threads take consecutive
// kx so that every z-plane access is coalesced.  Column kx = 0 arrives
// untangled by the y transform (App. A's packing applied again along y), so
// every slot is one column of Eq. 12; the two self-conjugate slots hold two
// real columns with different eigenvalues in their real and imaginary parts.
// The singular Neumann column (0, 0) is pinned (row 0 -> F_0 = 0); the
// removal of the dz-weighted mean of its right-hand side and of its solution
// is folded into the same two sweeps by linearity.
#include <atomic>

#include "chanfs_tma.cuh"
#include "chanfs_group.cuh"
#include "chanfs_alg2.cuh"

namespace chanfs {


constexpr int kThomasBlock = 64;
// Rows each thread keeps in flight ahead of its sweep (by arithmetic type):
// an FP64 sweep is bound by the FP64 pipe and needs few; an FP32 sweep is
// bound by memory latency.  (Deeper prefetch spills at the register budget
// of 14 blocks of 64 threads per SM.)
template <class CA> struct prefetch_rows { static constexpr int value = 3; };
template <> struct prefetch_rows<float2> { static constexpr int value = 6; };
// The same for a thread that sweeps two columns (sweep_pair): two rows per
// step.  DEEP (FP64 plans of moderate size): the launch fits in one wave at
// 6 (DEEP = 6) or 8 (DEEP = 4) blocks per SM, so each thread may keep a
// queue of DEEP rows; the sweep is bound by memory latency at the few warps
// per SM such a launch has (the channel's FP64 spectrum: 772 blocks, 6 rows
// measured 5 % faster than 4).
template <class CA, int DEEP> struct pair_prefetch_rows {
  static constexpr int value = DEEP ? DEEP : 2;
};
template <int DEEP> struct pair_prefetch_rows<float2, DEEP> { static constexpr int value = 3; };

template <class C> struct cplx_traits;
template <> struct cplx_traits<double2> {
  using T = double;
  __device__ static double2 mk(double x, double y) { return make_double2(x, y); }
};
template <> struct cplx_traits<float2> {
  using T = float;
  __device__ static float2 mk(float x, float y) { return make_float2(x, y); }
};
template <class CA, class CS> __device__ __forceinline__ CA cvt(CS v) {
  return cplx_traits<CA>::mk((typename cplx_traits<CA>::T)v.x, (typename cplx_traits<CA>::T)v.y);
}

// One column sweep: storage type CS (the spectrum), arithmetic type CA with
// its factor tables F (pairs) and B (scalars).  Pointers step by a row stride
// and each thread keeps the next prefetch_rows<CA> rows in flight while the recurrence
// consumes the current one (the sweep is sequential in k, and there are only
// a few warps per SM, so this in-thread prefetch is what hides the memory
// latency).  Real and imaginary parts use factor sets x and y, which differ
// only for the two self-conjugate slots of kx = 0 (a real F(0,ky) and a real
// F(Nx/2,ky) packed together; see fft_y.cu).
//
// Neumann (0, 0) column (real part of slot (0, 0)): singular.  Its system is
// pinned (row 0: F_0 = 0) and, by linearity, both projections are folded
// into the same two sweeps:
//   mu = sum_k wn_k E_k                   (dz-weighted mean of the rhs)
//   x  = T'^{-1} E' - mu h - nu,  E' = (0, E_1, ..)
//   nu = (g^T E' - mu g^T 1') / sum w     (dz-weighted mean of the solution)
// with h = T'^{-1} (0, 1, .., 1) and g = T'^{-T} w precomputed by the plan.
//
// ONE: the real and imaginary parts share factor set x (every column but
// kx = 0); fy0 and by0 are then not read.
template <class CS, class CA, bool ONE, int PF, class F2, class F1>
__device__ __forceinline__ void sweep_column(const ThomasArgs& a, CS* const s0, const F2* const fx0,
                                             const F2* const fy0, const F1* const bx0,
                                             const F1* const by0, const bool sing) {
  using T = typename cplx_traits<CA>::T;
  const int nz = a.nz;
  const long long rs = (long long)a.ny * a.M;         // spectrum row stride
  const long long rt = (long long)a.nky * (a.M + 1);  // factor row stride

  // forward: g_k = (s/piv_k) f_k - (A_k/piv_k) g_{k-1}, in place
  CS qu[PF];
  F2 qx[PF], qy[ONE ? 1 : PF];
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    if (i < nz) {
      qu[i] = s0[i * rs];
      qx[i] = fx0[i * rt];
      if (!ONE) qy[i] = fy0[i * rt];
    }
  }
  const CS* pu = s0 + PF * rs;  // next rows to prefetch
  const F2* px = fx0 + PF * rt;
  const F2* py = ONE ? px : fy0 + PF * rt;
  CS* ps = s0;                         // row being written
  CA g = cplx_traits<CA>::mk(T(0), T(0));
  double mu = 0.0, gam = 0.0;
  for (int k = 0; k < nz; k += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      if (k + i >= nz) break;
      CA u = cvt<CA>(qu[i]);
      const F2 fx = qx[i], fy = ONE ? fx : qy[i];
      if (k + i + PF < nz) {
        qu[i] = *pu;
        qx[i] = *px;
        if (!ONE) qy[i] = *py;
      }
      pu += rs;
      px += rt;
      if (!ONE) py += rt;
      if (sing) {
        mu = fma(a.sing[k + i], (double)u.x, mu);
        if (k + i > 0) gam = fma(a.sing[nz + k + i], (double)u.x, gam);
        else u.x = T(0);  // pinned row
      }
      g = cplx_traits<CA>::mk(fma(-fx.y, g.x, fx.x * u.x), fma(-fy.y, g.y, fy.x * u.y));
      *ps = cvt<CS>(g);
      ps += rs;
    }
  }
  const double nu = sing ? a.sing_sc * (gam - mu * a.sing_cg) : 0.0;

  // backward: x_k = g_k - (C_k/piv_k) x_{k+1}, from the top wall down
  CS qg[PF];
  F1 qbx[PF], qby[ONE ? 1 : PF];
  CS* const s1 = s0 + (long long)(nz - 1) * rs;
  const F1* const bx1 = bx0 + (long long)(nz - 1) * rt;
  const F1* const by1 = ONE ? bx1 : by0 + (long long)(nz - 1) * rt;
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    if (i < nz) {
      qg[i] = s1[-i * rs];
      qbx[i] = bx1[-i * rt];
      if (!ONE) qby[i] = by1[-i * rt];
    }
  }
  const CS* pg = s1 - PF * rs;
  const F1* pbx = bx1 - PF * rt;
  const F1* pby = by1 - PF * rt;
  ps = s1;
  CA x = cplx_traits<CA>::mk(T(0), T(0));
  for (int r = 0; r < nz; r += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      if (r + i >= nz) break;
      const CA gg = cvt<CA>(qg[i]);
      const F1 bx = qbx[i], by = ONE ? bx : qby[i];
      if (r + i + PF < nz) {
        qg[i] = *pg;
        qbx[i] = *pbx;
        if (!ONE) qby[i] = *pby;
      }
      pg -= rs;
      pbx -= rt;
      if (!ONE) pby -= rt;
      x = cplx_traits<CA>::mk(fma(-bx, x.x, gg.x), fma(-by, x.y, gg.y));
      CA out = x;
      if (sing) out.x = (T)(fma(-mu, a.sing[2 * nz + (nz - 1 - r - i)], (double)out.x) - nu);
      *ps = cvt<CS>(out);
      ps -= rs;
    }
  }
}

// One thread per spectrum column (kx = j in [0, M), slot ky in [0, Ny)),
// consecutive threads on consecutive kx (every z-plane access of a warp is
// one contiguous run).  With an FP32 spectrum (the inner solve of iterative
// refinement) the near-singular columns of small |kx|, |ky| -- the singular
// Neumann (0,0) one included -- are still solved in FP64 arithmetic with the
// FP64 factors, the rest in FP32.
//
// The columns split into two launches: the main kernel takes every column
// with kx >= 1 in the spectrum's own precision, whose real and imaginary
// parts share one factor set (fewer loads and registers, deeper prefetch);
// the special kernel takes column kx = 0 of every slot (two real columns, or
// the singular one) and, for FP32 spectra, the FP64 columns.

// Column (ky, j) in full generality; PF rows of prefetch.
template <class CS, int PF = 1>
__device__ __forceinline__ void thomas_column(const ThomasArgs& a, int ky, int j) {
  // factor sets of the real (x) and imaginary (y) parts
  int kx_x = j, kx_y = j, kp_x, kp_y;
  if (a.ywall) {  // every slot its own column; column 0 holds the real pair F(0) + i F(M)
    kp_x = kp_y = ky;
    if (j == 0) kx_y = a.M;
  } else if (j > 0) {
    kp_x = kp_y = min(ky, a.ny - ky);
  } else if (2 * ky == 0 || 2 * ky == a.ny) {  // real pair F(0,ky) + i F(M,ky)
    kp_x = kp_y = ky;
    kx_y = a.M;
  } else if (2 * ky < a.ny) {  // F(0, ky)
    kp_x = kp_y = ky;
  } else {  // F(M, Ny - ky)
    kx_x = kx_y = a.M;
    kp_x = kp_y = a.ny - ky;
  }
  const bool sing = a.neumann && j == 0 && ky == 0;
  CS* const s0 = reinterpret_cast<CS*>(a.S) + (long long)ky * a.M + j;
  const long long ox = (long long)kp_x * (a.M + 1) + kx_x;
  const long long oy = (long long)kp_y * (a.M + 1) + kx_y;
  const bool fp64 = sizeof(CS) == sizeof(double2) || sing ||
                    (kx_x < a.kx64 && kp_x < a.ky64 && kx_y < a.kx64 && kp_y < a.ky64);
  // (one row of prefetch: these few columns run beside the main ones, whose
  // register budget the kernel keeps)
  if (fp64)
    sweep_column<CS, double2, false, PF>(a, s0, a.fwd + ox, a.fwd + oy, a.bwd + ox, a.bwd + oy,
                                        sing);
  else
    sweep_column<CS, float2, false, PF>(a, s0, a.fwd32 + ox, a.fwd32 + oy, a.bwd32 + ox,
                                       a.bwd32 + oy, false);
}

// Columns (ky, j) and (Ny - ky, j) of a periodic-y spectrum share one factor
// set (the eigenvalue depends on |ky|): one thread sweeps both, so that the
// factors are read once for two columns and the two recurrences are
// independent work for the same thread (the sweeps are bound by memory
// latency).  ONE factor set (kx >= 1); both columns advance row by row.
template <class CS, class CA, int PF, class F2, class F1>
__device__ __forceinline__ void sweep_pair(const ThomasArgs& a, CS* const s0, CS* const t0,
                                           const F2* const fx0, const F1* const bx0) {
  using T = typename cplx_traits<CA>::T;
  const int nz = a.nz;
  const long long rs = (long long)a.ny * a.M;         // spectrum row stride
  const long long rt = (long long)a.nky * (a.M + 1);  // factor row stride

  // forward: g_k = (s/piv_k) f_k - (A_k/piv_k) g_{k-1}, in place, both columns
  CS qu[PF], qv[PF];
  F2 qx[PF];
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    if (i < nz) {
      qu[i] = s0[i * rs];
      qv[i] = t0[i * rs];
      qx[i] = fx0[i * rt];
    }
  }
  long long off = PF * rs;  // next row to prefetch (spectrum)
  const F2* px = fx0 + PF * rt;
  long long w = 0;          // row being written
  CA g = cplx_traits<CA>::mk(T(0), T(0)), h = g;
  for (int k = 0; k < nz; k += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      if (k + i >= nz) break;
      const CA u = cvt<CA>(qu[i]), v = cvt<CA>(qv[i]);
      const F2 fx = qx[i];
      if (k + i + PF < nz) {
        qu[i] = s0[off];
        qv[i] = t0[off];
        qx[i] = *px;
      }
      off += rs;
      px += rt;
      g = cplx_traits<CA>::mk(fma(-fx.y, g.x, fx.x * u.x), fma(-fx.y, g.y, fx.x * u.y));
      h = cplx_traits<CA>::mk(fma(-fx.y, h.x, fx.x * v.x), fma(-fx.y, h.y, fx.x * v.y));
      s0[w] = cvt<CS>(g);
      t0[w] = cvt<CS>(h);
      w += rs;
    }
  }

  // backward: x_k = g_k - (C_k/piv_k) x_{k+1}, from the top wall down
  CS qg[PF], qh[PF];
  F1 qb[PF];
  const long long top = (long long)(nz - 1) * rs;
  const F1* const bx1 = bx0 + (long long)(nz - 1) * rt;
#pragma unroll
  for (int i = 0; i < PF; ++i) {
    if (i < nz) {
      qg[i] = s0[top - i * rs];
      qh[i] = t0[top - i * rs];
      qb[i] = bx1[-i * rt];
    }
  }
  off = top - PF * rs;
  const F1* pb = bx1 - PF * rt;
  w = top;
  CA x = cplx_traits<CA>::mk(T(0), T(0)), y = x;
  for (int r = 0; r < nz; r += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      if (r + i >= nz) break;
      const CA gg = cvt<CA>(qg[i]), hh = cvt<CA>(qh[i]);
      const F1 b = qb[i];
      if (r + i + PF < nz) {
        qg[i] = s0[off];
        qh[i] = t0[off];
        qb[i] = *pb;
      }
      off -= rs;
      pb -= rt;
      x = cplx_traits<CA>::mk(fma(-b, x.x, gg.x), fma(-b, x.y, gg.y));
      y = cplx_traits<CA>::mk(fma(-b, y.x, hh.x), fma(-b, y.y, hh.y));
      s0[w] = cvt<CS>(x);
      t0[w] = cvt<CS>(y);
      w -= rs;
    }
  }
}

// Rows of main blocks: periodic y pairs the slots ky and Ny - ky (kp = 0 ..
// Ny/2); y walls have every slot its own column.
__host__ __device__ inline int main_rows(const ThomasArgs& a) {
  return a.ywall ? a.ny : a.ny / 2 + 1;
}

// Whether column (ky, j >= 1) of an FP32 spectrum is solved in FP64.
__device__ __forceinline__ bool fp64_column(const ThomasArgs& a, int ky, int j) {
  const int kp = a.ywall ? ky : min(ky, a.ny - ky);
  return j < a.kx64 && kp < a.ky64;
}

template <class CS, int DEEP>
__device__ __forceinline__ void thomas_body(const ThomasArgs& a, int blk) {
  const int ky = blk / a.nblk_x;  // (the pair index kp for periodic y)
  const int j = (blk % a.nblk_x) * kThomasBlock + threadIdx.x;
  if (j == 0 || j >= a.M) return;
  if (sizeof(CS) == sizeof(float2) && fp64_column(a, ky, j)) return;
  if (!a.ywall && ky > 0 && 2 * ky != a.ny) {  // slots ky and Ny - ky together
    CS* const s0 = reinterpret_cast<CS*>(a.S) + (long long)ky * a.M + j;
    CS* const t0 = reinterpret_cast<CS*>(a.S) + (long long)(a.ny - ky) * a.M + j;
    const long long o = (long long)ky * (a.M + 1) + j;
    if constexpr (sizeof(CS) == sizeof(double2))
      sweep_pair<CS, double2, pair_prefetch_rows<double2, DEEP>::value>(a, s0, t0, a.fwd + o,
                                                                  a.bwd + o);
    else
      sweep_pair<CS, float2, pair_prefetch_rows<float2, DEEP>::value>(a, s0, t0, a.fwd32 + o,
                                                                a.bwd32 + o);
    return;
  }
  const int kp = a.ywall ? ky : min(ky, a.ny - ky);
  CS* const s0 = reinterpret_cast<CS*>(a.S) + (long long)ky * a.M + j;
  const long long o = (long long)kp * (a.M + 1) + j;
  if constexpr (sizeof(CS) == sizeof(double2))
    sweep_column<CS, double2, true, prefetch_rows<double2>::value>(a, s0, a.fwd + o, a.fwd + o,
                                                                   a.bwd + o, a.bwd + o, false);
  else
    sweep_column<CS, float2, true, prefetch_rows<float2>::value>(
        a, s0, a.fwd32 + o, a.fwd32 + o, a.bwd32 + o, a.bwd32 + o, false);
}

// Columns per slot of the special kernel: kx = 0, and for FP32 spectra the
// FP64 columns kx < kx64.
template <class CS>
__host__ __device__ inline int special_width(const ThomasArgs& a) {
  if (sizeof(CS) == sizeof(double2)) return 1;
  const int w = a.kx64 > 1 ? a.kx64 : 1;
  return w < a.M ? w : a.M;
}

template <class CS, int PF = 1>
__device__ __forceinline__ void thomas_special_body(const ThomasArgs& a, int blk) {
  const int kxs = special_width<CS>(a);
  const int t = blk * kThomasBlock + threadIdx.x;
  const int j = t % kxs, ky = t / kxs;
  if (ky >= a.ny) return;
  if (j > 0 && !fp64_column(a, ky, j)) return;  // the main kernel's column
  thomas_column<CS, PF>(a, ky, j);
}

template <class CS>
__host__ __device__ inline int special_blocks(const ThomasArgs& a) {
  return (a.ny * special_width<CS>(a) + kThomasBlock - 1) / kThomasBlock;
}

// One launch: the special columns' blocks first (their sweeps are the
// longest-latency ones and overlap the main columns), then the main blocks.
template <class CS, int DEEP>
__device__ __forceinline__ void thomas_launch_body(const ThomasArgs& a, int blk) {
  const int nsp = special_blocks<CS>(a);
  if (blk < nsp) thomas_special_body<CS>(a, blk);
  else thomas_body<CS, DEEP>(a, blk - nsp);
}

// Resident blocks the register budget is sized for: 14 per SM, or 8 / 6
// with deeper prefetch queues (DEEP 4 / 6) for launches that fit in one wave
// of those.
template <class CS, int DEEP>
__global__ void __launch_bounds__(kThomasBlock, DEEP == 6 ? 6 : (DEEP == 4 ? 8 : 14))
    thomas_kernel(ThomasArgs a) {
  thomas_launch_body<CS, DEEP>(a, blockIdx.x);
}

// One launch for several boxes (FP32 inner solves of grouped refinement).
__global__ void __launch_bounds__(kThomasBlock, 14) thomas_group_kernel(const ThomasArgs* boxes,
                                                                        GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  thomas_launch_body<float2, 0>(boxes[b], blk);
}

template <class CS>
static cudaError_t launch_streaming(const ThomasArgs& a, cudaStream_t st) {
  const long long blocks = special_blocks<CS>(a) + (long long)a.nblk_x * main_rows(a);
  static std::atomic<int> sms{0};  // SMs of the device (the same on every GB300 of a process)
  int nsm = sms.load(std::memory_order_relaxed);
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    sms.store(nsm, std::memory_order_relaxed);
  }
  if constexpr (sizeof(CS) == sizeof(double2)) {
    if (blocks <= 6LL * nsm) {
      thomas_kernel<CS, 6><<<(unsigned)blocks, kThomasBlock, 0, st>>>(a);
      return cudaGetLastError();
    }
    if (blocks <= 8LL * nsm) {
      thomas_kernel<CS, 4><<<(unsigned)blocks, kThomasBlock, 0, st>>>(a);
      return cudaGetLastError();
    }
  }
  thomas_kernel<CS, 0><<<(unsigned)blocks, kThomasBlock, 0, st>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// FP32 spectra: Algorithm 2 (Sec. 2.2.4) over z-partitions held in registers.
// The streaming sweep above writes its forward intermediate to the spectrum
// and reads it back, and reads factor tables: about 2.3 times the one read and
// one write of the spectrum a z solve needs.  Here thread (q, c) of a CTA
// holds rows [8q, 8q + 8) of column c of a tile of C consecutive kx, for the
// slots ky and Ny - ky at once (they share the eigenvalue, so four real
// right-hand sides share one elimination; one slot with y walls).  Rows past
// Nz are identity rows x = 0, uncoupled because the wall row has C = 0.  A
// warp's loads and stores cover C consecutive complex values of one row.  The
// thread forms its rows of Eq. 12 on the fly from the plan's z operator and
// eigenvalues, divided by the inverse-FFT normalisation s,
//   (A_k F_{k-1} + (B_k + lx[kx] + ly[ky]) F_k + C_k F_{k+1}) / s = f_k
// (FP32 arithmetic is cheap on GB300; no per-column table is read), and runs
// Steps 1 and 2 of Algorithm 2 together, rows normalised:
//  * downward, with x_0 a parameter: piv_i = D_i - A_i c'_{i-1} (piv_1 = D_1),
//    c'_i = C_i / piv_i, g'_i = -A_i g'_{i-1} / piv_i (g'_1 = A_1 / D_1),
//    d'_i = (d_i - A_i d'_{i-1}) / piv_i; row i then reads
//    x_i + c'_i x_{i+1} + g'_i x_0 = d'_i  (i = 1 .. 7);
//  * upward, x_i = u_i - v_i x_0 - w_i x_7 for i = 6 .. 1 carried as scalars
//    into row 0: A_0 x_{-1} + (D_0 - C_0 v_1) x_0 - C_0 w_1 x_7 = d_0 - C_0 u_1.
// Row 0 and row 7 of every partition form the 2P-row reduced system of the
// column (Step 3), solved in shared memory by cyclic reduction (multipliers
// formed on the fly; O(P) work), and each thread then recovers its interior
// rows by back substitution in the downward form (Step 4),
// x_i = d'_i - c'_i x_{i+1} - g'_i x_0.  Per row a thread keeps d' (two
// complex values) and c', g' in registers; the spectrum is read once and
// written once.  The FP64 columns of an FP32 spectrum and the kx = 0 slots
// run in the launch's first blocks, as in the streaming kernel.
// ----------------------------------------------------------------------------
constexpr int kZPartThreads = 256;  // at most C * P threads per CTA
constexpr int kZPartMaxParts = 64;
constexpr int kZPartRows = 8;  // rows per partition (register arrays): Nz <= 512

// Reciprocals by the fast hardware approximation (a few ulp): the inner
// solve needs FP32 accuracy only, the refinement corrects the rest, and the
// correctly rounded form would add a slow-path call per row.
__device__ __forceinline__ float zp_rcp(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ float2 f2_fms(float2 a, float k, float2 b) {  // a - k b
  return make_float2(fmaf(-k, b.x, a.x), fmaf(-k, b.y, a.y));
}

// Shared memory of a tile: the operator rows of the column, partition by
// partition with one float4 of padding after each (so that the lanes of a
// warp, which read the same row of different partitions, hit different
// banks), then the reduced system: per row (sub, diag, sup, -) and the two
// slots' complex right-hand sides.
__host__ __device__ inline int zpart_rows_smem(int P, int MM) { return P * (MM + 1); }

__device__ __forceinline__ float4 f4_fms(float4 a, float k, float4 b) {  // a - k b
  return make_float4(fmaf(-k, b.x, a.x), fmaf(-k, b.y, a.y), fmaf(-k, b.z, a.z),
                     fmaf(-k, b.w, a.w));
}

template <int MM>
__device__ __forceinline__ void zpart_body(const ZPartArgs& z, int tile) {
  const ThomasArgs& a = z.t;
  const int C = z.C, P = z.P, J = 2 * P;
  const int kp = tile / z.ntx;  // slot ky (and its partner Ny - ky with periodic y)
  const bool live = (int)threadIdx.x < C * P;  // the others only join the barriers
  const int c = threadIdx.x % C, q = live ? threadIdx.x / C : 0;
  const int j = (tile % z.ntx) * C + c;
  const bool active = live && j >= 1 && j < a.M && !fp64_column(a, kp, j);
  const int ky2 = (!a.ywall && kp > 0 && 2 * kp != a.ny) ? a.ny - kp : kp;
  const bool two = active && ky2 != kp;
  const int r0 = q * MM;  // every partition MM rows; rows past nz are x = 0
  const long long rs = (long long)a.ny * a.M;
  float2* const base = reinterpret_cast<float2*>(a.S) + (long long)r0 * rs + (active ? j : 0);
  float2* const col = base + (long long)kp * a.M;
  float2* const col2 = base + (long long)ky2 * a.M;

  extern __shared__ __align__(16) unsigned char zsm[];
  float4* const srow = reinterpret_cast<float4*>(zsm);
  for (int k = threadIdx.x; k < P * MM; k += blockDim.x) srow[k + k / MM] = __ldg(z.zrow + k);
  float2 u[MM], v[MM];  // right-hand sides of the two slots, then d'
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    u[i] = v[i] = make_float2(0.0f, 0.0f);
    if (active && r0 + i < a.nz) u[i] = col[i * rs];
    if (two && r0 + i < a.nz) v[i] = col2[i * rs];
  }
  // (inactive lanes solve a harmless zero column with the largest shift)
  const float lam = active ? z.lam[j] + z.lam[a.M + 1 + kp] : z.lam[a.M];
  __syncthreads();
  const float4* const zr = srow + q * (MM + 1);

  // downward, rows normalised: x_i + c'_i x_{i+1} + g'_i x_0 = d'_i (i >= 1).
  // The rows and eigenvalues are divided by the normalisation s, so that the
  // solution comes out scaled by s.
  float cq[MM], gq[MM];
  {
    const float4 r = zr[1];
    const float ib = zp_rcp(fmaf(lam, r.w, r.y));
    cq[1] = r.z * ib;
    gq[1] = r.x * ib;
    u[1] = make_float2(u[1].x * ib, u[1].y * ib);
    v[1] = make_float2(v[1].x * ib, v[1].y * ib);
  }
  cq[0] = gq[0] = 0.0f;
#pragma unroll
  for (int i = 2; i < MM; ++i) {
    const float4 r = zr[i];
    const float ib = zp_rcp(fmaf(-r.x, cq[i - 1], fmaf(lam, r.w, r.y)));
    cq[i] = r.z * ib;
    gq[i] = -(r.x * ib) * gq[i - 1];
    const float2 t = f2_fms(u[i], r.x, u[i - 1]), w = f2_fms(v[i], r.x, v[i - 1]);
    u[i] = make_float2(t.x * ib, t.y * ib);
    v[i] = make_float2(w.x * ib, w.y * ib);
  }
  // upward to row 0: x_i = uu_i - vv_i x_0 - ww_i x_{MM-1}, carried as scalars
  float2 uu = u[MM - 2], uv = v[MM - 2];
  float vv = gq[MM - 2], ww = cq[MM - 2];
#pragma unroll
  for (int i = MM - 3; i >= 1; --i) {
    const float ci = cq[i];
    uu = f2_fms(u[i], ci, uu);
    uv = f2_fms(v[i], ci, uv);
    vv = fmaf(-ci, vv, gq[i]);
    ww = -ci * ww;
  }
  const float4 rz = zr[0];

  // the reduced system (Step 3): row 2q is the partition's row 0, row 2q + 1
  // its row MM-1; column c's row k at index k * C + c.  Solved by cyclic
  // reduction: at stride s the rows k = -1 mod 2s take away rows k -+ s,
  // down to the single row 2^L - 1; then back substitution.
  float4* const cA = srow + zpart_rows_smem(P, MM);  // (sub, diag, sup, -)
  float4* const cY = cA + J * C;                     // (slot 1, slot 2) right-hand sides
  if (live) {
    cA[(2 * q) * C + c] =
        make_float4(rz.x, fmaf(-rz.z, vv, fmaf(lam, rz.w, rz.y)), -rz.z * ww, 0.0f);
    cY[(2 * q) * C + c] = make_float4(fmaf(-rz.z, uu.x, u[0].x), fmaf(-rz.z, uu.y, u[0].y),
                                      fmaf(-rz.z, uv.x, v[0].x), fmaf(-rz.z, uv.y, v[0].y));
    cA[(2 * q + 1) * C + c] = make_float4(gq[MM - 1], 1.0f, cq[MM - 1], 0.0f);
    cY[(2 * q + 1) * C + c] = make_float4(u[MM - 1].x, u[MM - 1].y, v[MM - 1].x, v[MM - 1].y);
  }
  __syncthreads();
  const int k1 = 2 * q + 1;  // the odd row this thread updates
  int s = 1;
  for (; 2 * s <= J; s <<= 1) {
    if (live && ((k1 + 1) & (2 * s - 1)) == 0) {
      float4 m = cA[k1 * C + c];
      float4 y = cY[k1 * C + c];
      const float4 lo = cA[(k1 - s) * C + c];
      const float e1 = m.x * zp_rcp(lo.y);
      float diag = fmaf(-e1, lo.z, m.y);
      const float sub = -e1 * lo.x;
      float sup = 0.0f;
      y = f4_fms(y, e1, cY[(k1 - s) * C + c]);
      if (k1 + s < J) {
        const float4 hi = cA[(k1 + s) * C + c];
        const float e2 = m.z * zp_rcp(hi.y);
        diag = fmaf(-e2, hi.x, diag);
        sup = -e2 * hi.z;
        y = f4_fms(y, e2, cY[(k1 + s) * C + c]);
      }
      cA[k1 * C + c] = make_float4(sub, diag, sup, 0.0f);
      cY[k1 * C + c] = y;
    }
    __syncthreads();
  }
  // s is now the first stride with no update: the last row updated is s - 1
  if (live && k1 == s - 1) {
    const float id = zp_rcp(cA[k1 * C + c].y);
    const float4 y = cY[k1 * C + c];
    cY[k1 * C + c] = make_float4(y.x * id, y.y * id, y.z * id, y.w * id);
  }
  __syncthreads();
  for (int h = s >> 1; h >= 1; h >>= 1) {  // rows k = h - 1 mod 2h, from x_{k -+ h}
    const int k = (h == 1) ? 2 * q : k1;
    if (live && ((k + 1) & (2 * h - 1)) == h) {
      const float4 m = cA[k * C + c];
      float4 y = cY[k * C + c];
      if (k - h >= 0) y = f4_fms(y, m.x, cY[(k - h) * C + c]);
      if (k + h < J) y = f4_fms(y, m.z, cY[(k + h) * C + c]);
      const float id = zp_rcp(m.y);
      cY[k * C + c] = make_float4(y.x * id, y.y * id, y.z * id, y.w * id);
    }
    __syncthreads();
  }
  const float4 x0 = cY[(2 * q) * C + c], xl = cY[k1 * C + c];

  // back substitution in the downward form, rows MM-2 .. 1
  u[MM - 1] = make_float2(xl.x, xl.y);
  v[MM - 1] = make_float2(xl.z, xl.w);
#pragma unroll
  for (int i = MM - 2; i >= 1; --i) {
    u[i] = make_float2(fmaf(-cq[i], u[i + 1].x, fmaf(-gq[i], x0.x, u[i].x)),
                       fmaf(-cq[i], u[i + 1].y, fmaf(-gq[i], x0.y, u[i].y)));
    v[i] = make_float2(fmaf(-cq[i], v[i + 1].x, fmaf(-gq[i], x0.z, v[i].x)),
                       fmaf(-cq[i], v[i + 1].y, fmaf(-gq[i], x0.w, v[i].y)));
  }
  u[0] = make_float2(x0.x, x0.y);
  v[0] = make_float2(x0.z, x0.w);
#pragma unroll
  for (int i = 0; i < MM; ++i) {
    if (active && r0 + i < a.nz) col[i * rs] = u[i];
    if (two && r0 + i < a.nz) col2[i * rs] = v[i];
  }
}

// Block blk of one box: the FP64 and kx = 0 columns first, then the tiles.
template <int MM>
__device__ __forceinline__ void zpart_block(const ZPartArgs& z, int blk) {
  if (blk < z.nsp) {
    // (a deeper prefetch than in the streaming kernel: here the main columns
    // finish sooner, and these serial sweeps would be the launch's tail)
    if (threadIdx.x < kThomasBlock) thomas_special_body<float2, 4>(z.t, blk);
    return;
  }
  zpart_body<MM>(z, blk - z.nsp);
}

__global__ void __launch_bounds__(kZPartThreads, 2) zpart_kernel(ZPartArgs z) {
  zpart_block<kZPartRows>(z, (int)blockIdx.x);
}

// One launch for several boxes (FP32 inner solves of grouped refinement): the
// same blocks as each box alone, so the same bits.
__global__ void __launch_bounds__(kZPartThreads, 2) zpart_group_kernel(const ZPartArgs* boxes,
                                                                       GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  zpart_block<kZPartRows>(boxes[b], blk);
}

static ThomasArgs thomas_args(const cfs_plan* P, void* data);

// Rows per partition (MM) for nz rows; 0 if the partitioned solve does not
// apply.  The operator table holds ceil(nz / MM) MM <= nz + kZPartRowPad rows.
static int zpart_rows(int nz) {
  return (nz >= 3 && (nz + kZPartRows - 1) / kZPartRows <= kZPartMaxParts) ? kZPartRows : 0;
}

static bool zpart_ok(const cfs_plan* P) {
  return P->dtype == CFS_F32_REFINED && P->d_zrow32 && P->d_lam32 && zpart_rows(P->nz) > 0;
}

// The launch of one plan's partitioned solve on `data`; returns its blocks.
static int zpart_args(const cfs_plan* P, float* data, ZPartArgs* z) {
  z->t = thomas_args(P, data);
  z->zrow = P->d_zrow32;
  z->lam = P->d_lam32;
  z->mm = zpart_rows(P->nz);
  z->P = (P->nz + z->mm - 1) / z->mm;
  int C = 4;  // the widest tile within the thread budget (more than half of it)
  while (2 * C * z->P <= kZPartThreads) C *= 2;
  z->C = C;
  z->ntx = (P->M + C - 1) / C;
  z->nsp = special_blocks<float2>(z->t);
  return z->nsp + main_rows(z->t) * z->ntx;  // slot pairs (ky, Ny - ky), or slots (y walls)
}

static size_t zpart_smem(const ZPartArgs& z) {
  return sizeof(float4) * ((size_t)zpart_rows_smem(z.P, z.mm) + (size_t)2 * (2 * z.P) * z.C);
}

static cudaError_t launch_zpart(const cfs_plan* P, float* data, cudaStream_t st) {
  ZPartArgs z;
  const int blocks = zpart_args(P, data, &z);
  zpart_kernel<<<blocks, kZPartThreads, zpart_smem(z), st>>>(z);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Shared-memory tiles.  A CTA takes TW consecutive spectrum columns (kx in
// [j0, j0 + TW)) of one slot ky with all Nz rows: the Tensor Memory
// Accelerator copies the tile into shared memory (rows of TW complex values),
// both sweeps run there, and TMA writes the tile back.  Global memory sees one
// read and one write of the spectrum plus the factors; the streaming kernel
// above also writes g and reads it back.  One thread per real component:
// thread 2c + r sweeps the real (r = 0) or imaginary (r = 1) part of column c
// with the factor set of that part.  The factor rows of every thread stream
// through a per-thread ring in shared memory that cp.async fills DG groups of
// kTileG rows ahead of the sweep; a group's loads are issued together, so the
// shared-memory latency is paid once per group and not once per row.  CTAs
// are persistent over tiles, and several CTAs per SM overlap one tile's copies
// with another's sweeps.  Tiles run in the slot order ky = 0, Ny-1, 1, Ny-2,
// ... so that slots ky and Ny-ky, which share their factors, are swept close
// together in time.
// ----------------------------------------------------------------------------
constexpr int kTileG = 8;  // rows per prefetch group

template <class A> struct tile_fac;
template <> struct tile_fac<double> { using F2 = double2; };
template <> struct tile_fac<float> { using F2 = float2; };

// Both sweeps of one real component: col[k * NT] is its row k (storage type
// S, arithmetic type A); f2 / f1 point at its forward / backward factors of
// row 0 (row stride rt); ring is its slot 0 (16-byte slots, NT * 16 bytes
// apart).  `pin` marks the singular Neumann column: row 0 is pinned, and the
// output is corrected by mu * hs_k + nu (the two dz-weighted means).
template <class A, class S, int NT, int DG>
__device__ __forceinline__ void tile_sweeps(S* col, const typename tile_fac<A>::F2* f2,
                                            const A* f1, long long rt, int nz, bool pin,
                                            const double* hs, double mu, double nu,
                                            unsigned char* ring) {
  using F2 = typename tile_fac<A>::F2;
  constexpr int G = kTileG;
  constexpr int RG = DG + 1;  // ring groups: group q + DG refills the slots of group q - 1
  constexpr int SLOT = NT * 16;
  const int ng = (nz + G - 1) / G;

  // forward: g_k = (s/piv_k) u_k - (A_k/piv_k) g_{k-1}
  for (int q = 0; q < DG; ++q) {
    if (q < ng) {
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int k = q * G + i;
        if (k < nz) cp_async<(int)sizeof(F2)>(ring + (q * G + i) * SLOT, f2 + k * rt);
      }
    }
    cp_async_commit();
  }
  A g = A(0);
  int rg = 0;
  for (int q = 0; q < ng; ++q) {
    cp_async_wait<DG - 1>();
    const int k0 = q * G;
    F2 f[G];
    A u[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      if (k0 + i < nz) {
        f[i] = *reinterpret_cast<const F2*>(ring + (rg * G + i) * SLOT);
        u[i] = (A)col[(k0 + i) * NT];
      }
    }
    const int qn = q + DG;
    if (qn < ng) {
      const int rn = (rg + DG) % RG;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int k = qn * G + i;
        if (k < nz) cp_async<(int)sizeof(F2)>(ring + (rn * G + i) * SLOT, f2 + k * rt);
      }
    }
    cp_async_commit();
    rg = (rg + 1 == RG) ? 0 : rg + 1;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      if (k0 + i < nz) {
        const A uu = (pin && k0 + i == 0) ? A(0) : u[i];
        g = fma(-f[i].y, g, f[i].x * uu);
        col[(k0 + i) * NT] = (S)g;
      }
    }
  }
  cp_async_wait<0>();

  // backward, from the top wall down: x_k = g_k - (C_k/piv_k) x_{k+1}
  for (int q = 0; q < DG; ++q) {
    if (q < ng) {
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int k = nz - 1 - (q * G + i);
        if (k >= 0) {
          unsigned char* d = ring + (q * G + i) * SLOT;
          cp_async<(int)sizeof(A)>(d, f1 + k * rt);
          if (pin) cp_async<8>(d + 8, hs + k);
        }
      }
    }
    cp_async_commit();
  }
  A x = A(0);
  rg = 0;
  for (int q = 0; q < ng; ++q) {
    cp_async_wait<DG - 1>();
    const int k0 = nz - 1 - q * G;  // rows k0, k0 - 1, ..
    A b[G], gg[G];
    double h[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      if (k0 - i >= 0) {
        const unsigned char* d = ring + (rg * G + i) * SLOT;
        b[i] = *reinterpret_cast<const A*>(d);
        h[i] = pin ? *reinterpret_cast<const double*>(d + 8) : 0.0;
        gg[i] = (A)col[(k0 - i) * NT];
      }
    }
    const int qn = q + DG;
    if (qn < ng) {
      const int rn = (rg + DG) % RG;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int k = nz - 1 - (qn * G + i);
        if (k >= 0) {
          unsigned char* d = ring + (rn * G + i) * SLOT;
          cp_async<(int)sizeof(A)>(d, f1 + k * rt);
          if (pin) cp_async<8>(d + 8, hs + k);
        }
      }
    }
    cp_async_commit();
    rg = (rg + 1 == RG) ? 0 : rg + 1;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      if (k0 - i >= 0) {
        x = fma(-b[i], x, gg[i]);
        A out = x;
        if (pin) out = (A)(fma(-mu, h[i], (double)out) - nu);
        col[(k0 - i) * NT] = (S)out;
      }
    }
  }
  cp_async_wait<0>();
}

template <class CS, int TW, int DG>
__global__ void __launch_bounds__(2 * TW) thomas_tile_kernel(const __grid_constant__ CUtensorMap map,
                                                             ThomasArgs a, int bz, int nbox,
                                                             int* status) {
  using T = typename cplx_traits<CS>::T;
  constexpr int NT = 2 * TW;
  constexpr unsigned kMask = NT == 32 ? 0xffffffffu : ((1u << NT) - 1u);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* tile = reinterpret_cast<T*>(smem_raw + 128);  // [nbox * bz][NT]
  const int rows = nbox * bz;
  const int tid = threadIdx.x;
  unsigned char* ring = reinterpret_cast<unsigned char*>(tile + (size_t)rows * NT) + tid * 16;
  const int nbx = (a.M + TW - 1) / TW;
  const long long ntiles = (long long)nbx * a.ny;
  const uint32_t tile_bytes = (uint32_t)((size_t)rows * NT * sizeof(T));
  const long long rt = (long long)a.nky * (a.M + 1);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int sidx = (int)(t / nbx);
    const int j0 = (int)(t % nbx) * TW;
    const int ky = (sidx & 1) ? a.ny - ((sidx + 1) >> 1) : (sidx >> 1);
    if (tid == 0) {
      mbar_expect_tx(bar, tile_bytes);
      for (int b = 0; b < nbox; ++b)
        tma_load_3d(tile + (size_t)b * bz * NT, &map, bar, 2 * j0, ky, b * bz);
    }
    if (!cta_wait(bar, phase, status)) return;
    phase ^= 1u;
    // Singular Neumann column (real part of column 0, slot 0): the
    // dz-weighted mean of its right-hand side (mu) and, through g^T E', that
    // of the pinned solution (nu), reduced over the loaded tile.
    const bool sing_tile = a.neumann && ky == 0 && j0 == 0;
    double mu = 0.0, nu = 0.0;
    if (sing_tile) {
      double pm = 0.0, pg = 0.0;
      for (int k = tid; k < a.nz; k += NT) {
        const double e = (double)tile[(size_t)k * NT];
        pm = fma(a.sing[k], e, pm);
        if (k > 0) pg = fma(a.sing[a.nz + k], e, pg);
      }
#pragma unroll
      for (int o = NT / 2; o > 0; o >>= 1) {
        pm += __shfl_xor_sync(kMask, pm, o);
        pg += __shfl_xor_sync(kMask, pg, o);
      }
      mu = pm;
      nu = a.sing_sc * (pg - mu * a.sing_cg);
    }
    const int c = tid >> 1, comp = tid & 1;
    const int j = j0 + c;
    if (j < a.M) {
      int kx = j, kp;
      if (a.ywall) {
        kp = ky;
        if (j == 0 && comp) kx = a.M;
      } else if (j > 0) {
        kp = min(ky, a.ny - ky);
      } else if (2 * ky == 0 || 2 * ky == a.ny) {  // real pair F(0,ky) + i F(M,ky)
        kp = ky;
        kx = comp ? a.M : 0;
      } else if (2 * ky < a.ny) {  // F(0, ky)
        kp = ky;
      } else {  // F(M, Ny - ky)
        kx = a.M;
        kp = a.ny - ky;
      }
      const bool pin = sing_tile && tid == 0;
      const long long off = (long long)kp * (a.M + 1) + kx;
      T* col = tile + tid;
      if constexpr (sizeof(T) == 8) {
        tile_sweeps<double, T, NT, DG>(col, a.fwd + off, a.bwd + off, rt, a.nz, pin,
                                       a.sing + 2 * a.nz, mu, nu, ring);
      } else {
        if (pin || (kx < a.kx64 && kp < a.ky64))
          tile_sweeps<double, T, NT, DG>(col, a.fwd + off, a.bwd + off, rt, a.nz, pin,
                                         a.sing + 2 * a.nz, mu, nu, ring);
        else
          tile_sweeps<float, T, NT, DG>(col, a.fwd32 + off, a.bwd32 + off, rt, a.nz, false,
                                        nullptr, 0.0, 0.0, ring);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      for (int b = 0; b < nbox; ++b)
        tma_store_3d(&map, tile + (size_t)b * bz * NT, 2 * j0, ky, b * bz);
      tma_store_commit_and_wait_read();  // the tile may be reloaded
    }
  }
}

static ThomasArgs thomas_args(const cfs_plan* P, void* data) {
  ThomasArgs a;
  a.S = data;
  a.fwd = P->d_fwd;
  a.bwd = P->d_bwd;
  a.fwd32 = P->d_fwd32;
  a.bwd32 = P->d_bwd32;
  a.sing = P->d_sing;
  a.sing_cg = P->sing_cg;
  a.sing_sc = P->sing_sc;
  a.M = P->M;
  a.ny = P->ny;
  a.nz = P->nz;
  a.nky = P->nky;
  a.nblk_x = (P->M + kThomasBlock - 1) / kThomasBlock;
  a.neumann = P->has_null;
  a.kx64 = P->kx64;
  a.ky64 = P->ky64;
  a.ywall = (P->ybc != CFS_Y_PERIODIC);
  return a;
}

// Rows per TMA box: at most 256, even when rows are 64 bytes so that every
// box starts on a 128-byte boundary of the tile.
static void tile_boxes(int nz, int row_bytes, int* nbox, int* bz) {
  *nbox = (nz + 255) / 256;
  *bz = (nz + *nbox - 1) / *nbox;
  if ((row_bytes % 128) && (*bz % 2)) ++*bz;
}

template <class CS, int TW, int DG>
static size_t tile_smem(int nz) {
  using T = typename cplx_traits<CS>::T;
  int nbox, bz;
  tile_boxes(nz, 2 * TW * (int)sizeof(T), &nbox, &bz);
  return 128 + (size_t)nbox * bz * 2 * TW * sizeof(T) + (size_t)(DG + 1) * kTileG * 2 * TW * 16;
}

// CTAs of the tile kernel resident per SM (0 if it cannot run).
template <class CS, int TW, int DG>
static int tile_occupancy(int nz) {
  const size_t smem = tile_smem<CS, TW, DG>(nz);
  if (smem > 227 * 1024) return 0;
  auto kern = thomas_tile_kernel<CS, TW, DG>;
  if (allow_max_smem(kern) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 2 * TW, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

template <class CS, int TW, int DG>
static cudaError_t launch_tile(const cfs_plan* P, void* data, cudaStream_t st) {
  using T = typename cplx_traits<CS>::T;
  const int per_sm = tile_occupancy<CS, TW, DG>(P->nz);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  ThomasArgs a = thomas_args(P, data);
  int nbox, bz;
  tile_boxes(P->nz, 2 * TW * (int)sizeof(T), &nbox, &bz);
  CUtensorMap map;
  const cuuint64_t gdim[3] = {(cuuint64_t)(2 * P->M), (cuuint64_t)P->ny, (cuuint64_t)P->nz};
  const cuuint64_t gstride[2] = {(cuuint64_t)(2 * P->M) * sizeof(T),
                                 (cuuint64_t)(2 * P->M) * P->ny * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * TW), 1, (cuuint32_t)bz};
  if (!encode_map(&map, sizeof(T), 3, data, gdim, gstride, box)) return cudaErrorInvalidValue;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
  const long long ntiles = (long long)((P->M + TW - 1) / TW) * P->ny;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  thomas_tile_kernel<CS, TW, DG><<<(unsigned)grid, 2 * TW, tile_smem<CS, TW, DG>(P->nz), st>>>(
      map, a, bz, nbox, P->d_status);
  return cudaGetLastError();
}

// Prefetch depth (groups of kTileG rows) of the factor ring.  An FP64 sweep
// spends longer per row, so fewer rows in flight cover the same latency; the
// narrow tile leaves shared memory for a deeper ring.
template <class CS, int TW> struct tile_depth { static constexpr int DG = TW == 8 ? 6 : 2; };

// Tile width for this plan: the forced one, or the one that keeps more
// threads resident per SM (the wider tile on a tie); -1 = streaming kernel.
template <class CS>
static int pick_tile_width(const cfs_plan* P, int tw) {
  constexpr int D16 = tile_depth<CS, 16>::DG, D8 = tile_depth<CS, 8>::DG;
  if (tw == 1)  // the partitioned solve: FP32 spectra (FP64 sweeps stream)
    return sizeof(CS) == sizeof(float2) ? (zpart_ok(P) ? 1 : 0) : -1;
  // FP32 spectra take no tiles: their grouped solves have no tile variant,
  // and a box must give the same bits grouped as alone
  if constexpr (sizeof(CS) == sizeof(float2)) {
    return (tw == -1 || tw == 0 || tw == 8 || tw == 16) ? -1 : 0;
  } else {
    if (tw == -1) return -1;
    if (tw == 16) return tile_occupancy<CS, 16, D16>(P->nz) >= 1 ? 16 : 0;
    if (tw == 8) return tile_occupancy<CS, 8, D8>(P->nz) >= 1 ? 8 : 0;
    if (tw != 0) return 0;
    return -1;  // measured fastest at the workload sizes so far
  }
}

int thomas_tile_width(const cfs_plan* P, bool fp32, int tw) {
  return fp32 ? pick_tile_width<float2>(P, tw) : pick_tile_width<double2>(P, tw);
}

template <class CS>
static cudaError_t launch_thomas_t(const cfs_plan* P, void* data, cudaStream_t st) {
  const int tw = pick_tile_width<CS>(P, P->thomas_tw);
  if constexpr (sizeof(CS) == sizeof(float2))
    if (tw == 1) return launch_zpart(P, static_cast<float*>(data), st);
  if constexpr (sizeof(CS) == sizeof(double2)) {
    if (tw == 16) return launch_tile<CS, 16, tile_depth<CS, 16>::DG>(P, data, st);
    if (tw == 8) return launch_tile<CS, 8, tile_depth<CS, 8>::DG>(P, data, st);
  }
  return launch_streaming<CS>(thomas_args(P, data), st);
}

cudaError_t launch_thomas(const cfs_plan* P, double* data, cudaStream_t st) {
  return launch_thomas_t<double2>(P, data, st);
}

cudaError_t launch_thomas32(const cfs_plan* P, float* data, cudaStream_t st) {
  if (!P->d_fwd32) return cudaErrorInvalidValue;
  return launch_thomas_t<float2>(P, data, st);
}

// ----------------------------------------------------------------------------
// Plan-time factorisation, one thread per (kx, kyp), FP64 with true division.
// The Neumann (0, 0) system is pinned: row 0 becomes F_0 = 0 (B_0 -> 1,
// C_0 -> 0).
// ----------------------------------------------------------------------------
__global__ void thomas_factor_kernel(double2* fwd, double* bwd, float2* fwd32, float* bwd32,
                                     const double* A, const double* B, const double* C,
                                     const double* lamx, const double* lamy, int M, int nky, int nz,
                                     double s, int neumann) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int kyp = blockIdx.y;
  if (kx > M) return;
  const double lam = lamx[kx] + lamy[kyp];
  const double sc = s;
  const bool pin = neumann && kx == 0 && kyp == 0;
  double piv = 1.0, cprev = 0.0;
  for (int k = 0; k < nz; ++k) {
    double b = B[k] + lam;
    double c = C[k];
    if (k == 0) {
      if (pin) {
        b = 1.0;
        c = 0.0;
      }
      piv = b;
    } else {
      piv = b - A[k] * cprev / piv;
    }
    const long long t = ((long long)k * nky + kyp) * (M + 1) + kx;
    const double2 f = make_double2(sc / piv, (k == 0 ? 0.0 : A[k]) / piv);
    fwd[t] = f;
    bwd[t] = c / piv;
    if (fwd32) {  // rounded copies for the FP32 inner solves of refinement
      fwd32[t] = make_float2((float)f.x, (float)f.y);
      bwd32[t] = (float)(c / piv);
    }
    cprev = c;
  }
}

cudaError_t launch_thomas_factor_set(const cfs_plan* P, double2* fwd, double* bwd, int n,
                                     const double* dA, const double* dB, const double* dC,
                                     const double* dlx, const double* dly, cudaStream_t st) {
  const double s = 2.0 / ((double)P->nx * (double)P->ny);
  dim3 grid((P->M + 1 + 127) / 128, P->nky);
  thomas_factor_kernel<<<grid, 128, 0, st>>>(fwd, bwd, nullptr, nullptr, dA, dB, dC, dlx, dly,
                                             P->M, P->nky, n, s, 0);
  return cudaGetLastError();
}

cudaError_t launch_thomas_set(const cfs_plan* P, double* data, const double2* fwd,
                              const double* bwd, int n, cudaStream_t st) {
  ThomasArgs a = thomas_args(P, data);
  a.fwd = fwd;
  a.bwd = bwd;
  a.fwd32 = nullptr;
  a.bwd32 = nullptr;
  a.nz = n;
  a.neumann = 0;
  a.kx64 = a.ky64 = 0;  // (ywall as for the plan)
  return launch_streaming<double2>(a, st);
}

cudaError_t launch_thomas_factor(cfs_plan* P, const double* dA, const double* dB, const double* dC,
                                 const double* dlamx, const double* dlamy, cudaStream_t st) {
  const double s = 2.0 / ((double)P->nx * (double)P->ny);
  dim3 grid((P->M + 1 + 127) / 128, P->nky);
  thomas_factor_kernel<<<grid, 128, 0, st>>>(P->d_fwd, P->d_bwd, P->d_fwd32, P->d_bwd32, dA, dB,
                                             dC, dlamx, dlamy, P->M, P->nky, P->nz, s,
                                             P->has_null);
  return cudaGetLastError();
}

size_t thomas_group_box(const cfs_plan* P, ThomasArgs* box, int* blocks) {
  *box = thomas_args(P, P->d_r32);
  *blocks = special_blocks<float2>(*box) + box->nblk_x * main_rows(*box);
  return 0;
}

bool zpart_group_member(const cfs_plan* P) { return pick_tile_width<float2>(P, P->thomas_tw) == 1; }

size_t zpart_group_box(const cfs_plan* P, ZPartArgs* box, int* blocks) {
  *blocks = zpart_args(P, P->d_r32, box);
  return zpart_smem(*box);
}

cudaError_t launch_zpart_group(const ZPartArgs* boxes, GroupMap g, int total, size_t smem,
                               cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  zpart_group_kernel<<<total, kZPartThreads, smem, st>>>(boxes, g);
  return cudaGetLastError();
}

cudaError_t launch_thomas_group32(const ThomasArgs* boxes, GroupMap g, int total,
                                  cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  thomas_group_kernel<<<total, kThomasBlock, 0, st>>>(boxes, g);
  return cudaGetLastError();
}

}  // namespace chanfs
