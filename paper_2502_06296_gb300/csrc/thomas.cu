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
#include "chanfs_internal.cuh"

namespace chanfs {

struct ThomasArgs {
  void* S;               // spectrum (Nz, Ny, M) complex, double2 or float2
  const double2* fwd;    // FP64 factors (s/piv, A/piv) per (k, kyp, kx in [0, M])
  const double* bwd;     // FP64 C/piv
  const float2* fwd32;   // FP32 copies (refined plans only)
  const float* bwd32;
  const double* sing;    // Neumann (0,0): wn | gn | hs, 3*nz (see below)
  double sing_cg;        // g^T 1' / sum(w)
  double sing_sc;        // the factor scale of the (0,0) column
  int M, ny, nz, nky;
  int nblk_x;            // blocks along kx per ky
  int neumann;
  int kx64, ky64;        // FP32 spectra: columns kx < kx64, |ky| < ky64 in FP64
};

constexpr int kThomasBlock = 64;
constexpr int kPrefetch = 3;

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
// and each thread keeps the next kPrefetch rows in flight while the recurrence
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
template <class CS, class CA, class F2, class F1>
__device__ __forceinline__ void sweep_column(const ThomasArgs& a, CS* const s0, const F2* const fx0,
                                             const F2* const fy0, const F1* const bx0,
                                             const F1* const by0, const bool sing) {
  using T = typename cplx_traits<CA>::T;
  const int nz = a.nz;
  const long long rs = (long long)a.ny * a.M;         // spectrum row stride
  const long long rt = (long long)a.nky * (a.M + 1);  // factor row stride

  // forward: g_k = (s/piv_k) f_k - (A_k/piv_k) g_{k-1}, in place
  CS qu[kPrefetch];
  F2 qx[kPrefetch], qy[kPrefetch];
#pragma unroll
  for (int i = 0; i < kPrefetch; ++i) {
    if (i < nz) {
      qu[i] = s0[i * rs];
      qx[i] = fx0[i * rt];
      qy[i] = fy0[i * rt];
    }
  }
  const CS* pu = s0 + kPrefetch * rs;  // next rows to prefetch
  const F2* px = fx0 + kPrefetch * rt;
  const F2* py = fy0 + kPrefetch * rt;
  CS* ps = s0;                         // row being written
  CA g = cplx_traits<CA>::mk(T(0), T(0));
  double mu = 0.0, gam = 0.0;
  for (int k = 0; k < nz; k += kPrefetch) {
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      if (k + i >= nz) break;
      CA u = cvt<CA>(qu[i]);
      const F2 fx = qx[i], fy = qy[i];
      if (k + i + kPrefetch < nz) {
        qu[i] = *pu;
        qx[i] = *px;
        qy[i] = *py;
      }
      pu += rs;
      px += rt;
      py += rt;
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
  CS qg[kPrefetch];
  F1 qbx[kPrefetch], qby[kPrefetch];
  CS* const s1 = s0 + (long long)(nz - 1) * rs;
  const F1* const bx1 = bx0 + (long long)(nz - 1) * rt;
  const F1* const by1 = by0 + (long long)(nz - 1) * rt;
#pragma unroll
  for (int i = 0; i < kPrefetch; ++i) {
    if (i < nz) {
      qg[i] = s1[-i * rs];
      qbx[i] = bx1[-i * rt];
      qby[i] = by1[-i * rt];
    }
  }
  const CS* pg = s1 - kPrefetch * rs;
  const F1* pbx = bx1 - kPrefetch * rt;
  const F1* pby = by1 - kPrefetch * rt;
  ps = s1;
  CA x = cplx_traits<CA>::mk(T(0), T(0));
  for (int r = 0; r < nz; r += kPrefetch) {
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
      if (r + i >= nz) break;
      const CA gg = cvt<CA>(qg[i]);
      const F1 bx = qbx[i], by = qby[i];
      if (r + i + kPrefetch < nz) {
        qg[i] = *pg;
        qbx[i] = *pbx;
        qby[i] = *pby;
      }
      pg -= rs;
      pbx -= rt;
      pby -= rt;
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
template <class CS>
__global__ void __launch_bounds__(kThomasBlock, 11) thomas_kernel(ThomasArgs a) {
  const int ky = blockIdx.x / a.nblk_x;
  const int j = (blockIdx.x % a.nblk_x) * kThomasBlock + threadIdx.x;
  if (j >= a.M) return;
  // factor sets of the real (x) and imaginary (y) parts
  int kx_x = j, kx_y = j, kp_x, kp_y;
  if (j > 0) {
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
  if (fp64)
    sweep_column<CS, double2>(a, s0, a.fwd + ox, a.fwd + oy, a.bwd + ox, a.bwd + oy, sing);
  else
    sweep_column<CS, float2>(a, s0, a.fwd32 + ox, a.fwd32 + oy, a.bwd32 + ox, a.bwd32 + oy, false);
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
  a.neumann = (P->bc == CFS_BC_NEUMANN);
  a.kx64 = P->kx64;
  a.ky64 = P->ky64;
  return a;
}

cudaError_t launch_thomas(const cfs_plan* P, double* data, cudaStream_t st) {
  ThomasArgs a = thomas_args(P, data);
  thomas_kernel<double2><<<a.nblk_x * P->ny, kThomasBlock, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_thomas32(const cfs_plan* P, float* data, cudaStream_t st) {
  if (!P->d_fwd32) return cudaErrorInvalidValue;
  ThomasArgs a = thomas_args(P, data);
  thomas_kernel<float2><<<a.nblk_x * P->ny, kThomasBlock, 0, st>>>(a);
  return cudaGetLastError();
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

cudaError_t launch_thomas_factor(cfs_plan* P, const double* dA, const double* dB, const double* dC,
                                 const double* dlamx, const double* dlamy, cudaStream_t st) {
  const double s = 2.0 / ((double)P->nx * (double)P->ny);
  dim3 grid((P->M + 1 + 127) / 128, P->nky);
  thomas_factor_kernel<<<grid, 128, 0, st>>>(P->d_fwd, P->d_bwd, P->d_fwd32, P->d_bwd32, dA, dB,
                                             dC, dlamx, dlamy, P->M, P->nky, P->nz, s,
                                             P->bc == CFS_BC_NEUMANN);
  return cudaGetLastError();
}

}  // namespace chanfs
