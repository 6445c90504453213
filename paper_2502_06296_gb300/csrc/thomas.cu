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
// One thread owns the column pair ky and Ny-ky of one kx (they share the
// eigenvalue, hence the factors); consecutive threads take consecutive kx so
// that every z-plane access is coalesced.  kx = 0 is the packed pair of App. A:
// it holds F(0, ky) + i F(Nx/2, ky), which the thread untangles with the
// Hermitian partner ky' = Ny - ky, solves with the two factor sets, and packs
// back.  The singular Neumann column (0, 0) is pinned (row 0 -> F_0 = 0) after
// removing the dz-weighted mean of its right-hand side, and the dz-weighted
// mean of its solution is removed afterwards.
#include "chanfs_internal.cuh"

namespace chanfs {

struct ThomasArgs {
  double2* S;            // spectrum (Nz, Ny, M) complex
  const double2* fwd;    // (s/piv, A/piv) per (k, kyp, kx in [0, M])
  const double* bwd;     // C/piv
  const double* dzf;     // weights of the Neumann mean
  int M, ny, nz, nky;
  int neumann;
};

__device__ __forceinline__ long long sidx(const ThomasArgs& a, int k, int ky, int j) {
  return ((long long)k * a.ny + ky) * a.M + j;
}
__device__ __forceinline__ long long tidx(const ThomasArgs& a, int k, int kyp, int kx) {
  return ((long long)k * a.nky + kyp) * (a.M + 1) + kx;
}

// The (kx, ky) = (0, 0) pair under Neumann walls: P = 2 Re S is the singular
// column, Q = 2 Im S is the regular column (Nx/2, 0).
__device__ void thomas_singular(const ThomasArgs& a) {
  double sw = 0.0, swp = 0.0;
  for (int k = 0; k < a.nz; ++k) {
    sw += a.dzf[k];
    swp += a.dzf[k] * (2.0 * a.S[sidx(a, k, 0, 0)].x);
  }
  const double mu = swp / sw;
  double gp = 0.0, gq = 0.0;
  for (int k = 0; k < a.nz; ++k) {
    double2 s = a.S[sidx(a, k, 0, 0)];
    double p = (k == 0) ? 0.0 : 2.0 * s.x - mu;
    double q = 2.0 * s.y;
    double2 fp = a.fwd[tidx(a, k, 0, 0)], fq = a.fwd[tidx(a, k, 0, a.M)];
    gp = fma(-fp.y, gp, fp.x * p);
    gq = fma(-fq.y, gq, fq.x * q);
    a.S[sidx(a, k, 0, 0)] = make_double2(gp, gq);
  }
  double xp = 0.0, xq = 0.0, swx = 0.0;
  for (int k = a.nz - 1; k >= 0; --k) {
    double2 g = a.S[sidx(a, k, 0, 0)];
    xp = fma(-a.bwd[tidx(a, k, 0, 0)], xp, g.x);
    xq = fma(-a.bwd[tidx(a, k, 0, a.M)], xq, g.y);
    swx += a.dzf[k] * xp;
    a.S[sidx(a, k, 0, 0)] = make_double2(xp, xq);
  }
  const double nu = swx / sw;
  for (int k = 0; k < a.nz; ++k) a.S[sidx(a, k, 0, 0)].x -= nu;
}

__global__ void __launch_bounds__(128) thomas_kernel(ThomasArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int kyp = blockIdx.y;
  if (j >= a.M) return;
  const int kyq = (a.ny - kyp) % a.ny;
  const bool self = (kyq == kyp);
  const bool j0 = (j == 0);
  if (a.neumann && j0 && kyp == 0) {
    thomas_singular(a);
    return;
  }
  const int kxq = j0 ? a.M : j;  // factor set of the second column
  double2 gp = make_double2(0.0, 0.0), gq = gp;
  // forward sweep: g overwrites the right-hand side in place
  for (int k = 0; k < a.nz; ++k) {
    double2 u = a.S[sidx(a, k, kyp, j)];
    double2 v = a.S[sidx(a, k, kyq, j)];
    double2 P, Q;
    if (j0) {  // untangle F(0,ky) (times 2) and F(M,ky) (times 2)
      P = make_double2(u.x + v.x, u.y - v.y);
      Q = make_double2(u.y + v.y, v.x - u.x);
    } else {
      P = u;
      Q = v;
    }
    const double2 fp = a.fwd[tidx(a, k, kyp, j)];
    const double2 fq = j0 ? a.fwd[tidx(a, k, kyp, kxq)] : fp;
    gp = make_double2(fma(-fp.y, gp.x, fp.x * P.x), fma(-fp.y, gp.y, fp.x * P.y));
    gq = make_double2(fma(-fq.y, gq.x, fq.x * Q.x), fma(-fq.y, gq.y, fq.x * Q.y));
    if (j0 && self) {
      a.S[sidx(a, k, kyp, 0)] = make_double2(gp.x, gq.x);  // both columns are real
    } else {
      a.S[sidx(a, k, kyp, j)] = gp;
      a.S[sidx(a, k, kyq, j)] = gq;
    }
  }
  // backward sweep
  double2 xp = make_double2(0.0, 0.0), xq = xp;
  for (int k = a.nz - 1; k >= 0; --k) {
    double2 g1, g2;
    if (j0 && self) {
      double2 s = a.S[sidx(a, k, kyp, 0)];
      g1 = make_double2(s.x, 0.0);
      g2 = make_double2(s.y, 0.0);
    } else {
      g1 = a.S[sidx(a, k, kyp, j)];
      g2 = a.S[sidx(a, k, kyq, j)];
    }
    const double bp = a.bwd[tidx(a, k, kyp, j)];
    const double bq = j0 ? a.bwd[tidx(a, k, kyp, kxq)] : bp;
    xp = make_double2(fma(-bp, xp.x, g1.x), fma(-bp, xp.y, g1.y));
    xq = make_double2(fma(-bq, xq.x, g2.x), fma(-bq, xq.y, g2.y));
    if (j0) {  // pack back: Z(ky) = P + i Q, Z(Ny-ky) = conj P + i conj Q
      a.S[sidx(a, k, kyp, 0)] = make_double2(xp.x - xq.y, xp.y + xq.x);
      if (!self) a.S[sidx(a, k, kyq, 0)] = make_double2(xp.x + xq.y, xq.x - xp.y);
    } else {
      a.S[sidx(a, k, kyp, j)] = xp;
      a.S[sidx(a, k, kyq, j)] = xq;
    }
  }
}

cudaError_t launch_thomas(const cfs_plan* P, double* data, cudaStream_t st) {
  ThomasArgs a;
  a.S = reinterpret_cast<double2*>(data);
  a.fwd = P->d_fwd;
  a.bwd = P->d_bwd;
  a.dzf = P->d_dzf;
  a.M = P->M;
  a.ny = P->ny;
  a.nz = P->nz;
  a.nky = P->nky;
  a.neumann = (P->bc == CFS_BC_NEUMANN);
  dim3 grid((P->M + 127) / 128, P->nky);
  thomas_kernel<<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Plan-time factorisation, one thread per (kx, kyp), FP64 with true division.
// The x-pair kx = 0 and kx = M (untangled from the packed column, which
// doubles them) take s/2.  The Neumann (0, 0) system is pinned: row 0 becomes
// F_0 = 0 (B_0 -> 1, C_0 -> 0).
// ----------------------------------------------------------------------------
__global__ void thomas_factor_kernel(double2* fwd, double* bwd, const double* A, const double* B,
                                     const double* C, const double* lamx, const double* lamy,
                                     int M, int nky, int nz, double s, int neumann) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int kyp = blockIdx.y;
  if (kx > M) return;
  const double lam = lamx[kx] + lamy[kyp];
  const double sc = (kx == 0 || kx == M) ? 0.5 * s : s;
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
    fwd[t] = make_double2(sc / piv, (k == 0 ? 0.0 : A[k]) / piv);
    bwd[t] = c / piv;
    cprev = c;
  }
}

cudaError_t launch_thomas_factor(cfs_plan* P, const double* dA, const double* dB, const double* dC,
                                 const double* dlamx, const double* dlamy, cudaStream_t st) {
  const double s = 2.0 / ((double)P->nx * (double)P->ny);
  dim3 grid((P->M + 1 + 127) / 128, P->nky);
  thomas_factor_kernel<<<grid, 128, 0, st>>>(P->d_fwd, P->d_bwd, dA, dB, dC, dlamx, dlamy, P->M,
                                             P->nky, P->nz, s, P->bc == CFS_BC_NEUMANN);
  return cudaGetLastError();
}

}  // namespace chanfs
