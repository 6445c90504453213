// helm_thomas.cu -- the z-implicit Helmholtz systems (I - c L_z) u = rhs of
// Eq. 11 by a plain Thomas sweep per (x, y) column, the alternative to the
// paper's Algorithm 2 that the tuner may pick per size.
//
// Every column has the same coefficients, so the LU factors are computed
// once per (c, loc) on the host (beside Algorithm 2's Step 1):
//   fs_k = 1/piv_k, fa_k = A'_k/piv_k, fc_k = C'_k/piv_k,
//   piv_0 = B'_0, piv_k = B'_k - A'_k fc_{k-1},
// and a sweep is g_k = fs_k d_k - fa_k g_{k-1} up the column (g written to
// u), then u_k = g_k - fc_k u_{k+1} back down: 3 instructions per unknown
// against Algorithm 2's 5, for twice the field traffic (g goes through
// memory).  One thread per column, consecutive threads on consecutive x, so
// every z-row access of a warp is one contiguous run; each thread keeps the
// next PF rows of its column in flight (the sweep is sequential in z), and
// the factors sit in shared memory.  rhs == u is allowed: the forward sweep
// reads row k + PF before it writes row k.
#include "chanfs_group.cuh"

namespace chanfs {

constexpr int kHThBlock = 128;  // columns per block

template <class R> struct hth_prefetch { static constexpr int value = 8; };
template <> struct hth_prefetch<float> { static constexpr int value = 16; };

template <class R>
__device__ __forceinline__ void helm_thomas_body(const R* rhs, R* u, const R* __restrict__ fac,
                                                 long long ncols, int n, int nz, int face,
                                                 long long blk) {
  extern __shared__ __align__(16) unsigned char hth_smem[];
  R* sf = reinterpret_cast<R*>(hth_smem);  // fs | fa | fc
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) sf[i] = fac[i];
  __syncthreads();
  const long long col = blk * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  constexpr int PF = hth_prefetch<R>::value;
  const R* fs = sf;
  const R* fa = sf + n;
  const R* fc = sf + 2 * n;

  // forward: g_k = fs_k d_k - fa_k g_{k-1}
  R qd[PF];
#pragma unroll
  for (int i = 0; i < PF; ++i)
    if (i < n) qd[i] = rhs[(long long)i * ncols + col];
  R g = R(0);
  for (int k = 0; k < n; k += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      const int r = k + i;
      if (r >= n) break;
      const R d = qd[i];
      if (r + PF < n) qd[i] = rhs[(long long)(r + PF) * ncols + col];
      g = fma(-fa[r], g, fs[r] * d);
      u[(long long)r * ncols + col] = g;
    }
  }
  // backward: u_{n-1} = g_{n-1}, u_k = g_k - fc_k u_{k+1}
  R qg[PF];
#pragma unroll
  for (int i = 0; i < PF; ++i)
    if (i < n) qg[i] = u[(long long)(n - 1 - i) * ncols + col];
  R x = R(0);
  for (int k = 0; k < n; k += PF) {
#pragma unroll
    for (int i = 0; i < PF; ++i) {
      const int r = n - 1 - (k + i);
      if (r < 0) break;
      const R gg = qg[i];
      if (r - PF >= 0) qg[i] = u[(long long)(r - PF) * ncols + col];
      x = fma(-fc[r], x, gg);
      u[(long long)r * ncols + col] = x;
    }
  }
  if (face) u[(long long)(nz - 1) * ncols + col] = R(0);  // the wall slot
}

template <class R>
__global__ void __launch_bounds__(kHThBlock) helm_thomas_kernel(const R* rhs, R* u,
                                                                const R* __restrict__ fac,
                                                                long long ncols, int n, int nz,
                                                                int face) {
  helm_thomas_body<R>(rhs, u, fac, ncols, n, nz, face, blockIdx.x);
}

template <class R>
__global__ void __launch_bounds__(kHThBlock) helm_thomas_group_kernel(const HThomasBox* boxes,
                                                                      GroupMap g,
                                                                      const GroupIo* io) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const HThomasBox& x = boxes[b];
  // per-call fields (FP64 boxes) come from the call's table; FP32 inner
  // solves work in place on the plan's residual field
  const R* rhs = x.per_call ? reinterpret_cast<const R*>(io[b].f) : static_cast<const R*>(x.rhs);
  R* u = x.per_call ? reinterpret_cast<R*>(io[b].p) : static_cast<R*>(x.u);
  helm_thomas_body<R>(rhs, u, static_cast<const R*>(x.fac), x.ncols, x.n, x.nz, x.face, blk);
}

template <class R>
static cudaError_t launch_t(const cfs_plan* P, const HelmCoef& h, const R* fac, const R* rhs,
                            R* u, cudaStream_t st) {
  const long long ncols = (long long)P->nx * P->ny;
  const unsigned grid = (unsigned)((ncols + kHThBlock - 1) / kHThBlock);
  const size_t smem = 3 * sizeof(R) * (size_t)h.n;
  auto k = helm_thomas_kernel<R>;
  allow_max_smem(k);
  k<<<grid, kHThBlock, smem, st>>>(rhs, u, fac, ncols, h.n, P->nz, h.loc == CFS_LOC_FACE);
  return cudaGetLastError();
}

cudaError_t launch_helm_thomas(const cfs_plan* P, const HelmCoef& h, const double* rhs,
                               double* u, cudaStream_t st) {
  return launch_t<double>(P, h, h.d_th, rhs, u, st);
}

cudaError_t launch_helm_thomas32(const cfs_plan* P, const HelmCoef& h, const float* rhs,
                                 float* u, cudaStream_t st) {
  if (!h.d_th32) return cudaErrorInvalidValue;  // FP64 plans hold no FP32 factors
  return launch_t<float>(P, h, h.d_th32, rhs, u, st);
}

size_t helm_thomas_group_box(const cfs_plan* P, const HelmCoef& h, bool fp32, HThomasBox* box,
                             int* blocks) {
  box->ncols = (long long)P->nx * P->ny;
  box->n = h.n;
  box->nz = P->nz;
  box->face = h.loc == CFS_LOC_FACE;
  box->per_call = !fp32;
  box->rhs = fp32 ? static_cast<const void*>(P->d_r32) : nullptr;
  box->u = fp32 ? static_cast<void*>(P->d_r32) : nullptr;
  box->fac = fp32 ? static_cast<const void*>(h.d_th32) : static_cast<const void*>(h.d_th);
  *blocks = (int)((box->ncols + kHThBlock - 1) / kHThBlock);
  return 3 * (fp32 ? sizeof(float) : sizeof(double)) * (size_t)h.n;
}

cudaError_t launch_helm_thomas_group(const HThomasBox* boxes, GroupMap g, int total, size_t smem,
                                     bool fp32, const GroupIo* io, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  if (fp32) {
    auto k = helm_thomas_group_kernel<float>;
    allow_max_smem(k);
    k<<<total, kHThBlock, smem, st>>>(boxes, g, io);
  } else {
    auto k = helm_thomas_group_kernel<double>;
    allow_max_smem(k);
    k<<<total, kHThBlock, smem, st>>>(boxes, g, io);
  }
  return cudaGetLastError();
}

}  // namespace chanfs
