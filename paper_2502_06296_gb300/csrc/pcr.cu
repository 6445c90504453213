// pcr.cu -- z-implicit Helmholtz solve (I - c L_z) u = rhs (Eq. 11) by the
// reworked parallel cyclic reduction of Algorithm 2, Steps 2-4.
//
// Mapping: a CTA has one warp per z-partition and 32 lanes = 32 consecutive
// (x, y) columns, so every row access of a warp is one contiguous 256-byte
// run.  Each thread keeps its partition's m <= MMAX rows in registers:
//   Step 2: forward  d_i -= alpha_i d_{i-1}   (i = 2..m-1),
//           backward d_i -= beta_i  d_{i+1}   (i = m-3..0),
//   Step 3: the 2*nparts boundary unknowns of each column go to shared
//           memory; warp 0 solves every column's reduced tridiagonal system
//           (one lane per column) with the LU factors prepared on the host,
//   Step 4: d_i = ib_i d_i - ap_i x_0 - cp_i x_{m-1}.
// Only the right-hand side changes at run time (the point of Algorithm 2):
// 5 FP64 instructions per unknown, no division.  The coefficients, identical
// for every column, are staged once per CTA in shared memory and read as
// warp-uniform broadcasts.  CTAs loop over column tiles.
#include "chanfs_internal.cuh"

namespace chanfs {

struct PcrArgs {
  const double* rhs;
  double* u;
  long long ncols;  // Nx * Ny
  int n;            // unknowns per column
  int nparts;
  int face;         // face-located field: slot nz-1 is the wall, written 0
  int nz;
  const double* rows;  // alpha | beta | ib | ap | cp  (5n)
  const double* red;   // rl | rip | ripc            (3 * 2 nparts)
  int start[kPcrMaxParts + 1];
};

// MMAX = 16: up to 32 warps at <= 64 registers; MMAX = 32: up to 12 warps.
template <int MMAX>
__global__ void __launch_bounds__(MMAX == 16 ? 1024 : 384) pcr_kernel(PcrArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int n = a.n, J = 2 * a.nparts;
  double* s_rows = sm;             // 5n
  double* s_red = s_rows + 5 * n;  // 3J
  double* s_x = s_red + 3 * J;     // J x 32 boundary values
  for (int e = threadIdx.x; e < 5 * n; e += blockDim.x) s_rows[e] = a.rows[e];
  for (int e = threadIdx.x; e < 3 * J; e += blockDim.x) s_red[e] = a.red[e];
  __syncthreads();
  const double* alpha = s_rows;
  const double* beta = s_rows + n;
  const double* ib = s_rows + 2 * n;
  const double* ap = s_rows + 3 * n;
  const double* cp = s_rows + 4 * n;
  const double* rl = s_red;
  const double* rip = s_red + J;
  const double* ripc = s_red + 2 * J;

  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int s = a.start[q], m = a.start[q + 1] - s;
  const long long ntiles = (a.ncols + 31) / 32;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long col = tile * 32 + lane;
    const bool live = col < a.ncols;
    double v[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      v[i] = (live && i < m) ? a.rhs[(long long)(s + i) * a.ncols + col] : 0.0;
    // Step 2, forward then backward reduction of d only
#pragma unroll
    for (int i = 2; i < MMAX; ++i)
      if (i < m) v[i] = fma(-alpha[s + i], v[i - 1], v[i]);
#pragma unroll
    for (int i = MMAX - 3; i >= 0; --i)
      if (i <= m - 3) v[i] = fma(-beta[s + i], v[i + 1], v[i]);
    // v[m-1] without a run-time index (which would demote v to local memory)
    unsigned long long lastbits = 0ull;
#pragma unroll
    for (int i = 2; i < MMAX; ++i)
      lastbits |= (unsigned long long)__double_as_longlong(v[i]) &
                  (0ull - (unsigned long long)(i == m - 1));
    const double vlast = __longlong_as_double((long long)lastbits);
    s_x[(2 * q) * 32 + lane] = v[0];
    s_x[(2 * q + 1) * 32 + lane] = vlast;
    __syncthreads();
    // Step 3, reduced system [x_0^0, x_{m-1}^0, x_0^1, ...] per column
    if (q == 0) {
      double y = s_x[lane];
      for (int jj = 1; jj < J; ++jj) {
        y = fma(-rl[jj], y, s_x[jj * 32 + lane]);
        s_x[jj * 32 + lane] = y;
      }
      double x = rip[J - 1] * y;
      s_x[(J - 1) * 32 + lane] = x;
      for (int jj = J - 2; jj >= 0; --jj) {
        x = fma(-ripc[jj], x, rip[jj] * s_x[jj * 32 + lane]);
        s_x[jj * 32 + lane] = x;
      }
    }
    __syncthreads();
    // Step 4, reconstruction
    const double x0 = s_x[(2 * q) * 32 + lane];
    const double xm = s_x[(2 * q + 1) * 32 + lane];
    if (live) {
      double* out = a.u + col;
#pragma unroll
      for (int i = 0; i < MMAX; ++i) {
        if (i < m) {
          double r;
          if (i == 0) r = x0;
          else if (i == m - 1) r = xm;
          else r = fma(-cp[s + i], xm, fma(-ap[s + i], x0, ib[s + i] * v[i]));
          out[(long long)(s + i) * a.ncols] = r;
        }
      }
      if (a.face && q == a.nparts - 1) out[(long long)(a.nz - 1) * a.ncols] = 0.0;
    }
    __syncthreads();  // s_x is reused by the next tile
  }
}

template <int MMAX>
static cudaError_t launch_pcr_t(const PcrArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)(5 * a.n + 3 * 2 * a.nparts + 2 * a.nparts * 32);
  cudaFuncSetAttribute(pcr_kernel<MMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcr_kernel<MMAX>, 32 * a.nparts, smem);
  if (per_sm < 1) per_sm = 1;
  const long long ntiles = (a.ncols + 31) / 32;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  pcr_kernel<MMAX><<<(unsigned)grid, 32 * a.nparts, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pcr(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       cudaStream_t st) {
  PcrArgs a;
  a.rhs = rhs;
  a.u = u;
  a.ncols = (long long)P->nx * P->ny;
  a.n = h.n;
  a.nparts = h.nparts;
  a.face = (h.loc == CFS_LOC_FACE);
  a.nz = P->nz;
  a.rows = h.d_rows;
  a.red = h.d_red;
  for (int i = 0; i <= kPcrMaxParts; ++i) a.start[i] = (i <= h.nparts) ? h.start[i] : h.n;
  if (h.mmax <= 16) return launch_pcr_t<16>(a, st);
  return launch_pcr_t<32>(a, st);
}

}  // namespace chanfs
