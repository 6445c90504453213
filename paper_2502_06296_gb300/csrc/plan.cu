// plan.cu -- the C ABI of libchanfs: plans, tables, pre-processing and the
// orchestration of the Poisson and Helmholtz solves on the caller's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "chanfs_alg2.cuh"
#include "chanfs_internal.cuh"

using namespace chanfs;

// ----------------------------------------------------------------------------
// FFT radix plans and twiddles
// ----------------------------------------------------------------------------
namespace chanfs {

static const double kTwoPi = 6.283185307179586476925286766559;

// exp(-2 pi i e / n) with exact reduction of e modulo n.
static double2 root(long long e, long long n) {
  long long r = e % n;
  if (r < 0) r += n;
  double a = kTwoPi * (double)r / (double)n;
  return make_double2(cos(a), -sin(a));
}

bool make_fft_desc(int n, FftDesc* d, std::vector<double2>* tw, int max_radix) {
  memset(d, 0, sizeof(*d));
  d->n = n;
  int rest = n;
  std::vector<int> rad;
  if (max_radix >= 8)
    while (rest % 8 == 0) { rad.push_back(8); rest /= 8; }
  while (rest % 4 == 0) { rad.push_back(4); rest /= 4; }
  if (rest % 2 == 0) { rad.push_back(2); rest /= 2; }
  while (rest % 3 == 0) { rad.push_back(3); rest /= 3; }
  if (rest != 1 || (int)rad.size() > kMaxPasses) return false;
  tw->clear();
  int L = 1;
  d->npass = (int)rad.size();
  for (int p = 0; p < d->npass; ++p) {
    const int R = rad[p];
    d->radix[p] = R;
    d->span[p] = L;
    d->twoff[p] = (int)tw->size();
    for (int k = 0; k < L; ++k)
      for (int r = 1; r < R; ++r) tw->push_back(root((long long)r * k, (long long)L * R));
    L *= R;
  }
  d->ntw = (int)tw->size();
  if (tw->empty()) tw->push_back(make_double2(1.0, 0.0));  // keep a valid pointer
  return true;
}

}  // namespace chanfs

// ----------------------------------------------------------------------------
// Helpers
// ----------------------------------------------------------------------------
static bool is_23_smooth(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

template <typename T>
static int dev_upload(T** dst, const T* src, size_t count, size_t* acc) {
  if (cudaMalloc(dst, sizeof(T) * count) != cudaSuccess) return CFS_ENOMEM;
  *acc += sizeof(T) * count;
  if (src && cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return CFS_ECUDA;
  return CFS_OK;
}

// Guard words around the work buffers that kernels write (factor tables, the
// refinement's FP32 fields and reduction scratch): kGuardBytes of a fixed
// pattern before and after each, compared by cfs_plan_check_guards, so that a
// kernel storing past either end of its buffer is noticed at the next check.
// (A stand-in for a device memory checker in runs that cannot use one.)
constexpr size_t kGuardBytes = 256;   // keeps the buffer 256-byte aligned
constexpr uint32_t kGuardWord = 0x6A09E667u;

template <typename T>
static int dev_alloc_guarded(cfs_plan* P, T** dst, size_t count) {
  const size_t bytes = sizeof(T) * count;
  unsigned char* base = nullptr;
  if (cudaMalloc(&base, bytes + 2 * kGuardBytes) != cudaSuccess) return CFS_ENOMEM;
  P->guarded.push_back({base, bytes});
  P->device_bytes += bytes + 2 * kGuardBytes;
  const std::vector<uint32_t> pat(kGuardBytes / sizeof(uint32_t), kGuardWord);
  if (cudaMemcpy(base, pat.data(), kGuardBytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + kGuardBytes + bytes, pat.data(), kGuardBytes, cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return CFS_ECUDA;
  *dst = reinterpret_cast<T*>(base + kGuardBytes);
  return CFS_OK;
}

// z stencil of the staggered grid (Sec. 2.1, eta of Eq. 12), flux form:
//   (L_z p)_k = [(p_{k+1}-p_k)/dzc_k - (p_k-p_{k-1})/dzc_{k-1}] / dzf_k,
// centred unknowns with mirror ghosts at the walls (Neumann: p_{-1} = p_0;
// Dirichlet: u_{-1} = -u_0, ghost one cell width away), or, for face-located
// unknowns, the Nz-1 interior faces with w = 0 on both walls.
static int z_stencil(const std::vector<double>& dzf, int bc, int loc, std::vector<double>& A,
                     std::vector<double>& B, std::vector<double>& C) {
  const int nz = (int)dzf.size();
  const int n = (loc == CFS_LOC_CENTER) ? nz : nz - 1;
  A.assign(n, 0.0);
  B.assign(n, 0.0);
  C.assign(n, 0.0);
  for (int k = 0; k < n; ++k) z_operator_row(k, nz, dzf.data(), bc, loc, &A[k], &B[k], &C[k]);
  return n;
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? CFS_OK : CFS_ECUDA; }

// Thomas algorithm on the host (FP64): a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k.
static void thomas_host(const std::vector<double>& a, const std::vector<double>& b,
                        const std::vector<double>& c, const std::vector<double>& d,
                        std::vector<double>& x) {
  const int n = (int)b.size();
  std::vector<double> cp(n), dp(n);
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int k = 1; k < n; ++k) {
    const double piv = b[k] - a[k] * cp[k - 1];
    cp[k] = c[k] / piv;
    dp[k] = (d[k] - a[k] * dp[k - 1]) / piv;
  }
  x[n - 1] = dp[n - 1];
  for (int k = n - 2; k >= 0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
}

// ----------------------------------------------------------------------------
// Public ABI
// ----------------------------------------------------------------------------
std::recursive_mutex& chanfs::capture_mutex() {
  static std::recursive_mutex mu;
  return mu;
}

extern "C" int cfs_version(void) { return CHANFS_VERSION; }

extern "C" const char* cfs_status_string(int s) {
  switch (s) {
    case CFS_OK: return "ok";
    case CFS_EINVAL: return "invalid argument";
    case CFS_ENOMEM: return "out of memory";
    case CFS_EUNSUPPORTED: return "unsupported size or option";
    case CFS_ECUDA: return "CUDA runtime error";
    case CFS_ETIMEOUT: return "device-side wait timed out";
    case CFS_ENOTCONVERGED: return "not converged";
    case CFS_ECANCELED: return "cancelled";
    case CFS_EGUARD: return "guard words around a work buffer were overwritten";
    default: return "unknown status";
  }
}

static void plan_free(cfs_plan* P) {
  if (!P) return;
  for (const auto& g : P->guarded) cudaFree(g.first);  // guarded work buffers
  cudaFree(P->d_twx);
  cudaFree(P->d_twy);
  cudaFree(P->d_post);
  cudaFree(P->d_dzf);
  cudaFree(P->d_sing);
  cudaFree(P->d_stage);
  cudaFree(P->d_batch);
  for (cudaStream_t q : {P->copy_in, P->copy_out, P->copy_out2, P->compute2})
    if (q) cudaStreamDestroy(q);
  if (P->ev_entry) cudaEventDestroy(P->ev_entry);
  for (int k = 0; k < kBatchSlots; ++k) {
    for (cudaEvent_t e : {P->ev_done[k], P->ev_free[k]})
      if (e) cudaEventDestroy(e);
    for (int c = 0; c < kMaxStreamChunks; ++c)
      for (cudaEvent_t e : {P->ev_cin[k][c], P->ev_cdone[k][c]})
        if (e) cudaEventDestroy(e);
  }
  cudaFree(P->d_status);
  cudaFree(P->d_twx32);
  cudaFree(P->d_twy32);
  cudaFree(P->d_post32);
  cudaFree(P->d_zrow32);
  cudaFree(P->d_lam32);
  cudaFree(P->d_zk);
  cudaFree(P->d_wy);
  cudaFree(P->d_wy32);

  for (auto& h : P->helm) {
    cudaFree(h.d_rows);
    cudaFree(h.d_red);
    cudaFree(h.d_rows32);
    cudaFree(h.d_red32);
    cudaFree(h.d_abc);
  }
  for (auto& h : P->helm3) {
    cudaFree(h.d_fwd);
    cudaFree(h.d_bwd);
  }
  delete P;
}

extern "C" int cfs_plan_create(cfs_plan_t* out, int nx, int ny, int nz, double lx, double ly,
                               const double* dz, int poisson_bc, int dtype) {
  return cfs_plan_create_walls(out, nx, ny, nz, lx, ly, dz, poisson_bc, CFS_Y_PERIODIC, dtype);
}

extern "C" int cfs_plan_create_walls(cfs_plan_t* out, int nx, int ny, int nz, double lx,
                                     double ly, const double* dz, int poisson_bc, int ybc,
                                     int dtype) {
  CaptureLock lock(capture_mutex());
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (!dz || !(lx > 0) || !(ly > 0) || !isfinite(lx) || !isfinite(ly)) return CFS_EINVAL;
  if (poisson_bc != CFS_BC_NEUMANN && poisson_bc != CFS_BC_DIRICHLET) return CFS_EINVAL;
  if (ybc != CFS_Y_PERIODIC && ybc != CFS_Y_NEUMANN && ybc != CFS_Y_DIRICHLET) return CFS_EINVAL;
  if (dtype != CFS_F64 && dtype != CFS_F32_REFINED) return CFS_EUNSUPPORTED;
  // FP32 rows must be whole 16-byte units for the TMA copies
  if (dtype == CFS_F32_REFINED && nx % 4 != 0) return CFS_EUNSUPPORTED;
  if (nx < 2 || ny < 1 || nz < 3) return CFS_EINVAL;
  if (nx % 2 != 0 || nx > kMaxNx || !is_23_smooth(nx / 2)) return CFS_EUNSUPPORTED;
  if (ny > kMaxNy || !is_23_smooth(ny) || nz > kMaxNz) return CFS_EUNSUPPORTED;
  for (int k = 0; k < nz; ++k)
    if (!(dz[k] > 0) || !isfinite(dz[k])) return CFS_EINVAL;

  cfs_plan* P = new (std::nothrow) cfs_plan();
  if (!P) return CFS_ENOMEM;
  cudaGetDevice(&P->device);
  P->nx = nx;
  P->ny = ny;
  P->nz = nz;
  P->M = nx / 2;
  P->nky = (ybc == CFS_Y_PERIODIC) ? ny / 2 + 1 : ny;
  P->lx = lx;
  P->ly = ly;
  P->bc = poisson_bc;
  P->ybc = ybc;
  P->has_null = (poisson_bc == CFS_BC_NEUMANN && ybc != CFS_Y_DIRICHLET);
  P->dzf.assign(dz, dz + nz);
  P->helm_clock = 0;
  P->device_bytes = 0;
  P->dtype = dtype;
  P->tol = 1e-10;
  P->maxit = 4;
  P->last_iters = 0;
  P->last_rho = 0.0;
  const bool refined = (dtype == CFS_F32_REFINED);

  // y tile: columns per tile and TMA boxes (at most 256 rows per box)
  P->nbox = (ny + 255) / 256;
  if (ny % P->nbox != 0) {
    plan_free(P);
    return CFS_EUNSUPPORTED;
  }
  P->by = ny / P->nbox;
  // 8 columns per tile when the tile is small (or when 4 would leave a box
  // start off the 128-byte boundary TMA wants in shared memory), else 4
  P->tk = (ny <= 256 || P->by % 2 != 0) ? 8 : 4;
  if (P->tk > P->M) P->tk = P->M;
  if (P->nbox > 1 && ((size_t)P->by * P->tk * sizeof(double2)) % 128 != 0) {
    plan_free(P);
    return CFS_EUNSUPPORTED;
  }
  // FP32 tiles: twice the columns in the same bytes; an even count keeps the
  // 16-byte TMA box rows
  P->tk32 = (P->by % 2 != 0) ? 16 : 2 * P->tk;
  if (P->tk32 > P->M) P->tk32 = P->M + (P->M & 1);
  if (refined && P->nbox > 1 && ((size_t)P->by * P->tk32 * sizeof(float2)) % 128 != 0) {
    plan_free(P);
    return CFS_EUNSUPPORTED;
  }
  P->tk_auto = P->tk;
  P->tk32_auto = P->tk32;

  std::vector<double2> twx, twy;
  P->fft_radix = 8;
  P->emu_x = kEmuDefaultX;
  P->emu_y = kEmuDefaultY;
  if (!make_fft_desc(P->M, &P->fx, &twx, 8) || !make_fft_desc(ny, &P->fy, &twy, 8)) {
    plan_free(P);
    return CFS_EUNSUPPORTED;
  }
  // real-FFT untangling factors 0.5 * W_nx^k, k = 0..M/2
  std::vector<double2> post(P->M / 2 + 1);
  for (int k = 0; k <= P->M / 2; ++k) {
    double2 w = chanfs::root(k, nx);
    post[k] = make_double2(0.5 * w.x, 0.5 * w.y);
  }
  // modified wavenumbers of Eq. 12 for kx = 0..M and ky = 0..ny/2
  const double dx = lx / nx, dy = ly / ny;
  std::vector<double> lamx(P->M + 1), lamy(P->nky);
  for (int k = 0; k <= P->M; ++k) lamx[k] = 2.0 * (cos(kTwoPi * k / nx) - 1.0) / (dx * dx);
  for (int k = 0; k < P->nky; ++k) {
    // periodic: pairs +-ky; walls: cos(pi k (j+1/2)/Ny) (Neumann) or
    // sin(pi (k+1)(j+1/2)/Ny) (Dirichlet) eigenvectors of the mirrored stencil
    const double angle = (ybc == CFS_Y_PERIODIC) ? kTwoPi * k / ny
                         : (ybc == CFS_Y_NEUMANN) ? 0.5 * kTwoPi * k / ny
                                                  : 0.5 * kTwoPi * (k + 1) / ny;
    lamy[k] = 2.0 * (cos(angle) - 1.0) / (dy * dy);
  }
  // wall transforms: w_k = exp(-i pi k / 2Ny)
  std::vector<double2> wy;
  if (ybc != CFS_Y_PERIODIC)
    for (int k = 0; k < ny; ++k) wy.push_back(chanfs::root(k, 4 * ny));
  P->lamx_h = lamx;
  P->lamy_h = lamy;
  std::vector<double> A, B, C;
  z_stencil(P->dzf, poisson_bc, CFS_LOC_CENTER, A, B, C);

  // Neumann (0,0) column, pinned operator T' (row 0 -> identity):
  // h = T'^{-1} (0,1,..,1) and g = T'^{-T} w by Thomas in FP64
  std::vector<double> sing(3 * (size_t)nz, 0.0);
  P->sing_sc = 2.0 / ((double)nx * (double)ny);  // the factor scale s
  P->sing_cg = 0.0;
  if (P->has_null) {
    std::vector<double> a(A), b(B), c(C), rhs(nz, 1.0), h(nz), g(nz);
    b[0] = 1.0;
    c[0] = 0.0;
    rhs[0] = 0.0;
    thomas_host(a, b, c, rhs, h);
    // transpose: sub-diagonal c_{k-1}, super-diagonal a_{k+1}
    std::vector<double> at(nz, 0.0), ct(nz, 0.0);
    for (int k = 1; k < nz; ++k) at[k] = c[k - 1];
    for (int k = 0; k + 1 < nz; ++k) ct[k] = a[k + 1];
    thomas_host(at, b, ct, P->dzf, g);
    double sw = 0.0;
    for (int k = 0; k < nz; ++k) sw += P->dzf[k];
    for (int k = 0; k < nz; ++k) {
      sing[k] = P->dzf[k] / sw;
      sing[nz + k] = g[k] / sw;
      sing[2 * nz + k] = P->sing_sc * h[k];
    }
    for (int k = 1; k < nz; ++k) P->sing_cg += g[k];
    P->sing_cg /= sw;
  }

  // Refinement: the Poisson operator's z rows with the x/y diagonal folded in
  // (residual kernel), and the columns kept in FP64 by the FP32 z sweep: those
  // whose eigenvalue shift |lx + ly| is below 1e-3 of the largest z
  // eigenvalue, where an FP32 sweep would lose more than ~4 digits.
  std::vector<double> zop(3 * (size_t)nz);
  for (int k = 0; k < nz; ++k) {
    zop[k] = A[k];
    zop[nz + k] = B[k] - 2.0 / (dx * dx) - 2.0 / (dy * dy);
    zop[2 * nz + k] = C[k];
  }
  P->kx64 = P->ky64 = 0;
  if (refined) {
    double zmax = 0.0;
    for (int k = 0; k < nz; ++k) zmax = std::max(zmax, fabs(A[k]) + fabs(B[k]) + fabs(C[k]));
    const double thr = 1e-3 * zmax;
    while (P->kx64 <= P->M && fabs(lamx[P->kx64]) < thr) ++P->kx64;
    while (P->ky64 < P->nky && fabs(lamy[P->ky64]) < thr) ++P->ky64;
    P->kx64 = std::max(P->kx64, 1);
    P->ky64 = std::max(P->ky64, 1);
  }

  int rc = CFS_OK;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr, *dlx = nullptr, *dly = nullptr;
  size_t scratch = 0;
  const size_t nfac = (size_t)(P->M + 1) * P->nky * nz;
  if (!rc) rc = dev_upload(&P->d_twx, twx.data(), twx.size(), &P->device_bytes);
  if (!rc) rc = dev_upload(&P->d_twy, twy.data(), twy.size(), &P->device_bytes);
  if (!rc) rc = dev_upload(&P->d_post, post.data(), post.size(), &P->device_bytes);
  if (!rc) rc = dev_upload(&P->d_dzf, P->dzf.data(), (size_t)nz, &P->device_bytes);
  if (!rc) rc = dev_upload(&P->d_sing, sing.data(), sing.size(), &P->device_bytes);
  if (!rc && !wy.empty()) rc = dev_upload(&P->d_wy, wy.data(), wy.size(), &P->device_bytes);
  if (!rc) rc = dev_alloc_guarded(P, &P->d_fwd, nfac);
  if (!rc) rc = dev_alloc_guarded(P, &P->d_bwd, nfac);
  if (!rc) rc = dev_upload<int>(&P->d_status, nullptr, 1, &P->device_bytes);
  if (!rc) rc = cuda_status(cudaMemset(P->d_status, 0, sizeof(int)));
  if (!rc && refined) {
    auto f32 = [](const std::vector<double2>& v) {
      std::vector<float2> o(v.size());
      for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
      return o;
    };
    const std::vector<float2> twx32 = f32(twx), twy32 = f32(twy), post32 = f32(post);
    rc = dev_upload(&P->d_twx32, twx32.data(), twx32.size(), &P->device_bytes);
    if (!rc) rc = dev_upload(&P->d_twy32, twy32.data(), twy32.size(), &P->device_bytes);
    if (!rc) rc = dev_upload(&P->d_post32, post32.data(), post32.size(), &P->device_bytes);
    if (!rc && !wy.empty()) {
      const std::vector<float2> wy32 = f32(wy);
      rc = dev_upload(&P->d_wy32, wy32.data(), wy32.size(), &P->device_bytes);
    }
    if (!rc) rc = dev_alloc_guarded(P, &P->d_fwd32, nfac);
    if (!rc) rc = dev_alloc_guarded(P, &P->d_bwd32, nfac);
    {  // the partitioned FP32 z solve forms its rows from these, divided by
       // the inverse-FFT normalisation s (its solution then comes out scaled)
      const double is = ((double)nx * (double)ny) / 2.0;
      std::vector<float4> zrow(nz + kZPartRowPad, make_float4(0.0f, 1.0f, 0.0f, 0.0f));
      for (int k = 0; k < nz; ++k)
        zrow[k] = make_float4(k > 0 ? (float)(A[k] * is) : 0.0f, (float)(B[k] * is),
                              k + 1 < nz ? (float)(C[k] * is) : 0.0f, 1.0f);
      std::vector<float> lam;
      for (double v : lamx) lam.push_back((float)(v * is));
      for (double v : lamy) lam.push_back((float)(v * is));
      if (!rc) rc = dev_upload(&P->d_zrow32, zrow.data(), zrow.size(), &P->device_bytes);
      if (!rc) rc = dev_upload(&P->d_lam32, lam.data(), lam.size(), &P->device_bytes);
    }
    if (!rc) rc = dev_alloc_guarded(P, &P->d_r32, (size_t)nx * ny * nz);
    if (!rc)
      rc = dev_alloc_guarded(P, &P->d_red, (size_t)nz * start_chunks(nz) + 8);
    // The residual kernels' coefficients, each split as hi = fl32(v),
    // lo = fl32(v - hi), packed per plane (three float4: (A, C), (B', dz),
    // (D, dz)) and then (1/dx^2, 1/dy^2).  D_k = A_k + B'_k + C_k + 2/dx^2 +
    // 2/dy^2 is the centre weight left when the stencil is written in
    // differences (first residual); it is summed exactly (a TwoSum cascade:
    // in the interior it is the FP64 rounding residue of zero).
    auto split = [](double v, float* h, float* l) {
      *h = (float)v;
      *l = (float)(v - (double)*h);
    };
    std::vector<float4> zk(3 * (size_t)nz + 1);
    double wsum = 0.0;
    for (int k = 0; k < nz; ++k) {
      const double terms[5] = {zop[k], zop[nz + k], zop[2 * nz + k], 2.0 / (dx * dx),
                               2.0 / (dy * dy)};
      double sum = 0.0, err = 0.0;
      for (double v : terms) {
        const double t = sum + v, bb = t - sum;
        err += (sum - (t - bb)) + (v - bb);
        sum = t;
      }
      float4& ac = zk[3 * (size_t)k];
      float4& bw = zk[3 * (size_t)k + 1];
      float4& dw = zk[3 * (size_t)k + 2];
      split(zop[k], &ac.x, &ac.y);
      split(zop[2 * nz + k], &ac.z, &ac.w);
      split(zop[nz + k], &bw.x, &bw.y);
      split(P->dzf[k], &bw.z, &bw.w);
      split(sum + err, &dw.x, &dw.y);
      dw.z = bw.z;
      dw.w = bw.w;
      wsum += P->dzf[k];
    }
    float4& axy = zk[3 * (size_t)nz];
    split(1.0 / (dx * dx), &axy.x, &axy.y);
    split(1.0 / (dy * dy), &axy.z, &axy.w);
    if (!rc) rc = dev_upload(&P->d_zk, zk.data(), zk.size(), &P->device_bytes);
    P->inv_wn = 1.0 / (wsum * (double)nx * (double)ny);
    if (!rc)
      rc = dev_alloc_guarded(P, &P->d_mpart, ((size_t)nx * ny + 127) / 128);
    if (!rc) rc = dev_alloc_guarded(P, &P->d_r32b, (size_t)nx * ny * nz);
    if (!rc) rc = dev_alloc_guarded(P, &P->d_rlo, (size_t)nx * ny * nz);
    if (!rc) rc = dev_alloc_guarded(P, &P->d_w2, (size_t)nx * ny * nz);
  }

  if (!rc) rc = dev_upload(&dA, A.data(), A.size(), &scratch);
  if (!rc) rc = dev_upload(&dB, B.data(), B.size(), &scratch);
  if (!rc) rc = dev_upload(&dC, C.data(), C.size(), &scratch);
  if (!rc) rc = dev_upload(&dlx, lamx.data(), lamx.size(), &scratch);
  if (!rc) rc = dev_upload(&dly, lamy.data(), lamy.size(), &scratch);
  if (!rc) rc = cuda_status(launch_thomas_factor(P, dA, dB, dC, dlx, dly, 0));
  if (!rc) rc = cuda_status(cudaDeviceSynchronize());
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(dlx);
  cudaFree(dly);
  if (rc) {
    plan_free(P);
    return rc;
  }
  *out = P;
  return CFS_OK;
}

extern "C" int cfs_plan_destroy(cfs_plan_t P) {
  if (!P) return CFS_EINVAL;
  CaptureLock lock(capture_mutex());
  cudaDeviceSynchronize();
  plan_free(P);
  return CFS_OK;
}

extern "C" int cfs_plan_device_bytes(cfs_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CFS_EINVAL;
  *bytes = P->device_bytes;
  return CFS_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" int cfs_spectral_forward(cfs_plan_t P, const double* f, double* s, void* stream) {
  if (!P || !f || !s || !aligned16(f) || !aligned16(s)) return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_rfft_x(P, f, s, false, 1.0, st);
  if (e == cudaSuccess) e = launch_fft_y(P, s, false, st);
  return e == cudaErrorInvalidValue ? CFS_EINVAL : cuda_status(e);
}

extern "C" int cfs_spectral_inverse(cfs_plan_t P, const double* s, double* f, void* stream) {
  if (!P || !f || !s || !aligned16(f) || !aligned16(s)) return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the y pass works in place, so it runs on the output buffer
  cudaError_t e = cudaSuccess;
  if (s != f)
    e = cudaMemcpyAsync(f, s, sizeof(double) * (size_t)P->nx * P->ny * P->nz,
                        cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_fft_y(P, f, true, st);
  if (e == cudaSuccess) e = launch_rfft_x(P, f, f, true, 2.0 / ((double)P->nx * P->ny), st);
  return e == cudaErrorInvalidValue ? CFS_EINVAL : cuda_status(e);
}

static int ensure_stage(cfs_plan* P);

extern "C" int cfs_poisson_solve(cfs_plan_t P, const double* f, double* p, void* stream) {
  if (!P || !f || !p || !aligned16(f) || !aligned16(p)) return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (P->dtype == CFS_F32_REFINED) {
    if (f == p) {  // the residual needs f for every iteration
      int rc = ensure_stage(P);
      if (rc) return rc;
      if (cudaMemcpyAsync(P->d_stage, f, sizeof(double) * (size_t)P->nx * P->ny * P->nz,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return CFS_ECUDA;
      f = P->d_stage;
    }
    return refine_poisson(P, f, p, st);
  }
  cudaError_t e = launch_rfft_x(P, f, p, false, 1.0, st);
  if (e == cudaSuccess) e = launch_fft_y(P, p, false, st);
  if (e == cudaSuccess) e = launch_thomas(P, p, st);
  if (e == cudaSuccess) e = launch_fft_y(P, p, true, st);
  if (e == cudaSuccess) e = launch_rfft_x(P, p, p, true, 1.0, st);
  return e == cudaErrorInvalidValue ? CFS_EINVAL : cuda_status(e);
}

extern "C" int cfs_poisson_stage(cfs_plan_t P, int stage, const double* in, double* out,
                                 void* stream) {
  if (!P || !in || !out || !aligned16(in) || !aligned16(out)) return CFS_EINVAL;
  if (stage < CFS_STAGE_X_FORWARD || stage > CFS_STAGE_X_INVERSE) return CFS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (stage == CFS_STAGE_X_FORWARD) {
    e = launch_rfft_x(P, in, out, false, 1.0, st);
  } else if (stage == CFS_STAGE_X_INVERSE) {
    e = launch_rfft_x(P, in, out, true, 1.0, st);
  } else {
    if (in != out)
      e = cudaMemcpyAsync(out, in, sizeof(double) * (size_t)P->nx * P->ny * P->nz,
                          cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
      if (stage == CFS_STAGE_Y_FORWARD) e = launch_fft_y(P, out, false, st);
      else if (stage == CFS_STAGE_Y_INVERSE) e = launch_fft_y(P, out, true, st);
      else e = launch_thomas(P, out, st);
    }
  }
  return e == cudaErrorInvalidValue ? CFS_EINVAL : cuda_status(e);
}

// ----------------------------------------------------------------------------
// Helmholtz: Algorithm 2, Step 1 on the host in FP64 (Sec. 2.2.4: the
// coefficients are the same for every (x, y) column, so every GPU computes
// them locally instead of communicating them).
// ----------------------------------------------------------------------------
static HelmCoef* helm_find(cfs_plan* P, double c, int loc, int nparts) {
  for (auto& h : P->helm)
    if (h.c == c && h.loc == loc && (nparts == 0 || h.nparts == nparts)) return &h;
  return nullptr;
}

static int auto_parts(int n) { return alg2_auto_parts(n, kPcrMaxParts); }

// Frees one cached set (the device must be idle on it).
static void helm_release(cfs_plan* P, HelmCoef& h) {
  const size_t n = (size_t)h.n, p = (size_t)h.nparts;
  cudaFree(h.d_rows);
  cudaFree(h.d_red);
  cudaFree(h.d_th);
  P->device_bytes -= sizeof(double) * (5 * n + 6 * p + 3 * n);
  if (h.d_rows32) {
    cudaFree(h.d_rows32);
    cudaFree(h.d_red32);
    cudaFree(h.d_abc);
    cudaFree(h.d_th32);
    P->device_bytes -= sizeof(float) * (5 * n + 6 * p + 3 * n) + sizeof(double) * 3 * n;
  }
  if (h.d_lv32) {
    cudaFree(h.d_lv32);
    P->device_bytes -= sizeof(float) * (2 * (size_t)alg2_pcr_levels(2 * (int)p) + 1) * 2 * p;
  }
}

static int helm_prepare(cfs_plan* P, double c, int loc, int nparts, HelmCoef** res) {
  CaptureLock lock(capture_mutex());
  if (!(c >= 0) || !isfinite(c)) return CFS_EINVAL;
  if (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE) return CFS_EINVAL;
  if (nparts < 0 || nparts > kPcrMaxParts) return CFS_EUNSUPPORTED;
  if (HelmCoef* h = helm_find(P, c, loc, nparts)) {
    h->stamp = ++P->helm_clock;
    *res = h;
    return CFS_OK;
  }
  std::vector<double> A, B, C;
  const int n = z_stencil(P->dzf, CFS_BC_DIRICHLET, loc, A, B, C);
  for (int i = 0; i < n; ++i) {  // I - c L_z
    A[i] = -c * A[i];
    B[i] = 1.0 - c * B[i];
    C[i] = -c * C[i];
  }
  if (n < 3 || n > kPcrMaxUnknowns) return CFS_EUNSUPPORTED;
  const int np = nparts ? nparts : (P->pcr_parts ? P->pcr_parts : auto_parts(n));
  if (pcr_smem_bytes(n, np) > 227 * 1024) return CFS_EUNSUPPORTED;
  HelmCoef h;
  memset(&h, 0, sizeof(h));
  h.c = c;
  h.loc = loc;
  h.nparts = np;
  h.n = n;
  h.mmax = 0;
  for (int q = 0; q <= np; ++q) h.start[q] = alg2_part_start(q, n, np);
  for (int q = 0; q < np; ++q) {
    const int m = h.start[q + 1] - h.start[q];
    if (m < 3) return CFS_EUNSUPPORTED;
    h.mmax = std::max(h.mmax, m);
  }
  std::vector<double> rows(5 * (size_t)n, 0.0);
  double* alpha = rows.data();
  double* beta = alpha + n;
  double* ib = beta + n;
  double* ap = ib + n;
  double* cpv = ap + n;
  const int J = 2 * np;
  std::vector<double> ra(J), rb(J), rc(J);
  for (int q = 0; q < np; ++q) {
    const int o = h.start[q], m = h.start[q + 1] - o;
    // Step 1 of Algorithm 2, and the partition's two rows of the reduced system
    const ArrayRows row{A.data(), B.data(), C.data(), o};
    double first[3], last[3];
    alg2_factor_partition(m, row, alpha + o, beta + o, ib + o, ap + o, cpv + o, first, last);
    ra[2 * q] = first[0];
    rb[2 * q] = first[1];
    rc[2 * q] = first[2];
    ra[2 * q + 1] = last[0];
    rb[2 * q + 1] = last[1];
    rc[2 * q + 1] = last[2];
  }
  // LU of the reduced system (Step 3; no pivoting: diagonally dominant)
  std::vector<double> red(3 * (size_t)J);
  alg2_reduced_factor(J, ra.data(), rb.data(), rc.data(), red.data(), red.data() + J,
                      red.data() + 2 * J);
  // Thomas factors of the same system: fs = 1/piv, fa = A'/piv, fc = C'/piv
  std::vector<double> th(3 * (size_t)n);
  {
    double pv = B[0];
    for (int i = 0; i < n; ++i) {
      if (i > 0) pv = B[i] - A[i] * th[2 * (size_t)n + i - 1];
      th[i] = 1.0 / pv;
      th[(size_t)n + i] = (i > 0) ? A[i] / pv : 0.0;
      th[2 * (size_t)n + i] = (i < n - 1) ? C[i] / pv : 0.0;
    }
  }
  int rcode = dev_upload(&h.d_rows, rows.data(), rows.size(), &P->device_bytes);
  if (!rcode) rcode = dev_upload(&h.d_red, red.data(), red.size(), &P->device_bytes);
  if (!rcode) rcode = dev_upload(&h.d_th, th.data(), th.size(), &P->device_bytes);
  if (!rcode && P->dtype == CFS_F32_REFINED) {
    // FP32 copies for the inner solves; the FP64 rows of I - c L_z for the residual
    std::vector<float> rows32(rows.begin(), rows.end()), red32(red.begin(), red.end());
    std::vector<double> abc(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
      abc[i] = A[i];
      abc[n + i] = B[i];
      abc[2 * n + i] = C[i];
    }
    rcode = dev_upload(&h.d_rows32, rows32.data(), rows32.size(), &P->device_bytes);
    if (!rcode) rcode = dev_upload(&h.d_red32, red32.data(), red32.size(), &P->device_bytes);
    if (!rcode) rcode = dev_upload(&h.d_abc, abc.data(), abc.size(), &P->device_bytes);
    std::vector<float> th32(th.begin(), th.end());
    if (!rcode) rcode = dev_upload(&h.d_th32, th32.data(), th32.size(), &P->device_bytes);
    // the reduced system by parallel cyclic reduction (the one-pass refined solve)
    const int L = alg2_pcr_levels(J);
    std::vector<double> sub(ra), diag(rb), sup(rc), na(J), nb(J), nc(J);
    std::vector<double> lv((2 * (size_t)L + 1) * J);
    alg2_reduced_pcr(J, sub.data(), diag.data(), sup.data(), na.data(), nb.data(), nc.data(),
                     lv.data(), lv.data() + (size_t)L * J, lv.data() + 2 * (size_t)L * J);
    std::vector<float> lv32(lv.begin(), lv.end());
    if (!rcode) rcode = dev_upload(&h.d_lv32, lv32.data(), lv32.size(), &P->device_bytes);
  }
  if (rcode) {
    cudaFree(h.d_rows);
    cudaFree(h.d_red);
    cudaFree(h.d_th);
    cudaFree(h.d_rows32);
    cudaFree(h.d_red32);
    cudaFree(h.d_abc);
    cudaFree(h.d_th32);
    cudaFree(h.d_lv32);
    return rcode;
  }
  // bounded cache: evict the least recently used entry
  const size_t kMaxEntries = 32;
  if (P->helm.size() >= kMaxEntries) {
    auto it = std::min_element(P->helm.begin(), P->helm.end(),
                               [](const HelmCoef& x, const HelmCoef& y) { return x.stamp < y.stamp; });
    cudaDeviceSynchronize();
    helm_release(P, *it);
    P->helm.erase(it);
  }
  h.stamp = ++P->helm_clock;
  P->helm.push_back(h);
  *res = &P->helm.back();
  return CFS_OK;
}

int chanfs::plan_helm_prepare(cfs_plan* P, double c, int loc, int nparts, HelmCoef** out) {
  return helm_prepare(P, c, loc, nparts ? nparts : P->pcr_parts, out);
}

// Drops the cached Algorithm 2 sets of coefficient c (the tuner's probes).
void chanfs::plan_helm_forget(cfs_plan* P, double c) {
  CaptureLock lock(capture_mutex());
  cudaDeviceSynchronize();
  for (size_t i = 0; i < P->helm.size();) {
    if (P->helm[i].c == c) {
      helm_release(P, P->helm[i]);
      P->helm.erase(P->helm.begin() + i);
    } else {
      ++i;
    }
  }
}

// ----------------------------------------------------------------------------
// Fully implicit 3-D Helmholtz (Eq. 8): (I - c L) u = rhs on the Poisson
// machinery.  After the x and y transforms each (kx, ky) column solves
//   -c A_k U_{k-1} + (1 - c (B_k + lx + ly)) U_k - c C_k U_{k+1} = F_k
// on the Dirichlet rows of the field's location (n = nz centred, nz - 1
// face); the factors of every column are computed once per (c, loc) on the
// GPU and kept in a small LRU cache.
// ----------------------------------------------------------------------------
static int helm3_prepare(cfs_plan* P, double c, int loc, Helm3Coef** res) {
  CaptureLock lock(capture_mutex());
  if (!(c >= 0) || !isfinite(c)) return CFS_EINVAL;
  if (loc != CFS_LOC_CENTER && loc != CFS_LOC_FACE) return CFS_EINVAL;
  for (auto& h : P->helm3)
    if (h.c == c && h.loc == loc) {
      h.stamp = ++P->helm_clock;
      *res = &h;
      return CFS_OK;
    }
  std::vector<double> A, B, C;
  const int n = z_stencil(P->dzf, CFS_BC_DIRICHLET, loc, A, B, C);
  for (int i = 0; i < n; ++i) {  // -c A, 1 - c B, -c C; the x-y shift enters as -c lambda
    A[i] = -c * A[i];
    B[i] = 1.0 - c * B[i];
    C[i] = -c * C[i];
  }
  std::vector<double> lx(P->lamx_h), ly(P->lamy_h);
  for (double& v : lx) v *= -c;
  for (double& v : ly) v *= -c;
  Helm3Coef h;
  memset(&h, 0, sizeof(h));
  h.c = c;
  h.loc = loc;
  h.n = n;
  const size_t nfac = (size_t)(P->M + 1) * P->nky * n;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr, *dlx = nullptr, *dly = nullptr;
  size_t scratch = 0;
  int rc = dev_upload<double2>(&h.d_fwd, nullptr, nfac, &P->device_bytes);
  if (!rc) rc = dev_upload<double>(&h.d_bwd, nullptr, nfac, &P->device_bytes);
  if (!rc) rc = dev_upload(&dA, A.data(), (size_t)n, &scratch);
  if (!rc) rc = dev_upload(&dB, B.data(), (size_t)n, &scratch);
  if (!rc) rc = dev_upload(&dC, C.data(), (size_t)n, &scratch);
  if (!rc) rc = dev_upload(&dlx, lx.data(), lx.size(), &scratch);
  if (!rc) rc = dev_upload(&dly, ly.data(), ly.size(), &scratch);
  if (!rc) rc = cuda_status(launch_thomas_factor_set(P, h.d_fwd, h.d_bwd, n, dA, dB, dC, dlx, dly, 0));
  if (!rc) rc = cuda_status(cudaDeviceSynchronize());
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(dlx);
  cudaFree(dly);
  if (rc) {
    cudaFree(h.d_fwd);
    cudaFree(h.d_bwd);
    return rc;
  }
  const size_t kMaxEntries = 4;  // each set is as large as the Poisson factors
  if (P->helm3.size() >= kMaxEntries) {
    auto it = std::min_element(P->helm3.begin(), P->helm3.end(),
                               [](const Helm3Coef& x, const Helm3Coef& y) { return x.stamp < y.stamp; });
    cudaDeviceSynchronize();
    cudaFree(it->d_fwd);
    cudaFree(it->d_bwd);
    P->device_bytes -= (sizeof(double2) + sizeof(double)) * (size_t)(P->M + 1) * P->nky * it->n;
    P->helm3.erase(it);
  }
  h.stamp = ++P->helm_clock;
  P->helm3.push_back(h);
  *res = &P->helm3.back();
  return CFS_OK;
}

extern "C" int cfs_helmholtz3d_prepare(cfs_plan_t P, double c, int loc) {
  if (!P) return CFS_EINVAL;
  Helm3Coef* h = nullptr;
  return helm3_prepare(P, c, loc, &h);
}

extern "C" int cfs_helmholtz3d_solve(cfs_plan_t P, double c, int loc, const double* rhs,
                                     double* u, void* stream) {
  if (!P || !rhs || !u || !aligned16(rhs) || !aligned16(u)) return CFS_EINVAL;
  Helm3Coef* h = nullptr;
  int rc = helm3_prepare(P, c, loc, &h);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_rfft_x(P, rhs, u, false, 1.0, st);
  if (e == cudaSuccess) e = launch_fft_y(P, u, false, st);
  if (e == cudaSuccess) e = launch_thomas_set(P, u, h->d_fwd, h->d_bwd, h->n, st);
  const size_t plane = (size_t)P->nx * P->ny;
  if (e == cudaSuccess && h->n < P->nz)  // the wall slot of a face field
    e = cudaMemsetAsync(u + plane * (P->nz - 1), 0, sizeof(double) * plane, st);
  if (e == cudaSuccess) e = launch_fft_y(P, u, true, st);
  if (e == cudaSuccess) e = launch_rfft_x(P, u, u, true, 1.0, st);
  return cuda_status(e);
}

extern "C" int cfs_helmholtz_prepare(cfs_plan_t P, double c, int loc, int nparts) {
  if (!P) return CFS_EINVAL;
  HelmCoef* h = nullptr;
  return helm_prepare(P, c, loc, nparts, &h);
}

extern "C" int cfs_helmholtz_solve(cfs_plan_t P, double c, int loc, const double* rhs, double* u,
                                   void* stream) {
  if (!P || !rhs || !u || !aligned16(rhs) || !aligned16(u)) return CFS_EINVAL;
  HelmCoef* h = nullptr;
  int rc = helm_prepare(P, c, loc, P->pcr_parts, &h);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (P->dtype == CFS_F32_REFINED) {
    if (rhs == u && !P->helm_fp64) {
      rc = ensure_stage(P);
      if (rc) return rc;
      if (cudaMemcpyAsync(P->d_stage, rhs, sizeof(double) * (size_t)P->nx * P->ny * P->nz,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return CFS_ECUDA;
      rhs = P->d_stage;
    }
    if (!P->helm_fp64) return refine_helmholtz(P, *h, rhs, u, st);
    P->last_iters = 0;
    P->last_rho = 0.0;
  }
  return cuda_status(launch_helm64(P, *h, rhs, u, st));
}

cudaError_t chanfs::launch_helm64(const cfs_plan* P, const HelmCoef& h, const double* rhs,
                                  double* u, cudaStream_t st) {
  return P->helm_thomas ? launch_helm_thomas(P, h, rhs, u, st) : launch_pcr(P, h, rhs, u, st);
}

cudaError_t chanfs::launch_helm32(const cfs_plan* P, const HelmCoef& h, const float* rhs,
                                  float* u, cudaStream_t st) {
  return P->helm_thomas32 ? launch_helm_thomas32(P, h, rhs, u, st)
                          : launch_pcr32(P, h, rhs, u, st);
}

extern "C" int cfs_plan_set_refinement(cfs_plan_t P, double tol, int maxit) {
  if (!P || !(tol > 0) || !isfinite(tol) || maxit < 1 || maxit > 64) return CFS_EINVAL;
  P->tol = tol;
  P->maxit = maxit;
  return CFS_OK;
}

// Rebuilds the x and y radix plans with passes of at most max_radix (8 or 4)
// and replaces their twiddle tables (FP64, and FP32 for refined plans).  The
// table sizes do not change (n - 1 entries), so neither do the tiles.
int chanfs::plan_set_radix(cfs_plan* P, int max_radix) {
  if (P->fft_radix == max_radix) return CFS_OK;
  CaptureLock lock(capture_mutex());
  FftDesc fx, fy;
  std::vector<double2> twx, twy;
  if (!make_fft_desc(P->M, &fx, &twx, max_radix) || !make_fft_desc(P->ny, &fy, &twy, max_radix))
    return CFS_EUNSUPPORTED;
  cudaDeviceSynchronize();  // no solve may be reading the old tables
  auto put64 = [&](double2* dst, const std::vector<double2>& v) {
    return cudaMemcpy(dst, v.data(), sizeof(double2) * v.size(), cudaMemcpyHostToDevice);
  };
  auto put32 = [&](float2* dst, const std::vector<double2>& v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
    return cudaMemcpy(dst, o.data(), sizeof(float2) * o.size(), cudaMemcpyHostToDevice);
  };
  cudaError_t e = put64(P->d_twx, twx);
  if (e == cudaSuccess) e = put64(P->d_twy, twy);
  if (e == cudaSuccess && P->d_twx32) e = put32(P->d_twx32, twx);
  if (e == cudaSuccess && P->d_twy32) e = put32(P->d_twy32, twy);
  if (e != cudaSuccess) return CFS_ECUDA;
  P->fx = fx;
  P->fy = fy;
  P->fft_radix = max_radix;
  return CFS_OK;
}

// Chunks of a streamed FP64 batch field (CFS_OPT_STREAM_CHUNKS): z-plane
// ranges of a Poisson field, (x, y)-column ranges (whole y rows) of a
// Helmholtz field solved by Algorithm 2; 1 for the solves that take the whole
// field at once.  Automatic: about 200 MB per chunk (3 for a 604 MB channel
// field; on GB300 2, 3, 4 and 6 chunks gave 19.4, 19.0, 20.0 and 19.9 ms per
// channel step against 20.8 ms whole, and 8 chunks 23.2 ms), at most
// kMaxStreamChunks.
static int batch_chunks(const cfs_plan* P, int kind) {
  const size_t plane = (size_t)P->nx * P->ny;
  if (P->dtype != CFS_F64 || (P->nx & 1)) return 1;
  if (kind == CFS_REQ_HELMHOLTZ && (P->helm_thomas || sizeof(double) * plane > (1u << 30)))
    return 1;  // (Thomas sweeps take the field whole; 2-D copy pitches stay modest)
  const int extent = (kind == CFS_REQ_POISSON) ? P->nz : P->ny;
  int k = P->stream_chunks;
  if (k == 0)
    k = (int)std::min<size_t>(kMaxStreamChunks, sizeof(double) * plane * P->nz / (192u << 20));
  return std::max(1, std::min(k, extent));
}

extern "C" int cfs_plan_set_option(cfs_plan_t P, int option, int value) {
  if (!P) return CFS_EINVAL;
  switch (option) {
    case CFS_OPT_THOMAS_TILE: {
      if (value != 0 && value != -1 && value != 1 && value != 8 && value != 16) return CFS_EINVAL;
      const bool fp32 = (P->dtype == CFS_F32_REFINED);
      if (value == 1 && !fp32) return CFS_EUNSUPPORTED;  // the partitioned solve is FP32
      if (thomas_tile_width(P, false, value) == 0 ||
          (fp32 && thomas_tile_width(P, true, value) == 0))
        return CFS_EUNSUPPORTED;
      P->thomas_tw = value;
      return CFS_OK;
    }
    case CFS_OPT_X_LINES: {
      if (value < 0 || value > 64) return CFS_EINVAL;
      const size_t cs = (P->dtype == CFS_F32_REFINED) ? sizeof(float2) : sizeof(double2);
      if (value > 0 && x_smem_bytes(P, value, cs) > 227 * 1024) return CFS_EUNSUPPORTED;
      P->x_lines = value;
      return CFS_OK;
    }
    case CFS_OPT_Y_TILE: {
      const bool fp32 = (P->dtype == CFS_F32_REFINED);
      if (value < 0 || value > 32) return CFS_EINVAL;
      if (value > 0 && !y_tile_ok(P, value, fp32)) return CFS_EUNSUPPORTED;
      if (fp32) P->tk32 = value ? value : P->tk32_auto;
      else P->tk = value ? value : P->tk_auto;
      return CFS_OK;
    }
    case CFS_OPT_HELM_FP64:
      if (value != 0 && value != 1) return CFS_EINVAL;
      P->helm_fp64 = value;
      return CFS_OK;
    case CFS_OPT_HELM_THOMAS:
      if (value != 0 && value != 1) return CFS_EINVAL;
      P->helm_thomas = value;
      return CFS_OK;
    case CFS_OPT_FFT_RADIX:
      if (value != 0 && value != 4 && value != 8) return CFS_EINVAL;
      return plan_set_radix(P, value ? value : 8);
    case CFS_OPT_HELM_THOMAS32:
      if (value != 0 && value != 1) return CFS_EINVAL;
      if (value && P->dtype != CFS_F32_REFINED) return CFS_EUNSUPPORTED;
      P->helm_thomas32 = value;
      return CFS_OK;
    case CFS_OPT_F64_ADDS_X:
    case CFS_OPT_F64_ADDS_Y:
      if (value < 0 || value > 4) return CFS_EINVAL;
      (option == CFS_OPT_F64_ADDS_X ? P->emu_x : P->emu_y) = value;
      return CFS_OK;
    case CFS_OPT_STREAM_CHUNKS:
      if (value < 0 || value > kMaxStreamChunks) return CFS_EINVAL;
      P->stream_chunks = value;
      return CFS_OK;
    case CFS_OPT_PCR_PARTS: {
      if (value < 0 || value > kPcrMaxParts) return CFS_EINVAL;
      for (int n = P->nz - 1; value > 0 && n <= P->nz; ++n)  // face and centred fields
        if (n / value < 3 || pcr_smem_bytes(n, value) > 227 * 1024) return CFS_EUNSUPPORTED;
      P->pcr_parts = value;
      return CFS_OK;
    }
    default:
      return CFS_EINVAL;
  }
}

extern "C" int cfs_plan_get_option(cfs_plan_t P, int option, int* value) {
  if (!P || !value) return CFS_EINVAL;
  switch (option) {
    case CFS_OPT_THOMAS_TILE:
      *value = thomas_tile_width(P, P->dtype == CFS_F32_REFINED, P->thomas_tw);
      return CFS_OK;
    case CFS_OPT_X_LINES:
      *value = x_lines_per_cta(P, P->dtype == CFS_F32_REFINED ? sizeof(float2) : sizeof(double2));
      return CFS_OK;
    case CFS_OPT_Y_TILE:
      *value = (P->dtype == CFS_F32_REFINED) ? P->tk32 : P->tk;
      return CFS_OK;
    case CFS_OPT_PCR_PARTS:
      *value = P->pcr_parts ? P->pcr_parts : auto_parts(P->nz);
      return CFS_OK;
    case CFS_OPT_HELM_FP64:
      *value = (P->dtype == CFS_F32_REFINED) ? P->helm_fp64 : 1;
      return CFS_OK;
    case CFS_OPT_HELM_THOMAS:
      *value = P->helm_thomas;
      return CFS_OK;
    case CFS_OPT_FFT_RADIX:
      *value = P->fft_radix;
      return CFS_OK;
    case CFS_OPT_HELM_THOMAS32:
      *value = P->helm_thomas32;
      return CFS_OK;
    case CFS_OPT_F64_ADDS_X:
      *value = P->emu_x;
      return CFS_OK;
    case CFS_OPT_F64_ADDS_Y:
      *value = P->emu_y;
      return CFS_OK;
    case CFS_OPT_STREAM_CHUNKS:
      *value = batch_chunks(P, CFS_REQ_POISSON);
      return CFS_OK;
    default:
      return CFS_EINVAL;
  }
}

extern "C" int cfs_last_info(cfs_plan_t P, int* iters, double* rel_residual) {
  if (!P) return CFS_EINVAL;
  if (iters) *iters = P->last_iters;
  if (rel_residual) *rel_residual = P->last_rho;
  return CFS_OK;
}

// ----------------------------------------------------------------------------
// Host-buffer variants
// ----------------------------------------------------------------------------
int chanfs::plan_ensure_stage(cfs_plan* P) { return ensure_stage(P); }

static int ensure_stage(cfs_plan* P) {
  if (P->d_stage) return CFS_OK;
  CaptureLock lock(capture_mutex());
  const size_t bytes = sizeof(double) * (size_t)P->nx * P->ny * P->nz;
  if (cudaMalloc(&P->d_stage, bytes) != cudaSuccess) return CFS_ENOMEM;
  P->device_bytes += bytes;
  return CFS_OK;
}

extern "C" int cfs_poisson_solve_host(cfs_plan_t P, const double* f, double* p, void* stream) {
  if (!P || !f || !p) return CFS_EINVAL;
  int rc = ensure_stage(P);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)P->nx * P->ny * P->nz;
  if (cudaMemcpyAsync(P->d_stage, f, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CFS_ECUDA;
  rc = cfs_poisson_solve(P, P->d_stage, P->d_stage, stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(p, P->d_stage, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CFS_ECUDA;
  return cuda_status(cudaStreamSynchronize(st));
}

extern "C" int cfs_helmholtz_solve_host(cfs_plan_t P, double c, int loc, const double* rhs,
                                        double* u, void* stream) {
  if (!P || !rhs || !u) return CFS_EINVAL;
  int rc = ensure_stage(P);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)P->nx * P->ny * P->nz;
  if (cudaMemcpyAsync(P->d_stage, rhs, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return CFS_ECUDA;
  rc = cfs_helmholtz_solve(P, c, loc, P->d_stage, P->d_stage, stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(u, P->d_stage, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CFS_ECUDA;
  return cuda_status(cudaStreamSynchronize(st));
}

// Staging of batched host-buffer solves (grown to `slots` slots), its
// streams and events (made once).
static int ensure_batch(cfs_plan* P, int slots) {
  CaptureLock lock(capture_mutex());
  const size_t field = sizeof(double) * (size_t)P->nx * P->ny * P->nz;
  if (slots > P->batch_slots) {
    if (P->d_batch) {
      cudaDeviceSynchronize();  // no earlier batch may still use the old slots
      cudaFree(P->d_batch);
      P->device_bytes -= 2 * field * (size_t)P->batch_slots;
      P->d_batch = nullptr;
      P->batch_slots = 0;
    }
    if (cudaMalloc(&P->d_batch, 2 * field * (size_t)slots) != cudaSuccess) {
      P->d_batch = nullptr;
      return CFS_ENOMEM;
    }
    P->batch_slots = slots;
    P->device_bytes += 2 * field * (size_t)slots;
  }
  if (P->copy_in) return CFS_OK;
  cudaError_t e = cudaSuccess;
  for (cudaStream_t* q : {&P->copy_in, &P->copy_out, &P->copy_out2, &P->compute2})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(q, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_entry, cudaEventDisableTiming);
  for (int k = 0; k < kBatchSlots && e == cudaSuccess; ++k) {
    for (cudaEvent_t* v : {&P->ev_done[k], &P->ev_free[k]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(v, cudaEventDisableTiming);
    for (int c = 0; c < kMaxStreamChunks; ++c)
      for (cudaEvent_t* v : {&P->ev_cin[k][c], &P->ev_cdone[k][c]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(v, cudaEventDisableTiming);
  }
  return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
}

// n solves through host buffers, pipelined over up to kBatchSlots device
// slots (the job at position p of the processing order in slot p mod K): the
// inputs are copied in back to back on one copy stream as their slots free
// up; each solve starts when its input has arrived and its slot's previous
// output has been copied out; each result is copied out as soon as it is
// ready.  On FP64 plans the Helmholtz solves run on a second compute stream,
// beside the Poisson solves (the two kinds share no plan scratch; refined
// solves share the FP32 work fields and stay on the caller's stream), each
// compute stream with its own copy-out stream.  The copy of the next input is
// enqueued before solve p starts, so that it proceeds even while a refined
// solve waits on the host.
//
// FP64 plans stream their fields in chunks (batch_chunks): a Poisson field in
// ranges of z planes, whose forward x transforms start as each range lands and
// whose inverse x transforms hand each range to the copy-out stream as it is
// done; a Helmholtz field solved by Algorithm 2 in ranges of y rows (2-D
// copies), each solved and copied out on its own.  The host link then carries
// inputs and results at once from the first chunk on, instead of waiting for
// whole fields.  Every chunk is computed by the same kernels on the same
// columns or lines as a whole-field solve, so the results are the same bits.
// The first Helmholtz job of a batch that also holds Poisson jobs is taken
// first: its chunks come back while the Poisson input is still arriving.
extern "C" int cfs_solve_batch_host(cfs_plan_t P, int n, const int* kind, const double* c,
                                    const int* loc, const double* const* in, double* const* out,
                                    void* stream) {
  if (!P || n < 0 || (n > 0 && (!kind || !in || !out))) return CFS_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!in[i] || !out[i]) return CFS_EINVAL;
    if (kind[i] == CFS_REQ_HELMHOLTZ) {
      if (!c || !loc || !(c[i] >= 0) || !isfinite(c[i])) return CFS_EINVAL;
      if (loc[i] != CFS_LOC_CENTER && loc[i] != CFS_LOC_FACE) return CFS_EINVAL;
    } else if (kind[i] != CFS_REQ_POISSON) {
      return CFS_EINVAL;
    }
  }
  if (n == 0) return CFS_OK;
  const int K = std::min(n, kBatchSlots);
  int rc = ensure_batch(P, K);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool two = (P->dtype == CFS_F64);  // Helmholtz beside Poisson
  const size_t plane = (size_t)P->nx * P->ny;
  const size_t nf = plane * P->nz;
  const size_t bytes = sizeof(double) * nf;
  // processing order: the first Helmholtz job ahead when Poisson jobs are streamed too
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  if (two) {
    int first_h = -1;
    bool any_p = false;
    for (int i = 0; i < n; ++i) {
      if (kind[i] == CFS_REQ_HELMHOLTZ && first_h < 0) first_h = i;
      any_p = any_p || kind[i] == CFS_REQ_POISSON;
    }
    if (first_h > 0 && any_p && batch_chunks(P, CFS_REQ_HELMHOLTZ) > 1)
      std::rotate(ord.begin(), ord.begin() + first_h, ord.begin() + first_h + 1);
  }
  auto din = [&](int s) { return P->d_batch + (size_t)(2 * s) * nf; };
  auto dout = [&](int s) { return P->d_batch + (size_t)(2 * s + 1) * nf; };
  auto cstream = [&](int i) {
    return (two && kind[i] == CFS_REQ_HELMHOLTZ) ? P->compute2 : st;
  };
  auto ostream = [&](int i) {
    return (two && kind[i] == CFS_REQ_HELMHOLTZ) ? P->copy_out2 : P->copy_out;
  };
  // chunk q of job i: element offset, and the 2-D shape (rows x width
  // elements, rows nf / nz apart) for column ranges
  struct Chunk {
    size_t off, rows, width;
  };
  auto chunk = [&](int i, int q, int nq) {
    if (nq == 1) return Chunk{0, 1, nf};
    if (kind[i] == CFS_REQ_POISSON) {  // z planes [z0, z1)
      const size_t z0 = (size_t)P->nz * q / nq, z1 = (size_t)P->nz * (q + 1) / nq;
      return Chunk{z0 * plane, 1, (z1 - z0) * plane};
    }
    const size_t y0 = (size_t)P->ny * q / nq, y1 = (size_t)P->ny * (q + 1) / nq;  // y rows
    return Chunk{y0 * P->nx, (size_t)P->nz, (y1 - y0) * P->nx};
  };
  auto copy = [&](double* dst, const double* src, const Chunk& k, cudaMemcpyKind dir,
                  cudaStream_t q) {
    if (k.rows == 1)
      return cudaMemcpyAsync(dst + k.off, src + k.off, sizeof(double) * k.width, dir, q);
    return cudaMemcpy2DAsync(dst + k.off, sizeof(double) * plane, src + k.off,
                             sizeof(double) * plane, sizeof(double) * k.width, k.rows, dir, q);
  };
  // everything starts after the work already on the caller's stream
  cudaError_t e = cudaEventRecord(P->ev_entry, st);
  for (cudaStream_t q : {P->copy_in, P->copy_out, P->copy_out2, P->compute2})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(q, P->ev_entry, 0);
  auto copy_in = [&](int p) {
    const int i = ord[p], s = p % K, nq = batch_chunks(P, kind[i]);
    cudaError_t r = cudaSuccess;
    if (p >= K) r = cudaStreamWaitEvent(P->copy_in, P->ev_done[s], 0);  // solve p-K read it
    for (int q = 0; q < nq && r == cudaSuccess; ++q) {
      r = copy(din(s), in[i], chunk(i, q, nq), cudaMemcpyHostToDevice, P->copy_in);
      if (r == cudaSuccess) r = cudaEventRecord(P->ev_cin[s][q], P->copy_in);
    }
    return r;
  };
  if (e == cudaSuccess) e = copy_in(0);
  for (int p = 0; p < n && e == cudaSuccess; ++p) {
    const int i = ord[p], s = p % K, nq = batch_chunks(P, kind[i]);
    cudaStream_t cs = cstream(i);
    if (p + 1 < n) e = copy_in(p + 1);
    if (e == cudaSuccess && p >= K)  // the output of solve p-K has been copied out
      e = cudaStreamWaitEvent(cs, P->ev_free[s], 0);
    if (e != cudaSuccess) break;
    int r = CFS_OK;
    if (nq == 1) {
      e = cudaStreamWaitEvent(cs, P->ev_cin[s][0], 0);
      if (e != cudaSuccess) break;
      r = (kind[i] == CFS_REQ_POISSON)
              ? cfs_poisson_solve(P, din(s), dout(s), cs)
              : cfs_helmholtz_solve(P, c[i], loc[i], din(s), dout(s), cs);
      if (r == CFS_OK || r == CFS_ENOTCONVERGED) e = cudaEventRecord(P->ev_cdone[s][0], cs);
    } else if (kind[i] == CFS_REQ_POISSON) {  // the stages of cfs_poisson_solve, x by z ranges
      for (int q = 0; q < nq && e == cudaSuccess; ++q) {
        const Chunk k = chunk(i, q, nq);
        e = cudaStreamWaitEvent(cs, P->ev_cin[s][q], 0);
        if (e == cudaSuccess)
          e = launch_rfft_x(P, din(s) + k.off, dout(s) + k.off, false, 1.0, cs,
                            (long long)(k.width / P->nx));
      }
      if (e == cudaSuccess) e = launch_fft_y(P, dout(s), false, cs);
      if (e == cudaSuccess) e = launch_thomas(P, dout(s), cs);
      if (e == cudaSuccess) e = launch_fft_y(P, dout(s), true, cs);
      for (int q = 0; q < nq && e == cudaSuccess; ++q) {
        const Chunk k = chunk(i, q, nq);
        e = launch_rfft_x(P, dout(s) + k.off, dout(s) + k.off, true, 1.0, cs,
                          (long long)(k.width / P->nx));
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_cdone[s][q], cs);
      }
    } else {  // Algorithm 2 by y-row ranges of columns
      HelmCoef* h = nullptr;
      r = helm_prepare(P, c[i], loc[i], P->pcr_parts, &h);
      for (int q = 0; q < nq && r == CFS_OK && e == cudaSuccess; ++q) {
        const Chunk k = chunk(i, q, nq);
        e = cudaStreamWaitEvent(cs, P->ev_cin[s][q], 0);
        if (e == cudaSuccess)
          e = launch_pcr_cols(P, *h, din(s), dout(s), (long long)k.off, (long long)k.width, cs);
        if (e == cudaSuccess) e = cudaEventRecord(P->ev_cdone[s][q], cs);
      }
    }
    if (r != CFS_OK && r != CFS_ENOTCONVERGED) {
      rc = r;
      break;
    }
    if (e != cudaSuccess) break;
    if (r == CFS_ENOTCONVERGED && rc == CFS_OK) rc = r;
    cudaStream_t os = ostream(i);
    e = cudaEventRecord(P->ev_done[s], cs);
    for (int q = 0; q < nq && e == cudaSuccess; ++q) {
      e = cudaStreamWaitEvent(os, P->ev_cdone[s][q], 0);
      if (e == cudaSuccess)
        e = copy(out[i], dout(s), chunk(i, q, nq), cudaMemcpyDeviceToHost, os);
    }
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_free[s], os);
  }
  // every copy has landed (or the work stops here) before returning
  cudaError_t ef = cudaSuccess;
  for (cudaStream_t q : {P->copy_in, P->compute2, P->copy_out, P->copy_out2, st})
    if (cudaStreamSynchronize(q) != cudaSuccess) ef = cudaErrorUnknown;
  if (rc != CFS_OK && rc != CFS_ENOTCONVERGED) return rc;
  if (e == cudaErrorInvalidValue) return CFS_EINVAL;
  if (e != cudaSuccess || ef != cudaSuccess) return CFS_ECUDA;
  return rc;
}

extern "C" int cfs_plan_check_guards(cfs_plan_t P, int* damaged) {
  if (!P) return CFS_EINVAL;
  CaptureLock lock(capture_mutex());
  if (cudaDeviceSynchronize() != cudaSuccess) return CFS_ECUDA;
  std::vector<uint32_t> got(kGuardBytes / sizeof(uint32_t));
  int bad = 0;
  for (const auto& g : P->guarded) {
    unsigned char* ends[2] = {g.first, g.first + kGuardBytes + g.second};
    bool ok = true;
    for (unsigned char* at : ends) {
      if (cudaMemcpy(got.data(), at, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CFS_ECUDA;
      for (uint32_t w : got) ok = ok && (w == kGuardWord);
    }
    bad += ok ? 0 : 1;
  }
  if (damaged) *damaged = bad;
  return bad ? CFS_EGUARD : CFS_OK;
}

extern "C" int cfs_plan_debug_guard_poke(cfs_plan_t P, int buffer, int tail) {
  if (!P || buffer < 0 || buffer >= (int)P->guarded.size()) return CFS_EINVAL;
  CaptureLock lock(capture_mutex());
  const auto& g = P->guarded[buffer];
  unsigned char* at = tail ? g.first + kGuardBytes + g.second : g.first + kGuardBytes - 1;
  return cudaMemset(at, 0x5A, 1) == cudaSuccess ? CFS_OK : CFS_ECUDA;
}

extern "C" int cfs_plan_check(cfs_plan_t P, int* device_error) {
  if (!P) return CFS_EINVAL;
  CaptureLock lock(capture_mutex());
  cudaError_t e = cudaDeviceSynchronize();
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&bits, P->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && bits) e = cudaMemset(P->d_status, 0, sizeof(int));
  if (device_error) *device_error = bits;
  if (e != cudaSuccess) return CFS_ECUDA;
  return (bits & kErrTmaTimeout) ? CFS_ETIMEOUT : CFS_OK;
}
