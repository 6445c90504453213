// group.cu -- grouped refined solves: the Poisson solves of several plans
// (boxes of different sizes, grids and walls) run together, every stage of
// the FP32 inner solve and of the FP64 refinement launched once for all boxes.
//
// Each box follows exactly the iteration of its own refined solve (the same
// kernels' arithmetic and block partition, the same stopping rule on its own
// tolerance and FP32-solve budget), so a box's result does not depend on the
// group it is solved in.  Boxes that converge drop out of the later stages
// through a device-side mask; the host reads one word per iteration (are any
// boxes still iterating?) instead of one per box.
#include <string.h>

#include <algorithm>
#include <vector>

#include "chanfs_group.cuh"

using namespace chanfs;

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * src.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
  return e;
}

// Block offsets of a grouped launch from per-box block counts.
std::vector<int> offsets(const std::vector<int>& blocks, int* total) {
  std::vector<int> start(blocks.size() + 1, 0);
  for (size_t b = 0; b < blocks.size(); ++b) start[b + 1] = start[b] + blocks[b];
  *total = start.back();
  return start;
}

}  // namespace

// Descriptor tables of a bound group, at fixed offsets of one device buffer
// (and of its pinned host staging copy) sized for the group's capacity.
struct GroupTables {
  size_t xf, xi, y, th, res, sx, sy, sth, sres, splane, sone, ssub, bytes;
  explicit GroupTables(int cap) {
    size_t o = 0;
    auto take = [&](size_t n) {
      const size_t at = o;
      o += (n + 255) / 256 * 256;
      return at;
    };
    xf = take(sizeof(XBox) * cap);
    xi = take(sizeof(XBox) * cap);
    y = take(sizeof(YBox) * cap);
    th = take(sizeof(ThomasArgs) * cap);
    res = take(sizeof(ResBox) * cap);
    sx = take(sizeof(int) * (cap + 1));
    sy = take(sizeof(int) * (cap + 1));
    sth = take(sizeof(int) * (cap + 1));
    sres = take(sizeof(int) * (cap + 1));
    splane = take(sizeof(int) * (cap + 1));
    sone = take(sizeof(int) * (cap + 1));
    ssub = take(sizeof(int) * (cap + 1));
    bytes = o;
  }
};

struct cfs_group {
  int cap = 0;   // boxes the buffers hold
  int nbox = 0;  // boxes bound
  int device = 0;
  std::vector<cfs_plan*> plans;
  std::vector<int> neumann;
  GroupTables tab{1};
  unsigned char* d_tab = nullptr;
  unsigned char* h_tab = nullptr;  // pinned staging of the tables
  // per-kernel descriptors and block offsets (inside d_tab)
  XBox* d_xf = nullptr;
  XBox* d_xi = nullptr;
  YBox* d_y = nullptr;
  ThomasArgs* d_th = nullptr;
  ResBox* d_res = nullptr;
  int *d_sx = nullptr, *d_sy = nullptr, *d_sth = nullptr, *d_sres = nullptr;
  int *d_splane = nullptr, *d_sone = nullptr, *d_ssub = nullptr;
  int tx = 0, ty = 0, tth = 0, tres = 0, tplane = 0, tone = 0, tsub = 0;
  size_t smem_x = 0, smem_y = 0;
  // refinement state
  int* d_active = nullptr;  // boxes still iterating
  int* d_mean = nullptr;    // boxes whose mean is removed (Neumann, nonzero rhs)
  float* d_fmax = nullptr;
  double* d_tol = nullptr;
  int* d_maxit = nullptr;
  int* d_iters = nullptr;
  double* d_rho = nullptr;
  int* d_nactive = nullptr;
  GroupIo* d_io = nullptr;
  GroupIo* h_io = nullptr;  // pinned staging of the per-call pointers
  // Helmholtz: per-call Algorithm 2 and residual descriptors (c, loc vary)
  PcrBox* d_pcr = nullptr;
  PcrBox* h_pcr = nullptr;
  PcrBox64* d_pcr64 = nullptr;  // boxes whose plans solve Helmholtz in FP64 directly
  PcrBox64* h_pcr64 = nullptr;
  int* d_spcr64 = nullptr;
  ResBox* d_hres = nullptr;
  ResBox* h_hres = nullptr;
  int* d_spcr = nullptr;
  cudaEvent_t io_copied = nullptr;  // staging buffers free again after this
  std::vector<ResBox> res;          // host copy of the bound boxes' residual records
  std::vector<int> last_iters;
  std::vector<double> last_rho;
};

static void group_free(cfs_group* G) {
  void* ptrs[] = {G->d_tab,   G->d_active, G->d_mean, G->d_fmax, G->d_tol,  G->d_maxit,
                  G->d_iters, G->d_rho,    G->d_nactive, G->d_io, G->d_pcr, G->d_hres,
                  G->d_spcr, G->d_pcr64, G->d_spcr64};
  for (void* p : ptrs) cudaFree(p);
  if (G->h_pcr64) cudaFreeHost(G->h_pcr64);
  if (G->h_tab) cudaFreeHost(G->h_tab);
  if (G->h_io) cudaFreeHost(G->h_io);
  if (G->h_pcr) cudaFreeHost(G->h_pcr);
  if (G->h_hres) cudaFreeHost(G->h_hres);
  if (G->io_copied) cudaEventDestroy(G->io_copied);
  delete G;
}

static int group_alloc(cfs_group* G, int cap) {
  G->cap = cap;
  G->tab = GroupTables(cap);
  cudaError_t e = cudaMalloc(&G->d_tab, G->tab.bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_tab, G->tab.bytes);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_active, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_mean, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_fmax, sizeof(float) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_tol, sizeof(double) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_maxit, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_iters, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_rho, sizeof(double) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_nactive, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_io, sizeof(GroupIo) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_io, sizeof(GroupIo) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_pcr, sizeof(PcrBox) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_pcr, sizeof(PcrBox) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_hres, sizeof(ResBox) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_hres, sizeof(ResBox) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_spcr, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_pcr64, sizeof(PcrBox64) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_pcr64, sizeof(PcrBox64) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_spcr64, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->io_copied, cudaEventDisableTiming);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CFS_ENOMEM : CFS_ECUDA;
  const GroupTables& t = G->tab;
  G->d_xf = reinterpret_cast<XBox*>(G->d_tab + t.xf);
  G->d_xi = reinterpret_cast<XBox*>(G->d_tab + t.xi);
  G->d_y = reinterpret_cast<YBox*>(G->d_tab + t.y);
  G->d_th = reinterpret_cast<ThomasArgs*>(G->d_tab + t.th);
  G->d_res = reinterpret_cast<ResBox*>(G->d_tab + t.res);
  G->d_sx = reinterpret_cast<int*>(G->d_tab + t.sx);
  G->d_sy = reinterpret_cast<int*>(G->d_tab + t.sy);
  G->d_sth = reinterpret_cast<int*>(G->d_tab + t.sth);
  G->d_sres = reinterpret_cast<int*>(G->d_tab + t.sres);
  G->d_splane = reinterpret_cast<int*>(G->d_tab + t.splane);
  G->d_sone = reinterpret_cast<int*>(G->d_tab + t.sone);
  G->d_ssub = reinterpret_cast<int*>(G->d_tab + t.ssub);
  return CFS_OK;
}

static int check_plans(int nplans, const cfs_plan_t* plans, int dev) {
  for (int b = 0; b < nplans; ++b) {
    if (!plans[b]) return CFS_EINVAL;
    if (plans[b]->dtype != CFS_F32_REFINED || plans[b]->device != dev) return CFS_EUNSUPPORTED;
    for (int c = 0; c < b; ++c)
      if (plans[c] == plans[b]) return CFS_EINVAL;  // boxes share the plan's work field
  }
  return CFS_OK;
}

// Builds the descriptor tables of `plans` in the pinned staging buffer and
// copies them to the device on `st` (ordered before the solves on st).
static int group_bind(cfs_group* G, int nplans, const cfs_plan_t* plans, cudaStream_t st) {
  if (cudaEventSynchronize(G->io_copied) != cudaSuccess) return CFS_ECUDA;  // staging free
  const GroupTables& t = G->tab;
  XBox* xf = reinterpret_cast<XBox*>(G->h_tab + t.xf);
  XBox* xi = reinterpret_cast<XBox*>(G->h_tab + t.xi);
  YBox* y = reinterpret_cast<YBox*>(G->h_tab + t.y);
  ThomasArgs* th = reinterpret_cast<ThomasArgs*>(G->h_tab + t.th);
  ResBox* res = reinterpret_cast<ResBox*>(G->h_tab + t.res);
  std::vector<int> bx(nplans), by(nplans), bth(nplans), bres(nplans), bplane(nplans),
      bone(nplans, 1), bsub(nplans);
  G->plans.clear();
  G->neumann.clear();
  G->res.assign(nplans, ResBox{});
  G->smem_x = G->smem_y = 0;
  for (int b = 0; b < nplans; ++b) {
    cfs_plan* P = plans[b];
    G->plans.push_back(P);
    G->neumann.push_back(P->has_null);
    G->smem_x = std::max(G->smem_x, x_group_box(P, false, &xf[b], &bx[b]));
    x_group_box(P, true, &xi[b], &bx[b]);
    const size_t sy = y_group_box(P, &y[b], &by[b]);
    if (!sy) return CFS_ECUDA;
    G->smem_y = std::max(G->smem_y, sy);
    thomas_group_box(P, &th[b], &bth[b]);
    const long long nxy = (long long)P->nx * P->ny;
    ResBox& r = res[b];
    memset(&r, 0, sizeof(r));
    r.zop = P->d_zop;
    r.dzf = P->d_dzf;
    r.partial = P->d_red + 2;
    r.mean = P->d_red + 1;
    r.r32 = P->d_r32;
    r.r32b = P->d_r32b;
    r.rdf = P->d_rdf;
    r.zop2 = P->d_zop2;
    r.rmax = reinterpret_cast<unsigned int*>(P->d_red);
    r.nx = P->nx;
    r.ny = P->ny;
    r.nz = P->nz;
    r.n = P->nz;
    const double dx = P->lx / P->nx, dy = P->ly / P->ny;
    r.idx2 = 1.0 / (dx * dx);
    r.idy2 = 1.0 / (dy * dy);
    r.neumann = P->has_null;
    r.ybc = P->ybc;
    G->res[b] = r;
    bres[b] = (int)((nxy + 127) / 128);
    bplane[b] = P->nz;
    bsub[b] = (int)group_sub_blocks(nxy * P->nz);
  }
  auto put = [&](size_t at, const std::vector<int>& v) {
    memcpy(G->h_tab + at, v.data(), sizeof(int) * v.size());
  };
  put(t.sx, offsets(bx, &G->tx));
  put(t.sy, offsets(by, &G->ty));
  put(t.sth, offsets(bth, &G->tth));
  put(t.sres, offsets(bres, &G->tres));
  put(t.splane, offsets(bplane, &G->tplane));
  put(t.sone, offsets(bone, &G->tone));
  put(t.ssub, offsets(bsub, &G->tsub));
  cudaError_t e = cudaMemcpyAsync(G->d_tab, G->h_tab, t.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e != cudaSuccess) return CFS_ECUDA;
  G->nbox = nplans;
  G->last_iters.assign(nplans, 0);
  G->last_rho.assign(nplans, 0.0);
  return CFS_OK;
}

extern "C" int cfs_group_create(cfs_group_t* out, int nplans, const cfs_plan_t* plans) {
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (nplans < 1 || nplans > kMaxGroup || !plans) return CFS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CFS_ECUDA;
  int rc = check_plans(nplans, plans, dev);
  if (rc) return rc;
  cfs_group* G = new (std::nothrow) cfs_group();
  if (!G) return CFS_ENOMEM;
  G->device = dev;
  rc = group_alloc(G, nplans);
  if (!rc) rc = group_bind(G, nplans, plans, 0);
  if (!rc && cudaStreamSynchronize(0) != cudaSuccess) rc = CFS_ECUDA;
  if (rc) {
    group_free(G);
    return rc;
  }
  *out = G;
  return CFS_OK;
}

extern "C" int cfs_group_reserve(cfs_group_t* out, int capacity) {
  if (!out) return CFS_EINVAL;
  *out = nullptr;
  if (capacity < 1 || capacity > kMaxGroup) return CFS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CFS_ECUDA;
  cfs_group* G = new (std::nothrow) cfs_group();
  if (!G) return CFS_ENOMEM;
  G->device = dev;
  const int rc = group_alloc(G, capacity);
  if (rc) {
    group_free(G);
    return rc;
  }
  *out = G;
  return CFS_OK;
}

extern "C" int cfs_group_rebind(cfs_group_t G, int nplans, const cfs_plan_t* plans,
                                void* stream) {
  if (!G || !plans || nplans < 1) return CFS_EINVAL;
  if (nplans > G->cap) return CFS_EUNSUPPORTED;
  int rc = check_plans(nplans, plans, G->device);
  if (rc) return rc;
  return group_bind(G, nplans, plans, static_cast<cudaStream_t>(stream));
}

extern "C" int cfs_group_destroy(cfs_group_t G) {
  if (!G) return CFS_EINVAL;
  cudaDeviceSynchronize();
  group_free(G);
  return CFS_OK;
}

static int rc_of(cudaError_t e) { return e == cudaSuccess ? CFS_OK : CFS_ECUDA; }

extern "C" int cfs_group_poisson_solve(cfs_group_t G, const double* const* f, double* const* p,
                                       void* stream) {
  if (!G || !f || !p || G->nbox < 1) return CFS_EINVAL;
  const int nb = G->nbox;
  for (int b = 0; b < nb; ++b)
    if (!f[b] || !p[b] || static_cast<const void*>(f[b]) == static_cast<const void*>(p[b]))
      return CFS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the staging buffer of the previous call must have been copied
  cudaError_t e = cudaEventSynchronize(G->io_copied);
  for (int b = 0; b < nb && e == cudaSuccess; ++b) G->h_io[b] = GroupIo{f[b], p[b]};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_io, G->h_io, sizeof(GroupIo) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e != cudaSuccess) return CFS_ECUDA;

  // the plans' current refinement settings
  std::vector<double> tol(nb);
  std::vector<int> maxits(nb);
  for (int b = 0; b < nb; ++b) {
    tol[b] = G->plans[b]->tol;
    maxits[b] = G->plans[b]->maxit;
  }
  e = cudaMemcpyAsync(G->d_tol, tol.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_maxit, maxits.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return CFS_ECUDA;

  std::vector<int> on(nb), mean_on(nb);
  for (int b = 0; b < nb; ++b) mean_on[b] = G->neumann[b];
  const GroupMap all{nullptr, nullptr, nb};
  GroupMap g = all;
  // remove the dz-weighted mean of f (Neumann boxes)
  e = cudaMemcpyAsync(G->d_mean, mean_on.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    g.start = G->d_splane;
    g.active = G->d_mean;
    e = launch_group_refine_stage(GSTAGE_PLANE_SUM, G->d_res, g, G->tplane, G->d_io, 0, st);
  }
  if (e == cudaSuccess) {
    g.start = G->d_sone;
    e = launch_group_refine_stage(GSTAGE_MEAN_FINAL, G->d_res, g, G->tone, G->d_io, 0, st);
  }
  // r_0 = f - mean and its max-norm (the reference of each box)
  if (e == cudaSuccess) e = launch_group_zero_max(G->d_res, nb, st);
  if (e == cudaSuccess) {
    g.start = G->d_sres;
    g.active = nullptr;
    e = launch_group_refine_stage(GSTAGE_RESIDUAL, G->d_res, g, G->tres, G->d_io, 0, st);
  }
  if (e == cudaSuccess) e = launch_group_fmax(G->d_res, nb, G->d_fmax, st);
  std::vector<float> fmax(nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fmax.data(), G->d_fmax, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CFS_ECUDA;
  int nactive = 0;
  for (int b = 0; b < nb; ++b) {
    cfs_plan* P = G->plans[b];
    on[b] = fmax[b] != 0.0f;
    mean_on[b] = on[b] && G->neumann[b];
    nactive += on[b];
    G->last_iters[b] = 0;
    G->last_rho[b] = 0.0;
    if (!on[b])  // zero right-hand side: zero solution
      e = cudaMemsetAsync(p[b], 0, sizeof(double) * (size_t)P->nx * P->ny * P->nz, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_active, on.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_mean, mean_on.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  int maxit = 0;
  for (int b = 0; b < nb; ++b) maxit = std::max(maxit, G->plans[b]->maxit);
  g.active = G->d_active;
  for (int it = 0; it < maxit && nactive > 0 && e == cudaSuccess; ++it) {
    g.start = G->d_sx;
    e = launch_rfft_x_group32(G->d_xf, g, G->tx, G->smem_x, false, OUT_SAME, G->d_io, it >= 2,
                              st);
    if (e == cudaSuccess) {
      g.start = G->d_sy;
      e = launch_fft_y_group32(G->d_y, g, G->ty, G->smem_y, false, st);
    }
    if (e == cudaSuccess) {
      g.start = G->d_sth;
      e = launch_thomas_group32(G->d_th, g, G->tth, st);
    }
    if (e == cudaSuccess) {
      g.start = G->d_sy;
      e = launch_fft_y_group32(G->d_y, g, G->ty, G->smem_y, true, st);
    }
    if (e == cudaSuccess) {
      g.start = G->d_sx;
      e = launch_rfft_x_group32(G->d_xi, g, G->tx, G->smem_x, true, it > 0 ? OUT_ADD : OUT_SET,
                                G->d_io, 0, st);
    }
    if (e == cudaSuccess) {  // the first residual directly in FP64, then updates
      g.start = G->d_sres;
      e = launch_group_refine_stage(it == 0 ? GSTAGE_RESIDUAL : GSTAGE_UPDATE, G->d_res, g,
                                    G->tres, G->d_io, 1, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(G->d_nactive, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = launch_group_update(G->d_res, nb, G->d_fmax, G->d_tol, G->d_maxit, it, G->d_active,
                              G->d_iters, G->d_rho, G->d_nactive, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&nactive, G->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  // restore the zero dz-weighted mean of p (Neumann boxes), as the single solve does
  g.active = G->d_mean;
  if (e == cudaSuccess) {
    g.start = G->d_splane;
    e = launch_group_refine_stage(GSTAGE_PLANE_SUM, G->d_res, g, G->tplane, G->d_io, 1, st);
  }
  if (e == cudaSuccess) {
    g.start = G->d_sone;
    e = launch_group_refine_stage(GSTAGE_MEAN_FINAL, G->d_res, g, G->tone, G->d_io, 0, st);
  }
  if (e == cudaSuccess) {
    g.start = G->d_ssub;
    e = launch_group_refine_stage(GSTAGE_SUBTRACT, G->d_res, g, G->tsub, G->d_io, 0, st);
  }
  std::vector<int> iters(nb);
  std::vector<double> rho(nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(iters.data(), G->d_iters, sizeof(int) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rho.data(), G->d_rho, sizeof(double) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rc_of(e);
  int rc = CFS_OK;
  for (int b = 0; b < nb; ++b) {
    if (!on[b]) continue;
    G->last_iters[b] = iters[b];
    G->last_rho[b] = rho[b];
    G->plans[b]->last_iters = iters[b];
    G->plans[b]->last_rho = rho[b];
    if (!(rho[b] <= G->plans[b]->tol)) rc = CFS_ENOTCONVERGED;
  }
  return rc;
}

extern "C" int cfs_group_helmholtz_solve(cfs_group_t G, const double* c, const int* loc,
                                         const double* const* rhs, double* const* u,
                                         void* stream) {
  if (!G || !c || !loc || !rhs || !u || G->nbox < 1) return CFS_EINVAL;
  const int nb = G->nbox;
  for (int b = 0; b < nb; ++b)
    if (!rhs[b] || !u[b] || static_cast<const void*>(rhs[b]) == static_cast<const void*>(u[b]))
      return CFS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventSynchronize(G->io_copied);  // staging of the previous call is free
  if (e != cudaSuccess) return CFS_ECUDA;
  // Algorithm 2, Step 1 of every box (host, cached per plan), and the
  // per-call descriptors
  // Boxes whose plans take FP64 Algorithm 2 directly (CFS_OPT_HELM_FP64) run
  // in one FP64 launch; the others are refined together.
  std::vector<int> blocks(nb, 0), blocks64(nb, 0), on(nb, 0), refined(nb, 0);
  std::vector<double> tol(nb);
  std::vector<int> maxits(nb);
  int threads = 0, threads64 = 0, nref = 0;
  size_t smem = 0, smem64 = 0;
  for (int b = 0; b < nb; ++b) {
    cfs_plan* P = G->plans[b];
    HelmCoef* h = nullptr;
    int rc = plan_helm_prepare(P, c[b], loc[b], 0, &h);
    if (rc) return rc;
    int th = 0;
    refined[b] = !P->helm_fp64;
    nref += refined[b];
    if (refined[b]) {
      const size_t sm = pcr_group_box(P, *h, &G->h_pcr[b], &blocks[b], &th);
      if (!sm) return CFS_ECUDA;
      threads = std::max(threads, th);
      smem = std::max(smem, sm);
    } else {
      const size_t sm = pcr_group_box64(P, *h, rhs[b], u[b], &G->h_pcr64[b], &blocks64[b], &th);
      if (!sm) return CFS_ECUDA;
      threads64 = std::max(threads64, th);
      smem64 = std::max(smem64, sm);
    }
    G->h_hres[b] = G->res[b];
    G->h_hres[b].abc = h->d_abc;
    G->h_hres[b].n = h->n;
    G->h_io[b] = GroupIo{rhs[b], u[b]};
    tol[b] = P->tol;
    maxits[b] = P->maxit;
  }
  int tpcr = 0, tpcr64 = 0;
  std::vector<int> spcr = offsets(blocks, &tpcr), spcr64 = offsets(blocks64, &tpcr64);
  e = cudaMemcpyAsync(G->d_pcr, G->h_pcr, sizeof(PcrBox) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_hres, G->h_hres, sizeof(ResBox) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && tpcr64 > 0)
    e = cudaMemcpyAsync(G->d_pcr64, G->h_pcr64, sizeof(PcrBox64) * nb, cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_io, G->h_io, sizeof(GroupIo) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_spcr, spcr.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_spcr64, spcr64.data(), sizeof(int) * (nb + 1),
                        cudaMemcpyHostToDevice, st);
  // the FP64 boxes: one launch, no refinement
  if (e == cudaSuccess && tpcr64 > 0)
    e = launch_pcr_group64(G->d_pcr64, GroupMap{G->d_spcr64, nullptr, nb}, tpcr64, threads64,
                           smem64, st);
  for (int b = 0; b < nb; ++b)
    if (!refined[b]) {
      G->last_iters[b] = 0;
      G->last_rho[b] = 0.0;
      G->plans[b]->last_iters = 0;
      G->plans[b]->last_rho = 0.0;
    }
  if (nref == 0) return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_tol, tol.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_maxit, maxits.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  // r_0 = rhs and its max-norm (refined boxes)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_active, refined.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                        st);
  GroupMap g{G->d_sres, G->d_active, nb};
  if (e == cudaSuccess) e = launch_group_zero_max(G->d_hres, nb, st);
  if (e == cudaSuccess)
    e = launch_group_refine_stage(GSTAGE_HELM_RESIDUAL, G->d_hres, g, G->tres, G->d_io, 0, st);
  if (e == cudaSuccess) e = launch_group_fmax(G->d_hres, nb, G->d_fmax, st);
  std::vector<float> fmax(nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fmax.data(), G->d_fmax, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CFS_ECUDA;
  int nactive = 0, maxit = 0;
  for (int b = 0; b < nb; ++b) {
    if (!refined[b]) continue;
    cfs_plan* P = G->plans[b];
    on[b] = fmax[b] != 0.0f;
    nactive += on[b];
    maxit = std::max(maxit, P->maxit);
    G->last_iters[b] = 0;
    G->last_rho[b] = 0.0;
    if (!on[b])  // zero right-hand side: zero solution
      e = cudaMemsetAsync(u[b], 0, sizeof(double) * (size_t)P->nx * P->ny * P->nz, st);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G->d_active, on.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
  g.active = G->d_active;
  for (int it = 0; it < maxit && nactive > 0 && e == cudaSuccess; ++it) {
    g.start = G->d_spcr;
    e = launch_pcr_group32(G->d_pcr, g, tpcr, threads, smem, st);
    if (e == cudaSuccess) {
      g.start = G->d_sres;
      e = launch_group_refine_stage(GSTAGE_HELM_RESIDUAL, G->d_hres, g, G->tres, G->d_io,
                                    it == 0 ? 1 : 2, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(G->d_nactive, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = launch_group_update(G->d_hres, nb, G->d_fmax, G->d_tol, G->d_maxit, it, G->d_active,
                              G->d_iters, G->d_rho, G->d_nactive, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&nactive, G->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  std::vector<int> iters(nb);
  std::vector<double> rho(nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(iters.data(), G->d_iters, sizeof(int) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(rho.data(), G->d_rho, sizeof(double) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rc_of(e);
  int rc = CFS_OK;
  for (int b = 0; b < nb; ++b) {
    if (!on[b]) continue;
    G->last_iters[b] = iters[b];
    G->last_rho[b] = rho[b];
    G->plans[b]->last_iters = iters[b];
    G->plans[b]->last_rho = rho[b];
    if (!(rho[b] <= G->plans[b]->tol)) rc = CFS_ENOTCONVERGED;
  }
  return rc;
}

extern "C" int cfs_group_last_info(cfs_group_t G, int* iters, double* rel_residual) {
  if (!G) return CFS_EINVAL;
  for (int b = 0; b < G->nbox; ++b) {
    if (iters) iters[b] = G->last_iters[b];
    if (rel_residual) rel_residual[b] = G->last_rho[b];
  }
  return CFS_OK;
}

extern "C" int cfs_group_size(cfs_group_t G, int* nplans) {
  if (!G || !nplans) return CFS_EINVAL;
  *nplans = G->nbox;
  return CFS_OK;
}
