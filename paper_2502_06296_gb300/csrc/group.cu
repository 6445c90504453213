// group.cu -- grouped refined solves: the Poisson solves of several plans
// (boxes of different sizes, grids and walls) run together, every stage of
// the FP32 inner solve and of the FP64 refinement launched once for all boxes.
//
// Each box follows exactly the iteration of its own refined solve (the same
// kernels' arithmetic and block partition, the same stopping rule on its own
// tolerance and FP32-solve budget), so a box's result does not depend on the
// group it is solved in.  Boxes that converge drop out of the later stages
// through a device-side mask, and the iteration itself is driven from the
// device: a solve is one CUDA graph whose refinement loop is a conditional
// WHILE node; the kernel that closes an iteration sets the loop condition
// (any box still iterating?).  The host takes part only at the end, to read
// the iteration counts.  Graphs are keyed by launch shape and captured at a
// shape's second solve; other solves run the same launches directly with the
// loop on the host.
#include <stdint.h>
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
  size_t xf, xi, y, th, zp, res, sx, sy, sth, szp, sres, splane, sone, ssub, neu, bytes;
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
    zp = take(sizeof(ZPartArgs) * cap);
    res = take(sizeof(ResBox) * cap);
    sx = take(sizeof(int) * (cap + 1));
    sy = take(sizeof(int) * (cap + 1));
    sth = take(sizeof(int) * (cap + 1));
    szp = take(sizeof(int) * (cap + 1));
    sres = take(sizeof(int) * (cap + 1));
    splane = take(sizeof(int) * (cap + 1));
    sone = take(sizeof(int) * (cap + 1));
    ssub = take(sizeof(int) * (cap + 1));
    neu = take(sizeof(int) * cap);
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
  ThomasArgs* d_th = nullptr;  // streaming z sweeps
  ZPartArgs* d_zp = nullptr;    // partitioned z solves
  ResBox* d_res = nullptr;
  int *d_sx = nullptr, *d_sy = nullptr, *d_sth = nullptr, *d_szp = nullptr, *d_sres = nullptr;
  int *d_splane = nullptr, *d_sone = nullptr, *d_ssub = nullptr;
  int* d_neumann = nullptr;  // boxes whose operator has the constants as null space
  int tx = 0, ty = 0, tth = 0, tzp = 0, tres = 0, tplane = 0, tone = 0, tsub = 0;
  size_t smem_x = 0, smem_y = 0, smem_zp = 0;
  // refinement state
  int* d_active = nullptr;  // boxes still iterating
  int* d_mean = nullptr;    // boxes whose mean is removed (Neumann, nonzero rhs)
  int* d_one = nullptr;     // boxes on their first correction (p written at the end if they stop)
  int* d_zero = nullptr;    // boxes with a zero right-hand side (zero solution)
  int* d_elig = nullptr;    // Helmholtz: boxes that are refined (the others solve in FP64)
  GroupCtl* d_ctl = nullptr;
  double* d_fmax = nullptr;
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
  HThomasBox* d_hth = nullptr;  // boxes whose Helmholtz systems take Thomas sweeps
  HThomasBox* h_hth = nullptr;
  PcrRefineBox* d_fus = nullptr;  // boxes refined in one pass (FP32 Algorithm 2 on tiles)
  PcrRefineBox* h_fus = nullptr;
  int* d_sfus = nullptr;
  int* h_sfus = nullptr;
  unsigned int* d_fwords = nullptr;  // per such box: max|r|, max|rhs|, FP32 solves
  unsigned int* h_fwords = nullptr;
  int* h_fused = nullptr;
  int* d_sth32 = nullptr;  // block offsets: FP32 inner Thomas sweeps
  int* d_sth64 = nullptr;  // FP64 direct Thomas sweeps
  int* h_sth32 = nullptr;
  int* h_sth64 = nullptr;
  // pinned per-call staging: the copies of a solve (graph nodes included)
  // read these when they run
  double* h_tol = nullptr;
  int* h_maxit = nullptr;
  int* h_elig = nullptr;
  int* h_spcr = nullptr;
  int* h_spcr64 = nullptr;
  int* h_iters = nullptr;  // results, written by the solve's last copies
  double* h_rho = nullptr;
  GroupCtl* h_ctl = nullptr;
  // Graphs of solves, keyed by launch shape.  A graph's kernels read every
  // per-box record from the group's device tables, so a graph captured for
  // one binding serves any later binding with the same launch shape (number
  // of boxes, total blocks and shared memory of each stage).
  bool graphs = true;
  cudaStream_t cap_main = nullptr, cap_body = nullptr;
  struct Graph {
    std::vector<long long> sig;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> cache;  // least recently used first
  // launch shapes seen but not yet captured: a shape is captured at its
  // second solve, so that one-off shapes (a serving loop's varied batches)
  // run as direct launches and do not pay for a capture
  std::vector<std::vector<long long>> seen;
  cudaEvent_t io_copied = nullptr;  // staging buffers free again after this
  // Launch tracing (cfs_group_set_trace): while on, solves run as direct
  // launches with a pair of events around every copy and kernel they issue.
  bool trace = false;
  std::vector<cudaEvent_t> trace_ev;  // begin / end pairs, kTraceLaunches of them
  int trace_n = 0;                    // pairs recorded by the last solve
  std::vector<ResBox> res;          // host copy of the bound boxes' residual records
  std::vector<int> last_iters;
  std::vector<double> last_rho;
};

constexpr size_t kGraphCache = 128;  // graphs kept per group
constexpr size_t kSeenShapes = 512;  // uncaptured shapes remembered per group

static void drop_graphs(cfs_group* G) {
  for (auto& g : G->cache)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  G->cache.clear();
  G->seen.clear();
}

// The cached graph of launch shape `sig` (moved to the back), or null.
static cudaGraphExec_t find_graph(cfs_group* G, const std::vector<long long>& sig) {
  for (size_t i = 0; i < G->cache.size(); ++i)
    if (G->cache[i].sig == sig) {
      cfs_group::Graph g = G->cache[i];
      G->cache.erase(G->cache.begin() + (long)i);
      G->cache.push_back(g);
      return g.exec;
    }
  return nullptr;
}

// Whether a solve of launch shape `sig` should capture a graph: on the
// shape's second solve (the first runs as direct launches).
static bool capture_now(cfs_group* G, const std::vector<long long>& sig) {
  for (size_t i = 0; i < G->seen.size(); ++i)
    if (G->seen[i] == sig) {
      G->seen.erase(G->seen.begin() + (long)i);
      return true;
    }
  if (G->seen.size() >= kSeenShapes) G->seen.erase(G->seen.begin());
  G->seen.push_back(sig);
  return false;
}

static void keep_graph(cfs_group* G, const std::vector<long long>& sig, cudaGraphExec_t exec) {
  if (G->cache.size() >= kGraphCache) {
    cudaGraphExecDestroy(G->cache.front().exec);
    G->cache.erase(G->cache.begin());
  }
  G->cache.push_back({sig, exec});
}

constexpr int kTraceLaunches = 512;

// Runs f() (one copy or kernel launch on st), bracketed by a pair of trace
// events while tracing is on; launches past the pool run untraced.
template <class F>
static cudaError_t traced(cfs_group* G, cudaStream_t st, F&& f) {
  if (!G->trace || 2 * G->trace_n + 2 > (int)G->trace_ev.size()) return f();
  cudaError_t e = cudaEventRecord(G->trace_ev[2 * G->trace_n], st);
  if (e == cudaSuccess) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(G->trace_ev[2 * G->trace_n + 1], st);
  if (e == cudaSuccess) ++G->trace_n;
  return e;
}

static void group_free(cfs_group* G) {
  drop_graphs(G);
  for (cudaEvent_t ev : G->trace_ev) cudaEventDestroy(ev);
  void* ptrs[] = {G->d_tab,   G->d_active, G->d_mean, G->d_one, G->d_fmax, G->d_tol,  G->d_maxit,
                  G->d_iters, G->d_rho,    G->d_nactive, G->d_io, G->d_pcr, G->d_hres,
                  G->d_spcr, G->d_pcr64, G->d_spcr64, G->d_zero, G->d_elig, G->d_ctl,
                  G->d_hth, G->d_sth32, G->d_sth64, G->d_fus, G->d_sfus, G->d_fwords};
  for (void* p : ptrs) cudaFree(p);
  void* hptrs[] = {G->h_tol,   G->h_maxit, G->h_elig, G->h_spcr,  G->h_spcr64, G->h_iters,
                   G->h_rho,   G->h_ctl,   G->h_hth,  G->h_sth32, G->h_sth64,  G->h_fus,
                   G->h_sfus,  G->h_fwords, G->h_fused};
  for (void* p : hptrs)
    if (p) cudaFreeHost(p);
  if (G->cap_main) cudaStreamDestroy(G->cap_main);
  if (G->cap_body) cudaStreamDestroy(G->cap_body);
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
  if (e == cudaSuccess) e = cudaMalloc(&G->d_one, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_fmax, sizeof(double) * cap);
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
  if (e == cudaSuccess) e = cudaMalloc(&G->d_zero, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_elig, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_ctl, sizeof(GroupCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_tol, sizeof(double) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_maxit, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_elig, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_spcr, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_spcr64, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_iters, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_rho, sizeof(double) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_ctl, sizeof(GroupCtl));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_hth, sizeof(HThomasBox) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_hth, sizeof(HThomasBox) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_sth32, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_sth64, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_sth32, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_sth64, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_fus, sizeof(PcrRefineBox) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_fus, sizeof(PcrRefineBox) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&G->d_sfus, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_sfus, sizeof(int) * (cap + 1));
  if (e == cudaSuccess) e = cudaMalloc(&G->d_fwords, sizeof(unsigned int) * 3 * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_fwords, sizeof(unsigned int) * 3 * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&G->h_fused, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->cap_main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G->cap_body, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->io_copied, cudaEventDisableTiming);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CFS_ENOMEM : CFS_ECUDA;
  const GroupTables& t = G->tab;
  G->d_xf = reinterpret_cast<XBox*>(G->d_tab + t.xf);
  G->d_xi = reinterpret_cast<XBox*>(G->d_tab + t.xi);
  G->d_y = reinterpret_cast<YBox*>(G->d_tab + t.y);
  G->d_th = reinterpret_cast<ThomasArgs*>(G->d_tab + t.th);
  G->d_zp = reinterpret_cast<ZPartArgs*>(G->d_tab + t.zp);
  G->d_res = reinterpret_cast<ResBox*>(G->d_tab + t.res);
  G->d_sx = reinterpret_cast<int*>(G->d_tab + t.sx);
  G->d_sy = reinterpret_cast<int*>(G->d_tab + t.sy);
  G->d_sth = reinterpret_cast<int*>(G->d_tab + t.sth);
  G->d_szp = reinterpret_cast<int*>(G->d_tab + t.szp);
  G->d_sres = reinterpret_cast<int*>(G->d_tab + t.sres);
  G->d_splane = reinterpret_cast<int*>(G->d_tab + t.splane);
  G->d_sone = reinterpret_cast<int*>(G->d_tab + t.sone);
  G->d_ssub = reinterpret_cast<int*>(G->d_tab + t.ssub);
  G->d_neumann = reinterpret_cast<int*>(G->d_tab + t.neu);
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
  ZPartArgs* zp = reinterpret_cast<ZPartArgs*>(G->h_tab + t.zp);
  ResBox* res = reinterpret_cast<ResBox*>(G->h_tab + t.res);
  std::vector<int> bx(nplans), by(nplans), bth(nplans), bzp(nplans, 0), bres(nplans),
      bplane(nplans), bone(nplans, 1), bsub(nplans);
  G->plans.clear();
  G->neumann.clear();
  G->res.assign(nplans, ResBox{});
  G->smem_x = G->smem_y = G->smem_zp = 0;
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
    if (zpart_group_member(P)) {  // the z solve its plan takes alone
      G->smem_zp = std::max(G->smem_zp, zpart_group_box(P, &zp[b], &bzp[b]));
      bth[b] = 0;
    }
    const long long nxy = (long long)P->nx * P->ny;
    ResBox& r = res[b];
    memset(&r, 0, sizeof(r));
    r.dzf = P->d_dzf;
    r.partial = P->d_red + 3;
    r.mean = P->d_red + 1;
    r.r32 = P->d_r32;
    r.r32b = P->d_r32b;
    r.rlo = P->d_rlo;
    r.dcopy = P->d_w2;
    r.zk = P->d_zk;
    r.rmax = reinterpret_cast<unsigned int*>(P->d_red);
    r.nx = P->nx;
    r.ny = P->ny;
    r.nz = P->nz;
    r.n = P->nz;
    const double dx = P->lx / P->nx, dy = P->ly / P->ny;
    r.neumann = P->has_null;
    r.ybc = P->ybc;
    r.mpart = P->d_mpart;
    r.mnum = P->d_red + 2;
    r.inv_wn = P->inv_wn;
    G->res[b] = r;
    bres[b] = (int)((nxy + 127) / 128);
    bplane[b] = P->nz * start_chunks(P->nz);
    bsub[b] = (int)group_sub_blocks(nxy * P->nz);
  }
  auto put = [&](size_t at, const std::vector<int>& v) {
    memcpy(G->h_tab + at, v.data(), sizeof(int) * v.size());
  };
  put(t.sx, offsets(bx, &G->tx));
  put(t.sy, offsets(by, &G->ty));
  put(t.sth, offsets(bth, &G->tth));
  put(t.szp, offsets(bzp, &G->tzp));
  put(t.sres, offsets(bres, &G->tres));
  put(t.splane, offsets(bplane, &G->tplane));
  put(t.sone, offsets(bone, &G->tone));
  put(t.ssub, offsets(bsub, &G->tsub));
  put(t.neu, G->neumann);
  cudaError_t e = cudaMemcpyAsync(G->d_tab, G->h_tab, t.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e != cudaSuccess) return CFS_ECUDA;
  G->nbox = nplans;
  G->last_iters.assign(nplans, 0);
  G->last_rho.assign(nplans, 0.0);
  return CFS_OK;
}

extern "C" int cfs_group_create(cfs_group_t* out, int nplans, const cfs_plan_t* plans) {
  CaptureLock lock(capture_mutex());
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
  CaptureLock lock(capture_mutex());
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
  CaptureLock lock(capture_mutex());
  if (!G) return CFS_EINVAL;
  cudaDeviceSynchronize();
  group_free(G);
  return CFS_OK;
}

static int rc_of(cudaError_t e) { return e == cudaSuccess ? CFS_OK : CFS_ECUDA; }

// Fields are read and written by 16-byte bulk copies and vector loads.
static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

namespace {

constexpr cudaMemcpyKind kH2D = cudaMemcpyHostToDevice;
constexpr cudaMemcpyKind kD2H = cudaMemcpyDeviceToHost;

// Builds and instantiates the graph of one solve: head() (the stages up to
// the loop), a WHILE node whose body is one loop iteration, then tail().
// The kernels that close an iteration set the node's condition through
// `cond`; it is 0 at each launch until the head sets it.
template <class Head, class Body, class Tail>
cudaError_t build_graph(cfs_group* G, Head head, Body body, Tail tail, cudaGraphExec_t* out) {
  CaptureLock lock(capture_mutex());
  *out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle cond = 0;
  e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault);
  bool capturing = false;
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(G->cap_main, graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  capturing = e == cudaSuccess;
  if (e == cudaSuccess) e = head(G->cap_main, cond);
  // the loop node after everything captured so far
  cudaGraphNode_t loop = nullptr;
  cudaGraph_t loop_body = nullptr;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus status;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(G->cap_main, &status, nullptr, &cg, &deps, nullptr, &ndeps);
    if (e == cudaSuccess && status != cudaStreamCaptureStatusActive) e = cudaErrorStreamCaptureInvalidated;
    if (e == cudaSuccess) {
      cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
      np.conditional.handle = cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&loop, cg, deps, nullptr, ndeps, &np);
      if (e == cudaSuccess) loop_body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(G->cap_main, &loop, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
  }
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(G->cap_body, loop_body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      const cudaError_t eb = body(G->cap_body, cond);
      cudaGraph_t ended = nullptr;
      e = cudaStreamEndCapture(G->cap_body, &ended);
      if (eb != cudaSuccess) e = eb;
    }
  }
  if (e == cudaSuccess) e = tail(G->cap_main);
  if (capturing) {
    cudaGraph_t ended = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(G->cap_main, &ended);
    if (e == cudaSuccess) e = ee;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    cudaGetLastError();
  }
  return e;
}

// ---- Poisson: stages of one grouped solve --------------------------------

// Copies of the call's pointers and settings, the start pass (r_0 = f as
// FP32, its extremes, the plane sums of Neumann boxes), the dz-weighted mean
// of f (Neumann boxes), the reference norms and the start state, and the
// zero solution of boxes whose right-hand side is zero.
cudaError_t poisson_head(cfs_group* G, cudaStream_t st) {
  const int nb = G->nbox;
  cudaError_t e = traced(G, st, [&] {
    return cudaMemcpyAsync(G->d_io, G->h_io, sizeof(GroupIo) * nb, kH2D, st);
  });
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return cudaMemcpyAsync(G->d_tol, G->h_tol, sizeof(double) * nb, kH2D, st);
    });
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return cudaMemcpyAsync(G->d_maxit, G->h_maxit, sizeof(int) * nb, kH2D, st);
    });
  if (e == cudaSuccess) e = traced(G, st, [&] { return launch_group_zero_max(G->d_res, nb, st); });
  GroupMap g{G->d_splane, nullptr, nb};
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_refine_stage(GSTAGE_START, G->d_res, g, G->tplane, G->d_io, 0, st);
    });
  g = GroupMap{G->d_sone, G->d_neumann, nb};
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_refine_stage(GSTAGE_MEAN_FINAL, G->d_res, g, G->tone, G->d_io, 0, st);
    });
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_start(G->d_res, nb, 1, G->d_fmax, nullptr, G->d_active, G->d_mean,
                                G->d_zero, G->d_iters, G->d_rho, G->d_ctl, st, G->d_one);
    });
  g = GroupMap{G->d_ssub, G->d_zero, nb};
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_refine_stage(GSTAGE_ZERO, G->d_res, g, G->tsub, G->d_io, 0, st);
    });
  return e;
}

// One iteration: FP32 solve of the current residual, correction of p, new
// residual, stopping test.  kind 0: the first (the correction stays in FP32,
// first residual by differences); kind 1: the second (p = both corrections,
// double-float residual update); kind 2: the later ones (p += delta; as 1,
// the FP32 right-hand side read from r32b).
cudaError_t poisson_iteration(cfs_group* G, int kind, cudaGraphConditionalHandle cond,
                              int set_cond, cudaStream_t st) {
  const int nb = G->nbox;
  GroupMap g{G->d_sx, G->d_active, nb};
  cudaError_t e = traced(G, st, [&] {
    return launch_rfft_x_group32(G->d_xf, g, G->tx, G->smem_x, false, OUT_SAME, G->d_io,
                                 kind >= 1, st);
  });
  if (e == cudaSuccess) {
    g.start = G->d_sy;
    e = traced(G, st, [&] { return launch_fft_y_group32(G->d_y, g, G->ty, G->smem_y, false, st); });
  }
  if (e == cudaSuccess) {
    g.start = G->d_sth;
    e = traced(G, st, [&] { return launch_thomas_group32(G->d_th, g, G->tth, st); });
  }
  if (e == cudaSuccess) {
    g.start = G->d_szp;
    e = traced(G, st, [&] { return launch_zpart_group(G->d_zp, g, G->tzp, G->smem_zp, st); });
  }
  if (e == cudaSuccess) {
    g.start = G->d_sy;
    e = traced(G, st, [&] { return launch_fft_y_group32(G->d_y, g, G->ty, G->smem_y, true, st); });
  }
  if (e == cudaSuccess) {
    g.start = G->d_sx;
    // the first correction stays in FP32; the second pass writes p = both;
    // later passes add to p
    e = traced(G, st, [&] {
      return launch_rfft_x_group32(G->d_xi, g, G->tx, G->smem_x, true,
                                   kind == 0 ? OUT_SAME : kind == 1 ? OUT_SUM : OUT_ADD, G->d_io, 0,
                                   st);
    });
  }
  if (e == cudaSuccess) {
    g.start = G->d_sres;
    e = traced(G, st, [&] {
      return launch_group_refine_stage(kind == 0 ? GSTAGE_RESIDUAL : GSTAGE_UPDATE, G->d_res, g,
                                       G->tres, G->d_io, 1, st);
    });
  }
  if (e == cudaSuccess) {  // the weighted sum of p, correction by correction (Neumann boxes)
    g.start = G->d_sone;
    e = traced(G, st, [&] {
      return launch_group_refine_stage(GSTAGE_MEAN_ACC, G->d_res, g, G->tone, G->d_io, 0, st);
    });
  }
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_iter_end(G->d_res, nb, G->d_fmax, G->d_tol, G->d_maxit, G->d_active,
                                   G->d_mean, G->d_iters, G->d_rho, G->d_ctl, cond, set_cond, st,
                                   G->d_one);
    });
  return e;
}

// Boxes that stopped after one FP32 solve: p from that correction, less the
// solution's dz-weighted mean for Neumann boxes (from the running weighted
// sum of the corrections), as the single solve does; then the iteration
// counts and residuals copied out.
cudaError_t poisson_tail(cfs_group* G, cudaStream_t st) {
  const int nb = G->nbox;
  GroupMap g{G->d_sone, G->d_mean, nb};
  cudaError_t e =
      launch_group_refine_stage(GSTAGE_MEAN_FROM_NUM, G->d_res, g, G->tone, G->d_io, 0, st);
  g = GroupMap{G->d_ssub, G->d_one, nb};
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return launch_group_refine_stage(GSTAGE_FIRST_ONLY, G->d_res, g, G->tsub, G->d_io, 0, st);
    });
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return cudaMemcpyAsync(G->h_iters, G->d_iters, sizeof(int) * nb, kD2H, st);
    });
  if (e == cudaSuccess)
    e = traced(G, st, [&] {
      return cudaMemcpyAsync(G->h_rho, G->d_rho, sizeof(double) * nb, kD2H, st);
    });
  return e;
}

// Host-side loop: reads the count of boxes still iterating after each one.
cudaError_t read_nactive(cfs_group* G, cudaStream_t st, int* nactive) {
  cudaError_t e = cudaMemcpyAsync(G->h_ctl, G->d_ctl, sizeof(GroupCtl), kD2H, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *nactive = e == cudaSuccess ? G->h_ctl->nactive : 0;
  return e;
}

// Results of a finished solve (h_iters, h_rho) into the group and plans.
int finish(cfs_group* G, const int* skip) {
  int rc = CFS_OK;
  for (int b = 0; b < G->nbox; ++b) {
    G->last_iters[b] = G->h_iters[b];
    G->last_rho[b] = G->h_rho[b];
    G->plans[b]->last_iters = G->h_iters[b];
    G->plans[b]->last_rho = G->h_rho[b];
    if (skip && skip[b]) continue;
    if (!(G->h_rho[b] <= G->plans[b]->tol)) rc = CFS_ENOTCONVERGED;
  }
  return rc;
}

}  // namespace

extern "C" int cfs_group_poisson_solve(cfs_group_t G, const double* const* f, double* const* p,
                                       void* stream) {
  if (!G || !f || !p || G->nbox < 1) return CFS_EINVAL;
  const int nb = G->nbox;
  for (int b = 0; b < nb; ++b)
    if (!f[b] || !p[b] || static_cast<const void*>(f[b]) == static_cast<const void*>(p[b]) ||
        !aligned16(f[b]) || !aligned16(p[b]))
      return CFS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the staging buffers of the previous call must have been read
  cudaError_t e = cudaEventSynchronize(G->io_copied);
  if (e != cudaSuccess) return CFS_ECUDA;
  for (int b = 0; b < nb; ++b) {
    G->h_io[b] = GroupIo{f[b], p[b]};
    G->h_tol[b] = G->plans[b]->tol;
    G->h_maxit[b] = G->plans[b]->maxit;
  }
  G->trace_n = 0;
  const std::vector<long long> sig = {0,       nb,      G->tx,     G->ty,
                                      G->tth,  G->tzp,  G->tres,   G->tplane,
                                      G->tone, G->tsub, (long long)G->smem_x,
                                      (long long)G->smem_y, (long long)G->smem_zp};
  const bool graphs = G->graphs && !G->trace;
  cudaGraphExec_t exec = graphs ? find_graph(G, sig) : nullptr;
  if (exec || (graphs && capture_now(G, sig))) {
    if (!exec) {
      e = build_graph(
          G,
          [&](cudaStream_t s, cudaGraphConditionalHandle c) {
            cudaError_t r = poisson_head(G, s);
            if (r == cudaSuccess) r = poisson_iteration(G, 0, c, 1, s);
            if (r == cudaSuccess) r = poisson_iteration(G, 1, c, 1, s);
            return r;
          },
          [&](cudaStream_t s, cudaGraphConditionalHandle c) {
            return poisson_iteration(G, 2, c, 1, s);
          },
          [&](cudaStream_t s) { return poisson_tail(G, s); }, &exec);
      if (e != cudaSuccess) return CFS_ECUDA;
      keep_graph(G, sig, exec);
    }
    e = cudaGraphLaunch(exec, st);
  } else {
    e = poisson_head(G, st);
    int nactive = 0;
    if (e == cudaSuccess) e = poisson_iteration(G, 0, 0, 0, st);
    if (e == cudaSuccess) e = read_nactive(G, st, &nactive);
    for (int kind = 1; nactive > 0 && e == cudaSuccess; kind = 2) {
      e = poisson_iteration(G, kind, 0, 0, st);
      if (e == cudaSuccess) e = read_nactive(G, st, &nactive);
    }
    if (e == cudaSuccess) e = poisson_tail(G, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rc_of(e);
  return finish(G, nullptr);
}

// End of a grouped Helmholtz call whose work was issued on st with status e.
static int finish_helm(cfs_group* G, cudaError_t e, cudaStream_t st) {
  if (e == cudaSuccess) e = cudaEventRecord(G->io_copied, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rc_of(e);
  std::vector<int> fp64(G->nbox);
  for (int b = 0; b < G->nbox; ++b) {
    fp64[b] = !G->h_elig[b] && !G->h_fused[b];
    if (G->h_fused[b]) {  // refined in one pass: the words its tiles left
      const unsigned int* w = G->h_fwords + 3 * b;
      float rmax, amax;
      memcpy(&rmax, &w[0], sizeof(float));
      memcpy(&amax, &w[1], sizeof(float));
      G->h_iters[b] = (int)w[2];
      G->h_rho[b] = amax > 0.0f ? (double)rmax / (double)amax : 0.0;
    }
  }
  return finish(G, fp64.data());
}

extern "C" int cfs_group_helmholtz_solve(cfs_group_t G, const double* c, const int* loc,
                                         const double* const* rhs, double* const* u,
                                         void* stream) {
  if (!G || !c || !loc || !rhs || !u || G->nbox < 1) return CFS_EINVAL;
  const int nb = G->nbox;
  for (int b = 0; b < nb; ++b)
    if (!rhs[b] || !u[b] || static_cast<const void*>(rhs[b]) == static_cast<const void*>(u[b]) ||
        !aligned16(rhs[b]) || !aligned16(u[b]))
      return CFS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventSynchronize(G->io_copied);  // staging of the previous call is free
  if (e != cudaSuccess) return CFS_ECUDA;
  G->trace_n = 0;
  // Algorithm 2, Step 1 of every box (host, cached per plan), and the
  // per-call descriptors.  Boxes whose plans take FP64 Algorithm 2 directly
  // (CFS_OPT_HELM_FP64) run in one FP64 launch; the others are refined
  // together.
  std::vector<int> blocks(nb, 0), blocks64(nb, 0), bt32(nb, 0), bt64(nb, 0), bfus(nb, 0);
  int threads = 0, threads64 = 0, threads_f = 0, nref = 0, rows_f = 0;
  size_t smem = 0, smem64 = 0, smem_t32 = 0, smem_t64 = 0, smem_f = 0;
  // boxes refined in one pass share one kernel instance: the most rows per
  // thread any of them needs; a box with more threads than that instance
  // allows takes the loop instead
  std::vector<HelmCoef*> hs(nb, nullptr);
  for (int b = 0; b < nb; ++b) {
    cfs_plan* P = G->plans[b];
    int rc = plan_helm_prepare(P, c[b], loc[b], 0, &hs[b]);
    if (rc) return rc;
    if (!P->helm_fp64 && pcr_refine_fits(P, *hs[b]))
      rows_f = std::max(rows_f, pcr_refine_rows(*hs[b]));
  }
  for (int b = 0; b < nb; ++b) {
    cfs_plan* P = G->plans[b];
    HelmCoef* h = hs[b];
    int th = 0;
    G->h_elig[b] = !P->helm_fp64;
    G->h_fused[b] = G->h_elig[b] && pcr_refine_fits(P, *h) &&
                    kPcrTileColumns * h->nparts <= pcr_refine_thread_limit(rows_f);
    if (G->h_fused[b]) G->h_elig[b] = 0;  // refined in one pass, outside the loop
    nref += G->h_elig[b];
    memset(&G->h_hth[b], 0, sizeof(HThomasBox));
    if (G->h_fused[b]) {
      int rows_b = 0;
      const size_t sm = pcr_refine_group_box(P, *h, rhs[b], u[b], G->d_fwords + 3 * b,
                                             &G->h_fus[b], &bfus[b], &th, &rows_b);
      if (!sm) return CFS_ECUDA;
      threads_f = std::max(threads_f, th);
      smem_f = std::max(smem_f, sm);
    } else if (G->h_elig[b] && P->helm_thomas32) {
      smem_t32 = std::max(smem_t32, helm_thomas_group_box(P, *h, true, &G->h_hth[b], &bt32[b]));
    } else if (G->h_elig[b]) {
      const size_t sm = pcr_group_box(P, *h, &G->h_pcr[b], &blocks[b], &th);
      if (!sm) return CFS_ECUDA;
      threads = std::max(threads, th);
      smem = std::max(smem, sm);
    } else if (P->helm_thomas) {
      smem_t64 = std::max(smem_t64, helm_thomas_group_box(P, *h, false, &G->h_hth[b], &bt64[b]));
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
    G->h_tol[b] = P->tol;
    G->h_maxit[b] = P->maxit;
  }
  int tpcr = 0, tpcr64 = 0, tt32 = 0, tt64 = 0, tfus = 0;
  const std::vector<int> sfus = offsets(bfus, &tfus);
  memcpy(G->h_sfus, sfus.data(), sizeof(int) * (nb + 1));
  const std::vector<int> spcr = offsets(blocks, &tpcr), spcr64 = offsets(blocks64, &tpcr64);
  const std::vector<int> st32 = offsets(bt32, &tt32), st64 = offsets(bt64, &tt64);
  memcpy(G->h_spcr, spcr.data(), sizeof(int) * (nb + 1));
  memcpy(G->h_spcr64, spcr64.data(), sizeof(int) * (nb + 1));
  memcpy(G->h_sth32, st32.data(), sizeof(int) * (nb + 1));
  memcpy(G->h_sth64, st64.data(), sizeof(int) * (nb + 1));

  auto head = [&](cudaStream_t s) {
    cudaError_t r = traced(G, s, [&] {
      return cudaMemcpyAsync(G->d_pcr, G->h_pcr, sizeof(PcrBox) * nb, kH2D, s);
    });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_hres, G->h_hres, sizeof(ResBox) * nb, kH2D, s);
      });
    if (r == cudaSuccess && tpcr64 > 0)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_pcr64, G->h_pcr64, sizeof(PcrBox64) * nb, kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_io, G->h_io, sizeof(GroupIo) * nb, kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_spcr, G->h_spcr, sizeof(int) * (nb + 1), kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_spcr64, G->h_spcr64, sizeof(int) * (nb + 1), kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_tol, G->h_tol, sizeof(double) * nb, kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_maxit, G->h_maxit, sizeof(int) * nb, kH2D, s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_elig, G->h_elig, sizeof(int) * nb, kH2D, s);
      });
    if (r == cudaSuccess && tt32 + tt64 > 0) {
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_hth, G->h_hth, sizeof(HThomasBox) * nb, kH2D, s);
      });
      if (r == cudaSuccess)
        r = traced(G, s, [&] {
          return cudaMemcpyAsync(G->d_sth32, G->h_sth32, sizeof(int) * (nb + 1), kH2D, s);
        });
      if (r == cudaSuccess)
        r = traced(G, s, [&] {
          return cudaMemcpyAsync(G->d_sth64, G->h_sth64, sizeof(int) * (nb + 1), kH2D, s);
        });
    }
    // the boxes refined in one pass: one launch, the result words copied out
    if (r == cudaSuccess && tfus > 0)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_fus, G->h_fus, sizeof(PcrRefineBox) * nb, kH2D, s);
      });
    if (r == cudaSuccess && tfus > 0)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->d_sfus, G->h_sfus, sizeof(int) * (nb + 1), kH2D, s);
      });
    if (r == cudaSuccess && tfus > 0)
      r = traced(G, s, [&] {
        return cudaMemsetAsync(G->d_fwords, 0, sizeof(unsigned int) * 3 * nb, s);
      });
    if (r == cudaSuccess && tfus > 0)
      r = traced(G, s, [&] {
        return launch_pcr_refine_group(G->d_fus, GroupMap{G->d_sfus, nullptr, nb}, tfus, threads_f,
                                       smem_f, rows_f, s);
      });
    if (r == cudaSuccess && tfus > 0)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->h_fwords, G->d_fwords, sizeof(unsigned int) * 3 * nb, kD2H, s);
      });
    // the FP64 boxes: one launch per method, no refinement
    if (r == cudaSuccess && tpcr64 > 0)
      r = traced(G, s, [&] {
        return launch_pcr_group64(G->d_pcr64, GroupMap{G->d_spcr64, nullptr, nb}, tpcr64, threads64,
                                  smem64, s);
      });
    if (r == cudaSuccess && tt64 > 0)
      r = traced(G, s, [&] {
        return launch_helm_thomas_group(G->d_hth, GroupMap{G->d_sth64, nullptr, nb}, tt64, smem_t64,
                                        false, G->d_io, s);
      });
    if (nref == 0) return r;
    // r_0 = rhs and its max-norm (refined boxes), the start state, zero
    // solutions of zero right-hand sides
    GroupMap g{G->d_sres, G->d_elig, nb};
    if (r == cudaSuccess) r = traced(G, s, [&] { return launch_group_zero_max(G->d_hres, nb, s); });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_group_refine_stage(GSTAGE_HELM_RESIDUAL, G->d_hres, g, G->tres, G->d_io, 0,
                                         s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_group_start(G->d_hres, nb, 0, G->d_fmax, G->d_elig, G->d_active, nullptr,
                                  G->d_zero, G->d_iters, G->d_rho, G->d_ctl, s);
      });
    g = GroupMap{G->d_ssub, G->d_zero, nb};
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_group_refine_stage(GSTAGE_ZERO, G->d_hres, g, G->tsub, G->d_io, 0, s);
      });
    return r;
  };
  // one iteration: FP32 Algorithm 2 on the residual, u updated, new residual
  // (mode 1: u = delta, 2: u += delta), stopping test
  auto iteration = [&](int mode, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s) {
    GroupMap g{G->d_spcr, G->d_active, nb};
    cudaError_t r = traced(G, s, [&] {
      return launch_pcr_group32(G->d_pcr, g, tpcr, threads, smem, s);
    });
    g.start = G->d_sth32;
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_helm_thomas_group(G->d_hth, g, tt32, smem_t32, true, G->d_io, s);
      });
    g.start = G->d_sres;
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_group_refine_stage(GSTAGE_HELM_RESIDUAL, G->d_hres, g, G->tres, G->d_io, mode,
                                         s);
      });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return launch_group_iter_end(G->d_hres, nb, G->d_fmax, G->d_tol, G->d_maxit, G->d_active,
                                     nullptr, G->d_iters, G->d_rho, G->d_ctl, cond, set_cond, s);
      });
    return r;
  };
  auto tail = [&](cudaStream_t s) {
    cudaError_t r = traced(G, s, [&] {
      return cudaMemcpyAsync(G->h_iters, G->d_iters, sizeof(int) * nb, kD2H, s);
    });
    if (r == cudaSuccess)
      r = traced(G, s, [&] {
        return cudaMemcpyAsync(G->h_rho, G->d_rho, sizeof(double) * nb, kD2H, s);
      });
    return r;
  };

  if (nref == 0) {  // no box needs the refinement loop (FP64 or one-pass boxes)
    e = head(st);
    for (int b = 0; b < nb; ++b) {
      G->h_iters[b] = 0;
      G->h_rho[b] = 0.0;
    }
    return finish_helm(G, e, st);
  }
  const std::vector<long long> sig = {1,        nb,       tpcr,
                                      tpcr64,   threads,  threads64,
                                      (long long)smem,    (long long)smem64,
                                      tt32,     tt64,     (long long)smem_t32,
                                      (long long)smem_t64, G->tres, G->tsub,
                                      tfus,     threads_f, (long long)smem_f, rows_f};
  const bool graphs = G->graphs && !G->trace;
  cudaGraphExec_t exec = graphs ? find_graph(G, sig) : nullptr;
  if (exec || (graphs && capture_now(G, sig))) {
    if (!exec) {
      e = build_graph(
          G,
          [&](cudaStream_t s, cudaGraphConditionalHandle cnd) {
            cudaError_t r = head(s);
            if (r == cudaSuccess) r = iteration(1, cnd, 1, s);
            return r;
          },
          [&](cudaStream_t s, cudaGraphConditionalHandle cnd) { return iteration(2, cnd, 1, s); },
          tail, &exec);
      if (e != cudaSuccess) return CFS_ECUDA;
      keep_graph(G, sig, exec);
    }
    e = cudaGraphLaunch(exec, st);
  } else {
    e = head(st);
    int nactive = 0;
    if (e == cudaSuccess) e = iteration(1, 0, 0, st);
    if (e == cudaSuccess) e = read_nactive(G, st, &nactive);
    while (nactive > 0 && e == cudaSuccess) {
      e = iteration(2, 0, 0, st);
      if (e == cudaSuccess) e = read_nactive(G, st, &nactive);
    }
    if (e == cudaSuccess) e = tail(st);
  }
  return finish_helm(G, e, st);
}

extern "C" int cfs_group_set_graphs(cfs_group_t G, int on) {
  if (!G) return CFS_EINVAL;
  G->graphs = on != 0;
  return CFS_OK;
}

extern "C" int cfs_group_set_trace(cfs_group_t G, int on) {
  if (!G) return CFS_EINVAL;
  if (on && G->trace_ev.empty()) {
    G->trace_ev.assign(2 * kTraceLaunches, nullptr);
    for (cudaEvent_t& ev : G->trace_ev) {
      if (cudaEventCreate(&ev) != cudaSuccess) {
        for (cudaEvent_t& x : G->trace_ev)
          if (x) cudaEventDestroy(x);
        G->trace_ev.clear();
        return CFS_ECUDA;
      }
    }
  }
  G->trace = on != 0;
  G->trace_n = 0;
  return CFS_OK;
}

extern "C" int cfs_group_trace(cfs_group_t G, float* ms, int capacity, int* count) {
  if (!G || !count || capacity < 0 || (capacity > 0 && !ms)) return CFS_EINVAL;
  *count = G->trace_n;
  for (int i = 0; i < G->trace_n && i < capacity; ++i) {
    cudaError_t e = cudaEventSynchronize(G->trace_ev[2 * i + 1]);
    if (e == cudaSuccess)
      e = cudaEventElapsedTime(&ms[i], G->trace_ev[2 * i], G->trace_ev[2 * i + 1]);
    if (e != cudaSuccess) return CFS_ECUDA;
  }
  return CFS_OK;
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
