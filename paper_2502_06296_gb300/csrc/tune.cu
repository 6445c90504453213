// tune.cu -- per-size choice of kernel shapes by measurement.
//
// For one plan the tuner times, with CUDA events on the caller's stream, the
// candidates of each kernel-shape option (FFT radix plan, x-lines per CTA, y-tile width,
// Thomas sweep shape, Algorithm 2 partition count, Algorithm 2 or Thomas
// sweeps for the Helmholtz systems, refined or FP64 Helmholtz) on the plan's
// own work fields, and keeps the fastest of each.  The options do not interact through
// the arithmetic (each only reshapes one kernel's launch), so they are tuned
// one after the other.  Choices are remembered per process for the plan's
// (nx, ny, nz, dtype).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>

#include "chanfs_internal.cuh"

using namespace chanfs;

namespace {

struct Choice {
  int x_lines, y_tile, thomas, pcr_parts, helm_fp64, helm_thomas, helm_thomas32, radix;
};

std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, Choice> g_cache;

// Best of `reps` timings (after one warm-up) of fn() on st, in ms; a huge
// value if a launch fails.
template <class F>
float best_ms(cudaStream_t st, F fn, int reps = 3) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 1e30f;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return 1e30f;
  }
  float best = 1e30f;
  if (fn() == cudaSuccess) {
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(a, st);
      const cudaError_t e = fn();
      cudaEventRecord(b, st);
      float ms = 1e30f;
      if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
        break;
      if (ms < best) best = ms;
    }
  }
  cudaGetLastError();  // a failed candidate leaves no error behind
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

constexpr double kProbeC = 3.0517578125e-5;  // Helmholtz coefficient of the probes (2^-15)

}  // namespace

// Whether choice c can run on plan P (a choice read from a file may not).
static bool fits(const cfs_plan* P, const Choice& c) {
  const bool fp32 = (P->dtype == CFS_F32_REFINED);
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  if (c.x_lines < 1 || c.x_lines > 64 || x_smem_bytes(P, c.x_lines, cs) > 227 * 1024) return false;
  if (!y_tile_ok(P, c.y_tile, fp32)) return false;
  if (c.thomas != -1 && thomas_tile_width(P, fp32, c.thomas) != c.thomas) return false;
  if (c.pcr_parts < 0 || c.pcr_parts > kPcrMaxParts) return false;
  for (int n = P->nz - 1; c.pcr_parts > 0 && n <= P->nz; ++n)
    if (n / c.pcr_parts < 3 || pcr_smem_bytes(n, c.pcr_parts) > 227 * 1024) return false;
  if ((c.helm_fp64 | c.helm_thomas | c.helm_thomas32) & ~1) return false;
  if (c.helm_thomas32 && !fp32) return false;
  return c.radix == 4 || c.radix == 8;
}

static void apply(cfs_plan* P, const Choice& c) {
  plan_set_radix(P, c.radix);
  P->x_lines = c.x_lines;
  if (P->dtype == CFS_F32_REFINED) P->tk32 = c.y_tile;
  else P->tk = c.y_tile;
  P->thomas_tw = c.thomas;
  P->pcr_parts = c.pcr_parts;
  P->helm_fp64 = c.helm_fp64;
  P->helm_thomas = c.helm_thomas;
  P->helm_thomas32 = c.helm_thomas32;
}

extern "C" int cfs_plan_autotune(cfs_plan_t P, void* stream) {
  if (!P) return CFS_EINVAL;
  CaptureLock capture_lock(capture_mutex());
  const bool fp32 = (P->dtype == CFS_F32_REFINED);
  const auto key = std::make_tuple(P->nx, P->ny, P->nz, P->dtype);
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      if (fits(P, it->second)) {
        apply(P, it->second);
        return CFS_OK;
      }
      g_cache.erase(it);  // a loaded choice that does not fit this plan: time afresh
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool had_stage = P->d_stage != nullptr;
  int rc = plan_ensure_stage(P);
  if (rc) return rc;
  const size_t npts = (size_t)P->nx * P->ny * P->nz;
  if (cudaMemsetAsync(P->d_stage, 0, sizeof(double) * npts, st) != cudaSuccess) return CFS_ECUDA;
  if (fp32 && cudaMemsetAsync(P->d_r32, 0, sizeof(float) * npts, st) != cudaSuccess)
    return CFS_ECUDA;
  double* s64 = P->d_stage;
  float* s32 = P->d_r32;
  const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
  Choice best{};

  // radix plan of the x and y transforms (default tiles), all four passes
  {
    float tbest = 1e30f;
    best.radix = 8;
    for (int r : {8, 4}) {
      if (plan_set_radix(P, r) != CFS_OK) continue;
      const float t = best_ms(st, [&]() {
        cudaError_t e = fp32 ? launch_rfft_x32(P, s32, s32, false, st)
                             : launch_rfft_x(P, s64, s64, false, 1.0, st);
        if (e == cudaSuccess)
          e = fp32 ? launch_fft_y32(P, s32, false, st) : launch_fft_y(P, s64, false, st);
        if (e == cudaSuccess)
          e = fp32 ? launch_fft_y32(P, s32, true, st) : launch_fft_y(P, s64, true, st);
        if (e == cudaSuccess)
          e = fp32 ? launch_rfft_x32_to64(P, s32, s64, false, st)
                   : launch_rfft_x(P, s64, s64, true, 1.0, st);
        return e;
      });
      if (t < tbest) {
        tbest = t;
        best.radix = r;
      }
    }
    if (plan_set_radix(P, best.radix) != CFS_OK) return CFS_ECUDA;
  }
  // x-lines per CTA: forward and inverse x transform
  {
    float tbest = 1e30f;
    const long long nlines = (long long)P->ny * P->nz;
    for (int lines : {1, 2, 4, 8, 16, 32, 64}) {
      if (lines > nlines || x_smem_bytes(P, lines, cs) > 227 * 1024) continue;
      P->x_lines = lines;
      // the transforms of one refined solve (two forward, the inverse that
      // sets p and the one that adds to it), or of one FP64 solve
      const float t = best_ms(st, [&]() {
        cudaError_t e = fp32 ? launch_rfft_x32(P, s32, s32, false, st)
                             : launch_rfft_x(P, s64, s64, false, 1.0, st);
        if (e == cudaSuccess)
          e = fp32 ? launch_rfft_x32_to64(P, s32, s64, false, st)
                   : launch_rfft_x(P, s64, s64, true, 1.0, st);
        if (fp32 && e == cudaSuccess) e = launch_rfft_x32(P, s32, s32, false, st);
        if (fp32 && e == cudaSuccess) e = launch_rfft_x32_to64(P, s32, s64, true, st);
        return e;
      });
      if (t < tbest) {
        tbest = t;
        best.x_lines = lines;
      }
    }
    P->x_lines = best.x_lines;
  }
  // y-tile width: forward and inverse y transform
  {
    float tbest = 1e30f;
    int& tk = fp32 ? P->tk32 : P->tk;
    const int tk0 = tk;
    best.y_tile = tk0;
    for (int cand : {1, 2, 4, 8, 16, 32}) {
      if (!y_tile_ok(P, cand, fp32)) continue;
      tk = cand;
      const float t = best_ms(st, [&]() {
        cudaError_t e = fp32 ? launch_fft_y32(P, s32, false, st) : launch_fft_y(P, s64, false, st);
        if (e == cudaSuccess)
          e = fp32 ? launch_fft_y32(P, s32, true, st) : launch_fft_y(P, s64, true, st);
        return e;
      });
      if (t < tbest) {
        tbest = t;
        best.y_tile = cand;
      }
    }
    tk = best.y_tile;
  }
  // Thomas sweep shape
  {
    float tbest = 1e30f;
    best.thomas = -1;
    for (int cand : {-1, 1, 8, 16}) {
      if (thomas_tile_width(P, fp32, cand) != cand) continue;
      P->thomas_tw = cand;
      const float t = best_ms(st, [&]() {
        return fp32 ? launch_thomas32(P, s32, st) : launch_thomas(P, s64, st);
      });
      if (t < tbest) {
        tbest = t;
        best.thomas = cand;
      }
    }
    P->thomas_tw = best.thomas;
  }
  // Algorithm 2 partitions (centred field: n = nz unknowns)
  {
    float tbest = 1e30f;
    best.pcr_parts = 0;
    const int n = P->nz;
    for (int cand : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}) {
      if ((n - 1) / cand < 3 || n > kPcrMaxUnknowns || pcr_smem_bytes(n, cand) > 227 * 1024)
        continue;  // the face field has n - 1 unknowns
      HelmCoef* h = nullptr;
      if (plan_helm_prepare(P, kProbeC, CFS_LOC_CENTER, cand, &h) != CFS_OK) continue;
      const HelmCoef hc = *h;  // the cache may move while timing
      const float t = best_ms(st, [&]() {
        return fp32 ? launch_pcr32(P, hc, s32, s32, st) : launch_pcr(P, hc, s64, s64, st);
      });
      if (t < tbest) {
        tbest = t;
        best.pcr_parts = cand;
      }
    }
    plan_helm_forget(P, kProbeC);
  }
  // Helmholtz by Algorithm 2 (best partition count) or by Thomas sweeps: in
  // the plan's own arithmetic, and for refined plans also in FP64 (the FP64
  // direct solve of CFS_OPT_HELM_FP64)
  best.helm_thomas = best.helm_thomas32 = 0;
  float t_direct64 = 1e30f;
  {
    HelmCoef* h = nullptr;
    if (plan_helm_prepare(P, kProbeC, CFS_LOC_CENTER, best.pcr_parts, &h) == CFS_OK) {
      const HelmCoef hc = *h;
      const float tp64 = best_ms(st, [&]() { return launch_pcr(P, hc, s64, s64, st); });
      const float tt64 = best_ms(st, [&]() { return launch_helm_thomas(P, hc, s64, s64, st); });
      best.helm_thomas = tt64 < tp64;
      t_direct64 = std::min(tp64, tt64);
    }
    plan_helm_forget(P, kProbeC);
  }
  // Refined plans: the whole refined Helmholtz solve with Algorithm 2 inner
  // solves (one pass over the field where a tile fits in shared memory) and
  // with Thomas inner solves, against the FP64 direct solve (all three meet
  // the refinement target), on a constant right-hand side
  best.helm_fp64 = 0;
  if (fp32 && P->nz <= kPcrMaxUnknowns) {
    double* u = nullptr;
    HelmCoef* h = nullptr;
    if (cudaMalloc(&u, sizeof(double) * npts) == cudaSuccess &&
        cudaMemsetAsync(s64, 0x3f, sizeof(double) * npts, st) == cudaSuccess &&
        plan_helm_prepare(P, kProbeC, CFS_LOC_CENTER, best.pcr_parts, &h) == CFS_OK) {
      const HelmCoef hc = *h;
      float t32[2] = {1e30f, 1e30f};
      for (int th = 0; th < 2; ++th) {
        P->helm_thomas32 = th;
        t32[th] = best_ms(st, [&]() {
          return refine_helmholtz(P, hc, s64, u, st) == CFS_OK ? cudaSuccess : cudaErrorUnknown;
        });
      }
      best.helm_thomas32 = t32[1] < t32[0];
      best.helm_fp64 = t_direct64 < std::min(t32[0], t32[1]);
    }
    cudaStreamSynchronize(st);
    cudaFree(u);
    plan_helm_forget(P, kProbeC);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return CFS_ECUDA;
  if (!had_stage) {  // the scratch field was the tuner's own
    cudaFree(P->d_stage);
    P->d_stage = nullptr;
    P->device_bytes -= sizeof(double) * npts;
  }
  apply(P, best);
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache[key] = best;
  return CFS_OK;
}

// ---- remembered choices across processes ---------------------------------

// The current device's name with blanks replaced (one token of a line).
static bool device_name(std::string* out) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return false;
  std::string n(prop.name);
  for (char& ch : n)
    if (ch == ' ' || ch == '\t') ch = '_';
  *out = n.empty() ? std::string("unknown") : n;
  return true;
}

static const char kTuneTag[] = "chanfs-tune-1";

extern "C" int cfs_autotune_save(const char* path) {
  if (!path) return CFS_EINVAL;
  std::string name;
  if (!device_name(&name)) return CFS_ECUDA;
  FILE* fp = fopen(path, "w");
  if (!fp) return CFS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  bool ok = true;
  for (const auto& kv : g_cache) {
    const Choice& c = kv.second;
    ok = ok && fprintf(fp, "%s %s %d %d %d %d %d %d %d %d %d %d %d %d\n", kTuneTag, name.c_str(),
                       std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                       std::get<3>(kv.first), c.x_lines, c.y_tile, c.thomas, c.pcr_parts,
                       c.helm_fp64, c.helm_thomas, c.helm_thomas32, c.radix) > 0;
  }
  ok = (fclose(fp) == 0) && ok;
  return ok ? CFS_OK : CFS_EINVAL;
}

extern "C" int cfs_autotune_load(const char* path, int* loaded) {
  if (loaded) *loaded = 0;
  if (!path) return CFS_EINVAL;
  FILE* fp = fopen(path, "r");
  if (!fp) return CFS_EINVAL;
  std::string name;
  if (!device_name(&name)) {
    fclose(fp);
    return CFS_ECUDA;
  }
  int rc = CFS_OK, taken = 0;
  char line[512];
  while (fgets(line, sizeof(line), fp)) {
    char tag[32], gpu[256];
    int nx, ny, nz, dtype;
    Choice c{};
    if (line[0] == '\n' || line[0] == '#') continue;
    if (sscanf(line, "%31s %255s %d %d %d %d %d %d %d %d %d %d %d %d", tag, gpu, &nx, &ny, &nz,
               &dtype, &c.x_lines, &c.y_tile, &c.thomas, &c.pcr_parts, &c.helm_fp64,
               &c.helm_thomas, &c.helm_thomas32, &c.radix) != 14 ||
        strcmp(tag, kTuneTag) != 0) {
      rc = CFS_EINVAL;
      break;
    }
    if (name != gpu) continue;  // measured on another kind of GPU
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_cache.emplace(std::make_tuple(nx, ny, nz, dtype), c).second) ++taken;
  }
  fclose(fp);
  if (loaded) *loaded = taken;
  return rc;
}

extern "C" int cfs_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
  return CFS_OK;
}
