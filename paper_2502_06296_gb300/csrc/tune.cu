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
#include <string.h>

#include <algorithm>
#include <map>
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
      apply(P, it->second);
      return CFS_OK;
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
    for (int cand : {-1, 8, 16}) {
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
      if (fp32) {
        const float tp32 = best_ms(st, [&]() { return launch_pcr32(P, hc, s32, s32, st); });
        const float tt32 =
            best_ms(st, [&]() { return launch_helm_thomas32(P, hc, s32, s32, st); });
        best.helm_thomas32 = tt32 < tp32;
      }
    }
    plan_helm_forget(P, kProbeC);
  }
  // Refined plans: refined Helmholtz against the FP64 direct solve (both meet
  // the refinement target), on a constant right-hand side
  best.helm_fp64 = 0;
  if (fp32 && P->nz <= kPcrMaxUnknowns) {
    double* u = nullptr;
    HelmCoef* h = nullptr;
    P->helm_thomas32 = best.helm_thomas32;
    if (cudaMalloc(&u, sizeof(double) * npts) == cudaSuccess &&
        cudaMemsetAsync(s64, 0x3f, sizeof(double) * npts, st) == cudaSuccess &&
        plan_helm_prepare(P, kProbeC, CFS_LOC_CENTER, best.pcr_parts, &h) == CFS_OK) {
      const HelmCoef hc = *h;
      const float t32 = best_ms(st, [&]() {
        return refine_helmholtz(P, hc, s64, u, st) == CFS_OK ? cudaSuccess : cudaErrorUnknown;
      });
      best.helm_fp64 = t_direct64 < t32;
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
