// probe.cu -- cfs_probe_fma: the FMA issue rate of this GPU, measured.
//
// The FP64 path of the solver is bound by FP64 instructions (GB300 has two
// FP64 FMA lanes per SM per clock against 128 FP32 lanes), so its roofline
// peak is the FP64 FMA rate.  This diagnostic (no counterpart in the paper)
// measures it, or the FP32 rate: every thread of a grid of one full wave
// runs kChains independent FMA recurrences for `iters` steps, timed by CUDA
// events; rate = threads x kChains x iters / time.
#include "chanfs_tma.cuh"

namespace chanfs {

constexpr int kChains = 16;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

__device__ double g_probe_sink;

// x_j <- x_j * a_j + b per chain; each a_j (slightly below 1, in a register:
// operands from the constant bank are not what the solver's FMAs read) and a
// small b keep every value finite and normal for any iteration count.  The
// sum is written only if it equals a value it cannot reach, so no chain can
// be dropped as dead code.
template <class R>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(long long iters, R a, R b) {
  R x[kChains], m[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    x[j] = R(threadIdx.x + j) * R(1e-3);
    m[j] = a - R(j) * R(1e-9) * R(threadIdx.x & 1);
  }
  const R c = b * R(1 + (threadIdx.x & 1));
#pragma unroll 4
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], m[j], c);
  }
  R s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == R(-1)) g_probe_sink = (double)s;  // never true: the values stay positive
}

template <class R>
static int probe(long long iters, double* fma_per_s, double* ms_out) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CFS_ECUDA;
  // one full wave: as many blocks per SM as fit (at most kProbeBlocksPerSm)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<R>, kProbeThreads,
                                                    0) != cudaSuccess ||
      per_sm < 1)
    return CFS_ECUDA;
  const int blocks = nsm * (per_sm < kProbeBlocksPerSm ? per_sm : kProbeBlocksPerSm);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // warm-up (clocks ramp up, the module loads), then the timed launch
  if (e == cudaSuccess) {
    fma_probe_kernel<R><<<blocks, kProbeThreads>>>(iters / 8 + 1, R(0.999999), R(1e-7));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    fma_probe_kernel<R><<<blocks, kProbeThreads>>>(iters, R(0.999999), R(1e-7));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return CFS_ECUDA;
  *fma_per_s = (double)blocks * kProbeThreads * kChains * (double)iters / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return CFS_OK;
}

// The failure path of the kernels' bounded waits, made to run: each CTA
// arms an mbarrier for `bytes` bytes that no copy will deliver (none is
// issued, so nothing is in flight when the CTA leaves) and waits through
// cta_wait, the helper every TMA-fed kernel uses, with `polls` polls.
__global__ void wait_timeout_kernel(int* status, uint32_t polls, uint32_t bytes) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, bytes);
  if (!cta_wait(&bar, 0, status, polls)) return;
  if (threadIdx.x == 0) atomicOr(status, 1 << 30);  // not reached: the phase cannot complete
}

}  // namespace chanfs

extern "C" int cfs_selftest_wait_timeout(cfs_plan_t plan, int* device_status, unsigned polls,
                                         void* stream) {
  if ((plan == nullptr) == (device_status == nullptr) || polls < 1 || polls > (1u << 20))
    return CFS_EINVAL;
  int* status = plan ? plan->d_status : device_status;
  chanfs::wait_timeout_kernel<<<4, 128, 0, (cudaStream_t)stream>>>(status, polls, 4096);
  return cudaGetLastError() == cudaSuccess ? CFS_OK : CFS_ECUDA;
}

extern "C" int cfs_probe_fma(int bits, long long iters, double* fma_per_s, double* ms) {
  if (!fma_per_s || iters < 1 || iters > (1ll << 40) || (bits != 64 && bits != 32))
    return CFS_EINVAL;
  chanfs::CaptureLock lock(chanfs::capture_mutex());
  return bits == 64 ? chanfs::probe<double>(iters, fma_per_s, ms)
                    : chanfs::probe<float>(iters, fma_per_s, ms);
}
