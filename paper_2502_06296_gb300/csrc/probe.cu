// probe.cu -- cfs_probe_fma: the FMA issue rate of this GPU, measured.
//
// The FP64 path of the solver is bound by FP64 instructions (GB300 has two
// FP64 FMA lanes per SM per clock against 128 FP32 lanes), so its roofline
// peak is the FP64 FMA rate.  This diagnostic (no counterpart in the paper)
// measures it, or the FP32 rate: every thread of a grid of one full wave
// runs kChains independent FMA recurrences for `iters` steps, timed by CUDA
// events; rate = threads x kChains x iters / time.
#include <stdlib.h>

#include "chanfs_f64emu.cuh"
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

// ----------------------------------------------------------------------------
// The integer-unit FP64 additions (chanfs_f64emu.cuh) against the FP64
// pipe's.  Sample i is a pair of operands drawn by a splitmix64 hash of i, of
// one of eight kinds: any two bit patterns (every exponent, zeros,
// subnormals, infinities, NaNs); exponents at most 3 apart; exponent
// differences 0..70 (the alignment shift and its sticky bit); operands equal
// up to their last 16 bits, of either sign (cancellation); few significant
// bits (exact ties of the rounding); the ends of the integer path's exponent
// range; equal magnitudes (zero results); and values of FFT-like size.
// ----------------------------------------------------------------------------
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline void addsub_sample(uint64_t i, double* a, double* b) {
  const uint64_t z = mix64((2 * i + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t w = mix64((2 * i + 2) * 0x9E3779B97F4A7C15ull);
  const uint64_t keep = 0x800FFFFFFFFFFFFFull;  // sign and fraction
  uint64_t ua = z, ub = w;
  switch (i % 8) {
    case 0:
      break;
    case 1: {
      const uint64_t e = 64 + (z >> 52) % 1982, d = (w >> 58) % 4;
      ua = (z & keep) | (e << 52);
      ub = (w & keep) | ((e >= 64 + d ? e - d : e) << 52);
      break;
    }
    case 2: {
      const uint64_t e = 200 + (z >> 52) % 1700, d = (w >> 57) % 71;
      ua = (z & keep) | (e << 52);
      ub = (w & keep) | ((e - d) << 52);
      break;
    }
    case 3: {
      const uint64_t e = 64 + (z >> 52) % 1982;
      ua = (z & keep) | (e << 52);
      ub = (ua ^ (w & 0xFFFFull)) ^ (((w >> 20) & 1ull) << 63);
      break;
    }
    case 4: {
      const uint64_t e = 1000 + (z >> 52) % 50, d = (w >> 57) % 60;
      ua = (z & kEmuSign) | (e << 52) | (z & 0x000FFF0000000000ull);
      ub = (w & kEmuSign) | ((e - d) << 52) | (w & 0x000FF00000000000ull);
      break;
    }
    case 5: {
      const uint64_t e1 = (z >> 63) ? 2045 : 64, e2 = (w >> 63) ? 2045 : 64 + (w >> 40) % 3;
      ua = (z & keep) | (e1 << 52);
      ub = (w & keep) | (e2 << 52);
      break;
    }
    case 6:
      ub = (w & 1ull) ? (z ^ kEmuSign) : z;
      break;
    default: {  // |a| ~ 1, |b| within 2^-20 .. 2^20 of it
      const uint64_t e = 1023 - 2 + (z >> 60) % 4, d = (w >> 58) % 41;
      ua = (z & keep) | (e << 52);
      ub = (w & keep) | ((e + d - 20) << 52);
      break;
    }
  }
  *a = emu_double(ua);
  *b = emu_double(ub);
}

// Equal encodings, or both NaN (the NaN payload is not specified).
__host__ __device__ inline bool same_bits(double x, double y) {
  return emu_bits(x) == emu_bits(y) || (x != x && y != y);
}

__host__ __device__ inline int addsub_mismatch(uint64_t i) {
  double a, b, s, d;
  addsub_sample(i, &a, &b);
  f64_addsub(a, b, s, d);
  const volatile double va = a, vb = b;  // the hardware's sum and difference
  return !same_bits(s, va + vb) + !same_bits(d, va - vb);
}

__global__ void addsub_check_kernel(unsigned long long n, unsigned long long* bad) {
  unsigned long long local = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    local += addsub_mismatch(i);
  if (local) atomicAdd(bad, local);
}

// Throughput of butterfly pairs (x, y) <- (x + y, x - y): on the FP64 pipe
// (EMU false) or by f64_addsub.  Each pair step grows the values by about
// sqrt 2; every 256 steps the exponents are lowered by 128 with an integer
// subtraction, so they stay in the integer path's range.
template <bool EMU>
__global__ void __launch_bounds__(kProbeThreads) addsub_probe_kernel(long long iters) {
  double x[kChains / 2], y[kChains / 2];
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) {
    x[j] = 1.0 + (threadIdx.x + j) * 1e-3;
    y[j] = 0.75 - j * 1e-2;
  }
  for (long long i = 0; i < iters; i += 256) {
#pragma unroll 4
    for (int t = 0; t < 256; ++t) {
#pragma unroll
      for (int j = 0; j < kChains / 2; ++j) {
        double s, d;
        if (EMU) {
          f64_addsub(x[j], y[j], s, d);
        } else {
          s = x[j] + y[j];
          d = x[j] - y[j];
        }
        x[j] = s;
        y[j] = d;
      }
    }
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) {
      x[j] = emu_double(emu_bits(x[j]) - (128ull << 52));
      y[j] = emu_double(emu_bits(y[j]) - (128ull << 52));
    }
  }
  double sum = 0;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) sum += x[j] + y[j];
  if (sum == -12345.0) g_probe_sink = sum;
}

static int probe_addsub(bool emu, long long iters, double* pairs_per_s, double* ms_out) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CFS_ECUDA;
  auto kern = emu ? addsub_probe_kernel<true> : addsub_probe_kernel<false>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kProbeThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return CFS_ECUDA;
  const int blocks = nsm * (per_sm < kProbeBlocksPerSm ? per_sm : kProbeBlocksPerSm);
  iters = (iters + 255) / 256 * 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    kern<<<blocks, kProbeThreads>>>(256);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    kern<<<blocks, kProbeThreads>>>(iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return CFS_ECUDA;
  *pairs_per_s = (double)blocks * kProbeThreads * (kChains / 2) * (double)iters / (ms * 1e-3);
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

extern "C" int cfs_selfcheck_f64_addsub(unsigned long long samples, int on_device,
                                        unsigned long long* mismatches) {
  if (!mismatches || samples == 0 || (on_device != 0 && on_device != 1)) return CFS_EINVAL;
  if (!on_device) {
    unsigned long long bad = 0;
    for (unsigned long long i = 0; i < samples; ++i) bad += chanfs::addsub_mismatch(i);
    *mismatches = bad;
    return CFS_OK;
  }
  chanfs::CaptureLock lock(chanfs::capture_mutex());
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    chanfs::addsub_check_kernel<<<1216, 256>>>(samples, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(mismatches, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? CFS_OK : CFS_ECUDA;
}

extern "C" int cfs_f64_addsub_host(long long n, const double* a, const double* b, double* s,
                                   double* d) {
  if (n < 0 || (n > 0 && (!a || !b || !s || !d))) return CFS_EINVAL;
  for (long long i = 0; i < n; ++i) chanfs::f64_addsub(a[i], b[i], s[i], d[i]);
  return CFS_OK;
}

extern "C" int cfs_probe_addsub(int on_integer_units, long long iters, double* pairs_per_s,
                                double* ms) {
  if (!pairs_per_s || iters < 1 || iters > (1ll << 40) ||
      (on_integer_units != 0 && on_integer_units != 1))
    return CFS_EINVAL;
  chanfs::CaptureLock lock(chanfs::capture_mutex());
  return chanfs::probe_addsub(on_integer_units != 0, iters, pairs_per_s, ms);
}
