// fft_y.cu -- complex FFT along y on TMA-staged tiles.
//
// The spectrum after the x transform is M complex columns per (y, z) line,
// i.e. a (Nz, Ny, M) complex array with M fastest.  One CTA takes `tk`
// consecutive columns of one z plane: a tk x Ny tile that the Tensor Memory
// Accelerator copies into shared memory as one or more 2-D boxes (rows of
// tk complex values, so every global read is a contiguous 16*tk-byte run and
// no transpose pass exists).  The tile is transformed in place along y by
// Stockham passes with the columns as batches, and written back by TMA.
// Out-of-range columns of a ragged last tile are zero-filled on load and
// clipped on store by the TMA unit.
#include "chanfs_fft.cuh"

namespace chanfs {

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait on phase `parity`; returns false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

template <bool INV, class C>
__global__ void __launch_bounds__(128) fft_y_kernel(const __grid_constant__ CUtensorMap map,
                                                    FftDesc d, const C* __restrict__ twg,
                                                    int tk, int by, int nbox, int* status) {
  using T = typename cscal<C>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  C* buf1 = buf0 + tk * d.n;
  C* tw = buf1 + tk * d.n;
  const int x0 = 2 * tk * blockIdx.x;  // in reals: a 16-byte aligned coordinate
  const int z = blockIdx.y;

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)(nbox * by * tk * sizeof(C)));
    for (int b = 0; b < nbox; ++b) tma_load_3d(buf0 + b * by * tk, &map, bar, x0, b * by, z);
  }
  for (int e = threadIdx.x; e < d.ntw; e += blockDim.x) tw[e] = twg[e];
  // every thread waits (bounded); the CTA then agrees on one outcome, which
  // also publishes the twiddles
  const int ok = __syncthreads_and(mbar_wait(bar, 0) ? 1 : 0);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, kErrTmaTimeout);
    return;  // no pass ran; nothing is stored
  }
  const int ny = d.n;
  // Column kx = 0 of the first tile is the packed pair F(0,ky) + i F(Nx/2,ky)
  // (App. A).  Its y spectrum is stored untangled, App. A's packing applied
  // once more along y: slot ky (0 < 2ky < Ny) holds F(0,ky), slot Ny-ky holds
  // F(Nx/2,ky), and the self-conjugate slots (ky = 0, Ny/2) keep the real pair
  // F(0,ky) + i F(Nx/2,ky).  Every slot is then one column of Eq. 12.
  if (INV && blockIdx.x == 0) {  // re-tangle before the inverse transform
    for (int ky = 1 + threadIdx.x; 2 * ky < ny; ky += blockDim.x) {
      const C f0 = buf0[ky * tk], fm = buf0[(ny - ky) * tk];
      buf0[ky * tk] = mkc<C>(f0.x - fm.y, f0.y + fm.x);         // F0 + i FM
      buf0[(ny - ky) * tk] = mkc<C>(f0.x + fm.y, fm.x - f0.y);  // conj F0 + i conj FM
    }
    __syncthreads();
  }
  // element (y, c) of the tile sits at y*tk + c: element stride tk, batch stride 1
  C* res = stockham_smem<INV, true>(buf0, buf1, d, tk, tk, 1, tw);
  if (!INV && blockIdx.x == 0) {  // untangle after the forward transform
    for (int ky = 1 + threadIdx.x; 2 * ky < ny; ky += blockDim.x) {
      const C zz = res[ky * tk], zm = res[(ny - ky) * tk];
      // F0 = (Z + conj Zm)/2,  FM = -i (Z - conj Zm)/2
      const T h = T(0.5);
      res[ky * tk] = mkc<C>(h * (zz.x + zm.x), h * (zz.y - zm.y));
      res[(ny - ky) * tk] = mkc<C>(h * (zz.y + zm.y), h * (zm.x - zz.x));
    }
    __syncthreads();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_3d(&map, res + b * by * tk, x0, b * by, z);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <class C>
static cudaError_t launch_y(const cfs_plan* P, void* data, bool inverse, int tk, const C* tw,
                            cudaStream_t st) {
  if (P->ny == 1) return cudaSuccess;  // length-1 transform is the identity
  EncodeTiledFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  using T = typename cscal<C>::T;
  CUtensorMap map;
  cuuint64_t gdim[3] = {(cuuint64_t)(2 * P->M), (cuuint64_t)P->ny, (cuuint64_t)P->nz};
  cuuint64_t gstride[2] = {(cuuint64_t)(2 * P->M) * sizeof(T),
                           (cuuint64_t)(2 * P->M) * P->ny * sizeof(T)};
  cuuint32_t box[3] = {(cuuint32_t)(2 * tk), (cuuint32_t)P->by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt =
      sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(&map, dt, 3, data, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = 128 + sizeof(C) * (size_t)(2 * tk * P->ny + P->fy.ntw);
  dim3 grid((P->M + tk - 1) / tk, P->nz);
  if (!inverse) {
    auto k = fft_y_kernel<false, C>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, 128, smem, st>>>(map, P->fy, tw, tk, P->by, P->nbox, P->d_status);
  } else {
    auto k = fft_y_kernel<true, C>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<grid, 128, smem, st>>>(map, P->fy, tw, tk, P->by, P->nbox, P->d_status);
  }
  return cudaGetLastError();
}

cudaError_t launch_fft_y(const cfs_plan* P, double* data, bool inverse, cudaStream_t st) {
  return launch_y<double2>(P, data, inverse, P->tk, P->d_twy, st);
}

cudaError_t launch_fft_y32(const cfs_plan* P, float* data, bool inverse, cudaStream_t st) {
  return launch_y<float2>(P, data, inverse, P->tk32, P->d_twy32, st);
}

}  // namespace chanfs
