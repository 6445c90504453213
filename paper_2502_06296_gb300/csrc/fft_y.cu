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
#include "chanfs_tma.cuh"
#include "chanfs_group.cuh"

namespace chanfs {

// Walls in y (Sec. 2.2.1 names cosine / sine transforms for non-periodic
// directions).  A column of N values is transformed by DCT-II (Neumann walls)
// or DST-II (Dirichlet walls) through one complex FFT of length N:
//   v_n = x_{2n}, v_{N-1-n} = x_{2n+1}   (even samples up, odd samples down)
//   V = FFT(v),  X_k = (w_k V_k + conj(w_k) V_{N-k}) / 2,  w_k = exp(-i pi k / 2N)
// which holds for complex columns because the transform is real-linear.  The
// inverse recovers V_k = conj(w_k) (X_k - i X_{N-k}) (V_0 = X_0), transforms
// back and undoes the reordering; like the FFT it returns N times the column.
// DST-II is DCT-II of (-1)^j x_j with the output order reversed.
enum { Y_FFT = 0, Y_DCT = 1, Y_DST = 2 };

// Elements of one y-tile buffer: tk x n values (FP32 tiles: with room for
// the padded layout of stockham_fixed_cols) rounded up to 128 bytes.
__host__ __device__ inline int y_buf_elems(int tk, int n, int csize) {
  const int e = tk * n + (csize == (int)sizeof(float2) ? tk * n / 16 : 0);
  const int bytes = (e * csize + 127) / 128 * 128;
  return bytes / csize;
}

inline size_t y_smem_bytes(int tk, int n, int ntw, size_t csize) {
  return 128 + csize * (2 * (size_t)y_buf_elems(tk, n, (int)csize) + (size_t)ntw);
}

// Whether a tile reads its twiddles from the global table (L1-cached) rather
// than a shared-memory copy: FP32 FFT tiles of the compile-time lengths.  A
// tile is small (a few KB per column pair), so the per-CTA copy of the table
// was as much traffic as the tile and its shared memory cost occupancy.
__host__ __device__ inline bool y_global_tw(const FftDesc& d, int ytype, bool fp32) {
  return fp32 && ytype == Y_FFT && tile_fixed_len(d);
}

inline size_t y_smem_of(const cfs_plan* P, int tk, bool fp32) {
  const int ntw = y_global_tw(P->fy, P->ybc, fp32) ? 0 : P->fy.ntw;
  return y_smem_bytes(tk, P->ny, ntw, fp32 ? sizeof(float2) : sizeof(double2));
}

// Threads per tile: FP32 tiles are bound by latency (a tile's passes are
// short against its copies), so they take more warps per tile; FP64 tiles
// are bound by the FP64 pipe.
template <class C> constexpr int y_threads() { return sizeof(C) == sizeof(float2) ? 256 : 128; }

template <class C>
__device__ __forceinline__ C cmul_conj_a(C a, C b) {  // conj(a) * b
  return mkc<C>(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// The wall transform of a loaded tile (buf0), stored back by TMA.
template <bool INV, class C>
__device__ __forceinline__ void y_wall_transform(C* buf0, C* buf1, const FftDesc& d, int tk,
                                                 const C* tw, int ytype,
                                                 const C* __restrict__ wy, const CUtensorMap* map,
                                                 int by, int nbox, int x0, int z) {
  using T = typename cscal<C>::T;
  const int N = d.n;
  const bool dst = (ytype == Y_DST);
  const T h = T(0.5);
  C* res;
  if (!INV) {
    for (int e = threadIdx.x; e < N * tk; e += blockDim.x) {  // reorder (and signs)
      const int j = e / tk, c = e - j * tk;
      const int t = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
      C v = buf0[e];
      if (dst && (j & 1)) v = mkc<C>(-v.x, -v.y);
      buf1[t * tk + c] = v;
    }
    __syncthreads();
    res = stockham_smem<false, true>(buf1, buf0, d, tk, tk, 1, tw);
    C* out = (res == buf0) ? buf1 : buf0;
    for (int e = threadIdx.x; e < (N / 2 + 1) * tk; e += blockDim.x) {
      const int k = e / tk, c = e - k * tk;
      const int kn = (k == 0) ? 0 : N - k;
      const C vk = res[k * tk + c], vn = res[kn * tk + c];
      const C wk = wy[k], wn = wy[kn];
      const C a = cmul(wk, vk), b = cmul_conj_a(wk, vn);  // X_k
      out[(dst ? N - 1 - k : k) * tk + c] = mkc<C>(h * (a.x + b.x), h * (a.y + b.y));
      if (kn != k) {
        const C a2 = cmul(wn, vn), b2 = cmul_conj_a(wn, vk);  // X_{N-k}
        out[(dst ? N - 1 - kn : kn) * tk + c] = mkc<C>(h * (a2.x + b2.x), h * (a2.y + b2.y));
      }
    }
    res = out;
  } else {
    for (int e = threadIdx.x; e < (N / 2 + 1) * tk; e += blockDim.x) {
      const int k = e / tk, c = e - k * tk;
      const int kn = (k == 0) ? 0 : N - k;
      const C xk = buf0[(dst ? N - 1 - k : k) * tk + c];
      if (k == 0) {
        buf1[c] = xk;
        continue;
      }
      const C xn = buf0[(dst ? N - 1 - kn : kn) * tk + c];
      // V_k = conj(w_k) (X_k - i X_{N-k})
      buf1[k * tk + c] = cmul_conj_a(wy[k], mkc<C>(xk.x + xn.y, xk.y - xn.x));
      if (kn != k) buf1[kn * tk + c] = cmul_conj_a(wy[kn], mkc<C>(xn.x + xk.y, xn.y - xk.x));
    }
    __syncthreads();
    res = stockham_smem<true, true>(buf1, buf0, d, tk, tk, 1, tw);
    C* out = (res == buf0) ? buf1 : buf0;
    for (int e = threadIdx.x; e < N * tk; e += blockDim.x) {  // undo the reordering
      const int j = e / tk, c = e - j * tk;
      const int t = (j & 1) ? N - 1 - (j >> 1) : (j >> 1);
      C v = res[t * tk + c];
      if (dst && (j & 1)) v = mkc<C>(-v.x, -v.y);
      out[e] = v;
    }
    res = out;
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_3d(map, res + b * by * tk, x0, b * by, z);
    tma_store_commit_and_wait_read();
  }
}

// Tile bx (columns [bx * tk, bx * tk + tk)) of z plane z; ytype is Y_FFT for
// periodic y, else the wall transform, with wy[k] = exp(-i pi k / 2N).
template <bool INV, class C, int EMU = 0>
__device__ __forceinline__ void fft_y_body(const CUtensorMap* map, const FftDesc& d,
                                           const C* __restrict__ twg, int tk, int by, int nbox,
                                           int* status, int bx, int z, int ytype,
                                           const C* __restrict__ wy) {
  using T = typename cscal<C>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  C* buf0 = reinterpret_cast<C*>(smem_raw + 128);
  // both ping-pong buffers start on 128-byte boundaries: either may be the
  // source of the TMA store
  const int bstride = y_buf_elems(tk, d.n, (int)sizeof(C));
  C* buf1 = buf0 + bstride;
  C* tw = buf1 + bstride;
  const int x0 = 2 * tk * bx;  // in reals: a 16-byte aligned coordinate

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)(nbox * by * tk * sizeof(C)));
    for (int b = 0; b < nbox; ++b) tma_load_3d(buf0 + b * by * tk, map, bar, x0, b * by, z);
  }
  const bool gtw = y_global_tw(d, ytype, sizeof(C) == sizeof(float2));
  if (!gtw)
    for (int e = threadIdx.x; e < d.ntw; e += blockDim.x) tw[e] = twg[e];
  // every thread waits (bounded); the CTA then agrees on one outcome, which
  // also publishes the twiddles
  if (!cta_wait(bar, 0, status)) return;  // no pass ran; nothing is stored
  const int ny = d.n;
  // Column kx = 0 of the first tile is the packed pair F(0,ky) + i F(Nx/2,ky)
  // (App. A).  Its y spectrum is stored untangled, App. A's packing applied
  // once more along y: slot ky (0 < 2ky < Ny) holds F(0,ky), slot Ny-ky holds
  // F(Nx/2,ky), and the self-conjugate slots (ky = 0, Ny/2) keep the real pair
  // F(0,ky) + i F(Nx/2,ky).  Every slot is then one column of Eq. 12.
  if (ytype != Y_FFT) {  // walls: cosine or sine transform of every column
    y_wall_transform<INV>(buf0, buf1, d, tk, tw, ytype, wy, map, by, nbox, x0, z);
    return;
  }
  if (INV && bx == 0) {  // re-tangle before the inverse transform
    for (int ky = 1 + threadIdx.x; 2 * ky < ny; ky += blockDim.x) {
      const C f0 = buf0[ky * tk], fm = buf0[(ny - ky) * tk];
      buf0[ky * tk] = mkc<C>(f0.x - fm.y, f0.y + fm.x);         // F0 + i FM
      buf0[(ny - ky) * tk] = mkc<C>(f0.x + fm.y, fm.x - f0.y);  // conj F0 + i conj FM
    }
    __syncthreads();
  }
  // element (y, c) of the tile sits at y*tk + c: element stride tk, batch stride 1
  C* res = stockham_tile<INV, C, EMU>(buf0, buf1, d, tk, gtw ? twg : tw);
  if (!INV && bx == 0) {  // untangle after the forward transform
    for (int ky = 1 + threadIdx.x; 2 * ky < ny; ky += blockDim.x) {
      const C zz = res[ky * tk], zm = res[(ny - ky) * tk];
      // F0 = (Z + conj Zm)/2,  FM = -i (Z - conj Zm)/2
      const T h = T(0.5);
      res[ky * tk] = mkc<C>(h * (zz.x + zm.x), h * (zz.y - zm.y));
      res[(ny - ky) * tk] = mkc<C>(h * (zz.y + zm.y), h * (zm.x - zz.x));
    }
    __syncthreads();
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_3d(map, res + b * by * tk, x0, b * by, z);
    tma_store_commit_and_wait_read();
  }
}

// EMU (FP64 only): the butterfly additions that run on the integer units
// (kEmu* in chanfs_fft.cuh; the same bits as the FP64 pipe's).
template <bool INV, class C, int EMU = 0>
__global__ void __launch_bounds__(256) fft_y_kernel(const __grid_constant__ CUtensorMap map,
                                                    FftDesc d, const C* __restrict__ twg,
                                                    int tk, int by, int nbox, int* status,
                                                    int ytype, const C* __restrict__ wy) {
  fft_y_body<INV, C, EMU>(&map, d, twg, tk, by, nbox, status, blockIdx.x, blockIdx.y, ytype,
                          wy);
}

// One launch for several boxes (FP32 inner solves of grouped refinement).
template <bool INV>
__global__ void __launch_bounds__(256, 1) fft_y_group_kernel(const YBox* boxes, GroupMap g) {
  int b, blk;
  if (!group_block(g, &b, &blk)) return;
  const YBox& y = boxes[b];
  if (threadIdx.x == 0) tensormap_acquire(&y.map);  // thread 0 issues the TMA copies
  fft_y_body<INV, float2>(&y.map, y.d, static_cast<const float2*>(y.tw), y.tk, y.by, y.nbox,
                          y.status, blk % y.ntx, blk / y.ntx, y.ytype,
                          static_cast<const float2*>(y.wy));
}

template <class C, int EMU = 0>
static cudaError_t launch_y(const cfs_plan* P, void* data, bool inverse, int tk, const C* tw,
                            const C* wy, cudaStream_t st) {
  if (P->ny == 1) return cudaSuccess;  // length-1 transform is the identity
  using T = typename cscal<C>::T;
  CUtensorMap map;
  const cuuint64_t gdim[3] = {(cuuint64_t)(2 * P->M), (cuuint64_t)P->ny, (cuuint64_t)P->nz};
  const cuuint64_t gstride[2] = {(cuuint64_t)(2 * P->M) * sizeof(T),
                                 (cuuint64_t)(2 * P->M) * P->ny * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * tk), (cuuint32_t)P->by, 1};
  if (!encode_map(&map, sizeof(T), 3, data, gdim, gstride, box)) return cudaErrorInvalidValue;
  const size_t smem = y_smem_of(P, tk, sizeof(C) == sizeof(float2));
  dim3 grid((P->M + tk - 1) / tk, P->nz);
  if (!inverse) {
    auto k = fft_y_kernel<false, C, EMU>;
    allow_max_smem(k);
    k<<<grid, y_threads<C>(), smem, st>>>(map, P->fy, tw, tk, P->by, P->nbox, P->d_status,
                                          P->ybc, wy);
  } else {
    auto k = fft_y_kernel<true, C, EMU>;
    allow_max_smem(k);
    k<<<grid, y_threads<C>(), smem, st>>>(map, P->fy, tw, tk, P->by, P->nbox, P->d_status,
                                          P->ybc, wy);
  }
  return cudaGetLastError();
}

bool y_tile_ok(const cfs_plan* P, int tk, bool fp32) {
  const size_t csize = fp32 ? sizeof(float2) : sizeof(double2);
  if (tk < 1 || tk > 32 || (fp32 && tk % 2)) return false;  // 16-byte TMA box rows
  if (P->nbox > 1 && ((size_t)P->by * tk * csize) % 128 != 0) return false;
  return y_smem_of(P, tk, fp32) <= 227 * 1024;
}

cudaError_t launch_fft_y(const cfs_plan* P, double* data, bool inverse, cudaStream_t st) {
  // the plan's level L of integer-unit additions: kEmu* bits 0 .. L-1 (the
  // x transform's untangle bit has no work here)
  switch (P->emu_y) {
    case 1:
      return launch_y<double2, 1>(P, data, inverse, P->tk, P->d_twy, P->d_wy, st);
    case 2:
      return launch_y<double2, 3>(P, data, inverse, P->tk, P->d_twy, P->d_wy, st);
    case 3:
    case 4:
      return launch_y<double2, 7>(P, data, inverse, P->tk, P->d_twy, P->d_wy, st);
    default:
      return launch_y<double2, 0>(P, data, inverse, P->tk, P->d_twy, P->d_wy, st);
  }
}

cudaError_t launch_fft_y32(const cfs_plan* P, float* data, bool inverse, cudaStream_t st) {
  return launch_y<float2>(P, data, inverse, P->tk32, P->d_twy32, P->d_wy32, st);
}

size_t y_group_box(const cfs_plan* P, YBox* box, int* blocks) {
  const int tk = P->tk32;
  const cuuint64_t gdim[3] = {(cuuint64_t)(2 * P->M), (cuuint64_t)P->ny, (cuuint64_t)P->nz};
  const cuuint64_t gstride[2] = {(cuuint64_t)(2 * P->M) * sizeof(float),
                                 (cuuint64_t)(2 * P->M) * P->ny * sizeof(float)};
  const cuuint32_t bx[3] = {(cuuint32_t)(2 * tk), (cuuint32_t)P->by, 1};
  if (!encode_map(&box->map, sizeof(float), 3, P->d_r32, gdim, gstride, bx)) return 0;
  box->d = P->fy;
  box->tw = P->d_twy32;
  box->tk = tk;
  box->by = P->by;
  box->nbox = P->nbox;
  box->ntx = (P->M + tk - 1) / tk;
  box->status = P->d_status;
  box->ytype = P->ybc;
  box->wy = P->d_wy32;
  *blocks = (P->ny == 1) ? 0 : box->ntx * P->nz;  // a length-1 transform is the identity
  return y_smem_of(P, tk, true);
}

cudaError_t launch_fft_y_group32(const YBox* boxes, GroupMap g, int total, size_t smem,
                                 bool inverse, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  if (!inverse) {
    auto k = fft_y_group_kernel<false>;
    allow_max_smem(k);
    k<<<total, y_threads<float2>(), smem, st>>>(boxes, g);
  } else {
    auto k = fft_y_group_kernel<true>;
    allow_max_smem(k);
    k<<<total, y_threads<float2>(), smem, st>>>(boxes, g);
  }
  return cudaGetLastError();
}

}  // namespace chanfs
