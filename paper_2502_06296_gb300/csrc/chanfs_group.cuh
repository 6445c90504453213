// chanfs_group.cuh -- grouped launches: one kernel launch covers one stage of
// the solves of several plans (boxes of different sizes).
//
// Box b owns the blocks [start[b], start[b+1]) of a grouped grid; each box
// carries its own argument record, so boxes with different grids, tables and
// coefficients share one launch.  A per-box `active` word (may be null) lets
// iterative refinement drop boxes that have converged: their blocks return at
// once.  The field pointers that change from call to call (right-hand side
// and solution) sit in a small per-call table, GroupIo, read by the kernels
// that touch them.
#pragma once

#include "chanfs_internal.cuh"

namespace chanfs {

// Output modes of the FP32 inverse x transform: in place, FP64 result written
// to the solution, or added to it (the correction step p += delta).
enum { OUT_SAME = 0, OUT_SET = 1, OUT_ADD = 2, OUT_SUM = 3 };

struct GroupMap {
  const int* start;   // nbox + 1 block offsets
  const int* active;  // nbox flags, or nullptr (every box runs)
  int nbox;
};

struct GroupIo {
  const double* f;  // right-hand side
  double* p;        // solution
};

// Arguments of one box, per grouped kernel.
struct XBox {  // packed real FFT along x (fft_x.cu)
  FftDesc d;
  const void* in;
  const void* in2;  // forward transforms of later refinement iterations read this
  void* out;
  const void* tw;
  const void* post;
  long long nlines;
  int lb;
  int* status;
  const double* msum;  // inverse, correction pass: the solution's weighted sum (may be null)
  double minv;         // 1 / (sum of the cell widths * Nx * Ny)
  const void* add_src; // inverse, second pass (OUT_SUM): the first correction (FP32)
};

struct YBox {  // FFT along y on TMA tiles (fft_y.cu); the map is 64-byte aligned
  CUtensorMap map;
  FftDesc d;
  const void* tw;
  const void* wy;  // wall-transform factors (y walls)
  int tk, by, nbox, ntx;
  int ytype;       // 0 periodic y (FFT), 1 DCT-II, 2 DST-II
  int* status;
};

struct ThomasArgs {  // z sweeps of Eq. 12 (thomas.cu)
  void* S;               // spectrum (Nz, Ny, M) complex, double2 or float2
  const double2* fwd;    // FP64 factors (s/piv, A/piv) per (k, kyp, kx in [0, M])
  const double* bwd;     // FP64 C/piv
  const float2* fwd32;   // FP32 copies (refined plans only)
  const float* bwd32;
  const double* sing;    // Neumann (0,0): wn | gn | hs, 3*nz (see below)
  double sing_cg;        // g^T 1' / sum(w)
  double sing_sc;        // the factor scale of the (0,0) column
  int M, ny, nz, nky;
  int nblk_x;            // blocks along kx per ky
  int neumann;
  int kx64, ky64;        // FP32 spectra: columns kx < kx64, |ky| < ky64 in FP64
  int ywall;             // y walls: every slot ky is its own column (no +-ky pairs)
};

// The partitioned FP32 z solve of Eq. 12 (Algorithm 2 over register-resident
// z-partitions, thomas.cu).
struct ZPartArgs {
  ThomasArgs t;        // spectrum, sizes; the special columns' factors
  const float4* zrow;  // (A_k, B_k, C_k, 1) / s of the z operator for k < nz (s the
                       // inverse-FFT normalisation), then (0, 1, 0, 0) rows: x = 0,
                       // uncoupled (the wall row has C = 0)
  const float* lam;    // lx[0..M] then ly[0..nky), divided by s
  int P;               // partitions per column
  int C;               // columns per tile (C * P of the CTA's 256 threads work)
  int ntx;             // tiles along kx per slot pair
  int nsp;             // blocks of the special columns (first in the grid)
  int mm;              // rows per partition (8)
};

struct ResBox {  // refinement residual and norms (refine.cu)
  const double* abc;   // Helmholtz: A' | B' | C'
  const double* dzf;   // cell widths
  double* partial;     // nz * start_chunks(nz) plane-chunk sums of the start pass
  double* mean;        // dz-weighted mean
  float* r32;          // FP32 residual / correction
  float* r32b;         // FP32 residual of the later iterations
  float* rlo;          // low part of the residual kept between iterations (high part: r32b)
  float* dcopy;        // the first correction, kept for the second pass (OUT_SUM)
  const float4* zk;    // Poisson: packed double-float coefficients per plane (refine.cu)
  unsigned int* rmax;  // max |r| (float bits)
  int nx, ny, nz, n;   // n = Helmholtz unknowns per column
  int neumann;         // the operator has the constants as null space (mean removal)
  int ybc;             // 0 periodic y, 1 Neumann walls, 2 Dirichlet walls
  double* mpart;       // per-block weighted sums of a correction
  double* mnum;        // running weighted sum of the solution
  double inv_wn;       // 1 / (sum of the cell widths * Nx * Ny)
};

// Blocks of the grouped mean subtraction for a field of n points.
inline __host__ __device__ long long group_sub_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return b < 1216 ? b : 1216;
}

struct HThomasBox {  // Helmholtz Thomas sweep of one box (helm_thomas.cu)
  const void* rhs;     // FP32 inner solves: the plan's residual field (in place)
  void* u;
  const void* fac;     // fs | fa | fc, 3n
  long long ncols;     // Nx * Ny
  int n, nz, face;
  int per_call;        // FP64 boxes: rhs and u from the call's GroupIo table
};

template <class R>
struct PcrArgs {  // Algorithm 2 runtime (pcr.cu)
  R* u;                // output field (for the face wall row)
  long long ncols;     // columns solved: Nx * Ny, or a range of them
  long long zstride;   // elements between z rows (Nx * Ny)
  int n;               // unknowns per column
  int nparts;
  int face;            // face-located field: slot nz-1 is the wall, written 0
  int nz;
  int by, nbox;        // rows per TMA box, boxes per tile
  const R* rows;       // alpha | beta | ib | ap | cp  (5n)
  const R* red;        // rl | rip | ripc             (3 * 2p)
};

template <class R>
struct PcrBoxT {  // one field of a grouped Algorithm 2 launch; maps 64-byte aligned
  CUtensorMap in_map;
  CUtensorMap out_map;
  PcrArgs<R> a;
  int* status;
  int blocks;  // blocks of this box (they stride over its tiles)
};
using PcrBox = PcrBoxT<float>;     // FP32 inner solves of refinement
using PcrBox64 = PcrBoxT<double>;  // FP64 solves

// The refined Helmholtz solve in one pass (pcr.cu, pcr_refine_kernel): FP32
// Algorithm 2 solves and double-float residuals on tiles in shared memory.
struct PcrRefineArgs {
  double* u;            // output field (for the face wall row)
  long long ncols;      // Nx * Ny
  int n, nparts, nz, face, by, nbox;
  int maxit;            // FP32 solves per tile at most
  float tol;            // stop when max|r| <= tol max|rhs| over the tile
  const float* rows;    // FP32 Algorithm 2 factors, alpha | beta | ib | ap | cp (5n)
  const float* red;     // FP32 reduced LU, rl | rip | ripc (3 * 2p)
  const double* abc;    // FP64 rows of I - c L_z: A' | B' | C' (n each)
  const float* lv;      // reduced system by parallel cyclic reduction: K1 | K2 | 1/diag
  int nlv;              // its levels, ceil(log2 2p)
  unsigned int* words;  // [0] max |r|, [1] max |rhs| (float bits), [2] most FP32 solves
};

struct PcrRefineBox {  // one field of a grouped launch; maps 64-byte aligned
  CUtensorMap in_map;
  CUtensorMap out_map;
  PcrRefineArgs a;
  int* status;
  int blocks;
};

#ifdef __CUDACC__

// Box and box-local block of this block; false if the box is masked out.
__device__ __forceinline__ bool group_block(const GroupMap& g, int* box, int* blk) {
  const int b0 = (int)blockIdx.x;
  int lo = 0, hi = g.nbox;  // start[lo] <= b0 < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(g.start + mid) <= b0) lo = mid;
    else hi = mid;
  }
  *box = lo;
  *blk = b0 - __ldg(g.start + lo);
  if (!g.active) return true;
  return *(volatile const int*)(g.active + lo) != 0;
}

#endif  // __CUDACC__

// Grouped launchers (one per translation unit).  `total` = start[nbox];
// `smem` = the largest dynamic shared memory any box needs.
cudaError_t launch_rfft_x_group32(const XBox* boxes, GroupMap g, int total, size_t smem,
                                  bool inverse, int out_mode, const GroupIo* io, int alt_in,
                                  cudaStream_t st);
cudaError_t launch_fft_y_group32(const YBox* boxes, GroupMap g, int total, size_t smem,
                                 bool inverse, cudaStream_t st);
cudaError_t launch_thomas_group32(const ThomasArgs* boxes, GroupMap g, int total,
                                  cudaStream_t st);
cudaError_t launch_pcr_group32(const PcrBox* boxes, GroupMap g, int total, int threads,
                               size_t smem, cudaStream_t st);
size_t pcr_group_box(const cfs_plan* P, const HelmCoef& h, PcrBox* box, int* blocks,
                     int* threads);
// FP64 Algorithm 2 on the caller's fields (rhs -> u).
cudaError_t launch_pcr_group64(const PcrBox64* boxes, GroupMap g, int total, int threads,
                               size_t smem, cudaStream_t st);
size_t pcr_group_box64(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                       PcrBox64* box, int* blocks, int* threads);

// The refined Helmholtz solve in one pass (FP32 Algorithm 2 solves and
// double-float residuals in shared memory): whether plan P can take it for
// set h (shared memory, FP32 Algorithm 2 inner solves), and the launches;
// `words` receives max|r|, max|rhs| (float bits) and the most FP32 solves.
bool pcr_refine_fits(const cfs_plan* P, const HelmCoef& h);
size_t pcr_refine_smem(int n, int nparts);
cudaError_t launch_pcr_refine(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                              unsigned int* words, cudaStream_t st);
// Rows per thread of the kernel instance set h needs (8, 16, 24, 32; 0: none
// fits), and the threads a CTA of that instance may have.  A grouped launch
// runs one instance: `rows` (the largest of its boxes') selects it.
constexpr int kPcrTileColumns = 16;  // columns of an Algorithm 2 tile (one half-warp)
int pcr_refine_rows(const HelmCoef& h);
int pcr_refine_thread_limit(int rows);
size_t pcr_refine_group_box(const cfs_plan* P, const HelmCoef& h, const double* rhs, double* u,
                            unsigned int* words, PcrRefineBox* box, int* blocks, int* threads,
                            int* rows);
cudaError_t launch_pcr_refine_group(const PcrRefineBox* boxes, GroupMap g, int total, int threads,
                                    size_t smem, int rows, cudaStream_t st);

// Thomas sweeps of the Helmholtz systems (helm_thomas.cu): `fp32` boxes are
// the FP32 inner solves of refinement, the others FP64 solves on the call's
// fields.  Returns the box's shared memory; *blocks its block count.
size_t helm_thomas_group_box(const cfs_plan* P, const HelmCoef& h, bool fp32, HThomasBox* box,
                             int* blocks);
cudaError_t launch_helm_thomas_group(const HThomasBox* boxes, GroupMap g, int total, size_t smem,
                                     bool fp32, const GroupIo* io, cudaStream_t st);

// Grouped refinement kernels (refine.cu), launched by group.cu.
cudaError_t launch_group_refine_stage(int stage, const ResBox* boxes, GroupMap g, int total,
                                      const GroupIo* io, int flag, cudaStream_t st);
struct GroupCtl {  // device-side iteration state of a grouped refined solve
  int it;          // iterations done
  int nactive;     // boxes still iterating after the last one
};
cudaError_t launch_group_start(const ResBox* boxes, int nbox, int keys, double* fmax,
                               const int* eligible, int* active, int* mean_on, int* zero,
                               int* iters, double* rho, GroupCtl* ctl, cudaStream_t st,
                               int* one = nullptr);
// one (may be null): boxes still on their first correction, i.e. whose p is
// written by the FIRST_ONLY stage if they stop there
cudaError_t launch_group_iter_end(const ResBox* boxes, int nbox, const double* fmax,
                                  const double* tol, const int* maxit, int* active,
                                  int* mean_on, int* iters, double* rho, GroupCtl* ctl,
                                  cudaGraphConditionalHandle cond, int set_cond, cudaStream_t st,
                                  int* one = nullptr);
cudaError_t launch_group_zero_max(const ResBox* boxes, int nbox, cudaStream_t st);
enum {
  GSTAGE_MEAN_FINAL = 1,
  GSTAGE_RESIDUAL = 2,
  GSTAGE_HELM_RESIDUAL = 4,  // flag = mode of helm_residual_kernel
  GSTAGE_UPDATE = 5,         // r -= L delta (double-float), r32b and max
  GSTAGE_ZERO = 6,           // zero solution (boxes with a zero right-hand side)
  GSTAGE_START = 7,          // r_0 = f as FP32, its extremes, plane sums (plane x chunk blocks)
  GSTAGE_MEAN_ACC = 8,       // running weighted sum of the solution += the correction's
  GSTAGE_MEAN_FROM_NUM = 9,  // the solution's weighted mean from the running sum
  GSTAGE_FIRST_ONLY = 10     // p from the only correction (boxes stopped after one solve)
};

// Host-side descriptions of one plan's box for the grouped kernels.
size_t x_group_box(const cfs_plan* P, bool inverse, XBox* box, int* blocks);
size_t y_group_box(const cfs_plan* P, YBox* box, int* blocks);
size_t thomas_group_box(const cfs_plan* P, ThomasArgs* box, int* blocks);
// Boxes whose plans take the partitioned FP32 z solve (CFS_OPT_THOMAS_TILE 1)
// run it in their grouped solves too, so that a box's bits match its solve
// alone.
bool zpart_group_member(const cfs_plan* P);
size_t zpart_group_box(const cfs_plan* P, ZPartArgs* box, int* blocks);  // returns smem
cudaError_t launch_zpart_group(const ZPartArgs* boxes, GroupMap g, int total, size_t smem,
                               cudaStream_t st);

}  // namespace chanfs
