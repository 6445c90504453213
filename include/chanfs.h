/*
 * chanfs.h -- C ABI of libchanfs, a GB300-native (sm_103a) solver for the
 * pressure-Poisson and wall-normal implicit-diffusion Helmholtz equations of
 * incompressible channel flow on a staggered second-order finite-difference
 * grid, after Diez, Peeters & Costa, "A pencil-distributed finite-difference
 * solver for extreme-scale calculations of turbulent wall flows at high
 * Reynolds number" (arXiv 2502.06296).
 *
 * Grid and storage
 *   Nx x Ny x Nz cells; x and y periodic and uniform (dx = lx/Nx, dy = ly/Ny);
 *   z bounded by two walls and arbitrarily stretched, given by the Nz cell
 *   widths dz[k] (Sec. 2.1).  Every field is Nx*Ny*Nz contiguous doubles,
 *   x fastest: f[x + Nx*(y + Ny*z)].  Cell-centred fields hold p, u, v; a
 *   face-located field holds w at the top face of cell k in slot k, and slot
 *   Nz-1 (the top wall) is written as 0 by the solver.
 *
 * Calls and memory
 *   Field pointers are DEVICE pointers unless the name ends in _host.  They
 *   belong to the caller, must be 16-byte aligned, and stay valid until the
 *   work queued on `stream` has finished.  `stream` is a cudaStream_t passed
 *   as void* (NULL = legacy default stream).  Solves are asynchronous; input
 *   and output may be the same buffer (in place).  Plans own their tables and
 *   workspace; one plan may be used from one host thread at a time.
 *
 * Errors
 *   Every call returns a cfs_status.  Argument errors are detected on the host
 *   and return before anything is queued.  A device-side failure (a bounded
 *   wait that ran out) is recorded in the plan and reported by cfs_plan_check.
 */
#ifndef CHANFS_H
#define CHANFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHANFS_VERSION 100 /* 1.0.0 */

typedef struct cfs_plan* cfs_plan_t; /* opaque, owned by the library */

typedef enum {
  CFS_OK = 0,
  CFS_EINVAL = -1,         /* bad argument (null pointer, bad size, bad enum) */
  CFS_ENOMEM = -2,         /* device or host allocation failed */
  CFS_EUNSUPPORTED = -3,   /* size outside what the kernels implement */
  CFS_ECUDA = -4,          /* a CUDA runtime call failed */
  CFS_ETIMEOUT = -5,       /* a device-side bounded wait ran out */
  CFS_ENOTCONVERGED = -6,  /* iterative refinement missed its tolerance */
  CFS_ECANCELED = -7,      /* a served request was cancelled before it ran */
  CFS_EGUARD = -8          /* guard words around a plan work buffer were overwritten */
} cfs_status;

typedef enum { CFS_BC_NEUMANN = 0, CFS_BC_DIRICHLET = 1 } cfs_bc;   /* z walls */
typedef enum { CFS_LOC_CENTER = 0, CFS_LOC_FACE = 1 } cfs_loc;      /* z location */
typedef enum {
  CFS_F64 = 0,          /* FP64 transforms and sweeps */
  CFS_F32_REFINED = 1   /* FP32 transforms and sweeps + FP64 iterative refinement */
} cfs_dtype;

/* Library version (CHANFS_VERSION of the build). */
int cfs_version(void);

/* Human-readable text for a cfs_status; never NULL. */
const char* cfs_status_string(int status);

/*
 * cfs_plan_create -- set up a solver for one grid on the current CUDA device
 * (Sec. 2.2.1 "Fourier-based synthesis", Eq. 12; App. A for the layout).
 *   nx     cells along x; even, nx/2 = 2^a 3^b, 2 <= nx <= 4096.
 *   ny     cells along y; 2^a 3^b, 1 <= ny <= 4096.
 *   nz     cells along z; 3 <= nz <= 16384.
 *   lx,ly  domain lengths (> 0); dx = lx/nx, dy = ly/ny.
 *   dz     nz HOST doubles, the cell widths along z (all > 0); copied.
 *   poisson_bc  z-wall condition of the Poisson equation (cfs_bc).
 *   dtype  CFS_F64, or CFS_F32_REFINED: solves run FP32 transforms and
 *          sweeps and recover FP64 accuracy by iterative refinement (see
 *          cfs_plan_set_refinement); the plan then also holds FP32 tables and
 *          one FP32 work field, and nx must be a multiple of 4.
 * At creation the plan computes, in FP64 and once (the time-invariant
 * pre-processing of Sec. 2.2.4): the z metrics, the modified wavenumbers
 * 2(cos(2 pi k/N) - 1)/h^2 re-ordered to the packed layout (App. A), the FFT
 * twiddle tables and the LU factors of every (kx, ky) tridiagonal system of
 * Eq. 12.  Returns CFS_EUNSUPPORTED for sizes outside the ranges above.
 * On success *plan is set; on failure *plan is left NULL.
 */
int cfs_plan_create(cfs_plan_t* plan, int nx, int ny, int nz, double lx,
                    double ly, const double* dz, int poisson_bc, int dtype);

/*
 * cfs_plan_create_walls -- as cfs_plan_create, with walls in y as well
 * (Sec. 2.2.1 names cosine/sine transforms for non-periodic directions).
 *   ybc  CFS_Y_PERIODIC (what cfs_plan_create makes), CFS_Y_NEUMANN or
 *        CFS_Y_DIRICHLET: homogeneous walls at y = 0 and y = ly, cell-centred
 *        unknowns, mirror ghosts p_{-1} = +-p_0 and p_{Ny} = +-p_{Ny-1}.
 * With walls the y transform is DCT-II (Neumann) or DST-II (Dirichlet), each
 * computed by one complex FFT of length Ny; the eigenvalues are
 * 2(cos(pi k/Ny) - 1)/dy^2 and 2(cos(pi (k+1)/Ny) - 1)/dy^2, k < Ny.  The
 * solution's null space (constants) exists only with Neumann walls in both
 * y and z; the Neumann conventions above apply to it.  Every solve supports
 * y walls (the fully implicit Helmholtz uses the same y transforms).
 */
enum { CFS_Y_PERIODIC = 0, CFS_Y_NEUMANN = 1, CFS_Y_DIRICHLET = 2 };
int cfs_plan_create_walls(cfs_plan_t* plan, int nx, int ny, int nz, double lx, double ly,
                          const double* dz, int poisson_bc, int ybc, int dtype);

/* Release the plan and everything it owns.  Waits for the device. */
int cfs_plan_destroy(cfs_plan_t plan);

/* Device bytes held by the plan (tables, cached coefficients, staging). */
int cfs_plan_device_bytes(cfs_plan_t plan, size_t* bytes);

/*
 * cfs_poisson_solve -- solve L p = f (Eq. 4 / Eq. 12): the staggered 7-point
 * Laplacian, periodic in x and y, with the plan's z-wall condition.
 *   f  device field (read), p  device field (written); f == p allowed.
 * Steps (Sec. 2.2.3 without transposes): packed real FFT along x (App. A),
 * complex FFT along y, one tridiagonal solve along z per (kx, ky), inverse y
 * and x transforms.  With Neumann walls the dz-weighted mean of f is removed
 * (compatibility) and p is returned with zero dz-weighted mean.
 * No workspace beyond p is used.
 */
int cfs_poisson_solve(cfs_plan_t plan, const double* f, double* p,
                      void* stream);

/*
 * cfs_helmholtz_prepare -- Step 1 of Algorithm 2 (Sec. 2.2.4) for the matrix
 * I - c L_z with homogeneous Dirichlet walls at location `loc`: the reduction
 * coefficients of each of `nparts` z-partitions and the factors of the
 * reduced 2*nparts boundary system, computed on the host in FP64 and cached
 * in the plan under (c, loc, nparts).  nparts = 0 picks a partition count.
 *   c  the coefficient of Eq. 11 (gamma_k nu dt / 2, i.e. alpha nu dt), >= 0.
 * Each partition needs at least 3 rows; at most 64 partitions and 1024
 * unknowns per column (a tile of 16 columns lives in shared memory);
 * otherwise EUNSUPPORTED.
 * Calling it is optional: cfs_helmholtz_solve prepares on a cache miss.
 */
int cfs_helmholtz_prepare(cfs_plan_t plan, double c, int loc, int nparts);

/*
 * cfs_helmholtz_solve -- solve (I - c L_z) u = rhs in every (x, y) column
 * (Eq. 11) by Steps 2-4 of Algorithm 2: runtime forward/backward reduction of
 * the right-hand side only, the reduced boundary system, and reconstruction.
 *   rhs  device field (read), u  device field (written); rhs == u allowed.
 * Uses the set cached by cfs_helmholtz_prepare with the plan's
 * CFS_OPT_PCR_PARTS count (when that option is 0: any cached set of (c, loc),
 * else one prepared with nparts = 0 on a miss).
 */
int cfs_helmholtz_solve(cfs_plan_t plan, double c, int loc, const double* rhs,
                        double* u, void* stream);

/*
 * cfs_spectral_forward / cfs_spectral_inverse -- the transform stages of the
 * Poisson solve on their own.  Forward: unnormalised DFT along x stored in
 * the packed real format of App. A (pair j >= 1 of a line is X_j; pair 0 is
 * X_0 + i X_{nx/2}), then an unnormalised complex DFT along y of each pair.
 * Inverse: the exact inverse (normalised by 1/(nx ny)).  Both are nx*ny*nz
 * doubles; in == out allowed.
 */
int cfs_spectral_forward(cfs_plan_t plan, const double* f, double* s,
                         void* stream);
int cfs_spectral_inverse(cfs_plan_t plan, const double* s, double* f,
                         void* stream);

/*
 * cfs_poisson_stage -- one kernel of the Poisson solve on its own, for
 * stage-by-stage testing and profiling.  `in` is read, `out` written (the
 * y and z stages work in place on `out`, after copying `in` there when the
 * two differ).  Stages, in the order cfs_poisson_solve runs them:
 *   CFS_STAGE_X_FORWARD  packed real DFT along x (App. A), unnormalised
 *   CFS_STAGE_Y_FORWARD  complex DFT along y of each packed pair, unnormalised
 *   CFS_STAGE_Z_SOLVE    the tridiagonal solves of Eq. 12 on the spectrum,
 *                        scaled by 2/(nx ny) to absorb the inverse transforms
 *   CFS_STAGE_Y_INVERSE  unnormalised inverse complex DFT along y
 *   CFS_STAGE_X_INVERSE  inverse real DFT along x, scaled by nx/2
 */
typedef enum {
  CFS_STAGE_X_FORWARD = 0,
  CFS_STAGE_Y_FORWARD = 1,
  CFS_STAGE_Z_SOLVE = 2,
  CFS_STAGE_Y_INVERSE = 3,
  CFS_STAGE_X_INVERSE = 4
} cfs_stage;
int cfs_poisson_stage(cfs_plan_t plan, int stage, const double* in,
                      double* out, void* stream);

/*
 * Host-buffer variants: f/p and rhs/u are HOST pointers (pinned memory gives
 * full copy bandwidth; pageable memory works).  The plan stages the field in
 * a device buffer it allocates on first use, copies in, solves and copies
 * out on `stream`, then waits for the stream before returning.
 */
int cfs_poisson_solve_host(cfs_plan_t plan, const double* f, double* p,
                           void* stream);
int cfs_helmholtz_solve_host(cfs_plan_t plan, double c, int loc,
                             const double* rhs, double* u, void* stream);

/*
 * cfs_solve_batch_host -- n solves on one plan through host buffers (no
 * counterpart in the paper): kind[i] CFS_REQ_POISSON (in[i] = f, out[i] = p)
 * or CFS_REQ_HELMHOLTZ (in[i] = rhs, out[i] = u, coefficient c[i], location
 * loc[i]; c and loc may be null if no solve is a Helmholtz one).  The copy of
 * each field to the device and of each result back overlap the solves of
 * the others: up to 4 device slots of (input, output) fields (as many as the
 * batch has solves, kept with the plan at the largest size used), one
 * copy-in stream and a copy-out stream per compute stream.  The solves run
 * after the work already on `stream`: Poisson solves on `stream`, and on
 * CFS_F64 plans the Helmholtz solves on a second stream beside them (they
 * share no plan scratch; refined solves all run on `stream`).  On CFS_F64
 * plans whose fields are larger than about 200 MB (or with
 * CFS_OPT_STREAM_CHUNKS set) each field moves in chunks: a Poisson field in
 * ranges of z planes, transformed along x range by range as it lands and
 * copied out range by range as its inverse x transform finishes; a Helmholtz
 * field solved by Algorithm 2 in ranges of y rows, each solved and copied
 * out on its own (Thomas-sweep Helmholtz solves take the field whole); and
 * the batch's first Helmholtz solve is taken first when the batch also holds
 * Poisson solves and its fields move in chunks.  The results are the same
 * bits as whole-field solves.  Host buffers should be pinned for the copies to
 * overlap.  Returns when every result has
 * arrived: CFS_OK, the first error, or CFS_ENOTCONVERGED if a refined solve
 * missed its tolerance (every output is still written).  A step of the
 * channel workload is one call: the Poisson solve and the three Helmholtz
 * solves of u, v and w.
 */
int cfs_solve_batch_host(cfs_plan_t plan, int n, const int* kind, const double* c, const int* loc,
                         const double* const* in, double* const* out, void* stream);

/*
 * cfs_helmholtz_solve_noalloc -- the solve of cfs_helmholtz_solve without a
 * plan and without allocating any memory.  The paper has no counterpart; it
 * exists for callers that cannot allocate device memory where they solve:
 * cudaMalloc and cudaFree synchronise the whole device, stalling every other
 * stream in flight, and applications that reserve the device memory up front
 * for their own pool have none left to give.
 *   nx, ny, nz, dz  grid as for cfs_plan_create (dz: nz HOST doubles, read
 *                   before the call returns); nx*ny even.
 *   c, loc          as for cfs_helmholtz_solve; nparts as for
 *                   cfs_helmholtz_prepare (0 = about 32 rows per partition).
 *   rhs, u          device fields as for cfs_helmholtz_solve (rhs == u allowed).
 *   device_status   DEVICE pointer to one int owned by the caller (4-byte
 *                   aligned): the call sets it to 0 on `stream`, and the
 *                   solve ORs failure bits into it (nonzero: a bounded wait
 *                   inside the kernel ran out and u is not valid).  Read it
 *                   once the work on `stream` has finished.
 * The Algorithm 2 coefficients are computed by a small kernel on `stream`,
 * in FP64 from the cell widths (passed as kernel parameters), into a fixed
 * device array inside the library, sized for at most 1024 unknowns per
 * column and 64 partitions (about 44 KB, held by every GPU that loads the
 * library until the process exits); larger sizes return CFS_EUNSUPPORTED
 * before anything is queued.  The call queues that kernel and the solve and
 * returns without waiting for the device.  The first call on a device looks
 * up the array's address there (cudaGetSymbolAddress), so make it before any
 * stream capture.  Every call overwrites the whole coefficient set; there is
 * one array per device, so calls whose work overlaps on one GPU (other
 * streams, other host threads) race and may read each other's coefficients.
 * Calls on different devices do not share anything.
 */
int cfs_helmholtz_solve_noalloc(int nx, int ny, int nz, const double* dz,
                                double c, int loc, int nparts,
                                const double* rhs, double* u,
                                int* device_status, void* stream);

/*
 * Iterative refinement (plans created with CFS_F32_REFINED).  A solve starts
 * from x = 0 and repeats { delta = FP32 solve of r; x += delta in FP64;
 * r = b - A x } until ||r||_inf <= tol ||b||_inf or `maxit` FP32 solves were
 * done (defaults: tol = 1e-10, maxit = 4).  A is the staggered 7-point
 * Laplacian (Poisson; b is the right-hand side minus its dz-weighted mean for
 * Neumann walls) or I - c L_z (Helmholtz).  Helmholtz residuals are formed in
 * FP64.  Poisson residuals are formed in double-float arithmetic (the
 * coefficients split hi + lo, the residual kept as an FP32 pair): the first
 * with the stencil written in differences of the correction (exact in FP32),
 * as accurate as an FP64 evaluation for a solution resolved by the grid, the
 * later ones as r -= A delta.  With Neumann walls the running dz-weighted
 * mean of x is subtracted from each correction after the first, so x keeps
 * a zero mean up to the FP32 rounding of its last correction (a solve that
 * stops after one FP32 solve has its mean removed in FP64 at the end).  FP64
 * is also used for the accumulation, the coefficient pre-processing and the
 * z sweep of the near-singular low-wavenumber columns.  Each iteration reads
 * the residual norm back, so refined solves synchronise `stream`; when the
 * target is missed the solve returns CFS_ENOTCONVERGED with its best x.
 * cfs_last_info reports the FP32 solves done and the final relative residual
 * of the last refined solve.
 */
int cfs_plan_set_refinement(cfs_plan_t plan, double tol, int maxit);
int cfs_last_info(cfs_plan_t plan, int* iters, double* rel_residual);

/*
 * cfs_helmholtz3d_solve -- the fully implicit Helmholtz solve of Eq. 8,
 * (I - c L) u = rhs with L the whole staggered Laplacian (periodic x; y as
 * the plan's, periodic or walls; homogeneous Dirichlet z walls, cell-centred
 * or face-located field as in cfs_helmholtz_solve).  It runs on the Poisson machinery: packed x FFT, y
 * FFT, one tridiagonal system per (kx, ky) with the diagonal
 * 1 - c (B_k + lx + ly) and off-diagonals -c A_k, -c C_k, inverse transforms.
 * The factors of every (kx, ky) system are computed on the GPU once per
 * (c, loc) and cached (at most 4 sets, each as large as the Poisson factors);
 * cfs_helmholtz3d_prepare computes a set ahead of time.  FP64 on every plan;
 * c >= 0; rhs == u allowed; for a face field slot Nz-1 of u is written 0.
 */
int cfs_helmholtz3d_prepare(cfs_plan_t plan, double c, int loc);
int cfs_helmholtz3d_solve(cfs_plan_t plan, double c, int loc, const double* rhs, double* u,
                          void* stream);

/*
 * Grouped solves.  The paper has no counterpart (it spreads one box over many
 * GPUs; a group puts many independent boxes on one).  A group is built from
 * up to 4096 CFS_F32_REFINED plans of the current device, of any sizes, z
 * grids, walls and refinement settings.  Every stage of the refined Poisson
 * solve (start pass, FP32 transforms and z sweeps, residuals, means) is
 * then one kernel launch for all boxes, and the refinement loop runs on the
 * device: a solve is one CUDA graph whose loop is a conditional WHILE node,
 * the kernel that ends an iteration setting its condition; the host waits
 * once, at the end.  The graph reads every per-box record from the group's
 * tables, so it depends only on the launch shape (number of boxes, blocks and
 * shared memory of each stage) and is reused across rebindings.  A shape is
 * captured at its second solve (its first runs as direct launches with the
 * loop on the host, so one-off shapes pay no capture); 128 graphs are kept
 * per group.  Each box follows its own refined solve
 * exactly, stopping test included, so its result is bit-identical to
 * cfs_poisson_solve on its plan.
 *   cfs_group_create   plans: nplans distinct plan handles (not owned: keep
 *                      them alive while the group exists).  CFS_EUNSUPPORTED
 *                      if a plan is not CFS_F32_REFINED or lives on another
 *                      device.
 *   cfs_group_poisson_solve  f, p: host arrays of nplans device pointers,
 *                      box b sized as plan b's fields; f[b] != p[b] (the
 *                      right-hand side is read again after p is first
 *                      written).  The solve uses the plans' work fields:
 *                      solves on the same plans, grouped or not, must not
 *                      overlap on the device.  Returns CFS_ENOTCONVERGED if a
 *                      box missed its tolerance (every box is still written).
 *   cfs_group_last_info  per box: FP32 solves used and final relative
 *                      residual of the last grouped solve (arrays of nplans).
 */
typedef struct cfs_group* cfs_group_t;
int cfs_group_create(cfs_group_t* group, int nplans, const cfs_plan_t* plans);
/* cfs_group_reserve makes an empty group with room for `capacity` plans;
 * cfs_group_rebind (re)binds it to nplans <= capacity plans without
 * allocating, the tables copied on `stream` ahead of the next solves there
 * (a serving loop keeps one group per stream and rebinds it per batch). */
int cfs_group_reserve(cfs_group_t* group, int capacity);
int cfs_group_rebind(cfs_group_t group, int nplans, const cfs_plan_t* plans, void* stream);
int cfs_group_destroy(cfs_group_t group);
int cfs_group_size(cfs_group_t group, int* nplans);
int cfs_group_poisson_solve(cfs_group_t group, const double* const* f, double* const* p,
                            void* stream);
/* The z-implicit Helmholtz solves (I - c[b] L_z) u[b] = rhs[b] of the boxes
 * (Eq. 11, Algorithm 2 for the FP32 inner solves), grouped in the same way:
 * c, loc: host arrays of nplans coefficients and field locations (see
 * cfs_helmholtz_solve); rhs[b] != u[b]. */
int cfs_group_helmholtz_solve(cfs_group_t group, const double* c, const int* loc,
                              const double* const* rhs, double* const* u, void* stream);
int cfs_group_last_info(cfs_group_t group, int* iters, double* rel_residual);
/* on = 0: later solves of the group launch their stages directly and run the
 * refinement loop on the host (one wait per iteration); on != 0 (the
 * default): graphs as above.  Both give bit-identical results. */
int cfs_group_set_graphs(cfs_group_t group, int on);
/* Launch tracing, a measurement aid (the paper has no counterpart).  While
 * on != 0, the group's solves run as direct launches (no graph) and every
 * copy and kernel they issue on the caller's stream is bracketed by a pair
 * of CUDA events (the first 512 of a solve; later ones run untraced).  The
 * first call with on != 0 creates the events (CFS_ECUDA if that fails).
 * cfs_group_trace waits for the last solve's events and writes the device
 * time of each traced copy or kernel, in issue order, to ms[0 .. min(count,
 * capacity)) in milliseconds; *count receives how many were traced.  Their
 * sum against the time of the same solve as a graph bounds the idle time
 * between a graph's nodes. */
int cfs_group_set_trace(cfs_group_t group, int on);
int cfs_group_trace(cfs_group_t group, float* ms, int capacity, int* count);

/*
 * Serving.  The paper has no counterpart.  A server takes Poisson and
 * Helmholtz solve requests from many concurrently running simulations
 * ("runs", one grid each) and answers them with FP32 + FP64-refined solves
 * (tolerance 1e-10, at most 4 FP32 solves).  A run has up to slots_per_run
 * plans, so that as many of its requests can be solved at the same time;
 * each plan stays resident in device memory while the budget allows: it is
 * created when a request first needs it (and tuned with cfs_plan_autotune if
 * `autotune`), and idle plans are destroyed, least recently used first, when
 * a new plan would exceed hbm_budget_bytes.  `workers` threads, each with its
 * own CUDA stream, form batches continuously: a free worker takes the oldest
 * request whose run has a free plan slot, adds every pending request of the
 * same kind that finds a free slot (up to max_batch), and solves them as one
 * grouped solve; requests arriving meanwhile join the next batch, and batches
 * of different workers overlap on the device.  A result is bit-identical to
 * the refined solve of the run's plan alone.
 *   cfs_server_create  CFS_ECUDA if no worker could start (its stream or
 *       group); workers that cannot start leave, the others serve.
 *   cfs_server_add_run  a grid (as cfs_plan_create); nx % 4 == 0; returns the
 *       run index.  CFS_EUNSUPPORTED if its plan alone exceeds the budget.
 *   cfs_server_submit  kind CFS_REQ_POISSON (c, loc ignored) or
 *       CFS_REQ_HELMHOLTZ (c >= 0, loc a cfs_loc); rhs and out: device fields
 *       of the run's size, distinct, owned by the caller and left untouched
 *       until the request completes.  Returns a ticket.
 *   cfs_server_wait  waits up to timeout_s seconds (< 0: no limit) for the
 *       ticket; CFS_ETIMEOUT if not done (the ticket stays valid).  On
 *       success *status is the request's status (a solve's status, the
 *       status of a plan creation that failed for it, CFS_ECANCELED) and
 *       *latency_s the time from submission to completion, and the ticket is
 *       retired.  A failure is the request's own: the others go on.
 *   cfs_server_cancel  takes a request that no worker has taken yet off the
 *       queue (it completes with CFS_ECANCELED); CFS_EINVAL if the ticket is
 *       unknown, already running or done.
 *   cfs_server_pause  paused != 0: workers form no new batches (running ones
 *       finish; requests queue); 0 resumes.
 *   cfs_server_destroy  resumes, finishes the pending requests, stops the
 *       workers and destroys the plans; tickets never waited for are freed.
 *   cfs_server_inject_fault  host-side fault injection for tests:
 *       CFS_FAULT_PLAN_ALLOC makes the next `count` plan creations of server
 *       S fail with CFS_ENOMEM, as a refused device allocation would;
 *       CFS_FAULT_WORKER_START (S = NULL) makes the next `count` worker
 *       start-ups of servers created afterwards fail.
 */
typedef struct cfs_server* cfs_server_t;
enum { CFS_REQ_POISSON = 0, CFS_REQ_HELMHOLTZ = 1 };
enum { CFS_FAULT_PLAN_ALLOC = 1, CFS_FAULT_WORKER_START = 2 };
typedef struct {
  unsigned long long submitted, completed, failed, batches;
  int max_batch_seen, plans_created, plans_evicted, plans_resident;
  size_t bytes_in_use;  /* plan bytes held (reserved estimates included) */
  unsigned long long cancelled;
  int workers_alive, pending;
} cfs_server_stats_t;
int cfs_server_create(cfs_server_t* server, size_t hbm_budget_bytes, int workers, int max_batch,
                      int slots_per_run, int autotune);
int cfs_server_add_run(cfs_server_t server, int nx, int ny, int nz, double lx, double ly,
                       const double* dz, int poisson_bc, int* run);
int cfs_server_submit(cfs_server_t server, int run, int kind, double c, int loc, const double* rhs,
                      double* out, unsigned long long* ticket);
int cfs_server_wait(cfs_server_t server, unsigned long long ticket, double timeout_s, int* status,
                    double* latency_s);
int cfs_server_cancel(cfs_server_t server, unsigned long long ticket);
int cfs_server_pause(cfs_server_t server, int paused);
int cfs_server_inject_fault(cfs_server_t server, int fault, int count);
int cfs_server_stats(cfs_server_t server, cfs_server_stats_t* stats);
int cfs_server_destroy(cfs_server_t server);

/*
 * z-slabs over several GPUs: the paper's parallel tridiagonal solver
 * (P-TDMA, Sec. 2.2.3) with one slab of whole x-y planes per rank
 * (p_y = 1, p_z = nranks, the layout of its weak-scaling runs, Sec. 3).
 * The x and y transforms of a rank's planes are local; along z each column's
 * system is split over the ranks, each rank's planes one partition of
 * Algorithm 2 (Sec. 2.2.4).  A solve is two calls around one exchange:
 *   *_reduce  transforms (Poisson) and Step 2 on the rank's rows; writes the
 *             rank's boundary buffer `bnd` (cfs_slab_boundary_doubles
 *             doubles: the two boundary values of every column, plus for the
 *             Poisson solve two partial sums of the Neumann (0, 0) column).
 *   the caller gathers the buffers of all ranks into `bnd_all`, rank-major
 *             (rank r's buffer at offset r * count; an NCCL all-gather).
 *   *_finish  Step 3 (the reduced system of the 2 nranks boundary unknowns
 *             of every column, solved by every rank) and Step 4 on the rank's
 *             rows, then the inverse transforms (Poisson); writes the rank's
 *             planes of the solution.
 * The reduced systems' coefficients are computed by every rank for all
 * ranks when the slab is created (Poisson) or a coefficient is first used
 * (Helmholtz), so only right-hand-side data is exchanged.  Fields are the
 * rank's planes: nx*ny*(z1 - z0) doubles, x fastest; `work` is a field of
 * that size owned by the caller (work == p allowed for the Poisson solve;
 * the Helmholtz solve keeps rhs, work and u distinct).  Results equal the
 * single-GPU solve of the whole field up to rounding.  Periodic y only.
 *   cfs_slab_partition  planes [z0, z1) of `rank` (host arithmetic only).
 *   cfs_slab_create  the rank's slab of the global grid (dz: nz HOST
 *       doubles of the whole grid); every slab needs at least 4 planes;
 *       nranks <= 64.  Creates a plan for the rank's planes on the current
 *       device.
 */
typedef struct cfs_slab* cfs_slab_t;
int cfs_slab_partition(int nz, int nranks, int rank, int* z0, int* z1);
int cfs_slab_create(cfs_slab_t* slab, int nx, int ny, int nz, double lx, double ly,
                    const double* dz, int poisson_bc, int nranks, int rank);
int cfs_slab_destroy(cfs_slab_t slab);
int cfs_slab_extent(cfs_slab_t slab, int* z0, int* z1);
int cfs_slab_boundary_doubles(cfs_slab_t slab, int kind, size_t* count);
int cfs_slab_poisson_reduce(cfs_slab_t slab, const double* f, double* work, double* bnd,
                            void* stream);
int cfs_slab_poisson_finish(cfs_slab_t slab, const double* bnd_all, double* work, double* p,
                            void* stream);
int cfs_slab_helmholtz_reduce(cfs_slab_t slab, double c, int loc, const double* rhs,
                              double* work, double* bnd, void* stream);
int cfs_slab_helmholtz_finish(cfs_slab_t slab, double c, int loc, const double* bnd_all,
                              const double* work, double* u, void* stream);

/*
 * Kernel-shape options of a plan.  The paper has no counterpart: an option
 * chooses between launch shapes that compute the same thing (up to rounding
 * order), and defaults are picked per plan from the problem size.
 *   CFS_OPT_THOMAS_TILE  columns per shared-memory tile of the z sweeps of
 *       Eq. 12: 0 automatic (the default), 8 or 16, or -1 for the streaming
 *       kernel (one thread per column, rows through registers, the forward
 *       sweep's intermediate written to the spectrum and read back).  Tiles
 *       apply to FP64 sweeps only: the FP32 sweeps of refined plans stream
 *       (grouped solves have no tile variant, and a box gives the same bits
 *       grouped as alone), and get_option reports their shape.  Or, for
 *       the FP32 solves of CFS_F32_REFINED plans with Nz <= 512, 1: Algorithm 2
 *       (Sec. 2.2.4) over z-partitions of 8 rows in registers, the rows of
 *       Eq. 12 formed on the fly (the spectrum read and written once; the
 *       plan's FP64 sweeps then stream).  1 on an FP64 plan, or with Nz > 512,
 *       is CFS_EUNSUPPORTED.
 *   CFS_OPT_X_LINES  x-lines per CTA of the x transforms: 0 automatic (about
 *       16 KB of data per buffer) or 1..64.
 *   CFS_OPT_Y_TILE  complex columns per y-transform tile (of the precision the
 *       solves transform in): 0 automatic or 1..32 (even for refined plans).
 *   CFS_OPT_PCR_PARTS  z-partitions of Algorithm 2 for Helmholtz sets that
 *       are prepared without an explicit count: 0 automatic (about 32 rows
 *       per partition) or 1..64, each partition at least 3 rows.
 *   CFS_OPT_HELM_FP64  CFS_F32_REFINED plans: 1 solves Helmholtz by FP64
 *       Algorithm 2 directly (no refinement; its error is that of the FP64
 *       path, below the refinement target), 0 (default) refines FP32 solves.
 *       On hardware where FP64 is scarce the refinement's FP64 Helmholtz
 *       residual costs as much as the FP64 solve itself, so the tuner may
 *       pick 1.
 *   CFS_OPT_HELM_THOMAS  1: the FP64 Helmholtz solves of Eq. 11 run as one
 *       Thomas sweep per (x, y) column (factors of I - c L_z computed once per
 *       (c, loc), 3 FP64 instructions per unknown, the intermediate through
 *       memory); 0 (default): Algorithm 2.  Both are exact direct methods.
 *   CFS_OPT_HELM_THOMAS32  the same choice for the FP32 inner Helmholtz solves
 *       of CFS_F32_REFINED plans.
 *   CFS_OPT_FFT_RADIX  largest radix of the Stockham passes of the x and y
 *       transforms: 8 (0 or 8, the default: radix-8 passes, then 4, 2, 3s) or
 *       4 (radix-4 passes, then 2, 3s).  Setting it rebuilds the twiddle
 *       tables (it waits for the device); groups bound to the plan must be
 *       rebound.
 *   CFS_OPT_F64_ADDS_X, CFS_OPT_F64_ADDS_Y  how many kinds of butterfly
 *       additions of the FP64 x / y transforms run on the integer units
 *       instead of the FP64 pipe, 0..4 (cumulative: 1 the second level of
 *       every radix-4 core, 2 also the radix-2 combination of each DFT8,
 *       3 also the first level of the untwiddled passes, 4 also the real-FFT
 *       untangle of the x transform).  Those additions are exact IEEE-754
 *       binary64 round-to-nearest-even additions done in integer
 *       arithmetic, so every level gives the same bits; on GPUs whose FP64
 *       pipe is narrow it lets the integer units share the FP64 work.
 *   CFS_OPT_STREAM_CHUNKS  chunks in which cfs_solve_batch_host moves each
 *       field of an FP64 plan: 0 automatic (about 200 MB per chunk, at most
 *       8), 1 whole fields, or 2..8.  A Poisson field moves in ranges of z
 *       planes (its x transforms run range by range as the data lands and
 *       leaves), a Helmholtz field solved by Algorithm 2 in ranges of y rows;
 *       the results are the same bits for every value.  get_option reports
 *       the count a Poisson field of the plan takes.
 * cfs_plan_set_option returns CFS_EINVAL for an unknown option or value, and
 * CFS_EUNSUPPORTED if the value cannot run at this plan's size (a tile that
 * does not fit in shared memory).  cfs_plan_get_option reports the value in
 * effect, with automatic choices resolved (for CFS_F32_REFINED plans, the
 * choice of the FP32 inner solve).
 */
enum {
  CFS_OPT_THOMAS_TILE = 1,
  CFS_OPT_X_LINES = 2,
  CFS_OPT_Y_TILE = 3,
  CFS_OPT_PCR_PARTS = 4,
  CFS_OPT_HELM_FP64 = 5,
  CFS_OPT_HELM_THOMAS = 6,
  CFS_OPT_HELM_THOMAS32 = 7,
  CFS_OPT_FFT_RADIX = 8,
  CFS_OPT_F64_ADDS_X = 9,
  CFS_OPT_F64_ADDS_Y = 10,
  CFS_OPT_STREAM_CHUNKS = 11
};
int cfs_plan_set_option(cfs_plan_t plan, int option, int value);
int cfs_plan_get_option(cfs_plan_t plan, int option, int* value);

/*
 * cfs_plan_autotune -- choose the options above for this plan by timing the
 * candidates of each on the GPU (CUDA events on `stream`, the plan's own work
 * fields as scratch) and set the fastest.  Results are kept per process for
 * the plan's (nx, ny, nz, dtype), so later plans of that size take them
 * without timing.  The paper has no counterpart.  Solves on the plan must not
 * run meanwhile; the plan's cached Helmholtz sets are kept.
 */
int cfs_plan_autotune(cfs_plan_t plan, void* stream);

/*
 * The tuner's remembered choices across processes (no counterpart in the
 * paper).  cfs_autotune_save writes every choice of this process to a text
 * file at `path`, one line per (nx, ny, nz, dtype) with the name of the GPU
 * it was measured on.  cfs_autotune_load reads such a file and takes the
 * lines measured on a GPU of the current device's name (choices this
 * process already holds are kept); *loaded (may be null) receives the number
 * taken.  A taken choice is checked against the plan it is applied to (tile
 * sizes, shared memory) and timed afresh if it does not fit.  Both return
 * CFS_EINVAL if the file cannot be opened or a line is malformed (lines
 * before it are taken).  cfs_autotune_clear forgets every choice.
 */
int cfs_autotune_save(const char* path);
int cfs_autotune_load(const char* path, int* loaded);
int cfs_autotune_clear(void);

/*
 * cfs_selfcheck_conversions -- a diagnostic with no counterpart in the paper.
 * The refinement kernels convert between FP32 and FP64 on the integer units
 * (the hardware conversions share the scarce FP64 pipe); this runs `samples`
 * hashed operands (any double, exact rounding ties, binary32 subnormal
 * results and their ties, any float, float subnormals, and the double-float
 * split hi = fl32(x), lo = fl32(x - hi) of doubles in the binary32 range)
 * through both and reports in *mismatches how many results differ in any
 * bit (0 expected; NaN results compare equal whatever their payload, and a
 * lo below the normal binary32 range is not compared: the split returns 0).
 */
int cfs_selfcheck_conversions(unsigned long long samples, unsigned long long* mismatches);

/*
 * cfs_selfcheck_f64_addsub -- a diagnostic with no counterpart in the paper.
 * The FP64 x and y transforms may run part of their butterfly additions in
 * integer arithmetic (CFS_OPT_F64_ADDS_X / _Y): an exact IEEE-754 binary64
 * round-to-nearest-even a + b and a - b, with zeros, subnormals, operands
 * below 2^-959 or from 2^1023 up, infinities and NaNs left to the FP64
 * pipe.  This runs `samples` hashed operand pairs (any two bit patterns,
 * close and distant exponents, cancellation, exact rounding ties, the ends
 * of the integer range, equal magnitudes, FFT-sized values) through both on
 * the GPU (on_device = 1) or on the host CPU (on_device = 0, no GPU needed)
 * and reports in *mismatches how many of the 2 * samples results differ in
 * any bit (0 expected; NaN results compare equal whatever their payload).
 */
int cfs_selfcheck_f64_addsub(unsigned long long samples, int on_device,
                             unsigned long long* mismatches);

/*
 * cfs_f64_addsub_host -- a diagnostic with no counterpart in the paper: the
 * same integer-unit FP64 addition and subtraction, evaluated on the host CPU
 * for caller-chosen operands, s[i] = a[i] + b[i] and d[i] = a[i] - b[i]
 * (i < n).  All four pointers are HOST arrays of n doubles (s, d written);
 * n = 0 does nothing.  No GPU is needed.
 */
int cfs_f64_addsub_host(long long n, const double* a, const double* b, double* s, double* d);

/*
 * cfs_probe_fma -- a measurement with no counterpart in the paper: the FMA
 * rate of the current GPU in FP64 (bits = 64) or FP32 (bits = 32), the
 * roofline peak of kernels bound by those instructions.  Every thread of one
 * full wave of 256-thread blocks (as many per SM as fit, at most 8) runs 16
 * independent FMA chains for `iters` steps (1 <= iters <= 2^40); after one
 * shorter warm-up launch the timed launch is measured with CUDA events on
 * the legacy default stream.
 * *fma_per_s receives FMAs per second, *ms (may be NULL) the launch time.
 * Waits for the device.
 */
int cfs_probe_fma(int bits, long long iters, double* fma_per_s, double* ms);

/*
 * cfs_probe_addsub -- a measurement with no counterpart in the paper: the
 * rate of FP64 butterfly pairs (a + b, a - b) on the FP64 pipe
 * (on_integer_units = 0) or by the integer-unit additions of the transforms
 * (1).  Every thread of one full wave of 256-thread blocks runs 8
 * independent pair chains for `iters` steps (rounded up to a multiple of
 * 256; 1 <= iters <= 2^40), timed as cfs_probe_fma.  *pairs_per_s receives
 * pairs per second, *ms (may be NULL) the launch time.  Waits for the device.
 */
int cfs_probe_addsub(int on_integer_units, long long iters, double* pairs_per_s, double* ms);

/*
 * cfs_selftest_wait_timeout -- a test of the failure path, with no
 * counterpart in the paper.  Every kernel that waits for asynchronous copies
 * waits a bounded number of polls; when the bound runs out it records
 * CFS_ETIMEOUT's bit in the status word, waits once more (bounded) for the
 * copies still in flight and exits without storing.  This queues, on
 * `stream`, 4 CTAs that go through that same path with `polls` polls
 * (1 <= polls <= 2^20) on a barrier that no copy completes (no copy is
 * issued).  The bit lands in the plan's status word (read by cfs_plan_check)
 * when plan is given, else in the caller's device int `device_status`
 * (exactly one of the two).  The device stays usable.
 */
int cfs_selftest_wait_timeout(cfs_plan_t plan, int* device_status, unsigned polls, void* stream);

/*
 * cfs_plan_check -- wait for the device and report device-side failures
 * recorded since the last check (then clear them).  *device_error (may be
 * NULL) receives the raw failure bits.  Returns CFS_ETIMEOUT if a bounded
 * wait inside a kernel ran out, CFS_ECUDA if the device reported an error.
 */
int cfs_plan_check(cfs_plan_t plan, int* device_error);

/*
 * cfs_plan_check_guards -- a stand-in for a device memory checker (no
 * counterpart in the paper).  The work buffers of a plan that its kernels
 * write (the factor tables of Eq. 12, the FP32 fields and the reduction
 * scratch of refined plans) are allocated with 256 bytes of a fixed pattern
 * before and after them.  This waits for the device and compares every
 * pattern; *damaged (may be NULL) receives the number of buffers with an
 * overwritten guard.  Returns CFS_EGUARD if there is one, else CFS_OK.
 * cfs_plan_debug_guard_poke overwrites one byte of buffer `buffer`'s leading
 * (tail = 0: the byte just before the buffer) or trailing (tail != 0: the
 * byte just after it) guard with a host-side memset, for tests of the check;
 * CFS_EINVAL if the plan has no such buffer.
 */
int cfs_plan_check_guards(cfs_plan_t plan, int* damaged);
int cfs_plan_debug_guard_poke(cfs_plan_t plan, int buffer, int tail);

#ifdef __cplusplus
}
#endif
#endif /* CHANFS_H */
