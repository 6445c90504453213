/*
 * chanfs_oracle.h -- plain single-threaded FP64 reference implementation
 * ("oracle") of the pressure-Poisson and wall-normal implicit-diffusion
 * Helmholtz solves of Diez, Peeters & Costa, "A pencil-distributed
 * finite-difference solver for extreme-scale calculations of turbulent wall
 * flows at high Reynolds number" (arXiv 2502.06296).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * shares no code, header, table or helper with it.
 *
 * Conventions (shared by every function below):
 *  - Fields are Nx*Ny*Nz doubles, x fastest: f[x + Nx*(y + Ny*z)].
 *  - Complex arrays are interleaved (re, im) doubles.
 *  - Forward DFT: X_k = sum_j x_j exp(-2 pi i j k / n); inverse has +i and 1/n.
 *  - z grid: dzf[k] (k = 0..Nz-1) are the cell widths between faces z_f[k] and
 *    z_f[k+1]; cell centres are face midpoints.
 *  - bc: 0 = homogeneous Neumann at both z walls, 1 = homogeneous Dirichlet.
 *  - loc: 0 = cell-centred unknowns (p, u, v), 1 = face-located unknowns (w);
 *    a face field stores w at face z_f[k+1] in slot k, slot Nz-1 is the top
 *    wall and is returned as 0.
 *  - Return value: 0 on success, negative on invalid arguments.
 */
#ifndef CHANFS_ORACLE_H
#define CHANFS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Discrete Fourier transforms (Sec. 2.2.1 "Fourier-based synthesis"). */
int or_dft_naive(int n, const double* in, double* out, int sign);
int or_fft(int n, const double* in, double* out, int sign);

/* Appendix A packed real-to-complex format (Eqs. A.1-A.3). */
int or_rfft_packed(int n, const double* x, double* packed);
int or_irfft_packed(int n, const double* packed, double* x);
int or_packed_wavenumber(int n, int slot);

/* Modified wavenumbers lambda_i / dx^2 of Eq. (12), natural and packed order. */
int or_eig_periodic(int n, double h, double* lam);
int or_eig_packed(int n, double h, double* lam);

/* Stretched-grid metrics and the tridiagonal z stencil (eta of Eq. (12)). */
int or_dzc(int nz, const double* dzf, double* dzc);
int or_lz_coefficients(int nz, const double* dzf, int bc, int loc,
                       double* A, double* B, double* C);

/* Tridiagonal solvers for Eq. (13): a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k;
 * Algorithms 1 and 2 of Sec. 2.2.4. */
int or_thomas(int n, const double* a, const double* b, const double* c,
              const double* d, double* x);
int or_alg1_solve(int n, int p, const double* a, const double* b,
                  const double* c, const double* d, double* x);
int or_alg2_prepare(int m, const double* A, const double* B, const double* C,
                    double* a, double* b, double* c);
int or_alg2_runtime(int m, const double* A, const double* C, const double* b,
                    double* d);
int or_alg2_reconstruct(int m, const double* a, const double* b,
                        const double* c, double x0, double xm1, double* d);
int or_alg2_solve(int n, int p, const double* A, const double* B,
                  const double* C, const double* d, double* x);

/* 3-D operators (Sec. 2.1 staggered second-order discretisation). */
int or_apply_poisson(int nx, int ny, int nz, double lx, double ly,
                     const double* dzf, int bc, const double* p, double* out);
int or_apply_helmholtz(int nx, int ny, int nz, const double* dzf, double c,
                       int loc, const double* u, double* out);

/* Solvers: Poisson by Eq. (12); z-implicit Helmholtz of Eq. (11). */
int or_poisson_solve(int nx, int ny, int nz, double lx, double ly,
                     const double* dzf, int bc, const double* f, double* p);
int or_helmholtz_solve(int nx, int ny, int nz, const double* dzf, double c,
                       int loc, int method, int nparts, const double* rhs,
                       double* u);
/* Walls in y (ybc 0 periodic, 1 Neumann, 2 Dirichlet; cell-centred): the
 * DCT-II / DST-II and inverses by their definitions, the wall eigenvalues,
 * the operator and the Poisson solve. */
int or_dct2(int n, const double* x, double* X);
int or_idct2(int n, const double* X, double* x);
int or_dst2(int n, const double* x, double* X);
int or_idst2(int n, const double* X, double* x);
int or_eig_wall(int n, double h, int ybc, double* lam);
int or_apply_poisson_walls(int nx, int ny, int nz, double lx, double ly, const double* dzf,
                           int bc, int ybc, const double* p, double* out);
int or_poisson_solve_walls(int nx, int ny, int nz, double lx, double ly, const double* dzf,
                           int bc, int ybc, const double* f, double* p);

/* Fully implicit 3-D Helmholtz (Eq. 8), Dirichlet z walls: apply and solve. */
int or_apply_helmholtz3d(int nx, int ny, int nz, double lx, double ly,
                         const double* dzf, double c, int loc, const double* u,
                         double* out);
int or_helmholtz3d_solve(int nx, int ny, int nz, double lx, double ly,
                         const double* dzf, double c, int loc, const double* rhs,
                         double* u);
/* The same with walls in y (ybc 0 periodic, 1 Neumann, 2 Dirichlet). */
int or_apply_helmholtz3d_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc, const double* u,
                               double* out);
int or_helmholtz3d_solve_walls(int nx, int ny, int nz, double lx, double ly,
                               const double* dzf, double c, int loc, int ybc,
                               const double* rhs, double* u);

/* Spectral layout used by the solver: App. A packing along x, complex DFT
 * along y (pair j of a packed x-line read as one complex number), and pair 0
 * (F(0,ky) + i F(Nx/2,ky)) stored untangled by the same packing along y. */
int or_spectral_forward(int nx, int ny, int nz, const double* f, double* s);
int or_spectral_inverse(int nx, int ny, int nz, const double* s, double* f);

/* Dense LU with partial pivoting; A is n*n row-major, b overwritten by x. */
int or_dense_solve(int n, double* A, double* b);

#ifdef __cplusplus
}
#endif
#endif
