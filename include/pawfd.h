/*
 * pawfd.h -- C ABI of the GB300 (sm_103a) real-space PAW eigensolver-step library.
 *
 * The library applies the PAW Hamiltonian and overlap operators of Eq. (dh) of the PAW
 * section of the paper (arXiv 2310.14776),
 *
 *     H = -1/2 nabla^2 + v(r) + sum_a sum_ii' |p_i^a> dH^a_ii' <p_i'^a|
 *     S = 1               + sum_a sum_ii' |p_i^a> dS^a_ii' <p_i'^a|,
 *
 * to a block of wave functions on a uniform periodic grid (the finite-difference mode of
 * the wave-function section: the kinetic operator is a stencil on a uniform Cartesian
 * grid, here the order-6 central second difference), and performs the subspace
 * diagonalization that opens each SCF step (Kohn-Sham section, step 1) with a dense
 * Cholesky and eigensolver (parallelization section).  The generalized eigenproblem is
 * H psi = eps S psi (PAW section, the PAW form of the Kohn-Sham equations).
 *
 * Conventions shared by every entry point
 *   - Return value: PAWFD_OK (0) or a negative PAWFD_E* code; pawfd_last_error() gives text.
 *     No exception crosses this boundary.
 *   - Grid arrays are [band][i3][i2][i1] with i1 (x) fastest, bands contiguous with stride
 *     K = N1*N2*N3 elements.  Complex data is interleaved (re, im).
 *   - Array arguments are DEVICE pointers owned by the caller unless marked "host".  The
 *     library never frees caller memory.  It owns only what pawfd_create allocates
 *     (projector tables, the shifted local potential, scratch), released by pawfd_destroy.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous; a device-side
 *     failure (Cholesky pivot, eigensolver sweep cap, bounded wait) is recorded in the
 *     context and returned by pawfd_sync() (and by the next call that synchronizes).
 *   - Inputs and outputs may not alias unless stated.
 *   - A NULL context (or batch) is checked before anything else and touches no device:
 *     calls returning int give PAWFD_EINVAL, pawfd_nproj_total and pawfd_launch_count give
 *     PAWFD_EINVAL, pawfd_batch_is_graph and pawfd_batch_kernel_count give 0, and
 *     pawfd_last_error / pawfd_batch_last_error give a fixed text.
 */
#ifndef PAWFD_H
#define PAWFD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pawfd_ctx pawfd_ctx;

/* wave-function storage / arithmetic type of the band arrays and projections.
 * Gram matrices, eigenvalues and eigenvectors (C) are always FP64: double for the real
 * types, interleaved complex double for the complex types.  The FP32 types are the mixed
 * form: stencil, projections and back-add in FP32 arithmetic; Gram matrices and rotations as
 * exact products of BF16 digits of the FP32 values on the tensor cores (4 digits per value,
 * the products accumulated to about FP64 accuracy; with the option tensor_cores = 0, FP32
 * products instead); subspace solve in FP64. */
enum {
  PAWFD_R64 = 0,  /* real double, Gamma point (k must be 0)         */
  PAWFD_C128 = 1, /* complex double, Bloch vector k                  */
  PAWFD_R32 = 2,  /* real float, Gamma point (k must be 0)          */
  PAWFD_C64 = 3   /* complex float, Bloch vector k                   */
};

/* error codes */
enum {
  PAWFD_OK = 0,
  PAWFD_EINVAL = -1,    /* bad argument (size, pointer, layout)                          */
  PAWFD_ENOMEM = -2,    /* device allocation in pawfd_create failed                       */
  PAWFD_ENOTPD = -3,    /* S_nm not positive definite: Cholesky pivot <= 0 (column in text) */
  PAWFD_ENOCONV = -4,   /* Jacobi eigensolver hit its sweep cap                           */
  PAWFD_ETIMEDOUT = -5, /* a bounded device-side wait gave up                             */
  PAWFD_EDEVICE = -6    /* CUDA runtime error (text from the runtime)                     */
};

/* One periodic orthorhombic cell.  All pointers here are HOST pointers, read during
 * pawfd_create only (the library copies what it needs to the device).
 *
 * Projector p_i^a sampled on its box: the box of atom a covers the unwrapped grid indices
 * box_lo[a][c] .. box_lo[a][c] + box_n[a][c] - 1 along axis c (x, y, z); an unwrapped index
 * u stands for grid point u mod N_c in the cell translated by floor(u / N_c) * L_c, so boxes
 * may cross faces and may even be larger than the cell.  proj holds, for atom a starting
 * at proj_off[a], the values [I_a][box_n z][box_n y][box_n x].  dH and dS hold, for atom a
 * starting at dmat_off[a], the real symmetric I_a x I_a matrices dH^a and dS^a (row-major). */
typedef struct {
  int n[3];                 /* grid points N1, N2, N3 (x, y, z), each >= 1                   */
  double cell[3];           /* cell lengths L_c (bohr); spacing h_c = L_c / N_c              */
  double k[3];              /* Bloch vector (1/bohr); must be 0 for PAWFD_R64                */
  int dtype;                /* PAWFD_R64, PAWFD_C128, PAWFD_R32 or PAWFD_C64                 */
  int max_bands;            /* largest nb any later call will use (sizes the scratch)        */
  int natoms;               /* A >= 0                                                        */
  const int* nproj;         /* [A] I_a >= 1                                                  */
  const int* box_lo;        /* [A][3]                                                        */
  const int* box_n;         /* [A][3], each >= 1                                             */
  const double* proj;       /* concatenated projector boxes                                  */
  const long long* proj_off;/* [A+1]                                                         */
  const double* dH;         /* concatenated dH^a                                             */
  const double* dS;         /* concatenated dS^a                                             */
  const long long* dmat_off;/* [A+1]                                                         */
  const double* vloc;       /* [N3][N2][N1] local potential v(r) (Hartree)                   */
} pawfd_system_desc;

/* Create a context for one system; stream is a cudaStream_t (NULL = legacy default stream).
 * On success *out owns device tables sized for max_bands bands.  The description is checked
 * on the host before any CUDA call; PAWFD_EINVAL (with *out = NULL and the reason on stderr)
 * for a NULL out or desc, a grid size < 1 or above 2^31 - 1 points, a cell length <= 0, an
 * unknown dtype, a real dtype with k != 0, max_bands < 1, a NULL vloc, natoms < 0, missing
 * atom arrays, nproj outside 1..32, a box size < 1, or proj_off / dmat_off offsets that do
 * not match the box sizes and nproj.  PAWFD_ENOMEM or PAWFD_EDEVICE for device failures. */
int pawfd_create(pawfd_ctx** out, const pawfd_system_desc* desc, void* stream);
int pawfd_destroy(pawfd_ctx* ctx);
int pawfd_set_stream(pawfd_ctx* ctx, void* stream);

/* Wait for the context's stream; returns the first device-side error recorded since the
 * last pawfd_sync (and clears it), or PAWFD_OK. */
int pawfd_sync(pawfd_ctx* ctx);
const char* pawfd_last_error(const pawfd_ctx* ctx);

/* number of projector rows Ip = sum_a I_a */
int pawfd_nproj_total(const pawfd_ctx* ctx);

/* number of CUDA kernels this context has launched so far (host-side counter) */
long long pawfd_launch_count(const pawfd_ctx* ctx);

/* CUDA-event timing of the tensor-core Gram MMA kernel launches (pawfd_gram_hs, pawfd_gram,
 * pawfd_gram_hermitian and the steps built on them: each MMA kernel launch of a K block is
 * bracketed by a pair of events on the context's stream, up to 1024 launches between two
 * calls).  Returns, through total_ms and launches, the summed device time and the number of
 * timed launches since the previous call (launches = -1 if more than 1024 were made),
 * waiting for the last one; then turns timing on (enable = 1) or off. */
int pawfd_kernel_timing(pawfd_ctx* ctx, int enable, double* total_ms, long long* launches);

/* Select among equivalent implementations (for tests and measurements):
 *   "tensor_cores"    1 (default): Gram matrices and rotations on the tensor cores with exact
 *                     digit slices; 0: FMA kernels on the CUDA cores (FP64 products for the FP64
 *                     dtypes; FP32 products, about 1e-7 relative, for the FP32 dtypes).
 *   "stencil_variant" 0 (default): fastest kernel that applies to the shape; 1: skip the
 *                     bulk-copy ring kernels (FP32 real and FP32 complex); 2: always the
 *                     general kernel.
 *   "stencil_rows"    y rows per CTA of the bulk-copy ring kernels, 0 (default) automatic,
 *                     at most 64 (clamped further by the kernel's thread and memory limits).
 *   "stencil_yblock"  y rows per thread of the ring kernels: 0 (default) automatic, 1, 2 or 3.
 *   "stencil_ring"    ring kernels: planes in flight + in use, 0 (default: 8 for FP32 real, 6
 *                     for FP32 complex), 6, 8, 10 or 12 (the complex kernel takes 6 or 8, the
 *                     real one 8, 10 or 12; other values round to the nearest it takes).
 *   "stencil_zsplit"  general stencil kernel: the z range is split so that one launch has at
 *                     least this many CTAs per SM; 0 (default) means 4, at most 64.
 *   "tc_kblk"         tensor-core Gram: grid values per K block in units of 512 (0: the whole
 *                     slice buffer, 256 units); shorter blocks keep the digit slices in L2.
 *   "tc_scratch_mb"   size of the tensor-core digit-plane scratch, in MB: the Gram's K block is
 *                     as long as the planes of both operands fit in it, and the rotation's block
 *                     of grid points as long as their planes fit in it (0, the default: K
 *                     blocks of 256 x 512 values and rotation blocks of 512 MB).  Larger blocks
 *                     mean fewer launches and better balance across SMs at the cost of memory.
 *                     Waits for the context's stream, then frees and re-allocates the scratch;
 *                     on an allocation failure returns PAWFD_ENOMEM and turns the tensor-core
 *                     path off.
 *   "stencil_fx"      1 (default): the FP64 stencil (real bands, and complex Bloch bands in
 *                     16-byte aligned arrays) computes the order-6 sums exactly in 64-bit
 *                     integers on the band slab's FP64 grid (inputs rounded once to that grid,
 *                     Bloch factors of wrapped neighbours applied before that rounding, the
 *                     integer sum rounded once to FP64), the FP64 pipe only for the scaling
 *                     and v psi; 0: FP64 arithmetic.  "stencil_variant" 2 also selects FP64.
 *   "nonlocal_df"     1 (default): for real FP64 bands the projections and the nonlocal
 *                     back-add compute in double-float FP32 pairs (runs of 32 terms, then FP64
 *                     sums); 0: FP64 arithmetic.
 *   "jacobi_cluster"  0 (default): the Cholesky factorization and the Jacobi eigensolver run as
 *                     cooperative grids with a bounded software grid barrier; 1: on one
 *                     thread-block cluster (hardware cluster barrier) when their work fits 16 CTAs.
 *   "davidson_precond"  1 (default): pawfd_davidson_step forms its corrections with the kinetic
 *                     preconditioner of pawfd_kinetic_precond when every grid size factors into
 *                     2, 3 and 5 (the Jacobi one otherwise); 0: always the Jacobi preconditioner
 *                     of pawfd_residual_precond.
 *   "tridiag_dsm"     1 (default): the FP32 tridiagonal reduction of the subspace solve's far
 *                     path keeps the matrix in the distributed shared memory of one 16-CTA
 *                     cluster when it fits (n <= 512 complex, n <= 724 real); 0: in global
 *                     memory (L2), the form used for larger n.
 *   "test_barrier_missing"  0 (default); 1 (for tests of the error path only): the grid
 *                     barriers of the subspace solve wait for one CTA more than the launch has
 *                     and give up after 20 ms, so every such wait runs out: the kernels record
 *                     PAWFD_ETIMEDOUT, later kernels of the context return without work, and
 *                     pawfd_sync reports it.  Waits for the context's stream first.
 * Returns PAWFD_EINVAL for an unknown name or value. */
int pawfd_set_option(pawfd_ctx* ctx, const char* name, int value);

/* Projector overlaps P[i][n] = <p_i^a | psi_n> = dV sum_r conj(p_i^a(r)) psi_n(r), for
 * every atom a and projector i (global row i), n < nb.  Bloch phases exp(i k.T) of the
 * lattice translation T of each box point are applied (projector overlaps of the PAW
 * section; the atomic density matrix is built from them).
 *   psi: [nb][K] (dtype of the context);  P: [Ip][nb] (same dtype). */
int pawfd_project(pawfd_ctx* ctx, const void* psi, int nb, void* P);

/* hpsi = H psi for nb bands (Eq. (dh)).  If P_out is not NULL it receives the projections
 * of psi ([Ip][nb]); otherwise the context's scratch holds them.  psi, hpsi: [nb][K]. */
int pawfd_apply_H(pawfd_ctx* ctx, const void* psi, int nb, void* hpsi, void* P_out);

/* spsi = S psi for nb bands (PAW overlap operator).  P_out as for pawfd_apply_H. */
int pawfd_apply_S(pawfd_ctx* ctx, const void* psi, int nb, void* spsi, void* P_out);

/* The kinetic + local part alone: out = -1/2 Lap_FD psi + v psi (the finite-difference
 * stencil hot spot of the development section, fused with the local potential). */
int pawfd_apply_kinetic_local(pawfd_ctx* ctx, const void* psi, int nb, void* out);

/* Gram matrix M[n][m] = dV sum_r conj(A_n(r)) B_m(r), n, m < nb; A, B band arrays of the
 * context's dtype; M is [nb][nb] FP64 (double, or interleaved complex double for the complex
 * dtypes).  With B = H psi this is the
 * subspace Hamiltonian H_nm, with B = S psi the subspace overlap S_nm. */
int pawfd_gram(pawfd_ctx* ctx, const void* A, const void* B, int nb, void* M);

/* Hermitian Gram matrix for B = X A with X Hermitian (X = H or S, so that A^H X A is
 * Hermitian): computes M[n][m] = dV sum_r conj(A_n(r)) B_m(r) for n <= m only (tiles on or
 * above the diagonal, about half the work of pawfd_gram), sets M[m][n] = conj(M[n][m]) and
 * makes the diagonal exactly real.  Arguments and layout as pawfd_gram. */
int pawfd_gram_hermitian(pawfd_ctx* ctx, const void* A, const void* B, int nb, void* M);

/* H psi and S psi for nb bands with one set of projections (Eq. (dh) and the PAW overlap
 * operator; the projections of psi are computed once and serve both nonlocal terms).  If
 * P_out is not NULL it receives the projections ([Ip][nb]); otherwise the context's scratch
 * holds them.  psi, hpsi, spsi: [nb][K], pairwise distinct.  Asynchronous like the calls
 * above. */
int pawfd_apply_HS(pawfd_ctx* ctx, const void* psi, int nb, void* hpsi, void* spsi, void* P_out);

/* The two Gram matrices of the subspace step (SCF step 1 of the Kohn-Sham section):
 *   Hnm = dV psi^H (H psi)                         (as pawfd_gram_hermitian with B = H psi)
 *   Snm = dV psi^H psi + sum_a P_a^H dS^a P_a      (the PAW overlap <psi_n|S|psi_m>, its
 *                                                    projector term from the projections P)
 * P: the projections of psi ([Ip][nb], as written by pawfd_project / pawfd_apply_HS; may be
 * NULL only when the context has no atoms).  With the tensor-core contraction the digits of
 * psi are made once and serve both matrices.  Since H is Hermitian, some entries of Hnm may be
 * formed from the mirrored product ((H psi)_m^H psi_n conjugated, or psi_m^H (H psi)_n): equal
 * in exact arithmetic, with H psi in FP32 they differ at the FP32 level.  Hnm, Snm: [nb][nb]
 * FP64 of the context's kind, Hermitian (mirrored, real diagonal); they may not alias.
 * Asynchronous. */
int pawfd_gram_hs(pawfd_ctx* ctx, const void* psi, const void* hpsi, int nb, const void* P, void* Hnm, void* Snm);

/* Subspace diagonalization: given Hermitian H_nm and positive definite S_nm ([nb][nb],
 * FP64 of the context's kind: double or interleaved complex double), solve H C = S C diag(eps): symmetrize, S = L L^H, A = L^-1 H L^-H,
 * Jacobi A = U diag(eps) U^H, C = L^-H U.  eps (double [nb]) ascending with stable ties;
 * each column of C (FP64 of the same kind, [nb][nb], column m = eigenvector m) is S-normalized and
 * multiplied by a unit phase that makes its largest-magnitude entry (first on ties) real
 * and positive.  Hnm and Snm are overwritten (workspace).  Failures (PAWFD_ENOTPD with the
 * failing column, PAWFD_ENOCONV) are reported by pawfd_sync. */
int pawfd_subspace_diag(pawfd_ctx* ctx, int nb, void* Hnm, void* Snm, double* eps, void* C);

/* Band rotation psi_out_m = sum_n psi_n C[n][m] (the rotation that completes the subspace
 * diagonalization).  psi, psi_out: [nb][K] of the context's dtype; C: [nb][nb] FP64 (as
 * returned by pawfd_subspace_diag); psi_out must not alias psi.  With the tensor-core path
 * (the default) psi and C enter as exact sums of scaled BF16 digits (all 53 / 24 bits of
 * psi, C to at least 26 bits for the FP32 dtypes) and each output is accumulated to about
 * FP64 accuracy before the final rounding to the context's dtype. */
int pawfd_rotate(pawfd_ctx* ctx, const void* psi, int nb, const void* C, void* psi_out);

/* The band rotation onto the first nout columns of C: psi_out_m = sum_n psi_n C[n][m] for
 * m < nout (C: [nb][nb] FP64 of the context's kind; psi_out: [nout][K]).  nout = nb is
 * pawfd_rotate.  Returns PAWFD_EINVAL for nout outside 1..nb and as pawfd_rotate otherwise. */
int pawfd_rotate_n(pawfd_ctx* ctx, const void* psi, int nb, const void* C, int nout, void* psi_out);

/* Residuals of the generalized eigenproblem H psi = eps S psi (PAW section) and their
 * preconditioned corrections, as used by the iterative eigensolver (SCF step 2 of the
 * Kohn-Sham section; the paper names the Davidson method without its steps, so this is a
 * reading):
 *   R_n(r) = hpsi_n(r) - eps[n] spsi_n(r)               (the band's arithmetic),
 *   rnorm[n] = sqrt(dV sum_r |R_n(r)|^2)                  (FP64 sums in a fixed order),
 *   pr_n(r) = -R_n(r) / max(d(r) - eps[n], d0 / 10)      (weights in FP32),
 * with d(r) = v(r) + d0 the diagonal of the kinetic + local operator and d0 =
 * -1/2 c0 sum_c 1/h_c^2 the stencil's centre weight (a Jacobi preconditioner kept positive).
 * hpsi, spsi, pr: [nb][K] of the context's dtype (pr distinct from both); eps, rnorm: device
 * [nb] doubles.  Uses the subspace workspace of the context (no other call of the same
 * context may run concurrently). */
int pawfd_residual_precond(pawfd_ctx* ctx, const void* hpsi, const void* spsi, int nb, const double* eps, void* pr,
                           double* rnorm);

/* The kinetic preconditioner of the Davidson step (a reading: the paper names the Davidson
 * eigensolver without its preconditioner): out_n = -(T + sigma)^-1 R_n for every band, T the
 * order-6 FD kinetic operator of the grid with the Bloch condition, sigma = 0.5 Ha.  T is
 * diagonal on the grid's Bloch waves (symbol t(k+G) = -1/2 sum_c (w0 + 2 sum_m w_m cos(m q_c
 * h_c)) / h_c^2, q = k + G), so the solve is a forward FFT, a division and an inverse FFT on the
 * library's FFT kernels, in FP32 for every dtype (a search direction needs no more): two real
 * bands share one complex transform.
 *   R, out: [nb][K] band arrays of the context's dtype (out may be R); work: device scratch of
 *   8 K bytes per transform (ceil(nb / 2) transforms for real dtypes, nb for complex ones), not
 *   aliasing R or out.  The FFT tables are allocated by the first call (make it before any
 *   stream capture).  Returns PAWFD_EINVAL for nb outside 1..max_bands, null or aliased work,
 *   or a grid size with a prime factor other than 2, 3 and 5; PAWFD_ENOMEM if the tables cannot
 *   be allocated. */
int pawfd_kinetic_precond(pawfd_ctx* ctx, const void* R, int nb, void* out, void* work);

/* One block-Davidson step (the reading of the iterative eigensolver named in the Kohn-Sham
 * and parallelization sections; needs max_bands >= 2 nb):
 *   1. HX[0 .. nb) = H psi, SX = S psi for psi = X[0 .. nb) (Ritz vectors with Ritz values
 *      eps_in, e.g. from pawfd_rr_step or a previous step);
 *   2. X[nb .. 2nb) = the preconditioned corrections, rnorm the residual norms: the kinetic
 *      preconditioner of pawfd_kinetic_precond (its work in HX[nb .. 2nb), or for FP32 real
 *      bands and odd nb a context array allocated on first need) or, with option
 *      "davidson_precond" 0 or a grid size with another prime factor, the Jacobi corrections of
 *      pawfd_residual_precond;
 *   3. HX[nb .. 2nb) = H of the corrections; P = the projections of all 2 nb columns of X;
 *   4. Hnm, Snm = the Hermitian Gram matrices of X (as pawfd_gram_hs), scaled to a unit S
 *      diagonal (which leaves the Ritz values unchanged and keeps the factorization well
 *      conditioned when corrections are tiny), eps and C of their subspace diagonalization
 *      (2 nb Ritz pairs, ascending; C for the unscaled X; Hnm and Snm overwritten);
 *   5. psi_out = X C[:, 0 .. nb): the nb lowest Ritz vectors, with Ritz values eps[0 .. nb).
 * X, HX: [2 nb][K]; SX, psi_out: [nb][K] (context dtype, pairwise distinct); P: [Ip][2 nb];
 * Hnm, Snm, C: [2 nb][2 nb] FP64 of the context's kind; eps: [2 nb], rnorm: [nb] device
 * doubles.  All memory owned by the caller.  Errors as the individual calls. */
int pawfd_davidson_step(pawfd_ctx* ctx, void* X, int nb, const double* eps_in, void* HX, void* SX, void* P,
                        void* Hnm, void* Snm, double* eps, void* C, double* rnorm, void* psi_out);

/* The reductions that follow the eigensolver in the SCF loop (the density of step 4 of the
 * Kohn-Sham section; the PAW section's pseudo density and atomic density matrices), for one
 * spin channel and occupation numbers f (device [nb] doubles):
 *   rho[r] = sum_n f[n] |psi_n(r)|^2   (device [K] doubles; the pseudo density without
 *            compensation charges).  Real FP64 bands are summed in double-float FP32 pairs
 *            (about 2^-46 relative per term), complex FP64 bands in FP64, FP32 bands in FP32
 *            runs of 16 bands added in FP64.
 *   D[dmat_off[a] + i I_a + i'] = sum_n f[n] conj(P[row_a + i][n]) P[row_a + i'][n]
 *            (Eq. (atomicdensitymatrix): <psi_n|p_i^a><p_i'^a|psi_n> with P the projections
 *            of pawfd_project, row_a the atom's first projector row); FP64 (complex FP64 for
 *            the complex dtypes) in the packed per-atom layout of dH and dS.
 * Returns PAWFD_EINVAL for nb outside 1..max_bands or null arrays. */
int pawfd_density(pawfd_ctx* ctx, const void* psi, int nb, const double* f, double* rho);
int pawfd_atomic_density(pawfd_ctx* ctx, const void* P, int nb, const double* f, void* D);

/* The Hartree potential of a density (the Poisson solve of the potential update in the
 * Kohn-Sham section; the paper's solvers are Fourier-based or multigrid, this one iterates):
 * v solves lap_FD v = -4 pi (rho - <rho>) on the periodic grid with the order-6 Laplacian of
 * the kinetic stencil, i.e. T v = 2 pi (rho - <rho>) with T = -1/2 lap_FD, and has zero mean.
 * Conjugate gradients in FP64 (T applied by the stencil kernel of the context), stopped when
 * ||r|| <= tol ||b|| or after maxiter iterations (the residual is read every 25 iterations).
 *   ctx: a PAWFD_R64 context of a system with v = 0 and no atoms (the operator T alone);
 *   rho, v: device [K] doubles; work: device scratch of 4 K + 304 doubles;
 *   iters, resid (host, optional): iterations done and the final ||r|| / ||b||.
 * Returns PAWFD_EINVAL for another context, null arrays, tol <= 0 or maxiter < 1. */
int pawfd_poisson(pawfd_ctx* ctx, const double* rho, double* v, double tol, int maxiter, double* work, int* iters,
                  double* resid);

/* H and S in the plane-wave representation (the wave-function section writes a Bloch state
 * as psi_kn(r) = sum_G C_nG e^{i(k+G).r}; the paper's GPU port works in this representation).
 * This is a reading of the PW mode on the cell's FFT grid: G runs over the N1 x N2 x N3
 * frequencies of the grid, stored [nb][N3][N2][N1] in FFT order (index j_c for G_c = 2 pi f_c /
 * L_c, f_c = j_c for j_c < (N_c + 1) / 2, else j_c - N_c), and
 *   (H C)_G = |k+G|^2 / 2 C_G + [v psi + sum_a |p^a> dH^a <p^a|psi>]_G,
 *   (S C)_G = C_G + [sum_a |p^a> dS^a <p^a|psi>]_G,
 * with psi(r) = sum_G C_G e^{i(k+G).r} at the grid points and [f]_G = (1/K) sum_r
 * e^{-i(k+G).r} f(r): the kinetic operator is exact in this basis (not the finite-difference
 * stencil), v and the projector boxes are those of the context (Eq. (dh)).  ecut > 0 restricts
 * the basis to the sphere |k+G|^2 / 2 <= ecut (Hartree): the output is zero outside it (the
 * caller's C should be zero there too); ecut <= 0 keeps every G.
 *   ctx: a complex context (PAWFD_C128, or PAWFD_C64 for FP32 arithmetic), grid sizes with no
 *        prime factor other than 2, 3 and 5; the FFT tables (twiddles, e^{ik.r}, |k+G|^2 / 2) are
 *        allocated by the first plane-wave call on the context (it waits for the context's
 *        stream; make it before any stream capture);
 *   C, HC / SC: [nb][K] complex coefficients of the context's dtype; work: [2][nb][K] of the
 *        same dtype (psi on the grid and the local and nonlocal terms), all caller-owned and
 *        pairwise distinct.  The projections of psi are left in the context's scratch.
 * The Gram matrices of a plane-wave Rayleigh-Ritz step are those of pawfd_gram on the
 * coefficient arrays (they carry dV instead of the cell volume, a common factor K that leaves
 * the eigenvalues unchanged).  Returns PAWFD_EINVAL for a real context, another grid factor,
 * nb outside 1..max_bands, null or aliased arrays; PAWFD_ENOMEM if the tables cannot be
 * allocated.  Asynchronous like the calls above. */
int pawfd_pw_apply_H(pawfd_ctx* ctx, const void* C, int nb, double ecut, void* HC, void* work);
int pawfd_pw_apply_S(pawfd_ctx* ctx, const void* C, int nb, double ecut, void* SC, void* work);

/* The two representations of the same bands: psi(r) = sum_G C_G e^{i(k+G).r} at the grid
 * points (pawfd_pw_to_grid; C and psi [nb][K], distinct) and its inverse C_G = (1/K) sum_r
 * e^{-i(k+G).r} psi(r) (pawfd_pw_from_grid; work: [nb][K], a copy of psi that the transform
 * overwrites).  Arguments and errors as pawfd_pw_apply_H. */
int pawfd_pw_to_grid(pawfd_ctx* ctx, const void* C, int nb, void* psi);
int pawfd_pw_from_grid(pawfd_ctx* ctx, const void* psi, int nb, void* C, void* work);

/* The Hartree potential by the direct Fourier-transform route (the Kohn-Sham section names
 * direct solvers based on Fourier transforms as the default): the zero-mean v with
 * lap_FD v = -4 pi (rho - <rho>) for the order-6 Laplacian of the kinetic stencil, computed
 * as v(G) = -4 pi rho(G) / L(G) (G != 0; v(0) = 0) with L(G) the Laplacian's symbol
 * sum_c (w0 + 2 sum_m w_m cos(m G_c h_c)) / h_c^2 on the grid's FFT frequencies, on the
 * library's own FFT kernels (pawfd_pw_apply_H's); the same equation as pawfd_poisson solves
 * iteratively.
 *   ctx: a PAWFD_R64 context with v = 0 and no atoms, grid sizes with no prime factor other than
 *   2, 3 and 5 (the FFT tables and the K-point table of -4 pi / (K L(G)) are allocated by the
 *   first call; make it before any stream capture); rho, v: device [K] doubles; work: device
 *   scratch of K complex doubles (16 K bytes).  Returns PAWFD_EINVAL for another context, null
 *   or aliased arrays, another grid factor; PAWFD_ENOMEM if the tables cannot be allocated. */
int pawfd_poisson_fft(pawfd_ctx* ctx, const double* rho, double* v, void* work);

/* Final refinement of the mixed form (the paper is silent on it; this is the reading that
 * closes a mixed-precision eigensolver step).  ctx is an FP64 context (PAWFD_R64 or
 * PAWFD_C128) of the same system as the mixed context whose bands psi_lo (PAWFD_R32 or
 * PAWFD_C64 of the same kind, [nb][K], 16-byte aligned) are refined:
 *   1. psi = psi_lo promoted to FP64 (exact).  If C_lo is not NULL, psi_lo are the INPUT
 *      bands of a mixed Rayleigh-Ritz step and C_lo ([nb][nb] FP64 of the context's kind) the
 *      eigenvector matrix that step returned: then psi = psi_lo C_lo, rotated in FP64 (the
 *      digit-product rotation, accumulated to about FP64).  A nonsingular C_lo keeps the span
 *      of the input, so the refined eigenvalues are those of the FP64 step on the same input,
 *      while the bands are already near its Ritz vectors (the second solve is the cheap
 *      near-Ritz path).  If C_lo is NULL, psi_lo (e.g. rotated FP32 bands) are refined as given;
 *   2. hpsi = H psi and spsi = S psi in FP64 (Eq. (dh) and the overlap operator of the PAW
 *      section; one set of projections serves both);
 *   3. Hnm = dV psi^H hpsi, Snm = dV psi^H spsi (Hermitian Gram matrices, FP64);
 *   4. theta[n] = Re Hnm[n][n] / Re Snm[n][n] (FP64 Rayleigh quotients of the bands psi);
 *   5. a second subspace diagonalization of (Hnm, Snm) gives eps (ascending) and C, as
 *      pawfd_subspace_diag (Hnm and Snm are overwritten);
 *   6. resid[n] = sqrt(dV sum_r |hpsi_n(r) - eps[n] spsi_n(r)|^2).
 * psi, hpsi, spsi: caller-owned FP64 device work arrays [nb][K] (on return they hold steps
 * 1-2); Hnm, Snm, C: [nb][nb] of the context's kind; eps, theta, resid: device [nb] doubles.
 * The refined bands are psi C (pawfd_rotate on this context).
 * Returns PAWFD_EINVAL for a mixed context, nb outside 1..max_bands, null or aliased arrays,
 * or misaligned band arrays; device-side failures of step 5 are reported by pawfd_sync. */
int pawfd_refine(pawfd_ctx* ctx, const void* psi_lo, int nb, const void* C_lo, void* psi, void* hpsi, void* spsi,
                 void* Hnm, void* Snm, double* eps, double* theta, double* resid, void* C);

/* One Rayleigh-Ritz step of SCF step 1 (Kohn-Sham section) as a single call: hpsi = H psi
 * and spsi = S psi (Eq. (dh) and the overlap operator of the PAW section; one set of
 * projections serves both), Hnm = dV psi^H hpsi and Snm = dV psi^H spsi (Hermitian Gram),
 * the subspace diagonalization (eps ascending, C; Hnm and Snm are overwritten as in
 * pawfd_subspace_diag) and psi_out = psi C.
 *   psi, hpsi, spsi, psi_out: [nb][K] of the context's dtype, pairwise distinct;
 *   Hnm, Snm, C: [nb][nb] FP64 of the context's kind; eps: [nb] doubles.  All device memory
 *   owned by the caller.  Errors as the individual calls; device-side failures at pawfd_sync. */
int pawfd_rr_step(pawfd_ctx* ctx, const void* psi, int nb, void* hpsi, void* spsi, void* Hnm, void* Snm,
                  double* eps, void* C, void* psi_out);

/* A batch of independent Rayleigh-Ritz steps (no counterpart in the paper: the packaging of
 * many eigensolver instances of different sizes for one GPU).  Each job names its own
 * context (at most one job per context: a job uses its context's scratch) and the arrays of
 * pawfd_rr_step.  pawfd_batch_launch forks from `stream`, runs every job on a stream of the
 * batch's own (so the jobs' kernels overlap on the GPU) and joins back into `stream`.
 * With use_graph = 1, pawfd_batch_create captures that whole sequence once into a CUDA graph
 * and every launch is one graph launch; the arrays are then fixed for the batch's lifetime.
 * If the capture is refused the batch stays usable in eager mode (pawfd_batch_is_graph
 * returns 0 and pawfd_batch_last_error says why).  The contexts' own streams are not used;
 * check each context with pawfd_sync after the stream has been synchronized.
 * Returns PAWFD_EINVAL for null arguments, count < 1, a repeated context or a job whose
 * arrays fail the checks of pawfd_rr_step; PAWFD_EDEVICE for CUDA failures. */
typedef struct pawfd_rr_job {
  pawfd_ctx* ctx;
  const void* psi;
  int nb;
  void* hpsi;
  void* spsi;
  void* Hnm;
  void* Snm;
  double* eps;
  void* C;
  void* psi_out;
} pawfd_rr_job;
typedef struct pawfd_batch pawfd_batch;
int pawfd_batch_create(pawfd_batch** out, const pawfd_rr_job* jobs, int count, int use_graph);
int pawfd_batch_launch(pawfd_batch* batch, void* stream);
int pawfd_batch_is_graph(const pawfd_batch* batch);
/* kernels one launch of the batch runs (counted when the sequence was enqueued) */
long long pawfd_batch_kernel_count(const pawfd_batch* batch);
const char* pawfd_batch_last_error(const pawfd_batch* batch);
int pawfd_batch_destroy(pawfd_batch* batch);

/* Gram matrix for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a packaging variant of pawfd_gram.  It is for code
 * that must not call cudaMalloc where it needs the Gram matrix -- for example an application
 * whose device memory is wholly owned by its own pool allocator, or a serving loop that
 * cannot afford cudaMalloc's device synchronization and unbounded latency -- and which
 * therefore cannot create a pawfd context either.  It needs no context and allocates
 * nothing: M[n][m] = dV sum_r conj(A_n(r)) B_m(r) for n, m < nb, exactly as pawfd_gram,
 * with the split-K partial tiles kept in a fixed 8 MiB array that lives in the library's
 * device image.
 *   A, B:   device [nb][K] arrays of dtype (PAWFD_R64 or PAWFD_C128); M: device [nb][nb].
 *   stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 * Returns PAWFD_EINVAL for null pointers, K < 1, nb < 1, an unknown dtype, or when one
 * nb x nb partial does not fit in the 8 MiB array (nb > 1024 real, nb > 724 complex);
 * PAWFD_EDEVICE for a CUDA runtime failure.
 * Notes: every GPU that loads the library holds the 8 MiB array until the process exits.
 * The first call made with a given device and CUDA context current looks up the array's
 * device address on that device (set-up once per device and context, then cached under the
 * context's process-unique ID, so a device reset or another context is set up afresh); make
 * that first call before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU race on it.  Each call overwrites all the partial entries it
 * reads, so no clearing between calls is needed.  Launch failures are read from each launch's
 * own status: an error left in the runtime by earlier work is neither reported nor cleared. */
int pawfd_gram_noalloc(const void* A, const void* B, long long K, int nb, int dtype, double dV, void* M,
                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PAWFD_H */
