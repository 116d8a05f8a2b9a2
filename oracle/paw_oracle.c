/*
 * paw_oracle.c -- plain, slow FP64 CPU oracle for the real-space PAW eigensolver step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library.  It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * What it computes (the PAW section of the paper, Eq. (dh) and the overlap operator
 * after it; the Kohn-Sham section's SCF step 1, "diagonalization of the Hamiltonian in
 * the subspace of the current wave functions"; the parallelization section's dense
 * Cholesky + diagonalization):
 *
 *   (H psi)(r) = -1/2 sum_c d^2 psi/dx_c^2 (r) + v(r) psi(r) + sum_a sum_ii' p_i^a(r) dH^a_ii' P^a_i'
 *   (S psi)(r) =                                     psi(r)  + sum_a sum_ii' p_i^a(r) dS^a_ii' P^a_i'
 *   P^a_i     = <p_i^a | psi> = dV sum_r p_i^a(r) psi(r)          (projector overlaps)
 *   H_nm = dV sum_r conj(psi_n(r)) (H psi_m)(r),  S_nm likewise;  H C = S C diag(eps)
 *
 * The second derivative is the central finite difference of order 6 (three points each
 * side) on a uniform periodic grid; psi obeys the Bloch condition
 * psi(r + L_c e_c) = exp(i k_c L_c) psi(r).  Every loop below is the definition written
 * out, with no blocking or reordering: grid loops visit every point and band, projector
 * loops visit every box point, the Gram matrices are triple loops with compensated
 * summation, the Cholesky is the textbook column algorithm and the eigensolver is the
 * cyclic Jacobi method.
 *
 * Data layout: grid arrays are [band][i3][i2][i1] with i1 (x) fastest; complex arrays are
 * interleaved (re, im) pairs, read here as C99 double complex.  A projector box of atom a
 * covers unwrapped grid indices lo_c .. lo_c + n_c - 1; an unwrapped index u maps to the
 * grid point u mod N_c of the lattice translation T_c = floor(u / N_c) * L_c.  Projections
 * are stored [Ip][nb] (global projector row, band), Ip = sum_a I_a.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zdouble;

/* order-6 central second difference: f'' ~ (1/h^2) sum_{m=-3..3} c_|m| f(x + m h) */
static const double FD6_C[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};

int oracle_fd6_coefficients(double* out4) {
  for (int m = 0; m < 4; ++m) out4[m] = FD6_C[m];
  return 0;
}

/* --------------------------------------------------------------------------------------
 * grid geometry
 * ------------------------------------------------------------------------------------ */
typedef struct {
  int n[3];      /* N1, N2, N3 (x, y, z) */
  double L[3];   /* cell lengths (bohr) */
  double k[3];   /* Bloch vector (1/bohr) */
} orc_grid;

static long grid_index(const int* n, int i1, int i2, int i3) {
  return ((long)i3 * n[1] + i2) * n[0] + i1;
}

/* floor division for possibly negative u */
static int floor_div(int u, int n) { return (u >= 0) ? u / n : -((-u + n - 1) / n); }

/* --------------------------------------------------------------------------------------
 * a1: kinetic + local potential
 * ------------------------------------------------------------------------------------ */

/* real psi at Gamma:  out = -1/2 Lap_FD psi + v psi, periodic wrap */
int oracle_kinetic_local_real(const int* n, const double* L, const double* v, const double* psi,
                              long nb, double* out) {
  const long K = (long)n[0] * n[1] * n[2];
  double h[3];
  for (int c = 0; c < 3; ++c) h[c] = L[c] / n[c];
#pragma omp parallel for schedule(static)
  for (long b = 0; b < nb; ++b) {
    const double* f = psi + b * K;
    double* o = out + b * K;
    for (int i3 = 0; i3 < n[2]; ++i3)
      for (int i2 = 0; i2 < n[1]; ++i2)
        for (int i1 = 0; i1 < n[0]; ++i1) {
          int idx[3] = {i1, i2, i3};
          double lap = 0.0;
          for (int c = 0; c < 3; ++c)
            for (int m = -3; m <= 3; ++m) {
              int j[3] = {idx[0], idx[1], idx[2]};
              j[c] = ((j[c] + m) % n[c] + n[c]) % n[c];
              lap += FD6_C[abs(m)] / (h[c] * h[c]) * f[grid_index(n, j[0], j[1], j[2])];
            }
          long r = grid_index(n, i1, i2, i3);
          o[r] = -0.5 * lap + v[r] * f[r];
        }
  }
  return 0;
}

/* complex psi at Bloch vector k:  neighbours across a face pick up exp(+-i k_c L_c) */
int oracle_kinetic_local_bloch(const int* n, const double* L, const double* k, const double* v,
                               const double* psi_, long nb, double* out_) {
  const long K = (long)n[0] * n[1] * n[2];
  const zdouble* psi = (const zdouble*)psi_;
  zdouble* out = (zdouble*)out_;
  double h[3];
  for (int c = 0; c < 3; ++c) h[c] = L[c] / n[c];
#pragma omp parallel for schedule(static)
  for (long b = 0; b < nb; ++b) {
    const zdouble* f = psi + b * K;
    zdouble* o = out + b * K;
    for (int i3 = 0; i3 < n[2]; ++i3)
      for (int i2 = 0; i2 < n[1]; ++i2)
        for (int i1 = 0; i1 < n[0]; ++i1) {
          int idx[3] = {i1, i2, i3};
          zdouble lap = 0.0;
          for (int c = 0; c < 3; ++c)
            for (int m = -3; m <= 3; ++m) {
              int j[3] = {idx[0], idx[1], idx[2]};
              int u = j[c] + m;               /* unwrapped neighbour index along c */
              int t = floor_div(u, n[c]);     /* lattice translation in units of L_c */
              j[c] = u - t * n[c];
              zdouble phase = cexp(I * (k[c] * L[c] * t));
              lap += FD6_C[abs(m)] / (h[c] * h[c]) * phase * f[grid_index(n, j[0], j[1], j[2])];
            }
          long r = grid_index(n, i1, i2, i3);
          o[r] = -0.5 * lap + v[r] * f[r];
        }
  }
  return 0;
}

/* --------------------------------------------------------------------------------------
 * projector boxes (atoms)
 * ------------------------------------------------------------------------------------ */
typedef struct {
  int natoms;
  const int* nproj;      /* [A] I_a */
  const int* box_lo;     /* [A][3] */
  const int* box_n;      /* [A][3] */
  const double* proj;    /* per atom [I_a][bn3][bn2][bn1] */
  const long* proj_off;  /* [A+1] offsets into proj */
  const double* dmat;    /* per atom [I_a][I_a] (dH or dS) */
  const long* dmat_off;  /* [A+1] */
} orc_atoms;

/* Bloch phase exp(i k.T) of unwrapped box point u, and its wrapped grid index */
static long wrap_point(const orc_grid* g, const int* u, zdouble* phase) {
  int w[3];
  double kt = 0.0;
  for (int c = 0; c < 3; ++c) {
    int t = floor_div(u[c], g->n[c]);
    w[c] = u[c] - t * g->n[c];
    kt += g->k[c] * g->L[c] * t;
  }
  *phase = cexp(I * kt);
  return grid_index(g->n, w[0], w[1], w[2]);
}

/* a2: P[row_a + i][b] = dV sum_{u in box_a} p_i^a(u) exp(i k.T_u) psi_b(wrap u).  P is [Ip][nb] complex. */
static void project_all(const orc_grid* g, const orc_atoms* at, const zdouble* psi, long nb, zdouble* P) {
  const long K = (long)g->n[0] * g->n[1] * g->n[2];
  const double dV = (g->L[0] / g->n[0]) * (g->L[1] / g->n[1]) * (g->L[2] / g->n[2]);
  long Ip = 0;
  for (int a = 0; a < at->natoms; ++a) Ip += at->nproj[a];
  for (long x = 0; x < Ip * nb; ++x) P[x] = 0.0;
  long row = 0;
  for (int a = 0; a < at->natoms; ++a) {
    const int* lo = at->box_lo + 3 * a;
    const int* bn = at->box_n + 3 * a;
    const long bsize = (long)bn[0] * bn[1] * bn[2];
    const double* p = at->proj + at->proj_off[a];
#pragma omp parallel for schedule(static)
    for (long b = 0; b < nb; ++b)
      for (int j3 = 0; j3 < bn[2]; ++j3)
        for (int j2 = 0; j2 < bn[1]; ++j2)
          for (int j1 = 0; j1 < bn[0]; ++j1) {
            int u[3] = {lo[0] + j1, lo[1] + j2, lo[2] + j3};
            zdouble phase;
            long r = wrap_point(g, u, &phase);
            long jb = ((long)j3 * bn[1] + j2) * bn[0] + j1;
            for (int i = 0; i < at->nproj[a]; ++i)
              P[(row + i) * nb + b] += dV * p[i * bsize + jb] * phase * psi[b * K + r];
          }
    row += at->nproj[a];
  }
}

/* a3 + a4: out_b(wrap u) += sum_i p_i^a(u) exp(-i k.T_u) Q[row_a + i][b],  Q = dX P per atom */
static void nonlocal_add_all(const orc_grid* g, const orc_atoms* at, const zdouble* P, long nb, zdouble* out) {
  const long K = (long)g->n[0] * g->n[1] * g->n[2];
  long row = 0;
  for (int a = 0; a < at->natoms; ++a) {
    const int Ia = at->nproj[a];
    const double* dX = at->dmat + at->dmat_off[a];
    zdouble* Q = (zdouble*)calloc((size_t)Ia * nb, sizeof(zdouble));
    for (int i = 0; i < Ia; ++i)
      for (long b = 0; b < nb; ++b)
        for (int i2 = 0; i2 < Ia; ++i2) Q[i * nb + b] += dX[i * Ia + i2] * P[(row + i2) * nb + b];
    const int* lo = at->box_lo + 3 * a;
    const int* bn = at->box_n + 3 * a;
    const long bsize = (long)bn[0] * bn[1] * bn[2];
    const double* p = at->proj + at->proj_off[a];
    /* bands are independent; within one band the box points are visited in order, so a box
       that wraps onto itself (larger than the cell) still accumulates correctly */
#pragma omp parallel for schedule(static)
    for (long b = 0; b < nb; ++b)
      for (int j3 = 0; j3 < bn[2]; ++j3)
        for (int j2 = 0; j2 < bn[1]; ++j2)
          for (int j1 = 0; j1 < bn[0]; ++j1) {
            int u[3] = {lo[0] + j1, lo[1] + j2, lo[2] + j3};
            zdouble phase;
            long r = wrap_point(g, u, &phase);
            long jb = ((long)j3 * bn[1] + j2) * bn[0] + j1;
            zdouble s = 0.0;
            for (int i = 0; i < Ia; ++i) s += p[i * bsize + jb] * Q[i * nb + b];
            out[b * K + r] += conj(phase) * s;
          }
    free(Q);
    row += Ia;
  }
}

static void unpack(const int* n, const double* L, const double* k, orc_grid* g) {
  for (int c = 0; c < 3; ++c) {
    g->n[c] = n[c];
    g->L[c] = L[c];
    g->k[c] = k ? k[c] : 0.0;
  }
}

static void atoms_of(orc_atoms* at, int natoms, const int* nproj, const int* box_lo, const int* box_n,
                     const double* proj, const long* proj_off, const double* dmat, const long* dmat_off) {
  at->natoms = natoms;
  at->nproj = nproj;
  at->box_lo = box_lo;
  at->box_n = box_n;
  at->proj = proj;
  at->proj_off = proj_off;
  at->dmat = dmat;
  at->dmat_off = dmat_off;
}

static zdouble* to_complex(const double* x, long count, int is_complex) {
  zdouble* z = (zdouble*)malloc(sizeof(zdouble) * (size_t)(count > 0 ? count : 1));
  if (is_complex) memcpy(z, x, sizeof(zdouble) * (size_t)count);
  else
    for (long i = 0; i < count; ++i) z[i] = x[i];
  return z;
}

static void from_complex(const zdouble* z, long count, int is_complex, double* x) {
  if (is_complex) memcpy(x, z, sizeof(zdouble) * (size_t)count);
  else
    for (long i = 0; i < count; ++i) x[i] = creal(z[i]);
}

/* Projections P [Ip][nb]; real psi gives real P (k must be 0), complex psi gives complex P. */
int oracle_project(const int* n, const double* L, const double* k, int is_complex, int natoms, const int* nproj,
                   const int* box_lo, const int* box_n, const double* proj, const long* proj_off,
                   const double* psi, long nb, double* P) {
  orc_grid g;
  unpack(n, L, is_complex ? k : NULL, &g);
  orc_atoms at;
  atoms_of(&at, natoms, nproj, box_lo, box_n, proj, proj_off, NULL, NULL);
  const long K = (long)n[0] * n[1] * n[2];
  long Ip = 0;
  for (int a = 0; a < natoms; ++a) Ip += nproj[a];
  zdouble* zpsi = to_complex(psi, K * nb, is_complex);
  zdouble* zP = (zdouble*)calloc((size_t)(Ip * nb > 0 ? Ip * nb : 1), sizeof(zdouble));
  project_all(&g, &at, zpsi, nb, zP);
  from_complex(zP, Ip * nb, is_complex, P);
  free(zpsi);
  free(zP);
  return 0;
}

/* which = 0: H psi (kinetic + local + dH nonlocal);  which = 1: S psi (psi + dS nonlocal);
   which = 2: the nonlocal term alone, sum_a sum_ii' p_i^a dmat^a_ii' <p_i'^a|psi>.
   dmat holds dH or dS accordingly.  If P_out != NULL the projections are returned too. */
int oracle_apply(int which, const int* n, const double* L, const double* k, int is_complex, const double* v,
                 int natoms, const int* nproj, const int* box_lo, const int* box_n, const double* proj,
                 const long* proj_off, const double* dmat, const long* dmat_off, const double* psi, long nb,
                 double* out, double* P_out) {
  orc_grid g;
  unpack(n, L, is_complex ? k : NULL, &g);
  orc_atoms at;
  atoms_of(&at, natoms, nproj, box_lo, box_n, proj, proj_off, dmat, dmat_off);
  const long K = (long)n[0] * n[1] * n[2];
  long Ip = 0;
  for (int a = 0; a < natoms; ++a) Ip += nproj[a];
  zdouble* zpsi = to_complex(psi, K * nb, is_complex);
  zdouble* zout = (zdouble*)malloc(sizeof(zdouble) * (size_t)(K * nb));
  if (which == 0) {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(K * nb) * (is_complex ? 2 : 1));
    if (is_complex) oracle_kinetic_local_bloch(n, L, g.k, v, psi, nb, tmp);
    else oracle_kinetic_local_real(n, L, v, psi, nb, tmp);
    free(zout);
    zout = to_complex(tmp, K * nb, is_complex);
    free(tmp);
  } else if (which == 1) {
    memcpy(zout, zpsi, sizeof(zdouble) * (size_t)(K * nb));
  } else {
    memset(zout, 0, sizeof(zdouble) * (size_t)(K * nb));
  }
  zdouble* zP = (zdouble*)calloc((size_t)(Ip * nb > 0 ? Ip * nb : 1), sizeof(zdouble));
  project_all(&g, &at, zpsi, nb, zP);
  nonlocal_add_all(&g, &at, zP, nb, zout);
  from_complex(zout, K * nb, is_complex, out);
  if (P_out) from_complex(zP, Ip * nb, is_complex, P_out);
  free(zpsi);
  free(zout);
  free(zP);
  return 0;
}

/* --------------------------------------------------------------------------------------
 * a5: Gram matrix  M[n][m] = dV sum_r conj(A_n(r)) B_m(r)   (Neumaier-compensated sums)
 * ------------------------------------------------------------------------------------ */
static void neumaier_add(double* s, double* c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

int oracle_gram(int is_complex, const double* A, const double* B, long K, long nb, double dV, double* M) {
#pragma omp parallel for schedule(dynamic)
  for (long i = 0; i < nb; ++i)
    for (long j = 0; j < nb; ++j) {
      if (!is_complex) {
        double s = 0.0, c = 0.0;
        for (long r = 0; r < K; ++r) neumaier_add(&s, &c, A[i * K + r] * B[j * K + r]);
        M[i * nb + j] = dV * (s + c);
      } else {
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        for (long r = 0; r < K; ++r) {
          double ar = A[2 * (i * K + r)], ai = A[2 * (i * K + r) + 1];
          double br = B[2 * (j * K + r)], bi = B[2 * (j * K + r) + 1];
          /* conj(a) b = (ar br + ai bi) + i (ar bi - ai br) */
          neumaier_add(&sr, &cr, ar * br);
          neumaier_add(&sr, &cr, ai * bi);
          neumaier_add(&si, &ci, ar * bi);
          neumaier_add(&si, &ci, -ai * br);
        }
        M[2 * (i * nb + j)] = dV * (sr + cr);
        M[2 * (i * nb + j) + 1] = dV * (si + ci);
      }
    }
  return 0;
}

/* --------------------------------------------------------------------------------------
 * a6: dense linear algebra on the band x band problem (complex arithmetic throughout;
 *     real inputs are the special case with zero imaginary parts)
 * ------------------------------------------------------------------------------------ */

/* Cholesky S = L L^H (Golub & Van Loan, "Matrix Computations", Alg. 4.2.1 column form).
   Returns 0, or -(j+1) if the pivot of column j is not positive. L is lower, strict upper zeroed. */
static int cholesky(zdouble* S, long n) {
  for (long j = 0; j < n; ++j) {
    double d = creal(S[j * n + j]);
    for (long p = 0; p < j; ++p) d -= creal(S[j * n + p] * conj(S[j * n + p]));
    if (!(d > 0.0)) return (int)-(j + 1);
    double ljj = sqrt(d);
    S[j * n + j] = ljj;
    for (long i = j + 1; i < n; ++i) {
      zdouble s = S[i * n + j];
      for (long p = 0; p < j; ++p) s -= S[i * n + p] * conj(S[j * n + p]);
      S[i * n + j] = s / ljj;
    }
    for (long i = 0; i < j; ++i) S[i * n + j] = 0.0;
  }
  return 0;
}

/* X <- L^{-1} X  (forward substitution on every column of X, n x m) */
static void lower_solve(const zdouble* Lm, long n, zdouble* X, long m) {
  for (long col = 0; col < m; ++col)
    for (long i = 0; i < n; ++i) {
      zdouble s = X[i * m + col];
      for (long p = 0; p < i; ++p) s -= Lm[i * n + p] * X[p * m + col];
      X[i * m + col] = s / Lm[i * n + i];
    }
}

/* X <- L^{-H} X  (back substitution with L^H, upper triangular) */
static void lower_h_solve(const zdouble* Lm, long n, zdouble* X, long m) {
  for (long col = 0; col < m; ++col)
    for (long i = n - 1; i >= 0; --i) {
      zdouble s = X[i * m + col];
      for (long p = i + 1; p < n; ++p) s -= conj(Lm[p * n + i]) * X[p * m + col];
      X[i * m + col] = s / conj(Lm[i * n + i]);
    }
}

/* Cyclic Jacobi for a Hermitian matrix (Golub & Van Loan section 8.5, with the phase of each
   off-diagonal pivot removed first so the 2x2 problem is real symmetric).  A is overwritten
   by (nearly) diag(eigenvalues); V accumulates the rotations (A_in = V diag V^H).
   Stops when off(A) <= tol * ||A||_F; returns the number of sweeps, or -1 after max_sweeps. */
static int jacobi_eigh(zdouble* A, long n, zdouble* V, double tol, int max_sweeps) {
  for (long i = 0; i < n; ++i)
    for (long j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (long i = 0; i < n * n; ++i) fro += creal(A[i] * conj(A[i]));
  fro = sqrt(fro);
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double off = 0.0;
    for (long i = 0; i < n; ++i)
      for (long j = 0; j < n; ++j)
        if (i != j) off += creal(A[i * n + j] * conj(A[i * n + j]));
    if (sqrt(off) <= tol * fro) return sweep;
    if (sweep == max_sweeps) break;
    for (long p = 0; p < n - 1; ++p)
      for (long q = p + 1; q < n; ++q) {
        zdouble apq = A[p * n + q];
        double mag = cabs(apq);
        if (mag == 0.0) continue;
        /* unitary phase on column/row q: makes A[p][q] real and positive */
        zdouble ph = apq / mag; /* e^{i phi} */
        for (long i = 0; i < n; ++i) A[i * n + q] *= conj(ph);
        for (long i = 0; i < n; ++i) A[q * n + i] *= ph;
        for (long i = 0; i < n; ++i) V[i * n + q] *= conj(ph);
        double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
        double tau = (aqq - app) / (2.0 * mag);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* A <- J^T A J with J = [[c, s], [-s, c]] in the (p, q) plane */
        for (long i = 0; i < n; ++i) {
          zdouble aip = A[i * n + p], aiq = A[i * n + q];
          A[i * n + p] = c * aip - s * aiq;
          A[i * n + q] = s * aip + c * aiq;
        }
        for (long i = 0; i < n; ++i) {
          zdouble api = A[p * n + i], aqi = A[q * n + i];
          A[p * n + i] = c * api - s * aqi;
          A[q * n + i] = s * api + c * aqi;
        }
        A[p * n + q] = 0.0;
        A[q * n + p] = 0.0;
        for (long i = 0; i < n; ++i) {
          zdouble vip = V[i * n + p], viq = V[i * n + q];
          V[i * n + p] = c * vip - s * viq;
          V[i * n + q] = s * vip + c * viq;
        }
      }
  }
  return -1;
}

/* Solve H C = S C diag(eps) for Hermitian H and positive definite S (n x n, row-major,
   complex if is_complex).  Steps: symmetrize; S = L L^H; A = L^{-1} H L^{-H}; A = U diag U^H
   (Jacobi); C = L^{-H} U; sort ascending (stable); fix each column's phase so that its
   largest-magnitude entry (first on ties) is real and positive.
   Returns 0, -(j+1) for a Cholesky failure at column j, or -1000000 if Jacobi did not converge. */
int oracle_subspace_diag(int is_complex, long n, const double* Hnm, const double* Snm, double* eps, double* C,
                         int* sweeps_out) {
  zdouble* Hm = to_complex(Hnm, n * n, is_complex);
  zdouble* Sm = to_complex(Snm, n * n, is_complex);
  zdouble* A = (zdouble*)malloc(sizeof(zdouble) * (size_t)(n * n));
  zdouble* U = (zdouble*)malloc(sizeof(zdouble) * (size_t)(n * n));
  int rc = 0;
  for (long i = 0; i < n; ++i)
    for (long j = 0; j < n; ++j) {
      A[i * n + j] = 0.5 * (Hm[i * n + j] + conj(Hm[j * n + i]));
      U[i * n + j] = 0.5 * (Sm[i * n + j] + conj(Sm[j * n + i]));
    }
  memcpy(Sm, U, sizeof(zdouble) * (size_t)(n * n));
  rc = cholesky(Sm, n);
  if (rc == 0) {
    /* A <- L^{-1} A, then A <- (L^{-1} A^H)^H = L^{-1} H L^{-H} */
    lower_solve(Sm, n, A, n);
    for (long i = 0; i < n; ++i)
      for (long j = 0; j < n; ++j) U[j * n + i] = conj(A[i * n + j]);
    lower_solve(Sm, n, U, n);
    for (long i = 0; i < n; ++i)
      for (long j = 0; j < n; ++j) A[j * n + i] = conj(U[i * n + j]);
    /* exact Hermitian symmetry before the eigensolver */
    for (long i = 0; i < n; ++i)
      for (long j = i; j < n; ++j) {
        zdouble x = 0.5 * (A[i * n + j] + conj(A[j * n + i]));
        A[i * n + j] = x;
        A[j * n + i] = conj(x);
      }
    int sw = jacobi_eigh(A, n, U, 1e-14, 60);
    if (sweeps_out) *sweeps_out = sw;
    if (sw < 0) rc = -1000000;
    lower_h_solve(Sm, n, U, n); /* C = L^{-H} U */
    /* ascending order, stable */
    long* order = (long*)malloc(sizeof(long) * (size_t)n);
    for (long i = 0; i < n; ++i) order[i] = i;
    for (long i = 1; i < n; ++i) {
      long key = order[i];
      double kv = creal(A[key * n + key]);
      long j = i - 1;
      while (j >= 0 && creal(A[order[j] * n + order[j]]) > kv) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = key;
    }
    for (long m = 0; m < n; ++m) {
      long src = order[m];
      eps[m] = creal(A[src * n + src]);
      long best = 0;
      double bmag = -1.0;
      for (long i = 0; i < n; ++i) {
        double mag = cabs(U[i * n + src]);
        if (mag > bmag) {
          bmag = mag;
          best = i;
        }
      }
      zdouble ph = (bmag > 0.0) ? conj(U[best * n + src]) / bmag : 1.0;
      for (long i = 0; i < n; ++i) Hm[i * n + m] = U[i * n + src] * ph;
    }
    from_complex(Hm, n * n, is_complex, C);
    free(order);
  }
  free(Hm);
  free(Sm);
  free(A);
  free(U);
  return rc;
}

/* exposed pieces for the pin tests */
int oracle_cholesky(int is_complex, long n, const double* S, double* Lout) {
  zdouble* Sm = to_complex(S, n * n, is_complex);
  int rc = cholesky(Sm, n);
  from_complex(Sm, n * n, is_complex, Lout);
  free(Sm);
  return rc;
}

int oracle_jacobi_eigh(int is_complex, long n, const double* A_in, double* evals, double* V_out, int* sweeps) {
  zdouble* A = to_complex(A_in, n * n, is_complex);
  zdouble* V = (zdouble*)malloc(sizeof(zdouble) * (size_t)(n * n));
  int sw = jacobi_eigh(A, n, V, 1e-14, 60);
  if (sweeps) *sweeps = sw;
  for (long i = 0; i < n; ++i) evals[i] = creal(A[i * n + i]);
  from_complex(V, n * n, is_complex, V_out);
  free(A);
  free(V);
  return sw < 0 ? -1 : 0;
}

/* --------------------------------------------------------------------------------------
 * a7: rotation  psi'_m(r) = sum_n psi_n(r) C[n][m]
 * ------------------------------------------------------------------------------------ */
int oracle_rotate(int is_complex, const double* psi, long K, long nb, const double* C, double* out) {
  if (!is_complex) {
#pragma omp parallel for schedule(static)
    for (long m = 0; m < nb; ++m)
      for (long r = 0; r < K; ++r) {
        double s = 0.0;
        for (long nn = 0; nn < nb; ++nn) s += psi[nn * K + r] * C[nn * nb + m];
        out[m * K + r] = s;
      }
  } else {
    const zdouble* zp = (const zdouble*)psi;
    const zdouble* zc = (const zdouble*)C;
    zdouble* zo = (zdouble*)out;
#pragma omp parallel for schedule(static)
    for (long m = 0; m < nb; ++m)
      for (long r = 0; r < K; ++r) {
        zdouble s = 0.0;
        for (long nn = 0; nn < nb; ++nn) s += zp[nn * K + r] * zc[nn * nb + m];
        zo[m * K + r] = s;
      }
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
