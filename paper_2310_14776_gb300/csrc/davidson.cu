// davidson.cu -- one block-Davidson step of the iterative eigensolver (SCF step 2 of the
// Kohn-Sham section: "one or more steps through the iterative eigensolver"; the Davidson
// and RMM-DIIS methods of the parallelization section).
//
// The paper names the method but gives none of its steps; the reading implemented here:
//   given n Ritz vectors psi (columns of X[0 .. n)) with Ritz values eps_in,
//   1. H psi and S psi (Eq. (dh) and the overlap operator of the PAW section);
//   2. residuals R_n = H psi_n - eps_n S psi_n and their norms sqrt(dV sum_r |R_n(r)|^2);
//   3. preconditioned corrections X[n + m]: by default (option "davidson_precond" 1, grids whose
//      sizes factor into 2, 3 and 5) the kinetic preconditioner -(T + sigma)^-1 R_m, T the FD
//      kinetic operator, sigma = 0.5 Ha, applied in Fourier space on the library's FFT kernels
//      (pw.cu); otherwise the Jacobi one, -R_m / max(d(r) - eps_m, d0 / 10) with d(r) = v(r) + d0
//      the diagonal of the kinetic + local operator (d0 = -1/2 c0 sum_c 1/h_c^2, the stencil's
//      centre weight), floored so that it stays positive;
//   4. H of the corrections, the projections of all 2n columns, the Hermitian Gram matrices
//      of the 2n-dimensional subspace (H_nm and S_nm as pawfd_gram_hs), the subspace
//      diagonalization (2n Ritz pairs, ascending; the pencil is scaled to a unit S diagonal
//      first, which leaves the Ritz values unchanged), and the n lowest Ritz vectors
//      psi_out = X C[:, 0 .. n).
#include "pawfd_internal.cuh"

using namespace pawfd;

namespace {

constexpr int RB = 256;      // threads per residual block
constexpr int RG = 64;       // grid-point blocks per band (partial norms per band)

__device__ double rblock_sum(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < RB / 32; ++w) s += s_red[w];
  return s;   // valid in thread 0
}

// One band per blockIdx.y, RG blocks of grid points per band.  R = H psi - eps S psi in the
// band's arithmetic, the Jacobi correction -R / max(d - eps, d0 / 10) (or R itself, for the
// kinetic preconditioner that follows) written to pr, and each block's sum of |R|^2 (FP64) to
// part[band][blockIdx.x].
template <class T>
__global__ void __launch_bounds__(RB) residual_precond_kernel(const T* __restrict__ hpsi, const T* __restrict__ spsi,
                                                              long long K, const double* __restrict__ eps,
                                                              const real_t<T>* __restrict__ dshift, double d0,
                                                              T* __restrict__ pr, double* __restrict__ part,
                                                              int jacobi) {
  using R = real_t<T>;
  __shared__ double s_red[RB / 32];
  const int n = blockIdx.y;
  const R e = (R)eps[n];
  const float ef = (float)eps[n];
  const float floor_d = (float)(0.1 * d0);
  const long long off = (long long)n * K;
  double acc = 0.0;
  for (long long r = (long long)blockIdx.x * RB + threadIdx.x; r < K; r += (long long)gridDim.x * RB) {
    T res = hpsi[off + r];
    res -= e * spsi[off + r];
    acc += (double)absx2(res);
    // the preconditioner's weight needs no more than FP32 (any positive weight gives a valid
    // search direction; the subspace step is exact for whatever the corrections hold)
    const float d = (float)dshift[r] - ef;
    const float w = -1.0f / (d > floor_d ? d : floor_d);
    pr[off + r] = jacobi ? res * (R)w : res;
  }
  const double s = rblock_sum(acc, s_red);
  if (threadIdx.x == 0) part[(long long)n * gridDim.x + blockIdx.x] = s;
}

// rnorm[n] = sqrt(dV sum of the band's partial sums), in a fixed order
__global__ void residual_norm_kernel(const double* __restrict__ part, int nb, int G, double dV,
                                     double* __restrict__ rnorm) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nb) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += part[(long long)n * G + g];
  rnorm[n] = sqrt(dV * s);
}

// Jacobi scaling of the subspace pencil: d_i = 1 / sqrt(Re S_ii) (1 where S_ii <= 0), so that
// the scaled S has a unit diagonal.  The corrections of nearly converged bands are tiny;
// scaled, they are unit directions and the Cholesky factorization of S stays well
// conditioned.  Ritz values do not depend on the scaling; the eigenvectors C' of the scaled
// pencil give C = diag(d) C'.
template <class T>
__global__ void subspace_scale_diag_kernel(const T* __restrict__ S, int n, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = (double)realx(S[(long long)i * n + i]);
  d[i] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
}
template <class T>
__global__ void subspace_scale_kernel(T* __restrict__ H, T* __restrict__ S, int n, const double* __restrict__ d) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const double f = d[e / n] * d[e % n];
  H[e] = H[e] * f;
  S[e] = S[e] * f;
}
template <class T>
__global__ void scale_rows_kernel(T* __restrict__ C, int n, const double* __restrict__ d) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  C[e] = C[e] * d[e / n];
}

int check_bands(pawfd_ctx* c, int nb) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  return PAWFD_OK;
}

}  // namespace

namespace pawfd {

int launch_residual_precond(pawfd_ctx* c, const void* hpsi, const void* spsi, int nb, const double* eps, void* pr,
                            double* rnorm, bool jacobi) {
  const double d0 = -0.5 * FD6_W0 * (1.0 / (c->h[0] * c->h[0]) + 1.0 / (c->h[1] * c->h[1]) +
                                     1.0 / (c->h[2] * c->h[2]));
  // partial sums: RG doubles per band in the subspace workspace (7 max_bands^2 matrices of at
  // least 8 bytes per entry; consumed by the norm kernel before any later use of it)
  if ((size_t)nb * RG > (size_t)7 * c->max_bands * c->max_bands) return fail(c, PAWFD_EINVAL, "residual scratch");
  double* part = (double*)c->d_work;
  dim3 grid(RG, nb);
  int rc = dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    residual_precond_kernel<T><<<grid, RB, 0, c->stream>>>((const T*)hpsi, (const T*)spsi, (long long)c->K, eps,
                                                           (const real_t<T>*)c->d_vshift, d0, (T*)pr, part,
                                                           jacobi ? 1 : 0);
    return 0;
  });
  if (rc != PAWFD_OK) return rc;
  residual_norm_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(part, nb, RG, c->dV, rnorm);
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "residual launch");
}

}  // namespace pawfd

extern "C" int pawfd_residual_precond(pawfd_ctx* c, const void* hpsi, const void* spsi, int nb, const double* eps,
                                      void* pr, double* rnorm) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!hpsi || !spsi || !eps || !pr || !rnorm) return fail(c, PAWFD_EINVAL, "null array");
  if (pr == hpsi || pr == spsi) return fail(c, PAWFD_EINVAL, "pr may not alias hpsi or spsi");
  return launch_residual_precond(c, hpsi, spsi, nb, eps, pr, rnorm, true);
}

extern "C" int pawfd_rotate_n(pawfd_ctx* c, const void* psi, int nb, const void* C, int nout, void* psi_out) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (nout < 1 || nout > nb) return fail(c, PAWFD_EINVAL, "nout must be in 1..nb");
  if (!psi || !C || !psi_out) return fail(c, PAWFD_EINVAL, "null array");
  if (psi == psi_out) return fail(c, PAWFD_EINVAL, "psi_out may not alias psi");
  return launch_rotate(c, psi, nb, C, psi_out, nout);
}

extern "C" int pawfd_davidson_step(pawfd_ctx* c, void* X, int nb, const double* eps_in, void* HX, void* SX, void* P,
                                   void* Hnm, void* Snm, double* eps, void* C, double* rnorm, void* psi_out) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || 2 * nb > c->max_bands) return fail(c, PAWFD_EINVAL, "2 nb must be in 2..max_bands");
  if (!X || !eps_in || !HX || !SX || !Hnm || !Snm || !eps || !C || !rnorm || !psi_out || (!P && c->at.Ip > 0))
    return fail(c, PAWFD_EINVAL, "null array");
  if (X == HX || X == SX || X == psi_out || HX == SX || HX == psi_out || SX == psi_out || Hnm == Snm)
    return fail(c, PAWFD_EINVAL, "arrays may not alias");
  const size_t band_bytes = band_size(c) * c->K;
  char* X1 = (char*)X + band_bytes * nb;     // the corrections, columns n .. 2n
  char* HX1 = (char*)HX + band_bytes * nb;
  // 1. H psi and S psi
  int rc = launch_apply_hs(c, X, nb, HX, SX, c->d_P);
  // 2., 3. residuals, their norms, the preconditioned corrections (the kinetic preconditioner
  //    works through HX[nb .. 2nb), free until H of the corrections is formed)
  const bool kinetic = c->davidson_precond == 1 && kinetic_precond_available(c);
  if (rc == PAWFD_OK) rc = launch_residual_precond(c, HX, SX, nb, eps_in, X1, rnorm, !kinetic);
  if (rc == PAWFD_OK && kinetic) rc = launch_kinetic_precond(c, X1, nb, X1, HX1, band_bytes * nb);
  // 4. H of the corrections (S of them enters the Gram matrix through the projections)
  if (rc == PAWFD_OK) rc = launch_kinetic_local(c, X1, nb, HX1);
  if (rc == PAWFD_OK) rc = launch_project(c, X1, nb, c->d_P);
  if (rc == PAWFD_OK) rc = launch_nonlocal_add(c, c->d_P, nb, c->at.d_dH, HX1);
  //    projections of all 2n columns, the subspace matrices, their diagonalization, rotation
  if (rc == PAWFD_OK) rc = launch_project(c, X, 2 * nb, P ? P : c->d_P);
  if (rc == PAWFD_OK) rc = launch_gram_hs(c, X, HX, 2 * nb, P ? P : c->d_P, Hnm, Snm);
  const int m = 2 * nb;
  const unsigned eb = (unsigned)(((long long)m * m + 255) / 256);
  if (rc == PAWFD_OK) {
    if (is_complex(c)) {
      subspace_scale_diag_kernel<zd><<<(m + 127) / 128, 128, 0, c->stream>>>((const zd*)Snm, m, c->d_dscale);
      subspace_scale_kernel<zd><<<eb, 256, 0, c->stream>>>((zd*)Hnm, (zd*)Snm, m, c->d_dscale);
    } else {
      subspace_scale_diag_kernel<double><<<(m + 127) / 128, 128, 0, c->stream>>>((const double*)Snm, m, c->d_dscale);
      subspace_scale_kernel<double><<<eb, 256, 0, c->stream>>>((double*)Hnm, (double*)Snm, m, c->d_dscale);
    }
    c->launches += 2;
    rc = check_cuda(c, cudaGetLastError(), "subspace scaling launch");
  }
  if (rc == PAWFD_OK) rc = launch_subspace_diag(c, m, Hnm, Snm, eps, C);
  if (rc == PAWFD_OK) {
    if (is_complex(c)) scale_rows_kernel<zd><<<eb, 256, 0, c->stream>>>((zd*)C, m, c->d_dscale);
    else scale_rows_kernel<double><<<eb, 256, 0, c->stream>>>((double*)C, m, c->d_dscale);
    c->launches += 1;
    rc = check_cuda(c, cudaGetLastError(), "subspace scaling launch");
  }
  if (rc == PAWFD_OK) rc = launch_rotate(c, X, m, C, psi_out, nb);
  return rc;
}
