// refine.cu -- final refinement of the mixed form on an FP64 context.
//
// The paper does not describe a mixed-precision eigensolver step; the refinement follows the
// reading that closes one: the FP32 / complex64 input bands of the mixed step are promoted to
// FP64 and rotated by that step's FP64 eigenvector matrix in FP64 (psi' = psi C_lo, the
// digit-product rotation of an FP64 context: the span of the input is kept to FP64 rounding,
// where FP32-rounded rotated bands would move it by the FP32 rounding), H and S are applied in
// FP64 (Eq. (dh) and the overlap operator of the PAW section), FP64 Gram matrices give the
// Rayleigh quotients theta_n = H'_nn / S'_nn, a second FP64 subspace diagonalization (SCF step
// 1 of the Kohn-Sham section) gives the refined eigenvalues, and the residual norms
// ||H psi'_n - eps_n S psi'_n|| are reported.
#include <algorithm>

#include "pawfd_internal.cuh"

using namespace pawfd;

namespace {

constexpr int NT = 256;

// FP32 -> FP64 element copy (real or interleaved complex: `n` scalars)
__global__ void promote_kernel(const float* __restrict__ src, double* __restrict__ dst, long long n) {
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = __ldg((const float4*)src + i);
    ((double2*)dst)[2 * i] = make_double2(v.x, v.y);
    ((double2*)dst)[2 * i + 1] = make_double2(v.z, v.w);
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = (double)src[i];
}

template <class T>
__global__ void rayleigh_quotient_kernel(const T* __restrict__ H, const T* __restrict__ S, int nb,
                                         double* __restrict__ theta) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nb) theta[n] = realx(H[(size_t)n * nb + n]) / realx(S[(size_t)n * nb + n]);
}

// part[n][chunk] = sum over the chunk's points of |h_n - eps_n s_n|^2 (fixed summation order)
template <class T>
__global__ void residual_partial_kernel(const T* __restrict__ hpsi, const T* __restrict__ spsi,
                                        const double* __restrict__ eps, long long K, int nchunk,
                                        double* __restrict__ part) {
  const int n = blockIdx.y, chunk = blockIdx.x;
  const long long len = (K + nchunk - 1) / nchunk;
  const long long r0 = chunk * len, r1 = min(K, r0 + len);
  const T* h = hpsi + (size_t)n * K;
  const T* s = spsi + (size_t)n * K;
  const double e = eps[n];
  double acc = 0.0;
  for (long long r = r0 + threadIdx.x; r < r1; r += NT) {
    const T d = h[r] - e * s[r];
    acc += absx2(d);
  }
  __shared__ double red[NT];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)n * nchunk + chunk] = red[0];
}

__global__ void residual_final_kernel(const double* __restrict__ part, int nb, int nchunk, double dV,
                                      double* __restrict__ resid) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nb) return;
  double acc = 0.0;
  for (int j = 0; j < nchunk; ++j) acc += part[(size_t)n * nchunk + j];
  resid[n] = sqrt(dV * acc);
}

template <class T>
int refine_tail(pawfd_ctx* c, int nb, const void* hpsi, const void* spsi, void* Hnm, void* Snm, double* eps,
                double* theta, double* resid, void* C) {
  rayleigh_quotient_kernel<T><<<(nb + NT - 1) / NT, NT, 0, c->stream>>>((const T*)Hnm, (const T*)Snm, nb, theta);
  c->launches += 1;
  int rc = check_cuda(c, cudaGetLastError(), "rayleigh quotient launch");
  if (rc != PAWFD_OK) return rc;
  rc = launch_subspace_diag(c, nb, Hnm, Snm, eps, C);
  if (rc != PAWFD_OK) return rc;
  // the subspace solve is done with its workspace: its first nchunk * nb doubles hold partials
  const long long work_doubles = 7ll * c->max_bands * c->max_bands;
  const int nchunk = (int)std::max(1ll, std::min<long long>(64, work_doubles / nb));
  double* part = (double*)c->d_work;
  residual_partial_kernel<T><<<dim3(nchunk, nb), NT, 0, c->stream>>>((const T*)hpsi, (const T*)spsi, eps,
                                                                     (long long)c->K, nchunk, part);
  residual_final_kernel<<<(nb + NT - 1) / NT, NT, 0, c->stream>>>(part, nb, nchunk, c->dV, resid);
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "residual launch");
}

}  // namespace

extern "C" int pawfd_refine(pawfd_ctx* c, const void* psi_lo, int nb, const void* C_lo, void* psi, void* hpsi,
                            void* spsi, void* Hnm, void* Snm, double* eps, double* theta, double* resid, void* C) {
  if (!c) return PAWFD_EINVAL;
  if (c->dtype != PAWFD_R64 && c->dtype != PAWFD_C128)
    return fail(c, PAWFD_EINVAL, "refine needs an FP64 context (real or complex)");
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  if (!psi_lo || !psi || !hpsi || !spsi || !Hnm || !Snm || !eps || !theta || !resid || !C)
    return fail(c, PAWFD_EINVAL, "null array");
  if (psi == hpsi || psi == spsi || hpsi == spsi || psi_lo == psi || psi_lo == hpsi || Hnm == Snm)
    return fail(c, PAWFD_EINVAL, "work arrays may not alias");
  if (C_lo && (C_lo == C || C_lo == Hnm || C_lo == Snm))
    return fail(c, PAWFD_EINVAL, "C_lo may not alias an output matrix");
  if (((uintptr_t)psi_lo | (uintptr_t)psi | (uintptr_t)hpsi) & 15)
    return fail(c, PAWFD_EINVAL, "band arrays must be 16-byte aligned");
  // 1. promote the bands to FP64 (exact); with C_lo, into hpsi as a staging array, then
  //    psi = that * C_lo in FP64 (hpsi is written again by step 2)
  const long long scalars = (long long)nb * (long long)c->K * (is_complex(c) ? 2 : 1);
  const int blocks = (int)std::min<long long>(8ll * c->num_sms, (scalars / 4 + NT - 1) / NT + 1);
  promote_kernel<<<blocks, NT, 0, c->stream>>>((const float*)psi_lo, (double*)(C_lo ? hpsi : psi), scalars);
  c->launches += 1;
  int rc = check_cuda(c, cudaGetLastError(), "promote launch");
  if (rc == PAWFD_OK && C_lo) rc = launch_rotate(c, hpsi, nb, C_lo, psi);
  // 2. H psi' and S psi' in FP64, sharing one set of projections
  if (rc == PAWFD_OK) rc = launch_apply_hs(c, psi, nb, hpsi, spsi, c->d_P);
  // 3. FP64 Gram matrices
  if (rc == PAWFD_OK) rc = launch_gram_hs(c, psi, hpsi, nb, c->d_P, Hnm, Snm);
  if (rc != PAWFD_OK) return rc;
  // 4.-6. Rayleigh quotients, second subspace solve, residual norms
  if (is_complex(c)) return refine_tail<zd>(c, nb, hpsi, spsi, Hnm, Snm, eps, theta, resid, C);
  return refine_tail<double>(c, nb, hpsi, spsi, Hnm, Snm, eps, theta, resid, C);
}
