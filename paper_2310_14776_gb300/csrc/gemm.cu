// gemm.cu -- band x band contractions over the grid (FP64 / complex FP64 path).
//
//   Gram:    M[n][m] = dV sum_r conj(A_n(r)) B_m(r)      (subspace matrices H_nm, S_nm)
//   Rotate:  out_m(r) = sum_n psi_n(r) C[n][m]           (rotation after the subspace solve)
//
// Both are dense contractions (Kohn-Sham section, SCF step 1; the paper's BLAS hot spots).
// On GB300 the FP64 rate is the same for the vector units and the DMMA tensor path, so the
// FP64 kernels are register-tiled DFMA GEMMs: 64 x 64 output tiles, 256 threads, 4 x 4
// outputs per thread strided by 16 so that every shared-memory read is conflict free.
// The Gram kernel splits the long grid dimension across CTAs and reduces the partial
// tiles in a fixed order, so the result is deterministic.
#include <algorithm>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int TM = 64, TK = 16, NT = 256;

template <class T>
__global__ void __launch_bounds__(NT) gram_partial_kernel(const T* __restrict__ A, const T* __restrict__ B, int nb,
                                                          long long K, long long kchunk, T* __restrict__ part) {
  __shared__ T As[TK][TM];
  __shared__ T Bs[TK][TM];
  const int n0 = blockIdx.y * TM, m0 = blockIdx.x * TM;
  const long long k0 = (long long)blockIdx.z * kchunk;
  const long long k1 = min(K, k0 + kchunk);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int lrow = tid / 4, lk = (tid % 4) * 4;   // loader: 64 rows x 16 k, 4 consecutive k each
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
  const T* __restrict__ arow = A + (long long)(n0 + lrow) * K;
  const T* __restrict__ brow = B + (long long)(m0 + lrow) * K;
  const bool aok = n0 + lrow < nb, bok = m0 + lrow < nb;
  for (long long kk = k0; kk < k1; kk += TK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long k = kk + lk + e;
      As[lk + e][lrow] = (aok && k < k1) ? conjx(arow[k]) : zero<T>();
      Bs[lk + e][lrow] = (bok && k < k1) ? brow[k] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[j][ty + 16 * i];
        b[i] = Bs[j][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) fma_plain(acc[i][l], a[i], b[l]);
    }
    __syncthreads();
  }
  T* __restrict__ out = part + (long long)blockIdx.z * nb * nb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int n = n0 + ty + 16 * i, m = m0 + tx + 16 * l;
      if (n < nb && m < nb) out[(long long)n * nb + m] = acc[i][l];
    }
}

template <class T>
__global__ void gram_reduce_kernel(const T* __restrict__ part, int nsplit, int nb, double dV, T* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)nb * nb;
  if (e >= nn) return;
  T s = zero<T>();
  for (int p = 0; p < nsplit; ++p) s += part[p * nn + e];
  M[e] = dV * s;
}

template <class T>
__global__ void __launch_bounds__(NT) rotate_kernel(const T* __restrict__ psi, const T* __restrict__ C, int nb,
                                                    long long K, T* __restrict__ out) {
  __shared__ T Cs[TK][TM];
  __shared__ T Ps[TK][TM];
  const long long r0 = (long long)blockIdx.x * TM;
  const int m0 = blockIdx.y * TM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
  for (int n0 = 0; n0 < nb; n0 += TK) {
    for (int s = tid; s < TK * TM; s += NT) {
      const int j = s / TM, i = s - j * TM;
      const int n = n0 + j;
      Cs[j][i] = (n < nb && m0 + i < nb) ? C[(long long)n * nb + m0 + i] : zero<T>();
      Ps[j][i] = (n < nb && r0 + i < K) ? psi[(long long)n * K + r0 + i] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      T cm[4], pr[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cm[i] = Cs[j][ty + 16 * i];
        pr[i] = Ps[j][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) fma_plain(acc[i][l], cm[i], pr[l]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int m = m0 + ty + 16 * i;
      const long long r = r0 + tx + 16 * l;
      if (m < nb && r < K) out[(long long)m * K + r] = acc[i][l];
    }
}

template <class T>
int gram_impl(pawfd_ctx* c, const T* A, const T* B, int nb, T* M) {
  const long long K = (long long)c->K;
  const int tiles = ((nb + TM - 1) / TM) * ((nb + TM - 1) / TM);
  const size_t per = (size_t)nb * nb * sizeof(T);
  long long nsplit = std::max<long long>(1, (2ll * c->num_sms + tiles - 1) / tiles);
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, (long long)(c->gram_part_bytes / per)));
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, K / (4 * TK)));
  long long kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  dim3 grid((nb + TM - 1) / TM, (nb + TM - 1) / TM, (unsigned)nsplit);
  T* part = (T*)c->d_gram_part;
  gram_partial_kernel<T><<<grid, NT, 0, c->stream>>>(A, B, nb, K, kchunk, part);
  const long long nn = (long long)nb * nb;
  gram_reduce_kernel<T><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(part, (int)nsplit, nb, c->dV, M);
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "gram launch");
}

template <class T>
int rotate_impl(pawfd_ctx* c, const T* psi, int nb, const T* C, T* out) {
  const long long K = (long long)c->K;
  dim3 grid((unsigned)((K + TM - 1) / TM), (nb + TM - 1) / TM);
  rotate_kernel<T><<<grid, NT, 0, c->stream>>>(psi, C, nb, K, out);
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "rotate launch");
}

}  // namespace

int launch_gram(pawfd_ctx* c, const void* A, const void* B, int nb, void* M) {
  if (c->dtype == PAWFD_C128) return gram_impl<zd>(c, (const zd*)A, (const zd*)B, nb, (zd*)M);
  return gram_impl<double>(c, (const double*)A, (const double*)B, nb, (double*)M);
}

int launch_rotate(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out) {
  if (c->dtype == PAWFD_C128) return rotate_impl<zd>(c, (const zd*)psi, nb, (const zd*)C, (zd*)out);
  return rotate_impl<double>(c, (const double*)psi, nb, (const double*)C, (double*)out);
}

}  // namespace pawfd
