// density.cu -- the reductions that follow the eigensolver in the SCF loop (step 3 of the
// Kohn-Sham section feeds them): the pseudo density and the atomic density matrices.
//
//   rho(r) = sum_n f_n |psi_n(r)|^2                       (the pseudo density n~ of the PAW
//                                                           section, one spin channel, without
//                                                           compensation charges)
//   D^a_ii' = sum_n f_n <psi_n|p_i^a> <p_i'^a|psi_n>       (Eq. (atomicdensitymatrix))
//           = sum_n f_n conj(P_ani) P_ani'                  with P_ani = <p_ai|psi_n>
//
// rho is HBM-bound (one read of every band, 8 or 16 bytes per point-band); D is a tiny
// reduction over the projections.  Both are deterministic (fixed summation order).
#include <type_traits>

#include "df_arith.cuh"
#include "pawfd_internal.cuh"

using namespace pawfd;

namespace {

constexpr int DT = 256;     // threads per density block
constexpr int DV = 4;       // consecutive grid points per thread

// The DV values of one band at r0 (16-byte vector loads when the whole group is inside the
// grid and aligned; zero past the end).
__device__ __forceinline__ void load_group(const double* __restrict__ row, bool vec, long long left,
                                           double (&x)[DV]) {
  if (vec) {
    const double2 a = __ldg((const double2*)row), b = __ldg((const double2*)row + 1);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  } else {
#pragma unroll
    for (int v = 0; v < DV; ++v) x[v] = v < left ? row[v] : 0.0;
  }
}
__device__ __forceinline__ void load_group(const float* __restrict__ row, bool vec, long long left, float (&x)[DV]) {
  if (vec) {
    const float4 a = __ldg((const float4*)row);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  } else {
#pragma unroll
    for (int v = 0; v < DV; ++v) x[v] = v < left ? row[v] : 0.0f;
  }
}
template <class R>
__device__ __forceinline__ void load_group(const cplx<R>* __restrict__ row, bool, long long left, cplx<R> (&x)[DV]) {
#pragma unroll
  for (int v = 0; v < DV; ++v) x[v] = v < left ? row[v] : zero<cplx<R>>();
}

// f_n |x|^2 summed over the bands.  Real FP64 bands: in double-float FP32 pairs (x split into
// hi + lo with integer operations, x^2 and f_n x^2 as error-free products, about 2^-46 relative
// per term; the sum of positive terms keeps that relative accuracy), since the FP64 pipe
// (two FMAs per SM and clock) would bound the kernel well below the HBM rate.  Complex FP64:
// FP64.  FP32 bands: products in FP32 within runs of 16 bands, then FP64 (|x|^2 of an FP32
// value is exact to 2^-24; the sum over bands is the part that needs the wider type).
template <class T>
__global__ void __launch_bounds__(DT) density_kernel(const T* __restrict__ psi, int nb, long long K, bool aligned,
                                                     const double* __restrict__ f, double* __restrict__ rho) {
  using R = real_t<T>;
  const long long r0 = ((long long)blockIdx.x * DT + threadIdx.x) * DV;
  if (r0 >= K) return;
  const long long left = K - r0;
  const bool vec = aligned && left >= DV;
  if constexpr (std::is_same<T, double>::value) {
    dfa::DF acc[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) acc[v] = {0.0f, 0.0f};
    for (int n = 0; n < nb; ++n) {
      const dfa::DF fn = dfa::split64(__ldg(f + n));
      double x[DV];
      load_group(psi + (long long)n * K + r0, vec, left, x);
#pragma unroll
      for (int v = 0; v < DV; ++v) {
        const dfa::DF xs = dfa::split64(x[v]);
        dfa::DF x2 = {0.0f, 0.0f};
        dfa::fma_acc(x2, xs, xs);
        dfa::fma_acc(acc[v], fn, x2);
      }
    }
#pragma unroll
    for (int v = 0; v < DV; ++v)
      if (v < left) rho[r0 + v] = dfa::to_double(acc[v]);
  } else {
    double acc[DV];
#pragma unroll
    for (int v = 0; v < DV; ++v) acc[v] = 0.0;
    for (int n0 = 0; n0 < nb; n0 += 16) {
      const int n1 = min(nb, n0 + 16);
      R part[DV];
#pragma unroll
      for (int v = 0; v < DV; ++v) part[v] = (R)0;
      for (int n = n0; n < n1; ++n) {
        const R fn = (R)__ldg(f + n);
        T x[DV];
        load_group(psi + (long long)n * K + r0, vec, left, x);
#pragma unroll
        for (int v = 0; v < DV; ++v) {
          if constexpr (sizeof(R) == 8) acc[v] = fma((double)fn, (double)absx2(x[v]), acc[v]);
          else part[v] = fmaf(fn, absx2(x[v]), part[v]);
        }
      }
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int v = 0; v < DV; ++v) acc[v] += (double)part[v];
      }
    }
#pragma unroll
    for (int v = 0; v < DV; ++v)
      if (v < left) rho[r0 + v] = acc[v];
  }
}

// One CTA per atom: D^a[i][i'] = sum_n f_n conj(P[row_a + i][n]) P[row_a + i'][n], FP64 (or
// complex FP64) in the packed per-atom layout of dH / dS (offset dmat_off[a]).
template <class T>
__global__ void atomic_density_kernel(const T* __restrict__ P, int nb, const double* __restrict__ f,
                                      const int* __restrict__ nproj, const int* __restrict__ row_off,
                                      const long long* __restrict__ dmat_off, wide_t<T>* __restrict__ D) {
  using W = wide_t<T>;
  const int a = blockIdx.x;
  const int I = nproj[a], r0 = row_off[a];
  for (int e = threadIdx.x; e < I * I; e += blockDim.x) {
    const int i = e / I, ip = e % I;
    W acc = zero<W>();
    const T* pi = P + (long long)(r0 + i) * nb;
    const T* pj = P + (long long)(r0 + ip) * nb;
    for (int n = 0; n < nb; ++n) {
      W t = zero<W>();
      fma_conj(t, widen(pi[n]), widen(pj[n]));
      acc += f[n] * t;
    }
    D[dmat_off[a] + e] = acc;
  }
}

}  // namespace

extern "C" int pawfd_density(pawfd_ctx* c, const void* psi, int nb, const double* f, double* rho) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  if (!psi || !f || !rho) return fail(c, PAWFD_EINVAL, "null array");
  const long long K = (long long)c->K;
  const unsigned blocks = (unsigned)((K + (long long)DT * DV - 1) / ((long long)DT * DV));
  // 16-byte loads of the real types: band rows and the array start on 16-byte boundaries
  const bool aligned = (K * (long long)band_size(c)) % 16 == 0 && ((uintptr_t)psi & 15) == 0;
  int rc = dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    density_kernel<T><<<blocks, DT, 0, c->stream>>>((const T*)psi, nb, K, aligned, f, rho);
    return 0;
  });
  if (rc != PAWFD_OK) return rc;
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "density launch");
}

extern "C" int pawfd_atomic_density(pawfd_ctx* c, const void* P, int nb, const double* f, void* D) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  if (c->at.natoms == 0) return PAWFD_OK;
  if (!P || !f || !D) return fail(c, PAWFD_EINVAL, "null array");
  int rc = dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    atomic_density_kernel<T><<<c->at.natoms, 128, 0, c->stream>>>((const T*)P, nb, f, c->at.d_nproj, c->at.d_row_off,
                                                                  c->at.d_dmat_off, (wide_t<T>*)D);
    return 0;
  });
  if (rc != PAWFD_OK) return rc;
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "atomic density launch");
}
