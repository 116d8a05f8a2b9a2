// stencil.cu -- kinetic + local term  out = -1/2 Lap_FD psi + v psi  on a periodic / Bloch grid.
//
// The finite-difference stencil hot spot (development section: "applying a finite-difference
// stencil to a uniform grid"), order-6 central second difference per axis, fused with the
// local potential of Eq. (dh).  Bloch condition psi(r + L_c e_c) = exp(i k_c L_c) psi(r).
//
// Design: 2.5-D blocking.  A CTA owns a 32 x 8 (x, y) column of one band and marches along z;
// each z-plane of the tile plus a 3-point halo is staged in shared memory, the +-3 z
// neighbours of a thread's own column sit in a 7-register queue.  Halo points that leave the
// cell are wrapped (with the Bloch phase of the crossed face) on load, so the same code
// handles ragged tiles, boxes smaller than the stencil and every grid size >= 1.
#include <algorithm>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

// R: real type of the arithmetic (double for the FP64 dtypes, float for the FP32 ones)
template <class R>
struct StencilArgs {
  int n1, n2, n3;
  long long K;
  R wx[3], wy[3], wz[3];        // -1/2 w_m / h_c^2 for m = 1..3
  cplx<R> ph[3];                // exp(i k_c L_c)
  const R* vshift;              // v(r) - 1/2 w_0 sum_c 1/h_c^2
  int zchunk, nzc;
  void* cpy;                    // optional second output: a copy of psi (the 1 of S = 1 + ...)
};

template <class R>
__device__ __forceinline__ R phased(R v, int, int, int, const StencilArgs<R>&) { return v; }

template <class R>
__device__ __forceinline__ cplx<R> pow_phase(cplx<R> ph, int t) {
  cplx<R> r = {R(1), R(0)};
  const cplx<R> f = t > 0 ? ph : conjx(ph);
  for (int i = 0; i < (t > 0 ? t : -t); ++i) r = r * f;
  return r;
}

template <class R>
__device__ __forceinline__ cplx<R> phased(cplx<R> v, int t1, int t2, int t3, const StencilArgs<R>& a) {
  if (t1) v = v * pow_phase(a.ph[0], t1);
  if (t2) v = v * pow_phase(a.ph[1], t2);
  if (t3) v = v * pow_phase(a.ph[2], t3);
  return v;
}

// psi at unwrapped grid index (u1, u2, u3) of one band, Bloch phase included
template <class T>
__device__ __forceinline__ T load_wrapped(const T* __restrict__ src, int u1, int u2, int u3,
                                          const StencilArgs<real_t<T>>& a) {
  int t1 = 0, t2 = 0, t3 = 0;
  while (u1 < 0) { u1 += a.n1; --t1; }
  while (u1 >= a.n1) { u1 -= a.n1; ++t1; }
  while (u2 < 0) { u2 += a.n2; --t2; }
  while (u2 >= a.n2) { u2 -= a.n2; ++t2; }
  while (u3 < 0) { u3 += a.n3; --t3; }
  while (u3 >= a.n3) { u3 -= a.n3; ++t3; }
  const T v = src[((long long)u3 * a.n2 + u2) * a.n1 + u1];
  return phased(v, t1, t2, t3, a);
}

constexpr int TX = 32, TY = 8, HALO = 3;
constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO;

template <class T>
__global__ void __launch_bounds__(TX * TY) kinetic_local_kernel(const T* __restrict__ psi, T* __restrict__ out,
                                                                StencilArgs<real_t<T>> a) {
  __shared__ T tile[SY][SX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
  const int band = blockIdx.z / a.nzc, zc = blockIdx.z % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const T* __restrict__ src = psi + (long long)band * a.K;
  T* __restrict__ dst = out + (long long)band * a.K;
  T* __restrict__ cp = a.cpy ? (T*)a.cpy + (long long)band * a.K : nullptr;
  const int x = X0 + tx, y = Y0 + ty;
  const bool active = x < a.n1 && y < a.n2;

  T q[7];  // q[j] = psi(x, y, z - 3 + j)
#pragma unroll
  for (int j = 0; j < 6; ++j) q[j + 1] = active ? load_wrapped(src, x, y, z0 - 3 + j, a) : zero<T>();

  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 6; ++j) q[j] = q[j + 1];
    q[6] = active ? load_wrapped(src, x, y, z + 3, a) : zero<T>();
    __syncthreads();
    for (int s = ty * TX + tx; s < SX * SY; s += TX * TY) {
      const int ly = s / SX, lx = s - ly * SX;
      tile[ly][lx] = load_wrapped(src, X0 - HALO + lx, Y0 - HALO + ly, z, a);
    }
    __syncthreads();
    if (active) {
      const long long r = ((long long)z * a.n2 + y) * a.n1 + x;
      const T* row = &tile[ty + HALO][tx + HALO];
      T acc = a.vshift[r] * q[3];
      fma_real(acc, a.wx[0], row[1] + row[-1]);
      fma_real(acc, a.wx[1], row[2] + row[-2]);
      fma_real(acc, a.wx[2], row[3] + row[-3]);
      fma_real(acc, a.wy[0], tile[ty + HALO + 1][tx + HALO] + tile[ty + HALO - 1][tx + HALO]);
      fma_real(acc, a.wy[1], tile[ty + HALO + 2][tx + HALO] + tile[ty + HALO - 2][tx + HALO]);
      fma_real(acc, a.wy[2], tile[ty + HALO + 3][tx + HALO] + tile[ty + HALO - 3][tx + HALO]);
      fma_real(acc, a.wz[0], q[4] + q[2]);
      fma_real(acc, a.wz[1], q[5] + q[1]);
      fma_real(acc, a.wz[2], q[6] + q[0]);
      dst[r] = acc;
      if (cp) cp[r] = q[3];   // the point itself: no wrap, no phase
    }
  }
}

template <class T>
int kinetic_local_impl(pawfd_ctx* c, const T* psi, int nb, T* out, T* cpy) {
  using R = real_t<T>;
  StencilArgs<R> a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = (R)(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = (R)(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = (R)(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  for (int cc = 0; cc < 3; ++cc) {
    const double kl = c->k[cc] * c->cell[cc];
    a.ph[cc] = cplx<R>{(R)cos(kl), (R)sin(kl)};
  }
  a.vshift = (const R*)c->d_vshift;
  const int gx = (a.n1 + TX - 1) / TX, gy = (a.n2 + TY - 1) / TY;
  const long long tiles = (long long)gx * gy;
  // split z so that one launch has at least `per_sm` CTAs per SM (default 4)
  const long long per_sm = c->stencil_zsplit > 0 ? c->stencil_zsplit : 4;
  long long want = (per_sm * c->num_sms + tiles * nb - 1) / (tiles * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 3) / 4));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gx, gy, nbl * a.nzc), block(TX, TY);
    a.cpy = cpy ? (void*)(cpy + (size_t)b0 * c->K) : nullptr;
    kinetic_local_kernel<T><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local launch");
}

}  // namespace

int launch_kinetic_local_f32x4(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy);
int launch_kinetic_local_ring(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy);
int launch_kinetic_local_ring_c(pawfd_ctx* c, const zf* psi, int nb, zf* out, zf* cpy);
int launch_kinetic_local_fx(pawfd_ctx* c, const double* psi, int nb, double* out, double* cpy);
int launch_kinetic_local_fx_c(pawfd_ctx* c, const zd* psi, int nb, zd* out, zd* cpy);

// out = (-1/2 Lap + v) psi; with cpy != null the kernels also write psi to cpy (the first term
// of S psi = psi + sum |p> dS <p|psi>), which saves the separate copy pass
int launch_kinetic_local(pawfd_ctx* c, const void* psi, int nb, void* out, void* cpy) {
  if (c->dtype == PAWFD_R64 && c->stencil_fx && c->fast_stencil &&
      launch_kinetic_local_fx(c, (const double*)psi, nb, (double*)out, (double*)cpy) == PAWFD_OK)
    return PAWFD_OK;
  if (c->dtype == PAWFD_C128 && c->stencil_fx && c->fast_stencil &&
      launch_kinetic_local_fx_c(c, (const zd*)psi, nb, (zd*)out, (zd*)cpy) == PAWFD_OK)
    return PAWFD_OK;
  if (c->dtype == PAWFD_R32 && c->fast_stencil) {
    if (c->stencil_variant != 1 &&
        launch_kinetic_local_ring(c, (const float*)psi, nb, (float*)out, (float*)cpy) == PAWFD_OK)
      return PAWFD_OK;
    if (launch_kinetic_local_f32x4(c, (const float*)psi, nb, (float*)out, (float*)cpy) == PAWFD_OK)
      return PAWFD_OK;
  }
  if (c->dtype == PAWFD_C64 && c->fast_stencil && c->stencil_variant != 1 &&
      launch_kinetic_local_ring_c(c, (const zf*)psi, nb, (zf*)out, (zf*)cpy) == PAWFD_OK)
    return PAWFD_OK;
  return dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    return kinetic_local_impl<T>(c, (const T*)psi, nb, (T*)out, (T*)cpy);
  });
}

}  // namespace pawfd
