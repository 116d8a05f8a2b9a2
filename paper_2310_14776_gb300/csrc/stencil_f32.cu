// stencil_f32.cu -- bandwidth-oriented kinetic + local kernel for FP32 real band arrays.
//
// Same operator as stencil.cu (order-6 central second difference per axis, periodic wrap,
// fused local potential; Eq. (dh) of the PAW section), specialised for the mixed form where
// it is bound by HBM bandwidth: 8 bytes per point-band (read psi once, write once).
//
// Layout of the work: a CTA owns a TX x BY (x, y) tile of one band and marches along z.  Each
// thread computes 4 consecutive x points (float4 loads and stores).  The +-3 z neighbours
// live in a register queue (7 float4 per thread); the current z plane of the tile plus its
// y halo (3 rows each side) and x halo (one float4 each side) is staged in a double-buffered
// shared-memory plane, so x and y neighbours cost 9 shared-memory float4 reads per 4 points.
// The halo of plane z+1 is fetched into registers while plane z is computed.  Periodic wrap
// is plain modular row / column indexing (x in whole float4 units, hence N1 % 4 == 0).
#include <algorithm>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int BYMAX = 16;

struct F32Args {
  int n1, n2, n3;
  int n1v;                 // N1 / 4 (float4 per row)
  long long K;
  float wx[3], wy[3], wz[3];
  const float* vshift;
  int zchunk, nzc;
  float* cpy;              // optional copy of psi (first band of this launch), or null
};

__device__ __forceinline__ float4 ld4(const float* __restrict__ p) { return __ldg((const float4*)p); }

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// BX threads along x (4 points each), BY along y
template <int BX, int BY>
__global__ void __launch_bounds__(BX* BY) kinetic_local_f32x4_kernel(const float* __restrict__ psi,
                                                                      float* __restrict__ out, F32Args a) {
  constexpr int TX = 4 * BX;
  constexpr int SW = TX + 8;          // plane row: 4 halo floats each side
  constexpr int SH = BY + 6;
  __shared__ __align__(16) float plane[2][SH][SW];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * BY;
  const int band = blockIdx.z / a.nzc, zc = blockIdx.z % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const float* __restrict__ src = psi + (long long)band * a.K;
  float* __restrict__ dst = out + (long long)band * a.K;
  float* __restrict__ cp = a.cpy ? a.cpy + (long long)band * a.K : nullptr;
  const int x = X0 + 4 * tx, y = Y0 + ty;
  // plane row r holds global row wrap(Y0 - 3 + r); threads past the last row of a ragged tile
  // still load their (wrapped) row so that the y neighbours of the last rows are right
  const int yy = wrapi(y, a.n2);
  const bool loads = x < a.n1;
  const bool active = loads && y < a.n2;
  const long long rowlen = a.n1;
  auto at = [&](int zz, int yy) -> long long { return ((long long)zz * a.n2 + yy) * rowlen; };

  // halo work of this thread: y-halo rows (ty < 6, all BX columns), x-halo float4 (tx == 0
  // left, tx == BX - 1 right) of the own row
  const bool yhalo = ty < 6 && loads;
  const int hy = ty < 3 ? wrapi(Y0 - 3 + ty, a.n2) : wrapi(Y0 + BY + (ty - 3), a.n2);
  const int hrow = ty < 3 ? ty : BY + ty;   // plane row of this halo row
  const bool xl = tx == 0 && y < a.n2, xr = (tx == BX - 1 || x + 4 >= a.n1) && y < a.n2 && x < a.n1;
  const int xlv = wrapi(X0 / 4 - 1, a.n1v) * 4;
  const int xrv = wrapi(x / 4 + 1, a.n1v) * 4;

  float4 q[7];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int zz = wrapi(z0 - 3 + j, a.n3);
    q[j + 1] = loads ? ld4(src + at(zz, yy) + x) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // halo of the first plane
  float4 hy4 = make_float4(0.f, 0.f, 0.f, 0.f), hl4 = hy4, hr4 = hy4;
  {
    const int zz = wrapi(z0, a.n3);
    if (yhalo) hy4 = ld4(src + at(zz, hy) + x);
    if (xl) hl4 = ld4(src + at(zz, y) + xlv);
    if (xr) hr4 = ld4(src + at(zz, y) + xrv);
  }
  int buf = 0;
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 6; ++j) q[j] = q[j + 1];
    const int zn = wrapi(z + 3, a.n3);
    q[6] = loads ? ld4(src + at(zn, yy) + x) : make_float4(0.f, 0.f, 0.f, 0.f);
    // stage plane z
    float(*P)[SW] = plane[buf];
    if (loads) *(float4*)&P[ty + 3][4 + 4 * tx] = q[3];
    if (yhalo) *(float4*)&P[hrow][4 + 4 * tx] = hy4;
    if (xl) *(float4*)&P[ty + 3][0] = hl4;
    if (xr) *(float4*)&P[ty + 3][4 + 4 * tx + 4] = hr4;
    // prefetch the halo of plane z + 1
    if (z + 1 < z1) {
      const int zz = wrapi(z + 1, a.n3);
      if (yhalo) hy4 = ld4(src + at(zz, hy) + x);
      if (xl) hl4 = ld4(src + at(zz, y) + xlv);
      if (xr) hr4 = ld4(src + at(zz, y) + xrv);
    }
    __syncthreads();
    if (active) {
      const int c = 4 + 4 * tx;
      const float4 L = *(const float4*)&P[ty + 3][c - 4];
      const float4 C = *(const float4*)&P[ty + 3][c];
      const float4 R = *(const float4*)&P[ty + 3][c + 4];
      const float w[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, R.x, R.y, R.z, R.w};
      float4 ym[3], yp[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        ym[m] = *(const float4*)&P[ty + 2 - m][c];
        yp[m] = *(const float4*)&P[ty + 4 + m][c];
      }
      const float4 v = ld4(a.vshift + at(z, y) + x);
      float r[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float ctr = w[4 + i];
        float acc = (&v.x)[i] * ctr;
        acc = fmaf(a.wx[0], w[5 + i] + w[3 + i], acc);
        acc = fmaf(a.wx[1], w[6 + i] + w[2 + i], acc);
        acc = fmaf(a.wx[2], w[7 + i] + w[1 + i], acc);
        acc = fmaf(a.wy[0], (&yp[0].x)[i] + (&ym[0].x)[i], acc);
        acc = fmaf(a.wy[1], (&yp[1].x)[i] + (&ym[1].x)[i], acc);
        acc = fmaf(a.wy[2], (&yp[2].x)[i] + (&ym[2].x)[i], acc);
        acc = fmaf(a.wz[0], (&q[4].x)[i] + (&q[2].x)[i], acc);
        acc = fmaf(a.wz[1], (&q[5].x)[i] + (&q[1].x)[i], acc);
        acc = fmaf(a.wz[2], (&q[6].x)[i] + (&q[0].x)[i], acc);
        r[i] = acc;
      }
      *(float4*)(dst + at(z, y) + x) = make_float4(r[0], r[1], r[2], r[3]);
      if (cp) *(float4*)(cp + at(z, y) + x) = C;
    }
    buf ^= 1;
  }
}

template <int BX, int BY>
void launch_f32x4(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy, const F32Args& a0) {
  F32Args a = a0;
  const int gx = (a.n1 + 4 * BX - 1) / (4 * BX), gy = (a.n2 + BY - 1) / BY;
  const long long tiles = (long long)gx * gy;
  long long want = (4ll * c->num_sms + tiles * nb - 1) / (tiles * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 7) / 8));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gx, gy, nbl * a.nzc), block(BX, BY);
    a.cpy = cpy ? cpy + (size_t)b0 * c->K : nullptr;
    kinetic_local_f32x4_kernel<BX, BY><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K,
                                                                       out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
}

}  // namespace

// FP32 real band arrays with N1 a multiple of 4 (16-byte rows); returns PAWFD_EINVAL when the
// shape does not qualify, so the caller can use the general kernel.
int launch_kinetic_local_f32x4(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy) {
  if (c->dtype != PAWFD_R32 || c->n[0] % 4 != 0 || c->n[0] < 4) return PAWFD_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out | (uintptr_t)cpy) & 15) return PAWFD_EINVAL;
  F32Args a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.n1v = c->n[0] / 4;
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = (float)(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = (float)(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = (float)(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  a.vshift = (const float*)c->d_vshift;
  a.zchunk = a.n3;
  a.nzc = 1;
  const int n1v = a.n1v;
  if (n1v >= 32) launch_f32x4<32, BYMAX>(c, psi, nb, out, cpy, a);
  else if (n1v >= 24) launch_f32x4<24, BYMAX>(c, psi, nb, out, cpy, a);
  else if (n1v >= 16) launch_f32x4<16, BYMAX>(c, psi, nb, out, cpy, a);
  else launch_f32x4<8, BYMAX>(c, psi, nb, out, cpy, a);
  return check_cuda(c, cudaGetLastError(), "kinetic_local f32x4 launch");
}

}  // namespace pawfd
