// stencil_df.cu -- kinetic + local kernel for real FP64 bands, computed in double-float.
//
// Same operator as stencil.cu (order-6 central second difference per axis, periodic wrap,
// fused local potential; Eq. (dh) of the PAW section), for real FP64 band arrays.  GB300
// issues about two FP64 FMAs per SM and clock, 1/64 of its FP32 rate, so the FP64 stencil
// (19 FP64 operations per point) is bound by the FP64 pipe.  Here every value is carried as
// an unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits):
//   * the FP64 input is split into hi (rounded to 24 bits) and lo (the rest, rounded to 24
//     bits) with integer operations on the IEEE fields, off the FP64 pipe;
//   * the 19-term sum uses error-free transformations (TwoSum; products with FMA), about 190
//     FP32 operations per point, with relative error of order 2^-46 of the terms; the x, y
//     and z terms form three independent chains that are merged at the end;
//   * only the final hi + lo uses the FP64 pipe (one addition per point; both parts are
//     widened to FP64 with integer operations).
// Layout of the work as the general kernel: a CTA owns a 32 x 8 (x, y) column of one band and
// marches along z, the z neighbours in a register queue, the plane (with halo) in shared memory.
#include <algorithm>

#include "df_arith.cuh"
#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

using namespace dfa;

constexpr int TX = 32, TY = 8, HALO = 3;
constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO;

struct DFArgs {
  int n1, n2, n3;
  long long K;
  DF wx[3], wy[3], wz[3];   // -1/2 w_m / h_c^2 as hi + lo
  const float2* vshift;     // v(r) - 1/2 w_0 sum 1/h_c^2 as (hi, lo)
  int zchunk, nzc;
  double* cpy;              // optional copy of psi (first band of this launch), or null
};

// acc += w (p + m), acc kept as (hi exact FP32 sum, lo collecting every rounding error)
__device__ __forceinline__ void tap(DF& acc, DF w, DF p, DF m) {
  float s, e;
  two_sum(p.hi, m.hi, s, e);
  const float slo = e + (p.lo + m.lo);
  const float ph = s * w.hi;
  float pe = fmaf(s, w.hi, -ph);
  pe = fmaf(s, w.lo, pe);
  pe = fmaf(slo, w.hi, pe);
  float t, te;
  two_sum(acc.hi, ph, t, te);
  acc.hi = t;
  acc.lo += te + pe;
}

// w (p + m) as a new pair (hi: the rounded product, lo: every rounding error so far)
__device__ __forceinline__ DF tap0(DF w, DF p, DF m) {
  float s, e;
  two_sum(p.hi, m.hi, s, e);
  const float slo = e + (p.lo + m.lo);
  const float ph = s * w.hi;
  float pe = fmaf(s, w.hi, -ph);
  pe = fmaf(s, w.lo, pe);
  pe = fmaf(slo, w.hi, pe);
  return {ph, pe};
}

// acc += b (pairs): the high parts added error-free, the low parts and the error summed
__device__ __forceinline__ void merge(DF& acc, DF b) {
  float t, te;
  two_sum(acc.hi, b.hi, t, te);
  acc.hi = t;
  acc.lo += te + b.lo;
}

// wrapped index (|i| at most one period away from the cell, as for a stencil halo)
__device__ __forceinline__ int wrap1(int i, int n) {
  i = i < 0 ? i + n : i;
  return i >= n ? i - n : i;
}

__device__ __forceinline__ DF load_split(const double* __restrict__ src, int u1, int u2, int u3, const DFArgs& a) {
  return split64(src[((long long)wrap1(u3, a.n3) * a.n2 + wrap1(u2, a.n2)) * a.n1 + wrap1(u1, a.n1)]);
}

// halo cells of the (SY x SX) plane tile: HCELLS = SX SY - TX TY, at most HPER per thread
constexpr int HCELLS = SX * SY - TX * TY;
constexpr int HPER = (HCELLS + TX * TY - 1) / (TX * TY);

// (ly, lx) of halo cell h: the 3 rows above, the 3 rows below, then the 3 + 3 side columns of
// the TY interior rows
__device__ __forceinline__ void halo_cell(int h, int& ly, int& lx) {
  if (h < HALO * SX) {
    ly = h / SX;
    lx = h - ly * SX;
  } else if (h < 2 * HALO * SX) {
    h -= HALO * SX;
    ly = HALO + TY + h / SX;
    lx = h % SX;
  } else {
    h -= 2 * HALO * SX;
    ly = HALO + h / (2 * HALO);
    const int c = h % (2 * HALO);
    lx = c < HALO ? c : TX + c;
  }
}

// Requires N1 >= TX + 2 HALO + 2, N2 >= TY + 2 HALO, N3 >= HALO, so that every index a tile
// touches is at most one period outside the cell (one conditional wrap).
__global__ void __launch_bounds__(TX * TY) kinetic_local_df_kernel(const double* __restrict__ psi,
                                                                  double* __restrict__ out, DFArgs a) {
  __shared__ DF tile[2][SY][SX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
  const int band = blockIdx.z / a.nzc, zc = blockIdx.z % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const double* __restrict__ src = psi + (long long)band * a.K;
  double* __restrict__ dst = out + (long long)band * a.K;
  double* __restrict__ cp = a.cpy ? a.cpy + (long long)band * a.K : nullptr;
  const int x = X0 + tx, y = Y0 + ty;
  const bool active = x < a.n1 && y < a.n2;
  // this thread's halo cells
  int hy[HPER], hx[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k) {
    const int h = tid + k * TX * TY;
    if (h < HCELLS) halo_cell(h, hy[k], hx[k]);
    else hy[k] = hx[k] = -1;
  }

  // every thread carries its own (possibly wrapped) column: the tile's interior comes from it
  DF q[7];
#pragma unroll
  for (int j = 0; j < 6; ++j) q[j + 1] = load_split(src, x, y, z0 - 3 + j, a);
  DF hv[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k)
    if (hy[k] >= 0) hv[k] = load_split(src, X0 - HALO + hx[k], Y0 - HALO + hy[k], z0, a);

  int buf = 0;
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 6; ++j) q[j] = q[j + 1];
    q[6] = load_split(src, x, y, z + 3, a);
    // stage plane z (halo prefetched during the previous step) in this step's buffer
    DF(*T)[SX] = tile[buf];
    T[ty + HALO][tx + HALO] = q[3];
#pragma unroll
    for (int k = 0; k < HPER; ++k)
      if (hy[k] >= 0) T[hy[k]][hx[k]] = hv[k];
    __syncthreads();
    // prefetch the halo of plane z + 1 while plane z is computed
    if (z + 1 < z1) {
#pragma unroll
      for (int k = 0; k < HPER; ++k)
        if (hy[k] >= 0) hv[k] = load_split(src, X0 - HALO + hx[k], Y0 - HALO + hy[k], z + 1, a);
    }
    if (active) {
      const long long r = ((long long)z * a.n2 + y) * a.n1 + x;
      const float2 v = __ldg(a.vshift + r);
      const DF c = q[3];
      DF acc;
      acc.hi = v.x * c.hi;
      float pe = fmaf(v.x, c.hi, -acc.hi);
      pe = fmaf(v.x, c.lo, pe);
      acc.lo = fmaf(v.y, c.hi, pe);
      // three independent chains (x, y, z terms) for instruction-level parallelism, merged
      // into the potential term with the same error-free additions
      const DF* row = &T[ty + HALO][tx + HALO];
      DF ax = tap0(a.wx[0], row[1], row[-1]);
      DF ay = tap0(a.wy[0], T[ty + HALO + 1][tx + HALO], T[ty + HALO - 1][tx + HALO]);
      DF az = tap0(a.wz[0], q[4], q[2]);
      tap(ax, a.wx[1], row[2], row[-2]);
      tap(ay, a.wy[1], T[ty + HALO + 2][tx + HALO], T[ty + HALO - 2][tx + HALO]);
      tap(az, a.wz[1], q[5], q[1]);
      tap(ax, a.wx[2], row[3], row[-3]);
      tap(ay, a.wy[2], T[ty + HALO + 3][tx + HALO], T[ty + HALO - 3][tx + HALO]);
      tap(az, a.wz[2], q[6], q[0]);
      merge(ax, ay);
      merge(acc, az);
      merge(acc, ax);
      dst[r] = f2d(acc.hi) + f2d(acc.lo);   // one FP64 operation per point
      if (cp) cp[r] = src[r];                // exact value (the pair holds 48 bits); L1/L2 hit
    }
    buf ^= 1;
  }
}

DF split_host(double w) {
  const float hi = (float)w;
  return {hi, (float)(w - (double)hi)};
}

}  // namespace

// Real FP64 contexts with the double-float potential table; EINVAL otherwise.
int launch_kinetic_local_df(pawfd_ctx* c, const double* psi, int nb, double* out, double* cpy) {
  if (c->dtype != PAWFD_R64 || !c->d_vshift_df) return PAWFD_EINVAL;
  // one wrap per index must reach every point a tile touches (own points run up to TX - 1 and
  // halos HALO past the tile): smaller grids use the general kernel
  if (c->n[0] < TX + 2 * HALO + 2 || c->n[1] < TY + 2 * HALO || c->n[2] < HALO) return PAWFD_EINVAL;
  DFArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = split_host(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = split_host(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = split_host(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  a.vshift = (const float2*)c->d_vshift_df;
  const int gx = (a.n1 + TX - 1) / TX, gy = (a.n2 + TY - 1) / TY;
  const long long tiles = (long long)gx * gy;
  const long long per_sm = c->stencil_zsplit > 0 ? c->stencil_zsplit : 4;
  long long want = (per_sm * c->num_sms + tiles * nb - 1) / (tiles * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 3) / 4));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gx, gy, nbl * a.nzc), block(TX, TY);
    a.cpy = cpy ? cpy + (size_t)b0 * c->K : nullptr;
    kinetic_local_df_kernel<<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local double-float launch");
}

}  // namespace pawfd
