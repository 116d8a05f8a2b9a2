// stencil_fx.cu -- kinetic + local kernel for FP64 bands (real, and complex Bloch bands) in exact
// fixed-point arithmetic.
//
// Same operator as stencil.cu (order-6 central second difference per axis, periodic wrap,
// fused local potential; Eq. (dh) of the PAW section), for real FP64 band arrays.  GB300
// issues about two FP64 FMAs per SM and clock, so the 19 FP64 operations per point of the
// plain kernel bound it; this kernel moves the stencil itself to the integer pipes:
//   * the order-6 weights times 180 are the integers (-490, 270, -27, 2), so
//       180 sum_m w_|m| psi(r + m e_c) = -490 q0 + 270 (q+1 + q-1) - 27 (q+2 + q-2) + 2 (q+3 + q-3)
//     is exact in integer arithmetic once psi is an integer;
//   * every value of a CTA's slab (its 32 x 8 column over a range of z planes, with the
//     three-point halo) is rounded to an integer q = round(psi 2^(1073 - eb)), eb the largest
//     IEEE exponent field in the slab, so |q| <= 2^51: one rounding per value of at most half a
//     unit in 2^(eb - 1074), the size of an FP64 rounding of the slab's largest values;
//   * with |q| <= 2^51 the cubic-cell sum over the three axes is at most
//     (3 * 2 * 299 + 3 * 490) 2^51 < 2^63 and fits a 64-bit integer; other cells sum per axis;
//   * the exact integer sum is converted to FP64 once (one rounding, relative to the second
//     difference itself, not to the terms it cancels), scaled, and added to v psi with one
//     FP64 multiply and one FMA: two FP64 operations per point instead of nineteen (one more
//     for slabs of values so small that the folded scale factor would leave the normal range).
// So the error is that of rounding the inputs once to the slab's FP64 grid plus two roundings
// of the result, independent of the cancellation between the stencil's terms, which sets the
// error of a floating-point evaluation on smooth bands.
// Layout of the work: a CTA owns a 32 x 8 (x, y) column of one band and a range of z planes;
// it first reads its slab once for the largest exponent (the slab is short enough to stay in
// L2 for the second read), then marches along z with the z neighbours in a register queue and
// the current plane (with halo) in shared memory.  A slab holding an infinity or NaN is
// computed in plain FP64 arithmetic instead.
#include <algorithm>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int TX = 32, TY = 8, HALO = 3;
constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO;
constexpr int NTHR = TX * TY;
constexpr int HCELLS = SX * SY - TX * TY;
constexpr int HPER = (HCELLS + NTHR - 1) / NTHR;
constexpr int ZSLAB = 16;   // target z planes per CTA (the slab's two reads share L2)

struct FXArgs {
  int n1, n2, n3;
  long long K;
  double cs[3];        // -1 / (360 h_c^2)
  double ih2[3];       // 1 / h_c^2 (plain FP64 path)
  const double* v;     // v(r), FP64
  int zchunk, nzc;
  double* cpy;         // optional copy of psi (first band of this launch), or null
};

__device__ __forceinline__ int wrap1(int i, int n) {
  i = i < 0 ? i + n : i;
  return i >= n ? i - n : i;
}

__device__ __forceinline__ int exp_field(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu);
}

// q = round(x 2^(1073 - ebp)) for finite x whose exponent field is at most ebp (>= 1):
// |x| = m 2^(e' - 1075) with the 53-bit significand m and e' = max(e, 1), so
// q = m 2^-(ebp + 2 - e') rounded half away from zero, |q| <= 2^51.
__device__ __forceinline__ long long to_fixed(double x, int ebp) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FFu);
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  const int s = min(ebp + 2 - max(e, 1), 63);
  const unsigned long long q = (m + (1ull << (s - 1))) >> s;
  return (long long)((b >> 63) ? (0ull - q) : q);
}

// The FP64 value of v rounded to nearest, ties to even (IEEE 754), on the integer pipes: the
// magnitude is normalised so that its leading one sits at bit 63, its top 53 bits are the
// significand and the 11 below decide the rounding; adding the significand (hidden bit
// included) to (exponent - 1) << 52 carries a rounded-up 2^53 into the exponent by itself.
// The FP64 pipe, a few percent of the integer rate on this GPU, then only has the scaling
// FMA and v psi.
__device__ __forceinline__ double i64_to_f64(long long v) {
  const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  if (a == 0) return 0.0;
  const int lz = __clzll((long long)a);
  const unsigned long long nrm = a << lz;
  const unsigned long long m = nrm >> 11, r = nrm & 0x7FFull;
  const unsigned long long up = (r > 0x400ull || (r == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  const unsigned long long e = (unsigned long long)(1023 + 63 - lz);
  return __longlong_as_double((long long)(sign + ((e - 1ull) << 52) + m + up));
}

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

// The slab in plain FP64 arithmetic (only when it holds an infinity or NaN, so that those
// propagate as in a floating-point evaluation).
__device__ void fp64_slab(const double* __restrict__ src, double* __restrict__ dst, double* __restrict__ cp,
                          int x, int y, int z0, int z1, const FXArgs& a) {
  constexpr double w1 = 270.0 / 180.0, w2 = -27.0 / 180.0, w3 = 2.0 / 180.0, w0 = -490.0 / 180.0;
  for (int z = z0; z < z1; ++z) {
    auto at = [&](int u1, int u2, int u3) {
      return src[((long long)wrap1(u3, a.n3) * a.n2 + wrap1(u2, a.n2)) * a.n1 + wrap1(u1, a.n1)];
    };
    const long long r = ((long long)z * a.n2 + y) * a.n1 + x;
    const double c = src[r];
    double lap = 0.0;
    lap += a.ih2[0] * (w0 * c + w1 * (at(x + 1, y, z) + at(x - 1, y, z)) + w2 * (at(x + 2, y, z) + at(x - 2, y, z)) +
                       w3 * (at(x + 3, y, z) + at(x - 3, y, z)));
    lap += a.ih2[1] * (w0 * c + w1 * (at(x, y + 1, z) + at(x, y - 1, z)) + w2 * (at(x, y + 2, z) + at(x, y - 2, z)) +
                       w3 * (at(x, y + 3, z) + at(x, y - 3, z)));
    lap += a.ih2[2] * (w0 * c + w1 * (at(x, y, z + 1) + at(x, y, z - 1)) + w2 * (at(x, y, z + 2) + at(x, y, z - 2)) +
                       w3 * (at(x, y, z + 3) + at(x, y, z - 3)));
    dst[r] = a.v[r] * c - 0.5 * lap;
    if (cp) cp[r] = c;
  }
}

// Requires N1 >= TX + 2 HALO + 2, N2 >= TY + 2 HALO, N3 >= HALO, so that every index a tile
// touches is at most one period outside the cell (one conditional wrap).
template <bool CUBIC>
__global__ void __launch_bounds__(NTHR) kinetic_local_fx_kernel(const double* __restrict__ psi,
                                                                  double* __restrict__ out, FXArgs a) {
  __shared__ long long tile[2][SY][SX];
  __shared__ int s_emax[NTHR / 32];
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
  const long long plane = (long long)a.n1 * a.n2;
  // this thread's column and halo cells, as offsets within a plane (wrapped)
  const long long own = (long long)wrap1(y, a.n2) * a.n1 + wrap1(x, a.n1);
  int hy[HPER], hx[HPER];
  long long hoff[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k) {
    const int h = tid + k * NTHR;
    if (h < HCELLS) {
      halo_cell(h, hy[k], hx[k]);
      hoff[k] = (long long)wrap1(Y0 - HALO + hy[k], a.n2) * a.n1 + wrap1(X0 - HALO + hx[k], a.n1);
    } else {
      hy[k] = hx[k] = -1;
      hoff[k] = 0;
    }
  }

  // 1. the largest exponent field of the values the slab reads: the column over planes
  //    z0 - 3 .. z1 + 2, the halo over planes z0 .. z1 - 1
  int emax = 0;
  for (int z = z0 - HALO; z < z1 + HALO; ++z) {
    const double* p = src + (long long)wrap1(z, a.n3) * plane;
    emax = max(emax, exp_field(p[own]));
    if (z >= z0 && z < z1) {
#pragma unroll
      for (int k = 0; k < HPER; ++k)
        if (hy[k] >= 0) emax = max(emax, exp_field(p[hoff[k]]));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((tid & 31) == 0) s_emax[tid >> 5] = emax;
  __syncthreads();
  int eb = 0;
#pragma unroll
  for (int w = 0; w < NTHR / 32; ++w) eb = max(eb, s_emax[w]);
  if (eb == 0x7FF) {   // an infinity or NaN in the slab: plain FP64 (uniform over the CTA)
    if (active) fp64_slab(src, dst, cp, x, y, z0, z1, a);
    return;
  }
  const int ebp = max(eb, 1);
  // value of one integer unit: 2^(ebp - 1073).  Folded into the axis factors unless that
  // product could leave the normal range (slabs of values below about 2^-895); then the sums
  // are scaled by the axis factors first and by the unit after (one more FP64 multiply).
  const bool folded = ebp >= 128;
  const double unit = ldexp(1.0, ebp - 1073);
  double cs[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) cs[c] = folded ? a.cs[c] * unit : a.cs[c];

  // 2. the march along z: q[j] holds plane z - 3 + j of this thread's column, raw[j] the FP64
  //    values of planes z .. z + 3
  long long q[7];
  double raw[4];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const double val = src[(long long)wrap1(z0 - 3 + j, a.n3) * plane + own];
    q[j + 1] = to_fixed(val, ebp);
    if (j >= 3) raw[j - 2] = val;
  }
  double hv[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k)
    if (hy[k] >= 0) hv[k] = src[(long long)z0 * plane + hoff[k]];

  int buf = 0;
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 6; ++j) q[j] = q[j + 1];
#pragma unroll
    for (int j = 0; j < 3; ++j) raw[j] = raw[j + 1];
    raw[3] = src[(long long)wrap1(z + 3, a.n3) * plane + own];
    q[6] = to_fixed(raw[3], ebp);
    long long(*T)[SX] = tile[buf];
    T[ty + HALO][tx + HALO] = q[3];
#pragma unroll
    for (int k = 0; k < HPER; ++k)
      if (hy[k] >= 0) T[hy[k]][hx[k]] = to_fixed(hv[k], ebp);
    __syncthreads();
    // prefetch the halo of plane z + 1 while plane z is computed
    if (z + 1 < z1) {
#pragma unroll
      for (int k = 0; k < HPER; ++k)
        if (hy[k] >= 0) hv[k] = src[(long long)(z + 1) * plane + hoff[k]];
    }
    if (active) {
      const long long r = (long long)z * plane + (long long)y * a.n1 + x;
      const long long* row = &T[ty + HALO][tx + HALO];
      const long long c0 = q[3];
      const double vx = __ldg(a.v + r) * raw[0];
      double res;
      if (CUBIC) {
        const long long V1 = (row[1] + row[-1]) + (T[ty + HALO + 1][tx + HALO] + T[ty + HALO - 1][tx + HALO]) +
                             (q[4] + q[2]);
        const long long V2 = (row[2] + row[-2]) + (T[ty + HALO + 2][tx + HALO] + T[ty + HALO - 2][tx + HALO]) +
                             (q[5] + q[1]);
        const long long V3 = (row[3] + row[-3]) + (T[ty + HALO + 3][tx + HALO] + T[ty + HALO - 3][tx + HALO]) +
                             (q[6] + q[0]);
        const long long S = 270ll * V1 - 27ll * V2 + 2ll * V3 - 1470ll * c0;
        res = folded ? fma(i64_to_f64(S), cs[0], vx) : fma(i64_to_f64(S) * cs[0], unit, vx);
      } else {
        const long long c490 = 490ll * c0;
        const long long Sx = 270ll * (row[1] + row[-1]) - 27ll * (row[2] + row[-2]) + 2ll * (row[3] + row[-3]) - c490;
        const long long Sy = 270ll * (T[ty + HALO + 1][tx + HALO] + T[ty + HALO - 1][tx + HALO]) -
                             27ll * (T[ty + HALO + 2][tx + HALO] + T[ty + HALO - 2][tx + HALO]) +
                             2ll * (T[ty + HALO + 3][tx + HALO] + T[ty + HALO - 3][tx + HALO]) - c490;
        const long long Sz = 270ll * (q[4] + q[2]) - 27ll * (q[5] + q[1]) + 2ll * (q[6] + q[0]) - c490;
        if (folded) {
          res = fma(i64_to_f64(Sx), cs[0], fma(i64_to_f64(Sy), cs[1], fma(i64_to_f64(Sz), cs[2], vx)));
        } else {
          const double t = fma(i64_to_f64(Sx), cs[0], fma(i64_to_f64(Sy), cs[1], i64_to_f64(Sz) * cs[2]));
          res = fma(t, unit, vx);
        }
      }
      dst[r] = res;
      if (cp) cp[r] = raw[0];
    }
    buf ^= 1;
  }
}

// ------------------------------------------------------------------------------------------
// Complex (Bloch) FP64 bands: the same fixed-point scheme on the real and imaginary parts (the
// stencil's weights are real).  A neighbour that leaves the cell across face c carries the
// Bloch factor exp(+-i k_c L_c) (at most one crossing per index on the grids this tiling
// admits); it is applied in FP64 before the value is rounded to the slab's grid.  A rotated
// component can exceed the slab's largest component by up to a factor sqrt(2), so the grid
// unit is taken one exponent step higher, 2^(ebp - 1073) with ebp = eb + 1: |q| <= 2^51
// still holds, and every input is rounded once to within 2^(eb - 1073), twice the real
// kernel's half unit.  Slabs holding an infinity or NaN, values within a factor 2 of the top
// of the FP64 range (where a rotation could overflow), or only values below about 2^-896
// (where the unit folded into the axis factors would leave the normal range) are computed in
// plain FP64.

struct FXCArgs {
  int n1, n2, n3;
  long long K;
  double cs[3];        // -1 / (360 h_c^2)
  double ih2[3];       // 1 / h_c^2 (plain FP64 path)
  zd ph[3];            // exp(i k_c L_c)
  const double* v;     // v(r), FP64
  int zchunk, nzc;
  zd* cpy;             // optional copy of psi (first band of this launch), or null
};

__device__ __forceinline__ zd ldz(const zd* p) {
  const double2 t = __ldg((const double2*)p);
  return zd{t.x, t.y};
}
__device__ __forceinline__ void stz(zd* p, zd v) { *(double2*)p = make_double2(v.re, v.im); }

// -1, 0 or +1: the face an index at most one period outside [0, n) has crossed
__device__ __forceinline__ int crossing(int i, int n) { return i < 0 ? -1 : (i >= n ? 1 : 0); }

// the Bloch factor of the crossings t1, t2, t3
__device__ __forceinline__ zd bloch(int t1, int t2, int t3, const FXCArgs& a) {
  zd f = {1.0, 0.0};
  if (t1) f = f * (t1 > 0 ? a.ph[0] : conjx(a.ph[0]));
  if (t2) f = f * (t2 > 0 ? a.ph[1] : conjx(a.ph[1]));
  if (t3) f = f * (t3 > 0 ? a.ph[2] : conjx(a.ph[2]));
  return f;
}

// v times the Bloch factor of the crossings (t1, t2, t3).  Out of line: the wrapped case is
// rare (boundary tiles and planes), and inlined the compiler evaluated its FP64 products under
// a predicate for every halo and queue value (the FP64 pipe at 57 % for about 14 FP64
// instructions per point instead of four).
__device__ __noinline__ zd bloch_mul(zd v, int t1, int t2, int t3, zd p0, zd p1, zd p2) {
  if (t1) v = v * (t1 > 0 ? p0 : conjx(p0));
  if (t2) v = v * (t2 > 0 ? p1 : conjx(p1));
  if (t3) v = v * (t3 > 0 ? p2 : conjx(p2));
  return v;
}

__device__ void fp64_slab_c(const zd* __restrict__ src, zd* __restrict__ dst, zd* __restrict__ cp, int x, int y,
                            int z0, int z1, const FXCArgs& a) {
  constexpr double w1 = 270.0 / 180.0, w2 = -27.0 / 180.0, w3 = 2.0 / 180.0, w0 = -490.0 / 180.0;
  auto at = [&](int u1, int u2, int u3) -> zd {
    const int t1 = crossing(u1, a.n1), t2 = crossing(u2, a.n2), t3 = crossing(u3, a.n3);
    const zd v = src[((long long)wrap1(u3, a.n3) * a.n2 + wrap1(u2, a.n2)) * a.n1 + wrap1(u1, a.n1)];
    return (t1 | t2 | t3) ? v * bloch(t1, t2, t3, a) : v;
  };
  for (int z = z0; z < z1; ++z) {
    const long long r = ((long long)z * a.n2 + y) * a.n1 + x;
    const zd c = src[r];
    auto axis = [&](zd p1, zd m1, zd p2, zd m2, zd p3, zd m3) -> zd {
      return zd{w0 * c.re + w1 * (p1.re + m1.re) + w2 * (p2.re + m2.re) + w3 * (p3.re + m3.re),
                w0 * c.im + w1 * (p1.im + m1.im) + w2 * (p2.im + m2.im) + w3 * (p3.im + m3.im)};
    };
    const zd lx = axis(at(x + 1, y, z), at(x - 1, y, z), at(x + 2, y, z), at(x - 2, y, z), at(x + 3, y, z),
                       at(x - 3, y, z));
    const zd ly = axis(at(x, y + 1, z), at(x, y - 1, z), at(x, y + 2, z), at(x, y - 2, z), at(x, y + 3, z),
                       at(x, y - 3, z));
    const zd lz = axis(at(x, y, z + 1), at(x, y, z - 1), at(x, y, z + 2), at(x, y, z - 2), at(x, y, z + 3),
                       at(x, y, z - 3));
    const double vr = a.v[r];
    dst[r] = zd{vr * c.re - 0.5 * (a.ih2[0] * lx.re + a.ih2[1] * ly.re + a.ih2[2] * lz.re),
                vr * c.im - 0.5 * (a.ih2[0] * lx.im + a.ih2[1] * ly.im + a.ih2[2] * lz.im)};
    if (cp) cp[r] = c;
  }
}

// 180 x the order-6 second differences of one part at the thread's point: the cubic-cell sum
// over the three axes, or the per-axis sums (Sx, Sy, Sz)
__device__ __forceinline__ long long fx_sum_cubic(const long long (*T)[SX], int ty, int tx, const long long* q) {
  const long long* row = &T[ty + HALO][tx + HALO];
  const long long V1 = (row[1] + row[-1]) + (T[ty + HALO + 1][tx + HALO] + T[ty + HALO - 1][tx + HALO]) + (q[4] + q[2]);
  const long long V2 = (row[2] + row[-2]) + (T[ty + HALO + 2][tx + HALO] + T[ty + HALO - 2][tx + HALO]) + (q[5] + q[1]);
  const long long V3 = (row[3] + row[-3]) + (T[ty + HALO + 3][tx + HALO] + T[ty + HALO - 3][tx + HALO]) + (q[6] + q[0]);
  return 270ll * V1 - 27ll * V2 + 2ll * V3 - 1470ll * q[3];
}
__device__ __forceinline__ void fx_sum_axes(const long long (*T)[SX], int ty, int tx, const long long* q, long long& Sx,
                                            long long& Sy, long long& Sz) {
  const long long* row = &T[ty + HALO][tx + HALO];
  const long long c490 = 490ll * q[3];
  Sx = 270ll * (row[1] + row[-1]) - 27ll * (row[2] + row[-2]) + 2ll * (row[3] + row[-3]) - c490;
  Sy = 270ll * (T[ty + HALO + 1][tx + HALO] + T[ty + HALO - 1][tx + HALO]) -
       27ll * (T[ty + HALO + 2][tx + HALO] + T[ty + HALO - 2][tx + HALO]) +
       2ll * (T[ty + HALO + 3][tx + HALO] + T[ty + HALO - 3][tx + HALO]) - c490;
  Sz = 270ll * (q[4] + q[2]) - 27ll * (q[5] + q[1]) + 2ll * (q[6] + q[0]) - c490;
}

// Requires N1 >= TX + 2 HALO + 2, N2 >= TY + 2 HALO, N3 >= HALO (one crossing per index) and
// 16-byte aligned band arrays.
// Three CTAs per SM (80 registers, a little spilled) measured faster than two at 124 registers
// (38.3 against 42.5 ps per point at 144^3 x 128, before the out-of-line Bloch products took it
// to 33.0): the march is bound by the latency of each plane's loads, so more warps per SM pay
// more than the spilled registers cost.
template <bool CUBIC>
__global__ void __launch_bounds__(NTHR, 3) kinetic_local_fx_c_kernel(const zd* __restrict__ psi, zd* __restrict__ out,
                                                                    FXCArgs a) {
  __shared__ long long tile[2][2][SY][SX];   // [buffer][real / imaginary part]
  __shared__ int s_emax[NTHR / 32];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
  const int band = blockIdx.z / a.nzc, zc = blockIdx.z % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const zd* __restrict__ src = psi + (long long)band * a.K;
  zd* __restrict__ dst = out + (long long)band * a.K;
  zd* __restrict__ cp = a.cpy ? a.cpy + (long long)band * a.K : nullptr;
  const int x = X0 + tx, y = Y0 + ty;
  const bool active = x < a.n1 && y < a.n2;
  const long long plane = (long long)a.n1 * a.n2;
  // this thread's column (its x, y faces crossed when it lies past the cell's edge) and halo
  // cells, as wrapped offsets within a plane with their Bloch factors
  const long long own = (long long)wrap1(y, a.n2) * a.n1 + wrap1(x, a.n1);
  const int ox = crossing(x, a.n1), oy = crossing(y, a.n2);
  // halo cells: crossings of the x and y faces packed as (t1 + 1) + 3 (t2 + 1) (4: none); the
  // Bloch factor is formed when the value is rounded (boundary tiles only)
  int hy[HPER], hx[HPER], hcr[HPER];
  long long hoff[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k) {
    const int h = tid + k * NTHR;
    hcr[k] = 4;
    if (h < HCELLS) {
      halo_cell(h, hy[k], hx[k]);
      const int u1 = X0 - HALO + hx[k], u2 = Y0 - HALO + hy[k];
      hoff[k] = (long long)wrap1(u2, a.n2) * a.n1 + wrap1(u1, a.n1);
      hcr[k] = (crossing(u1, a.n1) + 1) + 3 * (crossing(u2, a.n2) + 1);
    } else {
      hy[k] = hx[k] = -1;
      hoff[k] = 0;
    }
  }

  // 1. the largest exponent field of the parts the slab reads
  int emax = 0;
  for (int z = z0 - HALO; z < z1 + HALO; ++z) {
    const zd* p = src + (long long)wrap1(z, a.n3) * plane;
    const zd v = ldz(p + own);
    emax = max(emax, max(exp_field(v.re), exp_field(v.im)));
    if (z >= z0 && z < z1) {
#pragma unroll
      for (int k = 0; k < HPER; ++k)
        if (hy[k] >= 0) {
          const zd w = ldz(p + hoff[k]);
          emax = max(emax, max(exp_field(w.re), exp_field(w.im)));
        }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((tid & 31) == 0) s_emax[tid >> 5] = emax;
  __syncthreads();
  int eb = 0;
#pragma unroll
  for (int w = 0; w < NTHR / 32; ++w) eb = max(eb, s_emax[w]);
  // plain FP64 for non-finite values, parts a rotation could overflow, and slabs of values so
  // small (below about 2^-895) that the unit folded into the axis factors would leave the
  // normal range: the march then has one form only (a per-CTA choice between two forms of the
  // final FMAs was evaluated under a predicate on both sides, FP64 work on every point)
  if (eb >= 0x7FE || eb < 126) {
    if (active) fp64_slab_c(src, dst, cp, x, y, z0, z1, a);
    return;
  }
  const int ebp = eb + 1;
  // 2^(ebp - 1073), a normal number for ebp >= 128, from its bit fields (no library call)
  const double unit = __longlong_as_double((long long)(ebp - 1073 + 1023) << 52);
  double cs[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) cs[c] = a.cs[c] * unit;
  // the own column's value of plane u3 on the grid: Bloch factor of the crossed faces, then
  // rounded
  auto own_fixed = [&](zd v, int u3, long long& qr, long long& qi) {
    const int t3 = crossing(u3, a.n3);
    if (ox | oy | t3) v = bloch_mul(v, ox, oy, t3, a.ph[0], a.ph[1], a.ph[2]);
    qr = to_fixed(v.re, ebp);
    qi = to_fixed(v.im, ebp);
  };

  // 2. the march along z: qr / qi[j] hold plane z - 3 + j of this thread's column on the grid;
  //    the FP64 value of the point itself (v psi, the copy) is read again when it is computed
  //    (from L1: the thread loaded it three planes earlier)
  long long qr[7], qi[7];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int u3 = z0 - 3 + j;
    const zd val = ldz(src + (long long)wrap1(u3, a.n3) * plane + own);
    own_fixed(val, u3, qr[j + 1], qi[j + 1]);
  }
  zd hv[HPER];
#pragma unroll
  for (int k = 0; k < HPER; ++k)
    if (hy[k] >= 0) hv[k] = ldz(src + (long long)z0 * plane + hoff[k]);

  int buf = 0;
  for (int z = z0; z < z1; ++z) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      qr[j] = qr[j + 1];
      qi[j] = qi[j + 1];
    }
    own_fixed(ldz(src + (long long)wrap1(z + 3, a.n3) * plane + own), z + 3, qr[6], qi[6]);
    long long(*TR)[SX] = tile[buf][0];
    long long(*TI)[SX] = tile[buf][1];
    TR[ty + HALO][tx + HALO] = qr[3];
    TI[ty + HALO][tx + HALO] = qi[3];
#pragma unroll
    for (int k = 0; k < HPER; ++k)
      if (hy[k] >= 0) {
        const zd w = hcr[k] != 4 ? bloch_mul(hv[k], hcr[k] % 3 - 1, hcr[k] / 3 - 1, 0, a.ph[0], a.ph[1], a.ph[2])
                                 : hv[k];
        TR[hy[k]][hx[k]] = to_fixed(w.re, ebp);
        TI[hy[k]][hx[k]] = to_fixed(w.im, ebp);
      }
    __syncthreads();
    if (z + 1 < z1) {
#pragma unroll
      for (int k = 0; k < HPER; ++k)
        if (hy[k] >= 0) hv[k] = ldz(src + (long long)(z + 1) * plane + hoff[k]);
    }
    if (active) {
      const long long r = (long long)z * plane + (long long)y * a.n1 + x;
      const zd c = ldz(src + r);
      const double vv = __ldg(a.v + r);
      const double vr = vv * c.re, vi = vv * c.im;
      double rre, rim;
      if (CUBIC) {
        rre = fma(i64_to_f64(fx_sum_cubic(TR, ty, tx, qr)), cs[0], vr);
        rim = fma(i64_to_f64(fx_sum_cubic(TI, ty, tx, qi)), cs[0], vi);
      } else {
        long long Sx, Sy, Sz;
        fx_sum_axes(TR, ty, tx, qr, Sx, Sy, Sz);
        rre = fma(i64_to_f64(Sx), cs[0], fma(i64_to_f64(Sy), cs[1], fma(i64_to_f64(Sz), cs[2], vr)));
        fx_sum_axes(TI, ty, tx, qi, Sx, Sy, Sz);
        rim = fma(i64_to_f64(Sx), cs[0], fma(i64_to_f64(Sy), cs[1], fma(i64_to_f64(Sz), cs[2], vi)));
      }
      stz(dst + r, zd{rre, rim});
      if (cp) stz(cp + r, c);
    }
    buf ^= 1;
  }
}

}  // namespace

// Real FP64 contexts on grids the tile fits (one wrap per index); EINVAL otherwise.
int launch_kinetic_local_fx(pawfd_ctx* c, const double* psi, int nb, double* out, double* cpy) {
  if (c->dtype != PAWFD_R64 || !c->d_vloc) return PAWFD_EINVAL;
  if (c->n[0] < TX + 2 * HALO + 2 || c->n[1] < TY + 2 * HALO || c->n[2] < HALO) return PAWFD_EINVAL;
  FXArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  for (int cc = 0; cc < 3; ++cc) {
    a.ih2[cc] = 1.0 / (c->h[cc] * c->h[cc]);
    a.cs[cc] = -1.0 / (360.0 * c->h[cc] * c->h[cc]);
  }
  a.v = (const double*)c->d_vloc;
  const bool cubic = c->h[0] == c->h[1] && c->h[1] == c->h[2];
  const int gx = (a.n1 + TX - 1) / TX, gy = (a.n2 + TY - 1) / TY;
  const long long tiles = (long long)gx * gy;
  // z slabs of about ZSLAB planes (their two reads meet in L2), more if a launch would
  // otherwise have fewer than `per_sm` CTAs per SM
  const long long per_sm = c->stencil_zsplit > 0 ? c->stencil_zsplit : 4;
  const long long want = std::max<long long>((per_sm * c->num_sms + tiles * nb - 1) / (tiles * nb),
                                             (a.n3 + ZSLAB - 1) / ZSLAB);
  const int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 3) / 4));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gx, gy, nbl * a.nzc), block(TX, TY);
    a.cpy = cpy ? cpy + (size_t)b0 * c->K : nullptr;
    if (cubic)
      kinetic_local_fx_kernel<true><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K, a);
    else
      kinetic_local_fx_kernel<false><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K,
                                                                    a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local fixed-point launch");
}

// Complex FP64 (Bloch) contexts on grids the tile fits, with 16-byte aligned band arrays;
// EINVAL otherwise.
int launch_kinetic_local_fx_c(pawfd_ctx* c, const zd* psi, int nb, zd* out, zd* cpy) {
  if (c->dtype != PAWFD_C128 || !c->d_vloc) return PAWFD_EINVAL;
  if (c->n[0] < TX + 2 * HALO + 2 || c->n[1] < TY + 2 * HALO || c->n[2] < HALO) return PAWFD_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out | (uintptr_t)cpy) & 15) return PAWFD_EINVAL;
  FXCArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  for (int cc = 0; cc < 3; ++cc) {
    a.ih2[cc] = 1.0 / (c->h[cc] * c->h[cc]);
    a.cs[cc] = -1.0 / (360.0 * c->h[cc] * c->h[cc]);
    const double kl = c->k[cc] * c->cell[cc];
    a.ph[cc] = zd{cos(kl), sin(kl)};
  }
  a.v = (const double*)c->d_vloc;
  const bool cubic = c->h[0] == c->h[1] && c->h[1] == c->h[2];
  const int gx = (a.n1 + TX - 1) / TX, gy = (a.n2 + TY - 1) / TY;
  const long long tiles = (long long)gx * gy;
  const long long per_sm = c->stencil_zsplit > 0 ? c->stencil_zsplit : 4;
  const long long want = std::max<long long>((per_sm * c->num_sms + tiles * nb - 1) / (tiles * nb),
                                             (a.n3 + ZSLAB - 1) / ZSLAB);
  const int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 3) / 4));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gx, gy, nbl * a.nzc), block(TX, TY);
    a.cpy = cpy ? cpy + (size_t)b0 * c->K : nullptr;
    if (cubic)
      kinetic_local_fx_c_kernel<true><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K, a);
    else
      kinetic_local_fx_c_kernel<false><<<grid, block, 0, c->stream>>>(psi + (size_t)b0 * c->K,
                                                                      out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local complex fixed-point launch");
}

}  // namespace pawfd
