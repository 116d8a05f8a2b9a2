// sliced_gram.cuh -- Gram matrices on the BF16 tensor cores with exact integer slices.
//
// Each real input value x (FP64 or FP32) of a row-chunk of KC grid values is written, relative
// to the chunk's largest binary exponent, as S balanced base-128 digits d_i in [-64, 64]:
//     x ~= 2^sigma * sum_i d_i 2^(-7 i),       sigma = E - bias - 5   (per row and chunk)
// The scaled digits d_i 2^(-7i) are exact in BF16, every digit product is exact in FP32, and
// the tcgen05 tensor core sums them in FP32.  Five TMEM accumulators per output element, one
// per digit order o = i + j (scaled digit products of order o are multiples of 2^(-7o) and at
// most 2^(12 - 7o) in magnitude, so a sum of n of them is exact while n 2^12 <= 2^24):
//     D0 = order 0 (1 product per grid value)   exact while KC <= 4096
//     D1 = order 1 (2 products)                 exact while KC <= 2048
//     D2 = order 2 (3 products)                 exact while KC <= 1365
//     D3 = order 3 (4 products)                 exact while KC <= 1024
//     D4 = orders 4 .. ORD, rounded in FP32 (each term is already 2^-28 below order 0)
// Five accumulators of BN = 96 columns use 480 of the 512 TMEM columns.  Chunks are KCG = 512
// values long for the Gram matrices (D0 .. D3 stay exact: with |d| <= 65 the order-2 sums
// reach 3 * 512 * 65^2 * 2^-14 < 2^10, inside the 2^(24-14) that keeps multiples of 2^-14
// exact, and the others have more room).  The rotation's contraction (the bands) is cut into
// chunks of KC = 256 when it is no longer than that (one chunk) and of KCG = 512 otherwise:
// every chunk costs the MMA warp a wait for the epilogue's TMEM drain, so fewer, longer
// chunks keep the tensor cores busier, and complex bands up to 256 stay one chunk (the
// persistent one-chunk form).  The FP32 drift of D4 stays small at either length.  After every chunk
// the epilogue adds 2^(sigma_a + sigma_b) (D0 + ... + D4) to a double-float (two FP32)
// accumulator with error-free transformations (Knuth's TwoSum), so the FP64 pipe is not
// needed per chunk; the scale is taken relative to the row's largest sigma of the K block.
// S = 7 digits and orders up to ORD = 6 keep 48 bits of each FP64 value (products accurate to
// ~2^-45 of the chunk maxima); S = 4 and ORD = 4 keep all 24 bits of an FP32 value.  Rounding
// to the digit grid may lift the top digit to 65; the exactness bounds above have room for it.  Digits are extracted from the IEEE bit fields with
// integer operations, so slicing needs no FP64 arithmetic.
#pragma once

#include <cuda_bf16.h>

#include "pawfd_internal.cuh"
#include "tc_common.cuh"

namespace pawfd {
namespace sg {

constexpr int KC = 256;           // contraction values per chunk of a rotation of at most 256 of them
constexpr int KCG = 512;          // grid values per exactness chunk of the Gram matrices
constexpr int BM = 128;           // output rows per CTA (TMEM lanes)
constexpr int BN = 96;            // output columns per CTA (MMA N)
constexpr int BK = 16;            // K per stage = one MMA (32-byte rows, 32B swizzle)
constexpr int NACC = 5;           // accumulators D0 .. D4 at columns 0, 96, 192, 288, 384
// Two epilogue warps per TMEM lane quarter (48 columns each) plus the TMA and MMA warps: ten
// warps, three on some SM sub-partitions, which caps registers at 168 per thread.
constexpr int EPI_WARPS = 8;
constexpr int EPI_COLS = BN / 2;
constexpr int NTHREADS = (EPI_WARPS + 2) * 32;
constexpr int TMEM_COLS = 512;

template <int S>
__host__ __device__ constexpr int a_slice_bytes() { return BM * BK * 2; }
__host__ __device__ constexpr int b_slice_bytes() { return BN * BK * 2; }
template <int S>
__host__ __device__ constexpr int stage_bytes() {
  static_assert(S >= 4 && S <= 7, "four to seven digits");
  return S * (BM + BN) * BK * 2;
}

// Hermitian tiling: tile rows of BM, tile columns of BN; a tile is needed when it holds an
// element with row <= column, i.e. column tile tc >= (BM tr) / BN.
__host__ __device__ inline int herm_first_col(int tr) { return (BM * tr) / BN; }
__host__ __device__ inline int herm_tiles(int n) {
  const int Tr = (n + BM - 1) / BM, Tc = (n + BN - 1) / BN;
  int t = 0;
  for (int r = 0; r < Tr; ++r) t += Tc > herm_first_col(r) ? Tc - herm_first_col(r) : 0;
  return t;
}
// pipeline depth: as many stages as fit in 200 KB of shared memory (4 for FP64, 7 for FP32)
template <int S>
__host__ __device__ constexpr int stages() { return (200 * 1024) / stage_bytes<S>() < 8 ? (200 * 1024) / stage_bytes<S>() : 8; }
template <int S>
__host__ __device__ constexpr int smem_bytes() { return stages<S>() * stage_bytes<S>() + 1024; }

// ------------------------------------------------------------------------------------------
// slicing
// ------------------------------------------------------------------------------------------
struct Fields {
  int exp;                 // biased exponent (0 for zero / subnormal, treated as zero)
  unsigned long long mant; // significand with the implicit bit
  bool neg;
};
__device__ __forceinline__ Fields fields(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  Fields f;
  f.exp = (int)((b >> 52) & 0x7FF);
  f.mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  f.neg = (b >> 63) != 0;
  return f;
}
__device__ __forceinline__ Fields fields(float x) {
  const unsigned b = __float_as_uint(x);
  Fields f;
  f.exp = (int)((b >> 23) & 0xFF);
  f.mant = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  f.neg = (b >> 31) != 0;
  return f;
}
template <class R> struct FloatBits;
template <> struct FloatBits<double> { static constexpr int bias = 1023, nb = 52; };
template <> struct FloatBits<float> { static constexpr int bias = 127, nb = 23; };

// x = src[r][k] of the real view, or for the "swapped" operand of a complex Gram the pair
// (re, im) -> (im, -re), so that sum_k a_k b''_k = Im(conj(a) . b).
template <class R>
__device__ __forceinline__ R slice_input(const R* __restrict__ src, long long ld, long long len, int r, long long k,
                                        bool swapped) {
  if (k >= len) return R(0);
  const R* row = src + (long long)r * ld;
  if (!swapped) return row[k];
  return (k & 1) ? -row[k - 1] : row[k + 1];
}

// Digit planes are stored in K steps: plane i, K step s (values 16 s .. 16 s + 15 of every
// row) is a slab of rows x 16 values.  Two layouts of a slab:
//  * row-major (plane_offset_rm): row r at 16 r, 32 contiguous bytes per row.  The Gram reads it
//    with 4-D TMA boxes (32-byte swizzle), which also zero-fill rows past the allocation.
//  * core matrices (plane_offset_cm): row group g = r / 8 holds the tensor cores' two K-major
//    core matrices (values 0-7 and 8-15 of the step) of 8 rows x 8 values (128 bytes each), so
//    the operand box of one plane (16 values of box_rows rows, box_rows a multiple of 8 from a
//    multiple of 8) is one contiguous block of box_rows * 32 bytes, copied with one bulk copy
//    and used as it lands (no swizzle).  The rotation's operands use this layout.
// rows is a multiple of 8 in both.
__device__ __forceinline__ long long plane_offset_rm(int i, long long k, int r, int rows, long long Lp) {
  return (((long long)i * (Lp / BK) + (k >> 4)) * rows + r) * BK + (k & 15);
}
__device__ __forceinline__ long long plane_offset_cm(int i, long long k, int r, int rows, long long Lp) {
  return ((long long)i * (Lp / BK) + (k >> 4)) * (long long)rows * BK + (long long)(r >> 3) * 128 +
         ((k >> 3) & 1) * 64 + (r & 7) * 8 + (k & 7);
}

// d 2^(-7 i) as a float for an integer |d| < 2^22, exactly, without a conversion instruction:
// the float 1.5 2^(23 - 7 i) has a unit in the last place of 2^(-7 i), so adding d to its bits
// and subtracting the float again leaves d 2^(-7 i).
__device__ __forceinline__ float digit_scaled(int d, int i) {
  const int m = ((150 - 7 * i) << 23) | 0x400000;
  return __int_as_float(m + d) - __int_as_float(m);
}
// Two floats that bf16 represents exactly (at most 8 significant bits) as a bf16x2 word, lo in
// the low half: the top 16 bits of each.
__device__ __forceinline__ uint32_t pack_bf16x2_exact(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

template <int S>
__device__ __forceinline__ void digits8_t(const double (&x)[8], int emax, uint32_t (&out)[S][4]);
template <int S>
__device__ __forceinline__ void digits8_t(const float (&x)[8], int emax, uint32_t (&out)[S][4]);

template <class R>
__device__ __forceinline__ void load8(const R* __restrict__ row, long long k0, long long len, bool swapped, R (&x)[8]) {
  if (k0 + 8 <= len && ((((uintptr_t)(row + k0)) & 15) == 0)) {
    if constexpr (sizeof(R) == 8) {
#pragma unroll
      for (int v = 0; v < 8; v += 2) {
        const double2 t = __ldg((const double2*)(row + k0 + v));
        x[v] = t.x;
        x[v + 1] = t.y;
      }
    } else {
      const float4 t0 = __ldg((const float4*)(row + k0)), t1 = __ldg((const float4*)(row + k0 + 4));
      x[0] = t0.x; x[1] = t0.y; x[2] = t0.z; x[3] = t0.w; x[4] = t1.x; x[5] = t1.y; x[6] = t1.z; x[7] = t1.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 8; ++v) x[v] = k0 + v < len ? row[k0 + v] : R(0);
  }
  if (swapped) {
    // (re, im) -> (im, -re): pairs start at even k, and k0 is a multiple of 8
#pragma unroll
    for (int v = 0; v < 8; v += 2) {
      const R re = x[v], im = x[v + 1];
      x[v] = im;
      x[v + 1] = -re;
    }
  }
}

// One warp per (row, chunk) of a K block: src points at the block's first value of row 0, rows
// are ld apart, len values per row are valid (the rest of the Lp-long block is zero).  out: S
// row-major digit planes of out_rows rows and Lp values (rows placed at row_offset); sig:
// [nchunks][sig_ld]; sigmax[row] (reset by the caller for every block) receives the largest
// sigma of the row.  Consecutive warps take consecutive rows of one chunk; each lane takes 8
// consecutive values of the 256-value chunk and writes 16 bytes per plane.
// (Memory-bound: the register cap keeps three CTAs per SM for FP64 values and six for FP32.)
template <class R, int S, int KCH>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 3 : 6)
    slice_kernel(const R* __restrict__ src, int rows, long long ld, long long len,
                                                    int nchunks, long long Lp, bool swapped, int row_offset,
                                                    int out_rows, __nv_bfloat16* __restrict__ out,
                                                    int* __restrict__ sig, int sig_ld, int* __restrict__ sigmax) {
  constexpr int NH = KCH / 256;   // runs of 256 values of the chunk: lane takes 8 values of each
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows * nchunks) return;
  const int r = warp % rows;
  const long long c = warp / rows;
  R x[NH][8];
#pragma unroll
  for (int h = 0; h < NH; ++h) load8(src + (long long)r * ld, c * KCH + h * 256 + lane * 8, len, swapped, x[h]);
  int emax = 0;
#pragma unroll
  for (int h = 0; h < NH; ++h)
#pragma unroll
    for (int v = 0; v < 8; ++v) emax = max(emax, fields(x[h][v]).exp);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  const int orow = row_offset + r;
  if (lane == 0) {
    sig[c * sig_ld + orow] = emax - FloatBits<R>::bias - 5;
    atomicMax(sigmax + orow, emax - FloatBits<R>::bias - 5);
  }
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    uint32_t o[S][4];
    digits8_t<S>(x[h], emax, o);
    const long long k0 = c * KCH + h * 256 + lane * 8;
#pragma unroll
    for (int i = 0; i < S; ++i)
      *(uint4*)(out + plane_offset_rm(i, k0, orow, out_rows, Lp)) = make_uint4(o[i][0], o[i][1], o[i][2], o[i][3]);
  }
}

// The same for core-matrix planes (the rotation's C operand): one warp per (group of 8 rows,
// chunk) of a K block; src, rows, ld, len, sig and sigmax as above; rows placed at row_offset,
// a multiple of 8.  Lane (r8, q) = (lane % 8, lane / 8)
// takes row r8 of the group and, in each of 8 passes j, the 8 values 32 j + 8 q of the chunk,
// so that one store instruction of the warp fills two whole K-step blocks of the row group's
// core matrices (2 x 256 contiguous bytes).  The chunk is read twice: once for its largest
// exponent, once (from L1/L2) for the digits.
template <class R, int S, int KCH>
__global__ void __launch_bounds__(256) slice_rg_kernel(const R* __restrict__ src, int rows, long long ld, long long len,
                                                       int nchunks, long long Lp, bool swapped, int row_offset,
                                                       int out_rows, __nv_bfloat16* __restrict__ out,
                                                       int* __restrict__ sig, int sig_ld, int* __restrict__ sigmax) {
  const int ngroups = (rows + 7) / 8;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)ngroups * nchunks) return;
  const int g = (int)(warp % ngroups);
  const long long c = warp / ngroups;
  const int r8 = lane & 7, q = lane >> 3;
  const int r = g * 8 + r8;
  const bool valid = r < rows;
  const R* row = src + (long long)(valid ? r : 0) * ld;
  int emax = 0;
#pragma unroll 2
  for (int j = 0; j < KCH / 32; ++j) {
    R x[8];
    if (valid) load8(row, c * KCH + 32 * j + 8 * q, len, swapped, x);
    else {
#pragma unroll
      for (int v = 0; v < 8; ++v) x[v] = R(0);
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) emax = max(emax, fields(x[v]).exp);
  }
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 8));
  emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 16));
  const int orow = row_offset + r;
  if (valid && q == 0) {
    sig[c * sig_ld + orow] = emax - FloatBits<R>::bias - 5;
    atomicMax(sigmax + orow, emax - FloatBits<R>::bias - 5);
  }
#pragma unroll 1
  for (int j = 0; j < KCH / 32; ++j) {
    const long long k0 = c * KCH + 32 * j + 8 * q;
    R x[8];
    uint32_t o[S][4];
    if (valid) {
      load8(row, k0, len, swapped, x);
      digits8_t<S>(x, emax, o);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) o[i][0] = o[i][1] = o[i][2] = o[i][3] = 0u;   // padding rows of the group
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
      *(uint4*)(out + plane_offset_cm(i, k0, orow, out_rows, Lp)) = make_uint4(o[i][0], o[i][1], o[i][2], o[i][3]);
  }
}

// Transposing slicer for the band rotation: operand rows are grid points r, the contraction
// index k runs over the bands (real: k = n; complex: k = 2 n + c, c = 0 real / 1 imaginary
// part).  One CTA per (16 grid points, chunk of KCH contraction values): the tile is read along
// r (coalesced), kept transposed in shared memory, the largest exponent of every grid point's
// chunk found, and each thread turns 8 consecutive k of one grid point into S 16-byte digit
// groups (a warp writes 512 contiguous bytes of a plane).  out: digit planes of out_rows rows (plane_offset);
// sig: [nchunks][sig_ld] (sig_ld >= rows).
constexpr int RT = 16;

// 8 values -> S planes of 8 bf16 digits (out[i][j]: plane i, values 2j, 2j+1), relative to the
// chunk's largest biased exponent emax (the digit scale of slice_kernel).
template <int S>
__device__ __forceinline__ void digits8_t(const double (&x)[8], int emax, uint32_t (&out)[S][4]) {
  constexpr int nbits = 52, g = 7 * S - 1 - nbits;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float dv[S][2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const Fields f = fields(x[2 * p + u]);
      unsigned long long G = 0;
      const int sh = emax - f.exp + 1;
      const int rs = sh - g;
      if (f.exp != 0 && rs < 64) G = rs > 0 ? (f.mant + (1ull << (rs - 1))) >> rs : f.mant << (-rs);
      int d[S];
#pragma unroll
      for (int i = 0; i < S; ++i) d[i] = (int)((G >> (7 * (S - 1 - i))) & 127ull);
#pragma unroll
      for (int i = S - 1; i >= 1; --i)
        if (d[i] >= 64) {
          d[i] -= 128;
          d[i - 1] += 1;
        }
#pragma unroll
      for (int i = 0; i < S; ++i) dv[i][u] = digit_scaled(f.neg ? -d[i] : d[i], i);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) out[i][p] = pack_bf16x2_exact(dv[i][0], dv[i][1]);
  }
}

// FP32 values: y = x 2^-sigma (|y| < 64), d_i = rint(y_i), y_{i+1} = 128 (y_i - d_i), all exact
// in FP32; the digits are balanced by construction.
template <int S>
__device__ __forceinline__ void digits8_t(const float (&x)[8], int emax, uint32_t (&out)[S][4]) {
  const int sigma = emax - 127 - 5;
  const float scale = (sigma > 126 || sigma < -126) ? 0.0f : __int_as_float((127 - sigma) << 23);
  float y[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) y[v] = x[v] * scale;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    float d[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      // round to the nearest integer (ties to even; |y| <= 64): adding and subtracting
      // 1.5 2^23 leaves the integer part
      d[v] = (y[v] + 12582912.0f) - 12582912.0f;
      y[v] = (y[v] - d[v]) * 128.0f;
    }
    const float w = __int_as_float((127 - 7 * i) << 23);
#pragma unroll
    for (int j = 0; j < 4; ++j) out[i][j] = pack_bf16x2_exact(d[2 * j] * w, d[2 * j + 1] * w);
  }
}

// Persistent, double-buffered form: each CTA walks tiles t = blockIdx.x, + gridDim.x, ...
// (chunk-major, so that CTAs running together read the same band rows) and copies the next
// tile into shared memory with cp.async while it slices the current one: 16 bytes per copy
// when the band rows and the block start allow it (vec16), else one value per copy; zero
// filled past the bands or the block's grid points.  The staged tile is dense and band-major:
// buf[n][q] (real) or buf[n][2 q + c] (complex), RT grid points q per band row.
template <class R, int KCH>
__host__ __device__ constexpr int slice_t_tile_values() { return KCH * RT; }
// two staged tiles of KCH contraction values x RT grid points
template <class R, int KCH>
__host__ __device__ constexpr int slice_t_smem() { return 2 * slice_t_tile_values<R, KCH>() * (int)sizeof(R); }

__device__ __forceinline__ void cp_async_zfill(void* sdst, const void* gsrc, int bytes, bool valid) {
  const int src_bytes = valid ? bytes : 0;
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(tc::smem_addr(sdst)), "l"(gsrc), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tc::smem_addr(sdst)), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
// 16 bytes, of which the first src_bytes (0 .. 16) are copied and the rest zero filled
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_addr(sdst)), "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <class R, int S, int KCH>
__global__ void __launch_bounds__(256) slice_t_kernel(const R* __restrict__ psi, int nb, long long K, int cplx,
                                                      long long r0, int rcount, long long Lp, int out_rows,
                                                      __nv_bfloat16* __restrict__ out, int* __restrict__ sig,
                                                      int sig_ld, int* __restrict__ sigmax, int nch, int vec16) {
  extern __shared__ __align__(16) unsigned char slice_t_smem_raw[];
  R* bufs = (R*)slice_t_smem_raw;                    // [2][KCH * RT] staged values
  __shared__ int pmax[16][RT];
  const int tid = threadIdx.x;
  const int nrt = (rcount + RT - 1) / RT;
  const int ntiles = nrt * nch;
  const int vals_per_row = cplx ? 2 * RT : RT;        // values of one band row of a tile
  const int rows_per_chunk = cplx ? KCH / 2 : KCH;    // band rows of one chunk
  constexpr int V16 = 16 / (int)sizeof(R);            // values per 16-byte copy
  // staged value (k, q) of a tile: real buf[k][q], complex buf[k / 2][2 q + k % 2]
  auto stage = [&](R* buf, int t) {
    const int rt = t % nrt, c = t / nrt;
    const int rl0 = rt * RT;
    const int nfirst = c * rows_per_chunk;
    if (vec16) {
      const int per_row = vals_per_row / V16;
      const int total = rows_per_chunk * per_row;
      for (int e = tid; e < total; e += 256) {
        const int nr = e / per_row, w = (e - nr * per_row) * V16;
        const int n = nfirst + nr;
        // values of this copy that lie inside the block's grid points
        const int left = cplx ? 2 * (rcount - rl0) - w : rcount - rl0 - w;
        const int nval = n < nb ? max(0, min(V16, left)) : 0;
        const long long gi = cplx ? (((long long)n * K + r0 + rl0) * 2 + w) : ((long long)n * K + r0 + rl0 + w);
        cp_async16(buf + nr * vals_per_row + w, nval > 0 ? psi + gi : psi, nval * (int)sizeof(R));
      }
      return;
    }
    const int total = rows_per_chunk * vals_per_row;
    for (int e = tid; e < total; e += 256) {
      const int nr = e / vals_per_row, w = e - nr * vals_per_row;
      const int n = nfirst + nr;
      const int q = cplx ? w >> 1 : w;
      const bool ok = n < nb && rl0 + q < rcount;
      const long long gi = cplx ? (((long long)n * K + r0 + rl0) * 2 + w) : ((long long)n * K + r0 + rl0 + w);
      cp_async_zfill(buf + nr * vals_per_row + w, ok ? psi + gi : psi, (int)sizeof(R), ok);
    }
  };
  auto val = [&](const R* buf, int k, int q) -> R {
    return cplx ? buf[(k >> 1) * (2 * RT) + 2 * q + (k & 1)] : buf[k * RT + q];
  };
  int it = 0;
  int t = blockIdx.x;
  if (t < ntiles) stage(bufs, t);
  cp_async_commit();
  for (; t < ntiles; t += gridDim.x, ++it) {
    R* cur = bufs + (it & 1) * slice_t_tile_values<R, KCH>();
    R* nxt = bufs + ((it + 1) & 1) * slice_t_tile_values<R, KCH>();
    if (t + (int)gridDim.x < ntiles) stage(nxt, t + gridDim.x);
    cp_async_commit();
    cp_async_wait1();   // this tile's copies have landed
    __syncthreads();
    const int rt = t % nrt, c = t / nrt;
    const int rl0 = rt * RT;
    // largest exponent of every grid point's chunk (zero fill beyond the bands contributes 0)
    {
      const int lr = tid % RT, kq = tid / RT;
      int em = 0;
      for (int kk = kq; kk < KCH; kk += 16) em = max(em, fields(val(cur, kk, lr)).exp);
      pmax[kq][lr] = em;
    }
    __syncthreads();
    if (tid < RT) {
      int m = 0;
      for (int q = 0; q < 16; ++q) m = max(m, pmax[q][tid]);
      pmax[0][tid] = m;
      if (rl0 + tid < rcount) {
        sig[(long long)c * sig_ld + rl0 + tid] = m - FloatBits<R>::bias - 5;
        atomicMax(sigmax + rl0 + tid, m - FloatBits<R>::bias - 5);
      }
    }
    __syncthreads();
    // items: (K step j, half h, grid point q); the 32 threads of a warp cover the 16 grid points
    // and both halves of one K step, i.e. 512 contiguous bytes of a digit plane
    for (int item = tid; item < RT * (KCH / 8); item += 256) {
      const int q = item % RT, k8 = (item / (2 * RT)) * 16 + ((item / RT) & 1) * 8;
      if (rl0 + q >= rcount) continue;
      R x[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) x[v] = val(cur, k8 + v, q);
      uint32_t o[S][4];
      digits8_t<S>(x, pmax[0][q], o);
#pragma unroll
      for (int i = 0; i < S; ++i)
        *(uint4*)(out + plane_offset_cm(i, (long long)c * KCH + k8, rl0 + q, out_rows, Lp)) =
            make_uint4(o[i][0], o[i][1], o[i][2], o[i][3]);
    }
    __syncthreads();   // the buffer and pmax are reused
  }
}

// ------------------------------------------------------------------------------------------
// Gram kernel
// ------------------------------------------------------------------------------------------
constexpr int COVER_TILES = 4;   // tiles of the symmetric cover (at most 256 rows)
constexpr int CB = 32;           // rows per block of the symmetric cover

struct GramArgs {
  const int* sigA = nullptr;      // [nchunks][sig_ldA]  (chunks of this K block)
  const int* sigB = nullptr;      // [nchunks][sig_ldB]
  const int* maxA = nullptr;      // [rows] largest sigma of each row in this K block
  const int* maxB = nullptr;
  int sig_ldA = 0, sig_ldB = 0;
  int rowsA = 0, rowsB = 0;     // valid rows of the two operands
  int tilesN = 0;           // column tiles (ceil(rowsB / BN))
  int herm = 0;             // only tiles with tile row <= tile column (within each half of B if halves > 1)
  int halves = 0;           // 2 for complex (B = [B'; B'']): tiles are enumerated per half
  int half_rows = 0;        // rows per half of B (complex: nb)
  int chunks_per_cta = 0;
  int nchunks = 0;          // chunks in this K block
  long long klen = 0;       // valid contraction values in this K block (0: all full chunks)
  int accumulate = 0;       // add to part instead of overwriting it (second and later K blocks)
  double* part = nullptr;         // [nsplit][rowsA][rowsB]
  DeviceStatus* st = nullptr;
  // band rotation: write every output value straight to the band array instead of partials.
  // Row `row` of the product is band row % rot_nb, real part for row < rot_nb and imaginary
  // part otherwise (complex); column `col` is grid point col of the block starting at rot_out.
  int rotation = 0;
  int rot_nb = 0;
  int rot_cplx = 0;
  int rot_fp32 = 0;
  long long rot_K = 0;  // grid points per band
  void* rot_out = nullptr;        // band array, already offset to the first grid point of the block
  int rot_vec = 0;                // real bands with 16-byte aligned rows: vector stores
  int rot_tiles = 0;              // output tiles of the rotation, shared out over the persistent CTAs
  // digit planes of the two operands (plane_offset layout, slabs of rows_alloc x 16 values)
  const __nv_bfloat16* gA = nullptr;
  const __nv_bfloat16* gB = nullptr;
  int rows_allocA = 0, rows_allocB = 0;
  long long ksteps = 0;           // K steps per plane (Lp / 16) of both buffers
  int half_stride = 0;            // B row of the second half's first row (complex; 0: half_rows)
  // Symmetric cover of a Hermitian Gram of at most 256 rows: tile t has A rows cov_row0[t] ..
  // + 127 and B rows from three 32-row blocks cov_seg[t][0..2] (one 32-row box of all planes
  // each; N = 32 MMAs per block); complex operands run the four tiles once per half of B
  // (CTA x = half x COVER_TILES + t).  A tile below the diagonal computes needed entries
  // mirrored (the imaginary half negated: Im G_mn = -Im G_nm).  Each pair of 32-row blocks (lo, hi), bit 8 lo + hi, belongs to one tile
  // (cov_own[t]); cov_tr[t] marks the pairs that tile writes from its mirrored orientation
  // (row block hi).  Entries of a diagonal block are written for row <= column.
  int cover = 0;
  int cov_row0[COVER_TILES] = {};
  int cov_seg[COVER_TILES][3] = {};
  unsigned long long cov_own[COVER_TILES] = {};
  unsigned long long cov_tr[COVER_TILES] = {};
};

// 2^e for the product scale; below the normal range the chunk contributes nothing (its
// digits are all zero) and 0 is returned
__device__ __forceinline__ double pow2(int e) {
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

// x 2^e as a double, assembled from the bit fields of the float x with integer operations (no
// FP64 conversion or multiply: the FP64 pipe is narrow); results below the normal FP64
// range, and float subnormals, give 0.
__device__ __forceinline__ double f2d_scaled(float x, int e) {
  const unsigned u = __float_as_uint(x);
  const int ef = (int)((u >> 23) & 0xFFu);
  const int ed = ef - 127 + 1023 + e;
  if (ef == 0 || ed <= 0) return 0.0;
  const unsigned hi = (u & 0x80000000u) | ((unsigned)ed << 20) | ((u >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(u << 29));
}
// the double-float (xh, xl) times 2^e: both parts exact, one FP64 add (the general path)
__device__ __noinline__ double df_to_double_slow(float xh, float xl, int e) {
  return f2d_scaled(xh, e) + f2d_scaled(xl, e);
}
// The same with integer operations only.  For a normalized pair (|xl| <= ulp(xh) / 2) the
// 53-bit significand of the result is xh's 24 bits followed by 29 zero bits, plus or minus xl's
// significand aligned to that last bit (xl's bits below it are dropped), renormalized by at
// most one bit: within one unit in the last place of the FP64 result.  Zero and subnormal
// parts, pairs that are not normalized and results outside the normal FP64 range take the
// FP64 path.
__device__ __forceinline__ double df_to_double(float xh, float xl, int e) {
  const unsigned uh = __float_as_uint(xh), ul = __float_as_uint(xl);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  const int d = eh - el;
  int ed = eh - 127 + 1023 + e;
  if (eh == 0 || (el != 0 && d < 21) || ed <= 1 || ed >= 2046) return df_to_double_slow(xh, xl, e);
  const unsigned mh = (uh & 0x7FFFFFu) | 0x800000u;
  unsigned hi = mh >> 3, lo = mh << 29;   // mh 2^29 as the high and low words of the significand
  unsigned L = 0;
  if (el != 0 && d < 53) {
    const unsigned ml = (ul & 0x7FFFFFu) | 0x800000u;
    L = d <= 29 ? ml << (29 - d) : ml >> (d - 29);
  }
  if ((uh ^ ul) & 0x80000000u) {
    const unsigned nlo = lo - L;
    hi -= nlo > lo ? 1u : 0u;
    lo = nlo;
  } else {
    const unsigned nlo = lo + L;
    hi += nlo < lo ? 1u : 0u;
    lo = nlo;
  }
  if (hi >= (1u << 21)) {
    lo = (lo >> 1) | (hi << 31);
    hi >>= 1;
    ++ed;
  } else if (hi < (1u << 20)) {
    hi = (hi << 1) | (lo >> 31);
    lo <<= 1;
    --ed;
  }
  return __hiloint2double((int)((uh & 0x80000000u) | ((unsigned)ed << 20) | (hi & 0xFFFFFu)), (int)lo);
}
// x 2^e in FP32 (x is the correctly rounded sum of the double-float pair).  The rare path is
// out of line so that it is not evaluated under a predicate for every value (FP64 pipe).
__device__ __noinline__ float f2f_scaled_slow(float x, int e) { return (float)((double)x * pow2(e)); }
__device__ __forceinline__ float f2f_scaled(float x, int e) {
  if (e >= -126 && e <= 127) return x * __int_as_float((e + 127) << 23);
  return f2f_scaled_slow(x, e);
}

// tile index -> (tile row, tile col) over the output [rowsA][rowsB]; tile columns are numbered
// per half of B (Tc = ceil(half_rows / BN) each)
__device__ __forceinline__ void gram_tile(const GramArgs& a, int t, int* tr, int* tc_) {
  if (!a.herm) {
    // tile rows fastest: the CTAs that share a B tile run together and read it once from DRAM
    const int Tr = (a.rowsA + BM - 1) / BM;
    *tr = t % Tr;
    *tc_ = t / Tr;
    return;
  }
  const int Tc = (a.half_rows + BN - 1) / BN;
  const int per_half = herm_tiles(a.half_rows);
  const int h = t / per_half;
  int u = t % per_half, row = 0;
  while (true) {
    const int first = herm_first_col(row), cnt = Tc > first ? Tc - first : 0;
    if (u < cnt) {
      *tr = row;
      *tc_ = h * Tc + first + u;
      return;
    }
    u -= cnt;
    ++row;
  }
}

// float 2^e for e <= 0 (0 below the normal range)
__device__ __forceinline__ float pow2f_nonpos(int e) { return e < -126 ? 0.0f : __int_as_float((e + 127) << 23); }

// error-free a + b = s + e (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += (xh, xl), double-float accumulation
__device__ __forceinline__ void df_add(float& hi, float& lo, float xh, float xl) {
  float s, e;
  two_sum(hi, xh, s, e);
  e += lo + xl;
  two_sum(s, e, hi, lo);
}

// BULK: the operands are core-matrix planes (plane_offset_cm), one bulk copy per plane and
// operand per stage, read by the tensor cores without swizzle; otherwise row-major planes
// (plane_offset_rm) through the 4-D TMA maps tA and tB with a 32-byte swizzle.
// tB32: the B planes with a box of CB rows (the symmetric cover's B blocks).  COVER: the Gram
// on the symmetric cover (a separate instance, so that the other instances carry none of its
// registers).
template <int S, int ORD, bool ONE, bool BULK, int KCH, bool COVER = false>
__global__ void __launch_bounds__(NTHREADS, 1) sliced_gram_kernel(const __grid_constant__ CUtensorMap tA,
                                                                  const __grid_constant__ CUtensorMap tB,
                                                                  const __grid_constant__ CUtensorMap tB32,
                                                                  const __grid_constant__ GramArgs a) {
  constexpr int STAGES = stages<S>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[STAGES], empty[STAGES], dfull, dempty;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // column tiles of the complex second half start at half_stride (a multiple of 8)
  const int T = (a.half_rows + BN - 1) / BN;
  const int HS = a.half_stride ? a.half_stride : a.half_rows;
  // Output tiles of this CTA: tile blockIdx.x; with ONE (a rotation whose contraction is one
  // chunk) every gridDim.x-th tile from blockIdx.x (a persistent CTA: the copies for the next
  // tile run while the epilogue of the last one drains TMEM and stores).
  const int ntiles = !ONE ? 1 : ((int)blockIdx.x < a.rot_tiles ? (a.rot_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0);
  auto tile_at = [&](int i, int& row0, int& col0, int& tcol) {
    if (COVER) {
      row0 = a.cov_row0[blockIdx.x % COVER_TILES];
      col0 = 0;
      tcol = 0;
      return;
    }
    int tr;
    gram_tile(a, (int)blockIdx.x + i * (int)gridDim.x, &tr, &tcol);
    row0 = tr * BM;
    col0 = (tcol / T) * HS + (tcol % T) * BN;
  };
  const int c_begin = blockIdx.y * a.chunks_per_cta;
  const int c_end = min(a.nchunks, c_begin + a.chunks_per_cta);
  const int nch = max(0, c_end - c_begin);
  const int steps_per_chunk = KCH / BK;
  // stages of chunk c (the last chunk of a block may hold fewer than KC valid values: no MMAs
  // on its zero padding)
  auto steps_of = [&](int c) {
    if (a.klen <= 0) return steps_per_chunk;
    const long long left = a.klen - (long long)(c_begin + c) * KCH;
    return (int)max(1ll, min((long long)steps_per_chunk, (left + BK - 1) / BK));
  };
  int steps_tile = 0;
  for (int c = 0; c < nch; ++c) steps_tile += steps_of(c);
  const int total_steps = steps_tile * ntiles;
  const int items = nch * ntiles;   // (tile, chunk) pairs, chunk fastest: one TMEM round each

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&dfull, 1);
    tc::mbar_init(&dempty, EPI_WARPS);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    tc::mbar_fence_init();
  }
  if (warp == EPI_WARPS) tc::tmem_alloc(&tmem_base, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == EPI_WARPS) {
    if (lane == 0 && items > 0) {   // TMA producer: S slices of A and S slices of B per stage
      int c = 0, q = 0, i = 0, row0, col0, tcol;
      tile_at(0, row0, col0, tcol);
      for (int g = 0; g < total_steps && !abort_flag; ++g) {
        const int s = g % STAGES;
        if (g >= STAGES && !tc::mbar_wait(&empty[s], ((g / STAGES) - 1) & 1)) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1001);
          break;
        }
        const int kx = (c_begin + c) * KCH + q * BK;
        unsigned char* sa = smem + s * stage_bytes<S>();
        unsigned char* sb = sa + S * a_slice_bytes<S>();
        tc::mbar_expect_tx(&full[s], stage_bytes<S>());
        const long long ks = kx / BK;
        if constexpr (BULK) {
          // one contiguous box per plane and operand (rows row0 .. row0 + BM - 1 of the slab)
#pragma unroll
          for (int pl = 0; pl < S; ++pl) {
            tc::bulk_load(sa + pl * a_slice_bytes<S>(),
                          a.gA + (pl * a.ksteps + ks) * a.rows_allocA * BK + (long long)row0 * BK, a_slice_bytes<S>(),
                          &full[s]);
            tc::bulk_load(sb + pl * b_slice_bytes(),
                          a.gB + (pl * a.ksteps + ks) * a.rows_allocB * BK + (long long)col0 * BK, b_slice_bytes(),
                          &full[s]);
          }
        } else {
          tc::tma_load_4d(sa, &tA, &full[s], 0, row0, (int)ks, 0);
          if constexpr (COVER) {
            // B rows from three blocks, each with its S planes in one box: block g's plane j
            // at (g S + j) KB of the stage's B area (the MMAs then take N = 32 per block)
            const int ct = blockIdx.x % COVER_TILES, boff = (blockIdx.x / COVER_TILES) * HS;
#pragma unroll
            for (int g3 = 0; g3 < 3; ++g3)
              tc::tma_load_4d(sb + g3 * (S * CB * BK * 2), &tB32, &full[s], 0, boff + a.cov_seg[ct][g3], (int)ks, 0);
          } else {
            tc::tma_load_4d(sb, &tB, &full[s], 0, col0, (int)ks, 0);
          }
        }
        issued = g + 1;
        if (++q == steps_of(c)) {
          q = 0;
          if (++c == nch) {
            c = 0;
            if (++i < ntiles) tile_at(i, row0, col0, tcol);
          }
        }
      }
    }
  } else if (warp == EPI_WARPS + 1) {
    // MMA issuer: the whole warp runs the loop (the waits, the stage's descriptors), so the
    // descriptors are warp-uniform values; one elected lane issues the MMAs and the commits.
    constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
    const bool leader = tc::elect_one();
    int g = 0;
    for (int it = 0; it < items; ++it) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      if (it > 0) {
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&dempty, (it - 1) & 1));
        if (!ok) {
          if (leader) {
            abort_flag = 1;
            set_status(a.st, PAWFD_ETIMEDOUT, 1002);
          }
          break;
        }
      }
      tc::fence_after_sync();
      const int steps = steps_of(it % nch);
      bool failed = false;
      for (int q = 0; q < steps; ++q, ++g) {
        const int s = g % STAGES;
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[s], (g / STAGES) & 1))) {
          if (leader) {
            abort_flag = 1;
            set_status(a.st, PAWFD_ETIMEDOUT, 1003);
          }
          failed = true;
          break;
        }
        tc::fence_after_sync();
        unsigned char* sa = smem + s * stage_bytes<S>();
        unsigned char* sb = sa + S * a_slice_bytes<S>();
        // plane i of a stage starts i slices after the stage's first plane; the start address
        // field (address / 16, 14 bits) does not overflow inside the 228 KB of shared memory
        const uint64_t da0 = BULK ? tc::smem_desc_nosw(sa, 128, 256) : tc::smem_desc(sa, BK * 2);
        const uint64_t db0 = BULK ? tc::smem_desc_nosw(sb, 128, 256) : tc::smem_desc(sb, BK * 2);
        if (COVER && leader) {
          // the symmetric cover: each product as three N = 32 MMAs, one per B block, into the
          // block's 32 columns of the accumulator; A plane i stays in the collector buffer over
          // all of them
          constexpr uint32_t idesc32 = tc::idesc_bf16_f32(BM, CB);
          bool touched[NACC] = {false, false, false, false, false};
#pragma unroll
          for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (i + j > ORD) continue;
              const int slot = (i + j) < NACC - 1 ? (i + j) : NACC - 1;
              const uint32_t acc = touched[slot] ? 1u : (q == 0 ? 0u : 1u);
              touched[slot] = true;
              const uint64_t da = da0 + (uint64_t)((i * a_slice_bytes<S>()) >> 4);
              const int jlast = (ORD - i) < (S - 1) ? (ORD - i) : (S - 1);
#pragma unroll
              for (int g3 = 0; g3 < 3; ++g3) {
                const uint32_t d = tmem + (uint32_t)(slot * BN + g3 * CB);
                const uint64_t db = db0 + (uint64_t)(((g3 * S + j) * (CB * BK * 2)) >> 4);
                if (j == 0 && g3 == 0)
                  tc::mma_bf16_ca<1>(d, da, db, idesc32, acc);
                else if (j == jlast && g3 == 2)
                  tc::mma_bf16_ca<3>(d, da, db, idesc32, acc);
                else
                  tc::mma_bf16_ca<2>(d, da, db, idesc32, acc);
              }
            }
          tc::mma_commit(&empty[s]);
          consumed = g + 1;
        } else if (leader) {
          bool touched[NACC] = {false, false, false, false, false};
#pragma unroll
          for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (i + j > ORD) continue;
              const int slot = (i + j) < NACC - 1 ? (i + j) : NACC - 1;
              const uint32_t d = tmem + (uint32_t)(slot * BN);
              // the first product written into an accumulator in this chunk overwrites it
              const uint32_t acc = touched[slot] ? 1u : (q == 0 ? 0u : 1u);
              touched[slot] = true;
              // A plane i serves the products (i, 0) .. (i, ORD - i) back to back: read it from
              // shared memory once and keep it in the collector buffer for the others
              const uint64_t da = da0 + (uint64_t)((i * a_slice_bytes<S>()) >> 4);
              const uint64_t db = db0 + (uint64_t)((j * b_slice_bytes()) >> 4);
              const int jlast = (ORD - i) < (S - 1) ? (ORD - i) : (S - 1);
              if (jlast == 0)
                tc::mma_bf16_ca<0>(d, da, db, idesc, acc);
              else if (j == 0)
                tc::mma_bf16_ca<1>(d, da, db, idesc, acc);
              else if (j < jlast)
                tc::mma_bf16_ca<2>(d, da, db, idesc, acc);
              else
                tc::mma_bf16_ca<3>(d, da, db, idesc, acc);
            }
          tc::mma_commit(&empty[s]);
          consumed = g + 1;
        }
        __syncwarp();
      }
      if (failed) break;
      if (leader) tc::mma_commit(&dfull);
      __syncwarp();
    }
  } else {
    if constexpr (ONE) {
    // One chunk per tile (the rotation of at most KCH contraction values): the value is (D0 + ... +
    // D4) 2^(sigma_a + sigma_b), summed exactly as a double-float and converted to the band
    // dtype.  TMEM is read in the 16 x 256-bit shape: in each 16-lane half h of the warp's
    // lane quarter, thread t holds rows t/4 and t/4 + 8 and columns 2 (t%4), 2 (t%4) + 1 of
    // each 8-column group, so four threads store four consecutive outputs of one row and a
    // store instruction writes 8 rows x 4 values (not 32 rows x 1 value).  The chunk
    // exponents of the tile's rows and columns are loaded while the tile's MMAs run (the
    // columns' in two registers per lane, handed to the column's threads by shuffles).
    static_assert(EPI_COLS % 8 == 0 && EPI_COLS <= 64, "8-column groups, two exponent registers per lane");
    constexpr int NG = EPI_COLS / 8;
    const int quarter = warp & 3, chalf = warp >> 2;
    const int cbase = chalf * EPI_COLS;
    const int trow = lane >> 2, tcol2 = (lane & 3) * 2;
    for (int i = 0; i < ntiles; ++i) {
      int row0, col0, tcol;
      tile_at(i, row0, col0, tcol);
      // this thread's rows: r = 2 h + p  ->  row0 + 32 quarter + 16 h + 8 p + trow
      int sga[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = row0 + quarter * 32 + (r >> 1) * 16 + (r & 1) * 8 + trow;
        sga[r] = row < a.rowsA ? __ldg(a.sigA + (long long)c_begin * a.sig_ldA + row) : 0;
      }
      const int cl0 = col0 + cbase + lane, cl1 = cl0 + 32;
      const int sgb0 = cl0 < a.rowsB ? __ldg(a.sigB + (long long)c_begin * a.sig_ldB + cl0) : 0;
      const int sgb1 = (lane + 32 < EPI_COLS && cl1 < a.rowsB) ? __ldg(a.sigB + (long long)c_begin * a.sig_ldB + cl1) : 0;
      bool ok = tc::mbar_wait(&dfull, i & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1004);
        }
        break;
      }
      tc::fence_after_sync();
      // TMEM -> the exact double-float sums (vh, vl) of the five orders
      float vh[2][NG][4], vl[2][NG][4];   // [h][group][2 p + c]
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          uint32_t d[NACC][4];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32 + h * 16) << 16) + (uint32_t)(cbase + g * 8);
#pragma unroll
          for (int o = 0; o < NACC; ++o) tc::tmem_ld_16x256b(taddr + o * BN, d[o]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float s1, e1, s2, e2, s3, e3;
            two_sum(__uint_as_float(d[0][e]), __uint_as_float(d[1][e]), s1, e1);
            two_sum(s1, __uint_as_float(d[2][e]), s2, e2);
            two_sum(s2, __uint_as_float(d[3][e]), s3, e3);
            two_sum(s3, ((e1 + e2) + e3) + __uint_as_float(d[4][e]), vh[h][g][e], vl[h][g][e]);
          }
        }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&dempty);
      // column exponents of this thread's columns 8 g + tcol2 + c (all lanes shuffle)
      int sgb[NG][2];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int cj = g * 8 + tcol2 + c;
          sgb[g][c] = __shfl_sync(0xffffffffu, g * 8 < 32 ? sgb0 : sgb1, cj & 31);
        }
      if (abort_flag) continue;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int h = r >> 1, p = r & 1;
        const int row = row0 + quarter * 32 + h * 16 + p * 8 + trow;
        if (row >= a.rowsA) continue;
        const int band = row % a.rot_nb, part = row / a.rot_nb;
        const long long base = (long long)band * a.rot_K;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const int col = col0 + cbase + g * 8 + tcol2;
          const bool vec = a.rot_vec && col + 1 < a.rowsB;
          if (a.rot_fp32) {
            const float v0 = f2f_scaled(vh[h][g][2 * p], sga[r] + sgb[g][0]);
            const float v1 = f2f_scaled(vh[h][g][2 * p + 1], sga[r] + sgb[g][1]);
            if (vec) {
              *(float2*)((float*)a.rot_out + base + col) = make_float2(v0, v1);
            } else {
              if (col < a.rowsB) ((float*)a.rot_out)[a.rot_cplx ? 2 * (base + col) + part : base + col] = v0;
              if (col + 1 < a.rowsB)
                ((float*)a.rot_out)[a.rot_cplx ? 2 * (base + col + 1) + part : base + col + 1] = v1;
            }
          } else {
            const double v0 = df_to_double(vh[h][g][2 * p], vl[h][g][2 * p], sga[r] + sgb[g][0]);
            const double v1 = df_to_double(vh[h][g][2 * p + 1], vl[h][g][2 * p + 1], sga[r] + sgb[g][1]);
            if (vec) {
              *(double2*)((double*)a.rot_out + base + col) = make_double2(v0, v1);
            } else {
              if (col < a.rowsB) ((double*)a.rot_out)[a.rot_cplx ? 2 * (base + col) + part : base + col] = v0;
              if (col + 1 < a.rowsB)
                ((double*)a.rot_out)[a.rot_cplx ? 2 * (base + col + 1) + part : base + col + 1] = v1;
            }
          }
        }
      }
    }
    } else if constexpr (BULK && S == 4) {
    // The rotation of FP32 bands with several chunks per tile (more than 512 contraction
    // values: complex bands beyond 256, real bands beyond 512): one tile per CTA, the chunks' five orders summed into double-float accumulators,
    // then one write-out with FP32 values rounded once from the double-float sums.  TMEM is
    // read in the 16 x 256-bit shape (as in the one-chunk form): thread t holds rows t/4 and
    // t/4 + 8 of each 16-lane half and columns 2 (t%4), 2 (t%4) + 1 of each 8-column group, so
    // that four threads store four consecutive values of one row.  (For FP64 bands the
    // general epilogue below measured faster: its wider TMEM loads drain each chunk in half
    // the load instructions, and the FP64 stores gain nothing from this layout.)
    constexpr int NG = EPI_COLS / 8;
    const int quarter = warp & 3, chalf = warp >> 2;
    int row0, col0, tcol;
    tile_at(0, row0, col0, tcol);
    const int cbase = chalf * EPI_COLS;
    const int trow = lane >> 2, tcol2 = (lane & 3) * 2;
    float ahi[2][NG][4], alo[2][NG][4];   // [h][group][2 p + c]
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ahi[h][g][e] = 0.0f;
          alo[h][g][e] = 0.0f;
        }
    // this thread's rows: r = 2 h + p  ->  row0 + 32 quarter + 16 h + 8 p + trow
    int rws[4], ra[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      rws[r] = row0 + quarter * 32 + (r >> 1) * 16 + (r & 1) * 8 + trow;
      ra[r] = rws[r] < a.rowsA ? __ldg(a.maxA + rws[r]) : 0;
    }
    // column exponents: two registers per lane (columns cbase + lane, cbase + 32 + lane), handed
    // to the column's threads by shuffles
    const int cl0 = col0 + cbase + lane, cl1 = cl0 + 32;
    const bool cv0 = cl0 < a.rowsB, cv1 = lane + 32 < EPI_COLS && cl1 < a.rowsB;
    const int mb0 = cv0 ? __ldg(a.maxB + cl0) : 0, mb1 = cv1 ? __ldg(a.maxB + cl1) : 0;
    for (int c = 0; c < nch; ++c) {
      const int chunk = c_begin + c;
      int sa[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        sa[r] = rws[r] < a.rowsA ? __ldg(a.sigA + (long long)chunk * a.sig_ldA + rws[r]) - ra[r] : 0;
      const int sb0 = cv0 ? __ldg(a.sigB + (long long)chunk * a.sig_ldB + cl0) - mb0 : 0;
      const int sb1 = cv1 ? __ldg(a.sigB + (long long)chunk * a.sig_ldB + cl1) - mb1 : 0;
      bool ok = tc::mbar_wait(&dfull, c & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1004);
        }
        break;
      }
      tc::fence_after_sync();
      int sbv[NG][2];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2)
          sbv[g][c2] = __shfl_sync(0xffffffffu, g * 8 < 32 ? sb0 : sb1, (g * 8 + tcol2 + c2) & 31);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          uint32_t d[NACC][4];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32 + h * 16) << 16) + (uint32_t)(cbase + g * 8);
#pragma unroll
          for (int o = 0; o < NACC; ++o) tc::tmem_ld_16x256b(taddr + o * BN, d[o]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float scale = pow2f_nonpos(sa[2 * h + (e >> 1)] + sbv[g][e & 1]);
            float s1, e1, s2, e2, s3, e3, vh, vl;
            two_sum(__uint_as_float(d[0][e]), __uint_as_float(d[1][e]), s1, e1);
            two_sum(s1, __uint_as_float(d[2][e]), s2, e2);
            two_sum(s2, __uint_as_float(d[3][e]), s3, e3);
            two_sum(s3, ((e1 + e2) + e3) + __uint_as_float(d[4][e]), vh, vl);
            df_add(ahi[h][g][e], alo[h][g][e], vh * scale, vl * scale);
          }
        }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&dempty);
    }
    // the columns' largest exponents, then the write-out (FP32 values rounded once from the
    // double-float sum, FP64 values assembled with integer operations)
    int mbv[NG][2];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
        mbv[g][c2] = __shfl_sync(0xffffffffu, g * 8 < 32 ? mb0 : mb1, (g * 8 + tcol2 + c2) & 31);
    if (!abort_flag) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int h = r >> 1, p = r & 1;
        if (rws[r] >= a.rowsA) continue;
        const int band = rws[r] % a.rot_nb, part = rws[r] / a.rot_nb;
        const long long base = (long long)band * a.rot_K;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          const int col = col0 + cbase + g * 8 + tcol2;
          const bool vec = a.rot_vec && col + 1 < a.rowsB;
          if (a.rot_fp32) {
            const float v0 = f2f_scaled(ahi[h][g][2 * p] + alo[h][g][2 * p], ra[r] + mbv[g][0]);
            const float v1 = f2f_scaled(ahi[h][g][2 * p + 1] + alo[h][g][2 * p + 1], ra[r] + mbv[g][1]);
            if (vec) {
              *(float2*)((float*)a.rot_out + base + col) = make_float2(v0, v1);
            } else {
              if (col < a.rowsB) ((float*)a.rot_out)[a.rot_cplx ? 2 * (base + col) + part : base + col] = v0;
              if (col + 1 < a.rowsB)
                ((float*)a.rot_out)[a.rot_cplx ? 2 * (base + col + 1) + part : base + col + 1] = v1;
            }
          } else {
            const double v0 = df_to_double(ahi[h][g][2 * p], alo[h][g][2 * p], ra[r] + mbv[g][0]);
            const double v1 = df_to_double(ahi[h][g][2 * p + 1], alo[h][g][2 * p + 1], ra[r] + mbv[g][1]);
            if (vec) {
              *(double2*)((double*)a.rot_out + base + col) = make_double2(v0, v1);
            } else {
              if (col < a.rowsB) ((double*)a.rot_out)[a.rot_cplx ? 2 * (base + col) + part : base + col] = v0;
              if (col + 1 < a.rowsB)
                ((double*)a.rot_out)[a.rot_cplx ? 2 * (base + col + 1) + part : base + col + 1] = v1;
            }
          }
        }
      }
    }
    } else {
    // epilogue warps: lane quarter (warp % 4), column half (warp / 4)
    const int quarter = warp & 3, chalf = warp >> 2;
    int row0, col0, tcol;
    tile_at(0, row0, col0, tcol);
    const int row = row0 + quarter * 32 + lane;
    const int cbase = chalf * EPI_COLS;
    float ahi[EPI_COLS], alo[EPI_COLS];
#pragma unroll
    for (int j = 0; j < EPI_COLS; ++j) {
      ahi[j] = 0.0f;
      alo[j] = 0.0f;
    }
    const int ra = (row < a.rowsA) ? __ldg(a.maxA + row) : 0;
    // B row of tile column tc (the symmetric cover gathers three 32-row blocks of its half)
    auto bcol = [&](int tcn) -> int {
      if (COVER)
        return (int)(blockIdx.x / COVER_TILES) * HS + a.cov_seg[blockIdx.x % COVER_TILES][tcn / CB] + tcn % CB;
      return col0 + tcn;
    };
    // column exponents: two registers per lane (columns cbase + lane, cbase + 32 + lane), handed
    // to the column's threads by shuffles; the chunk's exponents are loaded before its MMAs end
    const int cl0 = bcol(cbase + lane), cl1 = lane + 32 < EPI_COLS ? bcol(cbase + lane + 32) : a.rowsB;
    const bool cv0 = cl0 < a.rowsB, cv1 = lane + 32 < EPI_COLS && cl1 < a.rowsB;
    const int mb0 = cv0 ? __ldg(a.maxB + cl0) : 0, mb1 = cv1 ? __ldg(a.maxB + cl1) : 0;
    for (int c = 0; c < nch; ++c) {
      const int chunk = c_begin + c;
      const int sa = (row < a.rowsA) ? __ldg(a.sigA + (long long)chunk * a.sig_ldA + row) - ra : 0;
      const int sb0 = cv0 ? __ldg(a.sigB + (long long)chunk * a.sig_ldB + cl0) - mb0 : 0;
      const int sb1 = cv1 ? __ldg(a.sigB + (long long)chunk * a.sig_ldB + cl1) - mb1 : 0;
      bool ok = tc::mbar_wait(&dfull, c & 1);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1004);
        }
        break;
      }
      tc::fence_after_sync();
#pragma unroll
      for (int b = 0; b < EPI_COLS / 8; ++b) {
        uint32_t d[NACC][8];
        const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cbase + b * 8);
#pragma unroll
        for (int o = 0; o < NACC; ++o) tc::tmem_ld8(base + o * BN, d[o]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cj = b * 8 + j;
          const int sb = __shfl_sync(0xffffffffu, cj < 32 ? sb0 : sb1, cj & 31);
          const float scale = pow2f_nonpos(sa + sb);
          // D0 + D1 + D2 + D3 exactly as a double-float, then D4
          float s1, e1, s2, e2, s3, e3, vh, vl;
          two_sum(__uint_as_float(d[0][j]), __uint_as_float(d[1][j]), s1, e1);
          two_sum(s1, __uint_as_float(d[2][j]), s2, e2);
          two_sum(s2, __uint_as_float(d[3][j]), s3, e3);
          two_sum(s3, ((e1 + e2) + e3) + __uint_as_float(d[4][j]), vh, vl);
          df_add(ahi[b * 8 + j], alo[b * 8 + j], vh * scale, vl * scale);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&dempty);
    }
    // columns beyond this tile's half of B belong to the other half's tiles
    const int col_lim = min(a.rowsB, (tcol / T) * HS + a.half_rows);
    if (a.rotation) {
      if (row < a.rowsA && !abort_flag) {
        const int band = row % a.rot_nb, part = row / a.rot_nb;
        const long long base = (long long)band * a.rot_K;
        if (a.rot_vec) {
          // real bands, 16-byte aligned rows: 4 (FP32) or 2 (FP64) values per store
#pragma unroll
          for (int j = 0; j < EPI_COLS; j += 4) {
            const int col = col0 + cbase + j;
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              v[u] = col + u < a.rowsB ? df_to_double(ahi[j + u], alo[j + u], ra + __ldg(a.maxB + col + u)) : 0.0;
            if (col + 3 < a.rowsB) {
              if (a.rot_fp32) {
                *(float4*)((float*)a.rot_out + base + col) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
              } else {
                *(double2*)((double*)a.rot_out + base + col) = make_double2(v[0], v[1]);
                *(double2*)((double*)a.rot_out + base + col + 2) = make_double2(v[2], v[3]);
              }
            } else {
              for (int u = 0; u < 4 && col + u < a.rowsB; ++u) {
                if (a.rot_fp32) ((float*)a.rot_out)[base + col + u] = (float)v[u];
                else ((double*)a.rot_out)[base + col + u] = v[u];
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < EPI_COLS; ++j) {
            const int col = col0 + cbase + j;
            if (col < a.rowsB) {
              const double v = df_to_double(ahi[j], alo[j], ra + __ldg(a.maxB + col));
              const long long idx = a.rot_cplx ? 2 * (base + col) + part : base + col;
              if (a.rot_fp32) ((float*)a.rot_out)[idx] = (float)v;
              else ((double*)a.rot_out)[idx] = v;
            }
          }
        }
      }
    } else if (COVER) {
      // the symmetric cover: the entries of the block pairs this tile owns, at (min, max) of
      // its half
      if (row < a.rowsA && !abort_flag) {
        const int cov_t = blockIdx.x % COVER_TILES, cov_h = blockIdx.x / COVER_TILES;
        const unsigned long long own = a.cov_own[cov_t], trm = a.cov_tr[cov_t];
        const int bi = row / CB, hoff = cov_h * HS;
        double* base = a.part + (long long)blockIdx.y * a.rowsA * a.rowsB + hoff;
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) {
          const int col = bcol(cbase + j);    // B row
          const int m = col - hoff;           // band of the column
          if (m >= a.half_rows) continue;
          const int bj = m / CB, lo = min(bi, bj), hi = max(bi, bj);
          const int bit = lo * 8 + hi;
          if (!((own >> bit) & 1ull)) continue;
          const bool write = bi == bj ? row <= m : (((trm >> bit) & 1ull) ? bi == hi : bi == lo);
          if (!write) continue;
          double v = df_to_double(ahi[j], alo[j], ra + __ldg(a.maxB + col));
          if (cov_h == 1 && row > m) v = -v;
          double* o = base + (long long)min(row, m) * a.rowsB + max(row, m);
          *o = a.accumulate ? *o + v : v;
        }
      }
    } else if (row < a.rowsA && !abort_flag) {
      double* out = a.part + ((long long)blockIdx.y * a.rowsA + row) * a.rowsB;
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) {
        const int col = col0 + cbase + j;
        if (col < col_lim) {
          const double v = df_to_double(ahi[j], alo[j], ra + __ldg(a.maxB + col));
          out[col] = a.accumulate ? out[col] + v : v;
        }
      }
    }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0)   // let issued copies land before the CTA exits (bounded)
    for (int g = consumed; g < issued; ++g) tc::mbar_wait(&full[g % STAGES], (g / STAGES) & 1);
  __syncthreads();
  if (warp == EPI_WARPS) tc::tmem_free(tmem, TMEM_COLS);
}

}  // namespace sg
}  // namespace pawfd
