// fused_gram.cuh -- Gram matrices on the BF16 tensor cores, digits made inside the kernel.
//
// The same exact digit-product scheme as sliced_gram.cuh (balanced base-128 digits per row and
// 256-value chunk, five TMEM accumulators by digit order, double-float epilogue), but the
// digit planes never go through HBM: a TMA warp streams the raw FP64 / FP32 tiles of both
// operands into a shared-memory ring, eight worker warps turn every 16-value tile into S digit
// planes written straight into the 32-byte-swizzled layout the MMA descriptors read, and one
// warp issues the tcgen05 MMAs.  The workers also run the per-chunk epilogue.  The chunk
// exponents sigma come from a separate light pass (sigma_kernel), so a tile can be converted
// as soon as it lands.
//
//   FP32 data: y = x 2^-sigma (|y| < 64), then d_i = rint(y_i), y_{i+1} = 128 (y_i - d_i): every
//              step is exact in FP32, and the digits are balanced by construction.
//   FP64 data: the integer path of slice_kernel on the IEEE fields (no FP64 arithmetic).
#pragma once

#include <cuda_bf16.h>

#include "sliced_gram.cuh"

namespace pawfd {
namespace fg {

using sg::BK;
using sg::BM;
using sg::BN;
using sg::KC;
using sg::NACC;

constexpr int WORKERS = 8;                    // converter + epilogue warps
constexpr int NTHREADS = (WORKERS + 2) * 32;  // + TMA warp + MMA warp
constexpr int EPI_COLS = BN / 2;
constexpr int TMEM_COLS = 512;
constexpr int ROWS = BM + BN;                 // operand rows of one stage (A then B)

template <class R> struct Cfg;
template <> struct Cfg<double> { static constexpr int S = 7, ORD = 6, RAW = 4, DIG = 2; };
template <> struct Cfg<float> { static constexpr int S = 4, ORD = 4, RAW = 6, DIG = 4; };

template <class R> __host__ __device__ constexpr int raw_stage_bytes() { return ROWS * BK * (int)sizeof(R); }
template <class R> __host__ __device__ constexpr int dig_stage_bytes() { return Cfg<R>::S * ROWS * BK * 2; }
template <class R> __host__ __device__ constexpr int smem_bytes() {
  return Cfg<R>::DIG * dig_stage_bytes<R>() + Cfg<R>::RAW * raw_stage_bytes<R>() + 1024;
}

// ------------------------------------------------------------------------------------------
// chunk exponents
// ------------------------------------------------------------------------------------------
// One warp per (row, chunk): sig[chunk][row] = E - bias - 5 for the chunk's largest biased
// exponent E (the digit scale of slice_kernel), maxsig[row] = max over the row's chunks
// (reset to INT_MIN by the caller).  Values past len are zero.
template <class R>
__global__ void __launch_bounds__(256) sigma_kernel(const R* __restrict__ src, int rows, long long ld, long long len,
                                                    int nchunks, int* __restrict__ sig, int sig_ld,
                                                    int* __restrict__ maxsig) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)rows * nchunks) return;
  const int r = (int)(warp / nchunks);
  const long long c = warp % nchunks;
  const R* row = src + (long long)r * ld;
  int emax = 0;
  for (int t = lane; t < KC; t += 32) {
    const long long k = c * KC + t;
    if (k < len) emax = max(emax, sg::fields(row[k]).exp);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (lane == 0) {
    const int s = emax - sg::FloatBits<R>::bias - 5;
    sig[c * sig_ld + r] = s;
    atomicMax(maxsig + r, s);
  }
}

// ------------------------------------------------------------------------------------------
// conversion of 8 consecutive values of one row into S planes of 8 bf16 digits
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// out[i][j]: plane i, values 2j and 2j+1 of the N in word j.  sigma: the chunk's digit scale.
template <int S, int N>
__device__ __forceinline__ void digits(const float (&x)[N], int sigma, uint32_t (&out)[S][N / 2]) {
  // y = x 2^-sigma exactly (|y| < 64); a chunk below the normal range has all-zero digits
  const float scale = (sigma > 126 || sigma < -126) ? 0.0f : __int_as_float((127 - sigma) << 23);
  float y[N];
#pragma unroll
  for (int v = 0; v < N; ++v) y[v] = x[v] * scale;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    float d[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      d[v] = rintf(y[v]);
      y[v] = (y[v] - d[v]) * 128.0f;
    }
    const float w = __int_as_float((127 - 7 * i) << 23);   // 2^-7i
#pragma unroll
    for (int j = 0; j < N / 2; ++j) out[i][j] = pack_bf16x2(d[2 * j] * w, d[2 * j + 1] * w);
  }
}

template <int S, int N>
__device__ __forceinline__ void digits(const double (&x)[N], int sigma, uint32_t (&out)[S][N / 2]) {
  constexpr int bias = 1023, nbits = 52;
  constexpr int g = 7 * S - 1 - nbits;
  const int emax = sigma + bias + 5;
#pragma unroll
  for (int p = 0; p < N / 2; ++p) {
    float dv[S][2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const sg::Fields f = sg::fields(x[2 * p + u]);
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
      for (int i = 0; i < S; ++i) dv[i][u] = (f.neg ? -(float)d[i] : (float)d[i]) * __int_as_float((127 - 7 * i) << 23);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) out[i][p] = pack_bf16x2(dv[i][0], dv[i][1]);
  }
}

// values converted per work item: 4 for FP64 (register pressure), 8 for FP32
template <class R> __host__ __device__ constexpr int vpi() { return sizeof(R) == 8 ? 4 : 8; }

struct FusedArgs {
  sg::GramArgs g;            // tiles, scales, partials, rotation fields (as the sliced kernel)
  int braw_rows = 0;         // rows of B's raw tensor (complex: nb; B'' rows map onto them)
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          tc::smem_addr(dst)),
      "l"((uint64_t)map), "r"(tc::smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <class R>
__global__ void __launch_bounds__(NTHREADS, 1) fused_gram_kernel(const __grid_constant__ CUtensorMap tA,
                                                                 const __grid_constant__ CUtensorMap tB, FusedArgs fa) {
  constexpr int S = Cfg<R>::S, ORD = Cfg<R>::ORD, RAW = Cfg<R>::RAW, DIG = Cfg<R>::DIG;
  const sg::GramArgs& a = fa.g;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* dig = smem;                                  // [DIG][S][ROWS][32 B], swizzled
  unsigned char* raw = smem + DIG * dig_stage_bytes<R>();     // [RAW][ROWS][BK] R
  __shared__ uint64_t raw_full[RAW], raw_empty[RAW], dig_full[DIG], dig_empty[DIG], dfull, dempty, mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tr, tcol;
  sg::gram_tile(a, blockIdx.x, &tr, &tcol);
  const int row0 = tr * BM;
  const int T = (a.half_rows + BN - 1) / BN;
  const int half = tcol / T;                       // complex: 1 = the swapped half of B
  const int col0 = half * a.half_rows + (tcol % T) * BN;
  const int braw0 = col0 - half * a.half_rows;     // first raw row of B in this tile
  const bool swapped = half == 1;
  const int c_begin = blockIdx.y * a.chunks_per_cta;
  const int c_end = min(a.nchunks, c_begin + a.chunks_per_cta);
  const int nch = max(0, c_end - c_begin);
  constexpr int SPC = KC / BK;                     // stages per chunk
  const int total = nch * SPC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW; ++s) {
      tc::mbar_init(&raw_full[s], 1);
      tc::mbar_init(&raw_empty[s], WORKERS);
    }
    for (int s = 0; s < DIG; ++s) {
      tc::mbar_init(&dig_full[s], WORKERS);
      tc::mbar_init(&dig_empty[s], 1);
    }
    tc::mbar_init(&dfull, 1);
    tc::mbar_init(&dempty, WORKERS);
    tc::mbar_init(&mma_done, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    tc::mbar_fence_init();
  }
  if (warp == WORKERS) tc::tmem_alloc(&tmem_base, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == WORKERS) {
    if (lane == 0) {   // TMA producer: raw tiles of A (BM rows) and B (BN rows) per stage
      for (int g = 0; g < total && !abort_flag; ++g) {
        const int s = g % RAW;
        if (g >= RAW && !tc::mbar_wait(&raw_empty[s], ((g / RAW) - 1) & 1)) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1101);
          break;
        }
        const int kx = (c_begin + g / SPC) * KC + (g % SPC) * BK;
        unsigned char* ra = raw + s * raw_stage_bytes<R>();
        tc::mbar_expect_tx(&raw_full[s], raw_stage_bytes<R>());
        tma_load_2d(ra, &tA, &raw_full[s], kx, row0);
        tma_load_2d(ra + BM * BK * sizeof(R), &tB, &raw_full[s], kx, braw0);
        issued = g + 1;
      }
    }
  } else if (warp == WORKERS + 1) {
    if (lane == 0) {   // MMA issuer
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
      for (int c = 0; c < nch && !abort_flag; ++c) {
        if (c > 0 && !tc::mbar_wait(&dempty, (c - 1) & 1)) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1102);
          break;
        }
        tc::fence_after_sync();
        for (int q = 0; q < SPC && !abort_flag; ++q) {
          const int g = c * SPC + q;
          const int s = g % DIG;
          if (!tc::mbar_wait(&dig_full[s], (g / DIG) & 1)) {
            abort_flag = 1;
            set_status(a.st, PAWFD_ETIMEDOUT, 1103);
            break;
          }
          tc::fence_after_sync();
          unsigned char* sa = dig + s * dig_stage_bytes<R>();
          unsigned char* sb = sa + S * BM * BK * 2;
          bool touched[NACC] = {false, false, false, false, false};
#pragma unroll
          for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (i + j > ORD) continue;
              const int slot = (i + j) < NACC - 1 ? (i + j) : NACC - 1;
              const uint32_t d = tmem + (uint32_t)(slot * BN);
              const bool first = (q == 0) && !touched[slot];
              touched[slot] = true;
              tc::mma_bf16(d, tc::smem_desc(sa + i * BM * BK * 2, BK * 2), tc::smem_desc(sb + j * BN * BK * 2, BK * 2),
                           idesc, first ? 0u : 1u);
            }
          tc::mma_commit(&dig_empty[s]);
          consumed = g + 1;
        }
        tc::mma_commit(&dfull);
      }
      if (abort_flag) {
        // every MMA issued so far must be complete before the TMEM is released
        tc::mma_commit(&mma_done);
        tc::mbar_wait(&mma_done, 0);
      }
    }
  } else {
    // ---- workers: conversion of every stage, epilogue of every chunk ----
    const int tid = threadIdx.x;                      // 0 .. 255
    const int quarter = warp & 3, chalf = warp >> 2;
    const int erow = row0 + quarter * 32 + lane;      // epilogue row (TMEM lane)
    const int cbase = chalf * EPI_COLS;
    float ahi[EPI_COLS], alo[EPI_COLS];
#pragma unroll
    for (int j = 0; j < EPI_COLS; ++j) {
      ahi[j] = 0.0f;
      alo[j] = 0.0f;
    }
    const int ra = (erow < a.rowsA) ? __ldg(a.maxA + erow) : 0;
    bool ok = true;
    // chunk c's epilogue runs after the first `lead` stages of chunk c + 1 are converted, so
    // that the MMA has work as soon as the accumulators are free again
    constexpr int lead = DIG < SPC ? DIG : SPC;
    int next_epi = 0;
    auto epilogue = [&](int c) {
      bool got = tc::mbar_wait(&dfull, c & 1);
      got = __all_sync(0xffffffffu, got);
      if (!got) {
        if (lane == 0) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1104);
        }
        ok = false;
        return;
      }
      tc::fence_after_sync();
      const int chunk = c_begin + c;
      const int sa_ = (erow < a.rowsA) ? __ldg(a.sigA + (long long)chunk * a.sig_ldA + erow) - ra : 0;
#pragma unroll
      for (int b = 0; b < EPI_COLS / 8; ++b) {
        uint32_t d[NACC][8];
        const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cbase + b * 8);
#pragma unroll
        for (int o = 0; o < NACC; ++o) tc::tmem_ld8(base + o * BN, d[o]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int col = col0 + cbase + b * 8 + j;
          const int bcol = col - half * a.half_rows;   // raw row of B (sigma index)
          const int sb_ = (col < a.rowsB && bcol < fa.braw_rows)
                              ? __ldg(a.sigB + (long long)chunk * a.sig_ldB + bcol) - __ldg(a.maxB + bcol)
                              : 0;
          const float scale = sg::pow2f_nonpos(sa_ + sb_);
          float s1, e1, s2, e2, s3, e3, vh, vl;
          sg::two_sum(__uint_as_float(d[0][j]), __uint_as_float(d[1][j]), s1, e1);
          sg::two_sum(s1, __uint_as_float(d[2][j]), s2, e2);
          sg::two_sum(s2, __uint_as_float(d[3][j]), s3, e3);
          sg::two_sum(s3, ((e1 + e2) + e3) + __uint_as_float(d[4][j]), vh, vl);
          sg::df_add(ahi[b * 8 + j], alo[b * 8 + j], vh * scale, vl * scale);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&dempty);
    };

    // the rows a worker converts are the same in every stage: their chunk exponents are loaded
    // once per chunk
    constexpr int N = vpi<R>(), PER_ROW = BK / N;
    constexpr int ITEMS = ROWS * PER_ROW, KMAX = (ITEMS + WORKERS * 32 - 1) / (WORKERS * 32);
    int sig_reg[KMAX];
    for (int g = 0; g < total && ok && !abort_flag; ++g) {
      const int rs = g % RAW, ds = g % DIG;
      const int chunk = c_begin + g / SPC;
      if (g % SPC == 0) {
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
          const int item = tid + k * WORKERS * 32;
          const int r = item / PER_ROW;
          int sg_ = 0;
          if (item < ITEMS) {
            if (r < BM) {
              const int grow = row0 + r;
              if (grow < a.rowsA) sg_ = __ldg(a.sigA + (long long)chunk * a.sig_ldA + grow);
            } else {
              const int grow = braw0 + r - BM;
              if (grow < fa.braw_rows) sg_ = __ldg(a.sigB + (long long)chunk * a.sig_ldB + grow);
            }
          }
          sig_reg[k] = sg_;
        }
      }
      bool got = tc::mbar_wait(&raw_full[rs], (g / RAW) & 1);
      if (got && g >= DIG) got = tc::mbar_wait(&dig_empty[ds], ((g / DIG) - 1) & 1);
      got = __all_sync(0xffffffffu, got);
      if (!got) {
        if (lane == 0) {
          abort_flag = 1;
          set_status(a.st, PAWFD_ETIMEDOUT, 1105);
        }
        ok = false;
        break;
      }
      const R* rt = (const R*)(raw + rs * raw_stage_bytes<R>());
      unsigned char* dt = dig + ds * dig_stage_bytes<R>();
      // items: (row of the stage, which N of its 16 values)
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int item = tid + k * WORKERS * 32;
        if (item >= ITEMS) break;
        const int r = item / PER_ROW, v0 = (item % PER_ROW) * N;
        const bool isA = r < BM;
        const int orow = isA ? r : r - BM;             // row within its operand tile
        const int sigma = sig_reg[k];
        R x[N];
        const R* src = rt + r * BK + v0;
#pragma unroll
        for (int v = 0; v < N; ++v) x[v] = src[v];
        if (!isA && swapped) {
          // B'' = (im, -re) per complex pair (pairs never straddle an item: N is even)
#pragma unroll
          for (int v = 0; v < N; v += 2) {
            const R re = x[v], im = x[v + 1];
            x[v] = im;
            x[v + 1] = -re;
          }
        }
        uint32_t out[S][N / 2];
        digits<S, N>(x, sigma, out);
        // 32-byte rows; the two 16-byte halves are swapped on rows 4..7 of every 8 (32-byte swizzle)
        const int h = v0 >> 3;
        const int off = orow * 32 + ((h ^ ((orow >> 2) & 1)) << 4) + (v0 & 7) * 2;
        unsigned char* base = dt + (isA ? 0 : S * BM * BK * 2);
        const int plane = isA ? BM * BK * 2 : BN * BK * 2;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          if constexpr (N == 8)
            *(uint4*)(base + i * plane + off) = make_uint4(out[i][0], out[i][1], out[i][2], out[i][3]);
          else
            *(uint2*)(base + i * plane + off) = make_uint2(out[i][0], out[i][1]);
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&raw_empty[rs]);
        tc::mbar_arrive(&dig_full[ds]);
      }
      // epilogue of the previous chunk once `lead` stages of this chunk are converted
      if ((g % SPC) == lead - 1 && g / SPC > 0) {
        epilogue(next_epi);
        ++next_epi;
      }
    }
    while (ok && !abort_flag && next_epi < nch) {
      epilogue(next_epi);
      ++next_epi;
    }
    // write the tile (partials, or the rotated bands)
    const int col_lim = min(a.rowsB, (tcol / T + 1) * a.half_rows);
    if (ok && !abort_flag && erow < a.rowsA) {
      double* out = a.part + ((long long)blockIdx.y * a.rowsA + erow) * a.rowsB;
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) {
        const int col = col0 + cbase + j;
        const int bcol = col - half * a.half_rows;
        if (col < col_lim) {
          const double v = ((double)ahi[j] + (double)alo[j]) * sg::pow2(ra + __ldg(a.maxB + bcol));
          out[col] = v;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (abort_flag && threadIdx.x == 0)   // let the last copies of every raw slot land (bounded)
    for (int g = max(0, issued - RAW); g < issued; ++g) tc::mbar_wait(&raw_full[g % RAW], (g / RAW) & 1);
  __syncthreads();
  if (warp == WORKERS) tc::tmem_free(tmem, TMEM_COLS);
}

}  // namespace fg
}  // namespace pawfd
