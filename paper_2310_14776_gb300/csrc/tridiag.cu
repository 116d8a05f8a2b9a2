// tridiag.cu -- an FP32 eigendecomposition A ~= Z diag(lambda) Z^H of the reduced Hermitian
// matrix A = L^-1 H L^-H of the subspace solve: the starting basis of its FP64 Ogita-Aishima
// refinement (subspace.cu), which makes the result exact to FP64.
//
// The dense diagonalization is the step the paper hands to ScaLAPACK / ELPA or a single core
// (parallelization section).  GB300's FP64 rate is a small fraction of its FP32 rate, and a
// Jacobi sweep costs n - 1 device-wide synchronizations, so the far path computes its basis by
// the textbook route (Golub & Van Loan, "Matrix Computations", ch. 8) in FP32 instead:
//   1. Householder reduction Q^H A Q = T to a real symmetric tridiagonal T (the complex
//      reflectors are chosen so that the off-diagonal of T is real), one thread-block
//      cluster, two cluster barriers per column;
//   2. the eigenvalues of T by multisection on Sturm counts, one warp per eigenvalue;
//   3. the eigenvectors of T by inverse iteration with a partial-pivoting LU of T - sigma I,
//      the vectors of eigenvalues closer than 1e-5 ||T||_1 orthogonalized against each other
//      (modified Gram-Schmidt within each iteration), one warp per group of such eigenvalues;
//      then three Newton-Schulz steps Y <- Y (3 I - Y^T Y) / 2, which take the overlaps that
//      inverse iteration leaves between vectors of close but separate eigenvalues (about
//      eps ||T|| / gap, below 1e-2 outside the groups) down to FP32 rounding in parallel, where
//      Gram-Schmidt over a group of close eigenvalues would be one long sequential chain (a
//      narrow spectrum, such as the Ritz values of random bands, is one such group);
//   4. Z = Q Y, the reflectors applied to the eigenvectors of T, one warp per vector.
// Every step is deterministic (fixed reduction orders, a fixed pseudo-random start vector per
// eigenvector), so repeated solves of the same matrix give bitwise the same Z.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "device_sync.cuh"
#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

template <class T> struct Low;
template <> struct Low<double> { using F = float; };
template <> struct Low<zd> { using F = zf; };
template <class T> using low_t = typename Low<T>::F;

constexpr int TR_NT = 1024;    // threads per CTA of the reduction
constexpr int TR_CTAS = 16;    // CTAs of the reduction (one cluster where it can be launched)

__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ zf ldcg(const zf* p) {
  const float2 v = __ldcg((const float2*)p);
  return zf{v.x, v.y};
}
__device__ __forceinline__ float imagx(float) { return 0.f; }
__device__ __forceinline__ float imagx(zf x) { return x.im; }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ zf shfl_xor(zf v, int o) {
  return zf{__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}
template <class F> __device__ __forceinline__ F make_f(float re, float im);
template <> __device__ __forceinline__ float make_f<float>(float re, float) { return re; }
template <> __device__ __forceinline__ zf make_f<zf>(float re, float im) { return zf{re, im}; }

// butterfly sum: every lane ends with the same value (each level adds a pair in both orders,
// and IEEE addition is commutative)
template <class F> __device__ __forceinline__ F warp_sum(F v) {
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  return v;
}

// sum over the CTA, the same value in every thread (and in every CTA for the same inputs)
template <class F> __device__ F block_sum_all(F v, F* s_red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  F s = F{};
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w];
  return s;
}

// ------------------------------------------------------------------------------------------
// 1. Householder tridiagonalization.  Step k reduces column k below the subdiagonal with
//    H_k = I - tau v v^H (v_0 = 1), H_k^H x = (beta, 0, ..., 0), beta real (the LAPACK larfg
//    convention), and applies A22 <- H_k^H A22 H_k as A22 - v w^H - w v^H with p = tau A22 v,
//    w = p - (tau / 2)(p^H v) v.  A is kept full (both triangles), so column k is read as the
//    conjugate of row k.  Rows of the trailing block belong to warps (row r to warp r mod
//    warps).  On exit d, e hold T (e[k] = beta_k), tau[k] and v_k (in row k, columns
//    k+1 .. n-1) the reflectors.
// ------------------------------------------------------------------------------------------
template <class T, int MODE>
__global__ void __launch_bounds__(TR_NT) tridiag_kernel(const T* __restrict__ A, int n, low_t<T>* __restrict__ W,
                                                        low_t<T>* __restrict__ P, float* __restrict__ d,
                                                        float* __restrict__ e, low_t<T>* __restrict__ tau,
                                                        unsigned* bar, DeviceStatus* st, const int* gate) {
  using F = low_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* sv = (F*)smem_raw;   // v of this step [n]
  F* sw = sv + n;         // p, then w [n]
  __shared__ F s_red[32];
  __shared__ float s_redf[32];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const unsigned G = gridDim.x;
  const long long gthreads = (long long)G * blockDim.x;
  const long long nn = (long long)n * n;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < nn; x += gthreads)
    W[x] = narrow<F>(A[x]);
  if (!all_barrier<MODE>(bar, G, st, 800)) return;
  const int lane = threadIdx.x & 31;
  const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)(gthreads >> 5);
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    const F* rowk = W + (long long)k * n + k + 1;
    float xn2 = 0.f;   // ||x_1..||^2
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const F x = conjx(ldcg(rowk + j));
      sv[j] = x;
      if (j > 0) xn2 += absx2(x);
    }
    xn2 = block_sum_all(xn2, s_redf);   // ends with a barrier of the CTA: sv is complete
    const F alpha = sv[0];
    const float ar = realx(alpha), ai = imagx(alpha);
    const bool active = !(xn2 == 0.f && ai == 0.f);
    float beta = ar;
    F t = F{};
    F scale = F{};
    if (active) {
      const float nrm = sqrtf(ar * ar + ai * ai + xn2);
      beta = ar >= 0.f ? -nrm : nrm;
      t = make_f<F>((beta - ar) / beta, -ai / beta);
      // 1 / (alpha - beta)
      const float dr = ar - beta, di = ai, den = dr * dr + di * di;
      scale = make_f<F>(dr / den, -di / den);
    }
    __syncthreads();   // every thread has read sv[0]
    if (active)
      for (int j = threadIdx.x; j < m; j += blockDim.x) sv[j] = j == 0 ? make_f<F>(1.f, 0.f) : sv[j] * scale;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      d[k] = realx(ldcg(W + (long long)k * n + k));
      e[k] = beta;
      tau[k] = t;
    }
    __syncthreads();
    if (active) {
      // p = tau A22 v
      for (int i = gwarp; i < m; i += nwarps) {
        const F* row = W + (long long)(k + 1 + i) * n + k + 1;
        F acc = F{};
        for (int j = lane; j < m; j += 32) fma_plain(acc, ldcg(row + j), sv[j]);
        acc = warp_sum(acc);
        if (lane == 0) P[i] = t * acc;
      }
    }
    if (!all_barrier<MODE>(bar, G, st, 801)) return;
    if (active) {
      // w = p - (tau / 2)(p^H v) v
      F pv = F{};
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const F p = ldcg(P + j);
        sw[j] = p;
        fma_conj(pv, p, sv[j]);
      }
      pv = block_sum_all(pv, s_red);
      const F c = -0.5f * (t * pv);
      for (int j = threadIdx.x; j < m; j += blockDim.x) fma_plain(sw[j], c, sv[j]);
      __syncthreads();
      for (int i = gwarp; i < m; i += nwarps) {
        F* row = W + (long long)(k + 1 + i) * n + k + 1;
        const F vi = sv[i], wi = sw[i];
        for (int j = lane; j < m; j += 32) {
          F a = ldcg(row + j);
          a -= vi * conjx(sw[j]) + wi * conjx(sv[j]);
          row[j] = a;
        }
        // the reflector goes to row k, which no CTA reads after this step's first barrier
        if (lane == 0) W[(long long)k * n + k + 1 + i] = sv[i];
      }
    }
    if (!all_barrier<MODE>(bar, G, st, 802)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d[n - 1] = realx(ldcg(W + (long long)(n - 1) * n + n - 1));
    e[n - 1] = 0.f;
  }
}

// The same reduction with the trailing block resident in the cluster's shared memory (one
// cluster of TR_CTAS CTAs, when n^2 values fit): each warp keeps its rows (row r in warp
// r mod warps) in its CTA's shared memory for the whole reduction; p is scattered into every
// CTA's shared memory and the next pivot row is read from its owner's, both through the
// cluster's distributed shared memory, so a step is two cluster barriers and no global-memory
// round trip.  Only the gate may end the kernel early: it is the same word for every CTA, so
// no CTA leaves a cluster barrier without the others.
template <class T>
__global__ void __launch_bounds__(TR_NT) tridiag_dsm_kernel(const T* __restrict__ A, int n, int R,
                                                            low_t<T>* __restrict__ W, float* __restrict__ d,
                                                            float* __restrict__ e, low_t<T>* __restrict__ tau,
                                                            const int* gate) {
  using F = low_t<T>;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* rows = (F*)smem_raw;                 // [32 R][n] this CTA's rows
  F* sP = rows + (size_t)32 * R * n;      // [n] p of this step, written by every CTA
  F* sv = sP + n;                         // [n] v
  F* sw = sv + n;                         // [n] w
  __shared__ F s_red[32];
  __shared__ float s_redf[32];
  if (gated(gate)) return;
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();   // every CTA runs before the first access to its shared memory
  const int rank = (int)cl.block_rank();
  const int NW = 32 * (int)cl.num_blocks();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = 0; q < R; ++q) {
    const int r = rank * 32 + warp + q * NW;
    if (r < n)
      for (int j = lane; j < n; j += 32) rows[(size_t)(warp + 32 * q) * n + j] = narrow<F>(A[(long long)r * n + j]);
  }
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    // pivot row k: from A at k = 0, else from its owner's shared memory
    const int wk = k % NW;
    const F* prow = nullptr;
    if (k > 0) prow = cl.map_shared_rank(rows + (size_t)(wk % 32 + 32 * (k / NW)) * n, wk / 32);
    float xn2 = 0.f;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const F x = conjx(k == 0 ? narrow<F>(A[k + 1 + j]) : prow[k + 1 + j]);
      sv[j] = x;
      if (j > 0) xn2 += absx2(x);
    }
    xn2 = block_sum_all(xn2, s_redf);
    const F alpha = sv[0];
    const float ar = realx(alpha), ai = imagx(alpha);
    const bool active = !(xn2 == 0.f && ai == 0.f);
    float beta = ar;
    F t = F{};
    F scale = F{};
    if (active) {
      const float nrm = sqrtf(ar * ar + ai * ai + xn2);
      beta = ar >= 0.f ? -nrm : nrm;
      t = make_f<F>((beta - ar) / beta, -ai / beta);
      const float dr = ar - beta, di = ai, den = dr * dr + di * di;
      scale = make_f<F>(dr / den, -di / den);
    }
    __syncthreads();
    if (active)
      for (int j = threadIdx.x; j < m; j += blockDim.x) sv[j] = j == 0 ? make_f<F>(1.f, 0.f) : sv[j] * scale;
    if (rank == 0 && threadIdx.x == 0) {
      d[k] = realx(k == 0 ? narrow<F>(A[0]) : prow[k]);
      e[k] = beta;
      tau[k] = t;
    }
    __syncthreads();
    if (active) {
      if (rank == 0)
        for (int j = threadIdx.x; j < m; j += blockDim.x) W[(long long)k * n + k + 1 + j] = sv[j];
      for (int q = 0; q < R; ++q) {
        const int r = rank * 32 + warp + q * NW;
        if (r <= k || r >= n) continue;
        const F* row = rows + (size_t)(warp + 32 * q) * n + k + 1;
        F acc = F{};
        for (int j = lane; j < m; j += 32) fma_plain(acc, row[j], sv[j]);
        acc = warp_sum(acc);
        if (lane < (int)cl.num_blocks()) *cl.map_shared_rank(sP + (r - k - 1), lane) = t * acc;
      }
    }
    cl.sync();
    if (active) {
      F pv = F{};
      for (int j = threadIdx.x; j < m; j += blockDim.x) fma_conj(pv, sP[j], sv[j]);
      pv = block_sum_all(pv, s_red);
      const F c = -0.5f * (t * pv);
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        F w = sP[j];
        fma_plain(w, c, sv[j]);
        sw[j] = w;
      }
      __syncthreads();
      for (int q = 0; q < R; ++q) {
        const int r = rank * 32 + warp + q * NW;
        if (r <= k || r >= n) continue;
        F* row = rows + (size_t)(warp + 32 * q) * n + k + 1;
        const int i = r - k - 1;
        const F vi = sv[i], wi = sw[i];
        for (int j = lane; j < m; j += 32) row[j] -= vi * conjx(sw[j]) + wi * conjx(sv[j]);
      }
    }
    cl.sync();
  }
  if (rank == 0 && threadIdx.x == 0) {
    const int wk = (n - 1) % NW;
    const F* prow = cl.map_shared_rank(rows + (size_t)(wk % 32 + 32 * ((n - 1) / NW)) * n, wk / 32);
    d[n - 1] = n == 1 ? realx(narrow<F>(A[0])) : realx(prow[n - 1]);
    e[n - 1] = 0.f;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------------------------------------------
// 2. Eigenvalues of T, ascending: lambda_j by multisection.  Each lane of the warp of j counts
//    the eigenvalues below one of 32 points of the current interval (the signs of the pivots
//    of the LDL^T factorization of T - x I, pivots kept away from 0 by pivmin); the interval
//    shrinks to the two points around the place where the count passes j, 33 times per pass.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tri_bisect_kernel(const float* __restrict__ d, const float* __restrict__ e,
                                                         int n, float* __restrict__ lam, const DeviceStatus* st,
                                                         const int* gate) {
  extern __shared__ float sdf[];
  float* sd = sdf;       // [n] diagonal
  float* se2 = sdf + n;  // [n] squared off-diagonal
  __shared__ float s_lo[8], s_hi[8], s_e2[8];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  float lo = FLT_MAX, hi = -FLT_MAX, emax2 = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float di = d[i];
    const float ei = i + 1 < n ? e[i] : 0.f;
    const float em = i > 0 ? e[i - 1] : 0.f;
    const float r = fabsf(ei) + fabsf(em);
    sd[i] = di;
    se2[i] = ei * ei;
    lo = fminf(lo, di - r);
    hi = fmaxf(hi, di + r);
    emax2 = fmaxf(emax2, ei * ei);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax2 = fmaxf(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
    s_e2[warp] = emax2;
  }
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
  emax2 = s_e2[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    lo = fminf(lo, s_lo[w]);
    hi = fmaxf(hi, s_hi[w]);
    emax2 = fmaxf(emax2, s_e2[w]);
  }
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= n) return;
  const float pivmin = FLT_MIN * fmaxf(1.f, emax2);
  const float tnorm = fmaxf(fabsf(lo), fabsf(hi));
  float a = lo - 2.f * FLT_EPSILON * tnorm - 2.f * pivmin;
  float b = hi + 2.f * FLT_EPSILON * tnorm + 2.f * pivmin;
  for (int it = 0; it < 16; ++it) {
    const float x = a + (b - a) * (float)(lane + 1) / 33.f;
    int cnt = 0;
    float q = sd[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
    for (int i = 1; i < n; ++i) {
      q = (sd[i] - x) - __fdividef(se2[i - 1], q);
      if (fabsf(q) < pivmin) q = -pivmin;
      cnt += q < 0.f;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, cnt > j);
    const int f = ball ? __ffs(ball) - 1 : 32;
    const float na = f == 0 ? a : a + (b - a) * (float)f / 33.f;
    const float nb = f == 32 ? b : a + (b - a) * (float)(f + 1) / 33.f;
    a = na;
    b = nb;
    if (b - a <= 2.f * FLT_EPSILON * tnorm + pivmin) break;
  }
  if (lane == 0) lam[j] = 0.5f * (a + b);
}

// ------------------------------------------------------------------------------------------
// 3. Eigenvectors of T by inverse iteration.  The warp of j works only if j starts a group
//    (lambda_j - lambda_{j-1} > 1e-5 ||T||_1); it then computes the vectors of the group in
//    order.  Shifts within a group are kept at least 10 eps |lambda| apart.  Per vector: one
//    LU factorization of T - sigma I with partial pivoting (lane 0), three solves from a
//    fixed pseudo-random start, each followed by modified Gram-Schmidt against the group's
//    earlier vectors and normalization.  Row j of Yt receives vector j.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float start_value(int j, int i) {
  unsigned h = (unsigned)j * 0x9E3779B9u ^ ((unsigned)i * 0x85EBCA6Bu + 0x27D4EB2Fu);
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return (float)(h >> 8) * (2.f / 16777216.f) - 1.f;
}

__global__ void __launch_bounds__(32) tri_vectors_kernel(const float* __restrict__ d, const float* __restrict__ e,
                                                         const float* __restrict__ lam, int n, float* __restrict__ Yt,
                                                         const DeviceStatus* st, const int* gate) {
  extern __shared__ float svec[];
  float* u0 = svec;          // U diagonal
  float* u1 = svec + n;      // U first superdiagonal
  float* u2 = svec + 2 * n;  // U second superdiagonal
  float* ml = svec + 3 * n;  // multipliers
  float* y = svec + 4 * n;   // the iterate
  unsigned char* piv = (unsigned char*)(svec + 5 * n);
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const int j0 = blockIdx.x;
  const int lane = threadIdx.x;
  float tn = 0.f;   // ||T||_1
  for (int i = lane; i < n; i += 32) {
    const float r = fabsf(d[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i + 1 < n ? fabsf(e[i]) : 0.f);
    tn = fmaxf(tn, r);
  }
  for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  const float ortol = 1e-5f * tn;
  if (j0 > 0 && lam[j0] - lam[j0 - 1] <= ortol) return;
  int j1 = j0 + 1;
  while (j1 < n && lam[j1] - lam[j1 - 1] <= ortol) ++j1;
  const float tiny = fmaxf(FLT_EPSILON * tn, FLT_MIN);
  float sprev = 0.f;
  for (int j = j0; j < j1; ++j) {
    float sigma = lam[j];
    if (j > j0) {
      const float pertol = 10.f * FLT_EPSILON * fmaxf(fabsf(sigma), tiny);
      if (sigma - sprev < pertol) sigma = sprev + pertol;
    }
    sprev = sigma;
    if (lane == 0) {
      // P (T - sigma I) = L U; `c` is the row being eliminated (columns i, i+1)
      float c0 = d[0] - sigma, c1 = n > 1 ? e[0] : 0.f;
      for (int i = 0; i + 1 < n; ++i) {
        const float sub = e[i], dg = d[i + 1] - sigma, sup = i + 2 < n ? e[i + 1] : 0.f;
        if (fabsf(sub) > fabsf(c0)) {
          const float l = c0 / sub;
          u0[i] = sub; u1[i] = dg; u2[i] = sup; ml[i] = l; piv[i] = 1;
          c0 = c1 - l * dg;
          c1 = -l * sup;
        } else {
          const float p = fabsf(c0) < tiny ? (c0 < 0.f ? -tiny : tiny) : c0;
          const float l = sub / p;
          u0[i] = p; u1[i] = c1; u2[i] = 0.f; ml[i] = l; piv[i] = 0;
          c0 = dg - l * c1;
          c1 = sup;
        }
      }
      u0[n - 1] = fabsf(c0) < tiny ? (c0 < 0.f ? -tiny : tiny) : c0;
      u1[n - 1] = 0.f; u2[n - 1] = 0.f;
    }
    for (int i = lane; i < n; i += 32) y[i] = start_value(j, i);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) {
        // forward: the row operations of the factorization on y
        float bc = y[0];
        for (int i = 0; i + 1 < n; ++i) {
          const float bn = y[i + 1];
          if (piv[i]) { y[i] = bn; bc = bc - ml[i] * bn; }
          else { y[i] = bc; bc = bn - ml[i] * bc; }
        }
        y[n - 1] = bc;
        // backward: U y = rhs
        float y1 = 0.f, y2 = 0.f;
        for (int i = n - 1; i >= 0; --i) {
          const float v = (y[i] - u1[i] * y1 - u2[i] * y2) / u0[i];
          y[i] = v;
          y2 = y1;
          y1 = v;
        }
      }
      __syncwarp();
      // scale to unit max first (the solve grows y by about 1 / |lambda - sigma|)
      float mx = 0.f;
      for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(y[i]));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float inv = mx > 0.f ? 1.f / mx : 1.f;
      for (int i = lane; i < n; i += 32) y[i] *= inv;
      __syncwarp();
      // against the group's earlier vectors
      for (int p = j0; p < j; ++p) {
        const float* yp = Yt + (long long)p * n;
        float s = 0.f;
        for (int i = lane; i < n; i += 32) s = fmaf(yp[i], y[i], s);
        s = warp_sum(s);
        for (int i = lane; i < n; i += 32) y[i] = fmaf(-s, yp[i], y[i]);
        __syncwarp();
      }
      float nr = 0.f;
      for (int i = lane; i < n; i += 32) nr = fmaf(y[i], y[i], nr);
      nr = warp_sum(nr);
      const float r = nr > 0.f ? rsqrtf(nr) : 0.f;
      for (int i = lane; i < n; i += 32) y[i] *= r;
      __syncwarp();
    }
    float* yj = Yt + (long long)j * n;
    for (int i = lane; i < n; i += 32) yj[i] = y[i];
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// 3b. Newton-Schulz orthonormalization of the rows of Yt (the eigenvectors of T):
//     G = Yt Yt^T, then Yt <- (3 I - G) Yt / 2.  FP32 tiles of 64 x 64 (4 x 4 per thread),
//     16-deep slabs staged in shared memory.  BT: C = alpha A B^T + beta D, else
//     C = alpha A B + beta D (all n x n, row-major); the diagonal of C gets delta added.
// ------------------------------------------------------------------------------------------
template <bool BT>
__global__ void __launch_bounds__(256) ns_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                      const float* __restrict__ D, int n, float alpha, float beta,
                                                      float delta, float* __restrict__ C, const DeviceStatus* st,
                                                      const int* gate) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    // A tile: rows r0..r0+63, columns k0..k0+15 (stored transposed: As[k][r])
    for (int q = threadIdx.x; q < 64 * 16; q += 256) {
      const int r = q / 16, k = q % 16;
      const int gr = r0 + r, gk = k0 + k;
      As[k][r] = (gr < n && gk < n) ? A[(long long)gr * n + gk] : 0.f;
    }
    // B tile: op(B) rows k0..k0+15, columns c0..c0+63 (Bs[k][c])
    for (int q = threadIdx.x; q < 64 * 16; q += 256) {
      int k, cc;
      float v;
      if (BT) {   // op(B)[k][c] = B[c][k]
        cc = q / 16;
        k = q % 16;
        const int gc = c0 + cc, gk = k0 + k;
        v = (gc < n && gk < n) ? B[(long long)gc * n + gk] : 0.f;
      } else {
        k = q / 64;
        cc = q % 64;
        const int gc = c0 + cc, gk = k0 + k;
        v = (gc < n && gk < n) ? B[(long long)gk * n + gc] : 0.f;
      }
      Bs[k][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[k][ty + 16 * u];
        b[u] = Bs[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + ty + 16 * u, cc = c0 + tx + 16 * v;
      if (r < n && cc < n) {
        const long long o = (long long)r * n + cc;
        float x = alpha * acc[u][v];
        if (D) x = fmaf(beta, D[o], x);
        if (r == cc) x += delta;
        C[o] = x;
      }
    }
}

// ------------------------------------------------------------------------------------------
// 4. Z = Q Y = H_0 H_1 ... H_{n-2} Y: one warp per eigenvector (in shared memory), the
//    reflectors applied from the last to the first, RB of them staged in shared memory per
//    CTA barrier.  Z is written in FP64 (row i, column j = component i of vector j).
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void tri_back_kernel(const low_t<T>* __restrict__ W, const low_t<T>* __restrict__ tau,
                                const float* __restrict__ Yt, int n, int RB, T* __restrict__ Z,
                                const DeviceStatus* st, const int* gate) {
  using F = low_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  F* sy = (F*)smem_raw + (size_t)warp * n;          // this warp's vector
  F* sr = (F*)smem_raw + (size_t)nw * n;            // RB reflectors, RB x n
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const int j = blockIdx.x * nw + warp;
  if (j < n)
    for (int i = lane; i < n; i += 32) sy[i] = make_f<F>(Yt[(long long)j * n + i], 0.f);
  for (int kt = n - 2; kt >= 0; kt -= RB) {
    const int kb = max(0, kt - RB + 1);   // reflectors kb .. kt
    __syncthreads();
    for (int k = kb; k <= kt; ++k) {
      const int m = n - k - 1;
      for (int i = threadIdx.x; i < m; i += blockDim.x) sr[(size_t)(k - kb) * n + i] = W[(long long)k * n + k + 1 + i];
    }
    __syncthreads();
    if (j < n) {
      for (int k = kt; k >= kb; --k) {
        const F tk = tau[k];
        if (absx2(tk) == 0.f) continue;
        const int m = n - k - 1;
        const F* v = sr + (size_t)(k - kb) * n;
        F s = F{};
        for (int i = lane; i < m; i += 32) fma_conj(s, v[i], sy[k + 1 + i]);
        s = warp_sum(s);
        const F ts = -1.f * (tk * s);
        __syncwarp();
        for (int i = lane; i < m; i += 32) fma_plain(sy[k + 1 + i], ts, v[i]);
        __syncwarp();
      }
    }
  }
  if (j < n)
    for (int i = lane; i < n; i += 32) Z[(long long)i * n + j] = widen(sy[i]);
}

template <class T>
int eig32_impl(pawfd_ctx* c, int n, const T* A, T* Z, const int* gate) {
  using F = low_t<T>;
  cudaStream_t s = c->stream;
  char* base = (char*)c->d_eig;
  const size_t nn = (size_t)n * n;
  auto take = [&](size_t bytes) {
    char* p = base;
    base += (bytes + 255) / 256 * 256;
    return p;
  };
  F* W = (F*)take(nn * sizeof(F));
  float* Yt = (float*)take(nn * sizeof(float));
  float* Y2 = (float*)take(nn * sizeof(float));
  float* G = (float*)take(nn * sizeof(float));
  F* P = (F*)take((size_t)n * sizeof(F));
  F* tau = (F*)take((size_t)n * sizeof(F));
  float* d = (float*)take((size_t)n * sizeof(float));
  float* e = (float*)take((size_t)n * sizeof(float));
  float* lam = (float*)take((size_t)n * sizeof(float));
  int rc;
  // 1. reduction
  const size_t smem1 = 2 * (size_t)n * sizeof(F);
  if (smem1 > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(tridiag_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem1), "tridiag smem attribute");
    if (rc == PAWFD_OK)
      rc = check_cuda(c, cudaFuncSetAttribute(tridiag_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem1), "tridiag smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  // the shared-memory-resident form when the rows fit one cluster of TR_CTAS CTAs
  const int R = (n + 32 * TR_CTAS - 1) / (32 * TR_CTAS);
  const size_t smem_dsm = ((size_t)32 * R * n + 3 * (size_t)n) * sizeof(F);
  bool dsm = false;
  if (smem_dsm <= 220 * 1024 && c->tridiag_dsm) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(TR_CTAS);
    cfg.blockDim = dim3(TR_NT);
    cfg.dynamicSmemBytes = smem_dsm;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = TR_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaFuncSetAttribute(tridiag_dsm_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
        cudaFuncSetAttribute(tridiag_dsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dsm) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveClusters(&nclusters, tridiag_dsm_kernel<T>, &cfg) == cudaSuccess && nclusters >= 1) {
      rc = check_cuda(c, cudaLaunchKernelEx(&cfg, tridiag_dsm_kernel<T>, A, n, R, W, d, e, tau, gate),
                      "tridiag cluster launch");
      if (rc != PAWFD_OK) return rc;
      c->launches += 1;
      dsm = true;
    } else {
      cudaGetLastError();
    }
  }
  if (!dsm) {
    rc = launch_cluster_or_grid(c, tridiag_kernel<T, 1>, tridiag_kernel<T, 0>, TR_NT, smem1, TR_CTAS, true,
                                "tridiag launch", A, n, W, P, d, e, tau, c->d_barrier, c->d_status, gate);
    if (rc != PAWFD_OK) return rc;
  }
  // 2. eigenvalues
  const size_t smem2 = 2 * (size_t)n * sizeof(float);
  if (smem2 > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(tri_bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem2), "bisect smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  tri_bisect_kernel<<<(n + 7) / 8, 256, smem2, s>>>(d, e, n, lam, c->d_status, gate);
  // 3. eigenvectors of T
  const size_t smem3 = 5 * (size_t)n * sizeof(float) + (size_t)n;
  if (smem3 > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(tri_vectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem3), "vectors smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  tri_vectors_kernel<<<n, 32, smem3, s>>>(d, e, lam, n, Yt, c->d_status, gate);
  // 3b. three Newton-Schulz steps: G = Yt Yt^T; Yt <- 1.5 Yt - 0.5 G Yt (ping-pong Yt, Y2)
  {
    const dim3 g64((n + 63) / 64, (n + 63) / 64);
    float* cur = Yt;
    float* nxt = Y2;
    for (int it = 0; it < 3; ++it) {
      ns_gemm_kernel<true><<<g64, 256, 0, s>>>(cur, cur, nullptr, n, 1.f, 0.f, 0.f, G, c->d_status, gate);
      ns_gemm_kernel<false><<<g64, 256, 0, s>>>(G, cur, cur, n, -0.5f, 1.5f, 0.f, nxt, c->d_status, gate);
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
    Yt = cur;   // three steps: the result is in Y2
    c->launches += 6;
  }
  // 4. back-transformation: warps per CTA and reflectors per stage within 96 KB
  const size_t row = (size_t)n * sizeof(F);
  const int nw = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / row));
  const int RB = (int)std::max<size_t>(1, std::min<size_t>(16, (48 * 1024) / row));
  const size_t smem4 = (size_t)(nw + RB) * row;
  if (smem4 > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(tri_back_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem4), "back smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  tri_back_kernel<T><<<(n + nw - 1) / nw, 32 * nw, smem4, s>>>(W, tau, Yt, n, RB, Z, c->d_status, gate);
  c->launches += 3;
  return check_cuda(c, cudaGetLastError(), "eig32 launch");
}

}  // namespace

int launch_eig32(pawfd_ctx* c, int n, const double* A, double* Z, const int* gate) {
  return eig32_impl<double>(c, n, A, Z, gate);
}
int launch_eig32(pawfd_ctx* c, int n, const zd* A, zd* Z, const int* gate) {
  return eig32_impl<zd>(c, n, A, Z, gate);
}

}  // namespace pawfd
