// subspace.cu -- FP64 subspace diagonalization  H C = S C diag(eps)  on the device.
//
// The dense Cholesky + diagonalization of the band x band problem that the paper delegates
// to ScaLAPACK / ELPA or a single core (parallelization section), used by the subspace
// diagonalization of SCF step 1 (Kohn-Sham section).  Steps:
//   1. symmetrize H and S;
//   2. Cholesky S = L L^H (one CTA, right-looking, pivot <= 0 -> PAWFD_ENOTPD + column);
//   3. L^-1 by column-wise forward substitution (one CTA per column);
//   4. A = L^-1 H L^-H with two small GEMMs;
//   5. an FP32 eigendecomposition A ~= Z diag Z^H (tridiag.cu) refined in FP64 by two
//      Ogita-Aishima steps from X = Z; pairs of close eigenvalues the steps leave coupled go
//      to a parallel cyclic Jacobi on X^H A X (round-robin pair ordering: in each round n/2
//      disjoint rotations are applied at once, so every 2x2 block of A and every row pair of
//      V is updated independently; one grid-wide barrier per round, bounded in time; rounds
//      with no pair above the threshold are skipped);
//   6. stable ascending sort, C = L^-H U, phase fixing of each column.
// Bands that are already near the Ritz vectors (S_nm ~ I) skip steps 2-5: the Ogita-Aishima
// steps run on (H_nm, S_nm) from X = I.
#include <algorithm>
#include <cmath>

#include "device_sync.cuh"
#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

template <class T>
__global__ void symmetrize_kernel(const T* __restrict__ H, const T* __restrict__ S, int n, T* __restrict__ Hs,
                                  T* __restrict__ Ss) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const long long t = (long long)j * n + i;
  Hs[e] = 0.5 * (H[e] + conjx(H[t]));
  Ss[e] = 0.5 * (S[e] + conjx(S[t]));
}

// ------------------------------------------------------------------------------------------
// Blocked right-looking Cholesky S = L L^H of the lower triangle (in place; strict upper
// zeroed), Golub & Van Loan's outer-product form by panels of CH_NB columns:
//   (a) every CTA loads the panel's diagonal block and factors it with one warp in shared
//       memory (identical arithmetic in every CTA, so every CTA takes the same decision on a
//       pivot <= 0; CTA 0 writes the block back);
//   (b) the rows below solve x L11^H = a, one warp per row;
//   (c) the trailing lower triangle is updated, S22 -= L21 L21^H.
// Two all-CTA barriers per panel.
// ------------------------------------------------------------------------------------------
constexpr int CH_NB = 32;
constexpr int CH_NT = 512;

__device__ __forceinline__ double shfl_x(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ zd shfl_x(zd v, int src) {
  return zd{__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

template <class T, int MODE>
__global__ void __launch_bounds__(CH_NT) cholesky_kernel(T* __restrict__ S, int n, unsigned* bar, DeviceStatus* st,
                                                         const int* gate) {
  __shared__ T L11[CH_NB][CH_NB + 1];
  __shared__ double inv_d[CH_NB];
  __shared__ int s_fail;
  const unsigned G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gthreads = (int)G * CH_NT, gtid = (int)blockIdx.x * CH_NT + tid;
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;   // uniform: set before this launch
  for (int k0 = 0; k0 < n; k0 += CH_NB) {
    const int nb = min(CH_NB, n - k0);
    // (a) diagonal block
    for (int e = tid; e < nb * nb; e += CH_NT) L11[e / nb][e % nb] = ldcg(S + (long long)(k0 + e / nb) * n + k0 + e % nb);
    __syncthreads();
    if (warp == 0) {
      int fail = -1;
      for (int j = 0; j < nb; ++j) {
        const double d = realx(L11[j][j]);
        if (!(d > 0.0)) {
          fail = j;
          break;
        }
        const double ljj = sqrt(d), inv = 1.0 / ljj;
        __syncwarp();
        if (lane == j) {
          L11[j][j] = from_real<T>(ljj);
          inv_d[j] = inv;
        }
        if (lane > j && lane < nb) L11[lane][j] = inv * L11[lane][j];
        __syncwarp();
        if (lane > j && lane < nb) {
          const T lij = L11[lane][j];
          for (int k = j + 1; k <= lane; ++k) L11[lane][k] -= lij * conjx(L11[k][j]);
        }
        __syncwarp();
      }
      if (lane == 0) s_fail = fail;
    }
    __syncthreads();
    if (s_fail >= 0) {
      if (blockIdx.x == 0 && tid == 0) set_status(st, PAWFD_ENOTPD, k0 + s_fail);
      return;
    }
    // (b) rows below the block, one warp per row: x_j = (a_j - sum_{l<j} x_l conj(L_jl)) / L_jj
    const int m = n - k0 - nb;
    for (int r = (int)blockIdx.x * (CH_NT / 32) + warp; r < m; r += (int)G * (CH_NT / 32)) {
      const long long row = (long long)(k0 + nb + r) * n + k0;
      const T a = lane < nb ? ldcg(S + row + lane) : zero<T>();
      T sacc = zero<T>(), x = zero<T>();
      for (int j = 0; j < nb; ++j) {
        const T xj = shfl_x(inv_d[j] * (a - sacc), j);
        if (lane == j) x = xj;
        if (lane > j && lane < nb) sacc += xj * conjx(L11[lane][j]);
      }
      if (lane < nb) S[row + lane] = x;
    }
    if (!all_barrier<MODE>(bar, G, st, 700)) return;
    // every CTA has read the unfactored diagonal block: CTA 0 writes the factor back
    if (blockIdx.x == 0)
      for (int e = tid; e < nb * nb; e += CH_NT) {
        const int i = e / nb, k = e % nb;
        S[(long long)(k0 + i) * n + k0 + k] = k <= i ? L11[i][k] : zero<T>();
      }
    // (c) trailing lower triangle
    for (int e = gtid; e < m * m; e += gthreads) {
      const int r = e / m, q = e - r * m;
      if (q > r) continue;
      const long long i = k0 + nb + r, k = k0 + nb + q;
      T acc = ldcg(S + i * n + k);
      for (int j = 0; j < nb; ++j) acc -= ldcg(S + i * n + k0 + j) * conjx(ldcg(S + k * n + k0 + j));
      S[i * n + k] = acc;
    }
    if (!all_barrier<MODE>(bar, G, st, 701)) return;
  }
  for (int e = gtid; e < n * n; e += gthreads)
    if (e % n > e / n) S[e] = zero<T>();
}

// Linv column j = L^-1 e_j by forward substitution (one CTA per column).
template <class T>
__global__ void __launch_bounds__(256) tri_inverse_kernel(const T* __restrict__ L, int n, T* __restrict__ Linv,
                                                          const DeviceStatus* st, const int* gate) {
  extern __shared__ unsigned char smem_raw[];
  T* x = (T*)smem_raw;
  const int j = blockIdx.x, tid = threadIdx.x;
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  for (int k = tid; k < n; k += blockDim.x) x[k] = (k == j) ? from_real<T>(1.0) : zero<T>();
  for (int i = j; i < n; ++i) {
    __syncthreads();
    const T xi = (1.0 / realx(L[(long long)i * n + i])) * x[i];
    __syncthreads();
    if (tid == 0) x[i] = xi;
    for (int k = i + 1 + tid; k < n; k += blockDim.x) x[k] -= L[(long long)k * n + i] * xi;
  }
  __syncthreads();
  for (int k = tid; k < n; k += blockDim.x) Linv[(long long)k * n + j] = x[k];
}

// C = op(A) op(B) (+ D), n x n, op = identity or conjugate transpose.  With `skip` set on the
// device, C is a copy of `src` instead (the product is known to be that matrix).  `shape`
// skips the k-slabs that structure makes zero and, for a Hermitian product, half the tiles:
// SG_ALOW: op(A)[r][k] = 0 for k > r; SG_AUP: 0 for k < r; SG_BUP: op(B)[k][c] = 0 for k > c;
// SG_HERM: C is Hermitian, only tiles on or below the diagonal are computed and each entry
// below the diagonal is also stored, conjugated, above it.
enum { SG_ALOW = 1, SG_AUP = 2, SG_BUP = 4, SG_HERM = 8 };
template <class T>
__global__ void __launch_bounds__(256) small_gemm_kernel(const T* __restrict__ A, bool ha, const T* __restrict__ B,
                                                         bool hb, int n, T* __restrict__ C, const DeviceStatus* st,
                                                         const T* __restrict__ D = nullptr,
                                                         const int* skip = nullptr, const T* __restrict__ src = nullptr,
                                                         const int* gate = nullptr, int shape = 0) {
  __shared__ T As[16][17];
  __shared__ T Bs[16][17];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  if (skip && ld_volatile(skip)) {
    if (row < n && col < n) C[(long long)row * n + col] = src[(long long)row * n + col];
    return;
  }
  if ((shape & SG_HERM) && blockIdx.y < blockIdx.x) return;
  int kbeg = 0, kend = n;
  if (shape & SG_ALOW) kend = min(kend, (int)blockIdx.y * 16 + 16);
  if (shape & SG_AUP) kbeg = (int)blockIdx.y * 16;
  if (shape & SG_BUP) kend = min(kend, (int)blockIdx.x * 16 + 16);
  T acc = zero<T>();
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    {
      const int r = blockIdx.y * 16 + ty, k = k0 + tx;   // element (r, k) of op(A)
      T v = zero<T>();
      if (r < n && k < n) v = ha ? conjx(A[(long long)k * n + r]) : A[(long long)r * n + k];
      As[ty][tx] = v;
      const int kk = k0 + ty, cc = blockIdx.x * 16 + tx;  // element (kk, cc) of op(B)
      T w = zero<T>();
      if (kk < n && cc < n) w = hb ? conjx(B[(long long)cc * n + kk]) : B[(long long)kk * n + cc];
      Bs[ty][tx] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) fma_plain(acc, As[ty][k], Bs[k][tx]);
    __syncthreads();
  }
  if (row >= n || col >= n) return;
  if (shape & SG_HERM) {
    if (row < col) return;
    if (row == col) acc = from_real<T>(realx(acc));
    C[(long long)row * n + col] = acc;
    if (row != col) C[(long long)col * n + row] = conjx(acc);
    return;
  }
  C[(long long)row * n + col] = D ? acc + D[(long long)row * n + col] : acc;
}

template <class T>
__global__ void hermitize_kernel(T* __restrict__ A, int n, const DeviceStatus* st, const int* gate = nullptr) {
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (j < i) return;
  const long long t = (long long)j * n + i;
  const T v = 0.5 * (A[e] + conjx(A[t]));
  A[e] = v;
  A[t] = conjx(v);
}

struct Rot {
  double c, s;
  zd e;       // exp(-i phi) applied to column q (1 for real)
  int p, q;   // p < q; q == -1 marks an identity (pair with the padding index)
};

__device__ __forceinline__ double mul_e(double v, zd e) { return v * e.re; }
__device__ __forceinline__ zd mul_e(zd v, zd e) { return v * e; }
__device__ __forceinline__ double mul_ce(double v, zd e) { return v * e.re; }
__device__ __forceinline__ zd mul_ce(zd v, zd e) { return v * conjx(e); }
__device__ __forceinline__ zd phase_of(double apq, double mag) { return zd{apq / mag, 0.0}; }
__device__ __forceinline__ zd phase_of(zd apq, double mag) { return zd{apq.re / mag, -apq.im / mag}; }
__device__ __forceinline__ double absx(double x) { return fabs(x); }
__device__ __forceinline__ double absx(zd x) { return hypot(x.re, x.im); }

// Jacobi rotation of the pair (p, q) (p < q) that annihilates a_pq of a Hermitian matrix
template <class T>
__device__ __forceinline__ Rot make_rot(int p, int q, T apq, double app, double aqq) {
  Rot R;
  R.c = 1.0; R.s = 0.0; R.e = zd{1.0, 0.0}; R.p = p; R.q = q;
  const double mag = absx(apq);
  if (mag > 0.0) {
    const double tau = (aqq - app) / (2.0 * mag);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    R.c = 1.0 / sqrt(1.0 + t * t);
    R.s = t * R.c;
    R.e = phase_of(apq, mag);
  }
  return R;
}

// A'[P,Q] = J_P^H A[P,Q] J_Q on one 2x2 block with J = [[c, s], [-s e, c e]] on (p, q);
// a diagonal block (P == Q) comes out exactly diagonal with a real diagonal
template <class T>
__device__ __forceinline__ void rotate_block(const Rot& rp, const Rot& rq, bool diag, T& b00, T& b01, T& b10,
                                             T& b11) {
  if (rq.q >= 0) {
    const T x0 = rq.c * b00 - rq.s * mul_e(b01, rq.e);
    const T x1 = rq.s * b00 + rq.c * mul_e(b01, rq.e);
    const T y0 = rq.c * b10 - rq.s * mul_e(b11, rq.e);
    const T y1 = rq.s * b10 + rq.c * mul_e(b11, rq.e);
    b00 = x0; b01 = x1; b10 = y0; b11 = y1;
  }
  if (rp.q >= 0) {
    const T x0 = rp.c * b00 - rp.s * mul_ce(b10, rp.e);
    const T y0 = rp.s * b00 + rp.c * mul_ce(b10, rp.e);
    const T x1 = rp.c * b01 - rp.s * mul_ce(b11, rp.e);
    const T y1 = rp.s * b01 + rp.c * mul_ce(b11, rp.e);
    b00 = x0; b10 = y0; b01 = x1; b11 = y1;
  }
  if (diag && rp.q >= 0) {
    b01 = zero<T>();
    b10 = zero<T>();
    b00 = from_real<T>(realx(b00));
    b11 = from_real<T>(realx(b11));
  }
}

// player at position pos of round r of the circle (round-robin) schedule over npad players
__device__ __forceinline__ int rr_player(int pos, int r, int npad) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (npad - 1)) + 1;
}

__device__ double block_reduce_sum(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += s_red[w];
  return s;   // valid in thread 0
}

template <class T>
__global__ void identity_kernel(T* __restrict__ X, int n, const int* gate = nullptr) {
  if (gated(gate)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)n * n) X[e] = from_real<T>((e / n) == (e % n) ? 1.0 : 0.0);
}

// ---- Ogita-Aishima steps on many CTAs, for the generalized problem H x = lambda S x ----
// With an approximate basis X, A = X^H H X and B = X^H S X (B = null: B = I), the step of the
// single-CTA kernel above with R = I - B:  lambda_i = Re a_ii / Re b_ii,
//   e_ij = (a_ij + lambda_j r_ij) / (lambda_j - lambda_i)  off clusters, e_ij = r_ij / 2 on them,
// and X' = X + X E is S-orthonormal and diagonalizes H to second order.  Started from X = I
// (A = H_nm, B = S_nm), it replaces the Cholesky reduction when the bands are already close
// to the Ritz vectors (the iterated Rayleigh-Ritz step).

// Gate words of one subspace solve (oa_decide_kernel): a kernel given gate word g does nothing
// when flags[g] != 0.
// The far path's words: ZSKIP (the refinement from the FP32 basis Z), ZSTEP2 and ZSTEP3 (its
// second and third steps), ZFAIL (its fallback, the Jacobi sweeps from V = I), FAR_AM
// (X^H A X for the sweeps over coupled pairs), JACOBI_Z (the sweeps after refinement steps).
enum {
  GATE_NEAR = 0, GATE_FAR = 1, GATE_STEP2 = 2, GATE_AM = 3, GATE_JACOBI = 4, GATE_LAMBDA = 5,
  GATE_ZSKIP = 6, GATE_ZFAIL = 7, GATE_FAR_AM = 8, GATE_JACOBI_Z = 9, GATE_ZSTEP2 = 10, GATE_ZSTEP3 = 11
};

__device__ double block_reduce_max(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmax(m, s_red[w]);
  return m;   // valid in thread 0
}

// per-CTA partial sums of ||A - diag A||_F^2, ||A||_F^2, ||I - B||_F^2 into part[3 g + k], and
// lambda_i = Re a_ii / Re b_ii
template <class T>
__global__ void __launch_bounds__(256) oa_stats_kernel(const T* __restrict__ A, const T* __restrict__ B, int n,
                                                       double* __restrict__ part, double* __restrict__ lam,
                                                       const int* gate, const DeviceStatus* st) {
  __shared__ double s_red[32];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const long long nn = (long long)n * n;
  double off2 = 0.0, fro2 = 0.0, r2 = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const bool dg = (e / n) == (e % n);
    const double a2 = absx2(A[e]);
    fro2 += a2;
    if (!dg) off2 += a2;
    if (B) r2 += absx2(from_real<T>(dg ? 1.0 : 0.0) - B[e]);
  }
  off2 = block_reduce_sum(off2, s_red);
  if (threadIdx.x == 0) part[3 * blockIdx.x] = off2;
  fro2 = block_reduce_sum(fro2, s_red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 1] = fro2;
  r2 = block_reduce_sum(r2, s_red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 2] = r2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long d = (long long)i * n + i;
    lam[i] = realx(A[d]) / (B ? realx(B[d]) : 1.0);
  }
}

// E of one step (see above).  Pairs with |lambda_j - lambda_i| <= 1e-13 ||A||_F are a
// cluster; every other pair is corrected unless |e_ij| or |e_ji| would exceed sqrt(ebound2),
// in which case it is left to the Jacobi sweeps as well.  (Ogita and Aishima separate clusters
// by delta = 2 (||A - diag A|| + ||A|| ||R||); with Frobenius norms that bound sums the error of
// all n^2 entries and calls most pairs of a dense spectrum a cluster, so the bound on the
// corrections decides instead.)  Partials: part2[2 g] = pairs left coupled above the Jacobi
// threshold, part2[2 g + 1] = max |e_ij|^2.
template <class T>
__global__ void __launch_bounds__(256) oa_update_kernel(const T* __restrict__ A, const T* __restrict__ B, int n,
                                                        const double* __restrict__ lam, const double* __restrict__ part,
                                                        double tol, double ebound2,
                                                        T* __restrict__ E,
                                                        double* __restrict__ part2, const int* gate,
                                                        const DeviceStatus* st) {
  __shared__ double s_red[32];
  __shared__ double s_v[3];
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  if (threadIdx.x < 3) {   // the same sums, in the same order, in every CTA
    double v = 0.0;
    for (int g = 0; g < OA_G; ++g) v += part[3 * g + threadIdx.x];
    s_v[threadIdx.x] = v;
  }
  __syncthreads();
  const double fro2 = s_v[1];
  const double delta = 1e-13 * sqrt(fro2);
  const double thr2 = tol * tol * fro2 / ((double)n * n);
  const long long nn = (long long)n * n;
  double coupled = 0.0, emax2 = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const long long et = (long long)j * n + i;
    // the Hermitian parts of A and B (products X^H A X are Hermitian only up to rounding, and
    // e_ij + conj(e_ji) = r_ij holds exactly only for Hermitian inputs; otherwise the rounding
    // asymmetry, divided by a small gap, would spoil the orthogonality of X')
    const T a = 0.5 * (A[e] + conjx(A[et]));
    const T r = B ? from_real<T>(i == j ? 1.0 : 0.0) - 0.5 * (B[e] + conjx(B[et])) : zero<T>();
    T v = 0.5 * r;
    if (i != j) {
      const double li = lam[i], lj = lam[j];
      bool cluster = fabs(lj - li) <= delta;
      if (!cluster) {
        const T w = (1.0 / (lj - li)) * (a + lj * r);
        // the pair (j, i) makes the same decision: both corrections within the bound
        const T wt = (1.0 / (li - lj)) * (conjx(a) + li * conjx(r));
        if (absx2(w) <= ebound2 && absx2(wt) <= ebound2) v = w;
        else cluster = true;
      }
      if (cluster && absx2(a) > thr2) coupled += 1.0;
    }
    emax2 = fmax(emax2, absx2(v));
    E[e] = v;
  }
  coupled = block_reduce_sum(coupled, s_red);
  if (threadIdx.x == 0) part2[2 * blockIdx.x] = coupled;
  emax2 = block_reduce_max(emax2, s_red);
  if (threadIdx.x == 0) part2[2 * blockIdx.x + 1] = emax2;
}

// Path decision from the first step started at X = I (A = H_nm, B = S_nm): the near path when
// ||I - S_nm||_F <= 1e-4 and at most 2 n pairs are left coupled.  One step suffices when
// every |e_ij| <= 1e-8 (the error left is of its square); with no coupled pair either, the
// Jacobi sweeps are not needed and the eigenvalues are the lambda_i.
__global__ void oa_decide_kernel(const double* __restrict__ part, const double* __restrict__ part2, int n,
                                 int* __restrict__ flags) {
  if (threadIdx.x != 0) return;
  double r2 = 0.0, coupled = 0.0, emax2 = 0.0;
  for (int g = 0; g < OA_G; ++g) {
    r2 += part[3 * g + 2];
    coupled += part2[2 * g];
    emax2 = fmax(emax2, part2[2 * g + 1]);
  }
  const bool near = r2 <= 1e-8 && coupled <= 2.0 * n;
  const bool one = emax2 <= 1e-16;
  const bool nojac = one && coupled == 0.0;
  flags[GATE_NEAR] = near;
  flags[GATE_FAR] = !near;
  flags[GATE_STEP2] = !near || one;
  flags[GATE_AM] = !near || nojac;
  flags[GATE_JACOBI] = 1;
  flags[GATE_LAMBDA] = !(near && nojac);
  flags[GATE_ZSKIP] = near;
  flags[GATE_ZFAIL] = 1;
  flags[GATE_FAR_AM] = 1;
  flags[GATE_JACOBI_Z] = !near || nojac;
  flags[GATE_ZSTEP2] = 1;
  flags[GATE_ZSTEP3] = 1;
}

// Far path, after the first Ogita-Aishima step from the FP32 basis Z: Z is taken when the
// norms are finite and ||I - Z^H Z||_F <= 1e-2; otherwise the Jacobi sweeps diagonalize A
// from V = I.
__global__ void far_decide1_kernel(const double* __restrict__ part, int* __restrict__ flags, const int* gate) {
  if (threadIdx.x != 0 || gated(gate)) return;
  double r2 = 0.0, fro2 = 0.0;
  for (int g = 0; g < OA_G; ++g) {
    fro2 += part[3 * g + 1];
    r2 += part[3 * g + 2];
  }
  const bool ok = isfinite(r2) && isfinite(fro2) && r2 <= 1e-4;
  flags[GATE_ZSKIP] = !ok;
  flags[GATE_ZSTEP2] = !ok;
  flags[GATE_ZSTEP3] = 1;
  flags[GATE_ZFAIL] = ok;
  flags[GATE_JACOBI] = ok;
  flags[GATE_JACOBI_Z] = 1;
  flags[GATE_LAMBDA] = 1;
  flags[GATE_FAR_AM] = 1;
}

// Far path, after refinement step 2 (last = 0) or 3 (last = 1): with every |e_ij| <= 1e-8
// and no pair coupled, the step's basis is the eigenbasis to FP64 precision (the error left is
// of the order of |e|^2) and the eigenvalues are the step's lambda_i; otherwise, after step 2
// the third step runs, after step 3 the Jacobi sweeps run on X^H A X.
__global__ void far_decide_kernel(const double* __restrict__ part2, int last, int* __restrict__ flags,
                                  const int* gate) {
  if (threadIdx.x != 0 || gated(gate)) return;
  double coupled = 0.0, emax2 = 0.0;
  for (int g = 0; g < OA_G; ++g) {
    coupled += part2[2 * g];
    emax2 = fmax(emax2, part2[2 * g + 1]);
  }
  const bool done = emax2 <= 1e-16 && coupled == 0.0;
  if (!last && !done) {
    flags[GATE_ZSTEP3] = 0;
    return;
  }
  flags[GATE_JACOBI_Z] = done;
  flags[GATE_LAMBDA] = !done;
  flags[GATE_FAR_AM] = done;
}

// After the second step of the near path: when it left every |e_ij| <= 1e-8 and no pair
// coupled, X2 = X1 (I + E2) is the eigenvector basis to FP64 precision (the error left is of
// the order of |e|^2), so A = X2^H H X2 and the Jacobi sweeps are skipped and the eigenvalues
// are the step's lambda_i (Rayleigh quotients of X1, within |e|^2 of those of X2).
__global__ void oa_decide2_kernel(const double* __restrict__ part2, int* __restrict__ flags, const int* gate) {
  if (threadIdx.x != 0 || gated(gate)) return;
  double coupled = 0.0, emax2 = 0.0;
  for (int g = 0; g < OA_G; ++g) {
    coupled += part2[2 * g];
    emax2 = fmax(emax2, part2[2 * g + 1]);
  }
  if (emax2 <= 1e-16 && coupled == 0.0) {
    flags[GATE_AM] = 1;
    flags[GATE_JACOBI_Z] = 1;
    flags[GATE_LAMBDA] = 0;
  }
}

// X = I + E
template <class T>
__global__ void identity_plus_kernel(const T* __restrict__ E, int n, T* __restrict__ X, const int* gate,
                                     const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (long long)n * n) X[e] = E[e] + from_real<T>((e / n) == (e % n) ? 1.0 : 0.0);
}

template <class T>
__global__ void copy_kernel(const T* __restrict__ src, long long count, T* __restrict__ dst, const int* gate,
                            const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) dst[e] = src[e];
}

// the diagonal of A from lambda (the sort reads only the diagonal)
template <class T>
__global__ void lambda_diag_kernel(const double* __restrict__ lam, int n, T* __restrict__ A, const int* gate,
                                   const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(long long)i * n + i] = from_real<T>(lam[i]);
}

// sum over all CTAs of per-CTA partials, identical (same order) in every CTA
template <int MODE>
__device__ double grid_sum(double mine, double* red, double* s_red, double* s_bcast, unsigned* bar, unsigned G,
                           DeviceStatus* st, int id, bool* ok) {
  const double b = block_reduce_sum(mine, s_red);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!all_barrier<MODE>(bar, G, st, id)) {
    *ok = false;
    return 0.0;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (unsigned g = 0; g < G; ++g) s += __ldcg(red + g);
    *s_bcast = s;
  }
  __syncthreads();
  const double s = *s_bcast;
  // everyone has read red[] before anyone may overwrite it in the next reduction
  if (!all_barrier<MODE>(bar, G, st, id + 1)) *ok = false;
  return s;
}

template <class T, int MODE>
__global__ void __launch_bounds__(MODE == 1 ? 1024 : 256)
    jacobi_kernel(T* __restrict__ A0, T* __restrict__ A1, T* __restrict__ V, int n, double tol, int max_sweeps,
                  unsigned* bar, DeviceStatus* st, double* red, const int* gate) {
  // V holds the caller's starting basis; the rotations accumulate onto it
  extern __shared__ unsigned char smem_raw[];
  Rot* rot = (Rot*)smem_raw;
  __shared__ double s_red[32];
  __shared__ double s_bcast;
  const unsigned G = gridDim.x;
  const int npad = n + (n & 1);
  const int np = npad / 2;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gthreads = (long long)G * blockDim.x;
  bool ok = true;
  // Each round reads the rotation parameters and the 2x2 blocks from A and writes the
  // rotated blocks to the other buffer, so no CTA can see a half-updated round.
  T* A = A0;
  T* Anext = A1;
  if (ld_volatile(&st->code) != 0 || gated(gate)) return;   // an earlier step failed, or no sweeps needed


  double fro2 = 0.0;
  for (long long e = gtid; e < (long long)n * n; e += gthreads) fro2 += absx2(ldcg(A + e));
  fro2 = grid_sum<MODE>(fro2, red, s_red, &s_bcast, bar, G, st, 1, &ok);
  if (!ok) return;
  const double limit2 = tol * tol * fro2;

  // Threshold Jacobi: a pair is rotated only if |a_pq|^2 > thr2 (all off-diagonal entries at
  // that level would add up to the convergence limit), and a round whose pairs all fall below
  // it at the start of the sweep is skipped without a barrier.
  // The flags alternate between two arrays by sweep: a CTA may still read the flags of the
  // last rounds of sweep s while another clears those of sweep s + 1 (no barrier between them).
  const double thr2 = limit2 / ((double)n * n);
  for (int sweep = 0;; ++sweep) {
    unsigned* rflag = (unsigned*)(red + 2048) + (sweep & 1) * 3072;
    for (long long e = gtid; e < npad - 1; e += gthreads) rflag[e] = 0u;
    double off2 = 0.0;
    for (long long e = gtid; e < (long long)n * n; e += gthreads)
      if ((e / n) != (e % n)) off2 += absx2(ldcg(A + e));
    off2 = grid_sum<MODE>(off2, red, s_red, &s_bcast, bar, G, st, 3, &ok);
    if (!ok) return;
    if (off2 <= limit2 || sweep == max_sweeps) {
      if (off2 > limit2 && blockIdx.x == 0 && threadIdx.x == 0) set_status(st, PAWFD_ENOCONV, max_sweeps);
      if (A != A0)
        for (long long e = gtid; e < (long long)n * n; e += gthreads) A0[e] = ldcg(A + e);
      return;
    }
    for (long long w = gtid; w < (long long)(npad - 1) * np; w += gthreads) {
      const int r = (int)(w / np), k = (int)(w % np);
      int p = rr_player(k, r, npad), q = rr_player(npad - 1 - k, r, npad);
      if (p > q) { const int t = p; p = q; q = t; }
      if (q < n && absx2(ldcg(A + (long long)p * n + q)) > thr2) rflag[r] = 1u;
    }
    if (!all_barrier<MODE>(bar, G, st, 5)) return;
    for (int r = 0; r < npad - 1; ++r) {
      if (__ldcg(rflag + r) == 0u) continue;   // identical in every CTA
      // rotation parameters of this round's n/2 disjoint pairs, computed by every CTA
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int p = rr_player(k, r, npad), q = rr_player(npad - 1 - k, r, npad);
        if (p > q) { const int t = p; p = q; q = t; }
        Rot R;
        const T apq = q < n ? ldcg(A + (long long)p * n + q) : zero<T>();
        if (q >= n) {
          R.c = 1.0; R.s = 0.0; R.e = zd{1.0, 0.0}; R.p = p; R.q = -1;
        } else if (absx2(apq) <= thr2) {
          R.c = 1.0; R.s = 0.0; R.e = zd{1.0, 0.0}; R.p = p; R.q = q;
        } else {
          R = make_rot<T>(p, q, apq, realx(ldcg(A + (long long)p * n + p)), realx(ldcg(A + (long long)q * n + q)));
        }
        rot[k] = R;
      }
      __syncthreads();
      // 2x2 blocks: A'[P,Q] = J_P^H A[P,Q] J_Q with J = [[c, s], [-s e, c e]] on (p, q)
      for (long long w = gtid; w < (long long)np * np; w += gthreads) {
        const int P = (int)(w / np), Q = (int)(w % np);
        const Rot rp = rot[P], rq = rot[Q];
        const int i0 = rp.p, i1 = rp.q, j0 = rq.p, j1 = rq.q;
        T b00 = ldcg(A + (long long)i0 * n + j0);
        T b01 = j1 >= 0 ? ldcg(A + (long long)i0 * n + j1) : zero<T>();
        T b10 = i1 >= 0 ? ldcg(A + (long long)i1 * n + j0) : zero<T>();
        T b11 = (i1 >= 0 && j1 >= 0) ? ldcg(A + (long long)i1 * n + j1) : zero<T>();
        rotate_block<T>(rp, rq, P == Q, b00, b01, b10, b11);
        Anext[(long long)i0 * n + j0] = b00;
        if (j1 >= 0) Anext[(long long)i0 * n + j1] = b01;
        if (i1 >= 0) Anext[(long long)i1 * n + j0] = b10;
        if (i1 >= 0 && j1 >= 0) Anext[(long long)i1 * n + j1] = b11;
      }
      // V' = V J
      for (long long w = gtid; w < (long long)n * np; w += gthreads) {
        const int row = (int)(w / np), Q = (int)(w % np);
        const Rot rq = rot[Q];
        if (rq.q < 0) continue;
        const T v0 = ldcg(V + (long long)row * n + rq.p), v1 = ldcg(V + (long long)row * n + rq.q);
        V[(long long)row * n + rq.p] = rq.c * v0 - rq.s * mul_e(v1, rq.e);
        V[(long long)row * n + rq.q] = rq.s * v0 + rq.c * mul_e(v1, rq.e);
      }
      if (!all_barrier<MODE>(bar, G, st, 100 + r)) return;
      T* t = A; A = Anext; Anext = t;
    }
  }
}

// eps[rank(i)] = A[i][i] with ranks ascending, stable; U[:, rank(i)] = V[:, i]
template <class T>
__global__ void sort_kernel(const T* __restrict__ A, const T* __restrict__ V, int n, double* __restrict__ eps,
                            T* __restrict__ U, const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0) return;
  const int i = blockIdx.x;
  const double li = realx(A[(long long)i * n + i]);
  __shared__ int s_rank;
  if (threadIdx.x == 0) s_rank = 0;
  __syncthreads();
  int cnt = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double lj = realx(A[(long long)j * n + j]);
    if (lj < li || (lj == li && j < i)) ++cnt;
  }
  atomicAdd(&s_rank, cnt);
  __syncthreads();
  const int rk = s_rank;
  if (threadIdx.x == 0) eps[rk] = li;
  for (int r = threadIdx.x; r < n; r += blockDim.x) U[(long long)r * n + rk] = V[(long long)r * n + i];
}

// multiply column m by conj(x)/|x|, x its largest-magnitude entry (first on ties)
template <class T>
__global__ void phase_fix_kernel(T* __restrict__ C, int n, const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0) return;
  const int m = blockIdx.x;
  __shared__ double s_mag[256];
  __shared__ int s_idx[256];
  double best = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double mag = absx2(C[(long long)i * n + m]);
    if (mag > best) { best = mag; bi = i; }
  }
  s_mag[threadIdx.x] = best;
  s_idx[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double m2 = s_mag[threadIdx.x + o];
      const int i2 = s_idx[threadIdx.x + o];
      if (m2 > s_mag[threadIdx.x] || (m2 == s_mag[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
        s_mag[threadIdx.x] = m2;
        s_idx[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const T x = C[(long long)s_idx[0] * n + m];
  const double mag = sqrt(absx2(x));
  if (!(mag > 0.0)) return;
  const T f = (1.0 / mag) * conjx(x);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long e = (long long)i * n + m;
    if (i == s_idx[0]) C[e] = from_real<T>(mag);
    else C[e] = C[e] * f;
  }
}

// Jacobi on A (n x n, in place) accumulating V.  When one round's 2x2 blocks fit the threads
// of one thread-block cluster, the kernel runs as a single cluster and every round ends on a
// hardware cluster barrier; otherwise as a cooperative grid with a software grid barrier.
template <class T>
int launch_jacobi(pawfd_ctx* c, int n, T* Am, T* A2, T* Vm, const int* gate, double tol) {
  cudaStream_t s = c->stream;
  const int npad = n + (n & 1), np = npad / 2;
  const size_t rot_bytes = sizeof(Rot) * np;
  int max_sweeps = 60;
  unsigned* bar = c->d_barrier;
  DeviceStatus* st = c->d_status;
  double* red = c->d_reduce;
  int rc;
  const long long blocks = (long long)np * np;
  if (c->jacobi_cluster && blocks <= 16ll * 1024 * 2) {
    // one cluster of G CTAs x 1024 threads, G <= 16 (non-portable sizes above 8 when allowed)
    int G = (int)std::max(1ll, std::min<long long>(16, (blocks + 1023) / 1024));
    if (rot_bytes > 48 * 1024) {
      rc = check_cuda(c, cudaFuncSetAttribute(jacobi_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)rot_bytes), "jacobi smem attribute");
      if (rc != PAWFD_OK) return rc;
    }
    if (G > 8) {
      if (cudaFuncSetAttribute(jacobi_kernel<T, 1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
        cudaGetLastError();
        G = 8;
      }
    }
    for (;; G /= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(G);
      cfg.blockDim = dim3(1024);
      cfg.dynamicSmemBytes = rot_bytes;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = G;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_kernel<T, 1>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nclusters = 0;
      }
      if (nclusters >= 1) {
        rc = check_cuda(c, cudaLaunchKernelEx(&cfg, jacobi_kernel<T, 1>, Am, A2, Vm, n, tol, max_sweeps, bar, st, red,
                                              gate),
                        "jacobi cluster launch");
        c->launches += 1;
        return rc;
      }
      if (G == 1) break;
    }
  }
  // cooperative grid sized to the work of one round and to co-residency
  if (rot_bytes > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(jacobi_kernel<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)rot_bytes), "jacobi smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  int per_sm = 0;
  rc = check_cuda(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<T, 0>, 256, rot_bytes),
                  "occupancy");
  if (rc != PAWFD_OK) return rc;
  long long want = (blocks + 255) / 256;
  int G = (int)std::max(1ll, std::min<long long>(want, (long long)per_sm * c->num_sms));
  G = std::min(G, 2048);   // grid_sum partials live in red[0, 2048)
  rc = check_cuda(c, cudaMemsetAsync(c->d_barrier, 0, 2 * sizeof(unsigned), s), "barrier reset");
  if (rc != PAWFD_OK) return rc;
  void* args[] = {&Am, &A2, &Vm, &n, &tol, &max_sweeps, &bar, &st, &red, &gate};
  rc = check_cuda(c, cudaLaunchCooperativeKernel((const void*)jacobi_kernel<T, 0>, dim3(G), dim3(256), args,
                                                 rot_bytes, s),
                  "jacobi cooperative launch");
  c->launches += 1;
  return rc;
}

template <class T>
int subspace_impl(pawfd_ctx* c, int n, T* H, T* S, double* eps, T* C) {
  const long long nn = (long long)n * n;
  T* W = (T*)c->d_work;
  T* Hs = W;            // symmetrized H
  T* Lm = W + nn;       // symmetrized S; far path: then L
  T* Li = W + 2 * nn;   // far path: L^-1; near path: E of the first step (and of the second)
  T* T1 = W + 3 * nn;   // products, later U
  T* Am = W + 4 * nn;   // the matrix of the Jacobi sweeps, diagonalized in place
  T* Vm = W + 5 * nn;   // the basis X the rotations accumulate onto
  T* A2 = W + 6 * nn;   // second Jacobi buffer; near path: X^H H X of the second step
  cudaStream_t s = c->stream;
  const DeviceStatus* st = c->d_status;
  const int* flags = c->d_flags;
  const int* near = flags + GATE_NEAR;      // far-path kernels: skipped on the near path
  const int* far = flags + GATE_FAR;        // near-path kernels: skipped on the far path
  double* part = c->d_oa;                   // [3 OA_G] norms
  double* part2 = c->d_oa + 3 * OA_G;       // [2 OA_G] coupled pairs, max |e|^2
  double* lam = c->d_oa + 5 * OA_G;         // [n]
  const double tol = 1e-14;     // the sweeps from V = I (far-path fallback)
  // the sweeps after Ogita-Aishima steps: threshold 1e-12 ||A||_F / n, above the FP64 rounding
  // of the X^H A X they run on
  const double tol_z = 1e-12;
  const unsigned eb = (unsigned)((nn + 255) / 256);
  const dim3 gg((n + 15) / 16, (n + 15) / 16);
  symmetrize_kernel<T><<<eb, 256, 0, s>>>(H, S, n, Hs, Lm);
  // the first Ogita-Aishima step from X = I on (H, S), and the path decision
  oa_stats_kernel<T><<<OA_G, 256, 0, s>>>(Hs, Lm, n, part, lam, nullptr, st);
  oa_update_kernel<T><<<OA_G, 256, 0, s>>>(Hs, Lm, n, lam, part, tol_z, 1e-8, Li, part2, nullptr, st);
  oa_decide_kernel<<<1, 32, 0, s>>>(part, part2, n, c->d_flags);
  c->launches += 4;
  int rc = check_cuda(c, cudaGetLastError(), "subspace launch");
  if (rc != PAWFD_OK) return rc;

  // ---- far path: Cholesky S = L L^H, A = L^-1 H L^-H, its FP32 eigenbasis refined in FP64 ----
  // Cholesky: one cluster up to n = 256 (its flops fit 16 SMs), the whole GPU above
  {
    unsigned* bar = c->d_barrier;
    DeviceStatus* stw = c->d_status;
    const int want = n <= 256 ? 16 : c->num_sms;
    rc = launch_cluster_or_grid(c, cholesky_kernel<T, 1>, cholesky_kernel<T, 0>, CH_NT, 0, want, c->jacobi_cluster,
                                "cholesky launch", Lm, n, bar, stw, near);
    if (rc != PAWFD_OK) return rc;
  }
  tri_inverse_kernel<T><<<n, 256, sizeof(T) * n, s>>>(Lm, n, Li, st, near);
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(Li, false, Hs, false, n, T1, st, nullptr, nullptr, nullptr, near, SG_ALOW);
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(T1, false, Li, true, n, Am, st, nullptr, nullptr, nullptr, near,
                                          SG_BUP | SG_HERM);
  hermitize_kernel<T><<<eb, 256, 0, s>>>(Am, n, st, near);
  c->launches += 4;
  rc = check_cuda(c, cudaGetLastError(), "subspace launch");
  if (rc != PAWFD_OK) return rc;
  // FP32 eigendecomposition A ~= Z diag Z^H (tridiag.cu), then Ogita-Aishima steps in FP64
  // from X0 = Z: X_k = X_{k-1} (I + E_k), taking corrections up to 1e-2, 1e-4 and 1e-7 (each
  // step squares the error of the last; the first bound is wide because the FP32 basis couples
  // neighbours of a dense spectrum by about eps_32 ||A|| / gap); the third step runs only when
  // the second left a correction above 1e-8 or a coupled pair.  Pairs still coupled (close
  // eigenvalues) go to the Jacobi sweeps on X^H A X (threshold 1e-12 ||A||_F / n: the FP64
  // rounding of X^H A X stays below it); an unusable Z sends A to the sweeps from V = I.
  {
    const int* fam = flags + GATE_FAR_AM;
    rc = launch_eig32(c, n, Am, Vm, near);
    if (rc != PAWFD_OK) return rc;
    // one step from P: A P (Hs), S = P^H A P (Lm), B = P^H P (A2), E (Hs); then P + P E
    auto oa_step = [&](T* P, double ebound2, const int* gate) {
      small_gemm_kernel<T><<<gg, 256, 0, s>>>(Am, false, P, false, n, Hs, st, nullptr, nullptr, nullptr, gate);
      small_gemm_kernel<T><<<gg, 256, 0, s>>>(P, true, Hs, false, n, Lm, st, nullptr, nullptr, nullptr, gate, SG_HERM);
      small_gemm_kernel<T><<<gg, 256, 0, s>>>(P, true, P, false, n, A2, st, nullptr, nullptr, nullptr, gate, SG_HERM);
      oa_stats_kernel<T><<<OA_G, 256, 0, s>>>(Lm, A2, n, part, lam, gate, st);
      oa_update_kernel<T><<<OA_G, 256, 0, s>>>(Lm, A2, n, lam, part, tol_z, ebound2, Hs, part2, gate, st);
    };
    oa_step(Vm, 1e-4, near);
    far_decide1_kernel<<<1, 32, 0, s>>>(part, c->d_flags, near);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, false, Hs, false, n, T1, st, Vm, nullptr, nullptr,
                                            flags + GATE_ZSKIP);
    oa_step(T1, 1e-8, flags + GATE_ZSTEP2);
    far_decide_kernel<<<1, 32, 0, s>>>(part2, 0, c->d_flags, flags + GATE_ZSTEP2);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(T1, false, Hs, false, n, Vm, st, T1, nullptr, nullptr,
                                            flags + GATE_ZSTEP2);
    oa_step(Vm, 1e-14, flags + GATE_ZSTEP3);
    far_decide_kernel<<<1, 32, 0, s>>>(part2, 1, c->d_flags, flags + GATE_ZSTEP3);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, false, Hs, false, n, T1, st, Vm, nullptr, nullptr,
                                            flags + GATE_ZSTEP3);
    copy_kernel<T><<<eb, 256, 0, s>>>(T1, nn, Vm, flags + GATE_ZSTEP3, st);
    // A <- X^H A X for the sweeps over the coupled pairs
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Am, false, Vm, false, n, T1, st, nullptr, nullptr, nullptr, fam);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, true, T1, false, n, Am, st, nullptr, nullptr, nullptr, fam, SG_HERM);
    hermitize_kernel<T><<<eb, 256, 0, s>>>(Am, n, st, fam);
    // the fallback: the sweeps on A from V = I
    identity_kernel<T><<<eb, 256, 0, s>>>(Vm, n, flags + GATE_ZFAIL);
    c->launches += 30;
    rc = check_cuda(c, cudaGetLastError(), "far-path refinement");
    if (rc != PAWFD_OK) return rc;
  }

  // ---- near path: X1 = I + E1; a second step unless the first left |e| <= 1e-8; A = X^H H X
  // for the Jacobi sweeps unless a step left every |e| <= 1e-8 and no pair coupled (then the
  // eigenvalues are that step's lambda) ----
  {
    const int* step2 = flags + GATE_STEP2;
    const int* amg = flags + GATE_AM;
    identity_plus_kernel<T><<<eb, 256, 0, s>>>(Li, n, Vm, far, st);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Hs, false, Vm, false, n, T1, st, nullptr, nullptr, nullptr, step2);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, true, T1, false, n, A2, st, nullptr, nullptr, nullptr, step2, SG_HERM);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Lm, false, Vm, false, n, T1, st, nullptr, nullptr, nullptr, step2);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, true, T1, false, n, Am, st, nullptr, nullptr, nullptr, step2, SG_HERM);
    oa_stats_kernel<T><<<OA_G, 256, 0, s>>>(A2, Am, n, part, lam, step2, st);
    oa_update_kernel<T><<<OA_G, 256, 0, s>>>(A2, Am, n, lam, part, tol_z, 1e-14, Li, part2, step2, st);
    oa_decide2_kernel<<<1, 32, 0, s>>>(part2, c->d_flags, step2);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, false, Li, false, n, T1, st, Vm, nullptr, nullptr, step2);
    copy_kernel<T><<<eb, 256, 0, s>>>(T1, nn, Vm, step2, st);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Hs, false, Vm, false, n, T1, st, nullptr, nullptr, nullptr, amg);
    small_gemm_kernel<T><<<gg, 256, 0, s>>>(Vm, true, T1, false, n, Am, st, nullptr, nullptr, nullptr, amg, SG_HERM);
    hermitize_kernel<T><<<eb, 256, 0, s>>>(Am, n, st, amg);
    lambda_diag_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(lam, n, Am, flags + GATE_LAMBDA, st);
    c->launches += 14;
    rc = check_cuda(c, cudaGetLastError(), "near-path launch");
    if (rc != PAWFD_OK) return rc;
  }
  rc = launch_jacobi<T>(c, n, Am, A2, Vm, flags + GATE_JACOBI, tol);
  if (rc != PAWFD_OK) return rc;
  rc = launch_jacobi<T>(c, n, Am, A2, Vm, flags + GATE_JACOBI_Z, 1e-12);
  if (rc != PAWFD_OK) return rc;
  sort_kernel<T><<<n, 128, 0, s>>>(Am, Vm, n, eps, T1, c->d_status);
  // C = L^-H U (far path) or U (near path: a copy)
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(Li, true, T1, false, n, C, st, nullptr, near, T1, nullptr, SG_AUP);
  phase_fix_kernel<T><<<n, 256, 0, s>>>(C, n, c->d_status);
  c->launches += 3;
  return check_cuda(c, cudaGetLastError(), "subspace launch");
}

}  // namespace

int launch_subspace_diag(pawfd_ctx* c, int nb, void* Hnm, void* Snm, double* eps, void* C) {
  if (nb > 3072) return fail(c, PAWFD_EINVAL, "subspace_diag supports at most 3072 bands");
  if (is_complex(c)) return subspace_impl<zd>(c, nb, (zd*)Hnm, (zd*)Snm, eps, (zd*)C);
  return subspace_impl<double>(c, nb, (double*)Hnm, (double*)Snm, eps, (double*)C);
}

}  // namespace pawfd
