// subspace.cu -- FP64 subspace diagonalization  H C = S C diag(eps)  on the device.
//
// The dense Cholesky + diagonalization of the band x band problem that the paper delegates
// to ScaLAPACK / ELPA or a single core (parallelization section), used by the subspace
// diagonalization of SCF step 1 (Kohn-Sham section).  Steps:
//   1. symmetrize H and S;
//   2. Cholesky S = L L^H (one CTA, right-looking, pivot <= 0 -> PAWFD_ENOTPD + column);
//   3. L^-1 by column-wise forward substitution (one CTA per column);
//   4. A = L^-1 H L^-H with two small GEMMs;
//   5. parallel cyclic Jacobi on A (round-robin pair ordering: in each round n/2 disjoint
//      rotations are applied at once, so every 2x2 block of A and every row pair of V is
//      updated independently; one grid-wide barrier per round, bounded in time);
//   6. stable ascending sort, C = L^-H U, phase fixing of each column.
#include <algorithm>
#include <cmath>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr long long BARRIER_TIMEOUT_NS = 2000000000ll;   // a grid barrier gives up after 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(const volatile unsigned*)p; }
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  bar[0] counts
// arrivals, bar[1] is the generation.  The wait is bounded: after BARRIER_TIMEOUT_NS the
// CTA records PAWFD_ETIMEDOUT and every CTA stops at its next barrier.  Returns false if
// the kernel must stop.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, DeviceStatus* st, int id) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_volatile(&bar[1]);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_volatile(&bar[1]) == gen) {
        if (global_ns() - t0 > (unsigned long long)BARRIER_TIMEOUT_NS) {
          set_status(st, PAWFD_ETIMEDOUT, id);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (ld_volatile(&st->code) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// L2-only loads: data written by other CTAs of the same launch must not come from a stale L1
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zd ldcg(const zd* p) {
  const double2 v = __ldcg((const double2*)p);
  return zd{v.x, v.y};
}

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

// Right-looking Cholesky of the lower triangle of S (in place, one CTA).  Strict upper zeroed.
template <class T>
__global__ void __launch_bounds__(1024) cholesky_kernel(T* __restrict__ S, int n, DeviceStatus* st) {
  __shared__ int s_fail;
  __shared__ double s_ljj;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = realx(S[(long long)j * n + j]);
      if (!(d > 0.0)) {
        s_fail = 1;
        set_status(st, PAWFD_ENOTPD, j);
      } else {
        s_ljj = sqrt(d);
        S[(long long)j * n + j] = from_real<T>(s_ljj);
      }
    }
    __syncthreads();
    if (s_fail) return;
    const double inv = 1.0 / s_ljj;
    for (int i = j + 1 + tid; i < n; i += nt) S[(long long)i * n + j] = inv * S[(long long)i * n + j];
    __syncthreads();
    const int m = n - j - 1;
    for (long long e = tid; e < (long long)m * m; e += nt) {
      const int r = (int)(e / m), q = (int)(e % m);
      if (q > r) continue;
      const int i = j + 1 + r, k = j + 1 + q;
      T v = S[(long long)i * n + k];
      const T lij = S[(long long)i * n + j], lkj = S[(long long)k * n + j];
      v -= lij * conjx(lkj);
      S[(long long)i * n + k] = v;
    }
    __syncthreads();
  }
  for (long long e = tid; e < (long long)n * n; e += nt) {
    const int i = (int)(e / n), k = (int)(e % n);
    if (k > i) S[e] = zero<T>();
  }
}

// Linv column j = L^-1 e_j by forward substitution (one CTA per column).
template <class T>
__global__ void __launch_bounds__(256) tri_inverse_kernel(const T* __restrict__ L, int n, T* __restrict__ Linv,
                                                          const DeviceStatus* st) {
  extern __shared__ unsigned char smem_raw[];
  T* x = (T*)smem_raw;
  const int j = blockIdx.x, tid = threadIdx.x;
  if (ld_volatile(&st->code) != 0) return;
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

// C = op(A) op(B), n x n, op = identity or conjugate transpose
template <class T>
__global__ void __launch_bounds__(256) small_gemm_kernel(const T* __restrict__ A, bool ha, const T* __restrict__ B,
                                                         bool hb, int n, T* __restrict__ C, const DeviceStatus* st) {
  __shared__ T As[16][17];
  __shared__ T Bs[16][17];
  if (ld_volatile(&st->code) != 0) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  T acc = zero<T>();
  for (int k0 = 0; k0 < n; k0 += 16) {
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
  if (row < n && col < n) C[(long long)row * n + col] = acc;
}

template <class T>
__global__ void hermitize_kernel(T* __restrict__ A, int n, const DeviceStatus* st) {
  if (ld_volatile(&st->code) != 0) return;
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

// player at position pos of round r of the circle (round-robin) schedule over npad players
__device__ __forceinline__ int rr_player(int pos, int r, int npad) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (npad - 1)) + 1;
}

template <class T>
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

// sum over all CTAs of per-CTA partials, identical (same order) in every CTA
__device__ double grid_sum(double mine, double* red, double* s_red, double* s_bcast, unsigned* bar, unsigned G,
                           DeviceStatus* st, int id, bool* ok) {
  const double b = block_reduce_sum<double>(mine, s_red);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!grid_barrier(bar, G, st, id)) {
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
  if (!grid_barrier(bar, G, st, id + 1)) *ok = false;
  return s;
}

template <class T>
__global__ void __launch_bounds__(256) jacobi_kernel(T* __restrict__ A0, T* __restrict__ A1, T* __restrict__ V,
                                                     int n, double tol, int max_sweeps, unsigned* bar,
                                                     DeviceStatus* st, double* red) {
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
  if (ld_volatile(&st->code) != 0) return;   // an earlier step (Cholesky) failed

  // V = I
  for (long long e = gtid; e < (long long)n * n; e += gthreads) V[e] = from_real<T>((e / n) == (e % n) ? 1.0 : 0.0);

  double fro2 = 0.0;
  for (long long e = gtid; e < (long long)n * n; e += gthreads) fro2 += absx2(ldcg(A + e));
  fro2 = grid_sum(fro2, red, s_red, &s_bcast, bar, G, st, 1, &ok);
  if (!ok) return;
  const double limit2 = tol * tol * fro2;

  for (int sweep = 0;; ++sweep) {
    double off2 = 0.0;
    for (long long e = gtid; e < (long long)n * n; e += gthreads)
      if ((e / n) != (e % n)) off2 += absx2(ldcg(A + e));
    off2 = grid_sum(off2, red, s_red, &s_bcast, bar, G, st, 3, &ok);
    if (!ok) return;
    if (off2 <= limit2 || sweep == max_sweeps) {
      if (off2 > limit2 && blockIdx.x == 0 && threadIdx.x == 0) set_status(st, PAWFD_ENOCONV, max_sweeps);
      if (A != A0)
        for (long long e = gtid; e < (long long)n * n; e += gthreads) A0[e] = ldcg(A + e);
      return;
    }
    for (int r = 0; r < npad - 1; ++r) {
      // rotation parameters of this round's n/2 disjoint pairs, computed by every CTA
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int p = rr_player(k, r, npad), q = rr_player(npad - 1 - k, r, npad);
        if (p > q) { const int t = p; p = q; q = t; }
        Rot R;
        R.c = 1.0; R.s = 0.0; R.e = zd{1.0, 0.0}; R.p = p; R.q = q;
        if (q >= n) {
          R.q = -1;
        } else {
          const T apq = ldcg(A + (long long)p * n + q);
          const double mag = absx(apq);
          if (mag > 0.0) {
            const double app = realx(ldcg(A + (long long)p * n + p)), aqq = realx(ldcg(A + (long long)q * n + q));
            const double tau = (aqq - app) / (2.0 * mag);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            R.c = 1.0 / sqrt(1.0 + t * t);
            R.s = t * R.c;
            R.e = phase_of(apq, mag);
          }
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
        // columns: B J_Q
        if (j1 >= 0) {
          const T x0 = rq.c * b00 - rq.s * mul_e(b01, rq.e);
          const T x1 = rq.s * b00 + rq.c * mul_e(b01, rq.e);
          const T y0 = rq.c * b10 - rq.s * mul_e(b11, rq.e);
          const T y1 = rq.s * b10 + rq.c * mul_e(b11, rq.e);
          b00 = x0; b01 = x1; b10 = y0; b11 = y1;
        }
        // rows: J_P^H (.)
        if (i1 >= 0) {
          const T x0 = rp.c * b00 - rp.s * mul_ce(b10, rp.e);
          const T y0 = rp.s * b00 + rp.c * mul_ce(b10, rp.e);
          const T x1 = rp.c * b01 - rp.s * mul_ce(b11, rp.e);
          const T y1 = rp.s * b01 + rp.c * mul_ce(b11, rp.e);
          b00 = x0; b10 = y0; b01 = x1; b11 = y1;
        }
        if (P == Q && i1 >= 0) {
          b01 = zero<T>();
          b10 = zero<T>();
          b00 = from_real<T>(realx(b00));
          b11 = from_real<T>(realx(b11));
        }
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
      if (!grid_barrier(bar, G, st, 100 + r)) return;
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

template <class T>
int subspace_impl(pawfd_ctx* c, int n, T* H, T* S, double* eps, T* C) {
  const long long nn = (long long)n * n;
  T* W = (T*)c->d_work;
  T* Hs = W;            // symmetrized H
  T* Lm = W + nn;       // symmetrized S, then L
  T* Li = W + 2 * nn;   // L^-1
  T* T1 = W + 3 * nn;   // L^-1 H, later U
  T* Am = W + 4 * nn;   // L^-1 H L^-H, diagonalized in place
  T* Vm = W + 5 * nn;   // Jacobi rotations
  T* A2 = W + 6 * nn;   // second Jacobi buffer
  cudaStream_t s = c->stream;
  const unsigned eb = (unsigned)((nn + 255) / 256);
  symmetrize_kernel<T><<<eb, 256, 0, s>>>(H, S, n, Hs, Lm);
  cholesky_kernel<T><<<1, 1024, 0, s>>>(Lm, n, c->d_status);
  tri_inverse_kernel<T><<<n, 256, sizeof(T) * n, s>>>(Lm, n, Li, c->d_status);
  dim3 gg((n + 15) / 16, (n + 15) / 16);
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(Li, false, Hs, false, n, T1, c->d_status);
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(T1, false, Li, true, n, Am, c->d_status);
  hermitize_kernel<T><<<eb, 256, 0, s>>>(Am, n, c->d_status);
  c->launches += 6;
  int rc = check_cuda(c, cudaGetLastError(), "subspace launch");
  if (rc != PAWFD_OK) return rc;

  // Jacobi: cooperative launch sized to the work of one round and to co-residency
  const int npad = n + (n & 1), np = npad / 2;
  const size_t rot_bytes = sizeof(Rot) * np;
  if (rot_bytes > 48 * 1024) {
    rc = check_cuda(c, cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)rot_bytes), "jacobi smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  int per_sm = 0;
  rc = check_cuda(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<T>, 256, rot_bytes),
                  "occupancy");
  if (rc != PAWFD_OK) return rc;
  long long want = ((long long)np * np + 255) / 256;
  int G = (int)std::max(1ll, std::min<long long>(want, (long long)per_sm * c->num_sms));
  G = std::min(G, 4096);
  rc = check_cuda(c, cudaMemsetAsync(c->d_barrier, 0, 2 * sizeof(unsigned), s), "barrier reset");
  if (rc != PAWFD_OK) return rc;
  double tol = 1e-14;
  int max_sweeps = 60;
  unsigned* bar = c->d_barrier;
  DeviceStatus* st = c->d_status;
  double* red = c->d_reduce;
  void* args[] = {&Am, &A2, &Vm, &n, &tol, &max_sweeps, &bar, &st, &red};
  rc = check_cuda(c, cudaLaunchCooperativeKernel((const void*)jacobi_kernel<T>, dim3(G), dim3(256), args, rot_bytes, s),
                  "jacobi cooperative launch");
  if (rc != PAWFD_OK) return rc;
  sort_kernel<T><<<n, 128, 0, s>>>(Am, Vm, n, eps, T1, c->d_status);
  small_gemm_kernel<T><<<gg, 256, 0, s>>>(Li, true, T1, false, n, C, c->d_status);
  phase_fix_kernel<T><<<n, 256, 0, s>>>(C, n, c->d_status);
  c->launches += 4;
  return check_cuda(c, cudaGetLastError(), "subspace launch");
}

}  // namespace

int launch_subspace_diag(pawfd_ctx* c, int nb, void* Hnm, void* Snm, double* eps, void* C) {
  if (nb > 3072) return fail(c, PAWFD_EINVAL, "subspace_diag supports at most 3072 bands");
  if (is_complex(c)) return subspace_impl<zd>(c, nb, (zd*)Hnm, (zd*)Snm, eps, (zd*)C);
  return subspace_impl<double>(c, nb, (double*)Hnm, (double*)Snm, eps, (double*)C);
}

}  // namespace pawfd
