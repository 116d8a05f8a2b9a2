// nonlocal.cu -- projector overlaps and the nonlocal back-add of the PAW operators.
//
//   P[row_a + i][n] = dV sum_q conj(G_a[i][q]) psi_n(r_q)          (projections, PAW section)
//   out_n(r_q)     += sum_i G_a[i][q] Q[i][n],  Q = dX^a P_a       (Eq. (dh) nonlocal term)
//
// G_a is atom a's projector box folded onto its unique grid points r_q at context creation,
// with the Bloch phase exp(-i k.T) of each periodic image already multiplied in, so the
// kernels are a plain gather-contraction and scatter-contraction.  The back-add is
// deterministic without atomics: atoms are coloured so that the boxes of one launch never
// share a grid point, each (point, band) is written by exactly one thread per launch, and
// colours are applied in a fixed order.
#include <algorithm>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int BT = 32;      // bands per CTA
constexpr int CH = 32;      // box points per chunk
constexpr int NT = 256;     // threads per CTA
constexpr int IMAX = 32;    // largest projector count per atom handled by the kernels

struct AtomArgs {
  const int* nproj;
  const int* row_off;
  const int* npts;
  const long long* pt_off;
  const int* pts;
  const long long* g_off;
  const long long* dmat_off;
};

template <class T>
__global__ void __launch_bounds__(NT) project_kernel(const T* __restrict__ psi, T* __restrict__ P, int nb,
                                                     long long K, double dV, const T* __restrict__ g, AtomArgs at) {
  __shared__ T gs[IMAX][CH];
  __shared__ T ps[BT][CH + 1];
  const int a = blockIdx.x;
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a], row = at.row_off[a];
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const T* __restrict__ ga = g + at.g_off[a];
  const int tid = threadIdx.x;
  // each thread owns the (i, band) pairs tid, tid + NT, ... of the I x BT output block
  constexpr int MAXPAIRS = IMAX * BT / NT;
  T acc[MAXPAIRS];
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) acc[e] = zero<T>();
  for (int pc = 0; pc < np; pc += CH) {
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      gs[i][p] = (pc + p < np) ? conjx(ga[(long long)i * np + pc + p]) : zero<T>();
    }
    for (int s = tid; s < BT * CH; s += NT) {
      const int bl = s / CH, p = s - bl * CH;
      ps[bl][p] = (pc + p < np && b0 + bl < nb) ? psi[(long long)(b0 + bl) * K + pts[pc + p]] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < MAXPAIRS; ++e) {
      const int pair = tid + e * NT;
      const int i = pair / BT, bl = pair - i * BT;
      if (i < I) {
        T s = acc[e];
#pragma unroll 8
        for (int p = 0; p < CH; ++p) fma_plain(s, gs[i][p], ps[bl][p]);
        acc[e] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) {
    const int pair = tid + e * NT;
    const int i = pair / BT, bl = pair - i * BT;
    if (i < I && b0 + bl < nb) P[(long long)(row + i) * nb + b0 + bl] = (real_t<T>)dV * acc[e];
  }
}

template <class T>
__global__ void __launch_bounds__(NT) nonlocal_add_kernel(const T* __restrict__ P, int nb, long long K,
                                                          const real_t<T>* __restrict__ dmat, const T* __restrict__ g,
                                                          AtomArgs at, const int* __restrict__ atoms,
                                                          T* __restrict__ out) {
  __shared__ T Qs[IMAX][BT];
  __shared__ T gs[IMAX][CH];
  const int a = atoms[blockIdx.x];
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a], row = at.row_off[a];
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const T* __restrict__ ga = g + at.g_off[a];
  const real_t<T>* __restrict__ dX = dmat + at.dmat_off[a];
  const int tid = threadIdx.x;
  // Q[i][bl] = sum_i' dX[i][i'] P[row + i'][b0 + bl]
  for (int s = tid; s < I * BT; s += NT) {
    const int i = s / BT, bl = s - i * BT;
    T q = zero<T>();
    if (b0 + bl < nb)
      for (int i2 = 0; i2 < I; ++i2) fma_real(q, dX[i * I + i2], P[(long long)(row + i2) * nb + b0 + bl]);
    Qs[i][bl] = q;
  }
  const int p_local = tid % CH, bsub = tid / CH;   // 8 bands in flight per pass
  for (int pc = 0; pc < np; pc += CH) {
    __syncthreads();
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      gs[i][p] = (pc + p < np) ? ga[(long long)i * np + pc + p] : zero<T>();
    }
    __syncthreads();
    const int p = pc + p_local;
    if (p < np) {
      const long long r = pts[p];
      for (int bl = bsub; bl < BT && b0 + bl < nb; bl += NT / CH) {
        T s = zero<T>();
        for (int i = 0; i < I; ++i) fma_plain(s, gs[i][p_local], Qs[i][bl]);
        T* o = out + (long long)(b0 + bl) * K + r;
        *o += s;
      }
    }
  }
}

// Q[row_a + i][m] = sum_j dS^a[i][j] P[row_a + j][m] in FP64: one CTA per (atom, 256 bands)
template <class T>
__global__ void __launch_bounds__(256) overlap_q_kernel(const T* __restrict__ P, int nb,
                                                        const real_t<T>* __restrict__ dmat, AtomArgs at,
                                                        wide_t<T>* __restrict__ Q) {
  using W = wide_t<T>;
  const int a = blockIdx.x, m = blockIdx.y * 256 + threadIdx.x;
  if (m >= nb) return;
  const int I = at.nproj[a], row = at.row_off[a];
  const real_t<T>* __restrict__ dX = dmat + at.dmat_off[a];
  for (int i = 0; i < I; ++i) {
    W q = zero<W>();
    for (int j = 0; j < I; ++j) fma_real(q, (double)dX[i * I + j], widen(P[(long long)(row + j) * nb + m]));
    Q[(long long)(row + i) * nb + m] = q;
  }
}

// M[n][m] += sum_r conj(P[r][n]) Q[r][m] for n <= m, mirrored to M[m][n] (M Hermitian; the
// diagonal keeps its real part).  16 x 16 output tiles on or above the diagonal.
template <class T>
__global__ void __launch_bounds__(256) overlap_corr_kernel(const T* __restrict__ P, const wide_t<T>* __restrict__ Q,
                                                           int nb, int Ip, wide_t<T>* __restrict__ M) {
  using W = wide_t<T>;
  if (blockIdx.y > blockIdx.x) return;   // tile (row block y, column block x), y <= x
  __shared__ W Ps[16][17];
  __shared__ W Qs[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int n = blockIdx.y * 16 + ty, m = blockIdx.x * 16 + tx;
  W acc = zero<W>();
  for (int r0 = 0; r0 < Ip; r0 += 16) {
    const int r = r0 + tx, rq = r0 + ty;
    const int nn = blockIdx.y * 16 + ty, mm = blockIdx.x * 16 + tx;
    Ps[ty][tx] = (r < Ip && nn < nb) ? conjx(widen(P[(long long)r * nb + nn])) : zero<W>();
    Qs[ty][tx] = (rq < Ip && mm < nb) ? Q[(long long)rq * nb + mm] : zero<W>();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) fma_plain(acc, Ps[ty][k], Qs[k][tx]);
    __syncthreads();
  }
  if (n >= nb || m >= nb || n > m) return;
  if (n == m) {
    M[(long long)n * nb + n] = M[(long long)n * nb + n] + from_real<W>(realx(acc));
  } else {
    M[(long long)n * nb + m] = M[(long long)n * nb + m] + acc;
    M[(long long)m * nb + n] = M[(long long)m * nb + n] + conjx(acc);
  }
}

AtomArgs atom_args(const pawfd_ctx* c) {
  AtomArgs a;
  a.nproj = c->at.d_nproj;
  a.row_off = c->at.d_row_off;
  a.npts = c->at.d_npts;
  a.pt_off = c->at.d_pt_off;
  a.pts = c->at.d_pts;
  a.g_off = c->at.d_g_off;
  a.dmat_off = c->at.d_dmat_off;
  return a;
}

}  // namespace

int launch_project(pawfd_ctx* c, const void* psi, int nb, void* P) {
  if (c->at.natoms == 0) return PAWFD_OK;
  if (c->at.Imax > IMAX) return fail(c, PAWFD_EINVAL, "more than 32 projectors on one atom");
  dim3 grid(c->at.natoms, (nb + BT - 1) / BT);
  dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    project_kernel<T><<<grid, NT, 0, c->stream>>>((const T*)psi, (T*)P, nb, (long long)c->K, c->dV,
                                                   (const T*)c->at.d_g, atom_args(c));
    return 0;
  });
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "project launch");
}

int launch_nonlocal_add(pawfd_ctx* c, const void* P, int nb, const void* d_dmat, void* out) {
  if (c->at.natoms == 0) return PAWFD_OK;
  if (c->at.Imax > IMAX) return fail(c, PAWFD_EINVAL, "more than 32 projectors on one atom");
  for (size_t col = 0; col + 1 < c->at.color_off.size(); ++col) {
    const int first = c->at.color_off[col], count = c->at.color_off[col + 1] - first;
    dim3 grid(count, (nb + BT - 1) / BT);
    const int* atoms = c->at.d_color_atoms + first;
    dispatch_band(c, [&](auto tag) {
      using T = decltype(tag);
      nonlocal_add_kernel<T><<<grid, NT, 0, c->stream>>>((const T*)P, nb, (long long)c->K,
                                                          (const real_t<T>*)d_dmat, (const T*)c->at.d_g,
                                                          atom_args(c), atoms, (T*)out);
      return 0;
    });
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "nonlocal_add launch");
}

// S_nm += sum_a P_a^H dS^a P_a (the overlap's nonlocal term of the S Gram matrix); M is the
// Hermitian FP64 [nb][nb] matrix, P the projections [Ip][nb] of the context's band dtype
int launch_overlap_correction(pawfd_ctx* c, const void* P, int nb, void* M) {
  if (c->at.natoms == 0) return PAWFD_OK;
  if (c->at.Imax > IMAX) return fail(c, PAWFD_EINVAL, "more than 32 projectors on one atom");
  const int tb = (nb + 15) / 16;
  dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    using W = wide_t<T>;
    overlap_q_kernel<T><<<dim3(c->at.natoms, (nb + 255) / 256), 256, 0, c->stream>>>(
        (const T*)P, nb, (const real_t<T>*)c->at.d_dS, atom_args(c), (W*)c->d_Q);
    overlap_corr_kernel<T><<<dim3(tb, tb), 256, 0, c->stream>>>((const T*)P, (const W*)c->d_Q, nb, c->at.Ip, (W*)M);
    return 0;
  });
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "overlap correction launch");
}

}  // namespace pawfd
