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
#include <type_traits>

#include "df_arith.cuh"
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

// Partial projections of one work item (atom a, box points p0 .. p0 + NL_PCH - 1) for BT
// bands: part[item_row + i][band] = sum_p conj(G_a[i][p]) psi_band(r_p) over the item's points.
template <class T>
__global__ void __launch_bounds__(NT) project_kernel(const T* __restrict__ psi, T* __restrict__ part, int nb,
                                                     long long K, const T* __restrict__ g, AtomArgs at,
                                                     const int2* __restrict__ items,
                                                     const long long* __restrict__ item_row) {
  __shared__ T gs[IMAX][CH];
  __shared__ T ps[BT][CH + 1];
  const int2 item = items[blockIdx.x];
  const int a = item.x;
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a];
  const int p_end = min(np, item.y + NL_PCH);
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const T* __restrict__ ga = g + at.g_off[a];
  const int tid = threadIdx.x;
  // each thread owns the (i, band) pairs tid, tid + NT, ... of the I x BT output block
  constexpr int MAXPAIRS = IMAX * BT / NT;
  T acc[MAXPAIRS];
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) acc[e] = zero<T>();
  for (int pc = item.y; pc < p_end; pc += CH) {
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      gs[i][p] = (pc + p < p_end) ? conjx(ga[(long long)i * np + pc + p]) : zero<T>();
    }
    for (int s = tid; s < BT * CH; s += NT) {
      const int bl = s / CH, p = s - bl * CH;
      ps[bl][p] = (pc + p < p_end && b0 + bl < nb) ? psi[(long long)(b0 + bl) * K + pts[pc + p]] : zero<T>();
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
  const long long row = item_row[blockIdx.x];
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) {
    const int pair = tid + e * NT;
    const int i = pair / BT, bl = pair - i * BT;
    if (i < I && b0 + bl < nb) part[(row + i) * nb + b0 + bl] = acc[e];
  }
}

// P[row_a + i][band] = dV sum over the atom's items (in order) of the partials
template <class T>
__global__ void __launch_bounds__(256) project_reduce_kernel(const T* __restrict__ part, T* __restrict__ P, int nb,
                                                             double dV, AtomArgs at,
                                                             const int* __restrict__ atom_items,
                                                             const long long* __restrict__ item_row) {
  using W = wide_t<T>;
  const int a = blockIdx.x, m = blockIdx.y * 256 + threadIdx.x;
  if (m >= nb) return;
  const int I = at.nproj[a], row = at.row_off[a];
  const int it0 = atom_items[a], it1 = atom_items[a + 1];
  for (int i = 0; i < I; ++i) {
    W s = zero<W>();
    for (int it = it0; it < it1; ++it) s = s + widen(part[(item_row[it] + i) * nb + m]);
    P[(long long)(row + i) * nb + m] = narrow<T>(dV * s);
  }
}

// out1 += sum_i G_a[i] Q1[i] (and out2 with Q2 when out2 is set), Qk = dmat_k^a P_a, over one
// work item's box points.  Items of one launch belong to atoms of one colour, so no two
// threads of a launch touch the same grid point.
template <class T>
__global__ void __launch_bounds__(NT) nonlocal_add_kernel(const T* __restrict__ P, int nb, long long K,
                                                          const real_t<T>* __restrict__ dmat1,
                                                          const real_t<T>* __restrict__ dmat2,
                                                          const T* __restrict__ g, AtomArgs at,
                                                          const int2* __restrict__ items, T* __restrict__ out1,
                                                          T* __restrict__ out2) {
  __shared__ T Q1s[IMAX][BT];
  __shared__ T Q2s[IMAX][BT];
  __shared__ T gs[IMAX][CH];
  const int2 item = items[blockIdx.x];
  const int a = item.x;
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a], row = at.row_off[a];
  const int p_end = min(np, item.y + NL_PCH);
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const T* __restrict__ ga = g + at.g_off[a];
  const long long dmo = at.dmat_off[a];
  const int tid = threadIdx.x;
  const bool two = out2 != nullptr;
  // Qk[i][bl] = sum_i' dmat_k[i][i'] P[row + i'][b0 + bl]
  for (int s = tid; s < I * BT; s += NT) {
    const int i = s / BT, bl = s - i * BT;
    T q1 = zero<T>(), q2 = zero<T>();
    if (b0 + bl < nb)
      for (int i2 = 0; i2 < I; ++i2) {
        const T pv = P[(long long)(row + i2) * nb + b0 + bl];
        fma_real(q1, dmat1[dmo + i * I + i2], pv);
        if (two) fma_real(q2, dmat2[dmo + i * I + i2], pv);
      }
    Q1s[i][bl] = q1;
    Q2s[i][bl] = q2;
  }
  const int p_local = tid % CH, bsub = tid / CH;   // 8 bands in flight per pass
  for (int pc = item.y; pc < p_end; pc += CH) {
    __syncthreads();
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      gs[i][p] = (pc + p < p_end) ? ga[(long long)i * np + pc + p] : zero<T>();
    }
    __syncthreads();
    const int p = pc + p_local;
    if (p < p_end) {
      const long long r = pts[p];
      for (int bl = bsub; bl < BT && b0 + bl < nb; bl += NT / CH) {
        T s1 = zero<T>(), s2 = zero<T>();
        for (int i = 0; i < I; ++i) {
          fma_plain(s1, gs[i][p_local], Q1s[i][bl]);
          if (two) fma_plain(s2, gs[i][p_local], Q2s[i][bl]);
        }
        const long long o = (long long)(b0 + bl) * K + r;
        out1[o] += s1;
        if (two) out2[o] += s2;
      }
    }
  }
}

// ---- real FP64 bands in double-float arithmetic (FP32 pipe) ----
// The FP64 forms above are bound by GB300's FP64 rate (about two FMAs per SM and clock).
// Here the operands are pairs hi + lo (the projector values split once at create, psi and
// Q split on load) and every product-accumulate is dfa::fma_acc, about 15 FP32 operations of
// relative error ~2^-47; a run of CH terms is summed in pairs and then added to an FP64
// accumulator, so the pairs' error does not grow with the box size.

template <int I_UNUSED = 0>
__global__ void __launch_bounds__(NT) project_df_kernel(const double* __restrict__ psi, double* __restrict__ part,
                                                        int nb, long long K, const float2* __restrict__ gdf,
                                                        AtomArgs at, const int2* __restrict__ items,
                                                        const long long* __restrict__ item_row) {
  using dfa::DF;
  __shared__ DF gs[IMAX][CH];
  __shared__ DF ps[BT][CH + 1];
  const int2 item = items[blockIdx.x];
  const int a = item.x;
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a];
  const int p_end = min(np, item.y + NL_PCH);
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const float2* __restrict__ ga = gdf + at.g_off[a];
  const int tid = threadIdx.x;
  constexpr int MAXPAIRS = IMAX * BT / NT;
  double acc[MAXPAIRS];
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) acc[e] = 0.0;
  for (int pc = item.y; pc < p_end; pc += CH) {
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      const float2 gv = (pc + p < p_end) ? ga[(long long)i * np + pc + p] : make_float2(0.f, 0.f);
      gs[i][p] = {gv.x, gv.y};
    }
    for (int s = tid; s < BT * CH; s += NT) {
      const int bl = s / CH, p = s - bl * CH;
      ps[bl][p] = (pc + p < p_end && b0 + bl < nb) ? dfa::split64(psi[(long long)(b0 + bl) * K + pts[pc + p]])
                                                   : DF{0.f, 0.f};
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < MAXPAIRS; ++e) {
      const int pair = tid + e * NT;
      const int i = pair / BT, bl = pair - i * BT;
      if (i < I) {
        DF s = {0.f, 0.f};
#pragma unroll 8
        for (int p = 0; p < CH; ++p) dfa::fma_acc(s, gs[i][p], ps[bl][p]);
        acc[e] += dfa::to_double(s);
      }
    }
    __syncthreads();
  }
  const long long row = item_row[blockIdx.x];
#pragma unroll
  for (int e = 0; e < MAXPAIRS; ++e) {
    const int pair = tid + e * NT;
    const int i = pair / BT, bl = pair - i * BT;
    if (i < I && b0 + bl < nb) part[(row + i) * nb + b0 + bl] = acc[e];
  }
}

template <int I_UNUSED = 0>
__global__ void __launch_bounds__(NT) nonlocal_add_df_kernel(const double* __restrict__ P, int nb, long long K,
                                                             const double* __restrict__ dmat1,
                                                             const double* __restrict__ dmat2,
                                                             const float2* __restrict__ gdf, AtomArgs at,
                                                             const int2* __restrict__ items,
                                                             double* __restrict__ out1, double* __restrict__ out2) {
  using dfa::DF;
  __shared__ DF Q1s[IMAX][BT];
  __shared__ DF Q2s[IMAX][BT];
  __shared__ DF gs[IMAX][CH];
  const int2 item = items[blockIdx.x];
  const int a = item.x;
  const int b0 = blockIdx.y * BT;
  const int I = at.nproj[a], np = at.npts[a], row = at.row_off[a];
  const int p_end = min(np, item.y + NL_PCH);
  const int* __restrict__ pts = at.pts + at.pt_off[a];
  const float2* __restrict__ ga = gdf + at.g_off[a];
  const long long dmo = at.dmat_off[a];
  const int tid = threadIdx.x;
  const bool two = out2 != nullptr;
  // Qk[i][bl] = sum_i' dmat_k[i][i'] P[row + i'][b0 + bl] in FP64 (I^2 per band), then split
  for (int s = tid; s < I * BT; s += NT) {
    const int i = s / BT, bl = s - i * BT;
    double q1 = 0.0, q2 = 0.0;
    if (b0 + bl < nb)
      for (int i2 = 0; i2 < I; ++i2) {
        const double pv = P[(long long)(row + i2) * nb + b0 + bl];
        q1 = fma(dmat1[dmo + i * I + i2], pv, q1);
        if (two) q2 = fma(dmat2[dmo + i * I + i2], pv, q2);
      }
    Q1s[i][bl] = dfa::split64(q1);
    Q2s[i][bl] = dfa::split64(q2);
  }
  const int p_local = tid % CH, bsub = tid / CH;
  for (int pc = item.y; pc < p_end; pc += CH) {
    __syncthreads();
    for (int s = tid; s < I * CH; s += NT) {
      const int i = s / CH, p = s - i * CH;
      const float2 gv = (pc + p < p_end) ? ga[(long long)i * np + pc + p] : make_float2(0.f, 0.f);
      gs[i][p] = {gv.x, gv.y};
    }
    __syncthreads();
    const int p = pc + p_local;
    if (p < p_end) {
      const long long r = pts[p];
      for (int bl = bsub; bl < BT && b0 + bl < nb; bl += NT / CH) {
        DF s1 = {0.f, 0.f}, s2 = {0.f, 0.f};
        for (int i = 0; i < I; ++i) {
          dfa::fma_acc(s1, gs[i][p_local], Q1s[i][bl]);
          if (two) dfa::fma_acc(s2, gs[i][p_local], Q2s[i][bl]);
        }
        const long long o = (long long)(b0 + bl) * K + r;
        out1[o] += dfa::to_double(s1);
        if (two) out2[o] += dfa::to_double(s2);
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
  dim3 grid(c->at.nitems, (nb + BT - 1) / BT), rgrid(c->at.natoms, (nb + 255) / 256);
  dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    if (c->at.nitems > 0) {
      if (std::is_same<T, double>::value && c->at.d_g_df && c->nonlocal_df)
        project_df_kernel<><<<grid, NT, 0, c->stream>>>((const double*)psi, (double*)c->d_Ppart, nb, (long long)c->K,
                                                        (const float2*)c->at.d_g_df, atom_args(c), c->at.d_items,
                                                        c->at.d_item_row);
      else
        project_kernel<T><<<grid, NT, 0, c->stream>>>((const T*)psi, (T*)c->d_Ppart, nb, (long long)c->K,
                                                       (const T*)c->at.d_g, atom_args(c), c->at.d_items,
                                                       c->at.d_item_row);
    }
    project_reduce_kernel<T><<<rgrid, 256, 0, c->stream>>>((const T*)c->d_Ppart, (T*)P, nb, c->dV, atom_args(c),
                                                            c->at.d_atom_items, c->at.d_item_row);
    return 0;
  });
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "project launch");
}

int launch_nonlocal_add2(pawfd_ctx* c, const void* P, int nb, const void* dmat1, void* out1, const void* dmat2,
                         void* out2) {
  if (c->at.natoms == 0) return PAWFD_OK;
  if (c->at.Imax > IMAX) return fail(c, PAWFD_EINVAL, "more than 32 projectors on one atom");
  for (size_t col = 0; col + 1 < c->at.color_item_off.size(); ++col) {
    const int first = c->at.color_item_off[col], count = c->at.color_item_off[col + 1] - first;
    if (count == 0) continue;
    dim3 grid(count, (nb + BT - 1) / BT);
    const int2* items = c->at.d_color_items + first;
    dispatch_band(c, [&](auto tag) {
      using T = decltype(tag);
      if (std::is_same<T, double>::value && c->at.d_g_df && c->nonlocal_df)
        nonlocal_add_df_kernel<><<<grid, NT, 0, c->stream>>>((const double*)P, nb, (long long)c->K,
                                                             (const double*)dmat1, (const double*)dmat2,
                                                             (const float2*)c->at.d_g_df, atom_args(c), items,
                                                             (double*)out1, (double*)out2);
      else
        nonlocal_add_kernel<T><<<grid, NT, 0, c->stream>>>((const T*)P, nb, (long long)c->K,
                                                            (const real_t<T>*)dmat1, (const real_t<T>*)dmat2,
                                                            (const T*)c->at.d_g, atom_args(c), items, (T*)out1,
                                                            (T*)out2);
      return 0;
    });
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "nonlocal_add launch");
}

int launch_nonlocal_add(pawfd_ctx* c, const void* P, int nb, const void* d_dmat, void* out) {
  return launch_nonlocal_add2(c, P, nb, d_dmat, out, nullptr, nullptr);
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
