// tc_gram.cu -- Gram matrices on the tensor cores (sliced_gram.cuh) for every band dtype.
//
// Real inputs: M = dV A^T B over K.  Complex inputs: the interleaved arrays are read as real
// rows of length 2K; Re(conj(a).b) is the real dot product of the two rows and Im(conj(a).b) the
// dot product of a with the "swapped" row (im, -re) of b, so the complex Gram is one real
// Gram of A (nb rows) against B_ext = [B; B''] (2 nb rows).  K is processed in blocks whose
// slices fit the context's scratch; every block adds into FP64 split-K partials, and one
// reduce kernel sums the partials in a fixed order, applies dV and (for the Hermitian form)
// mirrors the upper triangle.
#include <cudaTypedefs.h>

#include <algorithm>

#include "pawfd_internal.cuh"
#include "sliced_gram.cuh"

namespace pawfd {
namespace {

// Split-K count of one K block.  The MMA kernel holds one CTA per SM (its shared memory and
// TMEM), so tiles x splits CTAs run in ceil(tiles x splits / SMs) waves of ceil(chunks / splits)
// chunks each.  The count with the fewest chunk-times wins, each wave's fixed cost (prologue,
// pipeline fill, partial store) counted as one chunk; ties go to fewer splits.  Filling the SMs
// once is not enough: 106 tiles (1024 complex bands) in one wave leave 46 of 152 SMs idle,
// ten splits run the same work in seven waves at 98 % occupancy.
int gram_splits(int tiles, int nch, int num_sms) {
  int best = 1;
  long long best_cost = -1;
  const int cap = std::min(nch, 2 * num_sms);
  for (int s = 1; s <= cap; ++s) {
    const int cpc = (nch + s - 1) / s, ns = (nch + cpc - 1) / cpc;
    const long long waves = ((long long)tiles * ns + num_sms - 1) / num_sms;
    const long long cost = waves * (cpc + 1);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = ns;
    }
  }
  return best;
}

// The symmetric cover of a Hermitian Gram of 192 < nb <= 256 rows (per half for complex bands).  Eight blocks of 32
// rows; a tile has A rows from block row_blk (four blocks, 128 rows) and B rows from three
// blocks.  With each tile's mirror (a tile below the diagonal computes the transposes of needed
// entries) the four tiles hold all 36 pairs of blocks; found by exhaustive search over the row
// starts and block triples.  The upper-triangle tiling needs five 128 x 96 tiles for the same
// matrix, so the cover does 20 % fewer digit products.
constexpr int kCoverRowBlk[sg::COVER_TILES] = {0, 0, 1, 4};
constexpr int kCoverSegBlk[sg::COVER_TILES][3] = {{0, 4, 5}, {1, 6, 7}, {2, 3, 4}, {5, 6, 7}};

bool use_cover(int nb) { return nb > 2 * sg::BN && nb <= 8 * sg::CB; }

// Fills the cover fields of a: each block pair goes to the first tile that holds it, written
// from the direct orientation (row block lo) when that tile has it, else mirrored.
void set_cover(sg::GramArgs& a) {
  a.cover = 1;
  unsigned long long owned = 0;
  for (int t = 0; t < sg::COVER_TILES; ++t) {
    a.cov_row0[t] = kCoverRowBlk[t] * sg::CB;
    for (int g = 0; g < 3; ++g) a.cov_seg[t][g] = kCoverSegBlk[t][g] * sg::CB;
    a.cov_own[t] = a.cov_tr[t] = 0;
    auto in_rows = [&](int b) { return b >= kCoverRowBlk[t] && b < kCoverRowBlk[t] + sg::BM / sg::CB; };
    auto in_cols = [&](int b) { return b == kCoverSegBlk[t][0] || b == kCoverSegBlk[t][1] || b == kCoverSegBlk[t][2]; };
    for (int lo = 0; lo < 8; ++lo)
      for (int hi = lo; hi < 8; ++hi) {
        const unsigned long long bit = 1ull << (lo * 8 + hi);
        if (owned & bit) continue;
        const bool direct = in_rows(lo) && in_cols(hi), mirrored = in_rows(hi) && in_cols(lo);
        if (!direct && !mirrored) continue;
        owned |= bit;
        a.cov_own[t] |= bit;
        if (!direct) a.cov_tr[t] |= bit;
      }
  }
}

// Tiles of the Hermitian Gram pair for nb bands
int pair_tiles(int nb, bool cplx) { return (cplx ? 2 : 1) * (use_cover(nb) ? sg::COVER_TILES : sg::herm_tiles(nb)); }

template <class W>
__global__ void tc_reduce_kernel(const double* __restrict__ part, int nsplit, int nb, int rowsB, int im_off, double dV,
                                 bool herm, W* __restrict__ M);

// real: part [nsplit][nb][nb]
template <>
__global__ void tc_reduce_kernel<double>(const double* __restrict__ part, int nsplit, int nb, int rowsB, int,
                                         double dV, bool herm, double* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  const int n = (int)(e / nb), m = (int)(e % nb);
  if (herm && m < n) return;
  double s = 0.0;
  for (int p = 0; p < nsplit; ++p) s += part[((long long)p * nb + n) * rowsB + m];
  s *= dV;
  M[e] = s;
  if (herm && m != n) M[(long long)m * nb + n] = s;
}

// complex: part [nsplit][nb][rowsB], real part in columns [0, nb), imaginary in [im_off, im_off + nb)
template <>
__global__ void tc_reduce_kernel<zd>(const double* __restrict__ part, int nsplit, int nb, int rowsB, int im_off,
                                     double dV, bool herm, zd* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nb * nb) return;
  const int n = (int)(e / nb), m = (int)(e % nb);
  if (herm && m < n) return;
  double re = 0.0, im = 0.0;
  for (int p = 0; p < nsplit; ++p) {
    const double* row = part + ((long long)p * nb + n) * rowsB;
    re += row[m];
    im += row[im_off + m];
  }
  re *= dV;
  im *= dV;
  if (herm && m == n) im = 0.0;
  M[e] = zd{re, im};
  if (herm && m != n) M[(long long)m * nb + n] = zd{re, -im};
}

template <class R, int S, int ORD>
int tc_gram_impl(pawfd_ctx* c, const R* A, const R* B, int nb, void* M, bool herm) {
  TcScratch& t = c->tc;
  const bool cplx = is_complex(c);
  const long long L = (long long)c->K * (cplx ? 2 : 1);            // real-view row length
  // complex: the swapped rows B'' start at a multiple of 8 (whole core-matrix row groups)
  const int nbp = (nb + 7) / 8 * 8;
  const int rowsB = cplx ? nbp + nb : nb;
  const int Tr = (nb + sg::BM - 1) / sg::BM, Tc = (nb + sg::BN - 1) / sg::BN;
  const int halves = cplx ? 2 : 1;
  const int tiles = herm ? halves * sg::herm_tiles(nb) : Tr * halves * Tc;
  // K block: the allocated slice length, or fewer chunks (the slices of a short block can stay
  // in L2 between the slicing kernels and the MMA kernel)
  const long long Kblk = c->tc_kblk_chunks > 0 ? std::min<long long>(t.kblk, (long long)c->tc_kblk_chunks * sg::KCG)
                                                 : t.kblk;
  const int nch0 = (int)((std::min(Kblk, L) + sg::KCG - 1) / sg::KCG);   // chunks of the first block
  int nsplit = gram_splits(tiles, nch0, c->num_sms);
  while (nsplit > 1 && (size_t)nsplit * nb * rowsB * sizeof(double) > t.part_bytes) --nsplit;
  __nv_bfloat16* sA = (__nv_bfloat16*)t.slicesA;
  __nv_bfloat16* sB = (__nv_bfloat16*)t.slicesB;
  int blk = 0;
  for (long long k0 = 0; k0 < L; k0 += Kblk, ++blk) {
    const long long len = std::min(Kblk, L - k0);
    const int nch = (int)((len + sg::KCG - 1) / sg::KCG);
    const int cpc = (nch + nsplit - 1) / nsplit;
    const int ns = (nch + cpc - 1) / cpc;
    // per-row largest sigma of this block: start from a very negative value
    cudaMemsetAsync(t.maxA, 0x80, sizeof(int) * t.rowsA_alloc, c->stream);
    cudaMemsetAsync(t.maxB, 0x80, sizeof(int) * t.rowsB_alloc, c->stream);
    // slices keep the allocated row length t.kblk (the tensor maps' layout); a shorter block
    // fills the first Kblk values of each row
    sg::slice_kernel<R, S, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
        A + k0, nb, L, len, nch, t.kblk, false, 0, t.rowsA_alloc, sA, t.sigA, t.rowsA_alloc, t.maxA);
    sg::slice_kernel<R, S, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
        B + k0, nb, L, len, nch, t.kblk, false, 0, t.rowsB_alloc, sB, t.sigB, t.rowsB_alloc, t.maxB);
    c->launches += 2;
    if (cplx) {
      sg::slice_kernel<R, S, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
          B + k0, nb, L, len, nch, t.kblk, true, nbp, t.rowsB_alloc, sB, t.sigB, t.rowsB_alloc, t.maxB);
      c->launches += 1;
    }
    sg::GramArgs a = {};
    a.gA = sA;
    a.gB = sB;
    a.rows_allocA = t.rowsA_alloc;
    a.rows_allocB = t.rowsB_alloc;
    a.ksteps = t.kblk / sg::BK;
    a.half_stride = cplx ? nbp : nb;
    a.sigA = t.sigA;
    a.sigB = t.sigB;
    a.sig_ldA = t.rowsA_alloc;
    a.sig_ldB = t.rowsB_alloc;
    a.maxA = t.maxA;
    a.maxB = t.maxB;
    a.rowsA = nb;
    a.rowsB = rowsB;
    a.tilesN = halves * Tc;
    a.herm = herm;
    a.halves = halves;
    a.half_rows = nb;
    a.chunks_per_cta = cpc;
    a.nchunks = nch;
    a.accumulate = blk > 0;
    a.klen = len;
    a.part = (double*)t.part;
    a.st = c->d_status;
    // slots written by the first block must cover every split later blocks add into
    if (blk == 0 && ns < nsplit) nsplit = ns;
    ktimer_begin(c);
    sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG><<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(
        t.mapA, t.mapB, t.mapB, a);
    ktimer_end(c);
    c->launches += 1;
  }
  const long long nn = (long long)nb * nb;
  if (cplx)
    tc_reduce_kernel<zd><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part, nsplit, nb, rowsB, nbp,
                                                                              c->dV, herm, (zd*)M);
  else
    tc_reduce_kernel<double><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part, nsplit, nb, rowsB,
                                                                                  nb, c->dV, herm, (double*)M);
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "tensor-core gram launch");
}

// The two Hermitian Gram matrices of the Rayleigh-Ritz step for real bands from one slicing
// of psi: M1 = dV psi^T B (B = H psi) and M2 = dV psi^T psi, the second with psi's digit
// planes as both operands.  Each K block slices psi and B once and runs the two MMA kernels.
template <class R, int S, int ORD>
int tc_gram_pair_impl(pawfd_ctx* c, const R* A, const R* B, int nb, double* M1, double* M2) {
  TcScratch& t = c->tc;
  const long long L = (long long)c->K;
  const bool cover = use_cover(nb);
  const int tiles = pair_tiles(nb, false);
  const long long Kblk = c->tc_kblk_chunks > 0 ? std::min<long long>(t.kblk, (long long)c->tc_kblk_chunks * sg::KCG)
                                                 : t.kblk;
  const int nch0 = (int)((std::min(Kblk, L) + sg::KCG - 1) / sg::KCG);
  int nsplit = gram_splits(tiles, nch0, c->num_sms);
  while (nsplit > 1 && (size_t)nsplit * nb * nb * sizeof(double) > t.part_bytes) --nsplit;
  __nv_bfloat16* sA = (__nv_bfloat16*)t.slicesA;
  __nv_bfloat16* sB = (__nv_bfloat16*)t.slicesB;
  // psi's digits of a single-block Gram may already be in place (gram_slice_psi)
  const bool presliced = t.presliced_gram == (const void*)A && t.presliced_gram_nb == nb && Kblk >= L;
  t.presliced_gram = nullptr;
  int blk = 0;
  for (long long k0 = 0; k0 < L; k0 += Kblk, ++blk) {
    const long long len = std::min(Kblk, L - k0);
    const int nch = (int)((len + sg::KCG - 1) / sg::KCG);
    const int cpc = (nch + nsplit - 1) / nsplit;
    const int ns = (nch + cpc - 1) / cpc;
    if (!presliced) {
      cudaMemsetAsync(t.maxA, 0x80, sizeof(int) * t.rowsA_alloc, c->stream);
      sg::slice_kernel<R, S, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
          A + k0, nb, L, len, nch, t.kblk, false, 0, t.rowsA_alloc, sA, t.sigA, t.rowsA_alloc, t.maxA);
    }
    cudaMemsetAsync(t.maxB, 0x80, sizeof(int) * t.rowsB_alloc, c->stream);
    sg::slice_kernel<R, S, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
        B + k0, nb, L, len, nch, t.kblk, false, 0, t.rowsB_alloc, sB, t.sigB, t.rowsB_alloc, t.maxB);
    sg::GramArgs a = {};
    a.gA = sA;
    a.gB = sB;
    a.rows_allocA = t.rowsA_alloc;
    a.rows_allocB = t.rowsB_alloc;
    a.ksteps = t.kblk / sg::BK;
    a.sigA = t.sigA;
    a.sigB = t.sigB;
    a.sig_ldA = t.rowsA_alloc;
    a.sig_ldB = t.rowsB_alloc;
    a.maxA = t.maxA;
    a.maxB = t.maxB;
    a.rowsA = nb;
    a.rowsB = nb;
    a.tilesN = (nb + sg::BN - 1) / sg::BN;
    a.herm = 1;
    a.halves = 1;
    a.half_rows = nb;
    a.chunks_per_cta = cpc;
    a.nchunks = nch;
    a.accumulate = blk > 0;
    a.klen = len;
    a.part = (double*)t.part;
    a.st = c->d_status;
    if (cover) set_cover(a);
    if (blk == 0 && ns < nsplit) nsplit = ns;
    ktimer_begin(c);
    if (cover)
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG, true>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB, t.mapB32, a);
    else
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB, t.mapB32, a);
    ktimer_end(c);
    // psi^T psi: psi's planes and exponents on both sides (psi's planes through a map with the
    // B operand's box)
    sg::GramArgs a2 = a;
    a2.gB = sA;
    a2.rows_allocB = t.rowsA_alloc;
    a2.sigB = t.sigA;
    a2.sig_ldB = t.rowsA_alloc;
    a2.maxB = t.maxA;
    a2.part = (double*)t.part2;
    ktimer_begin(c);
    if (cover)
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG, true>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapAB, t.mapAB32, a2);
    else
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapAB, t.mapAB32, a2);
    ktimer_end(c);
    c->launches += presliced ? 3 : 4;
  }
  const long long nn = (long long)nb * nb;
  tc_reduce_kernel<double><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part, nsplit, nb, nb, nb,
                                                                                c->dV, true, M1);
  tc_reduce_kernel<double><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part2, nsplit, nb, nb, nb,
                                                                                c->dV, true, M2);
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "tensor-core gram pair launch");
}

// The two Hermitian Gram matrices of the Rayleigh-Ritz step for complex bands from one slicing
// of psi and one of B = H psi.  B_ext = [psi; psi''] (psi and its swapped rows) is the second
// operand of both: M2 = dV psi^H psi takes psi's planes (rows [0, nb) of B_ext) as the first
// operand as well, and M1 takes B as the first operand, M1 = dV B^H psi.  For a Hermitian
// operator, (H psi)_n^H psi_m = conj(psi_m^H H psi_n) = H_nm, so M1 is psi^H H psi; the
// Hermitian tiling already rests on that symmetry (only the upper triangle is formed).  Three
// slicing passes per K block instead of the six of two separate Grams.
template <class R, int S, int ORD>
int tc_gram_pair_cplx_impl(pawfd_ctx* c, const R* A, const R* B, int nb, zd* M1, zd* M2) {
  TcScratch& t = c->tc;
  const long long L = 2LL * c->K;                                   // real-view row length
  const int nbp = (nb + 7) / 8 * 8;
  const int rowsB = nbp + nb;
  const int Tc = (nb + sg::BN - 1) / sg::BN;
  const bool cover = use_cover(nb);
  const int tiles = pair_tiles(nb, true);
  const long long Kblk = c->tc_kblk_chunks > 0 ? std::min<long long>(t.kblk, (long long)c->tc_kblk_chunks * sg::KCG)
                                                 : t.kblk;
  const int nch0 = (int)((std::min(Kblk, L) + sg::KCG - 1) / sg::KCG);
  int nsplit = gram_splits(tiles, nch0, c->num_sms);
  while (nsplit > 1 && (size_t)nsplit * nb * rowsB * sizeof(double) > t.part_bytes) --nsplit;
  __nv_bfloat16* sA = (__nv_bfloat16*)t.slicesA;
  __nv_bfloat16* sB = (__nv_bfloat16*)t.slicesB;
  t.presliced_gram = nullptr;
  int blk = 0;
  for (long long k0 = 0; k0 < L; k0 += Kblk, ++blk) {
    const long long len = std::min(Kblk, L - k0);
    const int nch = (int)((len + sg::KCG - 1) / sg::KCG);
    const int cpc = (nch + nsplit - 1) / nsplit;
    const int ns = (nch + cpc - 1) / cpc;
    cudaMemsetAsync(t.maxA, 0x80, sizeof(int) * t.rowsA_alloc, c->stream);
    cudaMemsetAsync(t.maxB, 0x80, sizeof(int) * t.rowsB_alloc, c->stream);
    const unsigned grid = (unsigned)(((long long)nb * nch + 7) / 8);
    sg::slice_kernel<R, S, sg::KCG><<<grid, 256, 0, c->stream>>>(B + k0, nb, L, len, nch, t.kblk, false, 0,
                                                                 t.rowsA_alloc, sA, t.sigA, t.rowsA_alloc, t.maxA);
    sg::slice_kernel<R, S, sg::KCG><<<grid, 256, 0, c->stream>>>(A + k0, nb, L, len, nch, t.kblk, false, 0,
                                                                 t.rowsB_alloc, sB, t.sigB, t.rowsB_alloc, t.maxB);
    sg::slice_kernel<R, S, sg::KCG><<<grid, 256, 0, c->stream>>>(A + k0, nb, L, len, nch, t.kblk, true, nbp,
                                                                 t.rowsB_alloc, sB, t.sigB, t.rowsB_alloc, t.maxB);
    sg::GramArgs a = {};
    a.gA = sA;
    a.gB = sB;
    a.rows_allocA = t.rowsA_alloc;
    a.rows_allocB = t.rowsB_alloc;
    a.ksteps = t.kblk / sg::BK;
    a.half_stride = nbp;
    a.sigA = t.sigA;
    a.sigB = t.sigB;
    a.sig_ldA = t.rowsA_alloc;
    a.sig_ldB = t.rowsB_alloc;
    a.maxA = t.maxA;
    a.maxB = t.maxB;
    a.rowsA = nb;
    a.rowsB = rowsB;
    a.tilesN = 2 * Tc;
    a.herm = 1;
    a.halves = 2;
    a.half_rows = nb;
    a.chunks_per_cta = cpc;
    a.nchunks = nch;
    a.accumulate = blk > 0;
    a.klen = len;
    a.part = (double*)t.part;
    a.st = c->d_status;
    if (cover) set_cover(a);
    if (blk == 0 && ns < nsplit) nsplit = ns;
    ktimer_begin(c);
    if (cover)
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG, true>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB, t.mapB32, a);
    else
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB, t.mapB32, a);
    ktimer_end(c);
    // psi^H psi: psi's planes (rows [0, nb) of B_ext, read through a map with the A box) as
    // the first operand; rows [nb, 128 Tr) of that box are zero or psi'' rows, whose output
    // rows (>= nb) are never stored
    sg::GramArgs a2 = a;
    a2.gA = sB;
    a2.rows_allocA = t.rowsB_alloc;
    a2.sigA = t.sigB;
    a2.sig_ldA = t.rowsB_alloc;
    a2.maxA = t.maxB;
    a2.part = (double*)t.part2;
    ktimer_begin(c);
    if (cover)
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG, true>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapBA, t.mapB, t.mapB32, a2);
    else
      sg::sliced_gram_kernel<S, ORD, false, false, sg::KCG>
          <<<dim3(tiles, ns), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapBA, t.mapB, t.mapB32, a2);
    ktimer_end(c);
    c->launches += 5;
  }
  const long long nn = (long long)nb * nb;
  tc_reduce_kernel<zd><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part, nsplit, nb, rowsB, nbp,
                                                                            c->dV, true, M1);
  tc_reduce_kernel<zd><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>((double*)t.part2, nsplit, nb, rowsB, nbp,
                                                                            c->dV, true, M2);
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "tensor-core complex gram pair launch");
}

// The rotation's first operand: A_ext[row][k] with k the contraction index, for the first
// nout columns m of C ([nb][nb]).  Real: A[m][n] = C[n][m].  Complex (C interleaved): rows
// m < nout give the real part of the output, A[m][2n] = Re C[n][m], A[m][2n+1] = -Im C[n][m];
// rows nout + m the imaginary part, A[nout+m][2n] = Im C[n][m], A[nout+m][2n+1] = Re C[n][m].
// Columns beyond the contraction and rows beyond the outputs are 0.
__global__ void rot_operand_kernel(const double* __restrict__ C, int nb, int nout, int cplx, double* __restrict__ A,
                                   long long Lc, int rows) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * Lc) return;
  const int row = (int)(e / Lc);
  const long long k = e % Lc;
  double v = 0.0;
  if (!cplx) {
    if (row < nout && k < nb) v = C[k * nb + row];
  } else if (row < 2 * nout && k < 2 * nb) {
    const int m = row % nout, n = (int)(k >> 1), re = (k & 1) == 0;
    const double cr = C[2 * ((long long)n * nb + m)], ci = C[2 * ((long long)n * nb + m) + 1];
    v = row < nout ? (re ? cr : -ci) : (re ? ci : cr);
  }
  A[e] = v;
}

// the transposed digits of psi for the rotation, one block of grid points r0 .. r0 + rcount
template <class R, int S, int KCH>
void rc_slice_psi_kc(pawfd_ctx* c, const R* psi, int nb, long long r0, int rcount, int nch) {
  TcScratch& t = c->tc;
  const bool cplx = is_complex(c);
  const long long K = (long long)c->K;
  cudaMemsetAsync(t.rotMaxB, 0x80, sizeof(int) * t.rot_rblk, c->stream);
  const int stiles = (rcount + sg::RT - 1) / sg::RT * nch;
  // 16-byte staging copies: band rows and the block start on 16-byte boundaries
  constexpr int v16 = 16 / (int)sizeof(R);
  const int per = cplx ? 2 : 1;
  const int vec16 = (per * K) % v16 == 0 && (per * r0) % v16 == 0 && (reinterpret_cast<uintptr_t>(psi) & 15) == 0;
  sg::slice_t_kernel<R, S, KCH><<<std::min(stiles, t.slice_t_ctas), 256, sg::slice_t_smem<R, KCH>(), c->stream>>>(
      psi, nb, K, cplx, r0, rcount, t.rot_Lc, (int)t.rot_rblk, (__nv_bfloat16*)t.rotSlicesB, t.rotSigB,
      (int)t.rot_rblk, t.rotMaxB, nch, vec16);
}

template <class R, int S>
void rc_slice_psi(pawfd_ctx* c, const R* psi, int nb, long long r0, int rcount, int nch) {
  if (c->tc.rot_kc == sg::KCG) rc_slice_psi_kc<R, S, sg::KCG>(c, psi, nb, r0, rcount, nch);
  else rc_slice_psi_kc<R, S, sg::KC>(c, psi, nb, r0, rcount, nch);
}

template <class R, int S, int ORD, int KCH>
int tc_rotate_kc(pawfd_ctx* c, const R* psi, int nb, const double* C, int nout, R* out) {
  TcScratch& t = c->tc;
  const bool cplx = is_complex(c);
  const int rowsA = cplx ? 2 * nout : nout;
  const long long Lk = (long long)nb * (cplx ? 2 : 1);
  const long long Lc = (Lk + KCH - 1) / KCH * KCH;
  const int nch = (int)(Lc / KCH);
  if (Lc > t.rot_Lc) return fail(c, PAWFD_EINVAL, "rotation scratch too small");
  const long long K = (long long)c->K;
  // operand A from C, then its digits
  rot_operand_kernel<<<(unsigned)((t.rot_rowsA_alloc * t.rot_Lc + 255) / 256), 256, 0, c->stream>>>(
      C, nb, nout, cplx, (double*)t.rotA, t.rot_Lc, t.rot_rowsA_alloc);
  cudaMemsetAsync(t.rotMaxA, 0x80, sizeof(int) * t.rot_rowsA_alloc, c->stream);
  {
    sg::slice_rg_kernel<double, S, KCH><<<(unsigned)(((rowsA + 7) / 8 * (long long)nch + 7) / 8), 256, 0, c->stream>>>(
        (const double*)t.rotA, rowsA, t.rot_Lc, Lk, nch, t.rot_Lc, false, 0, t.rot_rowsA_alloc,
        (__nv_bfloat16*)t.rotSlicesA, t.rotSigA, t.rot_rowsA_alloc, t.rotMaxA);
  }
  c->launches += 2;
  const int tilesM = (rowsA + sg::BM - 1) / sg::BM;
  // psi's digits of a single-block rotation may already be in place (rotate_slice_psi)
  const bool presliced = t.presliced_psi == (const void*)psi && t.presliced_nb == nb && t.rot_rblk >= K;
  t.presliced_psi = nullptr;
  for (long long r0 = 0; r0 < K; r0 += t.rot_rblk) {
    const int rcount = (int)std::min<long long>(t.rot_rblk, K - r0);
    if (!presliced) {
      rc_slice_psi_kc<R, S, KCH>(c, psi, nb, r0, rcount, nch);
      c->launches += 1;
    }
    sg::GramArgs a = {};
    a.gA = (const __nv_bfloat16*)t.rotSlicesA;
    a.gB = (const __nv_bfloat16*)t.rotSlicesB;
    a.rows_allocA = t.rot_rowsA_alloc;
    a.rows_allocB = (int)t.rot_rblk;
    a.ksteps = t.rot_Lc / sg::BK;
    a.sigA = t.rotSigA;
    a.sigB = t.rotSigB;
    a.sig_ldA = t.rot_rowsA_alloc;
    a.sig_ldB = (int)t.rot_rblk;
    a.maxA = t.rotMaxA;
    a.maxB = t.rotMaxB;
    a.rowsA = rowsA;
    a.rowsB = rcount;
    a.tilesN = (rcount + sg::BN - 1) / sg::BN;
    a.herm = 0;
    a.halves = 1;
    a.half_rows = rcount;
    a.chunks_per_cta = nch;
    a.nchunks = nch;
    a.accumulate = 0;
    a.part = nullptr;
    a.st = c->d_status;
    a.rotation = 1;
    a.rot_nb = nout;
    a.rot_cplx = cplx;
    a.rot_fp32 = sizeof(R) == 4;
    a.rot_K = K;
    a.rot_out = out + r0 * (cplx ? 2 : 1);
    a.rot_vec = !cplx && ((uintptr_t)a.rot_out % 16 == 0) && ((K * sizeof(R)) % 16 == 0);
    a.klen = Lk;
    a.rot_tiles = tilesM * a.tilesN;
    if (nch == 1)   // persistent CTAs, one per SM (the kernel's shared memory admits one)
      sg::sliced_gram_kernel<S, ORD, true, true, KCH>
          <<<dim3(std::min(a.rot_tiles, c->num_sms), 1), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB,
                                                                                                        t.mapB, a);
    else
      sg::sliced_gram_kernel<S, ORD, false, true, KCH>
          <<<dim3(a.rot_tiles, 1), sg::NTHREADS, sg::smem_bytes<S>(), c->stream>>>(t.mapA, t.mapB, t.mapB, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "tensor-core rotate launch");
}

template <class R, int S, int ORD>
int tc_rotate_impl(pawfd_ctx* c, const R* psi, int nb, const double* C, int nout, R* out) {
  if (c->tc.rot_kc == sg::KCG) return tc_rotate_kc<R, S, ORD, sg::KCG>(c, psi, nb, C, nout, out);
  return tc_rotate_kc<R, S, ORD, sg::KC>(c, psi, nb, C, nout, out);
}

}  // namespace

// The Gram digits of psi (the A operand of pawfd_gram_hs) for a following Gram pair of the
// same psi and nb, when the whole grid is one K block: enqueued early (on a stream ordered
// after psi is final) so that the Gram pair slices only H psi.  Returns false when the Gram
// would not use them.
bool gram_slice_psi(pawfd_ctx* c, const void* psi, int nb) {
  TcScratch& t = c->tc;
  const long long L = (long long)c->K;
  if (!c->use_tc || !t.ready || is_complex(c) || c->tc_kblk_chunks > 0 || t.kblk < L) return false;
  const int nch = (int)((L + sg::KCG - 1) / sg::KCG);
  cudaMemsetAsync(t.maxA, 0x80, sizeof(int) * t.rowsA_alloc, c->stream);
  if (is_fp32(c))
    sg::slice_kernel<float, 4, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
        (const float*)psi, nb, L, L, nch, t.kblk, false, 0, t.rowsA_alloc, (__nv_bfloat16*)t.slicesA, t.sigA,
        t.rowsA_alloc, t.maxA);
  else
    sg::slice_kernel<double, 7, sg::KCG><<<(unsigned)(((long long)nb * nch + 7) / 8), 256, 0, c->stream>>>(
        (const double*)psi, nb, L, L, nch, t.kblk, false, 0, t.rowsA_alloc, (__nv_bfloat16*)t.slicesA, t.sigA,
        t.rowsA_alloc, t.maxA);
  c->launches += 1;
  t.presliced_gram = psi;
  t.presliced_gram_nb = nb;
  return cudaGetLastError() == cudaSuccess;
}

// The digits of psi for a following rotation of the same psi and nb, when the rotation is one
// block of grid points: enqueued early (on any stream ordered after psi is final) so that the
// rotation skips them.  Returns false when the rotation would not use them.
bool rotate_slice_psi(pawfd_ctx* c, const void* psi, int nb) {
  TcScratch& t = c->tc;
  if (!c->use_tc || !t.ready || t.rot_rblk < (long long)c->K) return false;
  const long long Lk = (long long)nb * (is_complex(c) ? 2 : 1);
  const long long Lc = (Lk + t.rot_kc - 1) / t.rot_kc * t.rot_kc;
  if (Lc > t.rot_Lc) return false;
  const int nch = (int)(Lc / t.rot_kc);
  if (is_fp32(c)) rc_slice_psi<float, 4>(c, (const float*)psi, nb, 0, (int)c->K, nch);
  else rc_slice_psi<double, 7>(c, (const double*)psi, nb, 0, (int)c->K, nch);
  c->launches += 1;
  t.presliced_psi = psi;
  t.presliced_nb = nb;
  return cudaGetLastError() == cudaSuccess;
}

int launch_rotate_tc(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out, int nout) {
  if (!c->tc.ready) return fail(c, PAWFD_EINVAL, "tensor-core scratch not set up");
  if (is_fp32(c)) return tc_rotate_impl<float, 4, 4>(c, (const float*)psi, nb, (const double*)C, nout, (float*)out);
  return tc_rotate_impl<double, 7, 6>(c, (const double*)psi, nb, (const double*)C, nout, (double*)out);
}

// Hermitian Grams psi^H B and psi^H psi from one slicing of psi (false when this form does not apply)
bool gram_pair_tc(pawfd_ctx* c, const void* psi, const void* B, int nb, void* M1, void* M2, int* rc) {
  if (!c->tc.ready) return false;
  if (is_complex(c)) {
    if (is_fp32(c)) *rc = tc_gram_pair_cplx_impl<float, 4, 4>(c, (const float*)psi, (const float*)B, nb, (zd*)M1, (zd*)M2);
    else *rc = tc_gram_pair_cplx_impl<double, 7, 6>(c, (const double*)psi, (const double*)B, nb, (zd*)M1, (zd*)M2);
    return true;
  }
  if (is_fp32(c)) *rc = tc_gram_pair_impl<float, 4, 4>(c, (const float*)psi, (const float*)B, nb, (double*)M1, (double*)M2);
  else *rc = tc_gram_pair_impl<double, 7, 6>(c, (const double*)psi, (const double*)B, nb, (double*)M1, (double*)M2);
  return true;
}

int launch_gram_tc(pawfd_ctx* c, const void* A, const void* B, int nb, void* M, bool hermitian) {
  if (!c->tc.ready) return fail(c, PAWFD_EINVAL, "tensor-core Gram scratch not set up");
  if (is_fp32(c)) return tc_gram_impl<float, 4, 4>(c, (const float*)A, (const float*)B, nb, M, hermitian);
  return tc_gram_impl<double, 7, 6>(c, (const double*)A, (const double*)B, nb, M, hermitian);
}

// TMA descriptor of a row-major digit-plane buffer (S planes, K steps of rows x 16 values):
// boxes of 16 values x box_rows x S planes, 32-byte swizzle (the layout the tensor core reads
// through smem_desc(..., 32)); rows past the allocation read as zero.
int encode_slice_map(pawfd_ctx* c, CUtensorMap* map, void* base, int rows, long long Lp, int S, int box_rows,
                     int box_planes = 0) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(c, PAWFD_EDEVICE, "cuTensorMapEncodeTiled not available");
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  // row-major digit planes in K steps (sg::plane_offset_rm): dims (value in step, row, step, plane)
  const cuuint64_t ks = (cuuint64_t)(Lp / sg::BK);
  cuuint64_t dims[4] = {(cuuint64_t)sg::BK, (cuuint64_t)rows, ks, (cuuint64_t)S};
  cuuint64_t strides[3] = {(cuuint64_t)sg::BK * 2, (cuuint64_t)rows * sg::BK * 2, ks * rows * sg::BK * 2};
  cuuint32_t box[4] = {(cuuint32_t)sg::BK, (cuuint32_t)box_rows, 1, (cuuint32_t)(box_planes > 0 ? box_planes : S)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, PAWFD_EDEVICE, "cuTensorMapEncodeTiled failed");
  return PAWFD_OK;
}

// Scratch and TMA descriptors, sized for max_bands and one K block.
int setup_tc(pawfd_ctx* c) {
  TcScratch& t = c->tc;
  const int nb = c->max_bands;
  const bool cplx = is_complex(c);
  const int S = is_fp32(c) ? 4 : 7;
  const long long L = (long long)c->K * (cplx ? 2 : 1);
  t.rowsA_alloc = (nb + sg::BM - 1) / sg::BM * sg::BM;
  // complex: the swapped half starts at row nbp (a multiple of 8) and has its own column tiles
  const int nbp = (nb + 7) / 8 * 8, tcn = (nb + sg::BN - 1) / sg::BN;
  t.rowsB_alloc = cplx ? nbp + tcn * sg::BN : tcn * sg::BN;
  // K block: 256 chunks by default, or as many as the two operands' digit planes fit in the
  // requested scratch size; never longer than the padded row
  const long long Lpad = (L + sg::KCG - 1) / sg::KCG * sg::KCG;
  long long kblk = 256LL * sg::KCG;
  if (c->tc_scratch_mb > 0) {
    const long long per_value = (long long)S * (t.rowsA_alloc + t.rowsB_alloc) * 2;
    kblk = std::max<long long>(sg::KCG, ((long long)c->tc_scratch_mb << 20) / per_value / sg::KCG * sg::KCG);
  }
  t.kblk = std::min<long long>(kblk, Lpad);
  const size_t sa = (size_t)S * t.rowsA_alloc * t.kblk * 2, sb = (size_t)S * t.rowsB_alloc * t.kblk * 2;
  const int nchunks = (int)(t.kblk / sg::KC);
  const int rowsB = cplx ? nbp + nb : nb;
  const int tiles_min = pair_tiles(nb, cplx);
  const int nsplit = gram_splits(tiles_min, (int)(t.kblk / sg::KCG), c->num_sms);
  t.part_bytes = (size_t)nsplit * nb * rowsB * sizeof(double);
  int rc = check_cuda(c, cudaMalloc(&t.slicesA, sa), "cudaMalloc tc slices");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.slicesB, sb), "cudaMalloc tc slices");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.sigA, sizeof(int) * nchunks * t.rowsA_alloc), "cudaMalloc");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.sigB, sizeof(int) * nchunks * t.rowsB_alloc), "cudaMalloc");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.part, t.part_bytes), "cudaMalloc tc partials");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.part2, t.part_bytes), "cudaMalloc tc partials");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.maxA, sizeof(int) * t.rowsA_alloc), "cudaMalloc");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.maxB, sizeof(int) * t.rowsB_alloc), "cudaMalloc");
  if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  // rows beyond nb (and the imaginary half's padding) are never sliced: keep them zero
  rc = check_cuda(c, cudaMemset(t.slicesA, 0, sa), "memset");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(t.slicesB, 0, sb), "memset");
  if (rc != PAWFD_OK) return rc;
  rc = encode_slice_map(c, &t.mapA, t.slicesA, t.rowsA_alloc, t.kblk, S, sg::BM);
  if (rc == PAWFD_OK) rc = encode_slice_map(c, &t.mapB, t.slicesB, t.rowsB_alloc, t.kblk, S, sg::BN);
  if (rc == PAWFD_OK) rc = encode_slice_map(c, &t.mapAB, t.slicesA, t.rowsA_alloc, t.kblk, S, sg::BN);
  if (rc == PAWFD_OK) rc = encode_slice_map(c, &t.mapBA, t.slicesB, t.rowsB_alloc, t.kblk, S, sg::BM);
  if (rc == PAWFD_OK) rc = encode_slice_map(c, &t.mapB32, t.slicesB, t.rowsB_alloc, t.kblk, S, sg::CB);
  if (rc == PAWFD_OK) rc = encode_slice_map(c, &t.mapAB32, t.slicesA, t.rowsA_alloc, t.kblk, S, sg::CB);
  if (rc == PAWFD_OK) {
    const cudaFuncAttribute smem_attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    // the Gram (row-major planes, TMA maps) and the rotation (core-matrix planes, bulk copies;
    // persistent one-chunk form and general form)
    const void* fns7[] = {(const void*)sg::sliced_gram_kernel<7, 6, false, false, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<7, 6, true, true, sg::KC>,
                          (const void*)sg::sliced_gram_kernel<7, 6, false, true, sg::KC>,
                          (const void*)sg::sliced_gram_kernel<7, 6, true, true, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<7, 6, false, true, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<7, 6, false, false, sg::KCG, true>};
    const void* fns4[] = {(const void*)sg::sliced_gram_kernel<4, 4, false, false, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<4, 4, true, true, sg::KC>,
                          (const void*)sg::sliced_gram_kernel<4, 4, false, true, sg::KC>,
                          (const void*)sg::sliced_gram_kernel<4, 4, true, true, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<4, 4, false, true, sg::KCG>,
                          (const void*)sg::sliced_gram_kernel<4, 4, false, false, sg::KCG, true>};
    for (int f = 0; f < 6 && rc == PAWFD_OK; ++f)
      rc = check_cuda(c, cudaFuncSetAttribute(S == 7 ? fns7[f] : fns4[f], smem_attr,
                                              S == 7 ? sg::smem_bytes<7>() : sg::smem_bytes<4>()),
                      "smem attribute");
  }
  // rotation scratch: operand A (from C) and its digits, digits of a block of grid points
  if (rc == PAWFD_OK) {
    const long long Lk = (long long)nb * (cplx ? 2 : 1);
    t.rot_kc = Lk > sg::KC ? sg::KCG : sg::KC;
    t.rot_Lc = (Lk + t.rot_kc - 1) / t.rot_kc * t.rot_kc;
    t.rot_rowsA_alloc = ((cplx ? 2 * nb : nb) + sg::BM - 1) / sg::BM * sg::BM;
    const long long Kpad = ((long long)c->K + sg::BN - 1) / sg::BN * sg::BN;
    // bytes of grid-point digits per block
    const long long budget = c->tc_scratch_mb > 0 ? ((long long)c->tc_scratch_mb << 20) : (512ll << 20);
    long long rblk = budget / ((long long)S * t.rot_Lc * 2) / sg::BN * sg::BN;
    t.rot_rblk = std::max<long long>(sg::BN, std::min(rblk, Kpad));
    const int nchr = (int)(t.rot_Lc / t.rot_kc);
    const size_t a_bytes = sizeof(double) * t.rot_rowsA_alloc * t.rot_Lc;
    const size_t sa_bytes = (size_t)S * t.rot_rowsA_alloc * t.rot_Lc * 2;
    const size_t sb_bytes = (size_t)S * t.rot_rblk * t.rot_Lc * 2;
    rc = check_cuda(c, cudaMalloc(&t.rotA, a_bytes), "cudaMalloc rot");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotSlicesA, sa_bytes), "cudaMalloc rot");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotSlicesB, sb_bytes), "cudaMalloc rot");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotSigA, sizeof(int) * nchr * t.rot_rowsA_alloc), "cudaMalloc");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotSigB, sizeof(int) * nchr * t.rot_rblk), "cudaMalloc");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotMaxA, sizeof(int) * t.rot_rowsA_alloc), "cudaMalloc");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&t.rotMaxB, sizeof(int) * t.rot_rblk), "cudaMalloc");
    if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
    // persistent transposing slicer: as many CTAs as fit at once
    if (rc == PAWFD_OK) {
      const bool lk = t.rot_kc == sg::KCG;
      const void* fn = S == 7 ? (lk ? (const void*)sg::slice_t_kernel<double, 7, sg::KCG>
                                    : (const void*)sg::slice_t_kernel<double, 7, sg::KC>)
                              : (lk ? (const void*)sg::slice_t_kernel<float, 4, sg::KCG>
                                    : (const void*)sg::slice_t_kernel<float, 4, sg::KC>);
      const int smem = S == 7 ? (lk ? sg::slice_t_smem<double, sg::KCG>() : sg::slice_t_smem<double, sg::KC>())
                              : (lk ? sg::slice_t_smem<float, sg::KCG>() : sg::slice_t_smem<float, sg::KC>());
      rc = check_cuda(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "smem attribute");
      int per_sm = 0;
      if (rc == PAWFD_OK)
        rc = check_cuda(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem), "occupancy");
      t.slice_t_ctas = std::max(1, per_sm) * c->num_sms;
    }
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(t.rotSlicesA, 0, sa_bytes), "memset");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(t.rotSlicesB, 0, sb_bytes), "memset");
  }
  t.ready = rc == PAWFD_OK;
  return rc;
}

void free_tc(pawfd_ctx* c) {
  TcScratch& t = c->tc;
  void* p[] = {t.slicesA, t.slicesB, t.sigA, t.sigB, t.part, t.part2, t.maxA, t.maxB,
               t.rotA, t.rotSlicesA, t.rotSlicesB, t.rotSigA, t.rotSigB, t.rotMaxA, t.rotMaxB};
  for (void* q : p)
    if (q) cudaFree(q);
  t = TcScratch();
}

}  // namespace pawfd
