// gemm.cu -- band x band contractions over the grid (FP64 / complex FP64 path).
//
//   Gram:    M[n][m] = dV sum_r conj(A_n(r)) B_m(r)      (subspace matrices H_nm, S_nm)
//   Rotate:  out_m(r) = sum_n psi_n(r) C[n][m]           (rotation after the subspace solve)
//
// Both are dense contractions (Kohn-Sham section, SCF step 1; the paper's BLAS hot spots).
// On GB300 the FP64 rate is the same for the vector units and the DMMA tensor path, so the
// FP64 kernels are register-tiled DFMA GEMMs: 64 x 64 output tiles, 256 threads, 4 x 4
// outputs per thread strided by 16 so that every shared-memory read is conflict free.
// The Gram kernel splits the long grid dimension across CTAs and reduces the partial
// tiles in a fixed order, so the result is deterministic.
#include <algorithm>
#include <mutex>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int TM = 64, TK = 16, NT = 256;

// Output tile of this CTA.  HERM: only tiles on or above the diagonal are computed, listed
// row by row in blockIdx.x; otherwise blockIdx.y / blockIdx.x give the tile row / column.
template <bool HERM>
__device__ __forceinline__ void gram_tile(int nb, int* n0, int* m0) {
  if (!HERM) {
    *n0 = blockIdx.y * TM;
    *m0 = blockIdx.x * TM;
    return;
  }
  const int T = (nb + TM - 1) / TM;
  int t = blockIdx.x, row = 0;
  while (t >= T - row) {
    t -= T - row;
    ++row;
  }
  *n0 = row * TM;
  *m0 = (row + t) * TM;
}

template <class T, bool HERM = false>
__global__ void __launch_bounds__(NT) gram_partial_kernel(const T* __restrict__ A, const T* __restrict__ B, int nb,
                                                          long long K, long long kchunk, T* __restrict__ part) {
  __shared__ T As[TK][TM];
  __shared__ T Bs[TK][TM];
  int n0, m0;
  gram_tile<HERM>(nb, &n0, &m0);
  const long long k0 = (long long)blockIdx.z * kchunk;
  const long long k1 = min(K, k0 + kchunk);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int lrow = tid / 4, lk = (tid % 4) * 4;   // loader: 64 rows x 16 k, 4 consecutive k each
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
  const T* __restrict__ arow = A + (long long)(n0 + lrow) * K;
  const T* __restrict__ brow = B + (long long)(m0 + lrow) * K;
  const bool aok = n0 + lrow < nb, bok = m0 + lrow < nb;
  for (long long kk = k0; kk < k1; kk += TK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long k = kk + lk + e;
      As[lk + e][lrow] = (aok && k < k1) ? conjx(arow[k]) : zero<T>();
      Bs[lk + e][lrow] = (bok && k < k1) ? brow[k] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[j][ty + 16 * i];
        b[i] = Bs[j][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) fma_plain(acc[i][l], a[i], b[l]);
    }
    __syncthreads();
  }
  T* __restrict__ out = part + (long long)blockIdx.z * nb * nb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int n = n0 + ty + 16 * i, m = m0 + tx + 16 * l;
      if (n < nb && m < nb) out[(long long)n * nb + m] = acc[i][l];
    }
}

// Mixed-precision Gram partial for FP32 band arrays: products and sums in FP32 over runs of
// at most MIX_RUN grid points, then folded into FP64; partials written in FP64.
constexpr long long MIX_RUN = 4096;

template <class T, bool HERM>
__global__ void __launch_bounds__(NT) gram_partial_mixed_kernel(const T* __restrict__ A, const T* __restrict__ B,
                                                                int nb, long long K, long long kchunk,
                                                                wide_t<T>* __restrict__ part) {
  using W = wide_t<T>;
  __shared__ T As[TK][TM];
  __shared__ T Bs[TK][TM];
  int n0, m0;
  gram_tile<HERM>(nb, &n0, &m0);
  const long long k0 = (long long)blockIdx.z * kchunk;
  const long long k1 = min(K, k0 + kchunk);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int lrow = tid / 4, lk = (tid % 4) * 4;
  T acc[4][4];
  W wacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = zero<T>();
      wacc[i][j] = zero<W>();
    }
  const T* __restrict__ arow = A + (long long)(n0 + lrow) * K;
  const T* __restrict__ brow = B + (long long)(m0 + lrow) * K;
  const bool aok = n0 + lrow < nb, bok = m0 + lrow < nb;
  long long run_end = k0 + MIX_RUN;
  for (long long kk = k0; kk < k1; kk += TK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long k = kk + lk + e;
      As[lk + e][lrow] = (aok && k < k1) ? conjx(arow[k]) : zero<T>();
      Bs[lk + e][lrow] = (bok && k < k1) ? brow[k] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[j][ty + 16 * i];
        b[i] = Bs[j][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) fma_plain(acc[i][l], a[i], b[l]);
    }
    __syncthreads();
    if (kk + TK >= run_end || kk + TK >= k1) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          wacc[i][l] += widen(acc[i][l]);
          acc[i][l] = zero<T>();
        }
      run_end += MIX_RUN;
    }
  }
  W* __restrict__ out = part + (long long)blockIdx.z * nb * nb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int n = n0 + ty + 16 * i, m = m0 + tx + 16 * l;
      if (n < nb && m < nb) out[(long long)n * nb + m] = wacc[i][l];
    }
}

// Hermitian result from the upper-triangular partials: M[n][m] for n <= m, mirrored below,
// diagonal made exactly real.
__device__ __forceinline__ double herm_diag(double v) { return v; }
__device__ __forceinline__ zd herm_diag(zd v) { return zd{v.re, 0.0}; }

template <class T>
__global__ void gram_reduce_herm_kernel(const T* __restrict__ part, int nsplit, int nb, double dV,
                                        T* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)nb * nb;
  if (e >= nn) return;
  const int n = (int)(e / nb), m = (int)(e % nb);
  if (m < n) return;
  T s = zero<T>();
  for (int p = 0; p < nsplit; ++p) s += part[p * nn + e];
  s = dV * s;
  if (m == n) {
    M[e] = herm_diag(s);
  } else {
    M[e] = s;
    M[(long long)m * nb + n] = conjx(s);
  }
}

template <class T>
__global__ void gram_reduce_kernel(const T* __restrict__ part, int nsplit, int nb, double dV, T* __restrict__ M) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nn = (long long)nb * nb;
  if (e >= nn) return;
  T s = zero<T>();
  for (int p = 0; p < nsplit; ++p) s += part[p * nn + e];
  M[e] = dV * s;
}

template <class T>
__global__ void __launch_bounds__(NT) rotate_kernel(const T* __restrict__ psi, const wide_t<T>* __restrict__ C,
                                                    int nb, int nout, long long K, T* __restrict__ out) {
  __shared__ T Cs[TK][TM];
  __shared__ T Ps[TK][TM];
  const long long r0 = (long long)blockIdx.x * TM;
  const int m0 = blockIdx.y * TM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero<T>();
  for (int n0 = 0; n0 < nb; n0 += TK) {
    for (int s = tid; s < TK * TM; s += NT) {
      const int j = s / TM, i = s - j * TM;
      const int n = n0 + j;
      Cs[j][i] = (n < nb && m0 + i < nout) ? narrow<T>(C[(long long)n * nb + m0 + i]) : zero<T>();
      Ps[j][i] = (n < nb && r0 + i < K) ? psi[(long long)n * K + r0 + i] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TK; ++j) {
      T cm[4], pr[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cm[i] = Cs[j][ty + 16 * i];
        pr[i] = Ps[j][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) fma_plain(acc[i][l], cm[i], pr[l]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int m = m0 + ty + 16 * i;
      const long long r = r0 + tx + 16 * l;
      if (m < nout && r < K) out[(long long)m * K + r] = acc[i][l];
    }
}

template <class T>
int gram_impl(pawfd_ctx* c, const T* A, const T* B, int nb, T* M, bool herm) {
  const long long K = (long long)c->K;
  const int T1 = (nb + TM - 1) / TM;
  const int tiles = herm ? T1 * (T1 + 1) / 2 : T1 * T1;
  const size_t per = (size_t)nb * nb * sizeof(T);
  // about eight CTAs per SM, so that the split work spreads evenly over the SMs
  long long nsplit = std::max<long long>(1, (8ll * c->num_sms + tiles - 1) / tiles);
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, (long long)(c->gram_part_bytes / per)));
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, K / (4 * TK)));
  long long kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  T* part = (T*)c->d_gram_part;
  const long long nn = (long long)nb * nb;
  if (herm) {
    gram_partial_kernel<T, true><<<dim3(tiles, 1, (unsigned)nsplit), NT, 0, c->stream>>>(A, B, nb, K, kchunk, part);
    gram_reduce_herm_kernel<T><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(part, (int)nsplit, nb, c->dV,
                                                                                     M);
  } else {
    dim3 grid(T1, T1, (unsigned)nsplit);
    gram_partial_kernel<T><<<grid, NT, 0, c->stream>>>(A, B, nb, K, kchunk, part);
    gram_reduce_kernel<T><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(part, (int)nsplit, nb, c->dV, M);
  }
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "gram launch");
}

template <class T>
int rotate_impl(pawfd_ctx* c, const T* psi, int nb, const wide_t<T>* C, int nout, T* out) {
  const long long K = (long long)c->K;
  dim3 grid((unsigned)((K + TM - 1) / TM), (nout + TM - 1) / TM);
  rotate_kernel<T><<<grid, NT, 0, c->stream>>>(psi, C, nb, nout, K, out);
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "rotate launch");
}

template <class T>
int gram_mixed_impl(pawfd_ctx* c, const T* A, const T* B, int nb, wide_t<T>* M, bool herm) {
  using W = wide_t<T>;
  const long long K = (long long)c->K;
  const int T1 = (nb + TM - 1) / TM;
  const int tiles = herm ? T1 * (T1 + 1) / 2 : T1 * T1;
  const size_t per = (size_t)nb * nb * sizeof(W);
  // about eight CTAs per SM, so that the split work spreads evenly over the SMs
  long long nsplit = std::max<long long>(1, (8ll * c->num_sms + tiles - 1) / tiles);
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, (long long)(c->gram_part_bytes / per)));
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, K / (4 * TK)));
  long long kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  W* part = (W*)c->d_gram_part;
  const long long nn = (long long)nb * nb;
  if (herm) {
    gram_partial_mixed_kernel<T, true><<<dim3(tiles, 1, (unsigned)nsplit), NT, 0, c->stream>>>(A, B, nb, K, kchunk,
                                                                                               part);
    gram_reduce_herm_kernel<W><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(part, (int)nsplit, nb, c->dV,
                                                                                     M);
  } else {
    gram_partial_mixed_kernel<T, false><<<dim3(T1, T1, (unsigned)nsplit), NT, 0, c->stream>>>(A, B, nb, K, kchunk,
                                                                                              part);
    gram_reduce_kernel<W><<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(part, (int)nsplit, nb, c->dV, M);
  }
  c->launches += 2;
  return check_cuda(c, cudaGetLastError(), "gram launch");
}

}  // namespace

int launch_gram(pawfd_ctx* c, const void* A, const void* B, int nb, void* M, bool hermitian) {
  if (c->use_tc) return launch_gram_tc(c, A, B, nb, M, hermitian);
  switch (c->dtype) {
    case PAWFD_C128: return gram_impl<zd>(c, (const zd*)A, (const zd*)B, nb, (zd*)M, hermitian);
    case PAWFD_R64: return gram_impl<double>(c, (const double*)A, (const double*)B, nb, (double*)M, hermitian);
    case PAWFD_C64: return gram_mixed_impl<zf>(c, (const zf*)A, (const zf*)B, nb, (zd*)M, hermitian);
    case PAWFD_R32: return gram_mixed_impl<float>(c, (const float*)A, (const float*)B, nb, (double*)M, hermitian);
  }
  return fail(c, PAWFD_EINVAL, "unsupported dtype");
}

int launch_gram_hs(pawfd_ctx* c, const void* psi, const void* hpsi, int nb, const void* P, void* Hnm, void* Snm) {
  int rc = PAWFD_OK;
  if (!(c->use_tc && gram_pair_tc(c, psi, hpsi, nb, Hnm, Snm, &rc))) {
    rc = launch_gram(c, psi, hpsi, nb, Hnm, true);
    if (rc == PAWFD_OK) rc = launch_gram(c, psi, psi, nb, Snm, true);
  }
  if (rc != PAWFD_OK) return rc;
  return launch_overlap_correction(c, P, nb, Snm);
}

int launch_rotate(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out, int nout) {
  if (nout < 0) nout = nb;
  if (c->use_tc) return launch_rotate_tc(c, psi, nb, C, out, nout);
  return dispatch_band(c, [&](auto tag) {
    using T = decltype(tag);
    return rotate_impl<T>(c, (const T*)psi, nb, (const wide_t<T>*)C, nout, (T*)out);
  });
}

}  // namespace pawfd

// ------------------------------------------------------------------------------------------
// Gram matrix without any device allocation (pawfd_gram_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a Gram matrix:
// an application whose device memory is entirely claimed by its own pool allocator, or a
// latency-bound serving loop that must never call cudaMalloc (which can synchronize the
// device and has no bounded latency).  They cannot create a pawfd context either, since
// pawfd_create allocates.  This entry point runs the same split-K kernels as pawfd_gram but
// keeps the partial tiles in a fixed, file-scope device array instead of context scratch.
//
// Cost of that choice: every GPU that loads this library holds NOALLOC_SCRATCH_BYTES for the
// array until the process exits, and all calls share the one array, so calls whose work
// overlaps on the GPU (different streams, threads or processes sharing a context) race on
// it.  Each call writes every partial entry it later reads, so nothing has to be cleared
// between calls; the array simply keeps the last call's partials.  The array's device
// address is looked up at the first call made with a given device and context current and
// cached for that pair; that first call should come before any stream capture.
// ------------------------------------------------------------------------------------------
namespace pawfd {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;   // 8 MiB of split-K partials
constexpr int NOALLOC_CACHE = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// The device address of g_noalloc_scratch, looked up once per (device, CUDA context).  The
// context is named by its process-unique ID (cuCtxGetId), never reused, so a device reset or
// another context made current leads to a fresh look-up instead of a stale address.
struct NoallocSlot {
  int dev = -1;
  unsigned long long ctx_id = 0;
  void* ptr = nullptr;
  int sms = 0;
};
std::mutex g_noalloc_mu;
NoallocSlot g_noalloc_slots[NOALLOC_CACHE];
int g_noalloc_next = 0;

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

// ID of the calling thread's current context (0 if none is current yet)
int current_context_id(unsigned long long* id) {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1)
      return PAWFD_EDEVICE;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2)
      return PAWFD_EDEVICE;
    get_current = (ctx_get_current_fn)f1;
    get_id = (ctx_get_id_fn)f2;
  }
  CUcontext ctx = nullptr;
  *id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS) return PAWFD_EDEVICE;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return PAWFD_EDEVICE;
  return PAWFD_OK;
}

// Device address of g_noalloc_scratch for the current device and context.  In host code the
// array's name only stands for the device symbol; its address must be asked from the runtime
// with that device current (set-up done once per device and context, then cached).
int noalloc_scratch(void** out, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAWFD_EDEVICE;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc != PAWFD_OK) return rc;
  if (id != 0) {
    for (const NoallocSlot& e : g_noalloc_slots)
      if (e.ptr && e.dev == dev && e.ctx_id == id) {
        *out = e.ptr;
        *sms = e.sms;
        return PAWFD_OK;
      }
  }
  // set-up: the runtime's symbol look-up also makes the device's primary context current if
  // no context was current yet
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PAWFD_EDEVICE;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PAWFD_EDEVICE;
  rc = current_context_id(&id);
  if (rc != PAWFD_OK) return rc;
  if (id != 0) {
    NoallocSlot& e = g_noalloc_slots[g_noalloc_next];
    g_noalloc_next = (g_noalloc_next + 1) % NOALLOC_CACHE;
    e.dev = dev;
    e.ctx_id = id;
    e.ptr = p;
    e.sms = n;
  }
  *out = p;
  *sms = n;
  return PAWFD_OK;
}

template <class T>
int gram_noalloc_impl(const T* A, const T* B, long long K, int nb, double dV, T* M, cudaStream_t stream,
                      T* part, int num_sms) {
  const int tiles = ((nb + TM - 1) / TM) * ((nb + TM - 1) / TM);
  const long long per = (long long)nb * nb * (long long)sizeof(T);
  long long nsplit = std::max<long long>(1, (2ll * num_sms + tiles - 1) / tiles);
  nsplit = std::min<long long>(nsplit, (long long)NOALLOC_SCRATCH_BYTES / per);
  nsplit = std::min<long long>(nsplit, std::max<long long>(1, K / (4 * TK)));
  long long kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  // launched through cudaLaunchKernel so that each launch's own status is checked, without
  // reading (and clearing) an error that earlier, unrelated work left in the runtime
  const dim3 grid((nb + TM - 1) / TM, (nb + TM - 1) / TM, (unsigned)nsplit);
  void* partial_args[] = {(void*)&A, (void*)&B, (void*)&nb, (void*)&K, (void*)&kchunk, (void*)&part};
  if (cudaLaunchKernel((const void*)&gram_partial_kernel<T, false>, grid, dim3(NT), partial_args, 0, stream) !=
      cudaSuccess)
    return PAWFD_EDEVICE;
  const long long nn = (long long)nb * nb;
  const T* cpart = part;
  int ns = (int)nsplit;
  void* reduce_args[] = {(void*)&cpart, (void*)&ns, (void*)&nb, (void*)&dV, (void*)&M};
  if (cudaLaunchKernel((const void*)&gram_reduce_kernel<T>, dim3((unsigned)((nn + 255) / 256)), dim3(256),
                       reduce_args, 0, stream) != cudaSuccess)
    return PAWFD_EDEVICE;
  return PAWFD_OK;
}

}  // namespace
}  // namespace pawfd

extern "C" int pawfd_gram_noalloc(const void* A, const void* B, long long K, int nb, int dtype, double dV, void* M,
                                  void* stream) {
  using namespace pawfd;
  if (!A || !B || !M || K < 1 || nb < 1) return PAWFD_EINVAL;
  if (dtype != PAWFD_R64 && dtype != PAWFD_C128) return PAWFD_EINVAL;
  const size_t elem = dtype == PAWFD_C128 ? sizeof(zd) : sizeof(double);
  if ((size_t)nb * (size_t)nb * elem > NOALLOC_SCRATCH_BYTES) return PAWFD_EINVAL;   // one partial must fit
  void* scratch = nullptr;
  int sms = 0;
  const int rc = noalloc_scratch(&scratch, &sms);
  if (rc != PAWFD_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PAWFD_C128)
    return gram_noalloc_impl<zd>((const zd*)A, (const zd*)B, K, nb, dV, (zd*)M, s, (zd*)scratch, sms);
  return gram_noalloc_impl<double>((const double*)A, (const double*)B, K, nb, dV, (double*)M, s,
                                   (double*)scratch, sms);
}
