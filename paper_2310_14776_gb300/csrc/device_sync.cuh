// device_sync.cuh -- the bounded grid barrier, the cluster barrier and the launch helper that
// the multi-CTA dense kernels (subspace solve, tridiagonal eigensolver) share.
#pragma once

#include <algorithm>

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
    const unsigned need = nblocks + ld_volatile(&st->barrier_extra);
    const unsigned lim_ms = ld_volatile(&st->barrier_limit_ms);
    const unsigned long long limit = lim_ms ? 1000000ull * lim_ms : (unsigned long long)BARRIER_TIMEOUT_NS;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == need - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_volatile(&bar[1]) == gen) {
        if (global_ns() - t0 > limit) {
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

// Cluster-wide barrier (hardware).  Every CTA of the cluster reaches every call: the callers'
// control flow depends only on values that all CTAs compute identically.  The fence makes
// this CTA's global-memory writes visible before the arrive; readers use L2-only loads.
__device__ __forceinline__ void cluster_barrier() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// MODE 0: cooperative grid launch, software grid barrier (bounded); MODE 1: one thread-block
// cluster, hardware cluster barrier.  Returns false if the kernel must stop.
template <int MODE>
__device__ __forceinline__ bool all_barrier(unsigned* bar, unsigned nblocks, DeviceStatus* st, int id) {
  if (MODE == 1) {
    cluster_barrier();
    return true;
  }
  return grid_barrier(bar, nblocks, st, id);
}

// L2-only loads: data written by other CTAs of the same launch must not come from a stale L1
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zd ldcg(const zd* p) {
  const double2 v = __ldcg((const double2*)p);
  return zd{v.x, v.y};
}

// A kernel given a gate does nothing when the gate word is nonzero (a path of the subspace solve
// that the device decided against; the word is the same for every CTA of a launch).
__device__ __forceinline__ bool gated(const int* gate) { return gate && ld_volatile(gate) != 0; }

// Launch a kernel of the MODE 1 / MODE 0 pair: one thread-block cluster of up to `want` CTAs
// (non-portable sizes above 8 when allowed) when `cluster` is set and a cluster fits, else a
// cooperative grid of up to `want` co-resident CTAs.
template <class K1, class K0, class... Args>
int launch_cluster_or_grid(pawfd_ctx* c, K1 kernel1, K0 kernel0, int nthreads, size_t smem, int want, bool cluster,
                           const char* what, Args... args) {
  cudaStream_t s = c->stream;
  int rc;
  if (cluster) {
    int G = std::max(1, std::min(16, want));
    if (G > 8 && cudaFuncSetAttribute(kernel1, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      G = 8;
    }
    for (;; G = (G + 1) / 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(G);
      cfg.blockDim = dim3(nthreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = G;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kernel1, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nclusters = 0;
      }
      if (nclusters >= 1) {
        rc = check_cuda(c, cudaLaunchKernelEx(&cfg, kernel1, args...), what);
        c->launches += 1;
        return rc;
      }
      if (G == 1) break;
    }
  }
  int per_sm = 0;
  rc = check_cuda(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel0, nthreads, smem), "occupancy");
  if (rc != PAWFD_OK) return rc;
  const int G = std::max(1, std::min(want, per_sm * c->num_sms));
  rc = check_cuda(c, cudaMemsetAsync(c->d_barrier, 0, 2 * sizeof(unsigned), s), "barrier reset");
  if (rc != PAWFD_OK) return rc;
  void* argv[] = {&args...};
  rc = check_cuda(c, cudaLaunchCooperativeKernel((const void*)kernel0, dim3(G), dim3(nthreads), argv, smem, s), what);
  c->launches += 1;
  return rc;
}

}  // namespace
}  // namespace pawfd
