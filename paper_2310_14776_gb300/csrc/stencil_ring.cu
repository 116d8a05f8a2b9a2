// stencil_ring.cu -- kinetic + local kernel for FP32 real band arrays, fed by bulk async copies.
//
// Same operator as stencil.cu (order-6 central second difference per axis, periodic wrap,
// fused local potential; Eq. (dh) of the PAW section).  In the mixed form this kernel is
// bound by HBM bandwidth (8 bytes per point-band), so the design keeps many bytes in flight:
//
//  * a CTA owns BY full x rows (N1 points, N1 % 4 == 0) of one band and marches along z;
//  * every z plane of the tile plus 3 halo rows on each side is brought into a ring of D
//    shared-memory planes by cp.async.bulk row copies (one 16-byte-aligned row of N1 floats
//    per copy, any wrapped source row, so the periodic y wrap costs nothing) completing on one
//    mbarrier per slot; planes z+1 .. z+D-1 are in flight while plane z is computed;
//  * x neighbours wrap inside the staged row, y neighbours are read from the plane, and the
//    +-3 z neighbours come from a per-thread register queue fed by one shared-memory read per
//    plane, so a thread reads 9 float4 from shared memory per 4 points;
//  * every wait is bounded; a stall is reported through the context's status word.
#include <algorithm>

#include "pawfd_internal.cuh"
#include "tc_common.cuh"

namespace pawfd {
namespace {

constexpr int RING = 8;   // planes in the shared-memory ring

struct RingArgs {
  int n1, n2, n3, n1v;
  long long K;
  float wx[3], wy[3], wz[3];
  const float* vshift;
  int zchunk, nzc, by;
  DeviceStatus* st;
};

__device__ __forceinline__ int wrapr(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
      : "memory");
}

// blockDim = (N1 / 4, BY); dynamic shared memory: RING planes of (BY + 6) rows x N1 floats
__global__ void __launch_bounds__(768) kinetic_local_ring_kernel(const float* __restrict__ psi,
                                                                  float* __restrict__ out, RingArgs a) {
  extern __shared__ __align__(128) float ring[];
  __shared__ uint64_t bar[RING];
  const int tx = threadIdx.x, ty = threadIdx.y, BY = a.by;
  const int tid = ty * blockDim.x + tx;
  const int rows = BY + 6;
  const int plane_floats = rows * a.n1;
  const int Y0 = blockIdx.x * BY;
  const int band = blockIdx.y / a.nzc, zc = blockIdx.y % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const int nz = z1 - z0;
  const float* __restrict__ src = psi + (long long)band * a.K;
  float* __restrict__ dst = out + (long long)band * a.K;
  const int x = 4 * tx, y = Y0 + ty;
  const bool active = y < a.n2;

  if (tid == 0) {
    for (int s = 0; s < RING; ++s) tc::mbar_init(&bar[s], 1);
    tc::mbar_fence_init();
  }
  __syncthreads();

  // plane p = z0 - 3 + j (j = 0 .. nz + 5) goes to slot j % RING; warp 0 issues its row copies
  const int nplanes = nz + 6;
  int last_issued = -1;   // meaningful in warp 0 only
  auto issue = [&](int j) {
    last_issued = j;
    if (tid < 32) {
      const int zz = wrapr(z0 - 3 + j, a.n3);
      float* pl = ring + (j % RING) * plane_floats;
      const uint32_t row_bytes = (uint32_t)a.n1 * 4u;
      if (tid == 0) tc::mbar_expect_tx(&bar[j % RING], row_bytes * rows);
      __syncwarp(__activemask());
      for (int r = tid; r < rows; r += 32) {
        const int gy = wrapr(Y0 - 3 + r, a.n2);
        bulk_copy(pl + r * a.n1, src + ((long long)zz * a.n2 + gy) * a.n1, row_bytes, &bar[j % RING]);
      }
    }
  };
  for (int j = 0; j < min(RING, nplanes); ++j) issue(j);

  float4 q[7];
  bool ok = true;
  int j_fail = 0;
  // prime the z queue with planes z0-3 .. z0+2 (j = 0 .. 5)
  for (int j = 0; j < 6; ++j) {
    const bool got = tc::mbar_wait(&bar[j % RING], (j / RING) & 1);
    if (!__syncthreads_and(got)) {
      ok = false;
      j_fail = j;
      break;
    }
    const float* pl = ring + (j % RING) * plane_floats;
    q[j + 1] = *(const float4*)(pl + (ty + 3) * a.n1 + x);
  }
  // planes z0-3 .. z0-1 (slots 0..2) now live only in registers: reuse their slots
  __syncthreads();
  if (ok)
    for (int j = RING; j < RING + 3 && j < nplanes; ++j) issue(j);
  for (int z = z0, j = 6; z < z1 && ok; ++z, ++j) {
    // plane z is j - 3, the new queue entry is plane z + 3 = j
    const bool got = tc::mbar_wait(&bar[j % RING], (j / RING) & 1);
    if (!__syncthreads_and(got)) {
      ok = false;
      j_fail = j;
      break;
    }
    const float* pj = ring + (j % RING) * plane_floats;
#pragma unroll
    for (int i = 0; i < 6; ++i) q[i] = q[i + 1];
    q[6] = *(const float4*)(pj + (ty + 3) * a.n1 + x);
    const float* P = ring + ((j - 3) % RING) * plane_floats;
    if (active) {
      const float* row = P + (ty + 3) * a.n1;
      const float4 L = *(const float4*)(row + (x == 0 ? a.n1 - 4 : x - 4));
      const float4 C = q[3];
      const float4 R = *(const float4*)(row + (x + 4 == a.n1 ? 0 : x + 4));
      const float w[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, R.x, R.y, R.z, R.w};
      float4 ym[3], yp[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        ym[m] = *(const float4*)(P + (ty + 2 - m) * a.n1 + x);
        yp[m] = *(const float4*)(P + (ty + 4 + m) * a.n1 + x);
      }
      const long long g = ((long long)z * a.n2 + y) * a.n1 + x;
      const float4 v = __ldg((const float4*)(a.vshift + g));
      float r[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float acc = (&v.x)[i] * w[4 + i];
        acc = fmaf(a.wx[0], w[5 + i] + w[3 + i], acc);
        acc = fmaf(a.wx[1], w[6 + i] + w[2 + i], acc);
        acc = fmaf(a.wx[2], w[7 + i] + w[1 + i], acc);
        acc = fmaf(a.wy[0], (&yp[0].x)[i] + (&ym[0].x)[i], acc);
        acc = fmaf(a.wy[1], (&yp[1].x)[i] + (&ym[1].x)[i], acc);
        acc = fmaf(a.wy[2], (&yp[2].x)[i] + (&ym[2].x)[i], acc);
        acc = fmaf(a.wz[0], (&q[4].x)[i] + (&q[2].x)[i], acc);
        acc = fmaf(a.wz[1], (&q[5].x)[i] + (&q[1].x)[i], acc);
        acc = fmaf(a.wz[2], (&q[6].x)[i] + (&q[0].x)[i], acc);
        r[i] = acc;
      }
      *(float4*)(dst + g) = make_float4(r[0], r[1], r[2], r[3]);
    }
    // every thread is past plane j - 3: its slot takes plane j - 3 + RING
    __syncthreads();
    if (j - 3 + RING < nplanes) issue(j - 3 + RING);
  }
  // after a stall: report it, and wait (bounded) for the copies this CTA still has in flight
  if (!ok && tid == 0) {
    set_status(a.st, PAWFD_ETIMEDOUT, 2001);
    for (int p = j_fail; p <= last_issued; ++p) tc::mbar_wait(&bar[p % RING], (p / RING) & 1);
  }
  __syncthreads();
}

}  // namespace

// FP32 real band arrays with N1 % 4 == 0 and 8 <= N1 <= 3072; EINVAL when the shape does
// not qualify (the caller then uses the general kernel).
int launch_kinetic_local_ring(pawfd_ctx* c, const float* psi, int nb, float* out) {
  if (c->dtype != PAWFD_R32 || c->n[0] % 4 != 0 || c->n[0] < 8 || c->n[0] > 3072) return PAWFD_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out) & 15) return PAWFD_EINVAL;
  RingArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.n1v = c->n[0] / 4;
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = (float)(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = (float)(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = (float)(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  a.vshift = (const float*)c->d_vshift;
  a.st = c->d_status;
  // rows per CTA: as many as fit 768 threads and ~100 KB of ring, at most 16
  int by = std::min(16, 768 / a.n1v);
  while (by > 1 && (size_t)RING * (by + 6) * a.n1 * 4 > 100 * 1024) --by;
  by = std::min(by, a.n2);
  a.by = by;
  const size_t smem = (size_t)RING * (by + 6) * a.n1 * 4;
  if (smem > 200 * 1024) return PAWFD_EINVAL;
  const int gy = (a.n2 + by - 1) / by;
  long long want = (3ll * c->num_sms + (long long)gy * nb - 1) / ((long long)gy * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 15) / 16));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  int rc = check_cuda(c, cudaFuncSetAttribute(kinetic_local_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem), "ring smem attribute");
  if (rc != PAWFD_OK) return rc;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gy, nbl * a.nzc), block(a.n1v, by);
    kinetic_local_ring_kernel<<<grid, block, smem, c->stream>>>(psi + (size_t)b0 * c->K, out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local ring launch");
}

}  // namespace pawfd
