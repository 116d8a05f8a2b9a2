// stencil_ring.cu -- kinetic + local kernel for FP32 real band arrays, fed by bulk async copies.
//
// Same operator as stencil.cu (order-6 central second difference per axis, periodic wrap,
// fused local potential; Eq. (dh) of the PAW section).  In the mixed form this kernel is
// bound by HBM bandwidth (8 bytes per point-band), so the design keeps bytes in flight and
// spends few instructions per point:
//
//  * a CTA owns BY full x rows (N1 points, N1 % 4 == 0) of one band and marches along z;
//  * one producer warp brings every z plane of the tile plus 3 halo rows on each side into a
//    ring of RING shared-memory planes with cp.async.bulk row copies (one 16-byte-aligned row
//    per copy from any wrapped source row, so the periodic y wrap costs nothing); a "full"
//    mbarrier per slot counts the bytes in, an "empty" mbarrier per slot counts the consumer
//    warps out, so there is no CTA-wide barrier in the z loop and warps drift freely;
//  * consumer threads compute 4 consecutive x points each: x neighbours wrap inside the staged
//    row, y neighbours come from the plane, and the +-3 z neighbours from a per-thread register
//    queue fed by one shared-memory read per plane; the z loop is unrolled seven times so the
//    queue rotates by renaming rather than by moves;
//  * y and z terms use Blackwell's packed FP32x2 add / FMA on aligned register pairs, in the
//    same per-point operation order as the float4 kernel (bitwise-equal outputs);
//  * every wait is bounded; a stall is reported through the context's status word, and the
//    producer waits (bounded) for its copies in flight before it exits.
#include <algorithm>

#include "pawfd_internal.cuh"
#include "tc_common.cuh"

namespace pawfd {
namespace {

constexpr int PAD = 4;           // floats of padding after each staged row

struct RingArgs {
  int n1, n2, n3, n1v, pitch;
  long long K;
  float wx[3], wy[3], wz[3];
  const float* vshift;
  int zchunk, nzc, by, ncw;
  DeviceStatus* st;
  float* cpy;            // optional copy of psi (first band of this launch), or null
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

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

template <int R>
struct Consumer {
  const float* ring;
  uint64_t* full;
  uint64_t* empty;
  int own;               // offset of this thread's first row (4 points) in a staged plane
  int offL, offR;        // x neighbours (float4 to the left / right, wrapped) relative to own
  int plane_floats, pitch, n1;
  bool valid;            // the thread's rows lie inside the CTA's tile
  bool act[R];           // row r of the thread is a grid row (y < N2)
  float* dst;            // output at (z, y, x) of the current step, first row
  float* cpy;            // copy of psi at the same place, or null
  const float* v;        // shifted potential at (z + 1, y, x), first row (prefetched a step ahead)
  float4 vcur[R];        // shifted potential of the current step
  long long plane_stride;
};

// One z step for ring plane j (the queue's new entry z + 3); the centre plane is j - 3.
// Queue rotation B: q[(B + i) % 7][r] holds row r of plane z - 3 + i.
template <int B, int R, int RING>
__device__ __forceinline__ bool consume(Consumer<R>& c, const RingArgs& a, int j, int jend, float4 (&q)[7][R]) {
  const int s = (unsigned)j % RING, sc = (unsigned)(j - 3) % RING;
  // the potential of the next z step is loaded one step ahead (an L2 round trip per step)
  float4 vnext[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    vnext[r] = (c.act[r] && j + 1 < jend) ? __ldg((const float4*)(c.v + r * c.n1)) : make_float4(0.f, 0.f, 0.f, 0.f);
  const bool got = tc::mbar_wait(&c.full[s], ((unsigned)j / RING) & 1);
  if (!__all_sync(0xffffffffu, got)) return false;
  if (c.valid) {
    const float* N = c.ring + s * c.plane_floats + c.own;
#pragma unroll
    for (int r = 0; r < R; ++r) q[(B + 6) % 7][r] = *(const float4*)(N + r * c.pitch);
    const float* P = c.ring + sc * c.plane_floats + c.own;
    // rows -3 .. R + 2 of the centre plane relative to the first row; own rows from the queue
    float4 h[R + 6];
#pragma unroll
    for (int i = 0; i < R + 6; ++i) {
      const int rel = i - 3;
      if (rel >= 0 && rel < R) h[i] = q[(B + 3) % 7][rel];
      else h[i] = *(const float4*)(P + rel * c.pitch);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!c.act[r]) continue;
      const float4 C = h[r + 3];
      const float4 L = *(const float4*)(P + r * c.pitch + c.offL);
      const float4 Rt = *(const float4*)(P + r * c.pitch + c.offR);
      const float4 v = c.vcur[r];
      float2 acc0 = __fmul2_rn(lo2(v), lo2(C)), acc1 = __fmul2_rn(hi2(v), hi2(C));
      // x terms in scalar arithmetic: the shifted neighbour pairs are not aligned register pairs
      const float w[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, Rt.x, Rt.y, Rt.z, Rt.w};
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        acc0.x = fmaf(a.wx[m], w[5 + m] + w[3 - m], acc0.x);
        acc0.y = fmaf(a.wx[m], w[6 + m] + w[4 - m], acc0.y);
        acc1.x = fmaf(a.wx[m], w[7 + m] + w[5 - m], acc1.x);
        acc1.y = fmaf(a.wx[m], w[8 + m] + w[6 - m], acc1.y);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float4 yp = h[r + 4 + m], ym = h[r + 2 - m];
        const float2 wy2 = make_float2(a.wy[m], a.wy[m]);
        acc0 = __ffma2_rn(wy2, __fadd2_rn(lo2(yp), lo2(ym)), acc0);
        acc1 = __ffma2_rn(wy2, __fadd2_rn(hi2(yp), hi2(ym)), acc1);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float4 zp = q[(B + 4 + m) % 7][r], zm = q[(B + 2 - m + 7) % 7][r];
        const float2 wz2 = make_float2(a.wz[m], a.wz[m]);
        acc0 = __ffma2_rn(wz2, __fadd2_rn(lo2(zp), lo2(zm)), acc0);
        acc1 = __ffma2_rn(wz2, __fadd2_rn(hi2(zp), hi2(zm)), acc1);
      }
      *(float4*)(c.dst + r * c.n1) = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
      if (c.cpy) *(float4*)(c.cpy + r * c.n1) = C;
    }
  }
  c.dst += c.plane_stride;
  if (c.cpy) c.cpy += c.plane_stride;
  c.v += c.plane_stride;
#pragma unroll
  for (int r = 0; r < R; ++r) c.vcur[r] = vnext[r];
  // this warp is done with the centre plane: release its slot
  __syncwarp();
  if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&c.empty[sc]);
  return true;
}

template <int R>
constexpr int max_threads() {
  return R == 1 ? 512 : (R == 2 ? 512 : 384);
}

// 1-D block: a.ncw consumer warps (thread t -> rows R (t / N1v) .. + R - 1, float4 column
// t % N1v) and one producer warp.  Dynamic shared memory: RING planes of (BY + 6) rows x
// pitch floats.  BY is a multiple of R.
template <int R, int RING>
__global__ void __launch_bounds__(max_threads<R>(), 1)
    kinetic_local_ring_kernel(const float* __restrict__ psi, float* __restrict__ out, RingArgs a) {
  extern __shared__ __align__(128) float ring[];
  __shared__ uint64_t full[RING], empty[RING];
  const int tid = threadIdx.x;
  const int rows = a.by + 6;
  const int plane_floats = rows * a.pitch;
  const int Y0 = blockIdx.x * a.by;
  const int band = blockIdx.y / a.nzc, zc = blockIdx.y % a.nzc;
  const int z0 = zc * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.n3);
  const int nplanes = (z1 - z0) + 6;   // plane j is z0 - 3 + j

  if (tid == 0) {
    for (int s = 0; s < RING; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], a.ncw);
    }
    tc::mbar_fence_init();
  }
  __syncthreads();

  if (tid >= 32 * a.ncw) {
    // ---- producer warp ----
    const int lane = tid & 31;
    const float* src = psi + (long long)band * a.K;
    const uint32_t row_bytes = (uint32_t)a.n1 * 4u;
    int last = -1;
    bool ok = true;
    for (int j = 0; j < nplanes; ++j) {
      const int s = j % RING;
      if (j >= RING) {
        // every consumer warp has released plane j - RING
        const bool got = tc::mbar_wait(&empty[s], ((j / RING) - 1) & 1);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
      }
      if (lane == 0) tc::mbar_expect_tx(&full[s], row_bytes * rows);
      __syncwarp();
      const int zz = wrapr(z0 - 3 + j, a.n3);
      float* pl = ring + s * plane_floats;
      for (int r = lane; r < rows; r += 32) {
        const int gy = wrapr(Y0 - 3 + r, a.n2);
        bulk_copy(pl + r * a.pitch, src + ((long long)zz * a.n2 + gy) * a.n1, row_bytes, &full[s]);
      }
      last = j;
    }
    if (!ok && lane == 0) set_status(a.st, PAWFD_ETIMEDOUT, 2002);
    // the copies still in flight must land before the CTA may exit
    if (lane == 0)
      for (int p = max(0, last - RING + 1); p <= last; ++p) tc::mbar_wait(&full[p % RING], (p / RING) & 1);
    return;
  }

  // ---- consumer warps ----
  const int tr = tid / a.n1v, tx = tid % a.n1v;
  const int x = 4 * tx, y = Y0 + R * tr;
  Consumer<R> c;
  c.ring = ring;
  c.full = full;
  c.empty = empty;
  c.valid = R * tr < a.by;
#pragma unroll
  for (int r = 0; r < R; ++r) c.act[r] = c.valid && y + r < a.n2;
  c.pitch = a.pitch;
  c.n1 = a.n1;
  c.plane_floats = plane_floats;
  c.own = (min(R * tr, a.by - R) + 3) * a.pitch + x;
  c.offL = (x == 0 ? a.n1 - 4 : x - 4) - x;
  c.offR = (x + 4 == a.n1 ? 0 : x + 4) - x;
  c.plane_stride = (long long)a.n1 * a.n2;
  const long long g0 = ((long long)z0 * a.n2 + (c.act[0] ? y : 0)) * a.n1 + x;
  c.dst = out + (long long)band * a.K + g0;
  c.cpy = a.cpy ? a.cpy + (long long)band * a.K + g0 : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r)
    c.vcur[r] = c.act[r] ? __ldg((const float4*)(a.vshift + g0 + r * a.n1)) : make_float4(0.f, 0.f, 0.f, 0.f);
  c.v = a.vshift + g0 + c.plane_stride;

  float4 q[7][R];
  bool ok = true;
  // prime the queue with planes z0-3 .. z0+2 (j = 0 .. 5) in q[1] .. q[6]
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const bool got = tc::mbar_wait(&full[j], 0);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      break;
    }
    if (c.valid)
#pragma unroll
      for (int r = 0; r < R; ++r) q[j + 1][r] = *(const float4*)(ring + j * plane_floats + c.own + r * a.pitch);
  }
  // planes z0-3 .. z0-1 are never centre planes: release their slots
  __syncwarp();
  if (ok && (tid & 31) == 0)
    for (int s = 0; s < 3; ++s) tc::mbar_arrive(&empty[s]);
  // q[0] is free for the first step, which loads plane z0 + 3 into it
  int j = 6;
  const int jend = nplanes;
#define PAWFD_RING_STEP(B)                     \
  if (ok && j < jend) {                        \
    ok = consume<B, R, RING>(c, a, j, jend, q);      \
    ++j;                                       \
  }
  while (ok && j < jend) {
    PAWFD_RING_STEP(1)
    PAWFD_RING_STEP(2)
    PAWFD_RING_STEP(3)
    PAWFD_RING_STEP(4)
    PAWFD_RING_STEP(5)
    PAWFD_RING_STEP(6)
    PAWFD_RING_STEP(0)
  }
#undef PAWFD_RING_STEP
  if (!ok && (tid & 31) == 0) set_status(a.st, PAWFD_ETIMEDOUT, 2001);
}

template <int R, int RING>
int launch_ring(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy, RingArgs a, int rows_hint) {
  // rows per CTA: a multiple of R within the thread limit and ~100 KB of ring
  const int max_rows = R * ((max_threads<R>() - 32) / a.n1v);
  if (max_rows < R) return PAWFD_EINVAL;
  int by = std::min(rows_hint, max_rows);
  by = std::min(by, R * ((a.n2 + R - 1) / R));
  by = std::max(R, by / R * R);
  while (by > R && (size_t)RING * (by + 6) * a.pitch * 4 > 100 * 1024) by -= R;
  a.by = by;
  a.ncw = (a.n1v * (by / R) + 31) / 32;
  const size_t smem = (size_t)RING * (by + 6) * a.pitch * 4;
  if (smem > 200 * 1024) return PAWFD_EINVAL;
  const int gy = (a.n2 + by - 1) / by;
  long long want = (3ll * c->num_sms + (long long)gy * nb - 1) / ((long long)gy * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 15) / 16));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  int rc = check_cuda(c, cudaFuncSetAttribute(kinetic_local_ring_kernel<R, RING>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                      "ring smem attribute");
  if (rc != PAWFD_OK) return rc;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gy, nbl * a.nzc), block(32 * (a.ncw + 1));
    a.cpy = cpy ? cpy + (size_t)b0 * c->K : nullptr;
    kinetic_local_ring_kernel<R, RING><<<grid, block, smem, c->stream>>>(psi + (size_t)b0 * c->K,
                                                                    out + (size_t)b0 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local ring launch");
}

}  // namespace

// FP32 real band arrays with N1 % 4 == 0 and 8 <= N1 <= 3072; EINVAL when the shape does
// not qualify (the caller then uses another kernel).
int launch_kinetic_local_ring(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy) {
  if (c->dtype != PAWFD_R32 || c->n[0] % 4 != 0 || c->n[0] < 8 || c->n[0] > 3072) return PAWFD_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out | (uintptr_t)cpy) & 15) return PAWFD_EINVAL;
  RingArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.n1v = c->n[0] / 4;
  a.pitch = c->n[0] + PAD;
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = (float)(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = (float)(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = (float)(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  a.vshift = (const float*)c->d_vshift;
  a.st = c->d_status;
  // measured at 96^3 x 256 bands: 3 rows per thread and about 96 consumer threads per CTA
  // (several CTAs per SM, each with deep register reuse) beat every other combination
  const int yb = c->stencil_yblock > 0 ? c->stencil_yblock : 3;
  const int rows = c->stencil_rows > 0 ? c->stencil_rows : yb * std::max(1, (96 + a.n1v / 2) / a.n1v);
  const int depth = c->stencil_ring > 0 ? c->stencil_ring : 8;
  if (depth == 10) {
    switch (yb) {
      case 1: return launch_ring<1, 10>(c, psi, nb, out, cpy, a, rows);
      case 2: return launch_ring<2, 10>(c, psi, nb, out, cpy, a, rows);
      default: return launch_ring<3, 10>(c, psi, nb, out, cpy, a, rows);
    }
  }
  if (depth == 12) {
    switch (yb) {
      case 1: return launch_ring<1, 12>(c, psi, nb, out, cpy, a, rows);
      case 2: return launch_ring<2, 12>(c, psi, nb, out, cpy, a, rows);
      default: return launch_ring<3, 12>(c, psi, nb, out, cpy, a, rows);
    }
  }
  switch (yb) {
    case 1: return launch_ring<1, 8>(c, psi, nb, out, cpy, a, rows);
    case 2: return launch_ring<2, 8>(c, psi, nb, out, cpy, a, rows);
    default: return launch_ring<3, 8>(c, psi, nb, out, cpy, a, rows);
  }
}

}  // namespace pawfd
