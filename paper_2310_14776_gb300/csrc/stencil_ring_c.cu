// stencil_ring_c.cu -- kinetic + local kernel for FP32 complex (Bloch) band arrays, fed by
// bulk async copies.
//
// The operator of stencil.cu (order-6 central second difference per axis, fused local
// potential; Eq. (dh) of the PAW section) with the Bloch condition
// psi(r + L_c e_c) = exp(i k_c L_c) psi(r).  In the mixed form of the Bloch workloads it is
// bound by HBM bandwidth (16 bytes per point-band: read psi, write the result), so it follows
// the FP32 real ring kernel (stencil_ring.cu):
//
//  * a CTA owns BY full x rows of one band and marches along z; one producer warp brings every
//    z plane of the tile plus 3 halo rows on each side into a ring of shared-memory planes with
//    cp.async.bulk row copies from the wrapped source rows; full / empty mbarriers per slot,
//    no CTA-wide barrier in the z loop;
//  * a consumer thread computes 2 consecutive complex points (one float4) of R rows.  The real
//    stencil weights act on the real and imaginary parts alike, so every term is a packed
//    FP32x2 FMA on an aligned (re, im) pair: the x neighbours at distance 1..3 are the halves
//    of the float4s at -2 .. +2 along the row;
//  * the copies are raw values of the periodic array; the Bloch phase of a crossed face is
//    applied by the consumer: exp(-i k_x L_x) or exp(i k_x L_x) on x neighbours that wrap
//    around the row, exp(+-i k_y L_y) on staged rows outside [0, N2), exp(+-i k_z L_z) on
//    queue entries from planes outside [0, N3) (N2, N3 >= 3, so a neighbour wraps at most
//    once);
//  * every wait is bounded; a stall is reported through the context's status word, and the
//    producer waits (bounded) for its copies in flight before it exits.
#include <algorithm>

#include "pawfd_internal.cuh"
#include "tc_common.cuh"

namespace pawfd {
namespace {

constexpr int PADC = 4;   // floats of padding after each staged row

struct RingCArgs {
  int n1, n2, n3, n1v, pitch;   // n1 complex points per row; n1v = n1 / 2 float4 per row
  long long K;
  float wx[3], wy[3], wz[3];
  float2 ph[3];                 // exp(i k_c L_c)
  const float* vshift;
  int zchunk, nzc, by, ncw;
  DeviceStatus* st;
  float* cpy;                   // optional copy of psi (first band of this launch), or null
};

__device__ __forceinline__ int wrapc(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ void bulk_copy_c(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// both complex values of a float4 times the complex factor f, with the rounding fixed by
// explicit intrinsics (no contraction choice left to the compiler), so that every tiling and
// instantiation of the kernel gives bitwise the same result
__device__ __forceinline__ float4 cmul4(float4 a, float2 f) {
  return make_float4(fmaf(a.x, f.x, -__fmul_rn(a.y, f.y)), fmaf(a.x, f.y, __fmul_rn(a.y, f.x)),
                     fmaf(a.z, f.x, -__fmul_rn(a.w, f.y)), fmaf(a.z, f.y, __fmul_rn(a.w, f.x)));
}

// the phase for a neighbour t faces away (t = -1, 0, +1): conj(ph), 1, ph
__device__ __forceinline__ float4 phase_by(float4 a, int t, float2 ph) {
  if (t == 0) return a;
  return cmul4(a, t > 0 ? ph : make_float2(ph.x, -ph.y));
}

template <int R>
struct ConsumerC {
  const float* ring;
  uint64_t* full;
  uint64_t* empty;
  int own;                    // float offset of this thread's first row (2 points) in a staged plane
  int offL, offLL, offR, offRR;   // float offsets of the float4 neighbours along the row (wrapped)
  int tL, tLL, tR, tRR;       // the faces those neighbours cross: -1, 0, +1
  int plane_floats, pitch, n1, n2, n3, y, z0;
  bool valid;                 // the thread's rows lie inside the CTA's tile
  bool act[R];                // row r of the thread is a grid row (y + r < N2)
  float* dst;                 // output at (z, y, x) of the current step, first row
  float* cpy;                 // copy of psi at the same place, or null
  const float* v;             // shifted potential at (z + 1, y, x), first row (prefetched a step ahead)
  float2 vcur[R];             // the potential of the two points of each row, this step
  long long plane_pts;        // points per z plane
};

// One z step for ring plane j (the queue's new entry, plane z + 3); the centre plane is j - 3.
// Queue rotation B: q[(B + i) % 7][r] holds row r of plane z - 3 + i, Bloch phase applied.
template <int B, int R, int RING>
__device__ __forceinline__ bool consume_c(ConsumerC<R>& c, const RingCArgs& a, int j, int jend,
                                          float4 (&q)[7][R]) {
  const int s = (unsigned)j % RING, sc = (unsigned)(j - 3) % RING;
  float2 vnext[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    vnext[r] = (c.act[r] && j + 1 < jend) ? __ldg((const float2*)(c.v + r * c.n1)) : make_float2(0.f, 0.f);
  const bool got = tc::mbar_wait(&c.full[s], ((unsigned)j / RING) & 1);
  if (!__all_sync(0xffffffffu, got)) return false;
  if (c.valid) {
    const int zu = c.z0 - 3 + j;
    const int t3 = zu < 0 ? -1 : (zu >= c.n3 ? 1 : 0);
    const float* N = c.ring + s * c.plane_floats + c.own;
#pragma unroll
    for (int r = 0; r < R; ++r) q[(B + 6) % 7][r] = phase_by(*(const float4*)(N + r * c.pitch), t3, a.ph[2]);
    const float* P = c.ring + sc * c.plane_floats + c.own;
    // rows -3 .. R + 2 of the centre plane relative to the first row: the thread's own grid
    // rows from the queue, the others staged (with the y phase of a wrapped row)
    float4 h[R + 6];
#pragma unroll
    for (int i = 0; i < R + 6; ++i) {
      const int rel = i - 3;
      if (rel >= 0 && rel < R && c.act[rel]) {
        h[i] = q[(B + 3) % 7][rel];
      } else {
        const int yu = c.y + rel;
        const int t2 = yu < 0 ? -1 : (yu >= c.n2 ? 1 : 0);
        h[i] = phase_by(*(const float4*)(P + rel * c.pitch), t2, a.ph[1]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!c.act[r]) continue;
      const float* row = P + r * c.pitch;
      const float4 C = h[r + 3];
      const float4 L = phase_by(*(const float4*)(row + c.offL), c.tL, a.ph[0]);
      const float4 LL = phase_by(*(const float4*)(row + c.offLL), c.tLL, a.ph[0]);
      const float4 Rt = phase_by(*(const float4*)(row + c.offR), c.tR, a.ph[0]);
      const float4 RR = phase_by(*(const float4*)(row + c.offRR), c.tRR, a.ph[0]);
      const float2 v = c.vcur[r];
      float2 acc0 = __fmul2_rn(make_float2(v.x, v.x), lo2(C));
      float2 acc1 = __fmul2_rn(make_float2(v.y, v.y), hi2(C));
      // x: point 0's neighbours at +-1, +-2, +-3 are C.hi | L.hi, Rt.lo | L.lo, Rt.hi | LL.hi;
      // point 1's are Rt.lo | C.lo, Rt.hi | L.hi, RR.lo | L.lo
      const float2 wx0 = make_float2(a.wx[0], a.wx[0]), wx1 = make_float2(a.wx[1], a.wx[1]),
                   wx2 = make_float2(a.wx[2], a.wx[2]);
      acc0 = __ffma2_rn(wx0, __fadd2_rn(hi2(C), hi2(L)), acc0);
      acc1 = __ffma2_rn(wx0, __fadd2_rn(lo2(Rt), lo2(C)), acc1);
      acc0 = __ffma2_rn(wx1, __fadd2_rn(lo2(Rt), lo2(L)), acc0);
      acc1 = __ffma2_rn(wx1, __fadd2_rn(hi2(Rt), hi2(L)), acc1);
      acc0 = __ffma2_rn(wx2, __fadd2_rn(hi2(Rt), hi2(LL)), acc0);
      acc1 = __ffma2_rn(wx2, __fadd2_rn(lo2(RR), lo2(L)), acc1);
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
      *(float4*)(c.dst + 2 * r * c.n1) = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
      if (c.cpy) *(float4*)(c.cpy + 2 * r * c.n1) = C;
    }
  }
  c.dst += 2 * c.plane_pts;
  if (c.cpy) c.cpy += 2 * c.plane_pts;
  c.v += c.plane_pts;
#pragma unroll
  for (int r = 0; r < R; ++r) c.vcur[r] = vnext[r];
  __syncwarp();
  if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&c.empty[sc]);
  return true;
}

// 1-D block: a.ncw consumer warps (thread t -> rows R (t / N1v) .. + R - 1, float4 column
// t % N1v) and one producer warp.  Dynamic shared memory: RING planes of (BY + 6) rows x pitch
// floats.  BY is a multiple of R.
constexpr int RC_THREADS = 384;   // consumers + the producer warp (register budget: 170 per thread)

template <int R, int RING>
__global__ void __launch_bounds__(RC_THREADS, 1)
    kinetic_local_ring_c_kernel(const float* __restrict__ psi, float* __restrict__ out, RingCArgs a) {
  extern __shared__ __align__(128) float ringc[];
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
    // ---- producer warp: raw rows of the periodic array (the consumers apply the phases) ----
    const int lane = tid & 31;
    const float* src = psi + (long long)band * 2 * a.K;
    const uint32_t row_bytes = (uint32_t)a.n1 * 8u;
    int last = -1;
    bool ok = true;
    for (int j = 0; j < nplanes; ++j) {
      const int s = j % RING;
      if (j >= RING) {
        const bool got = tc::mbar_wait(&empty[s], ((j / RING) - 1) & 1);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
      }
      if (lane == 0) tc::mbar_expect_tx(&full[s], row_bytes * rows);
      __syncwarp();
      const int zz = wrapc(z0 - 3 + j, a.n3);
      float* pl = ringc + s * plane_floats;
      for (int r = lane; r < rows; r += 32) {
        const int gy = wrapc(Y0 - 3 + r, a.n2);
        bulk_copy_c(pl + r * a.pitch, src + 2 * (((long long)zz * a.n2 + gy) * a.n1), row_bytes, &full[s]);
      }
      last = j;
    }
    if (!ok && lane == 0) set_status(a.st, PAWFD_ETIMEDOUT, 2003);
    if (lane == 0)
      for (int p = max(0, last - RING + 1); p <= last; ++p) tc::mbar_wait(&full[p % RING], (p / RING) & 1);
    return;
  }

  // ---- consumer warps ----
  const int tr = tid / a.n1v, tx = tid % a.n1v;
  const int x = 2 * tx, y = Y0 + R * tr;
  ConsumerC<R> c;
  c.ring = ringc;
  c.full = full;
  c.empty = empty;
  c.valid = R * tr < a.by;
#pragma unroll
  for (int r = 0; r < R; ++r) c.act[r] = c.valid && y + r < a.n2;
  c.pitch = a.pitch;
  c.n1 = a.n1;
  c.n2 = a.n2;
  c.n3 = a.n3;
  c.y = y;
  c.z0 = z0;
  c.plane_floats = plane_floats;
  c.own = (min(R * tr, a.by - R) + 3) * a.pitch + 4 * tx;
  const int iL = tx - 1, iLL = tx - 2, iR = tx + 1, iRR = tx + 2;
  c.tL = iL < 0 ? -1 : 0;
  c.tLL = iLL < 0 ? -1 : 0;
  c.tR = iR >= a.n1v ? 1 : 0;
  c.tRR = iRR >= a.n1v ? 1 : 0;
  c.offL = 4 * (wrapc(iL, a.n1v) - tx);
  c.offLL = 4 * (wrapc(iLL, a.n1v) - tx);
  c.offR = 4 * (wrapc(iR, a.n1v) - tx);
  c.offRR = 4 * (wrapc(iRR, a.n1v) - tx);
  c.plane_pts = (long long)a.n1 * a.n2;
  const long long g0 = ((long long)z0 * a.n2 + (c.act[0] ? y : 0)) * a.n1 + x;
  c.dst = out + (long long)band * 2 * a.K + 2 * g0;
  c.cpy = a.cpy ? a.cpy + (long long)band * 2 * a.K + 2 * g0 : nullptr;
#pragma unroll
  for (int r = 0; r < R; ++r)
    c.vcur[r] = c.act[r] ? __ldg((const float2*)(a.vshift + g0 + r * a.n1)) : make_float2(0.f, 0.f);
  c.v = a.vshift + g0 + c.plane_pts;

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
    if (c.valid) {
      const int zu = z0 - 3 + j;
      const int t3 = zu < 0 ? -1 : (zu >= a.n3 ? 1 : 0);
#pragma unroll
      for (int r = 0; r < R; ++r)
        q[j + 1][r] = phase_by(*(const float4*)(ringc + j * plane_floats + c.own + r * a.pitch), t3, a.ph[2]);
    }
  }
  // planes z0-3 .. z0-1 are never centre planes: release their slots
  __syncwarp();
  if (ok && (tid & 31) == 0)
    for (int s = 0; s < 3; ++s) tc::mbar_arrive(&empty[s]);
  int j = 6;
  const int jend = nplanes;
#define PAWFD_RINGC_STEP(B)                         \
  if (ok && j < jend) {                             \
    ok = consume_c<B, R, RING>(c, a, j, jend, q);   \
    ++j;                                            \
  }
  while (ok && j < jend) {
    PAWFD_RINGC_STEP(1)
    PAWFD_RINGC_STEP(2)
    PAWFD_RINGC_STEP(3)
    PAWFD_RINGC_STEP(4)
    PAWFD_RINGC_STEP(5)
    PAWFD_RINGC_STEP(6)
    PAWFD_RINGC_STEP(0)
  }
#undef PAWFD_RINGC_STEP
  if (!ok && (tid & 31) == 0) set_status(a.st, PAWFD_ETIMEDOUT, 2004);
}

template <int R, int RING>
int launch_ring_c(pawfd_ctx* c, const float* psi, int nb, float* out, float* cpy, RingCArgs a, int rows_hint) {
  const int max_rows = R * ((RC_THREADS - 32) / a.n1v);
  if (max_rows < R) return PAWFD_EINVAL;
  int by = std::min(rows_hint, max_rows);
  by = std::min(by, R * ((a.n2 + R - 1) / R));
  by = std::max(R, by / R * R);
  while (by > R && (size_t)RING * (by + 6) * a.pitch * 4 > 110 * 1024) by -= R;
  a.by = by;
  a.ncw = (a.n1v * (by / R) + 31) / 32;
  const size_t smem = (size_t)RING * (by + 6) * a.pitch * 4;
  if (smem > 200 * 1024) return PAWFD_EINVAL;
  const int gy = (a.n2 + by - 1) / by;
  long long want = (3ll * c->num_sms + (long long)gy * nb - 1) / ((long long)gy * nb);
  int nzc = (int)std::max(1ll, std::min<long long>(want, (a.n3 + 15) / 16));
  a.zchunk = (a.n3 + nzc - 1) / nzc;
  a.nzc = (a.n3 + a.zchunk - 1) / a.zchunk;
  int rc = check_cuda(c, cudaFuncSetAttribute(kinetic_local_ring_c_kernel<R, RING>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                      "complex ring smem attribute");
  if (rc != PAWFD_OK) return rc;
  const int bands_per_launch = std::max(1, 65535 / a.nzc);
  for (int b0 = 0; b0 < nb; b0 += bands_per_launch) {
    const int nbl = std::min(bands_per_launch, nb - b0);
    dim3 grid(gy, nbl * a.nzc), block(32 * (a.ncw + 1));
    a.cpy = cpy ? cpy + (size_t)b0 * 2 * c->K : nullptr;
    kinetic_local_ring_c_kernel<R, RING><<<grid, block, smem, c->stream>>>(psi + (size_t)b0 * 2 * c->K,
                                                                          out + (size_t)b0 * 2 * c->K, a);
    c->launches += 1;
  }
  return check_cuda(c, cudaGetLastError(), "kinetic_local complex ring launch");
}

}  // namespace

// FP32 complex band arrays (PAWFD_C64) with N1 even, 8 <= N1 <= 1536 and N2, N3 >= 3;
// PAWFD_EINVAL when the shape does not qualify (the caller then uses the general kernel).
int launch_kinetic_local_ring_c(pawfd_ctx* c, const zf* psi, int nb, zf* out, zf* cpy) {
  if (c->dtype != PAWFD_C64 || c->n[0] % 2 != 0 || c->n[0] < 8 || c->n[0] > 1536 || c->n[1] < 3 || c->n[2] < 3)
    return PAWFD_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out | (uintptr_t)cpy) & 15) return PAWFD_EINVAL;
  RingCArgs a;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.n1v = c->n[0] / 2;
  a.pitch = 2 * c->n[0] + PADC;
  a.K = (long long)c->K;
  const double wm[3] = {FD6_W1, FD6_W2, FD6_W3};
  for (int m = 0; m < 3; ++m) {
    a.wx[m] = (float)(-0.5 * wm[m] / (c->h[0] * c->h[0]));
    a.wy[m] = (float)(-0.5 * wm[m] / (c->h[1] * c->h[1]));
    a.wz[m] = (float)(-0.5 * wm[m] / (c->h[2] * c->h[2]));
  }
  for (int cc = 0; cc < 3; ++cc) {
    const double kl = c->k[cc] * c->cell[cc];
    a.ph[cc] = make_float2((float)cos(kl), (float)sin(kl));
  }
  a.vshift = (const float*)c->d_vshift;
  a.st = c->d_status;
  a.cpy = nullptr;
  const int yb = c->stencil_yblock > 0 ? c->stencil_yblock : 2;
  // measured at 144^3 (n1v = 72): two rows per thread and about 288 consumer threads per CTA
  // (1 CTA per SM at 156 registers) beat the other tilings and ring depths
  const int rows = c->stencil_rows > 0 ? c->stencil_rows : yb * std::max(1, 288 / a.n1v);
  const int depth = c->stencil_ring > 0 ? c->stencil_ring : 6;
  const float* p = (const float*)psi;
  float* o = (float*)out;
  float* cp = (float*)cpy;
  if (depth >= 8) {
    switch (yb) {
      case 1: return launch_ring_c<1, 8>(c, p, nb, o, cp, a, rows);
      case 3: return launch_ring_c<3, 8>(c, p, nb, o, cp, a, rows);
      default: return launch_ring_c<2, 8>(c, p, nb, o, cp, a, rows);
    }
  }
  switch (yb) {
    case 1: return launch_ring_c<1, 6>(c, p, nb, o, cp, a, rows);
    case 3: return launch_ring_c<3, 6>(c, p, nb, o, cp, a, rows);
    default: return launch_ring_c<2, 6>(c, p, nb, o, cp, a, rows);
  }
}

}  // namespace pawfd
