// poisson.cu -- the Hartree potential of a density on the same grid (the Poisson solve of the
// Kohn-Sham section's potential update: "direct solvers based on Fourier transforms ... and
// iterative multi-grid solvers"; this is an iterative one).
//
// Solves  lap_FD v = -4 pi (rho - <rho>)  on the periodic grid, with the order-6 Laplacian of
// the kinetic stencil (T = -1/2 lap_FD, so the system is T v = 2 pi (rho - <rho>)), and
// returns the solution of zero mean.  T is symmetric positive definite on zero-mean grid
// functions, so conjugate gradients apply.  All scalars of the iteration stay on the device;
// the host reads the residual every CHECK iterations, and each batch of CHECK iterations is
// one CUDA graph launch.
#include <cmath>

#include "pawfd_internal.cuh"

using namespace pawfd;

namespace {

constexpr int PT = 256;           // threads per block
constexpr int PG = 296;           // blocks of the reductions (two per SM, fixed: deterministic sums)
constexpr int CHECK = 25;         // iterations between residual reads

// device scalars
enum { S_MEAN = 0, S_RR = 1, S_PAP = 2, S_ALPHA = 3, S_BETA = 4, S_BB = 5, S_RRNEW = 6, S_COUNT = 8 };

__device__ double pblock_sum(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < PT / 32; ++w) s += s_red[w];
  return s;
}

// part[block] = sum of a[r] b[r] (b = nullptr: sum of a[r]) over the block's grid-stride points
__global__ void __launch_bounds__(PT) dot_partial_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                         long long K, double* __restrict__ part) {
  __shared__ double s_red[PT / 32];
  double acc = 0.0;
  for (long long r = (long long)blockIdx.x * PT + threadIdx.x; r < K; r += (long long)gridDim.x * PT)
    acc += b ? a[r] * b[r] : a[r];
  const double s = pblock_sum(acc, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// the partial sums in a fixed order, then the scalar update of the iteration:
//   mode 0: scal[S_MEAN] = sum / K
//   mode 1: scal[S_BB] = scal[S_RR] = sum            (b.b = r.r at the start)
//   mode 2: scal[S_PAP] = sum, scal[S_ALPHA] = scal[S_RR] / sum
//   mode 3: scal[S_RRNEW] = sum, scal[S_BETA] = sum / scal[S_RR], scal[S_RR] = sum
__global__ void finish_kernel(const double* __restrict__ part, int G, long long K, int mode, double* __restrict__ scal) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += part[g];
  if (mode == 0) {
    scal[S_MEAN] = s / (double)K;
  } else if (mode == 1) {
    scal[S_BB] = s;
    scal[S_RR] = s;
  } else if (mode == 2) {
    scal[S_PAP] = s;
    scal[S_ALPHA] = s > 0.0 ? scal[S_RR] / s : 0.0;
  } else {
    scal[S_RRNEW] = s;
    scal[S_BETA] = scal[S_RR] > 0.0 ? s / scal[S_RR] : 0.0;
    scal[S_RR] = s;
  }
}

// b = 2 pi (rho - <rho>); x = 0; r = p = b
__global__ void cg_init_kernel(const double* __restrict__ rho, long long K, const double* __restrict__ scal,
                               double* __restrict__ x, double* __restrict__ r, double* __restrict__ p) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const double b = 2.0 * M_PI * (rho[i] - scal[S_MEAN]);
  x[i] = 0.0;
  r[i] = b;
  p[i] = b;
}

// x += alpha p; r -= alpha Ap; part[block] = the block's sum of r^2
__global__ void __launch_bounds__(PT) cg_xr_kernel(double* __restrict__ x, double* __restrict__ r,
                                                   const double* __restrict__ p, const double* __restrict__ Ap,
                                                   long long K, const double* __restrict__ scal,
                                                   double* __restrict__ part) {
  __shared__ double s_red[PT / 32];
  const double alpha = scal[S_ALPHA];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * PT + threadIdx.x; i < K; i += (long long)gridDim.x * PT) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    acc += ri * ri;
  }
  const double s = pblock_sum(acc, s_red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// p = r + beta p
__global__ void cg_p_kernel(double* __restrict__ p, const double* __restrict__ r, long long K,
                            const double* __restrict__ scal) {
  const double beta = scal[S_BETA];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (long long)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * p[i];
}

// v = x - <x>
__global__ void shift_kernel(const double* __restrict__ x, long long K, const double* __restrict__ scal,
                             double* __restrict__ v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) v[i] = x[i] - scal[S_MEAN];
}

}  // namespace

namespace {
int solve(pawfd_ctx* c, const double* rho, double* v, double tol, int maxiter, double* work, int* iters,
          double* resid);
}  // namespace

extern "C" int pawfd_poisson(pawfd_ctx* c, const double* rho, double* v, double tol, int maxiter, double* work,
                             int* iters, double* resid) {
  if (!c) return PAWFD_EINVAL;
  if (c->dtype != PAWFD_R64) return fail(c, PAWFD_EINVAL, "pawfd_poisson needs a real FP64 context");
  if (!c->free_operator) return fail(c, PAWFD_EINVAL, "pawfd_poisson needs a context with v = 0 and no atoms");
  if (!rho || !v || !work) return fail(c, PAWFD_EINVAL, "null array");
  if (!(tol > 0.0) || maxiter < 1) return fail(c, PAWFD_EINVAL, "tol must be > 0 and maxiter >= 1");
  // the solve runs on the context's auxiliary non-blocking stream (graph capture is not
  // possible on the legacy default stream), ordered after the work already on c->stream and
  // joined back to it at the end
  {
    const int e = ensure_aux_stream(c);
    if (e != PAWFD_OK) return e;
  }
  cudaStream_t caller = c->stream;
  int rc0 = check_cuda(c, cudaEventRecord(c->aux_fork, caller), "event record");
  if (rc0 == PAWFD_OK) rc0 = check_cuda(c, cudaStreamWaitEvent(c->aux_stream, c->aux_fork, 0), "stream wait");
  if (rc0 != PAWFD_OK) return rc0;
  c->stream = c->aux_stream;
  const int rcs = solve(c, rho, v, tol, maxiter, work, iters, resid);
  c->stream = caller;
  int rc1 = check_cuda(c, cudaEventRecord(c->aux_join, c->aux_stream), "event record");
  if (rc1 == PAWFD_OK) rc1 = check_cuda(c, cudaStreamWaitEvent(caller, c->aux_join, 0), "stream wait");
  return rcs != PAWFD_OK ? rcs : rc1;
}

namespace {
int solve(pawfd_ctx* c, const double* rho, double* v, double tol, int maxiter, double* work, int* iters,
          double* resid) {
  const long long K = (long long)c->K;
  double* x = work;
  double* r = work + K;
  double* p = work + 2 * K;
  double* Ap = work + 3 * K;
  double* part = work + 4 * K;          // PG partial sums
  double* scal = part + PG;             // S_COUNT scalars
  cudaStream_t s = c->stream;
  const unsigned eb = (unsigned)((K + PT - 1) / PT);
  dot_partial_kernel<<<PG, PT, 0, s>>>(rho, nullptr, K, part);
  finish_kernel<<<1, 32, 0, s>>>(part, PG, K, 0, scal);
  cg_init_kernel<<<eb, PT, 0, s>>>(rho, K, scal, x, r, p);
  dot_partial_kernel<<<PG, PT, 0, s>>>(r, r, K, part);
  finish_kernel<<<1, 32, 0, s>>>(part, PG, K, 1, scal);
  c->launches += 5;
  int rc = check_cuda(c, cudaGetLastError(), "poisson launch");
  double h[S_COUNT] = {};
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s), "copy");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamSynchronize(s), "sync");
  if (rc != PAWFD_OK) return rc;
  const double bnorm = std::sqrt(h[S_BB]);
  double rnorm = bnorm;
  int k = 0;
  // one iteration: Ap = T p, alpha, x and r, r.r and beta, p
  auto iteration = [&]() {
    int e = launch_kinetic_local(c, p, 1, Ap);
    dot_partial_kernel<<<PG, PT, 0, s>>>(p, Ap, K, part);
    finish_kernel<<<1, 32, 0, s>>>(part, PG, K, 2, scal);
    cg_xr_kernel<<<PG, PT, 0, s>>>(x, r, p, Ap, K, scal, part);
    finish_kernel<<<1, 32, 0, s>>>(part, PG, K, 3, scal);
    cg_p_kernel<<<PG, PT, 0, s>>>(p, r, K, scal);
    c->launches += 5;
    return e;
  };
  // CHECK iterations captured once into a CUDA graph (the pointers do not change between
  // iterations), so that a batch is one launch; eager launches if capture is not available
  cudaGraphExec_t exec = nullptr;
  {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int e = PAWFD_OK;
      for (int j = 0; j < CHECK && e == PAWFD_OK; ++j) e = iteration();
      const cudaError_t ce = cudaStreamEndCapture(s, &graph);
      if (e != PAWFD_OK || ce != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();   // a failed capture leaves no error behind for the eager path
  }
  while (k < maxiter && rnorm > tol * bnorm && bnorm > 0.0) {
    const int batch = std::min(CHECK, maxiter - k);
    if (exec && batch == CHECK) {
      rc = check_cuda(c, cudaGraphLaunch(exec, s), "poisson graph launch");
    } else {
      for (int j = 0; j < batch && rc == PAWFD_OK; ++j) rc = iteration();
    }
    k += batch;
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaGetLastError(), "poisson launch");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s), "copy");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamSynchronize(s), "sync");
    if (rc != PAWFD_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return rc;
    }
    rnorm = std::sqrt(h[S_RRNEW]);
  }
  if (exec) cudaGraphExecDestroy(exec);
  // the zero-mean solution
  dot_partial_kernel<<<PG, PT, 0, s>>>(x, nullptr, K, part);
  finish_kernel<<<1, 32, 0, s>>>(part, PG, K, 0, scal);
  shift_kernel<<<eb, PT, 0, s>>>(x, K, scal, v);
  c->launches += 3;
  if (iters) *iters = k;
  if (resid) *resid = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  return check_cuda(c, cudaGetLastError(), "poisson launch");
}
}  // namespace
