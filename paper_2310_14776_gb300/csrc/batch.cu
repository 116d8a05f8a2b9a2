// batch.cu -- one Rayleigh-Ritz step as a single call, and batches of independent steps.
//
// pawfd_rr_step enqueues the whole eigensolver step of SCF step 1 (Kohn-Sham section) for one
// context: H psi and S psi (Eq. (dh) and the overlap operator of the PAW section, with one set
// of projections serving both), the Hermitian Gram matrices (S_nm as dV psi^H psi plus the
// projector term, from the same slicing of psi as H_nm), the subspace diagonalization and the
// band rotation.
//
// A batch holds many such steps for independent contexts (different grids, band counts and
// atoms).  Each job runs on a stream of its own, forked from and joined back to the caller's
// stream, so the jobs' kernels overlap on the GPU; with graph mode the whole fork / steps /
// join sequence is captured once into a CUDA graph and every later launch of the batch is a
// single cudaGraphLaunch.
#include <vector>

#include "pawfd_internal.cuh"

using namespace pawfd;

struct pawfd_batch {
  std::vector<pawfd_rr_job> jobs;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;   // kernels enqueued by one launch of the batch
  std::string err;
};

namespace {

int enqueue_rr_step(pawfd_ctx* c, const pawfd_rr_job& j) {
  const int nb = j.nb;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  if (!j.psi || !j.hpsi || !j.spsi || !j.Hnm || !j.Snm || !j.eps || !j.C || !j.psi_out)
    return fail(c, PAWFD_EINVAL, "null array");
  if (j.psi == j.psi_out || j.psi == j.hpsi || j.psi == j.spsi || j.hpsi == j.spsi || j.Hnm == j.Snm)
    return fail(c, PAWFD_EINVAL, "arrays may not alias");
  // The Gram digits of psi and the rotation's digits of psi depend on psi alone: outside graph
  // capture the first are made on the auxiliary stream while H psi and S psi are applied, the
  // second while the latency-bound subspace solve runs.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool aux_ok = c->use_tc && c->tc.ready && cudaStreamIsCapturing(c->stream, &cap) == cudaSuccess &&
                      cap == cudaStreamCaptureStatusNone && ensure_aux_stream(c) == PAWFD_OK;
  int rc = PAWFD_OK;
  if (aux_ok) {
    cudaStream_t main = c->stream;
    rc = check_cuda(c, cudaEventRecord(c->aux_fork, main), "event record");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamWaitEvent(c->aux_stream, c->aux_fork, 0), "stream wait");
    if (rc == PAWFD_OK) {
      c->stream = c->aux_stream;
      gram_slice_psi(c, j.psi, nb);
      c->stream = main;
      rc = check_cuda(c, cudaEventRecord(c->aux_join, c->aux_stream), "event record");
    }
    if (rc == PAWFD_OK) rc = launch_apply_hs(c, j.psi, nb, j.hpsi, j.spsi, c->d_P);
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamWaitEvent(main, c->aux_join, 0), "stream wait");
  } else {
    rc = launch_apply_hs(c, j.psi, nb, j.hpsi, j.spsi, c->d_P);
  }
  if (rc == PAWFD_OK) rc = launch_gram_hs(c, j.psi, j.hpsi, nb, c->d_P, j.Hnm, j.Snm);
  c->tc.presliced_gram = nullptr;   // consumed by the Gram pair, or void after an error
  const bool overlap = rc == PAWFD_OK && aux_ok && c->tc.rot_rblk >= (long long)c->K;
  if (overlap) {
    cudaStream_t main = c->stream;
    rc = check_cuda(c, cudaEventRecord(c->aux_fork, main), "event record");
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamWaitEvent(c->aux_stream, c->aux_fork, 0), "stream wait");
    if (rc == PAWFD_OK) {
      c->stream = c->aux_stream;
      rotate_slice_psi(c, j.psi, nb);
      c->stream = main;
      rc = check_cuda(c, cudaEventRecord(c->aux_join, c->aux_stream), "event record");
    }
    if (rc == PAWFD_OK) rc = launch_subspace_diag(c, nb, j.Hnm, j.Snm, j.eps, j.C);
    if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamWaitEvent(main, c->aux_join, 0), "stream wait");
  } else if (rc == PAWFD_OK) {
    rc = launch_subspace_diag(c, nb, j.Hnm, j.Snm, j.eps, j.C);
  }
  if (rc == PAWFD_OK) rc = launch_rotate(c, j.psi, nb, j.C, j.psi_out);
  c->tc.presliced_psi = nullptr;   // consumed by the rotation, or void after an error
  return rc;
}

// fork from `origin`, one step per job on its own stream, join back into `origin`
int enqueue_batch(pawfd_batch* b, cudaStream_t origin, long long* kernels) {
  if (cudaEventRecord(b->fork, origin) != cudaSuccess) return PAWFD_EDEVICE;
  long long k = 0;
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    pawfd_ctx* c = b->jobs[i].ctx;
    if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return PAWFD_EDEVICE;
    cudaStream_t saved = c->stream;
    const long long l0 = c->launches;
    c->stream = b->streams[i];
    const int rc = enqueue_rr_step(c, b->jobs[i]);
    c->stream = saved;
    k += c->launches - l0;
    if (rc != PAWFD_OK) {
      b->err = "job " + std::to_string(i) + ": " + c->err;
      return rc;
    }
    if (cudaEventRecord(b->joins[i], b->streams[i]) != cudaSuccess) return PAWFD_EDEVICE;
    if (cudaStreamWaitEvent(origin, b->joins[i], 0) != cudaSuccess) return PAWFD_EDEVICE;
  }
  if (kernels) *kernels = k;
  return PAWFD_OK;
}

void free_batch(pawfd_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // namespace

extern "C" int pawfd_rr_step(pawfd_ctx* c, const void* psi, int nb, void* hpsi, void* spsi, void* Hnm, void* Snm,
                             double* eps, void* C, void* psi_out) {
  if (!c) return PAWFD_EINVAL;
  pawfd_rr_job j = {c, psi, nb, hpsi, spsi, Hnm, Snm, eps, C, psi_out};
  return enqueue_rr_step(c, j);
}

extern "C" int pawfd_batch_create(pawfd_batch** out, const pawfd_rr_job* jobs, int count, int use_graph) {
  if (!out || !jobs || count < 1) return PAWFD_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!jobs[i].ctx) return PAWFD_EINVAL;
    for (int k = 0; k < i; ++k)
      if (jobs[k].ctx == jobs[i].ctx) return PAWFD_EINVAL;   // one job per context (its scratch)
  }
  pawfd_batch* b = new pawfd_batch;
  b->jobs.assign(jobs, jobs + count);
  b->streams.assign(count, nullptr);
  b->joins.assign(count, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < count; ++i)
    ok = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch(b);
    return PAWFD_EDEVICE;
  }
  if (use_graph) {
    cudaStream_t cap = nullptr;
    int rc = PAWFD_EDEVICE;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      rc = enqueue_batch(b, cap, &b->kernels);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cap, &g);
      if (rc == PAWFD_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
        b->graph = g;
      } else {
        if (g) cudaGraphDestroy(g);
        if (rc == PAWFD_OK) rc = PAWFD_EDEVICE;
      }
    }
    if (cap) cudaStreamDestroy(cap);
    if (rc != PAWFD_OK) {
      // capture refused (or a job failed its checks): report, leave the batch in eager mode
      if (b->err.empty()) b->err = std::string("graph capture failed: ") + cudaGetErrorString(cudaGetLastError());
      cudaGetLastError();
      if (rc == PAWFD_EINVAL) {
        const int r = rc;
        free_batch(b);
        return r;
      }
    }
  }
  *out = b;
  return PAWFD_OK;
}

extern "C" int pawfd_batch_launch(pawfd_batch* b, void* stream) {
  if (!b) return PAWFD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (b->exec) return cudaGraphLaunch(b->exec, s) == cudaSuccess ? PAWFD_OK : PAWFD_EDEVICE;
  long long k = 0;
  const int rc = enqueue_batch(b, s, &k);
  b->kernels = k;
  return rc;
}

extern "C" int pawfd_batch_is_graph(const pawfd_batch* b) { return b && b->exec ? 1 : 0; }

extern "C" long long pawfd_batch_kernel_count(const pawfd_batch* b) { return b ? b->kernels : 0; }

extern "C" const char* pawfd_batch_last_error(const pawfd_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int pawfd_batch_destroy(pawfd_batch* b) {
  if (!b) return PAWFD_EINVAL;
  free_batch(b);
  return PAWFD_OK;
}
