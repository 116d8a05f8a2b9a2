// api.cu -- extern "C" entry points: argument checks, then the kernel sequences.
#include "pawfd_internal.cuh"

using namespace pawfd;

namespace {

int check_bands(pawfd_ctx* c, int nb) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  return PAWFD_OK;
}

int apply_X(pawfd_ctx* c, int which, const void* psi, int nb, void* out, void* P_out) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || !out) return fail(c, PAWFD_EINVAL, "null array");
  if (psi == out) return fail(c, PAWFD_EINVAL, "psi and output may not alias");
  void* P = P_out ? P_out : c->d_P;
  if (which == 0) {
    rc = launch_kinetic_local(c, psi, nb, out);
  } else {
    rc = check_cuda(c, cudaMemcpyAsync(out, psi, band_size(c) * c->K * (size_t)nb, cudaMemcpyDeviceToDevice,
                                       c->stream), "copy psi");
  }
  if (rc != PAWFD_OK) return rc;
  rc = launch_project(c, psi, nb, P);
  if (rc != PAWFD_OK) return rc;
  return launch_nonlocal_add(c, P, nb, which == 0 ? c->at.d_dH : c->at.d_dS, out);
}

}  // namespace

namespace pawfd {
int launch_apply_hs(pawfd_ctx* c, const void* psi, int nb, void* hpsi, void* spsi, void* P) {
  // the stencil pass also writes S psi's first term (psi itself), so psi is read once
  int rc = launch_kinetic_local(c, psi, nb, hpsi, spsi);
  if (rc == PAWFD_OK) rc = launch_project(c, psi, nb, P);
  if (rc == PAWFD_OK) rc = launch_nonlocal_add2(c, P, nb, c->at.d_dH, hpsi, c->at.d_dS, spsi);
  return rc;
}
}  // namespace pawfd

extern "C" int pawfd_apply_HS(pawfd_ctx* c, const void* psi, int nb, void* hpsi, void* spsi, void* P_out) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || !hpsi || !spsi) return fail(c, PAWFD_EINVAL, "null array");
  if (psi == hpsi || psi == spsi || hpsi == spsi) return fail(c, PAWFD_EINVAL, "arrays may not alias");
  return launch_apply_hs(c, psi, nb, hpsi, spsi, P_out ? P_out : c->d_P);
}

extern "C" int pawfd_gram_hs(pawfd_ctx* c, const void* psi, const void* hpsi, int nb, const void* P, void* Hnm,
                             void* Snm) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || !hpsi || !Hnm || !Snm || (!P && c->at.Ip > 0)) return fail(c, PAWFD_EINVAL, "null array");
  if (Hnm == Snm) return fail(c, PAWFD_EINVAL, "Hnm and Snm may not alias");
  return launch_gram_hs(c, psi, hpsi, nb, P, Hnm, Snm);
}

extern "C" int pawfd_apply_kinetic_local(pawfd_ctx* c, const void* psi, int nb, void* out) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || !out || psi == out) return fail(c, PAWFD_EINVAL, "bad arrays");
  return launch_kinetic_local(c, psi, nb, out);
}

extern "C" int pawfd_project(pawfd_ctx* c, const void* psi, int nb, void* P) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || (!P && c->at.Ip > 0)) return fail(c, PAWFD_EINVAL, "null array");
  return launch_project(c, psi, nb, P);
}

extern "C" int pawfd_apply_H(pawfd_ctx* c, const void* psi, int nb, void* hpsi, void* P_out) {
  return apply_X(c, 0, psi, nb, hpsi, P_out);
}

extern "C" int pawfd_apply_S(pawfd_ctx* c, const void* psi, int nb, void* spsi, void* P_out) {
  return apply_X(c, 1, psi, nb, spsi, P_out);
}

extern "C" int pawfd_gram(pawfd_ctx* c, const void* A, const void* B, int nb, void* M) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!A || !B || !M) return fail(c, PAWFD_EINVAL, "null array");
  return launch_gram(c, A, B, nb, M, false);
}

extern "C" int pawfd_gram_hermitian(pawfd_ctx* c, const void* A, const void* B, int nb, void* M) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!A || !B || !M) return fail(c, PAWFD_EINVAL, "null array");
  return launch_gram(c, A, B, nb, M, true);
}

extern "C" int pawfd_subspace_diag(pawfd_ctx* c, int nb, void* Hnm, void* Snm, double* eps, void* C) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!Hnm || !Snm || !eps || !C) return fail(c, PAWFD_EINVAL, "null array");
  return launch_subspace_diag(c, nb, Hnm, Snm, eps, C);
}

extern "C" int pawfd_rotate(pawfd_ctx* c, const void* psi, int nb, const void* C, void* psi_out) {
  int rc = check_bands(c, nb);
  if (rc != PAWFD_OK) return rc;
  if (!psi || !C || !psi_out) return fail(c, PAWFD_EINVAL, "null array");
  if (psi == psi_out) return fail(c, PAWFD_EINVAL, "psi_out may not alias psi");
  return launch_rotate(c, psi, nb, C, psi_out);
}
