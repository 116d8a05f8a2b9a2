// pawfd_internal.cuh -- shared definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pawfd.h"

namespace pawfd {

// ------------------------------------------------------------------------------------------
// complex double with the few operations the kernels need
// ------------------------------------------------------------------------------------------
struct alignas(16) zd {
  double re, im;
};

__host__ __device__ inline zd make_zd(double r, double i) { return zd{r, i}; }
__host__ __device__ inline zd operator+(zd a, zd b) { return zd{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline zd operator-(zd a, zd b) { return zd{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline zd operator*(zd a, zd b) { return zd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline zd operator*(double s, zd a) { return zd{s * a.re, s * a.im}; }
__host__ __device__ inline zd operator*(zd a, double s) { return zd{s * a.re, s * a.im}; }
__host__ __device__ inline zd& operator+=(zd& a, zd b) { a.re += b.re; a.im += b.im; return a; }
__host__ __device__ inline zd& operator-=(zd& a, zd b) { a.re -= b.re; a.im -= b.im; return a; }

// scalar traits: T is double (real, Gamma point) or zd (complex, Bloch)
__host__ __device__ inline double conjx(double x) { return x; }
__host__ __device__ inline zd conjx(zd x) { return zd{x.re, -x.im}; }
__host__ __device__ inline double absx2(double x) { return x * x; }
__host__ __device__ inline double absx2(zd x) { return x.re * x.re + x.im * x.im; }
__host__ __device__ inline double realx(double x) { return x; }
__host__ __device__ inline double realx(zd x) { return x.re; }
template <class T> __host__ __device__ inline T zero();
template <> __host__ __device__ inline double zero<double>() { return 0.0; }
template <> __host__ __device__ inline zd zero<zd>() { return zd{0.0, 0.0}; }
template <class T> __host__ __device__ inline T from_real(double x);
template <> __host__ __device__ inline double from_real<double>(double x) { return x; }
template <> __host__ __device__ inline zd from_real<zd>(double x) { return zd{x, 0.0}; }
// acc += conj(a) * b
__host__ __device__ inline void fma_conj(double& acc, double a, double b) { acc = fma(a, b, acc); }
__host__ __device__ inline void fma_conj(zd& acc, zd a, zd b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// acc += a * b
__host__ __device__ inline void fma_plain(double& acc, double a, double b) { acc = fma(a, b, acc); }
__host__ __device__ inline void fma_plain(zd& acc, zd a, zd b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += s * a (s real)
__host__ __device__ inline void fma_real(double& acc, double s, double a) { acc = fma(s, a, acc); }
__host__ __device__ inline void fma_real(zd& acc, double s, zd a) {
  acc.re = fma(s, a.re, acc.re);
  acc.im = fma(s, a.im, acc.im);
}

// ------------------------------------------------------------------------------------------
// device status word: first error wins
// ------------------------------------------------------------------------------------------
struct DeviceStatus {
  int code;    // 0 or a negative PAWFD_E* code
  int detail;  // e.g. failing Cholesky column, or the barrier that timed out
};

__device__ inline void set_status(DeviceStatus* st, int code, int detail) {
  if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// ------------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------------
struct AtomTables {
  int natoms = 0;
  int Ip = 0;
  int Imax = 0;
  // host copies
  std::vector<int> nproj, row_off, npts;
  std::vector<long long> pt_off, g_off, dmat_off;
  std::vector<std::vector<int>> colors;  // atoms grouped so that boxes of one group never share a point
  // device
  int* d_nproj = nullptr;
  int* d_row_off = nullptr;
  int* d_npts = nullptr;
  long long* d_pt_off = nullptr;
  int* d_pts = nullptr;              // wrapped grid index of every box point (unique per atom)
  long long* d_g_off = nullptr;
  void* d_g = nullptr;               // folded projector values [I_a][npts_a], scalar type of the context
  long long* d_dmat_off = nullptr;
  double* d_dH = nullptr;
  double* d_dS = nullptr;
  int* d_color_atoms = nullptr;      // atoms listed color by color
  std::vector<int> color_off;        // [ncolors+1] into d_color_atoms
};

}  // namespace pawfd

struct pawfd_ctx {
  int n[3];
  double cell[3], h[3], k[3], dV;
  int dtype;
  int max_bands;
  size_t K;
  cudaStream_t stream;
  double* d_vshift = nullptr;                 // v(r) - 1/2 c0 sum_c 1/h_c^2
  pawfd::AtomTables at;
  void* d_P = nullptr;                        // [Ip][max_bands] projection scratch
  void* d_gram_part = nullptr;                // split-K partial Gram matrices
  size_t gram_part_bytes = 0;
  void* d_work = nullptr;                     // subspace workspace (5 matrices of max_bands^2)
  double* d_evals = nullptr;                  // [max_bands] unsorted eigenvalues
  unsigned* d_barrier = nullptr;              // grid-barrier counters
  pawfd::DeviceStatus* d_status = nullptr;
  pawfd::DeviceStatus* h_status = nullptr;    // pinned mirror
  double* d_reduce = nullptr;                 // [max grid] partial sums for in-kernel reductions
  int num_sms = 0;
  long long launches = 0;                     // kernels this context has launched
  std::string err;
};

namespace pawfd {

inline size_t scalar_size(const pawfd_ctx* c) { return c->dtype == PAWFD_C128 ? 16 : 8; }

int fail(pawfd_ctx* c, int code, const std::string& msg);
int check_cuda(pawfd_ctx* c, cudaError_t e, const char* what);

// kernels (launchers), each enqueued on c->stream; return PAWFD_OK or an error code
int launch_kinetic_local(pawfd_ctx* c, const void* psi, int nb, void* out);
int launch_project(pawfd_ctx* c, const void* psi, int nb, void* P);
int launch_nonlocal_add(pawfd_ctx* c, const void* P, int nb, const double* d_dmat, void* out);
int launch_gram(pawfd_ctx* c, const void* A, const void* B, int nb, void* M);
int launch_rotate(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out);
int launch_subspace_diag(pawfd_ctx* c, int nb, void* Hnm, void* Snm, double* eps, void* C);

// order-6 central second-difference weights: f'' ~ (1/h^2) sum_m w_|m| f(x + m h)
constexpr double FD6_W0 = -49.0 / 18.0;
constexpr double FD6_W1 = 3.0 / 2.0;
constexpr double FD6_W2 = -3.0 / 20.0;
constexpr double FD6_W3 = 1.0 / 90.0;

}  // namespace pawfd
