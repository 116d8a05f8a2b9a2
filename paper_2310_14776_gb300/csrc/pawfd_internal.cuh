// pawfd_internal.cuh -- shared definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pawfd.h"

namespace pawfd {

// ------------------------------------------------------------------------------------------
// scalars: double / float (real, Gamma point) and zd / zf (complex, Bloch), with the few
// operations the kernels need
// ------------------------------------------------------------------------------------------
template <class R>
struct alignas(2 * sizeof(R)) cplx {
  R re, im;
};
using zd = cplx<double>;
using zf = cplx<float>;

template <class R> __host__ __device__ inline cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __host__ __device__ inline cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, R s) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ inline cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a.re += b.re; a.im += b.im; return a; }
template <class R> __host__ __device__ inline cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a.re -= b.re; a.im -= b.im; return a; }

template <class T> struct Traits;
template <> struct Traits<double> { using R = double; using D = double; static constexpr bool complex = false; };
template <> struct Traits<float> { using R = float; using D = double; static constexpr bool complex = false; };
template <> struct Traits<zd> { using R = double; using D = zd; static constexpr bool complex = true; };
template <> struct Traits<zf> { using R = float; using D = zd; static constexpr bool complex = true; };
template <class T> using real_t = typename Traits<T>::R;
template <class T> using wide_t = typename Traits<T>::D;   // the FP64 type of the same kind

__host__ __device__ inline double conjx(double x) { return x; }
__host__ __device__ inline float conjx(float x) { return x; }
template <class R> __host__ __device__ inline cplx<R> conjx(cplx<R> x) { return {x.re, -x.im}; }
__host__ __device__ inline double absx2(double x) { return x * x; }
__host__ __device__ inline float absx2(float x) { return x * x; }
template <class R> __host__ __device__ inline R absx2(cplx<R> x) { return x.re * x.re + x.im * x.im; }
__host__ __device__ inline double realx(double x) { return x; }
__host__ __device__ inline float realx(float x) { return x; }
template <class R> __host__ __device__ inline R realx(cplx<R> x) { return x.re; }
template <class T> __host__ __device__ inline T zero() { return T{}; }
template <class T> __host__ __device__ inline T from_real(real_t<T> x);
template <> __host__ __device__ inline double from_real<double>(double x) { return x; }
template <> __host__ __device__ inline float from_real<float>(float x) { return x; }
template <> __host__ __device__ inline zd from_real<zd>(double x) { return zd{x, 0.0}; }
template <> __host__ __device__ inline zf from_real<zf>(float x) { return zf{x, 0.0f}; }
// widening / narrowing conversions between the FP32 and FP64 scalar of the same kind
__host__ __device__ inline double widen(float x) { return (double)x; }
__host__ __device__ inline double widen(double x) { return x; }
__host__ __device__ inline zd widen(zf x) { return zd{(double)x.re, (double)x.im}; }
__host__ __device__ inline zd widen(zd x) { return x; }
template <class T> __host__ __device__ inline T narrow(wide_t<T> x);
template <> __host__ __device__ inline double narrow<double>(double x) { return x; }
template <> __host__ __device__ inline float narrow<float>(double x) { return (float)x; }
template <> __host__ __device__ inline zd narrow<zd>(zd x) { return x; }
template <> __host__ __device__ inline zf narrow<zf>(zd x) { return zf{(float)x.re, (float)x.im}; }

// acc += conj(a) * b
template <class R> __host__ __device__ inline void fma_conj(R& acc, R a, R b) { acc = fma(a, b, acc); }
template <class R> __host__ __device__ inline void fma_conj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// acc += a * b
template <class R> __host__ __device__ inline void fma_plain(R& acc, R a, R b) { acc = fma(a, b, acc); }
template <class R> __host__ __device__ inline void fma_plain(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += s * a (s real)
template <class R> __host__ __device__ inline void fma_real(R& acc, R s, R a) { acc = fma(s, a, acc); }
template <class R> __host__ __device__ inline void fma_real(cplx<R>& acc, R s, cplx<R> a) {
  acc.re = fma(s, a.re, acc.re);
  acc.im = fma(s, a.im, acc.im);
}

// ------------------------------------------------------------------------------------------
// device status word: first error wins
// ------------------------------------------------------------------------------------------
struct DeviceStatus {
  int code;    // 0 or a negative PAWFD_E* code
  int detail;  // e.g. failing Cholesky column, or the barrier that timed out
  // test setting ("test_barrier_missing"): grid barriers wait for this many CTAs more than
  // the launch has, and give up after barrier_limit_ms (0: the default limit)
  unsigned barrier_extra;
  unsigned barrier_limit_ms;
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
  void* d_g = nullptr;               // folded projector values [I_a][npts_a], band scalar type
  void* d_g_df = nullptr;            // real FP64: the same values as (hi, lo) FP32 pairs
  long long* d_dmat_off = nullptr;
  void* d_dH = nullptr;              // dH^a, real type of the band arithmetic (double or float)
  void* d_dS = nullptr;
  int* d_color_atoms = nullptr;      // atoms listed color by color
  std::vector<int> color_off;        // [ncolors+1] into d_color_atoms
  // work items of the projector kernels: (atom, first box point) of up to NL_PCH box points
  int nitems = 0;
  long long part_rows = 0;           // rows of the projection partials (sum over items of I_a)
  int2* d_items = nullptr;           // [nitems], atom by atom
  long long* d_item_row = nullptr;   // [nitems] first partial row of each item
  int* d_atom_items = nullptr;       // [natoms + 1] item range of each atom
  int2* d_color_items = nullptr;     // items listed color by color
  std::vector<int> color_item_off;   // [ncolors+1] into d_color_items
};
constexpr int NL_PCH = 256;          // box points per work item of the projector kernels

// Scratch of the tensor-core Gram: digit slices of one K block of each operand, their scale
// exponents, FP64 split-K partials, and the TMA descriptors of the slice buffers.
struct TcScratch {
  bool ready = false;
  long long kblk = 0;          // real-view values per K block (multiple of the exactness chunk)
  int rowsA_alloc = 0, rowsB_alloc = 0;
  void* slicesA = nullptr;
  void* slicesB = nullptr;
  int* sigA = nullptr;
  int* sigB = nullptr;
  int* maxA = nullptr;         // per-row largest scale exponent of the current K block
  int* maxB = nullptr;
  void* part = nullptr;
  size_t part_bytes = 0;
  CUtensorMap mapA;            // row-major planes of the Gram operands (4-D TMA boxes)
  CUtensorMap mapB;
  CUtensorMap mapAB;           // slicesA with the B operand's box (the Gram of psi with itself)
  CUtensorMap mapBA;           // slicesB with the A operand's box (complex Gram pair: psi's planes as A)
  CUtensorMap mapB32;          // slicesB with a box of 32 rows (symmetric cover)
  CUtensorMap mapAB32;         // slicesA with a box of 32 rows (symmetric cover, psi^T psi)
  void* part2 = nullptr;       // partials of the second Gram of a pair
  // band rotation
  long long rot_Lc = 0;        // contraction length (bands, x2 for complex) padded to chunks
  int rot_kc = 0;              // rotation chunk: 256 contraction values, or 512 beyond 256
  int rot_rowsA_alloc = 0;
  long long rot_rblk = 0;      // grid points per block
  void* rotA = nullptr;        // FP64 operand built from C
  void* rotSlicesA = nullptr;
  void* rotSlicesB = nullptr;
  int* rotSigA = nullptr;
  int* rotSigB = nullptr;
  int* rotMaxA = nullptr;
  int* rotMaxB = nullptr;
  int slice_t_ctas = 0;        // CTAs of the persistent transposing slicer
  const void* presliced_psi = nullptr;   // psi whose rotation digits are already in rotSlicesB
  int presliced_nb = 0;
  const void* presliced_gram = nullptr;  // psi whose Gram digits are already in slicesA
  int presliced_gram_nb = 0;
};

}  // namespace pawfd

// CUDA-event timing of the Gram MMA kernel launches (off by default; pawfd_kernel_timing)
struct KernelTimer {
  static constexpr int CAP = 1024;    // launches timed between two reads
  bool on = false;
  int used = 0;
  bool overflow = false;
  bool capturing = false;             // the bracketed launch is being captured into a graph
  cudaEvent_t start[CAP] = {}, stop[CAP] = {};
};

namespace pawfd {
// Plane-wave representation (pw.cu): FFT tables of the cell's grid, made on first use.
struct PwPlan {
  bool ready = false;
  int nf[3] = {0, 0, 0};          // radix stages per axis
  int fac[3][16] = {};            // radices per axis
  void* tw[3] = {nullptr, nullptr, nullptr};   // e^{-2 pi i j / N_c}, complex of the band precision
  void* phase = nullptr;          // e^{i k.r} at the grid points [K]
  void* kin = nullptr;            // |k+G|^2 / 2 [K], real of the band precision
  void* pois = nullptr;           // real FP64 contexts: -4 pi / (K L(G)) of the Poisson solve [K]
  void* tab = nullptr;            // kinetic preconditioner (FP32 plan): -1 / (K (t(k+G) + sigma)) [K]
};
}  // namespace pawfd

struct pawfd_ctx {
  KernelTimer ktimer;
  int n[3];
  double cell[3], h[3], k[3], dV;
  int dtype;
  int max_bands;
  size_t K;
  cudaStream_t stream;
  void* d_vshift = nullptr;                   // v(r) - 1/2 c0 sum_c 1/h_c^2 (double or float)
  void* d_vloc = nullptr;                     // v(r) itself in the band precision (double or float)
  pawfd::AtomTables at;
  void* d_P = nullptr;                        // [Ip][max_bands] projection scratch
  void* d_Q = nullptr;                        // [Ip][max_bands] FP64 dS P of the overlap correction
  void* d_Ppart = nullptr;                    // [part_rows][max_bands] projection partials
  void* d_gram_part = nullptr;                // split-K partial Gram matrices
  size_t gram_part_bytes = 0;
  void* d_work = nullptr;                     // subspace workspace (7 matrices of max_bands^2)
  int* d_flags = nullptr;                     // [16] subspace-solve path decisions (device-side gates)
  double* d_oa = nullptr;                     // Ogita-Aishima partial sums and eigenvalue estimates
  void* d_eig = nullptr;                      // FP32 eigendecomposition scratch (eig32_scratch_bytes)
  double* d_evals = nullptr;                  // [max_bands] unsorted eigenvalues
  double* d_dscale = nullptr;                 // [max_bands] column scaling of a Davidson subspace
  unsigned* d_barrier = nullptr;              // grid-barrier counters
  pawfd::DeviceStatus* d_status = nullptr;
  pawfd::DeviceStatus* h_status = nullptr;    // pinned mirror
  double* d_reduce = nullptr;                 // [8192]: in-kernel partial sums, Jacobi round flags
  int num_sms = 0;
  long long launches = 0;                     // kernels this context has launched
  bool use_tc = true;                         // Gram matrices on the tensor cores (sliced digits)
  bool fast_stencil = true;                   // shape-specialised stencil kernels where they apply
  int stencil_variant = 0;                    // 0: ring (bulk copies) first, 1: register float4 kernel
  int stencil_rows = 0;                       // y rows per CTA of the ring kernel (0: automatic)
  int stencil_yblock = 0;                     // y rows per thread of the ring kernel (0: automatic)
  int stencil_zsplit = 0;                     // general stencil: target CTAs per SM of a launch (0: 4)
  int stencil_ring = 0;                       // ring stencil: planes in the ring (0: 8; 8, 10 or 12)
  bool jacobi_cluster = false;                // Cholesky / Jacobi on one thread-block cluster where they fit
  bool tridiag_dsm = true;                    // FP32 tridiagonal reduction in the cluster's shared memory where it fits
  int tc_kblk_chunks = 0;                     // tensor-core Gram: K block in 512-value chunks (0: allocation)
  int tc_scratch_mb = 0;                      // digit-plane scratch per operand set in MB (0: default sizes)
  bool stencil_fx = true;                     // real FP64 stencil in exact fixed-point arithmetic
  bool free_operator = false;                 // v = 0 and no atoms: kinetic_local is T alone (Poisson)
  cudaStream_t aux_stream = nullptr;          // non-blocking stream for captured work (created on use)
  cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
  bool nonlocal_df = true;                    // real FP64 projector kernels in double-float arithmetic
  pawfd::TcScratch tc;
  pawfd::PwPlan pw;
  pawfd::PwPlan pc;                           // FP32 FFT plan of the Davidson kinetic preconditioner
  void* d_pc_work = nullptr;                  // its work array when the caller's is too small (lazy)
  size_t pc_work_bytes = 0;
  int davidson_precond = 1;                   // 1: kinetic (grids of 2, 3, 5 factors), 0: Jacobi
  std::string err;
};

namespace pawfd {

inline bool is_complex(const pawfd_ctx* c) { return c->dtype == PAWFD_C128 || c->dtype == PAWFD_C64; }
inline bool is_fp32(const pawfd_ctx* c) { return c->dtype == PAWFD_R32 || c->dtype == PAWFD_C64; }
// bytes of one band-array element / of one subspace-matrix element (always FP64)
inline size_t band_size(const pawfd_ctx* c) {
  return c->dtype == PAWFD_C128 ? 16 : (c->dtype == PAWFD_R32 ? 4 : 8);
}
inline size_t mat_size(const pawfd_ctx* c) { return is_complex(c) ? 16 : 8; }

// Call f(T{}) with T the band scalar type of the context (double, zd, float, zf).
template <class F>
int dispatch_band(const pawfd_ctx* c, F&& f) {
  switch (c->dtype) {
    case PAWFD_R64: return f(double{});
    case PAWFD_C128: return f(zd{});
    case PAWFD_R32: return f(float{});
    case PAWFD_C64: return f(zf{});
  }
  return PAWFD_EINVAL;
}

int fail(pawfd_ctx* c, int code, const std::string& msg);
int check_cuda(pawfd_ctx* c, cudaError_t e, const char* what);

// kernels (launchers), each enqueued on c->stream; return PAWFD_OK or an error code
int launch_kinetic_local(pawfd_ctx* c, const void* psi, int nb, void* out, void* cpy = nullptr);
int launch_project(pawfd_ctx* c, const void* psi, int nb, void* P);
int launch_nonlocal_add(pawfd_ctx* c, const void* P, int nb, const void* d_dmat, void* out);
// out1 += sum |p> dmat1 P and out2 += sum |p> dmat2 P in one pass over the boxes
int launch_nonlocal_add2(pawfd_ctx* c, const void* P, int nb, const void* dmat1, void* out1, const void* dmat2,
                         void* out2);
int launch_gram(pawfd_ctx* c, const void* A, const void* B, int nb, void* M, bool hermitian);
int launch_gram_tc(pawfd_ctx* c, const void* A, const void* B, int nb, void* M, bool hermitian);
int launch_rotate_tc(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out, int nout);
bool rotate_slice_psi(pawfd_ctx* c, const void* psi, int nb);
bool gram_slice_psi(pawfd_ctx* c, const void* psi, int nb);
// the context's auxiliary non-blocking stream and its fork / join events (created on first use)
int ensure_aux_stream(pawfd_ctx* c);
int setup_tc(pawfd_ctx* c);
void free_tc(pawfd_ctx* c);
void free_pw(pawfd_ctx* c);
size_t kinetic_precond_work_bytes(const pawfd_ctx* c, int nb);
int launch_kinetic_precond(pawfd_ctx* c, const void* R, int nb, void* out, void* work, size_t work_bytes);
int launch_rotate(pawfd_ctx* c, const void* psi, int nb, const void* C, void* out, int nout = -1);
// bracket one timed kernel launch on the context's stream (no-ops unless timing is on)
void ktimer_begin(pawfd_ctx* c);
void ktimer_end(pawfd_ctx* c);
// residuals H psi - eps S psi, their norms and the preconditioned corrections (davidson.cu)
int launch_residual_precond(pawfd_ctx* c, const void* hpsi, const void* spsi, int nb, const double* eps, void* pr,
                            double* rnorm, bool jacobi = true);
// the kinetic preconditioner applies: grid sizes with no prime factor other than 2, 3 and 5
bool kinetic_precond_available(const pawfd_ctx* c);
int launch_subspace_diag(pawfd_ctx* c, int nb, void* Hnm, void* Snm, double* eps, void* C);
// FP32 eigendecomposition of a Hermitian n x n FP64 matrix A (full storage): Z (FP64 storage)
// the eigenvectors, ascending eigenvalues; nothing happens when *gate != 0 (tridiag.cu)
int launch_eig32(pawfd_ctx* c, int n, const double* A, double* Z, const int* gate);
int launch_eig32(pawfd_ctx* c, int n, const zd* A, zd* Z, const int* gate);
int launch_overlap_correction(pawfd_ctx* c, const void* P, int nb, void* M);
bool gram_pair_tc(pawfd_ctx* c, const void* psi, const void* B, int nb, void* M1, void* M2, int* rc);
// H psi and S psi with one set of projections P of psi (written to P)
int launch_apply_hs(pawfd_ctx* c, const void* psi, int nb, void* hpsi, void* spsi, void* P);
// H_nm = dV psi^H H psi and S_nm = dV psi^H psi + sum_a P_a^H dS^a P_a (P: projections of psi)
int launch_gram_hs(pawfd_ctx* c, const void* psi, const void* hpsi, int nb, const void* P, void* Hnm, void* Snm);
// CTAs of the Ogita-Aishima element kernels and the doubles of their scratch for nb bands
constexpr int OA_G = 64;
inline size_t oa_scratch_doubles(int nb) { return 5 * (size_t)OA_G + (size_t)nb; }
// the working matrix (FP32 of the band kind), the eigenvectors of T (two float buffers), their
// Gram matrix and five vectors,
// each rounded up to 256 bytes
inline size_t eig32_scratch_bytes(int nb, bool complex) {
  const size_t f = complex ? 8 : 4, n = (size_t)nb;
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  return r(n * n * f) + 3 * r(n * n * 4) + 2 * r(n * f) + 3 * r(n * 4);
}

// order-6 central second-difference weights: f'' ~ (1/h^2) sum_m w_|m| f(x + m h)
constexpr double FD6_W0 = -49.0 / 18.0;
constexpr double FD6_W1 = 3.0 / 2.0;
constexpr double FD6_W2 = -3.0 / 20.0;
constexpr double FD6_W3 = 1.0 / 90.0;

}  // namespace pawfd
