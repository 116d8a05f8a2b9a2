// pw.cu -- H and S in the plane-wave representation, on the library's own FFT kernels.
//
// The wave-function section writes a Bloch state in plane waves,
//     psi_kn(r) = sum_G C_nG e^{i (k + G).r},
// the representation of the paper's GPU port.  On the cell's FFT grid (the grid of the
// finite-difference operator, G over the N1 x N2 x N3 frequencies in FFT order) the
// generalized eigenproblem of Eq. (dh) reads H C = eps S C with
//     (H C)_G = |k+G|^2 / 2 C_G + [v psi + sum_a |p^a> dH^a <p^a|psi>]_G,
//     (S C)_G = C_G + [sum_a |p^a> dS^a <p^a|psi>]_G,
// psi(r) = e^{ik.r} sum_G C_G e^{iG.r} at the grid points and [f]_G = (1/K) sum_r
// e^{-i(k+G).r} f(r): the kinetic operator is exact in this basis, the local potential and the
// projectors (the same grid-sampled boxes as the finite-difference operator) act on the grid.
// With an energy cutoff the basis is the sphere |k+G|^2 / 2 <= ecut and the output is zero
// outside it.
//
// FFTs: three passes, one per axis, each a batch of 1-D transforms of the lines along that
// axis.  A CTA stages a group of lines in shared memory and runs a mixed-radix Stockham
// transform (radices 4, 2, 3, 5; autosorting, so no bit reversal), ping-ponging between two
// buffers, with twiddles from a table e^{-2 pi i j / N} in shared memory.  Lines along x are
// contiguous; lines along y and z are gathered as tiles of consecutive x, so that both the
// loads and the stores of every pass are coalesced.  The Bloch phase, the local potential, the
// 1/K normalisation, the kinetic (or identity) term and the cutoff are applied in the first
// or last pass of each transform.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pawfd_internal.cuh"

namespace pawfd {
namespace {

constexpr int FFT_NT = 256;
constexpr int MAX_FAC = 16;

template <class R>
struct FftArgs {
  int N;                       // transform length (the axis' grid size)
  int nf;                      // number of radix stages
  int fac[MAX_FAC];            // radices, in order
  const cplx<R>* tw;           // e^{-2 pi i j / N}, j < N
  int inverse;                 // 1: e^{+i ...}, no normalisation
  int axis;                    // 0 (x), 1 (y), 2 (z)
  int n1, n2, n3;
  long long K;
  int nl;                      // lines per CTA
  int tiles;                   // axes 1, 2: tiles of nl consecutive x per row (ceil(n1 / nl))
  long long nlines;            // axis 0: nb n2 n3 lines
  const cplx<R>* in;
  cplx<R>* out;
  // prologue: 1 = multiply every input value by conj(phase[r]); 2 = the input is the real
  // array rin (imaginary part 0); 3 = the input is band array xin of the context's dtype
  // (xdouble: FP64, else FP32): real (xreal) bands 2 p and 2 p + 1 (0 past xnb) as the real
  // and imaginary parts of batch p, complex band p times conj(phase[r])
  int pre;
  const void* xin;
  void* xout;
  int xdouble, xreal, xnb;
  const cplx<R>* phase;
  const R* rin;
  // epilogue: 0 = store; 1 = store y phase[r] (psi), and v[r] psi into out2 (0 if v is null);
  // 2 = store y scale, plus kin[r] Cin (add_kin) or Cin (otherwise) when Cin is set, where
  // kin[r] <= ecut (or ecut <= 0), else 0; 3 = store y tab[r]; 4 = store Re(y) into rout;
  // 5 = the reverse of prologue 3 into xout: Re(y) to band 2 p and Im(y) to band 2 p + 1 (real),
  // or y phase[r] to band p (complex)
  int post;
  const R* tab;
  R* rout;
  cplx<R>* out2;
  const R* v;
  const R* kin;
  const cplx<R>* Cin;
  R scale;
  double ecut;
  int add_kin;
  // butterfly constants: sqrt(3)/2, cos(2 pi/5), cos(4 pi/5), sin(2 pi/5), sin(4 pi/5)
  R s3, c51, c52, s51, s52;
  // xy = 1: an x pass whose CTA holds one whole xy plane (nl = N2 lines) and transforms its
  // columns too (length N2, radices fac2, twiddles tw2) before the store
  int xy;
  int N2, nf2;
  int fac2[MAX_FAC];
  const cplx<R>* tw2;
};

// i s z
template <class R>
__device__ __forceinline__ cplx<R> imul(R s, cplx<R> z) {
  return cplx<R>{-s * z.im, s * z.re};
}

// The elements of this CTA's lines.  Line l's element i sits at grid point r = r0[l] + i s and
// global index g = g0[l] + i s (band offset band[l] K included), with s = 1 along x, N1 along y
// and N1 N2 along z; r0[l] < 0 marks a line past the grid.  The bases are formed once per CTA
// (64-bit divisions there only), so the per-element index arithmetic is an add and a multiply.
struct LineBase {
  long long g0;
  int r0;
  int band;
};

template <class R, int NT>
__device__ __forceinline__ void line_bases(const FftArgs<R>& a, LineBase* lb) {
  for (int l = threadIdx.x; l < a.nl; l += NT) {
    LineBase b;
    if (a.axis == 0) {
      const long long L = (long long)blockIdx.x * a.nl + l;
      const long long per_band = (long long)a.n2 * a.n3;
      if (L >= a.nlines) {
        b = {0, -1, 0};
      } else {
        b.band = (int)(L / per_band);
        b.r0 = (int)((L - (long long)b.band * per_band) * a.n1);
        b.g0 = (long long)b.band * a.K + b.r0;
      }
    } else {
      const int xt = blockIdx.x % a.tiles;
      const long long row = blockIdx.x / a.tiles;   // (band, z) for axis 1, (band, y) for axis 2
      const int x = xt * a.nl + l;
      const int m = a.axis == 1 ? a.n3 : a.n2;
      b.band = (int)(row / m);
      const int zy = (int)(row - (long long)b.band * m);
      if (x >= a.n1) {
        b = {0, -1, 0};
      } else {
        b.r0 = a.axis == 1 ? zy * a.n2 * a.n1 + x : zy * a.n1 + x;
        b.g0 = (long long)b.band * a.K + b.r0;
      }
    }
    lb[l] = b;
  }
}

// One radix-Rd butterfly of a Stockham stage: inputs x[r xs] (r < Rd), the r-th times the
// twiddle W[r k step], outputs y[r ys]
template <class R>
__device__ __forceinline__ void stockham_butterfly(const cplx<R>* x, int xs, cplx<R>* y, int ys, const cplx<R>* W,
                                                   int k, int step, int Rd, R sg, const FftArgs<R>& a) {
  if (Rd == 4) {
    cplx<R> v0 = x[0], v1 = x[xs] * W[k * step], v2 = x[2 * xs] * W[2 * k * step], v3 = x[3 * xs] * W[3 * k * step];
    const cplx<R> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, t3 = imul(sg, v1 - v3);
    y[0] = t0 + t2;
    y[ys] = t1 + t3;
    y[2 * ys] = t0 - t2;
    y[3 * ys] = t1 - t3;
  } else if (Rd == 2) {
    const cplx<R> v0 = x[0], v1 = x[xs] * W[k * step];
    y[0] = v0 + v1;
    y[ys] = v0 - v1;
  } else if (Rd == 3) {
    const cplx<R> v0 = x[0], v1 = x[xs] * W[k * step], v2 = x[2 * xs] * W[2 * k * step];
    const cplx<R> b = v1 + v2;
    const cplx<R> c = v0 - R(0.5) * b;
    const cplx<R> d = imul(sg * a.s3, v1 - v2);
    y[0] = v0 + b;
    y[ys] = c + d;
    y[2 * ys] = c - d;
  } else {   // 5
    const cplx<R> v0 = x[0], v1 = x[xs] * W[k * step], v2 = x[2 * xs] * W[2 * k * step],
                  v3 = x[3 * xs] * W[3 * k * step], v4 = x[4 * xs] * W[4 * k * step];
    const cplx<R> A = v1 + v4, B = v2 + v3, D = v1 - v4, E = v2 - v3;
    const cplx<R> t1 = v0 + a.c51 * A + a.c52 * B, t2 = v0 + a.c52 * A + a.c51 * B;
    const cplx<R> u1 = imul(sg, a.s51 * D + a.s52 * E), u2 = imul(sg, a.s52 * D - a.s51 * E);
    y[0] = v0 + A + B;
    y[ys] = t1 + u1;
    y[4 * ys] = t1 - u1;
    y[2 * ys] = t2 + u2;
    y[3 * ys] = t2 - u2;
  }
}

template <class R, int NT>
__global__ void __launch_bounds__(NT) fft_pass_kernel(const FftArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* W = (cplx<R>*)smem_raw;
  cplx<R>* W2 = W + a.N;                          // the columns' twiddles (xy passes)
  cplx<R>* X = W2 + (a.xy ? a.N2 : 0);
  // lines at a pitch of N + 1 values: the y and z passes fill and drain the buffer across lines
  // (consecutive x in consecutive threads), which at a pitch of N would put a warp's accesses
  // in one bank for every even N
  const int pitch = a.N + 1;
  cplx<R>* Y = X + (size_t)a.nl * pitch;
  LineBase* lb = (LineBase*)(Y + (size_t)a.nl * pitch);
  const int N = a.N, nl = a.nl, tid = threadIdx.x;
  const int stride = a.axis == 0 ? 1 : (a.axis == 1 ? a.n1 : a.n1 * a.n2);
  line_bases<R, NT>(a, lb);
  for (int j = tid; j < N; j += NT) {
    const cplx<R> w = a.tw[j];
    W[j] = a.inverse ? cplx<R>{w.re, -w.im} : w;
  }
  if (a.xy)
    for (int j = tid; j < a.N2; j += NT) {
      const cplx<R> w = a.tw2[j];
      W2[j] = a.inverse ? cplx<R>{w.re, -w.im} : w;
    }
  __syncthreads();   // the line bases
  // element e of the CTA's nl N is (line l, position i): e = l N + i along x (contiguous lines),
  // e = i nl + l along y and z (consecutive x); (l, i) advance by NT elements per iteration
  // without a division
  const bool xline = a.axis == 0;
  const int inner = xline ? N : nl;                     // the fast index's range
  const int d_fast = NT % inner, d_slow = NT / inner;
  const int f0 = tid % inner, s0 = tid / inner;
  // load: x lines along the line (contiguous), y / z lines across the tile (consecutive x)
  for (int e = tid, fi = f0, si = s0; e < nl * N; e += NT) {
    const int l = xline ? si : fi;
    const int i = xline ? fi : si;
    fi += d_fast;
    si += d_slow;
    if (fi >= inner) {
      fi -= inner;
      ++si;
    }
    cplx<R> v = {R(0), R(0)};
    const LineBase b = lb[l];
    if (b.r0 >= 0) {
      const int r = b.r0 + i * stride;
      const long long g = b.g0 + (long long)i * stride;
      if (a.pre == 2) {
        v = cplx<R>{a.rin[g], R(0)};
      } else if (a.pre == 3) {
        const long long p = b.band;
        if (a.xreal) {
          const long long ga = 2 * p * a.K + r, gb = ga + a.K;
          const bool hb = 2 * p + 1 < a.xnb;
          if (a.xdouble) {
            const double* X = (const double*)a.xin;
            v = cplx<R>{(R)X[ga], hb ? (R)X[gb] : R(0)};
          } else {
            const float* X = (const float*)a.xin;
            v = cplx<R>{(R)X[ga], hb ? (R)X[gb] : R(0)};
          }
        } else {
          if (a.xdouble) {
            const zd z = ((const zd*)a.xin)[g];
            v = cplx<R>{(R)z.re, (R)z.im};
          } else {
            const zf z = ((const zf*)a.xin)[g];
            v = cplx<R>{(R)z.re, (R)z.im};
          }
          const cplx<R> ph = a.phase[r];
          v = v * cplx<R>{ph.re, -ph.im};
        }
      } else {
        v = a.in[g];
        if (a.pre == 1) {
          const cplx<R> p = a.phase[r];
          v = v * cplx<R>{p.re, -p.im};
        }
      }
    }
    X[l * pitch + i] = v;
  }
  __syncthreads();
  // Stockham stages: after the stages with radices r_0 .. r_{s-1} (product Ns), transforms of
  // length Ns R are formed from R of length Ns
  const R sg = a.inverse ? R(1) : R(-1);
  int Ns = 1;
  for (int s = 0; s < a.nf; ++s) {
    const int Rd = a.fac[s], M = N / Rd, step = N / (Ns * Rd);
    // butterfly e = l M + j, j = jq Ns + k (M is a multiple of Ns); all advanced incrementally
    const int dj = NT % M, dl = NT / M, dk = dj % Ns, djq = dj / Ns, mq = M / Ns;
    int l = tid / M, j = tid - (tid / M) * M;
    int jq = j / Ns, k = j - jq * Ns;
    for (int e = tid; e < nl * M; e += NT) {
      stockham_butterfly(X + l * pitch + j, M, Y + l * pitch + jq * Ns * Rd + k, Ns, W, k, step, Rd, sg, a);
      j += dj;
      l += dl;
      k += dk;
      jq += djq;
      if (k >= Ns) {
        k -= Ns;
        ++jq;
      }
      if (j >= M) {
        j -= M;
        ++l;
        jq -= mq;
      }
    }
    __syncthreads();
    cplx<R>* t = X;
    X = Y;
    Y = t;
    Ns *= Rd;
  }
  // xy passes: the columns of the plane (element i of column x at X[i pitch + x]); butterfly
  // e = j N + x with x fastest, so that a warp touches consecutive columns (no bank conflicts)
  if (a.xy) {
    const int Ny = a.N2;
    int Ns2 = 1;
    for (int s = 0; s < a.nf2; ++s) {
      const int Rd = a.fac2[s], M = Ny / Rd, step = Ny / (Ns2 * Rd);
      const int dx = NT % N, dj = NT / N, dk = dj % Ns2, djq = dj / Ns2;
      int x = tid % N, j = tid / N;
      int jq = j / Ns2, k = j - jq * Ns2;
      for (int e = tid; e < M * N; e += NT) {
        stockham_butterfly(X + j * pitch + x, M * pitch, Y + (jq * Ns2 * Rd + k) * pitch + x, Ns2 * pitch, W2, k, step,
                           Rd, sg, a);
        x += dx;
        j += dj;
        k += dk;
        jq += djq;
        if (k >= Ns2) {
          k -= Ns2;
          ++jq;
        }
        if (x >= N) {
          x -= N;
          ++j;
          if (++k >= Ns2) {
            k -= Ns2;
            ++jq;
          }
        }
      }
      __syncthreads();
      cplx<R>* t = X;
      X = Y;
      Y = t;
      Ns2 *= Rd;
    }
  }
  // store, with the epilogue
  for (int e = tid, fi = f0, si = s0; e < nl * N; e += NT) {
    const int l = xline ? si : fi;
    const int i = xline ? fi : si;
    fi += d_fast;
    si += d_slow;
    if (fi >= inner) {
      fi -= inner;
      ++si;
    }
    const LineBase b = lb[l];
    if (b.r0 < 0) continue;
    const int r = b.r0 + i * stride;
    const long long g = b.g0 + (long long)i * stride;
    const cplx<R> y = X[l * pitch + i];
    if (a.post == 0) {
      a.out[g] = y;
    } else if (a.post == 3) {
      a.out[g] = y * a.tab[r];
    } else if (a.post == 4) {
      a.rout[g] = y.re;
    } else if (a.post == 5) {
      const long long p = b.band;
      if (a.xreal) {
        const long long ga = 2 * p * a.K + r, gb = ga + a.K;
        const bool hb = 2 * p + 1 < a.xnb;
        if (a.xdouble) {
          double* X = (double*)a.xout;
          X[ga] = (double)y.re;
          if (hb) X[gb] = (double)y.im;
        } else {
          float* X = (float*)a.xout;
          X[ga] = (float)y.re;
          if (hb) X[gb] = (float)y.im;
        }
      } else {
        const cplx<R> z = y * a.phase[r];
        if (a.xdouble) ((zd*)a.xout)[g] = zd{(double)z.re, (double)z.im};
        else ((zf*)a.xout)[g] = zf{(float)z.re, (float)z.im};
      }
    } else if (a.post == 1) {
      const cplx<R> psi = y * a.phase[r];
      a.out[g] = psi;
      if (a.out2) a.out2[g] = a.v ? a.v[r] * psi : cplx<R>{R(0), R(0)};
    } else {
      const R kn = a.kin[r];
      cplx<R> o = {R(0), R(0)};
      if (a.ecut <= 0.0 || (double)kn <= a.ecut) {
        o = y * a.scale;
        if (a.Cin) {
          const cplx<R> cg = a.Cin[g];
          o += a.add_kin ? kn * cg : cg;
        }
      }
      a.out[g] = o;
    }
  }
}

// radices of n from {4, 2, 3, 5} (fours first); false for other prime factors
bool factorize(int n, int* fac, int* nf) {
  *nf = 0;
  while (n % 4 == 0 && *nf < MAX_FAC) {
    fac[(*nf)++] = 4;
    n /= 4;
  }
  for (int r : {2, 3, 5})
    while (n % r == 0 && *nf < MAX_FAC) {
      fac[(*nf)++] = r;
      n /= r;
    }
  return n == 1;
}

template <class R>
int setup_pw_impl(pawfd_ctx* c) {
  PwPlan& p = c->pw;
  int rc = PAWFD_OK;
  for (int ax = 0; ax < 3; ++ax) {
    if (!factorize(c->n[ax], p.fac[ax], &p.nf[ax]))
      return fail(c, PAWFD_EINVAL, "plane-wave mode: grid sizes must have no prime factor other than 2, 3 and 5");
    const int N = c->n[ax];
    std::vector<cplx<R>> tw(N);
    for (int j = 0; j < N; ++j) {
      const double t = 2.0 * M_PI * (double)j / (double)N;
      tw[j] = cplx<R>{(R)std::cos(t), (R)-std::sin(t)};
    }
    rc = check_cuda(c, cudaMalloc(&p.tw[ax], sizeof(cplx<R>) * N), "cudaMalloc pw twiddles");
    if (rc == PAWFD_OK)
      rc = check_cuda(c, cudaMemcpy(p.tw[ax], tw.data(), sizeof(cplx<R>) * N, cudaMemcpyHostToDevice), "memcpy");
    if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  }
  const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2];
  std::vector<cplx<R>> ph(c->K);
  std::vector<R> kin(c->K);
  std::vector<double> qx(n1), qy(n2), qz(n3);
  auto freq = [](int i, int n) { return (double)(i < (n + 1) / 2 ? i : i - n); };
  for (int i = 0; i < n1; ++i) qx[i] = c->k[0] + 2.0 * M_PI * freq(i, n1) / c->cell[0];
  for (int i = 0; i < n2; ++i) qy[i] = c->k[1] + 2.0 * M_PI * freq(i, n2) / c->cell[1];
  for (int i = 0; i < n3; ++i) qz[i] = c->k[2] + 2.0 * M_PI * freq(i, n3) / c->cell[2];
  for (int i3 = 0; i3 < n3; ++i3)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < n1; ++i1) {
        const size_t r = ((size_t)i3 * n2 + i2) * n1 + i1;
        const double kr = c->k[0] * i1 * c->h[0] + c->k[1] * i2 * c->h[1] + c->k[2] * i3 * c->h[2];
        ph[r] = cplx<R>{(R)std::cos(kr), (R)std::sin(kr)};
        kin[r] = (R)(0.5 * (qx[i1] * qx[i1] + qy[i2] * qy[i2] + qz[i3] * qz[i3]));
      }
  // the Poisson solve's multiplier -4 pi / (K L(G)) (0 at G = 0), L(G) the symbol of the order-6
  // FD Laplacian, sum_c (w0 + 2 sum_m w_m cos(m G_c h_c)) / h_c^2 (real FP64 contexts)
  std::vector<double> pois;
  if (c->dtype == PAWFD_R64) {
    const double w[4] = {FD6_W0, FD6_W1, FD6_W2, FD6_W3};
    std::vector<double> lx(n1), ly(n2), lz(n3);
    auto sym = [&](std::vector<double>& out, int n, double L, double h) {
      for (int i = 0; i < n; ++i) {
        const double g = 2.0 * M_PI * freq(i, n) / L;
        double acc = w[0];
        for (int m = 1; m <= 3; ++m) acc += 2.0 * w[m] * std::cos(m * g * h);
        out[i] = acc / (h * h);
      }
    };
    sym(lx, n1, c->cell[0], c->h[0]);
    sym(ly, n2, c->cell[1], c->h[1]);
    sym(lz, n3, c->cell[2], c->h[2]);
    pois.resize(c->K);
    for (int i3 = 0; i3 < n3; ++i3)
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1) {
          const size_t r = ((size_t)i3 * n2 + i2) * n1 + i1;
          const double L = lx[i1] + ly[i2] + lz[i3];
          pois[r] = (r == 0) ? 0.0 : -4.0 * M_PI / ((double)c->K * L);
        }
    rc = check_cuda(c, cudaMalloc(&p.pois, sizeof(double) * c->K), "cudaMalloc poisson table");
    if (rc == PAWFD_OK)
      rc = check_cuda(c, cudaMemcpy(p.pois, pois.data(), sizeof(double) * c->K, cudaMemcpyHostToDevice), "memcpy");
    if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  }
  rc = check_cuda(c, cudaMalloc(&p.phase, sizeof(cplx<R>) * c->K), "cudaMalloc pw phase");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&p.kin, sizeof(R) * c->K), "cudaMalloc pw kinetic");
  if (rc == PAWFD_OK)
    rc = check_cuda(c, cudaMemcpy(p.phase, ph.data(), sizeof(cplx<R>) * c->K, cudaMemcpyHostToDevice), "memcpy");
  if (rc == PAWFD_OK)
    rc = check_cuda(c, cudaMemcpy(p.kin, kin.data(), sizeof(R) * c->K, cudaMemcpyHostToDevice), "memcpy");
  if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  p.ready = true;
  return PAWFD_OK;
}

// Tables on first use: twiddles per axis, the Bloch phase and the kinetic energies.
int ensure_pw(pawfd_ctx* c, bool need_complex = true) {
  if (need_complex && !is_complex(c))
    return fail(c, PAWFD_EINVAL, "plane-wave mode needs a complex context (PAWFD_C128 or PAWFD_C64)");
  if (c->pw.ready) return PAWFD_OK;
  int rc = check_cuda(c, cudaStreamSynchronize(c->stream), "stream sync");
  if (rc != PAWFD_OK) return rc;
  rc = is_fp32(c) ? setup_pw_impl<float>(c) : setup_pw_impl<double>(c);
  if (rc != PAWFD_OK) free_pw(c);
  return rc;
}

template <class R>
int fft_pass_plan(pawfd_ctx* c, const PwPlan& p, int axis, const cplx<R>* in, cplx<R>* out, int nb, bool inverse,
                  FftArgs<R> a) {
  a.N = c->n[axis];
  a.nf = p.nf[axis];
  for (int s = 0; s < p.nf[axis]; ++s) a.fac[s] = p.fac[axis][s];
  a.tw = (const cplx<R>*)p.tw[axis];
  a.inverse = inverse ? 1 : 0;
  a.axis = axis;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  a.in = in;
  a.out = out;
  a.s3 = (R)(0.5 * std::sqrt(3.0));
  a.c51 = (R)std::cos(2.0 * M_PI / 5.0);
  a.c52 = (R)std::cos(4.0 * M_PI / 5.0);
  a.s51 = (R)std::sin(2.0 * M_PI / 5.0);
  a.s52 = (R)std::sin(4.0 * M_PI / 5.0);
  // lines per CTA: about 1024 (FP64) or 2048 (FP32) complex values per buffer (measured a
  // little faster than twice that: more CTAs per SM)
  const int cap = sizeof(R) == 8 ? 1024 : 2048;
  long long grid;
  if (axis == 0) {
    a.nl = std::max(1, std::min(64, cap / a.N));
    a.nlines = (long long)nb * a.n2 * a.n3;
    a.tiles = 1;
    grid = (a.nlines + a.nl - 1) / a.nl;
  } else {
    a.nl = std::max(1, std::min(std::min(32, a.n1), cap / a.N));
    a.tiles = (a.n1 + a.nl - 1) / a.nl;
    a.nlines = 0;
    grid = (long long)nb * (axis == 1 ? a.n3 : a.n2) * a.tiles;
  }
  const size_t smem =
      sizeof(cplx<R>) * ((size_t)a.N + 2 * (size_t)a.nl * (a.N + 1)) + sizeof(LineBase) * (size_t)a.nl;
  if (smem > 48 * 1024) {
    const int rc = check_cuda(
        c, cudaFuncSetAttribute(fft_pass_kernel<R, FFT_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "fft smem attribute");
    if (rc != PAWFD_OK) return rc;
  }
  if (grid > 2147483647ll) return fail(c, PAWFD_EINVAL, "plane-wave mode: too many lines for one launch");
  fft_pass_kernel<R, FFT_NT><<<(unsigned)grid, FFT_NT, smem, c->stream>>>(a);
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "fft launch");
}

// The fused xy pass: one CTA of XY_NT threads per xy plane (both buffers of the plane in
// shared memory), x then y transforms, a's prologue on load and epilogue on store.  FP32 only,
// and only while the plane's two buffers fit XY_SMEM_MAX bytes (96^2: 149 KB).
constexpr int XY_NT = 1024;
constexpr size_t XY_SMEM_MAX = 200 * 1024;

template <class R>
size_t xy_smem(const pawfd_ctx* c) {
  const size_t n1 = (size_t)c->n[0], n2 = (size_t)c->n[1];
  return sizeof(cplx<R>) * (n1 + n2 + 2 * n2 * (n1 + 1)) + sizeof(LineBase) * n2;
}
template <class R>
bool xy_fits(const pawfd_ctx* c) { return sizeof(R) == 4 && xy_smem<R>(c) <= XY_SMEM_MAX; }

template <class R>
int fft_xy_pass_plan(pawfd_ctx* c, const PwPlan& p, const cplx<R>* in, cplx<R>* out, int nb, bool inverse,
                     FftArgs<R> a) {
  a.N = c->n[0];
  a.nf = p.nf[0];
  for (int s = 0; s < p.nf[0]; ++s) a.fac[s] = p.fac[0][s];
  a.tw = (const cplx<R>*)p.tw[0];
  a.xy = 1;
  a.N2 = c->n[1];
  a.nf2 = p.nf[1];
  for (int s = 0; s < p.nf[1]; ++s) a.fac2[s] = p.fac[1][s];
  a.tw2 = (const cplx<R>*)p.tw[1];
  a.inverse = inverse ? 1 : 0;
  a.axis = 0;
  a.n1 = c->n[0];
  a.n2 = c->n[1];
  a.n3 = c->n[2];
  a.K = (long long)c->K;
  a.in = in;
  a.out = out;
  a.s3 = (R)(0.5 * std::sqrt(3.0));
  a.c51 = (R)std::cos(2.0 * M_PI / 5.0);
  a.c52 = (R)std::cos(4.0 * M_PI / 5.0);
  a.s51 = (R)std::sin(2.0 * M_PI / 5.0);
  a.s52 = (R)std::sin(4.0 * M_PI / 5.0);
  a.nl = c->n[1];                                   // one xy plane per CTA
  a.nlines = (long long)nb * c->n[1] * c->n[2];
  a.tiles = 1;
  const long long grid = (long long)nb * c->n[2];
  const size_t smem = xy_smem<R>(c);
  int rc = check_cuda(c, cudaFuncSetAttribute(fft_pass_kernel<R, XY_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem),
                      "fft xy smem attribute");
  if (rc != PAWFD_OK) return rc;
  if (grid > 2147483647ll) return fail(c, PAWFD_EINVAL, "plane-wave mode: too many planes for one launch");
  fft_pass_kernel<R, XY_NT><<<(unsigned)grid, XY_NT, smem, c->stream>>>(a);
  c->launches += 1;
  return check_cuda(c, cudaGetLastError(), "fft xy launch");
}

// The x and y transforms of every xy plane: the fused pass where it applies, else the x pass
// (with a's prologue, in -> out) and the y pass (with a's epilogue, in place in out).
template <class R>
int fft_xy(pawfd_ctx* c, const PwPlan& p, const cplx<R>* in, cplx<R>* out, int nb, bool inverse, FftArgs<R> a) {
  if (xy_fits<R>(c)) return fft_xy_pass_plan<R>(c, p, in, out, nb, inverse, a);
  FftArgs<R> ax = a, ay = a;
  ax.post = 0;
  ay.pre = 0;
  ay.xin = nullptr;
  int rc = fft_pass_plan<R>(c, p, 0, in, out, nb, inverse, ax);
  if (rc == PAWFD_OK) rc = fft_pass_plan<R>(c, p, 1, out, out, nb, inverse, ay);
  return rc;
}

template <class R>
int fft_pass(pawfd_ctx* c, int axis, const cplx<R>* in, cplx<R>* out, int nb, bool inverse, FftArgs<R> a) {
  return fft_pass_plan<R>(c, c->pw, axis, in, out, nb, inverse, a);
}

// psi(r) = e^{ik.r} sum_G C_G e^{iG.r}: the inverse transform (unnormalised), the phase in the
// last pass; with loc != null also loc = v psi (v != null) or 0
template <class R>
int pw_inverse(pawfd_ctx* c, const cplx<R>* C, int nb, cplx<R>* psi, cplx<R>* loc, const R* v) {
  FftArgs<R> a = {};
  int rc;
  if (xy_fits<R>(c)) {
    // z first, then x and y in one pass with the phase epilogue (the axes commute)
    rc = fft_pass<R>(c, 2, C, psi, nb, true, a);
    a.post = 1;
    a.phase = (const cplx<R>*)c->pw.phase;
    a.out2 = loc;
    a.v = v;
    if (rc == PAWFD_OK) rc = fft_xy_pass_plan<R>(c, c->pw, psi, psi, nb, true, a);
    return rc;
  }
  rc = fft_pass<R>(c, 0, C, psi, nb, true, a);
  if (rc == PAWFD_OK) rc = fft_pass<R>(c, 1, psi, psi, nb, true, a);
  a.post = 1;
  a.phase = (const cplx<R>*)c->pw.phase;
  a.out2 = loc;
  a.v = v;
  if (rc == PAWFD_OK) rc = fft_pass<R>(c, 2, psi, psi, nb, true, a);
  return rc;
}

// out_G = (1/K) sum_r e^{-i(k+G).r} f(r) (+ kin_G Cin_G or + Cin_G, masked by the cutoff)
template <class R>
int pw_forward(pawfd_ctx* c, cplx<R>* f, int nb, cplx<R>* out, const cplx<R>* Cin, bool add_kin, double ecut) {
  FftArgs<R> a = {};
  a.pre = 1;
  a.phase = (const cplx<R>*)c->pw.phase;
  int rc = fft_xy<R>(c, c->pw, f, f, nb, false, a);
  a.pre = 0;
  a.post = 2;
  a.kin = (const R*)c->pw.kin;
  a.Cin = Cin;
  a.add_kin = add_kin ? 1 : 0;
  a.ecut = ecut;
  a.scale = (R)(1.0 / (double)c->K);
  if (rc == PAWFD_OK) rc = fft_pass<R>(c, 2, f, out, nb, false, a);
  return rc;
}

template <class R>
int pw_apply_impl(pawfd_ctx* c, int which, const cplx<R>* C, int nb, double ecut, cplx<R>* out, cplx<R>* work) {
  cplx<R>* psi = work;
  cplx<R>* loc = work + (size_t)nb * c->K;
  int rc = pw_inverse<R>(c, C, nb, psi, loc, which == 0 ? (const R*)c->d_vloc : nullptr);
  if (rc == PAWFD_OK && c->at.natoms > 0) {
    rc = launch_project(c, psi, nb, c->d_P);
    if (rc == PAWFD_OK) rc = launch_nonlocal_add(c, c->d_P, nb, which == 0 ? c->at.d_dH : c->at.d_dS, loc);
  }
  if (rc == PAWFD_OK) rc = pw_forward<R>(c, loc, nb, out, C, which == 0, ecut);
  return rc;
}

// v = the zero-mean solution of lap_FD v = -4 pi rho on the periodic grid: rho's transform
// times -4 pi / (K L(G)) (0 at G = 0), transformed back; the imaginary part of the result is
// rounding only and is dropped.
int poisson_fft_impl(pawfd_ctx* c, const double* rho, double* v, zd* work) {
  FftArgs<double> a = {};
  a.pre = 2;
  a.rin = rho;
  int rc = fft_pass<double>(c, 0, nullptr, work, 1, false, a);
  a.pre = 0;
  a.rin = nullptr;
  if (rc == PAWFD_OK) rc = fft_pass<double>(c, 1, work, work, 1, false, a);
  a.post = 3;
  a.tab = (const double*)c->pw.pois;
  if (rc == PAWFD_OK) rc = fft_pass<double>(c, 2, work, work, 1, false, a);
  a.post = 0;
  a.tab = nullptr;
  if (rc == PAWFD_OK) rc = fft_pass<double>(c, 0, work, work, 1, true, a);
  if (rc == PAWFD_OK) rc = fft_pass<double>(c, 1, work, work, 1, true, a);
  a.post = 4;
  a.rout = v;
  if (rc == PAWFD_OK) rc = fft_pass<double>(c, 2, work, work, 1, true, a);
  return rc;
}

// ---- the kinetic preconditioner of the Davidson step ----
// -(T + sigma)^-1 R for every band R: T is diagonal on the grid's Bloch waves, with the FD
// kinetic symbol t(k + G) = -1/2 sum_c (w0 + 2 sum_m w_m cos(m q_c h_c)) / h_c^2, q = k + G.
// A search direction needs no FP64, so the transforms are FP32 whatever the context's dtype:
// two real bands form one complex transform (the multiplier is real and even in G, so the real
// and imaginary parts stay apart), complex bands carry e^{-ik.r} in and e^{ik.r} out.
constexpr double KINETIC_SHIFT = 0.5;   // sigma, Hartree

int setup_pc_impl(pawfd_ctx* c) {
  PwPlan& p = c->pc;
  int rc = PAWFD_OK;
  for (int ax = 0; ax < 3; ++ax) {
    if (!factorize(c->n[ax], p.fac[ax], &p.nf[ax]))
      return fail(c, PAWFD_EINVAL, "kinetic preconditioner: grid sizes must have no prime factor other than 2, 3 and 5");
    const int N = c->n[ax];
    std::vector<zf> tw(N);
    for (int j = 0; j < N; ++j) {
      const double t = 2.0 * M_PI * (double)j / (double)N;
      tw[j] = zf{(float)std::cos(t), (float)-std::sin(t)};
    }
    rc = check_cuda(c, cudaMalloc(&p.tw[ax], sizeof(zf) * N), "cudaMalloc preconditioner twiddles");
    if (rc == PAWFD_OK)
      rc = check_cuda(c, cudaMemcpy(p.tw[ax], tw.data(), sizeof(zf) * N, cudaMemcpyHostToDevice), "memcpy");
    if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  }
  const int n1 = c->n[0], n2 = c->n[1], n3 = c->n[2];
  const double w[4] = {FD6_W0, FD6_W1, FD6_W2, FD6_W3};
  auto freq = [](int i, int n) { return (double)(i < (n + 1) / 2 ? i : i - n); };
  auto sym = [&](std::vector<double>& out, int n, int ax) {
    out.resize(n);
    const double h = c->h[ax];
    for (int i = 0; i < n; ++i) {
      const double q = c->k[ax] + 2.0 * M_PI * freq(i, n) / c->cell[ax];
      double acc = w[0];
      for (int m = 1; m <= 3; ++m) acc += 2.0 * w[m] * std::cos(m * q * h);
      out[i] = -0.5 * acc / (h * h);
    }
  };
  std::vector<double> tx, ty, tz;
  sym(tx, n1, 0);
  sym(ty, n2, 1);
  sym(tz, n3, 2);
  std::vector<float> tab(c->K);
  std::vector<zf> ph(c->K);
  for (int i3 = 0; i3 < n3; ++i3)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < n1; ++i1) {
        const size_t r = ((size_t)i3 * n2 + i2) * n1 + i1;
        tab[r] = (float)(-1.0 / ((double)c->K * (tx[i1] + ty[i2] + tz[i3] + KINETIC_SHIFT)));
        const double kr = c->k[0] * i1 * c->h[0] + c->k[1] * i2 * c->h[1] + c->k[2] * i3 * c->h[2];
        ph[r] = zf{(float)std::cos(kr), (float)std::sin(kr)};
      }
  rc = check_cuda(c, cudaMalloc(&p.tab, sizeof(float) * c->K), "cudaMalloc preconditioner table");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMalloc(&p.phase, sizeof(zf) * c->K), "cudaMalloc preconditioner phase");
  if (rc == PAWFD_OK)
    rc = check_cuda(c, cudaMemcpy(p.tab, tab.data(), sizeof(float) * c->K, cudaMemcpyHostToDevice), "memcpy");
  if (rc == PAWFD_OK)
    rc = check_cuda(c, cudaMemcpy(p.phase, ph.data(), sizeof(zf) * c->K, cudaMemcpyHostToDevice), "memcpy");
  if (rc != PAWFD_OK) return fail(c, PAWFD_ENOMEM, c->err);
  p.ready = true;
  return PAWFD_OK;
}

void free_plan(PwPlan& p) {
  void* ptrs[] = {p.tw[0], p.tw[1], p.tw[2], p.phase, p.kin, p.pois, p.tab};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p = PwPlan();
}

int ensure_pc(pawfd_ctx* c) {
  if (c->pc.ready) return PAWFD_OK;
  int rc = check_cuda(c, cudaStreamSynchronize(c->stream), "stream sync");
  if (rc != PAWFD_OK) return rc;
  rc = setup_pc_impl(c);
  if (rc != PAWFD_OK) free_plan(c->pc);
  return rc;
}

int kinetic_precond_impl(pawfd_ctx* c, const void* R, int nb, void* out, zf* work) {
  const int nbat = is_complex(c) ? nb : (nb + 1) / 2;
  FftArgs<float> a = {};
  a.xdouble = is_fp32(c) ? 0 : 1;
  a.xreal = is_complex(c) ? 0 : 1;
  a.xnb = nb;
  a.phase = (const zf*)c->pc.phase;
  a.pre = 3;
  a.xin = R;
  // forward: x and y (reading the bands), z (times the table); inverse: z, then x and y
  // (writing the bands); the axes commute
  int rc = fft_xy<float>(c, c->pc, nullptr, work, nbat, false, a);
  a.pre = 0;
  a.xin = nullptr;
  a.post = 3;
  a.tab = (const float*)c->pc.tab;
  if (rc == PAWFD_OK) rc = fft_pass_plan<float>(c, c->pc, 2, work, work, nbat, false, a);
  a.post = 0;
  a.tab = nullptr;
  if (rc == PAWFD_OK) rc = fft_pass_plan<float>(c, c->pc, 2, work, work, nbat, true, a);
  a.post = 5;
  a.xout = out;
  if (rc == PAWFD_OK) rc = fft_xy<float>(c, c->pc, work, work, nbat, true, a);
  return rc;
}

int check_pw_call(pawfd_ctx* c, const void* a, const void* b, int nb) {
  if (!c) return PAWFD_EINVAL;
  if (!a || !b) return fail(c, PAWFD_EINVAL, "null array");
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  return ensure_pw(c);
}

}  // namespace

void free_pw(pawfd_ctx* c) {
  free_plan(c->pw);
  free_plan(c->pc);
  if (c->d_pc_work) cudaFree(c->d_pc_work);
  c->d_pc_work = nullptr;
  c->pc_work_bytes = 0;
}

bool kinetic_precond_available(const pawfd_ctx* c) {
  int fac[MAX_FAC], nf;
  for (int ax = 0; ax < 3; ++ax)
    if (!factorize(c->n[ax], fac, &nf)) return false;
  return true;
}

size_t kinetic_precond_work_bytes(const pawfd_ctx* c, int nb) {
  return sizeof(zf) * (size_t)c->K * (size_t)(is_complex(c) ? nb : (nb + 1) / 2);
}

// -(T + sigma)^-1 of nb band arrays R into out (may be R), through work (at least
// kinetic_precond_work_bytes, or null: the context's own, allocated on first need)
int launch_kinetic_precond(pawfd_ctx* c, const void* R, int nb, void* out, void* work, size_t work_bytes) {
  int rc = ensure_pc(c);
  if (rc != PAWFD_OK) return rc;
  const size_t need = kinetic_precond_work_bytes(c, nb);
  if (!work || work_bytes < need) {
    if (c->pc_work_bytes < need) {
      rc = check_cuda(c, cudaStreamSynchronize(c->stream), "stream sync");
      if (rc != PAWFD_OK) return rc;
      if (c->d_pc_work) cudaFree(c->d_pc_work);
      c->d_pc_work = nullptr;
      c->pc_work_bytes = 0;
      if (cudaMalloc(&c->d_pc_work, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PAWFD_ENOMEM, "kinetic preconditioner work array");
      }
      c->pc_work_bytes = need;
    }
    work = c->d_pc_work;
  }
  return kinetic_precond_impl(c, R, nb, out, (zf*)work);
}

}  // namespace pawfd

using namespace pawfd;

static int pw_apply(pawfd_ctx* c, int which, const void* C, int nb, double ecut, void* out, void* work) {
  int rc = check_pw_call(c, C, out, nb);
  if (rc != PAWFD_OK) return rc;
  if (!work) return fail(c, PAWFD_EINVAL, "null work array");
  if (C == out || C == work || out == work) return fail(c, PAWFD_EINVAL, "C, out and work may not alias");
  if (is_fp32(c)) return pw_apply_impl<float>(c, which, (const zf*)C, nb, ecut, (zf*)out, (zf*)work);
  return pw_apply_impl<double>(c, which, (const zd*)C, nb, ecut, (zd*)out, (zd*)work);
}

extern "C" int pawfd_pw_apply_H(pawfd_ctx* c, const void* C, int nb, double ecut, void* HC, void* work) {
  return pw_apply(c, 0, C, nb, ecut, HC, work);
}

extern "C" int pawfd_pw_apply_S(pawfd_ctx* c, const void* C, int nb, double ecut, void* SC, void* work) {
  return pw_apply(c, 1, C, nb, ecut, SC, work);
}

extern "C" int pawfd_poisson_fft(pawfd_ctx* c, const double* rho, double* v, void* work) {
  if (!c) return PAWFD_EINVAL;
  if (c->dtype != PAWFD_R64) return fail(c, PAWFD_EINVAL, "pawfd_poisson_fft needs a real FP64 context");
  if (!c->free_operator) return fail(c, PAWFD_EINVAL, "pawfd_poisson_fft needs a context with v = 0 and no atoms");
  if (!rho || !v || !work) return fail(c, PAWFD_EINVAL, "null array");
  if ((const void*)rho == work || (void*)v == work) return fail(c, PAWFD_EINVAL, "work may not alias rho or v");
  const int rc = ensure_pw(c, false);
  if (rc != PAWFD_OK) return rc;
  return poisson_fft_impl(c, rho, v, (zd*)work);
}

extern "C" int pawfd_kinetic_precond(pawfd_ctx* c, const void* R, int nb, void* out, void* work) {
  if (!c) return PAWFD_EINVAL;
  if (nb < 1 || nb > c->max_bands) return fail(c, PAWFD_EINVAL, "nb must be in 1..max_bands");
  if (!R || !out || !work) return fail(c, PAWFD_EINVAL, "null array");
  if (work == R || work == out) return fail(c, PAWFD_EINVAL, "work may not alias R or out");
  return launch_kinetic_precond(c, R, nb, out, work, kinetic_precond_work_bytes(c, nb));
}

extern "C" int pawfd_pw_to_grid(pawfd_ctx* c, const void* C, int nb, void* psi) {
  int rc = check_pw_call(c, C, psi, nb);
  if (rc != PAWFD_OK) return rc;
  if (C == psi) return fail(c, PAWFD_EINVAL, "C and psi may not alias");
  if (is_fp32(c)) return pw_inverse<float>(c, (const zf*)C, nb, (zf*)psi, nullptr, nullptr);
  return pw_inverse<double>(c, (const zd*)C, nb, (zd*)psi, nullptr, nullptr);
}

extern "C" int pawfd_pw_from_grid(pawfd_ctx* c, const void* psi, int nb, void* C, void* work) {
  int rc = check_pw_call(c, psi, C, nb);
  if (rc != PAWFD_OK) return rc;
  if (!work) return fail(c, PAWFD_EINVAL, "null work array");
  if (psi == C || psi == work || C == work) return fail(c, PAWFD_EINVAL, "psi, C and work may not alias");
  const size_t bytes = (is_fp32(c) ? sizeof(zf) : sizeof(zd)) * (size_t)nb * c->K;
  rc = check_cuda(c, cudaMemcpyAsync(work, psi, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy");
  if (rc != PAWFD_OK) return rc;
  if (is_fp32(c)) return pw_forward<float>(c, (zf*)work, nb, (zf*)C, nullptr, false, 0.0);
  return pw_forward<double>(c, (zd*)work, nb, (zd*)C, nullptr, false, 0.0);
}
