// context.cu -- context creation: validates the system description and builds the device
// tables (shifted local potential, folded projector boxes, atom colouring, scratch).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "pawfd_internal.cuh"

namespace pawfd {

int fail(pawfd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int check_cuda(pawfd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PAWFD_OK;
  return fail(c, PAWFD_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

template <class T>
T* dev_alloc(pawfd_ctx* c, size_t count, int* rc) {
  if (*rc != PAWFD_OK) return nullptr;
  T* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    *rc = fail(c, PAWFD_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return nullptr;
  }
  return p;
}

template <class T>
void upload(pawfd_ctx* c, T* dst, const T* src, size_t count, int* rc) {
  if (*rc != PAWFD_OK || count == 0) return;
  *rc = check_cuda(c, cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice), "cudaMemcpy H2D");
}

long long floor_div(long long u, long long n) { return (u >= 0) ? u / n : -((-u + n - 1) / n); }

struct BoxPoint {
  long long grid;   // wrapped grid index
  long long j;      // index inside the box
  double kt;        // k . T of the image this point belongs to
};

// Fold atom a's box onto the grid: G[i][q] = sum over box points j that wrap onto the q-th
// unique grid point of p_i(j) * exp(-i k.T_j).  The projection uses conj(G), the back-add G.
void fold_atom(const pawfd_system_desc* d, int a, std::vector<int>& pts, std::vector<double>& g_re,
               std::vector<double>& g_im) {
  const int* lo = d->box_lo + 3 * a;
  const int* bn = d->box_n + 3 * a;
  const long long bsize = (long long)bn[0] * bn[1] * bn[2];
  const int I = d->nproj[a];
  std::vector<BoxPoint> bp;
  bp.reserve(bsize);
  for (int j3 = 0; j3 < bn[2]; ++j3)
    for (int j2 = 0; j2 < bn[1]; ++j2)
      for (int j1 = 0; j1 < bn[0]; ++j1) {
        long long u[3] = {(long long)lo[0] + j1, (long long)lo[1] + j2, (long long)lo[2] + j3};
        long long w[3];
        double kt = 0.0;
        for (int c = 0; c < 3; ++c) {
          long long t = floor_div(u[c], d->n[c]);
          w[c] = u[c] - t * d->n[c];
          kt += d->k[c] * d->cell[c] * (double)t;
        }
        long long grid = (w[2] * d->n[1] + w[1]) * d->n[0] + w[0];
        bp.push_back(BoxPoint{grid, ((long long)j3 * bn[1] + j2) * bn[0] + j1, kt});
      }
  std::stable_sort(bp.begin(), bp.end(), [](const BoxPoint& x, const BoxPoint& y) { return x.grid < y.grid; });
  pts.clear();
  std::vector<size_t> first;
  for (size_t q = 0; q < bp.size(); ++q)
    if (q == 0 || bp[q].grid != bp[q - 1].grid) {
      pts.push_back((int)bp[q].grid);
      first.push_back(q);
    }
  first.push_back(bp.size());
  const size_t np = pts.size();
  g_re.assign((size_t)I * np, 0.0);
  g_im.assign((size_t)I * np, 0.0);
  const double* p = d->proj + d->proj_off[a];
  for (size_t q = 0; q < np; ++q)
    for (size_t e = first[q]; e < first[q + 1]; ++e) {
      const double cr = std::cos(bp[e].kt), ci = -std::sin(bp[e].kt);
      for (int i = 0; i < I; ++i) {
        const double val = p[(size_t)i * bsize + bp[e].j];
        g_re[(size_t)i * np + q] += val * cr;
        g_im[(size_t)i * np + q] += val * ci;
      }
    }
}

int validate(const pawfd_system_desc* d, std::string& why) {
  if (!d) return why = "desc is NULL", PAWFD_EINVAL;
  for (int c = 0; c < 3; ++c) {
    if (d->n[c] < 1) return why = "grid size must be >= 1", PAWFD_EINVAL;
    if (!(d->cell[c] > 0.0)) return why = "cell lengths must be > 0", PAWFD_EINVAL;
  }
  if ((long long)d->n[0] * d->n[1] * d->n[2] > (1ll << 31) - 1) return why = "grid too large", PAWFD_EINVAL;
  if (d->dtype < PAWFD_R64 || d->dtype > PAWFD_C64) return why = "unsupported dtype", PAWFD_EINVAL;
  if ((d->dtype == PAWFD_R64 || d->dtype == PAWFD_R32) && (d->k[0] != 0.0 || d->k[1] != 0.0 || d->k[2] != 0.0))
    return why = "real wave functions need k = 0", PAWFD_EINVAL;
  if (d->max_bands < 1) return why = "max_bands must be >= 1", PAWFD_EINVAL;
  if (!d->vloc) return why = "vloc is NULL", PAWFD_EINVAL;
  if (d->natoms < 0) return why = "natoms < 0", PAWFD_EINVAL;
  if (d->natoms > 0) {
    if (!d->nproj || !d->box_lo || !d->box_n || !d->proj || !d->proj_off || !d->dH || !d->dS || !d->dmat_off)
      return why = "atom arrays missing", PAWFD_EINVAL;
    for (int a = 0; a < d->natoms; ++a) {
      if (d->nproj[a] < 1 || d->nproj[a] > 32) return why = "nproj must be in 1..32", PAWFD_EINVAL;
      for (int c = 0; c < 3; ++c)
        if (d->box_n[3 * a + c] < 1) return why = "box sizes must be >= 1", PAWFD_EINVAL;
      const long long bsize = (long long)d->box_n[3 * a] * d->box_n[3 * a + 1] * d->box_n[3 * a + 2];
      if (d->proj_off[a + 1] - d->proj_off[a] != bsize * d->nproj[a])
        return why = "proj_off inconsistent with box sizes", PAWFD_EINVAL;
      if (d->dmat_off[a + 1] - d->dmat_off[a] != (long long)d->nproj[a] * d->nproj[a])
        return why = "dmat_off inconsistent with nproj", PAWFD_EINVAL;
    }
  }
  return PAWFD_OK;
}

}  // namespace

int build_tables(pawfd_ctx* c, const pawfd_system_desc* d) {
  int rc = PAWFD_OK;
  AtomTables& at = c->at;
  at.natoms = d->natoms;
  const bool cplx = is_complex(c);
  const bool fp32 = is_fp32(c);
  std::vector<int> all_pts;
  std::vector<double> all_re, all_im;
  at.pt_off.assign(1, 0);
  at.g_off.assign(1, 0);
  at.row_off.assign(1, 0);
  at.dmat_off.assign(d->dmat_off, d->dmat_off + d->natoms + 1);
  for (int a = 0; a < d->natoms; ++a) {
    std::vector<int> pts;
    std::vector<double> re, im;
    fold_atom(d, a, pts, re, im);
    at.nproj.push_back(d->nproj[a]);
    at.npts.push_back((int)pts.size());
    all_pts.insert(all_pts.end(), pts.begin(), pts.end());
    all_re.insert(all_re.end(), re.begin(), re.end());
    all_im.insert(all_im.end(), im.begin(), im.end());
    at.pt_off.push_back(at.pt_off.back() + (long long)pts.size());
    at.g_off.push_back(at.g_off.back() + (long long)re.size());
    at.row_off.push_back(at.row_off.back() + d->nproj[a]);
    at.Imax = std::max(at.Imax, d->nproj[a]);
  }
  at.Ip = at.row_off.back();

  // colouring: atoms whose folded boxes share a grid point get different colours
  std::vector<uint64_t> used((size_t)c->K, 0);
  std::vector<int> color_of(d->natoms, 0);
  int ncolors = 0;
  for (int a = 0; a < d->natoms; ++a) {
    uint64_t forbidden = 0;
    for (long long q = at.pt_off[a]; q < at.pt_off[a + 1]; ++q) forbidden |= used[all_pts[q]];
    int col = 0;
    while (col < 64 && (forbidden >> col) & 1ull) ++col;
    if (col == 64) return fail(c, PAWFD_EINVAL, "more than 64 mutually overlapping projector boxes");
    color_of[a] = col;
    ncolors = std::max(ncolors, col + 1);
    for (long long q = at.pt_off[a]; q < at.pt_off[a + 1]; ++q) used[all_pts[q]] |= (1ull << col);
  }
  std::vector<int> color_atoms;
  at.color_off.assign(1, 0);
  at.colors.assign(ncolors, {});
  for (int col = 0; col < ncolors; ++col) {
    for (int a = 0; a < d->natoms; ++a)
      if (color_of[a] == col) {
        color_atoms.push_back(a);
        at.colors[col].push_back(a);
      }
    at.color_off.push_back((int)color_atoms.size());
  }

  // work items: each atom's box points in runs of NL_PCH, so that large boxes spread over
  // many CTAs (the FP64 rate of one SM would otherwise bound a whole box)
  std::vector<int2> items, color_items;
  std::vector<long long> item_row;
  std::vector<int> atom_items(1, 0);
  for (int a = 0; a < d->natoms; ++a) {
    for (int p0 = 0; p0 < at.npts[a]; p0 += NL_PCH) {
      items.push_back(make_int2(a, p0));
      item_row.push_back(at.part_rows);
      at.part_rows += at.nproj[a];
    }
    atom_items.push_back((int)items.size());
  }
  at.nitems = (int)items.size();
  at.color_item_off.assign(1, 0);
  for (int col = 0; col < ncolors; ++col) {
    for (int a : at.colors[col])
      for (int p0 = 0; p0 < at.npts[a]; p0 += NL_PCH) color_items.push_back(make_int2(a, p0));
    at.color_item_off.push_back((int)color_items.size());
  }

  const int A = d->natoms;
  at.d_items = dev_alloc<int2>(c, std::max<size_t>(1, items.size()), &rc);
  at.d_item_row = dev_alloc<long long>(c, std::max<size_t>(1, item_row.size()), &rc);
  at.d_atom_items = dev_alloc<int>(c, atom_items.size(), &rc);
  at.d_color_items = dev_alloc<int2>(c, std::max<size_t>(1, color_items.size()), &rc);
  upload(c, at.d_items, items.data(), items.size(), &rc);
  upload(c, at.d_item_row, item_row.data(), item_row.size(), &rc);
  upload(c, at.d_atom_items, atom_items.data(), atom_items.size(), &rc);
  upload(c, at.d_color_items, color_items.data(), color_items.size(), &rc);
  at.d_nproj = dev_alloc<int>(c, A, &rc);
  at.d_row_off = dev_alloc<int>(c, A + 1, &rc);
  at.d_npts = dev_alloc<int>(c, A, &rc);
  at.d_pt_off = dev_alloc<long long>(c, A + 1, &rc);
  at.d_pts = dev_alloc<int>(c, all_pts.size(), &rc);
  at.d_g_off = dev_alloc<long long>(c, A + 1, &rc);
  at.d_dmat_off = dev_alloc<long long>(c, A + 1, &rc);
  const long long ndm = A ? d->dmat_off[A] : 0;
  at.d_color_atoms = dev_alloc<int>(c, color_atoms.size(), &rc);
  upload(c, at.d_nproj, at.nproj.data(), A, &rc);
  upload(c, at.d_row_off, at.row_off.data(), A + 1, &rc);
  upload(c, at.d_npts, at.npts.data(), A, &rc);
  upload(c, at.d_pt_off, at.pt_off.data(), A + 1, &rc);
  upload(c, at.d_pts, all_pts.data(), all_pts.size(), &rc);
  upload(c, at.d_g_off, at.g_off.data(), A + 1, &rc);
  upload(c, at.d_dmat_off, at.dmat_off.data(), A + 1, &rc);
  if (fp32) {
    std::vector<float> h(d->dH, d->dH + ndm), s(d->dS, d->dS + ndm);
    float* dh = dev_alloc<float>(c, ndm, &rc);
    float* ds = dev_alloc<float>(c, ndm, &rc);
    upload(c, dh, h.data(), ndm, &rc);
    upload(c, ds, s.data(), ndm, &rc);
    at.d_dH = dh;
    at.d_dS = ds;
  } else {
    double* dh = dev_alloc<double>(c, ndm, &rc);
    double* ds = dev_alloc<double>(c, ndm, &rc);
    upload(c, dh, d->dH, ndm, &rc);
    upload(c, ds, d->dS, ndm, &rc);
    at.d_dH = dh;
    at.d_dS = ds;
  }
  upload(c, at.d_color_atoms, color_atoms.data(), color_atoms.size(), &rc);
  if (cplx && !fp32) {
    std::vector<zd> g(all_re.size());
    for (size_t q = 0; q < g.size(); ++q) g[q] = zd{all_re[q], all_im[q]};
    zd* dg = dev_alloc<zd>(c, g.size(), &rc);
    upload(c, dg, g.data(), g.size(), &rc);
    at.d_g = dg;
  } else if (cplx) {
    std::vector<zf> g(all_re.size());
    for (size_t q = 0; q < g.size(); ++q) g[q] = zf{(float)all_re[q], (float)all_im[q]};
    zf* dg = dev_alloc<zf>(c, g.size(), &rc);
    upload(c, dg, g.data(), g.size(), &rc);
    at.d_g = dg;
  } else if (fp32) {
    std::vector<float> g(all_re.begin(), all_re.end());
    float* dg = dev_alloc<float>(c, g.size(), &rc);
    upload(c, dg, g.data(), g.size(), &rc);
    at.d_g = dg;
  } else {
    double* dg = dev_alloc<double>(c, all_re.size(), &rc);
    upload(c, dg, all_re.data(), all_re.size(), &rc);
    at.d_g = dg;
    // the same values as (hi, lo) pairs for the double-float projector kernels
    std::vector<float2> gdf(all_re.size());
    for (size_t q = 0; q < gdf.size(); ++q) {
      const float hi = (float)all_re[q];
      gdf[q] = make_float2(hi, (float)(all_re[q] - (double)hi));
    }
    float2* dgdf = dev_alloc<float2>(c, gdf.size(), &rc);
    upload(c, dgdf, gdf.data(), gdf.size(), &rc);
    at.d_g_df = dgdf;
  }
  return rc;
}

void free_ctx(pawfd_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->d_vshift, c->at.d_nproj, c->at.d_row_off, c->at.d_npts, c->at.d_pt_off, c->at.d_pts,
                  c->at.d_g_off, c->at.d_g, c->at.d_dmat_off, c->at.d_dH, c->at.d_dS, c->at.d_color_atoms,
                  c->d_P, c->d_gram_part, c->d_work, c->d_evals, c->d_dscale, c->d_barrier, c->d_status, c->d_reduce,
                  c->d_flags, c->d_oa, c->d_eig, c->d_Q, c->d_Ppart, c->at.d_items, c->at.d_item_row,
                  c->at.d_atom_items, c->at.d_color_items, c->at.d_g_df, c->d_vloc};
  free_pw(c);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->aux_fork) cudaEventDestroy(c->aux_fork);
  if (c->aux_join) cudaEventDestroy(c->aux_join);
  for (int i = 0; i < KernelTimer::CAP; ++i) {
    if (c->ktimer.start[i]) cudaEventDestroy(c->ktimer.start[i]);
    if (c->ktimer.stop[i]) cudaEventDestroy(c->ktimer.stop[i]);
  }
  if (c->h_status) cudaFreeHost(c->h_status);
  free_tc(c);
  delete c;
}

}  // namespace pawfd

using namespace pawfd;

extern "C" int pawfd_create(pawfd_ctx** out, const pawfd_system_desc* d, void* stream) {
  if (!out) return PAWFD_EINVAL;
  *out = nullptr;
  pawfd_ctx* c = new pawfd_ctx();
  std::string why;
  int rc = validate(d, why);
  if (rc != PAWFD_OK) {
    delete c;
    fprintf(stderr, "pawfd_create: %s\n", why.c_str());
    return rc;
  }
  for (int i = 0; i < 3; ++i) {
    c->n[i] = d->n[i];
    c->cell[i] = d->cell[i];
    c->k[i] = d->k[i];
    c->h[i] = d->cell[i] / d->n[i];
  }
  c->dV = c->h[0] * c->h[1] * c->h[2];
  c->dtype = d->dtype;
  c->max_bands = d->max_bands;
  c->K = (size_t)d->n[0] * d->n[1] * d->n[2];
  c->stream = (cudaStream_t)stream;
  int dev = 0;
  rc = check_cuda(c, cudaGetDevice(&dev), "cudaGetDevice");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev), "attr");

  // shifted local potential: the centre weight of the three 1-D stencils folded into v
  if (rc == PAWFD_OK) {
    std::vector<double> vs(c->K);
    const double centre = -0.5 * FD6_W0 * (1.0 / (c->h[0] * c->h[0]) + 1.0 / (c->h[1] * c->h[1]) +
                                           1.0 / (c->h[2] * c->h[2]));
    bool vzero = true;
    for (size_t r = 0; r < c->K; ++r) {
      vs[r] = d->vloc[r] + centre;
      vzero = vzero && d->vloc[r] == 0.0;
    }
    c->free_operator = vzero && d->natoms == 0;
    // and v itself (the fixed-point stencil, whose centre weight is an exact integer, and the
    // plane-wave representation, whose kinetic term is separate)
    if (is_fp32(c)) {
      std::vector<float> vf(vs.begin(), vs.end());
      float* p = dev_alloc<float>(c, c->K, &rc);
      upload(c, p, vf.data(), c->K, &rc);
      c->d_vshift = p;
      std::vector<float> v0(d->vloc, d->vloc + c->K);
      float* q = dev_alloc<float>(c, c->K, &rc);
      upload(c, q, v0.data(), c->K, &rc);
      c->d_vloc = q;
    } else {
      double* p = dev_alloc<double>(c, c->K, &rc);
      upload(c, p, vs.data(), c->K, &rc);
      c->d_vshift = p;
      double* q = dev_alloc<double>(c, c->K, &rc);
      upload(c, q, d->vloc, c->K, &rc);
      c->d_vloc = q;
    }
  }
  if (rc == PAWFD_OK) rc = build_tables(c, d);
  const size_t ss = mat_size(c);
  const size_t nb = (size_t)c->max_bands;
  if (rc == PAWFD_OK) {
    c->d_P = dev_alloc<char>(c, band_size(c) * std::max<size_t>(1, (size_t)c->at.Ip) * nb, &rc);
    c->d_Q = dev_alloc<char>(c, mat_size(c) * std::max<size_t>(1, (size_t)c->at.Ip) * nb, &rc);
    c->d_Ppart = dev_alloc<char>(c, band_size(c) * std::max<size_t>(1, (size_t)c->at.part_rows) * nb, &rc);
    // split-K partials: about eight 64 x 64 tiles per SM at max_bands (Hermitian tiling),
    // capped at 256 MB
    const size_t t1 = (nb + 63) / 64, tiles = t1 * (t1 + 1) / 2;
    size_t nsplit = std::max<size_t>(1, std::min<size_t>(256, (8 * (size_t)c->num_sms + tiles - 1) / tiles));
    while (nsplit > 1 && nsplit * nb * nb * ss > (256ull << 20)) --nsplit;
    c->gram_part_bytes = nsplit * nb * nb * ss;
    c->d_gram_part = dev_alloc<char>(c, c->gram_part_bytes, &rc);
    c->d_work = dev_alloc<char>(c, 7 * nb * nb * ss, &rc);
    c->d_evals = dev_alloc<double>(c, nb, &rc);
    c->d_dscale = dev_alloc<double>(c, nb, &rc);
    c->d_barrier = dev_alloc<unsigned>(c, 4, &rc);
    c->d_status = dev_alloc<DeviceStatus>(c, 1, &rc);
    c->d_reduce = dev_alloc<double>(c, 8192, &rc);   // [0, 2048): partial sums; then Jacobi round flags
    c->d_flags = dev_alloc<int>(c, 16, &rc);
    c->d_oa = dev_alloc<double>(c, oa_scratch_doubles(nb), &rc);
    c->d_eig = dev_alloc<char>(c, eig32_scratch_bytes((int)nb, is_complex(c)), &rc);
  }
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMallocHost(&c->h_status, sizeof(DeviceStatus)), "cudaMallocHost");
  if (rc == PAWFD_OK && c->use_tc) rc = setup_tc(c);
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(c->d_barrier, 0, 4 * sizeof(unsigned)), "memset");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(c->d_flags, 0, 16 * sizeof(int)), "memset");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaMemset(c->d_status, 0, sizeof(DeviceStatus)), "memset");
  // the uploads and memsets above ran on the legacy default stream: wait for those only, not
  // for other work on the device (a server creates contexts while jobs run on their streams)
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamSynchronize(cudaStreamLegacy), "create sync");
  if (rc != PAWFD_OK) {
    fprintf(stderr, "pawfd_create: %s\n", c->err.c_str());
    free_ctx(c);
    return rc;
  }
  *out = c;
  return PAWFD_OK;
}

extern "C" int pawfd_destroy(pawfd_ctx* c) {
  if (!c) return PAWFD_EINVAL;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return PAWFD_OK;
}

extern "C" int pawfd_set_stream(pawfd_ctx* c, void* stream) {
  if (!c) return PAWFD_EINVAL;
  c->stream = (cudaStream_t)stream;
  return PAWFD_OK;
}

extern "C" const char* pawfd_last_error(const pawfd_ctx* c) { return c ? c->err.c_str() : "no context"; }

extern "C" int pawfd_nproj_total(const pawfd_ctx* c) { return c ? c->at.Ip : PAWFD_EINVAL; }

extern "C" long long pawfd_launch_count(const pawfd_ctx* c) { return c ? c->launches : PAWFD_EINVAL; }

extern "C" int pawfd_set_option(pawfd_ctx* c, const char* name, int value) {
  if (!c || !name) return PAWFD_EINVAL;
  const std::string n(name);
  if (n == "tensor_cores" && (value == 0 || value == 1)) {
    if (value == 1 && !c->tc.ready) return fail(c, PAWFD_EINVAL, "tensor-core scratch not set up");
    c->use_tc = value == 1;
    return PAWFD_OK;
  }
  if (n == "stencil_variant" && value >= 0 && value <= 2) {
    c->stencil_variant = value;
    c->fast_stencil = value != 2;
    return PAWFD_OK;
  }
  if (n == "stencil_rows" && value >= 0 && value <= 64) {
    c->stencil_rows = value;
    return PAWFD_OK;
  }
  if (n == "jacobi_cluster" && (value == 0 || value == 1)) {
    c->jacobi_cluster = value == 1;
    return PAWFD_OK;
  }
  if (n == "davidson_precond" && (value == 0 || value == 1)) {
    c->davidson_precond = value;
    return PAWFD_OK;
  }
  if (n == "tridiag_dsm" && (value == 0 || value == 1)) {
    c->tridiag_dsm = value == 1;
    return PAWFD_OK;
  }
  if (n == "test_barrier_missing" && (value == 0 || value == 1)) {
    // test setting: grid barriers wait for one CTA more than the launch has, for 20 ms, so
    // that every grid-barrier wait runs out and reports PAWFD_ETIMEDOUT
    const unsigned f[2] = {(unsigned)value, value ? 20u : 0u};
    int rc = check_cuda(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (rc == PAWFD_OK)
      rc = check_cuda(c, cudaMemcpy(&c->d_status->barrier_extra, f, sizeof f, cudaMemcpyHostToDevice), "memcpy");
    return rc;
  }
  if (n == "stencil_fx" && (value == 0 || value == 1)) {
    c->stencil_fx = value == 1;
    return PAWFD_OK;
  }
  if (n == "nonlocal_df" && (value == 0 || value == 1)) {
    c->nonlocal_df = value == 1;
    return PAWFD_OK;
  }
  if (n == "tc_scratch_mb" && value >= 0 && value <= (1 << 20)) {
    // re-size the digit-plane scratch: wait for the work in flight, free, allocate again
    c->tc_scratch_mb = value;
    if (!c->tc.ready) return PAWFD_OK;
    int rc = check_cuda(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (rc != PAWFD_OK) return rc;
    free_tc(c);
    rc = setup_tc(c);
    if (rc != PAWFD_OK) {
      free_tc(c);
      c->use_tc = false;
    }
    return rc;
  }
  if (n == "tc_kblk" && value >= 0 && value <= 4096) {
    c->tc_kblk_chunks = value;
    return PAWFD_OK;
  }
  if (n == "stencil_ring" && (value == 0 || value == 6 || value == 8 || value == 10 || value == 12)) {
    c->stencil_ring = value;
    return PAWFD_OK;
  }
  if (n == "stencil_zsplit" && value >= 0 && value <= 64) {
    c->stencil_zsplit = value;
    return PAWFD_OK;
  }
  if (n == "stencil_yblock" && value >= 0 && value <= 3) {
    c->stencil_yblock = value;
    return PAWFD_OK;
  }
  return fail(c, PAWFD_EINVAL, "unknown option or value");
}

namespace pawfd {
int ensure_aux_stream(pawfd_ctx* c) {
  if (c->aux_stream) return PAWFD_OK;
  int e = check_cuda(c, cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking), "aux stream");
  if (e == PAWFD_OK) e = check_cuda(c, cudaEventCreateWithFlags(&c->aux_fork, cudaEventDisableTiming), "event");
  if (e == PAWFD_OK) e = check_cuda(c, cudaEventCreateWithFlags(&c->aux_join, cudaEventDisableTiming), "event");
  return e;
}

void ktimer_begin(pawfd_ctx* c) {
  KernelTimer& t = c->ktimer;
  if (!t.on) return;
  // launches captured into a CUDA graph are not timed (their events would only be recorded
  // when the graph runs); ktimer_end sees the same answer
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    t.capturing = true;
    return;
  }
  t.capturing = false;
  if (t.used >= KernelTimer::CAP) {
    t.overflow = true;
    return;
  }
  if (!t.start[t.used]) {
    cudaEventCreate(&t.start[t.used]);
    cudaEventCreate(&t.stop[t.used]);
  }
  cudaEventRecord(t.start[t.used], c->stream);
}
void ktimer_end(pawfd_ctx* c) {
  KernelTimer& t = c->ktimer;
  if (!t.on || t.capturing || t.used >= KernelTimer::CAP) return;
  cudaEventRecord(t.stop[t.used], c->stream);
  ++t.used;
}
}  // namespace pawfd

extern "C" int pawfd_kernel_timing(pawfd_ctx* c, int enable, double* total_ms, long long* launches) {
  if (!c) return PAWFD_EINVAL;
  KernelTimer& t = c->ktimer;
  double ms = 0.0;
  int rc = PAWFD_OK;
  if (t.used > 0) {
    rc = check_cuda(c, cudaEventSynchronize(t.stop[t.used - 1]), "timing event");
    for (int i = 0; i < t.used && rc == PAWFD_OK; ++i) {
      float e = 0.0f;
      rc = check_cuda(c, cudaEventElapsedTime(&e, t.start[i], t.stop[i]), "timing event");
      ms += e;
    }
  }
  if (total_ms) *total_ms = ms;
  if (launches) *launches = t.overflow ? -1 : t.used;
  t.used = 0;
  t.overflow = false;
  t.on = enable != 0;
  return rc;
}

extern "C" int pawfd_sync(pawfd_ctx* c) {
  if (!c) return PAWFD_EINVAL;
  int rc = check_cuda(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DeviceStatus), cudaMemcpyDeviceToHost,
                                         c->stream), "status copy");
  if (rc == PAWFD_OK) rc = check_cuda(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (rc != PAWFD_OK) return rc;
  const DeviceStatus st = *c->h_status;
  if (st.code == 0) return PAWFD_OK;
  cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream);   // code and detail only
  cudaStreamSynchronize(c->stream);
  char buf[160];
  switch (st.code) {
    case PAWFD_ENOTPD: snprintf(buf, sizeof buf, "S_nm not positive definite: Cholesky pivot <= 0 at column %d", st.detail); break;
    case PAWFD_ENOCONV: snprintf(buf, sizeof buf, "Jacobi eigensolver did not converge within %d sweeps", st.detail); break;
    case PAWFD_ETIMEDOUT: snprintf(buf, sizeof buf, "device barrier wait gave up (barrier %d)", st.detail); break;
    default: snprintf(buf, sizeof buf, "device error %d (detail %d)", st.code, st.detail); break;
  }
  return fail(c, st.code, buf);
}
