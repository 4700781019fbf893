// Scene construction, the lockstep Newton / PN / PPN driver and the C ABI.
//
// One time step (backward Euler as incremental-potential minimisation,
// Sec. 2.1 / 5.1) runs Newton's method (Sec. 3) with, per mode:
//   NEWTON  unprojected H; on negative curvature the solver's last iterate is
//           the step (Newton-CG, Sec. 4.1)
//   PN      every element clamped before assembly (Sec. 3)
//   PPN     Algorithm 1: solve on the unprojected H; while the solver reports
//           indefiniteness, select elements with ||S^e g||_inf > delta (delta
//           initialised to alpha ||g||_inf, tightened by alpha), clamp them and
//           update H in place (Sec. 4.1), solve again; relax delta by beta.
// followed by a backtracking line search for sufficient decrease (Sec. 5.1).
//
// Several scenes step together as a "group": every phase is one launch over
// the scenes still taking part in it, and every host decision is taken per
// scene after one device->host copy of all scenes' control blocks.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>

#include "driver.h"

namespace ppn {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

const char* kFamilyNames[FAM_COUNT] = {"element", "gradient", "assemble", "select", "project",
                                       "update",  "pcg",      "energy",   "vector"};


// ------------------------------------------------------------------ staging
Staging::~Staging() {
  if (base) cudaFreeHost(base);
}

void* Staging::take(size_t n, cudaStream_t st) {
  n = (n + 255) & ~size_t(255);
  if (!base) {
    cap = std::max<size_t>(4 << 20, 2 * n);
    if (cudaMallocHost(&base, cap) != cudaSuccess) {
      base = nullptr;
      return nullptr;
    }
  }
  if (off + n > cap) {
    // every earlier upload must have been consumed before the slot is reused
    cudaStreamSynchronize(st);
    off = 0;
    if (n > cap) {
      cudaFreeHost(base);
      cap = 2 * n;
      if (cudaMallocHost(&base, cap) != cudaSuccess) {
        base = nullptr;
        return nullptr;
      }
    }
  }
  void* p = base + off;
  off += n;
  return p;
}

// ------------------------------------------------------------------ timers
KernelTimer::~KernelTimer() {
  for (auto& r : pending) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}
cudaEvent_t KernelTimer::ev() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
void KernelTimer::begin(int fam, cudaStream_t st, double b) {
  if (!on) return;
  Rec r{fam, ev(), ev(), b};
  cudaEventRecord(r.a, st);
  pending.push_back(r);
}
void KernelTimer::end(cudaStream_t st) {
  if (!on || pending.empty()) return;
  cudaEventRecord(pending.back().b, st);
}
void KernelTimer::collect() {
  for (auto& r : pending) {
    float ms_ = 0.f;
    if (cudaEventElapsedTime(&ms_, r.a, r.b) == cudaSuccess) {
      ms[r.fam] += ms_;
      launches[r.fam] += 1;
      bytes[r.fam] += r.bytes;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
}
void KernelTimer::reset() {
  collect();
  for (int i = 0; i < 16; ++i) {
    launches[i] = 0;
    ms[i] = 0;
    bytes[i] = 0;
  }
}

// ------------------------------------------------------------------ scene
template <typename T>
template <typename X>
X* SceneImpl<T>::alloc(size_t n) {
  if (n == 0) n = 1;
  void* p = dev_alloc(dalloc, n * sizeof(X));
  if (!p) return nullptr;
  allocs.push_back(p);
  dev_bytes += n * sizeof(X);
  return reinterpret_cast<X*>(p);
}

template <typename T>
SceneImpl<T>::~SceneImpl() {
  if (stream) cudaStreamSynchronize(stream);
  for (void* p : allocs) dev_free(dalloc, p);
  if (h_ctl) cudaFreeHost(h_ctl);
  if (ev_a) cudaEventDestroy(ev_a);
  if (ev_b) cudaEventDestroy(ev_b);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

static std::vector<TileRef> make_tiles(int scene, int n_items, int tile) {
  std::vector<TileRef> t;
  const int n = (n_items + tile - 1) / tile;
  t.reserve(n);
  for (int i = 0; i < n; ++i) t.push_back({scene, i});
  return t;
}

template <typename T>
ppn_status SceneImpl<T>::init(const double* rest_xyz, int64_t n_verts, const int32_t* tets,
                              int64_t n_tets, const ppn_material* mat, double dt_, const int32_t* fixed,
                              int64_t n_fixed, const ppn_params* p) {
  if (!rest_xyz || !tets || !mat || n_verts <= 0 || n_tets <= 0 || n_fixed < 0 ||
      (n_fixed > 0 && !fixed)) {
    set_error("null pointer or empty mesh");
    return PPN_ERR_INVALID_ARG;
  }
  if (n_tets >= (1ll << 27) || n_verts >= (1ll << 30)) {
    set_error("mesh too large for 32-bit element maps");
    return PPN_ERR_INVALID_ARG;
  }
  if (!(dt_ > 0) || !(mat->rho > 0) || !(mat->E > 0) || !(mat->nu > -1.0 && mat->nu < 0.5)) {
    set_error("invalid material or time step");
    return PPN_ERR_INVALID_ARG;
  }
  params = p ? *p : ppn_default_params();
  if ((params.projection != PPN_PROJ_CLAMP && params.projection != PPN_PROJ_MIRROR) || params.pdn_countdown < 0 ||
      !(params.alpha > 0 && params.alpha < 1) || !(params.beta >= 1) || !(params.eig_eps >= 0)) {
    set_error("invalid parameters (projection kind, pdn_countdown, alpha in (0,1), beta >= 1, eig_eps >= 0)");
    return PPN_ERR_INVALID_ARG;
  }
  if (!(params.dirichlet_penalty >= 0.0) || !std::isfinite(params.dirichlet_penalty)) {
    set_error("dirichlet_penalty must be finite and >= 0");
    return PPN_ERR_INVALID_ARG;
  }
  if (!(params.tie_band >= 0.0) || !std::isfinite(params.tie_band)) {
    set_error("tie_band must be finite and >= 0");
    return PPN_ERR_INVALID_ARG;
  }
  const bool penalty = params.dirichlet_penalty > 0.0;
  dt = dt_;
  nv = (int)n_verts;
  nt = (int)n_tets;
  nfixed = (int)n_fixed;
  rest.assign(rest_xyz, rest_xyz + 3 * n_verts);

  // --- tets: range check, orientation, Dm^-1, volume, lumped mass
  const double mu = mat->E / (2.0 * (1.0 + mat->nu));
  const double lam = mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu)) + mu;
  std::vector<int4> h_tets(nt);
  std::vector<T> h_tetc((size_t)nt * TETC_STRIDE);
  std::vector<double> mass(nv, 0.0);
  for (int e = 0; e < nt; ++e) {
    int v[4];
    for (int a = 0; a < 4; ++a) {
      v[a] = tets[4 * (int64_t)e + a];
      if (v[a] < 0 || v[a] >= nv) {
        set_error("tet index out of range at tet " + std::to_string(e));
        return PPN_ERR_INVALID_ARG;
      }
    }
    double D[9];
    auto build = [&](double* M) {
      for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) M[3 * i + a] = rest[3 * v[a + 1] + i] - rest[3 * v[0] + i];
    };
    build(D);
    double C[9];
    cof3(D, C);
    double det = D[0] * C[0] + D[1] * C[1] + D[2] * C[2];
    double hmax = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double l2 = 0;
        for (int k = 0; k < 3; ++k) {
          const double d = rest[3 * v[a] + k] - rest[3 * v[b] + k];
          l2 += d * d;
        }
        hmax = std::max(hmax, std::sqrt(l2));
      }
    if (!(std::fabs(det) > 1e-14 * hmax * hmax * hmax)) {
      set_error("degenerate tet " + std::to_string(e));
      return PPN_ERR_DEGENERATE_TET;
    }
    if (det < 0) {
      std::swap(v[2], v[3]);
      build(D);
      cof3(D, C);
      det = -det;
    }
    h_tets[e] = make_int4(v[0], v[1], v[2], v[3]);
    T* tc = &h_tetc[(size_t)e * TETC_STRIDE];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) tc[3 * i + j] = (T)(C[3 * j + i] / det);  // Dm^-1 = cof^T / det
    tc[9] = (T)(det / 6.0);
    tc[10] = (T)mu;
    tc[11] = (T)lam;
    for (int a = 0; a < 4; ++a) mass[v[a]] += mat->rho * (det / 6.0) / 4.0;
  }
  std::vector<uint8_t> fixed_flag(nv, 0);
  fixed_list.resize(nfixed);
  for (int f = 0; f < nfixed; ++f) {
    const int v = fixed[f];
    if (v < 0 || v >= nv || fixed_flag[v]) {
      set_error("fixed index out of range or repeated");
      return PPN_ERR_INVALID_ARG;
    }
    fixed_flag[v] = 1;
    fixed_list[f] = v;
  }
  for (int v = 0; v < nv; ++v)
    if ((penalty || !fixed_flag[v]) && !(mass[v] > 0)) {
      set_error("free vertex " + std::to_string(v) + " has no incident tet");
      return PPN_ERR_INVALID_ARG;
    }

  // --- BSR pattern (full symmetric, sorted, diagonal always present)
  std::vector<uint64_t> keys;
  keys.reserve((size_t)16 * nt + nv);
  for (int e = 0; e < nt; ++e) {
    const int v[4] = {h_tets[e].x, h_tets[e].y, h_tets[e].z, h_tets[e].w};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) keys.push_back(((uint64_t)v[a] << 32) | (uint32_t)v[b]);
  }
  for (int v = 0; v < nv; ++v) keys.push_back(((uint64_t)v << 32) | (uint32_t)v);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  if (keys.size() >= (size_t)INT32_MAX) {
    set_error("pattern too large");
    return PPN_ERR_INVALID_ARG;
  }
  nnzb = (int)keys.size();
  h_row_ptr.assign(nv + 1, 0);
  h_col.resize(nnzb);
  std::vector<int> blk_row(nnzb), diag_idx(nv);
  for (int k = 0; k < nnzb; ++k) {
    const int i = (int)(keys[k] >> 32), j = (int)(keys[k] & 0xffffffffu);
    h_col[k] = j;
    blk_row[k] = i;
    h_row_ptr[i + 1]++;
    if (i == j) diag_idx[i] = k;
  }
  for (int i = 0; i < nv; ++i) h_row_ptr[i + 1] += h_row_ptr[i];
  keys.clear();
  keys.shrink_to_fit();
  auto find_block = [&](int i, int j) {
    const int* b = h_col.data() + h_row_ptr[i];
    const int* e = h_col.data() + h_row_ptr[i + 1];
    return (int)(std::lower_bound(b, e, j) - h_col.data());
  };
  // block -> (tet, a, b) contributions, element order within each block
  std::vector<int> blk_ptr(nnzb + 1, 0), blk_src((size_t)16 * nt);
  std::vector<int> blk_of((size_t)16 * nt);
  for (int e = 0; e < nt; ++e) {
    const int v[4] = {h_tets[e].x, h_tets[e].y, h_tets[e].z, h_tets[e].w};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const int k = find_block(v[a], v[b]);
        blk_of[(size_t)16 * e + 4 * a + b] = k;
        blk_ptr[k + 1]++;
      }
  }
  for (int k = 0; k < nnzb; ++k) blk_ptr[k + 1] += blk_ptr[k];
  {
    std::vector<int> fill(blk_ptr.begin(), blk_ptr.end() - 1);
    for (int e = 0; e < nt; ++e)
      for (int ab = 0; ab < 16; ++ab) {
        const int k = blk_of[(size_t)16 * e + ab];
        blk_src[fill[k]++] = (e << 4) | ab;
      }
  }
  nmap = 16 * nt;
  // vertex -> (tet, corner)
  std::vector<int> vt_ptr(nv + 1, 0), vt_src((size_t)4 * nt);
  for (int e = 0; e < nt; ++e) {
    vt_ptr[h_tets[e].x + 1]++;
    vt_ptr[h_tets[e].y + 1]++;
    vt_ptr[h_tets[e].z + 1]++;
    vt_ptr[h_tets[e].w + 1]++;
  }
  for (int v = 0; v < nv; ++v) vt_ptr[v + 1] += vt_ptr[v];
  {
    std::vector<int> fill(vt_ptr.begin(), vt_ptr.end() - 1);
    for (int e = 0; e < nt; ++e) {
      const int v[4] = {h_tets[e].x, h_tets[e].y, h_tets[e].z, h_tets[e].w};
      for (int a = 0; a < 4; ++a) vt_src[fill[v[a]]++] = (e << 2) | a;
    }
  }

  // --- device allocation and upload
  PPN_CU(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
  own_stream = true;
  PPN_CU(cudaEventCreate(&ev_a));
  PPN_CU(cudaEventCreate(&ev_b));
  n_vtiles = (nv + TILE - 1) / TILE;
  n_ttiles = (nt + TILE - 1) / TILE;
  n_btiles = (nnzb + TILE - 1) / TILE;
  n_ptiles = (nv + PCG_TILE - 1) / PCG_TILE;
  using V4 = vec4_t<T>;
  SceneDev<T> s{};
  s.nv = nv;
  s.nt = nt;
  s.nnzb = nnzb;
  s.nmap = nmap;
  s.n_vtiles = n_vtiles;
  s.n_ttiles = n_ttiles;
  s.n_ptiles = n_ptiles;
  int4* d_tets = alloc<int4>(nt);
  T* d_tetc = alloc<T>((size_t)nt * TETC_STRIDE);
  double* d_mass = alloc<double>(nv);
  uint8_t* d_fixed = alloc<uint8_t>(nv);
  uint8_t* d_con = alloc<uint8_t>(nv);
  s.tgt = alloc<double4>(nv);
  double4* d_X = alloc<double4>(nv);
  int* d_vt_ptr = alloc<int>(nv + 1);
  int* d_vt_src = alloc<int>((size_t)4 * nt);
  int* d_row_ptr = alloc<int>(nv + 1);
  int* d_col = alloc<int>(nnzb);
  int* d_blk_row = alloc<int>(nnzb);
  int* d_blk_ptr = alloc<int>(nnzb + 1);
  int* d_blk_src = alloc<int>((size_t)16 * nt);
  unsigned char* d_blk_lane = alloc<unsigned char>((size_t)16 * nt);
  int* d_diag = alloc<int>(nv);
  int* d_tet_blk = alloc<int>((size_t)16 * nt);
  s.blk_mark = alloc<int>(nnzb);
  s.touched = alloc<int>(nnzb);
  s.u = alloc<double4>(nv);
  s.u_n = alloc<double4>(nv);
  s.vel = alloc<double4>(nv);
  s.uhat = alloc<double4>(nv);
  s.u_probe = alloc<double4>(nv);
  s.ge = alloc<double>((size_t)nt * GE_STRIDE);
  s.He = alloc<T>((size_t)nt * HE_STRIDE);
  s.dH = alloc<T>((size_t)nt * HE_STRIDE);
  s.g = alloc<double4>(nv);
  s.gmax = alloc<double>(nv);
  s.val = alloc<T>((size_t)9 * nnzb);
  s.proj_stamp = alloc<int>(nt);
  s.cproj_stamp = alloc<int>(nv);
  d_obs = alloc<ObstSet>(1);
  s.obs = d_obs;
  s.cround_stamp = alloc<int>(nv);
  s.dHc = alloc<T>((size_t)9 * nv);
  s.Hc = alloc<T>((size_t)9 * nv);
  s.round_stamp = alloc<int>(nt);
  s.sel_list = alloc<int>(nt);
  s.dx = alloc<V4>(nv);
  s.r = alloc<V4>(nv);
  s.z = alloc<V4>(nv);
  s.q = alloc<V4>(nv);
  s.d0 = alloc<V4>(nv);
  s.d1 = alloc<V4>(nv);
  s.Pinv = alloc<T>((size_t)9 * nv);
  s.vpart = alloc<double>((size_t)4 * n_vtiles);
  s.tpart = alloc<double>((size_t)4 * (n_vtiles + n_ttiles));
  s.ppart = alloc<double>((size_t)4 * n_ptiles);
  s.pword = alloc<unsigned long long>((size_t)8 * n_ptiles * pword_stride(n_ptiles));
  s.zrec = sizeof(T) == 4 ? alloc<T>((size_t)16 * nv) : nullptr;
  s.ctl = alloc<Ctl>(1);
  d_desc = alloc<SceneDev<T>>(1);
  d_ids = alloc<int>(1);
  d_bar = alloc<GridBar>(1);
  d_fixed_list = alloc<int>(nfixed);
  d_targets = alloc<double>((size_t)3 * nfixed);
  d_xyz = alloc<double>((size_t)3 * nv);
  const auto tt = make_tiles(0, nt, TILE), vt = make_tiles(0, nv, TILE), bt = make_tiles(0, nnzb, TILE),
             pt = make_tiles(0, nv, PCG_TILE), jt = make_tiles(0, nt, PROJ_CTA);
  std::vector<TileRef> et;
  for (int i = 0; i < n_ttiles + n_vtiles; ++i) et.push_back({0, i});
  d_ttiles = alloc<TileRef>(tt.size());
  d_vtiles = alloc<TileRef>(vt.size());
  d_btiles = alloc<TileRef>(bt.size());
  d_ptiles = alloc<TileRef>(pt.size());
  d_etiles = alloc<TileRef>(et.size());
  d_projtiles = alloc<TileRef>(jt.size());
  if (!d_tets || !d_tetc || !d_mass || !d_fixed || !d_con || !s.tgt || !d_X || !d_vt_ptr || !d_vt_src || !d_row_ptr ||
      !d_col || !d_blk_row || !d_blk_ptr || !d_blk_src || !d_blk_lane || !d_diag || !d_tet_blk || !s.blk_mark || !s.touched || !s.u || !s.u_n || !s.vel ||
      !s.uhat || !s.u_probe || !s.ge || !s.He || !s.dH || !s.g || !s.gmax || !s.val ||
      !s.proj_stamp || !s.round_stamp || !s.cproj_stamp || !d_obs || !s.cround_stamp || !s.dHc || !s.Hc || !s.sel_list || !s.dx || !s.r || !s.z || !s.q || !s.d0 ||
      !s.d1 || !s.Pinv || !s.vpart || !s.tpart || !s.ppart || !s.pword || (sizeof(T) == 4 && !s.zrec) || !s.ctl || !d_desc || !d_ids ||
      !d_bar || !d_fixed_list || !d_targets || !d_xyz || !d_ttiles || !d_vtiles || !d_btiles ||
      !d_ptiles || !d_etiles || !d_projtiles) {
    set_error("cudaMalloc failed (scene needs more device memory than is free)");
    return PPN_ERR_OOM;
  }
  std::vector<double4> X4(nv);
  for (int v = 0; v < nv; ++v) X4[v] = make_double4(rest[3 * v], rest[3 * v + 1], rest[3 * v + 2], 0.0);
  std::vector<int> rp32(h_row_ptr.begin(), h_row_ptr.end());
  std::vector<double> tg((size_t)3 * nfixed);
  for (int f = 0; f < nfixed; ++f)
    for (int k = 0; k < 3; ++k) tg[3 * f + k] = rest[3 * fixed_list[f] + k];
  auto up = [&](void* dst, const void* src, size_t n) { return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice); };
  PPN_CU(up(d_tets, h_tets.data(), sizeof(int4) * nt));
  PPN_CU(up(d_tetc, h_tetc.data(), sizeof(T) * h_tetc.size()));
  PPN_CU(up(d_mass, mass.data(), sizeof(double) * nv));
  // elimination: the Dirichlet vertices are fixed; penalty: they are free and constrained
  const std::vector<uint8_t> none(nv, 0);
  PPN_CU(up(d_fixed, penalty ? none.data() : fixed_flag.data(), nv));
  PPN_CU(up(d_con, penalty ? fixed_flag.data() : none.data(), nv));
  PPN_CU(cudaMemset(s.tgt, 0, sizeof(double4) * nv));  // targets start at the rest positions
  PPN_CU(up(d_X, X4.data(), sizeof(double4) * nv));
  PPN_CU(up(d_vt_ptr, vt_ptr.data(), sizeof(int) * (nv + 1)));
  PPN_CU(up(d_vt_src, vt_src.data(), sizeof(int) * vt_src.size()));
  PPN_CU(up(d_row_ptr, rp32.data(), sizeof(int) * (nv + 1)));
  PPN_CU(up(d_col, h_col.data(), sizeof(int) * nnzb));
  PPN_CU(up(d_blk_row, blk_row.data(), sizeof(int) * nnzb));
  PPN_CU(up(d_blk_ptr, blk_ptr.data(), sizeof(int) * (nnzb + 1)));
  PPN_CU(up(d_blk_src, blk_src.data(), sizeof(int) * blk_src.size()));
  {
    std::vector<unsigned char> lane((size_t)16 * nt);
    for (int k = 0; k < nnzb; ++k)
      for (int cc = blk_ptr[k]; cc < blk_ptr[k + 1]; ++cc) lane[cc] = (unsigned char)(k & 31);
    PPN_CU(up(d_blk_lane, lane.data(), lane.size()));
  }
  PPN_CU(up(d_diag, diag_idx.data(), sizeof(int) * nv));
  PPN_CU(up(d_tet_blk, blk_of.data(), sizeof(int) * blk_of.size()));
  PPN_CU(cudaMemset(s.blk_mark, 0xff, sizeof(int) * nnzb));
  if (nfixed) {
    PPN_CU(up(d_fixed_list, fixed_list.data(), sizeof(int) * nfixed));
    PPN_CU(up(d_targets, tg.data(), sizeof(double) * tg.size()));
  }
  PPN_CU(up(d_ttiles, tt.data(), sizeof(TileRef) * tt.size()));
  PPN_CU(up(d_vtiles, vt.data(), sizeof(TileRef) * vt.size()));
  PPN_CU(up(d_btiles, bt.data(), sizeof(TileRef) * bt.size()));
  PPN_CU(up(d_ptiles, pt.data(), sizeof(TileRef) * pt.size()));
  PPN_CU(up(d_etiles, et.data(), sizeof(TileRef) * et.size()));
  PPN_CU(up(d_projtiles, jt.data(), sizeof(TileRef) * jt.size()));
  const int zero = 0;
  PPN_CU(up(d_ids, &zero, sizeof(int)));
  PPN_CU(cudaMemset(s.u, 0, sizeof(double4) * nv));
  PPN_CU(cudaMemset(s.vel, 0, sizeof(double4) * nv));
  PPN_CU(cudaMemset(s.dx, 0, sizeof(V4) * nv));
  PPN_CU(cudaMemset(s.proj_stamp, 0xff, sizeof(int) * nt));
  PPN_CU(cudaMemset(s.cproj_stamp, 0xff, sizeof(int) * nv));
  PPN_CU(cudaMemset(d_obs, 0, sizeof(ObstSet)));
  PPN_CU(cudaMemset(s.cround_stamp, 0xff, sizeof(int) * nv));
  PPN_CU(cudaMemset(s.round_stamp, 0xff, sizeof(int) * nt));
  PPN_CU(cudaMemset(s.ctl, 0, sizeof(Ctl)));
  PPN_CU(cudaMemset(s.vpart, 0, sizeof(double) * 4 * n_vtiles));
  PPN_CU(cudaMemset(s.tpart, 0, sizeof(double) * 4 * (n_vtiles + n_ttiles)));
  PPN_CU(cudaMemset(s.ppart, 0, sizeof(double) * 4 * n_ptiles));
  s.tets = d_tets;
  s.tetc = d_tetc;
  s.mass = d_mass;
  s.fixed = d_fixed;
  s.X = d_X;
  s.vt_ptr = d_vt_ptr;
  s.vt_src = d_vt_src;
  s.row_ptr = d_row_ptr;
  s.col = d_col;
  s.blk_row = d_blk_row;
  s.blk_ptr = d_blk_ptr;
  s.blk_src = d_blk_src;
  s.blk_lane = d_blk_lane;
  s.diag_idx = d_diag;
  s.tet_blk = d_tet_blk;
  s.dt = dt;
  s.inv_dt2 = 1.0 / (dt * dt);
  for (int k = 0; k < 3; ++k) s.grav[k] = params.gravity[k];
  s.eps_delta = params.eps_delta;
  s.eig_eps = params.eig_eps;
  // the tie band of the selection: the resolution of r_e against delta in each precision
  s.tie_band = params.tie_band > 0.0 ? params.tie_band : (sizeof(T) == sizeof(double) ? 1e-12 : 1e-5);
  s.kappa = params.contact_kappa;
  s.dhat = params.contact_dhat;
  s.pen_k = params.dirichlet_penalty;
  s.con = d_con;
  s.proj_kind = params.projection;
  s.init_guess = params.init_guess;
  s.delta = std::numeric_limits<double>::infinity();
  s.pcg_tol2 = params.pcg_rel_tol * params.pcg_rel_tol;
  s.pcg_max_iter = params.pcg_max_iter > 0 ? params.pcg_max_iter : std::max(1000, 3 * nv);
  s.it_id = 0;
  s.round_id = 0;
  s.active = 1;
  d = s;
  PPN_CU(up(d_desc, &s, sizeof(SceneDev<T>)));  // for single-scene launches outside a step
  PPN_CU(cudaMallocHost(&h_ctl, sizeof(Ctl)));
  int dev = 0;
  PPN_CU(cudaGetDevice(&dev));
  pcg_group = 4;
  if (const char* g = std::getenv("PPN_PCG_GROUP")) pcg_group = (std::atoi(g) == 8) ? 8 : 4;
  pcg_grid = pcg_max_grid(pcg_group, dev);
  if (pcg_grid <= 0) {
    set_error("PCG kernel cannot be made co-resident on this device");
    return PPN_ERR_CUDA;
  }
  return PPN_OK;
}

// ------------------------------------------------------------------ groups
// A group is a set of scenes that step together; a single scene is a group
// of one.  The group owns the device copies of its members' descriptors, the
// concatenated tile tables, one contiguous control-block array and the PCG
// grid barrier.
template <typename T>
struct GroupCache {
  std::map<std::vector<const void*>, std::unique_ptr<Group<T>>> groups;
};

template <typename T>
static GroupCache<T>& group_cache() {
  static GroupCache<T> c;
  return c;
}
static std::mutex g_cache_mu;

template <typename T>
static Group<T>* get_group(const std::vector<SceneImpl<T>*>& members, ppn_status* rc) {
  std::vector<const void*> key(members.begin(), members.end());
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto& c = group_cache<T>().groups;
  auto it = c.find(key);
  if (it != c.end()) {
    // stream may have changed since the group was built
    it->second->st = members[0]->stream;
    *rc = PPN_OK;
    return it->second.get();
  }
  auto g = std::make_unique<Group<T>>();
  *rc = g->build(members);
  if (*rc) return nullptr;
  Group<T>* p = g.get();
  c.emplace(key, std::move(g));
  return p;
}

template <typename T>
static void drop_groups_of(const SceneImpl<T>* s) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto& c = group_cache<T>().groups;
  for (auto it = c.begin(); it != c.end();) {
    if (std::find(it->first.begin(), it->first.end(), (const void*)s) != it->first.end())
      it = c.erase(it);
    else
      ++it;
  }
}

template <typename T>
static ppn_status step_scenes(const std::vector<SceneImpl<T>*>& members, const int* modes, double tol,
                              std::vector<ppn_step_stats>* out) {
  ppn_status rc;
  Group<T>* G = get_group<T>(members, &rc);
  if (!G) return rc;
  // sync descriptor scalars from the scenes (ids advance across groups)
  for (size_t i = 0; i < members.size(); ++i) {
    G->h_desc[i].it_id = members[i]->d.it_id;
    G->h_desc[i].round_id = members[i]->d.round_id;
    G->h_desc[i].delta = std::numeric_limits<double>::infinity();
  }
  Driver<T> D(*G);
  rc = D.step(modes, tol);
  if (out) {
    out->resize(members.size());
    for (size_t i = 0; i < members.size(); ++i) (*out)[i] = D.H[i].tot;
  }
  if (rc) return rc;
  for (size_t i = 0; i < members.size(); ++i)
    if (D.H[i].status != PPN_OK) return (ppn_status)D.H[i].status;
  return PPN_OK;
}

// upload host positions as a displacement into `dst` (u = x - X)
template <typename T>
static ppn_status upload_positions(SceneImpl<T>& s, const double* x, double4* dst) {
  std::vector<double4> u(s.nv);
  for (int v = 0; v < s.nv; ++v)
    u[v] = make_double4(x[3 * v] - s.rest[3 * v], x[3 * v + 1] - s.rest[3 * v + 1], x[3 * v + 2] - s.rest[3 * v + 2], 0.0);
  PPN_CU(cudaMemcpyAsync(dst, u.data(), sizeof(double4) * s.nv, cudaMemcpyHostToDevice, s.stream));
  PPN_CU(cudaStreamSynchronize(s.stream));
  return PPN_OK;
}

// ------------------------------------------------------------------ probes
template <typename T>
struct Probe {
  SceneImpl<T>& s;
  Group<T>* G = nullptr;
  explicit Probe(SceneImpl<T>& s_) : s(s_) {}
  ppn_status begin() {
    ppn_status rc;
    G = get_group<T>({&s}, &rc);
    if (!G) return rc;
    G->h_desc[0].active = 1;
    G->h_desc[0].it_id = ++s.it_counter;
    G->h_desc[0].round_id = ++s.round_counter;
    s.d.it_id = G->h_desc[0].it_id;
    s.d.round_id = G->h_desc[0].round_id;
    G->h_desc[0].gamma = 0.0;
    return G->upload_desc();
  }
};

template <typename T>
static ppn_status probe_elements(SceneImpl<T>& s, const double* x, double* psi, double* ge, double* He) {
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  if ((rc = upload_positions(s, x, s.d.u_probe))) return rc;
  launch_element<T>(p.G->d_desc, p.G->d_ttiles, p.G->n_ttiles, 1, s.stream);
  PPN_CU(cudaGetLastError());
  PPN_CU(cudaStreamSynchronize(s.stream));
  if (ge) {
    PPN_CU(cudaMemcpy(ge, s.d.ge, sizeof(double) * (size_t)s.nt * GE_STRIDE, cudaMemcpyDeviceToHost));
  }
  if (He) {
    std::vector<T> h((size_t)s.nt * HE_STRIDE);
    PPN_CU(cudaMemcpy(h.data(), s.d.He, sizeof(T) * h.size(), cudaMemcpyDeviceToHost));
    for (int e = 0; e < s.nt; ++e)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
              const T v = a <= b ? h[(size_t)e * HE_STRIDE + 9 * tri4(a, b) + 3 * i + k]
                                 : h[(size_t)e * HE_STRIDE + 9 * tri4(b, a) + 3 * k + i];
              He[(size_t)144 * e + 12 * (3 * a + i) + 3 * b + k] = (double)v;
            }
  }
  if (psi) {
    double* d_psi = nullptr;
    PPN_CU(cudaMalloc(&d_psi, sizeof(double) * s.nt));
    p.G->h_desc[0].psi_out = d_psi;
    ppn_status rc2 = p.G->upload_desc();
    if (rc2 == PPN_OK) {
      launch_energy<T>(p.G->d_desc, p.G->d_etiles, p.G->n_etiles, 1, s.stream);
      cudaMemcpyAsync(psi, d_psi, sizeof(double) * s.nt, cudaMemcpyDeviceToHost, s.stream);
      cudaStreamSynchronize(s.stream);
    }
    p.G->h_desc[0].psi_out = nullptr;
    cudaFree(d_psi);
    if (rc2) return rc2;
    PPN_CU(cudaGetLastError());
  }
  return PPN_OK;
}

template <typename T>
static ppn_status probe_gradient(SceneImpl<T>& s, const double* x, const double* xhat, double* g,
                                 double* norms, double* energy) {
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  if ((rc = upload_positions(s, x, s.d.u_probe))) return rc;
  if ((rc = upload_positions(s, xhat, s.d.uhat))) return rc;
  launch_element<T>(p.G->d_desc, p.G->d_ttiles, p.G->n_ttiles, 1, s.stream);
  launch_gradient<T>(p.G->d_desc, p.G->d_vtiles, p.G->n_vtiles, 1, s.stream);
  if (energy) launch_energy<T>(p.G->d_desc, p.G->d_etiles, p.G->n_etiles, 1, s.stream);
  PPN_CU(cudaGetLastError());
  if ((rc = p.G->sync_ctl())) return rc;
  if (norms) {
    norms[0] = std::sqrt(p.G->h_ctl[0].grad[0]);
    norms[1] = p.G->h_ctl[0].grad[3];
  }
  if (energy) *energy = p.G->h_ctl[0].energy[0];
  if (g) {
    std::vector<double4> h(s.nv);
    PPN_CU(cudaMemcpy(h.data(), s.d.g, sizeof(double4) * s.nv, cudaMemcpyDeviceToHost));
    for (int v = 0; v < s.nv; ++v) {
      g[3 * v] = h[v].x;
      g[3 * v + 1] = h[v].y;
      g[3 * v + 2] = h[v].z;
    }
  }
  return PPN_OK;
}

template <typename T>
static ppn_status read_bsr(SceneImpl<T>& s, double* vals) {
  std::vector<T> h((size_t)9 * s.nnzb);
  PPN_CU(cudaMemcpy(h.data(), s.d.val, sizeof(T) * h.size(), cudaMemcpyDeviceToHost));
  for (int k = 0; k < s.nnzb; ++k)
    for (int c = 0; c < 9; ++c) vals[(size_t)9 * k + c] = (double)h[(size_t)c * s.nnzb + k];
  return PPN_OK;
}

// clamp the listed elements at the probe positions (fills dH, sets the count)
template <typename T>
static ppn_status probe_clamp_list(SceneImpl<T>& s, Probe<T>& p, const std::vector<int>& sel) {
  if (sel.empty()) return PPN_OK;
  PPN_CU(cudaMemcpy(s.d.sel_list, sel.data(), sizeof(int) * sel.size(), cudaMemcpyHostToDevice));
  const int n = (int)sel.size();
  PPN_CU(cudaMemcpy(&p.G->d_ctl[0].n_new, &n, sizeof(int), cudaMemcpyHostToDevice));
  const bool warp = project_warp_form(true);  // as a PPN selection round
  const int per = warp ? PROJW_TETS : PROJ_CTA;
  std::vector<TileRef> jt;
  for (int t = 0; t < (n + per - 1) / per; ++t) jt.push_back({0, t});
  ppn_status rc = p.G->upload(p.G->d_projtiles, jt.data(), sizeof(TileRef) * jt.size());
  if (rc) return rc;
  launch_project<T>(p.G->d_desc, p.G->d_projtiles, (int)jt.size(), 1, s.stream, warp);
  PPN_CU(cudaGetLastError());
  PPN_CU(cudaStreamSynchronize(s.stream));
  return PPN_OK;
}

template <typename T>
static ppn_status probe_assemble(SceneImpl<T>& s, const double* x, const uint8_t* proj, double* vals) {
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  if ((rc = upload_positions(s, x, s.d.u_probe))) return rc;
  launch_element<T>(p.G->d_desc, p.G->d_ttiles, p.G->n_ttiles, 1, s.stream);
  PPN_CU(cudaGetLastError());
  std::vector<int> stamp(s.nt, -1), sel;
  if (proj)
    for (int e = 0; e < s.nt; ++e)
      if (proj[e]) {
        stamp[e] = p.G->h_desc[0].it_id;
        sel.push_back(e);
      }
  PPN_CU(cudaMemcpyAsync(s.d.proj_stamp, stamp.data(), sizeof(int) * s.nt, cudaMemcpyHostToDevice, s.stream));
  if ((rc = probe_clamp_list(s, p, sel))) return rc;
  // the contact Hessians come from the gradient pass at the same positions
  if (s.n_obst > 0) launch_gradient<T>(p.G->d_desc, p.G->d_vtiles, p.G->n_vtiles, 1, s.stream);
  launch_assemble<T>(p.G->d_desc, p.G->d_btiles, p.G->n_btiles, p.G->d_vtiles, p.G->n_vtiles, s.stream, 1);
  PPN_CU(cudaGetLastError());
  PPN_CU(cudaStreamSynchronize(s.stream));
  return read_bsr(s, vals);
}

template <typename T>
static ppn_status probe_select(SceneImpl<T>& s, const double* g, double delta, const uint8_t* already,
                               uint8_t* out_new, int64_t* n_new, int64_t* n_ties) {
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  std::vector<double4> g4(s.nv);
  for (int v = 0; v < s.nv; ++v) g4[v] = make_double4(g[3 * v], g[3 * v + 1], g[3 * v + 2], 0.0);
  PPN_CU(cudaMemcpy(s.d.g, g4.data(), sizeof(double4) * s.nv, cudaMemcpyHostToDevice));
  std::vector<int> stamp(s.nt, -1);
  if (already)
    for (int e = 0; e < s.nt; ++e)
      if (already[e]) stamp[e] = p.G->h_desc[0].it_id;
  PPN_CU(cudaMemcpy(s.d.proj_stamp, stamp.data(), sizeof(int) * s.nt, cudaMemcpyHostToDevice));
  p.G->h_desc[0].delta = delta;
  if ((rc = p.G->upload_desc())) return rc;
  PPN_CU(cudaMemsetAsync(&p.G->d_ctl[0].n_new, 0, 3 * sizeof(int), s.stream));  // n_new, n_new_c, n_ties
  launch_gmax<T>(p.G->d_desc, p.G->d_vtiles, p.G->n_vtiles, s.stream);
  launch_select<T>(p.G->d_desc, p.G->d_ttiles, p.G->n_ttiles, s.stream);
  PPN_CU(cudaGetLastError());
  if ((rc = p.G->sync_ctl())) return rc;
  const int nn = p.G->h_ctl[0].n_new;
  std::vector<int> list(nn);
  if (nn) PPN_CU(cudaMemcpy(list.data(), s.d.sel_list, sizeof(int) * nn, cudaMemcpyDeviceToHost));
  if (out_new) {
    std::memset(out_new, 0, s.nt);
    for (int e : list) out_new[e] = 1;
  }
  if (n_new) *n_new = nn;
  if (n_ties) *n_ties = p.G->h_ctl[0].n_ties;
  return PPN_OK;
}

template <typename T>
static ppn_status probe_project(SceneImpl<T>& s, const double* x, const int32_t* sel, int64_t n_sel,
                                double* dH) {
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  for (int64_t i = 0; i < n_sel; ++i)
    if (sel[i] < 0 || sel[i] >= s.nt) {
      set_error("element index out of range");
      return PPN_ERR_INVALID_ARG;
    }
  if ((rc = upload_positions(s, x, s.d.u_probe))) return rc;
  std::vector<int> list(sel, sel + n_sel);
  // unique elements only (each owns one dH record)
  std::vector<int> uniq(list);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  if ((rc = probe_clamp_list(s, p, uniq))) return rc;
  std::vector<T> rec(HE_STRIDE);
  for (int64_t i = 0; i < n_sel; ++i) {
    PPN_CU(cudaMemcpy(rec.data(), s.d.dH + (size_t)list[i] * HE_STRIDE, sizeof(T) * HE_STRIDE,
                      cudaMemcpyDeviceToHost));
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            const T v = a <= b ? rec[9 * tri4(a, b) + 3 * r + c] : rec[9 * tri4(b, a) + 3 * c + r];
            dH[(size_t)144 * i + 12 * (3 * a + r) + 3 * b + c] = (double)v;
          }
  }
  return PPN_OK;
}

template <typename T>
static ppn_status probe_pcg(SceneImpl<T>& s, const double* vals, const double* b, double rel_tol,
                            int max_iter, double* x, int* info) {
  using V4 = vec4_t<T>;
  Probe<T> p(s);
  ppn_status rc = p.begin();
  if (rc) return rc;
  std::vector<T> h((size_t)9 * s.nnzb);
  for (int k = 0; k < s.nnzb; ++k)
    for (int c = 0; c < 9; ++c) h[(size_t)c * s.nnzb + k] = (T)vals[(size_t)9 * k + c];
  PPN_CU(cudaMemcpy(s.d.val, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  std::vector<V4> r(s.nv);
  for (int v = 0; v < s.nv; ++v) {
    r[v].x = (T)b[3 * v];
    r[v].y = (T)b[3 * v + 1];
    r[v].z = (T)b[3 * v + 2];
    r[v].w = (T)0;
  }
  PPN_CU(cudaMemcpy(s.d.r, r.data(), sizeof(V4) * s.nv, cudaMemcpyHostToDevice));
  p.G->h_desc[0].pcg_tol2 = rel_tol * rel_tol;
  p.G->h_desc[0].pcg_max_iter = max_iter > 0 ? max_iter : s.d.pcg_max_iter;
  Driver<T> D(*p.G);
  rc = D.solve(std::vector<char>{1}, 0);
  p.G->h_desc[0].pcg_tol2 = s.d.pcg_tol2;
  p.G->h_desc[0].pcg_max_iter = s.d.pcg_max_iter;
  if (rc) return rc;
  if ((rc = p.G->sync_ctl())) return rc;
  if ((rc = D.check_errors(std::vector<char>{1}))) return rc;
  const Ctl& c = p.G->h_ctl[0];
  if (info) {
    info[0] = c.pcg_iters;
    info[1] = c.pcg_ind;
    info[2] = c.pcg_precond_fail;
    info[3] = c.pcg_hit_max;
  }
  std::vector<V4> xo(s.nv);
  PPN_CU(cudaMemcpy(xo.data(), s.d.dx, sizeof(V4) * s.nv, cudaMemcpyDeviceToHost));
  for (int v = 0; v < s.nv; ++v) {
    x[3 * v] = (double)xo[v].x;
    x[3 * v + 1] = (double)xo[v].y;
    x[3 * v + 2] = (double)xo[v].z;
  }
  return PPN_OK;
}

}  // namespace ppn

// ====================================================================== C ABI
using namespace ppn;

template <typename F>
static ppn_status dispatch(ppn_scene* s, F&& f) {
  if (!s) {
    set_error("null scene");
    return PPN_ERR_INVALID_ARG;
  }
  if (s->f) return f(*s->f);
  return f(*s->d);
}
template <typename F>
static ppn_status dispatch_c(const ppn_scene* s, F&& f) {
  return dispatch(const_cast<ppn_scene*>(s), f);
}

// the allocator ppn_set_allocator installed (cudaMalloc when none)
namespace ppn {
namespace {
std::mutex g_alloc_mu;
DevAllocator g_alloc;
}  // namespace
DevAllocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}
}  // namespace ppn

extern "C" {

ppn_params ppn_default_params(void) {
  ppn_params p;
  p.alpha = 0.5;
  p.beta = 2.0;
  p.eps_delta = 1e-12;
  p.eig_eps = 1e-8;
  p.pdn_countdown = 4;
  p.projection = PPN_PROJ_CLAMP;
  p.grad_floor = 1e-12;
  p.ls_slack = 1e-12;
  p.contact_kappa = 1e3;
  p.contact_dhat = 1e-3;
  p.ccd_safety = 0.9;
  p.dirichlet_penalty = 0.0;
  p.tie_band = 0.0;
  p.pcg_rel_tol = 1e-4;
  p.armijo_c = 1e-4;
  p.gravity[0] = 0.0;
  p.gravity[1] = -9.81;
  p.gravity[2] = 0.0;
  p.pcg_max_iter = 0;
  p.newton_max_iter = 100;
  p.ls_max_halvings = 30;
  p.precision = PPN_PREC_MIXED;
  p.tol_kind = 0;
  p.init_guess = 0;
  return p;
}

const char* ppn_status_string(ppn_status s) {
  switch (s) {
    case PPN_OK: return "ok";
    case PPN_ERR_INVALID_ARG: return "invalid argument";
    case PPN_ERR_OOM: return "out of device memory";
    case PPN_ERR_CUDA: return "CUDA error";
    case PPN_ERR_DEGENERATE_TET: return "degenerate tet";
    case PPN_ERR_LINESEARCH: return "line search failed";
    case PPN_ERR_NEWTON_MAXITER: return "Newton iteration cap reached";
    case PPN_ERR_PCG_MAXITER: return "PCG iteration cap reached";
    case PPN_ERR_NONFINITE: return "non-finite value";
    case PPN_ERR_TIMEOUT: return "device wait timed out";
    case PPN_ERR_ADMISSION: return "admission refused";
  }
  return "unknown status";
}

const char* ppn_last_error(void) { return g_last_error.c_str(); }

ppn_status ppn_create_scene(const double* rest_xyz, int64_t n_verts, const int32_t* tets, int64_t n_tets,
                            const ppn_material* mat, double dt, const int32_t* fixed, int64_t n_fixed,
                            const ppn_params* params, ppn_scene** out) {
  if (!out) {
    set_error("null output pointer");
    return PPN_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const ppn_params p = params ? *params : ppn_default_params();
  auto s = std::make_unique<ppn_scene>();
  s->precision = p.precision;
  ppn_status rc;
  if (p.precision == PPN_PREC_FP64) {
    s->d = std::make_unique<SceneImpl<double>>();
    rc = s->d->init(rest_xyz, n_verts, tets, n_tets, mat, dt, fixed, n_fixed, &p);
  } else if (p.precision == PPN_PREC_MIXED) {
    s->f = std::make_unique<SceneImpl<float>>();
    rc = s->f->init(rest_xyz, n_verts, tets, n_tets, mat, dt, fixed, n_fixed, &p);
  } else {
    set_error("unknown precision");
    return PPN_ERR_INVALID_ARG;
  }
  if (rc != PPN_OK) return rc;
  *out = s.release();
  return PPN_OK;
}

void ppn_destroy_scene(ppn_scene* s) {
  if (!s) return;
  if (s->f) drop_groups_of(s->f.get());
  if (s->d) drop_groups_of(s->d.get());
  delete s;
}

ppn_status ppn_scene_get_info(const ppn_scene* s, ppn_scene_info* out) {
  if (!out) return PPN_ERR_INVALID_ARG;
  return dispatch_c(s, [&](auto& x) {
    out->n_verts = x.nv;
    out->n_tets = x.nt;
    out->n_fixed = x.nfixed;
    out->nnzb = x.nnzb;
    out->n_map = x.nmap;
    out->device_bytes = (int64_t)x.dev_bytes;
    out->precision = s->precision;
    out->pcg_layout = x.last_pcg_layout;
    return PPN_OK;
  });
}

ppn_status ppn_set_allocator(ppn_device_alloc_fn alloc_fn, ppn_device_free_fn free_fn, void* ctx) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) {
    ppn::set_error("ppn_set_allocator: give both functions or neither");
    return PPN_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(ppn::g_alloc_mu);
  ppn::g_alloc = ppn::DevAllocator{alloc_fn, free_fn, alloc_fn ? ctx : nullptr};
  return PPN_OK;
}

ppn_status ppn_set_stream(ppn_scene* s, void* cuda_stream) {
  return dispatch(s, [&](auto& x) {
    cudaStreamSynchronize(x.stream);
    if (cuda_stream) {
      if (x.own_stream) cudaStreamDestroy(x.stream);
      x.own_stream = false;
      x.stream = (cudaStream_t)cuda_stream;
    } else if (!x.own_stream) {
      PPN_CU(cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking));
      x.own_stream = true;
    }
    return PPN_OK;
  });
}

ppn_status ppn_set_kinematic_targets(ppn_scene* s, const double* xyz) {
  return dispatch(s, [&](auto& x) {
    if (x.nfixed == 0) return PPN_OK;
    if (!xyz) {
      set_error("null targets");
      return PPN_ERR_INVALID_ARG;
    }
    PPN_CU(cudaMemcpyAsync(x.d_targets, xyz, sizeof(double) * 3 * x.nfixed, cudaMemcpyHostToDevice, x.stream));
    // a penalty's targets take effect at once (positions are set at the next step)
    if (x.params.dirichlet_penalty > 0.0)
      launch_apply_targets(x.d_desc, 0, x.d_fixed_list, x.d_targets, x.nfixed, 2, x.stream);
    PPN_CU(cudaGetLastError());
    PPN_CU(cudaStreamSynchronize(x.stream));
    x.ext_targets = nullptr;
    return PPN_OK;
  });
}

ppn_status ppn_set_obstacles(ppn_scene* s, const ppn_obstacle* obs, int n) {
  if (n < 0 || n > PPN_MAX_OBSTACLES || (n > 0 && !obs)) {
    set_error("obstacle count out of range");
    return PPN_ERR_INVALID_ARG;
  }
  ObstSet h{};
  h.n = n;
  for (int k = 0; k < n; ++k) {
    const ppn_obstacle& o = obs[k];
    const double na = std::sqrt(o.a[0] * o.a[0] + o.a[1] * o.a[1] + o.a[2] * o.a[2]);
    const bool dir = o.type == PPN_OBST_SPHERE_OUT || std::fabs(na - 1.0) < 1e-9;
    const bool rad = o.type == PPN_OBST_PLANE || o.r > 0.0;
    if (o.type < PPN_OBST_PLANE || o.type > PPN_OBST_SPHERE_OUT || !dir || !rad) {
      set_error("invalid obstacle " + std::to_string(k) + " (type, unit direction, radius)");
      return PPN_ERR_INVALID_ARG;
    }
    h.o[k].type = o.type;
    for (int c = 0; c < 3; ++c) {
      h.o[k].p[c] = o.p[c];
      h.o[k].a[c] = o.a[c];
    }
    h.o[k].r = o.r;
  }
  // Requested poses.  A plane of the same normal as before is moved toward the
  // bodies at the next step only as far as keeps that step's initial iterate
  // feasible (ccd_safety x the smallest vertex distance), the rest in later steps;
  // other obstacles, and a set of another size, kind or normal, apply at once.
  return dispatch(s, [&](auto& x) {
    bool same = x.obs_app.n == n;
    for (int k = 0; same && k < n; ++k)
      same = x.obs_app.o[k].type == h.o[k].type && x.obs_app.o[k].a[0] == h.o[k].a[0] &&
             x.obs_app.o[k].a[1] == h.o[k].a[1] && x.obs_app.o[k].a[2] == h.o[k].a[2];
    x.obs_req = h;
    if (!same) x.obs_app = h;
    for (int k = 0; k < n; ++k)
      if (h.o[k].type != PPN_OBST_PLANE) x.obs_app.o[k] = h.o[k];
    PPN_CU(cudaStreamSynchronize(x.stream));
    PPN_CU(cudaMemcpy(x.d_obs, &x.obs_app, sizeof(ObstSet), cudaMemcpyHostToDevice));
    x.n_obst = n;
    return PPN_OK;
  });
}

ppn_status ppn_set_kinematic_targets_device(ppn_scene* s, const double* xyz) {
  return dispatch(s, [&](auto& x) {
    x.ext_targets = xyz;
    return PPN_OK;
  });
}

ppn_status ppn_step(ppn_scene* s, ppn_mode mode, double tol, double* out_xyz, ppn_step_stats* out) {
  if (mode < PPN_MODE_NEWTON || mode > PPN_MODE_PDN || !(tol >= 0)) {
    set_error("invalid mode or tolerance");
    return PPN_ERR_INVALID_ARG;
  }
  return dispatch(s, [&](auto& x) {
    std::vector<ppn_step_stats> st;
    const int m = (int)mode;
    using SI = std::remove_reference_t<decltype(x)>;
    ppn_status rc = step_scenes(std::vector<SI*>{&x}, &m, tol, &st);
    if (out && !st.empty()) *out = st[0];
    if (rc != PPN_OK && rc != PPN_ERR_NEWTON_MAXITER && rc != PPN_ERR_LINESEARCH) return rc;
    if (out_xyz) {
      const ppn_status r2 = read_positions(x, out_xyz);
      if (r2) return r2;
    }
    return rc;
  });
}

ppn_status ppn_step_batch(ppn_scene* const* scenes, int n, const ppn_mode* modes, double tol,
                          ppn_step_stats* out) {
  if (!scenes || n <= 0 || !modes) {
    set_error("invalid batch");
    return PPN_ERR_INVALID_ARG;
  }
  const int prec = scenes[0] ? scenes[0]->precision : -1;
  for (int i = 0; i < n; ++i)
    if (!scenes[i] || scenes[i]->precision != prec) {
      set_error("batch scenes must be non-null and share the precision");
      return PPN_ERR_INVALID_ARG;
    }
  std::vector<int> m(modes, modes + n);
  for (int i = 0; i < n; ++i)
    if (m[i] < PPN_MODE_NEWTON || m[i] > PPN_MODE_PDN) {
      set_error("invalid mode in batch");
      return PPN_ERR_INVALID_ARG;
    }
  if (!(tol >= 0)) {
    set_error("invalid tolerance");
    return PPN_ERR_INVALID_ARG;
  }
  std::vector<ppn_step_stats> st;
  ppn_status rc;
  if (prec == PPN_PREC_FP64) {
    std::vector<SceneImpl<double>*> v;
    for (int i = 0; i < n; ++i) v.push_back(scenes[i]->d.get());
    rc = step_scenes(v, m.data(), tol, &st);
  } else {
    std::vector<SceneImpl<float>*> v;
    for (int i = 0; i < n; ++i) v.push_back(scenes[i]->f.get());
    rc = step_scenes(v, m.data(), tol, &st);
  }
  if (out)
    for (int i = 0; i < n && i < (int)st.size(); ++i) out[i] = st[i];
  return rc;
}

ppn_status ppn_get_iter_stats(const ppn_scene* s, ppn_iter_stats* buf, int cap, int* n_written) {
  return dispatch_c(s, [&](auto& x) {
    const int n = (int)x.iters.size();
    for (int i = 0; i < n && i < cap; ++i) buf[i] = x.iters[i];
    if (n_written) *n_written = n;
    return PPN_OK;
  });
}

ppn_status ppn_get_attempts(const ppn_scene* s, ppn_attempt* buf, int cap, int* n_written) {
  return dispatch_c(s, [&](auto& x) {
    const int n = (int)x.attempts.size();
    for (int i = 0; i < n && i < cap; ++i) buf[i] = x.attempts[i];
    if (n_written) *n_written = n;
    return PPN_OK;
  });
}

ppn_status ppn_get_pcg_tuning(ppn_pcg_tuning* buf, int cap, int* n_written) {
  if (cap < 0 || (cap > 0 && !buf)) {
    set_error("cap < 0, or a null buffer with cap > 0");
    return PPN_ERR_INVALID_ARG;
  }
  const auto recs = pcg_tuner().snapshot();
  int i = 0;
  for (const auto& kv : recs) {
    if (i < cap) {
      ppn_pcg_tuning& o = buf[i];
      o.tiles_per_cta = kv.first[0];
      o.blocks_per_row = kv.first[1];
      o.log2_matrix_mb = kv.first[2];
      const PcgTuner::Rec& r = kv.second;
      bool done = true;
      int best = -1;
      double bt = 0.0;
      for (int k = 0; k < PcgTuner::kChoices; ++k) {
        o.launches[k] = r.n[k];
        o.us_per_iter[k] = r.iters[k] > 0 ? 1e3 * r.ms[k] / (double)r.iters[k] : 0.0;
        if (!((r.allowed >> k) & 1u)) continue;
        if (r.n[k] < PcgTuner::kExplore) done = false;
        if (r.iters[k] > 0 && (best < 0 || o.us_per_iter[k] < bt)) {
          best = k;
          bt = o.us_per_iter[k];
        }
      }
      o.choice = done ? best : -1;
    }
    ++i;
  }
  if (n_written) *n_written = i;
  return PPN_OK;
}

ppn_status ppn_set_record_selection(ppn_scene* s, int on) {
  return dispatch(s, [&](auto& x) {
    x.record_sel = on != 0;
    x.attempt_sel.clear();
    x.iter_g.clear();
    return PPN_OK;
  });
}

ppn_status ppn_get_iteration_gradient(const ppn_scene* s, int newton_iter, double* g) {
  if (!g) return PPN_ERR_INVALID_ARG;
  return dispatch_c(s, [&](auto& x) {
    if (newton_iter < 0 || newton_iter >= (int)x.iter_g.size()) {
      set_error("no recorded gradient for Newton iteration " + std::to_string(newton_iter));
      return PPN_ERR_INVALID_ARG;
    }
    std::memcpy(g, x.iter_g[newton_iter].data(), sizeof(double) * x.iter_g[newton_iter].size());
    return PPN_OK;
  });
}

ppn_status ppn_get_attempt_selection(const ppn_scene* s, int idx, int32_t* buf, int64_t cap, int64_t* n) {
  if (cap < 0 || (cap > 0 && !buf)) {
    set_error("cap < 0, or a null buffer with cap > 0");
    return PPN_ERR_INVALID_ARG;
  }
  return dispatch_c(s, [&](auto& x) {
    if (idx < 0 || idx >= (int)x.attempt_sel.size()) {
      set_error("no recorded selection for attempt " + std::to_string(idx) +
                " (recording off during the step, or index out of range)");
      return PPN_ERR_INVALID_ARG;
    }
    const std::vector<int>& l = x.attempt_sel[idx];
    for (int64_t k = 0; k < (int64_t)l.size() && k < cap; ++k) buf[k] = l[k];
    if (n) *n = (int64_t)l.size();
    return PPN_OK;
  });
}

ppn_status ppn_get_state(const ppn_scene* s, double* xo, double* vo) {
  return dispatch_c(s, [&](auto& x) {
    if (xo) {
      ppn_status rc = read_positions(x, xo);
      if (rc) return rc;
    }
    if (vo) {
      using SI = std::remove_reference_t<decltype(x)>;
      using TT = typename std::conditional<std::is_same<SI, SceneImpl<float>>::value, float, double>::type;
      k_vel_out<TT><<<(x.nv + 255) / 256, 256, 0, x.stream>>>(x.d.vel, x.d_xyz, x.nv);
      PPN_CU(cudaGetLastError());
      PPN_CU(cudaMemcpyAsync(vo, x.d_xyz, sizeof(double) * 3 * x.nv, cudaMemcpyDeviceToHost, x.stream));
      PPN_CU(cudaStreamSynchronize(x.stream));
    }
    return PPN_OK;
  });
}

ppn_status ppn_set_state(ppn_scene* s, const double* xi, const double* vi) {
  return dispatch(s, [&](auto& x) {
    if (xi) {
      ppn_status rc = upload_positions(x, xi, x.d.u);
      if (rc) return rc;
    }
    if (vi) {
      std::vector<double4> w(x.nv);
      for (int v = 0; v < x.nv; ++v) w[v] = make_double4(vi[3 * v], vi[3 * v + 1], vi[3 * v + 2], 0.0);
      PPN_CU(cudaMemcpy(x.d.vel, w.data(), sizeof(double4) * x.nv, cudaMemcpyHostToDevice));
    }
    return PPN_OK;
  });
}

ppn_status ppn_get_displacement(const ppn_scene* s, double* uo, double* vo) {
  return dispatch_c(s, [&](auto& x) {
    std::vector<double4> h(x.nv);
    double* outs[2] = {uo, vo};
    double4* src[2] = {x.d.u, x.d.vel};
    PPN_CU(cudaStreamSynchronize(x.stream));
    for (int k = 0; k < 2; ++k) {
      if (!outs[k]) continue;
      PPN_CU(cudaMemcpy(h.data(), src[k], sizeof(double4) * x.nv, cudaMemcpyDeviceToHost));
      for (int v = 0; v < x.nv; ++v) {
        outs[k][3 * v] = h[v].x;
        outs[k][3 * v + 1] = h[v].y;
        outs[k][3 * v + 2] = h[v].z;
      }
    }
    return PPN_OK;
  });
}

ppn_status ppn_set_displacement(ppn_scene* s, const double* ui, const double* vi) {
  return dispatch(s, [&](auto& x) {
    std::vector<double4> h(x.nv);
    const double* ins[2] = {ui, vi};
    double4* dst[2] = {x.d.u, x.d.vel};
    PPN_CU(cudaStreamSynchronize(x.stream));
    for (int k = 0; k < 2; ++k) {
      if (!ins[k]) continue;
      for (int v = 0; v < x.nv; ++v) h[v] = make_double4(ins[k][3 * v], ins[k][3 * v + 1], ins[k][3 * v + 2], 0.0);
      PPN_CU(cudaMemcpy(dst[k], h.data(), sizeof(double4) * x.nv, cudaMemcpyHostToDevice));
    }
    return PPN_OK;
  });
}

ppn_status ppn_set_profiling(ppn_scene* s, int on) {
  return dispatch(s, [&](auto& x) {
    x.timer.on = on != 0;
    x.timer.reset();
    return PPN_OK;
  });
}

ppn_status ppn_get_kernel_times(const ppn_scene* s, ppn_kernel_time* buf, int cap, int* n_written) {
  return dispatch_c(s, [&](auto& x) {
    int n = 0;
    for (int f = 0; f < FAM_COUNT; ++f) {
      if (n < cap && buf) {
        std::memset(&buf[n], 0, sizeof(ppn_kernel_time));
        std::snprintf(buf[n].name, sizeof(buf[n].name), "%s", kFamilyNames[f]);
        buf[n].launches = x.timer.launches[f];
        buf[n].total_ms = x.timer.ms[f];
        buf[n].bytes = x.timer.bytes[f];
      }
      ++n;
    }
    if (n_written) *n_written = n;
    return PPN_OK;
  });
}

ppn_status ppn_probe_elements(ppn_scene* s, const double* x, double* psi_e, double* ge, double* He) {
  if (!x) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_elements(sc, x, psi_e, ge, He); });
}

ppn_status ppn_probe_halo_tables(int n_scenes, const int64_t* const* row_ptr, const int32_t* const* col,
                                 const int64_t* n_verts, int grid, int32_t* out, int64_t out_cap,
                                 int64_t* out_len, int32_t* max_halo) {
  if (!row_ptr || !col || !n_verts || !out_len || !max_halo || n_scenes < 1 || n_scenes > HALO_MAX_SCENES)
    return PPN_ERR_INVALID_ARG;
  std::vector<HaloPattern> pats;
  for (int k = 0; k < n_scenes; ++k) {
    if (!row_ptr[k] || !col[k] || n_verts[k] < 1 || n_verts[k] >= (1 << HALO_ROW_BITS)) return PPN_ERR_INVALID_ARG;
    pats.push_back({(int)n_verts[k], row_ptr[k], col[k]});
  }
  std::vector<int> tab;
  const int mh = build_halo_tables(pats, grid, tab);
  if (mh < 0) {
    set_error("ppn_probe_halo_tables: grid outside 1..tiles");
    return PPN_ERR_INVALID_ARG;
  }
  *out_len = (int64_t)tab.size();
  *max_halo = mh;
  if (!out || out_cap < (int64_t)tab.size()) {
    set_error("ppn_probe_halo_tables: output buffer too small");
    return PPN_ERR_INVALID_ARG;
  }
  std::memcpy(out, tab.data(), sizeof(int32_t) * tab.size());
  return PPN_OK;
}

ppn_status ppn_probe_pattern(const ppn_scene* s, int64_t* row_ptr, int32_t* col) {
  return dispatch_c(s, [&](auto& x) {
    if (row_ptr) std::memcpy(row_ptr, x.h_row_ptr.data(), sizeof(int64_t) * x.h_row_ptr.size());
    if (col) std::memcpy(col, x.h_col.data(), sizeof(int32_t) * x.h_col.size());
    return PPN_OK;
  });
}

ppn_status ppn_probe_gradient(ppn_scene* s, const double* x, const double* xhat, double* g,
                              double* norms, double* energy) {
  if (!x || !xhat) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_gradient(sc, x, xhat, g, norms, energy); });
}

ppn_status ppn_probe_assemble(ppn_scene* s, const double* x, const uint8_t* proj, double* vals) {
  if (!x || !vals) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_assemble(sc, x, proj, vals); });
}

ppn_status ppn_probe_select(ppn_scene* s, const double* g, double delta, const uint8_t* already,
                            uint8_t* out_new, int64_t* n_new, int64_t* n_ties) {
  if (!g) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_select(sc, g, delta, already, out_new, n_new, n_ties); });
}

ppn_status ppn_probe_tets(const ppn_scene* s, int32_t* tets) {
  if (!tets) return PPN_ERR_INVALID_ARG;
  return dispatch_c(s, [&](auto& x) {
    PPN_CU(cudaMemcpy(tets, x.d.tets, sizeof(int4) * (size_t)x.nt, cudaMemcpyDeviceToHost));
    return PPN_OK;
  });
}

ppn_status ppn_probe_project(ppn_scene* s, const double* x, const int32_t* sel, int64_t n_sel,
                             double* dH) {
  if (!x || (n_sel > 0 && (!sel || !dH)) || n_sel < 0) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_project(sc, x, sel, n_sel, dH); });
}

ppn_status ppn_probe_bounded_wait(int n_words, int spin_limit, int preset) {
  if (n_words < 1 || n_words > 4096 || spin_limit < 1 || spin_limit > (1 << 20)) {
    set_error("n_words in [1, 4096], spin_limit in [1, 2^20]");
    return PPN_ERR_INVALID_ARG;
  }
  unsigned long long* w = nullptr;
  int* out = nullptr;
  PPN_CU(cudaMalloc(&w, sizeof(unsigned long long) * n_words));
  if (cudaMalloc(&out, sizeof(int)) != cudaSuccess) {
    cudaFree(w);
    set_error("cudaMalloc failed");
    return PPN_ERR_OOM;
  }
  const unsigned long long stamp = 1;
  std::vector<unsigned long long> h(n_words, preset ? stamp : 0ull);
  int timed_out = -1;
  cudaError_t e = cudaMemcpy(w, h.data(), sizeof(unsigned long long) * n_words, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_wait_probe(w, n_words, stamp, (unsigned)spin_limit, out, 0);
  if (e == cudaSuccess) e = cudaMemcpy(&timed_out, out, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(w);
  cudaFree(out);
  if (e != cudaSuccess) {
    set_error(std::string("bounded-wait probe: ") + cudaGetErrorString(e));
    return PPN_ERR_CUDA;
  }
  if (timed_out) {
    set_error("bounded-wait probe: the wait ran out");
    return PPN_ERR_TIMEOUT;
  }
  return PPN_OK;
}

ppn_status ppn_probe_pcg(ppn_scene* s, const double* vals, const double* b, double rel_tol,
                         int max_iter, double* x, int* info) {
  if (!vals || !b || !x) return PPN_ERR_INVALID_ARG;
  return dispatch(s, [&](auto& sc) { return probe_pcg(sc, vals, b, rel_tol, max_iter, x, info); });
}

}  // extern "C"
