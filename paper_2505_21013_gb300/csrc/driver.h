// Scene groups and the lockstep Newton / PN / PPN / PDN driver.
//
// A Group holds the device tables of a set of scenes that step together: one
// descriptor per scene, tile tables for every kernel family, control blocks.
// The Driver runs Newton iterations over a group: every phase is one launch
// over the scenes still taking part in it, and every host decision is taken
// per scene after one device->host copy of all scenes' control blocks.  A time
// step is begin() for the scenes that start it, tick() (one Newton iteration
// of every running scene) until they stop, and finish().  Scenes may join a
// group at an iteration boundary, which is how the serving loop batches
// requests continuously.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "halo.h"
#include "scene.h"

namespace ppn {

#define PPN_CU(call)                                                                      \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) {                                                              \
      set_error(std::string(#call) + ": " + cudaGetErrorString(_e));                      \
      return _e == cudaErrorMemoryAllocation ? PPN_ERR_OOM : PPN_ERR_CUDA;                \
    }                                                                                     \
  } while (0)

// Online choice of the launch configuration of the single-reduction FP32 PCG among
// configurations that give bitwise-identical results: the streamed layouts (vectors in
// shared memory with the blocks streamed, or everything in global memory) and the L2
// priority of the streamed blocks (evict-first, which keeps the vectors resident while a
// matrix larger than L2 streams past, or normal, which lets a smaller matrix stay
// resident across iterations).  A choice is layout (0 streamed, 1 global) + 2 x priority
// (0 evict-first, 1 normal).  Per shape class (CTA tiles, blocks per row, log2 of the
// launch's matrix in MB) the first launches try every allowed choice kExplore times,
// each timed by CUDA events on the launching stream; later launches take the choice
// with the smallest time per CG iteration.  Shared by all groups of the process.
struct PcgTuner {
  static constexpr int kExplore = 2, kChoices = 4;
  using Key = std::array<int, 3>;
  struct Rec {
    double ms[kChoices] = {0.0, 0.0, 0.0, 0.0};
    long long iters[kChoices] = {0, 0, 0, 0};
    int n[kChoices] = {0, 0, 0, 0};
    unsigned allowed = 0;
  };
  std::mutex mu;
  std::map<Key, Rec> recs;
  int choose(const Key& key, unsigned allowed) {
    std::lock_guard<std::mutex> lk(mu);
    Rec& r = recs[key];
    r.allowed = allowed;
    int pick = -1;
    for (int k = 0; k < kChoices; ++k)  // explore: the least-tried allowed choice
      if ((allowed >> k) & 1u && r.n[k] < kExplore && (pick < 0 || r.n[k] < r.n[pick])) pick = k;
    if (pick >= 0) return pick;
    double best = 0.0;
    for (int k = 0; k < kChoices; ++k) {
      if (!((allowed >> k) & 1u)) continue;
      const double t = r.ms[k] / (double)std::max(1ll, r.iters[k]);
      if (pick < 0 || t < best) {
        pick = k;
        best = t;
      }
    }
    return pick;
  }
  void report(const Key& key, int k, double ms, long long iters) {
    if (iters <= 0 || !(ms > 0.0)) return;
    std::lock_guard<std::mutex> lk(mu);
    Rec& r = recs[key];
    r.ms[k] += ms;
    r.iters[k] += iters;
    r.n[k] += 1;
  }
  // the records, for ppn_get_pcg_tuning
  std::vector<std::pair<Key, Rec>> snapshot() {
    std::lock_guard<std::mutex> lk(mu);
    return std::vector<std::pair<Key, Rec>>(recs.begin(), recs.end());
  }
};
inline PcgTuner& pcg_tuner() {
  static PcgTuner t;
  return t;
}

template <typename T>
struct Group {
  std::vector<SceneImpl<T>*> S;
  std::vector<SceneDev<T>> h_desc;
  SceneDev<T>* d_desc = nullptr;
  Ctl* d_ctl = nullptr;
  Ctl* h_ctl = nullptr;
  GridBar* h_bar = nullptr;
  TileRef *d_ttiles = nullptr, *d_vtiles = nullptr, *d_btiles = nullptr, *d_ptiles = nullptr,
          *d_etiles = nullptr, *d_projtiles = nullptr;
  int n_ttiles = 0, n_vtiles = 0, n_btiles = 0, n_ptiles = 0, n_etiles = 0;
  int* d_ids = nullptr;
  TileRef* d_pcgtiles = nullptr;
  TileRef* d_touchtiles = nullptr;  // (selected element, corner pair) tiles of the touched-block update
  unsigned pcg_launch_seq = 0;
  std::vector<int> pcg_ids;  // slots of the tile table currently on the device
  int pcg_ntiles = 0;
  size_t pcg_smem_bytes = 0;  // > 0: resident PCG layout chosen for that table
  int pcg_smem_blocks = 0, pcg_smem_grid = 0;
  bool pcg_sr = false;          // the single-reduction FP32 kernel was chosen for that table
  int pcg_sr_mode = 0;          // its layout (SR_RES, SR_STREAM, SR_GLOBAL)
  // layout chosen per launch by the tuner (SR_STREAM and SR_GLOBAL both fit)
  bool pcg_tune = false;
  PcgTuner::Key tune_key{0, 0, 0};
  unsigned tune_allowed = 0;      // allowed tuner choices for that table
  size_t tune_bytes[2] = {0, 0};  // dynamic shared memory of SR_STREAM, SR_GLOBAL
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  bool tune_pending = false;      // a timed launch awaits its sync
  int tune_choice = 0;
  std::vector<int> tune_slots;
  unsigned long long* d_flags = nullptr;  // its per-CTA publication flags
  // SR_HALO tables of that tile table (PcgLaunch): offsets, local columns, halo rows
  int* d_halo = nullptr;
  size_t cap_halo = 0;
  const int *halo_off = nullptr, *halo_col = nullptr, *halo_ref = nullptr;
  int halo_cap = 0;
  GridBar* d_bar = nullptr;
  cudaStream_t st = nullptr;
  Staging staging;
  KernelTimer* timer = nullptr;
  int pcg_grid = 0, pcg_group = 8;
  DevAllocator dalloc = current_allocator();
  std::vector<void*> allocs;
  // capacities of the device tables (a group can be rebuilt for new members)
  size_t cap_n = 0, cap_tt = 0, cap_vt = 0, cap_bt = 0, cap_pt = 0, cap_et = 0, cap_proj = 0;
  ~Group() {
    release();
    for (cudaEvent_t& e : tune_ev)
      if (e) cudaEventDestroy(e);
  }
  void release() {
    if (st) cudaStreamSynchronize(st);
    tune_pending = false;
    for (void* p : allocs) dev_free(dalloc, p);
    allocs.clear();
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_bar) cudaFreeHost(h_bar);
    h_ctl = nullptr;
    h_bar = nullptr;
    d_halo = nullptr;
    cap_halo = 0;
    cap_n = cap_tt = cap_vt = cap_bt = cap_pt = cap_et = cap_proj = 0;
  }
  template <typename X>
  X* alloc(size_t n) {
    void* p = dev_alloc(dalloc, std::max<size_t>(1, n) * sizeof(X));
    if (!p) return nullptr;
    allocs.push_back(p);
    return reinterpret_cast<X*>(p);
  }
  // (Re)build the group's tables for `members`.  Device tables are reused when
  // they are large enough and regrown (with headroom) otherwise.
  ppn_status build(const std::vector<SceneImpl<T>*>& members) {
    if (st) cudaStreamSynchronize(st);
    S = members;
    const int n = (int)S.size();
    st = S[0]->stream;
    timer = &S[0]->timer;
    pcg_grid = S[0]->pcg_grid;
    pcg_group = S[0]->pcg_group;
    h_desc.resize(n);
    std::vector<TileRef> tt, vt, bt, pt, et;
    size_t projcap = 0;
    for (int i = 0; i < n; ++i) {
      const SceneImpl<T>& s = *S[i];
      for (int t = 0; t < s.n_ttiles; ++t) tt.push_back({i, t});
      for (int t = 0; t < s.n_vtiles; ++t) vt.push_back({i, t});
      for (int t = 0; t < s.n_btiles; ++t) bt.push_back({i, t});
      for (int t = 0; t < s.n_ptiles; ++t) pt.push_back({i, t});
      for (int t = 0; t < s.n_ttiles + s.n_vtiles; ++t) et.push_back({i, t});
      projcap += (s.nt + PROJW_TETS - 1) / PROJW_TETS;  // (the warp form's tiles are the smaller)
    }
    n_ttiles = (int)tt.size();
    n_vtiles = (int)vt.size();
    n_btiles = (int)bt.size();
    n_ptiles = (int)pt.size();
    n_etiles = (int)et.size();
    if (n > (int)cap_n || tt.size() > cap_tt || vt.size() > cap_vt || bt.size() > cap_bt || pt.size() > cap_pt ||
        et.size() > cap_et || projcap > cap_proj) {
      const bool grow = !allocs.empty();
      release();
      auto room = [&](size_t x) { return grow ? x + x / 2 : x; };
      cap_n = room(n);
      cap_tt = room(tt.size());
      cap_vt = room(vt.size());
      cap_bt = room(bt.size());
      cap_pt = room(pt.size());
      cap_et = room(et.size());
      cap_proj = room(projcap);
      d_desc = alloc<SceneDev<T>>(cap_n);
      d_ctl = alloc<Ctl>(cap_n);
      d_ttiles = alloc<TileRef>(cap_tt);
      d_vtiles = alloc<TileRef>(cap_vt);
      d_btiles = alloc<TileRef>(cap_bt);
      d_ptiles = alloc<TileRef>(cap_pt);
      d_etiles = alloc<TileRef>(cap_et);
      d_projtiles = alloc<TileRef>(cap_proj);
      d_ids = alloc<int>(cap_n);
      d_pcgtiles = alloc<TileRef>(cap_pt);
      d_touchtiles = alloc<TileRef>(cap_bt);
      d_flags = alloc<unsigned long long>(XCH_MAX_CTAS_HOST);
      d_bar = alloc<GridBar>(1);
      if (!d_desc || !d_ctl || !d_ttiles || !d_vtiles || !d_btiles || !d_ptiles || !d_etiles ||
          !d_projtiles || !d_ids || !d_bar || !d_pcgtiles || !d_touchtiles) {
        set_error("cudaMalloc failed for a scene group");
        return PPN_ERR_OOM;
      }
      PPN_CU(cudaMallocHost(&h_ctl, sizeof(Ctl) * cap_n));
      PPN_CU(cudaMallocHost(&h_bar, sizeof(GridBar)));
    }
    pcg_ids.clear();
    pcg_ntiles = 0;
    pcg_smem_bytes = 0;
    pcg_sr = false;
    std::memset(h_bar, 0, sizeof(GridBar));
    PPN_CU(cudaMemset(d_bar, 0, sizeof(GridBar)));
    PPN_CU(cudaMemcpy(d_ttiles, tt.data(), sizeof(TileRef) * tt.size(), cudaMemcpyHostToDevice));
    PPN_CU(cudaMemcpy(d_vtiles, vt.data(), sizeof(TileRef) * vt.size(), cudaMemcpyHostToDevice));
    PPN_CU(cudaMemcpy(d_btiles, bt.data(), sizeof(TileRef) * bt.size(), cudaMemcpyHostToDevice));
    PPN_CU(cudaMemcpy(d_ptiles, pt.data(), sizeof(TileRef) * pt.size(), cudaMemcpyHostToDevice));
    PPN_CU(cudaMemcpy(d_etiles, et.data(), sizeof(TileRef) * et.size(), cudaMemcpyHostToDevice));
    std::vector<Ctl> c0(n);
    std::memset(c0.data(), 0, sizeof(Ctl) * n);
    for (auto& c : c0) c.pcg_done = 1;
    PPN_CU(cudaMemcpy(d_ctl, c0.data(), sizeof(Ctl) * n, cudaMemcpyHostToDevice));
    for (int i = 0; i < n; ++i) {
      h_desc[i] = S[i]->d;
      h_desc[i].ctl = d_ctl + i;
      h_desc[i].active = 0;
    }
    return PPN_OK;
  }
  // write the per-step descriptor scalars of the members back to their scenes
  // (before the group is rebuilt for other members)
  void stash() {
    for (size_t i = 0; i < S.size() && i < h_desc.size(); ++i) {
      S[i]->d.it_id = h_desc[i].it_id;
      S[i]->d.round_id = h_desc[i].round_id;
      S[i]->d.delta = h_desc[i].delta;
      S[i]->d.gamma = h_desc[i].gamma;
    }
  }
  ppn_status upload_desc() {
    const size_t b = sizeof(SceneDev<T>) * h_desc.size();
    void* p = staging.take(b, st);
    if (!p) {
      set_error("pinned staging allocation failed");
      return PPN_ERR_OOM;
    }
    std::memcpy(p, h_desc.data(), b);
    PPN_CU(cudaMemcpyAsync(d_desc, p, b, cudaMemcpyHostToDevice, st));
    return PPN_OK;
  }
  ppn_status upload(void* dst, const void* src, size_t b) {
    void* p = staging.take(b, st);
    if (!p) {
      set_error("pinned staging allocation failed");
      return PPN_ERR_OOM;
    }
    std::memcpy(p, src, b);
    PPN_CU(cudaMemcpyAsync(dst, p, b, cudaMemcpyHostToDevice, st));
    return PPN_OK;
  }
  ppn_status sync_ctl() {
    PPN_CU(cudaMemcpyAsync(h_ctl, d_ctl, sizeof(Ctl) * S.size(), cudaMemcpyDeviceToHost, st));
    PPN_CU(cudaMemcpyAsync(h_bar, d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
    PPN_CU(cudaStreamSynchronize(st));
    staging.reset();
    if (timer) timer->collect();
    if (tune_pending) {  // the timed PCG launch has finished: its time per CG iteration
      tune_pending = false;
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, tune_ev[0], tune_ev[1]) == cudaSuccess) {
        int it = 0;
        for (int k : tune_slots) it = std::max(it, h_ctl[k].pcg_iters);
        pcg_tuner().report(tune_key, tune_choice, ms, it);
      } else {
        cudaGetLastError();
      }
    }
    return PPN_OK;
  }
  void set_active(const std::vector<char>& on) {
    for (size_t i = 0; i < S.size(); ++i) h_desc[i].active = on[i] ? 1 : 0;
  }
};

// Per-scene host state of the lockstep Newton loop.
struct HostState {
  int mode = 0;
  int status = PPN_OK;
  bool running = true;
  int k = 0;
  double delta = 0, g0 = -1, gn2 = 0, ginf = 0;
  int n_proj = 0;
  bool ind = false, fallback = false;
  int precond_fail = 0, pcg_iters_last = 0;
  double E0 = 0, dd = 0, dxmax = 0, gamma = 1;
  bool has_next = false;  // E_next holds the incremental potential at the current iterate
  double E_next = 0;      // (the last accepted trial energy of this time step)
  int halvings = 0;
  int countdown = 0;  // PDN: iterations left that assemble projected
  int ties_pending = 0;          // selection ties of the rounds since the last solve
  std::vector<int> sel_pending;  // elements those rounds selected (recorded on request)
  bool pre = false;   // this iteration projects every element before assembly
  int n_elem = 0;     // elements of the current iteration: tets + contact elements
  double tol = 0;     // Newton tolerance of the current step
  ppn_iter_stats cur{};
  ppn_step_stats tot{};
};

template <typename T>
struct Driver {
  Group<T>& G;
  std::vector<HostState> H;
  explicit Driver(Group<T>& g) : G(g) {}
  // parameters of scene i (scenes of one batch may differ)
  const ppn_params& Pi(int i) const { return G.S[i]->params; }

  double pcg_iter_bytes() const {
    double b = 0;
    for (auto* s : G.S) b += (double)s->nnzb * (9 * sizeof(T) + 4) + (double)s->nv * (4 + 12 * sizeof(T) + 9 * sizeof(T) + 12 * 4 * sizeof(T));
    return b;
  }

  template <typename F>
  void timed(int fam, double bytes, F&& f) {
    G.timer->begin(fam, G.st, bytes);
    f();
    G.timer->end(G.st);
  }

  ppn_status check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("kernel launch: ") + cudaGetErrorString(e));
      return PPN_ERR_CUDA;
    }
    return PPN_OK;
  }

  // PCG over the scenes flagged in `on`; results land in each scene's Ctl
  ppn_status solve(const std::vector<char>& on, int b_from_g) {
    std::vector<int> ids;
    for (size_t i = 0; i < on.size(); ++i)
      if (on[i]) ids.push_back((int)i);
    if (ids.empty()) return PPN_OK;
    G.set_active(on);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    // slots of at most PCG_MAX_SCENES scenes per launch
    for (size_t b = 0; b < ids.size(); b += PCG_MAX_SCENES) {
      const size_t e = std::min(ids.size(), b + PCG_MAX_SCENES);
      std::vector<int> sl(ids.begin() + b, ids.begin() + e);
      if (sl != G.pcg_ids) {
        std::vector<TileRef> tt;
        for (size_t k = 0; k < sl.size(); ++k)
          for (int t = 0; t < G.S[sl[k]]->n_ptiles; ++t) tt.push_back({(int)k, t});
        if ((rc = G.upload(G.d_ids, sl.data(), sizeof(int) * sl.size()))) return rc;
        if ((rc = G.upload(G.d_pcgtiles, tt.data(), sizeof(TileRef) * tt.size()))) return rc;
        G.pcg_ids = sl;
        G.pcg_ntiles = (int)tt.size();
        plan_smem(sl, tt);
      }
      const int n_tiles = G.pcg_ntiles;
      PcgLaunch L;
      L.n_tiles = n_tiles;
      L.tiles = G.d_pcgtiles;
      L.n_scenes = (int)sl.size();
      L.scene_ids = G.d_ids;
      L.bar = G.d_bar;
      L.grid = G.pcg_smem_bytes ? G.pcg_smem_grid : std::min(G.pcg_grid, n_tiles);
      L.group = G.pcg_group;
      L.use_b_from_g = b_from_g;
      L.smem_bytes = G.pcg_smem_bytes;
      L.smem_blocks = G.pcg_smem_blocks;
      L.sr_mode = G.pcg_sr_mode;
      L.halo_off = G.halo_off;
      L.halo_col = G.halo_col;
      L.halo_ref = G.halo_ref;
      L.halo_cap = G.halo_cap;
      for (size_t k = 0; k < sl.size() && k < (size_t)HALO_MAX_SCENES; ++k) {
        L.zrec[k] = G.h_desc[sl[k]].zrec;
        L.zrec_bytes[k] = sizeof(T) * 16 * (size_t)G.S[sl[k]]->nv;
      }
      const bool tune = G.pcg_sr && G.pcg_tune && ids.size() <= (size_t)PCG_MAX_SCENES;
      L.l2_keep = std::getenv("PPN_PCG_L2_KEEP") ? 1 : 0;
      if (tune) {
        G.tune_choice = pcg_tuner().choose(G.tune_key, G.tune_allowed);
        L.sr_mode = (G.tune_choice & 1) ? SR_GLOBAL : SR_STREAM;
        L.l2_keep = G.tune_choice >> 1;
        L.smem_bytes = G.tune_bytes[G.tune_choice & 1];
        for (cudaEvent_t& e : G.tune_ev)
          if (!e && cudaEventCreate(&e) != cudaSuccess) {
            set_error("cudaEventCreate failed");
            return PPN_ERR_CUDA;
          }
        PPN_CU(cudaEventRecord(G.tune_ev[0], G.st));
      }
      for (int k : sl) G.S[k]->last_pcg_layout = G.pcg_sr ? L.sr_mode : L.smem_bytes ? 4 : 5;
      L.launch_seq = ++G.pcg_launch_seq;
      L.flags = G.d_flags;
      L.n_pword = (int)sl.size();
      for (size_t k = 0; k < sl.size(); ++k) {
        L.pword[k] = G.h_desc[sl[k]].pword;
        L.pword_bytes[k] = sizeof(unsigned long long) * 8 * G.S[sl[k]]->n_ptiles * pword_stride(G.S[sl[k]]->n_ptiles);
      }
      double bytes = 0.0;
      cudaError_t err = cudaSuccess;
      timed(FAM_PCG, bytes, [&] {
        if constexpr (sizeof(T) == sizeof(float)) {
          if (G.pcg_sr) {
            err = launch_pcg_sr(reinterpret_cast<const SceneDev<float>*>(G.d_desc), L, G.st);
            return;
          }
        }
        err = L.smem_bytes ? launch_pcg_smem<T>(G.d_desc, L, G.st) : launch_pcg<T>(G.d_desc, L, G.st);
      });
      if (err != cudaSuccess) {
        set_error(std::string("PCG launch: ") + cudaGetErrorString(err));
        return PPN_ERR_CUDA;
      }
      if (tune) {
        PPN_CU(cudaEventRecord(G.tune_ev[1], G.st));
        G.tune_pending = true;
        G.tune_slots = sl;
      }
    }
    return PPN_OK;
  }

  // SR_HALO tables for `grid` CTAs over the launch's tile table (every PCG tile
  // of each slot, slot after slot, as solve() builds it): build_halo_tables.
  int build_halo(const std::vector<int>& sl, int grid, std::vector<int>& tab) {
    std::vector<HaloPattern> pats;
    for (int k : sl) {
      const SceneImpl<T>& sc = *G.S[k];
      pats.push_back({sc.nv, sc.h_row_ptr.data(), sc.h_col.data()});
    }
    return build_halo_tables(pats, grid, tab);
  }

  // Choose the PCG kernel for the launch's tile table.  FP32 (unless
  // PPN_PCG_STD is set): the single-reduction kernel, with the rows' BSR blocks
  // and vectors resident in shared memory and the halo replicated when they fit
  // (unless PPN_PCG_NO_HALO is set), else without the halo, else the vectors
  // alone, else neither.  Otherwise the standard resident kernel when its
  // layout fits, else the global-memory kernel.
  void plan_smem(const std::vector<int>& sl, const std::vector<TileRef>& tt) {
    G.pcg_smem_bytes = 0;
    G.pcg_sr = false;
    G.pcg_tune = false;
    G.halo_off = G.halo_col = G.halo_ref = nullptr;
    G.halo_cap = 0;
    if (std::getenv("PPN_PCG_GLOBAL")) return;
    const int n_tiles = (int)tt.size();
    // largest rows / blocks of one CTA when n_tiles are split over `grid` CTAs, and the
    // largest slot count of the single-reduction kernel's resident layouts (per 16-row
    // group, 32 slots per step of ceil(longest row / 2))
    int max_slots = 0;
    auto layout = [&](int grid, int& max_items, int& max_blocks) {
      max_items = max_blocks = max_slots = 0;
      for (int b = 0; b < grid; ++b) {
        const int t0 = (int)(((long long)b * n_tiles) / grid), t1 = (int)(((long long)(b + 1) * n_tiles) / grid);
        int blocks = 0, slots = 0;
        for (int t = t0; t < t1; ++t) {
          const SceneImpl<T>& sc = *G.S[sl[tt[t].scene]];
          const int r0 = tt[t].tile * PCG_TILE, r1 = std::min(sc.nv, r0 + PCG_TILE);
          if (r1 > r0) blocks += (int)(sc.h_row_ptr[r1] - sc.h_row_ptr[r0]);
          for (int g = r0; g < r1; g += 16) {
            int m = 0;
            for (int r = g; r < std::min(r1, g + 16); ++r) m = std::max(m, (int)(sc.h_row_ptr[r + 1] - sc.h_row_ptr[r]));
            slots += 32 * ((m + 1) / 2);
          }
        }
        max_items = std::max(max_items, (t1 - t0) * PCG_TILE);
        max_blocks = std::max(max_blocks, blocks);
        max_slots = std::max(max_slots, slots);
      }
    };
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int max_items = 0, max_blocks = 0;
    if (sizeof(T) == sizeof(float) && !std::getenv("PPN_PCG_STD")) {
      const int grid = std::min(n_tiles, std::min(n_sm, 1024));  // one CTA per SM
      layout(grid, max_items, max_blocks);
      // blocks resident when they fit; otherwise the streamed layouts, chosen per
      // launch by the tuner when both fit (PPN_PCG_STREAM / PPN_PCG_SR_GLOBAL:
      // start at the streamed / global layout, no tuning)
      const bool f_str = std::getenv("PPN_PCG_STREAM") != nullptr, f_gl = std::getenv("PPN_PCG_SR_GLOBAL") != nullptr;
      const int first = f_gl ? SR_GLOBAL : f_str ? SR_STREAM : SR_RES;
      bool fits[3] = {false, false, false};
      size_t bytes[3];
      for (int mode = first; mode <= SR_GLOBAL; ++mode) {
        bytes[mode] = pcg_sr_smem_bytes(max_items, mode == SR_RES ? max_slots : 0, 0, mode);
        fits[mode] = bytes[mode] <= (size_t)212 * 1024 && pcg_sr_max_grid(dev, bytes[mode], mode) >= grid;
        if (fits[mode] && (mode == SR_RES || f_str || f_gl)) break;
      }
      if (first == SR_RES && fits[SR_RES] && sl.size() <= (size_t)HALO_MAX_SCENES && max_items <= SR_HALO_MAX_ROWS &&
          !std::getenv("PPN_PCG_NO_HALO")) {
        std::vector<int> tab;
        const int nh = build_halo(sl, grid, tab);
        const size_t hb = nh < 0 ? 0 : pcg_sr_smem_bytes(max_items, max_slots, nh, SR_HALO);
        if (nh >= 0 && hb <= (size_t)227 * 1024 && pcg_sr_max_grid(dev, hb, SR_HALO) >= grid) {
          if (tab.size() > G.cap_halo) {
            if (G.d_halo) {  // (cudaFree waits for launches that may still read it)
              const auto old = std::find(G.allocs.begin(), G.allocs.end(), (void*)G.d_halo);
              if (old != G.allocs.end()) G.allocs.erase(old);
              dev_free(G.dalloc, G.d_halo);
            }
            G.d_halo = G.template alloc<int>(tab.size());
            G.cap_halo = G.d_halo ? tab.size() : 0;
          }
          if (G.d_halo && G.upload(G.d_halo, tab.data(), sizeof(int) * tab.size()) == PPN_OK) {
            G.halo_off = G.d_halo;
            G.halo_col = G.d_halo + 2 * (grid + 1);
            G.halo_ref = G.halo_col + tab[2 * grid];
            G.halo_cap = nh;
            G.pcg_smem_bytes = hb;
            G.pcg_smem_blocks = max_slots;
            G.pcg_smem_grid = grid;
            G.pcg_sr = true;
            G.pcg_sr_mode = SR_HALO;
            return;
          }
        }
      }
      for (int mode = first; mode <= SR_GLOBAL; ++mode) {
        if (!fits[mode]) continue;
        G.pcg_smem_bytes = bytes[mode];
        G.pcg_smem_blocks = mode == SR_RES ? max_slots : 0;
        G.pcg_smem_grid = grid;
        G.pcg_sr = true;
        G.pcg_sr_mode = mode;
        // tuned: the streamed layouts that fit, each at both L2 priorities (not when a
        // switch fixes the layout)
        G.pcg_tune = (mode == SR_STREAM || mode == SR_GLOBAL) && !f_str && !f_gl;
        if (G.pcg_tune) {
          double mat = 0.0;
          for (int k : sl) mat += (double)G.S[k]->nnzb * (9 * sizeof(float) + 4);
          int lg = 0;
          while (lg < 30 && (double)(1ll << (lg + 1)) <= mat / 1e6) ++lg;
          G.tune_key = {(max_items + PCG_TILE - 1) / PCG_TILE, max_blocks / std::max(1, max_items), lg};
          G.tune_allowed = (mode == SR_STREAM ? 0x5u : 0u) | (fits[SR_GLOBAL] ? 0xAu : 0u);
          G.tune_bytes[0] = bytes[SR_STREAM];
          G.tune_bytes[1] = bytes[SR_GLOBAL];
        }
        return;
      }
    }
    const int grid = std::min(G.pcg_grid, n_tiles);
    if (grid > 1024) return;
    layout(grid, max_items, max_blocks);
    const size_t bytes = pcg_smem_bytes(max_items, max_blocks, (int)sizeof(T));
    if (bytes > (size_t)196 * 1024) return;
    const int mg = pcg_smem_max_grid(G.pcg_group, dev, bytes, (int)sizeof(T));
    if (mg < grid) return;
    G.pcg_smem_bytes = bytes;
    G.pcg_smem_blocks = max_blocks;
    G.pcg_smem_grid = grid;
  }

  // Start a time step for the flagged slots (their H[i].mode and H[i].tol set):
  // predictor, Dirichlet targets, delta = infinity (Algorithm 1, before the Newton loop).
  ppn_status begin(const std::vector<char>& on) {
    const int n = (int)G.S.size();
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const int mode = H[i].mode;
      const double tol = H[i].tol;
      H[i] = HostState();
      H[i].mode = mode;
      H[i].tol = tol;
      H[i].delta = std::numeric_limits<double>::infinity();
      G.h_desc[i].delta = H[i].delta;
      G.S[i]->iters.clear();
      G.S[i]->attempts.clear();
      G.S[i]->attempt_sel.clear();
      G.S[i]->iter_g.clear();
    }
    G.set_active(on);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    timed(FAM_VECTOR, 0, [&] { launch_predict<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st); });
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      SceneImpl<T>& s = *G.S[i];
      const double* tg = s.ext_targets ? s.ext_targets : s.d_targets;
      launch_apply_targets<T>(G.d_desc, i, s.d_fixed_list, tg, s.nfixed, 0, G.st);
      s.ext_targets = nullptr;
    }
    ppn_status rc2 = check_launch();
    if (rc2) return rc2;
    return advance_obstacles(on);
  }

  // Feasibility of the initial iterates against the applied obstacles, and the
  // advance of moving planes toward their requested poses (at most ccd_safety x
  // the smallest free-vertex distance per step).
  ppn_status advance_obstacles(const std::vector<char>& on) {
    const int n = (int)G.S.size();
    std::vector<char> ob(n, 0);
    int kmax = 0;
    for (int i = 0; i < n; ++i)
      if (on[i] && G.S[i]->n_obst > 0) {
        ob[i] = 1;
        kmax = std::max(kmax, G.S[i]->n_obst);
      }
    if (kmax == 0) return PPN_OK;
    G.set_active(ob);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    std::vector<std::vector<double>> gap(n, std::vector<double>(MAX_OBST, 0.0));
    for (int k0 = 0; k0 < kmax; k0 += 4) {
      launch_obst_gap<T>(G.d_desc, G.d_vtiles, G.n_vtiles, k0, G.st);
      if ((rc = check_launch())) return rc;
      if ((rc = G.sync_ctl())) return rc;
      for (int i = 0; i < n; ++i)
        if (ob[i])
          for (int j = 0; j < 4 && k0 + j < MAX_OBST; ++j) gap[i][k0 + j] = G.h_ctl[i].gap[j];
    }
    for (int i = 0; i < n; ++i) {
      if (!ob[i]) continue;
      SceneImpl<T>& s = *G.S[i];
      bool moved = false;
      for (int k = 0; k < s.n_obst; ++k) {
        if (!(gap[i][k] < std::numeric_limits<double>::infinity())) {
          set_error("the state is not feasible for obstacle " + std::to_string(k));
          H[i].status = PPN_ERR_INVALID_ARG;
          H[i].running = false;
          break;
        }
        ObstDev& o = s.obs_app.o[k];
        const ObstDev& q = s.obs_req.o[k];
        if (o.type != OBST_PLANE) continue;
        const double adv = o.a[0] * (q.p[0] - o.p[0]) + o.a[1] * (q.p[1] - o.p[1]) + o.a[2] * (q.p[2] - o.p[2]);
        const double m = gap[i][k] > 0.0 ? 1.0 / gap[i][k] : std::numeric_limits<double>::infinity();
        const double f = adv > 0.0 ? std::min(1.0, Pi(i).ccd_safety * m / adv) : 1.0;
        for (int c = 0; c < 3; ++c) {
          const double pc = o.p[c] + f * (q.p[c] - o.p[c]);
          moved |= pc != o.p[c];
          o.p[c] = pc;
        }
      }
      if (moved) PPN_CU(cudaMemcpyAsync(s.d_obs, &s.obs_app, sizeof(ObstSet), cudaMemcpyHostToDevice, G.st));
    }
    return PPN_OK;
  }

  bool any_running() const {
    for (const HostState& h : H)
      if (h.running) return true;
    return false;
  }

  // One Newton iteration of every running slot (lockstep over the group).
  ppn_status tick() {
    const int n = (int)G.S.size();
    ppn_status rc = PPN_OK;
    std::vector<char> run(n, 0);
    bool any = false;
    for (int i = 0; i < n; ++i) {
      run[i] = H[i].running;
      any |= H[i].running;
    }
    if (!any) return PPN_OK;
    // ---- element evaluation and gradient
    for (int i = 0; i < n; ++i)
      if (run[i]) {
        G.h_desc[i].it_id = ++G.S[i]->it_counter;
        G.h_desc[i].gamma = 0.0;
      }
    G.set_active(run);
    if ((rc = G.upload_desc())) return rc;
    timed(FAM_ELEMENT, 0, [&] { launch_element<T>(G.d_desc, G.d_ttiles, G.n_ttiles, 0, G.st); });
    timed(FAM_GRADIENT, 0, [&] { launch_gradient<T>(G.d_desc, G.d_vtiles, G.n_vtiles, 0, G.st); });
    if ((rc = check_launch())) return rc;
    if ((rc = G.sync_ctl())) return rc;
    for (int i = 0; i < n; ++i)  // the iteration's assembled gradient, on request (diagnostics)
      if (run[i] && G.S[i]->record_sel) {
        SceneImpl<T>& s = *G.S[i];
        std::vector<double4> g4(s.nv);
        PPN_CU(cudaMemcpyAsync(g4.data(), s.d.g, sizeof(double4) * s.nv, cudaMemcpyDeviceToHost, G.st));
        PPN_CU(cudaStreamSynchronize(G.st));
        std::vector<double> g3(3 * (size_t)s.nv);
        for (int v = 0; v < s.nv; ++v) {
          g3[3 * v] = g4[v].x;
          g3[3 * v + 1] = g4[v].y;
          g3[3 * v + 2] = g4[v].z;
        }
        s.iter_g.push_back(std::move(g3));
      }
    std::vector<char> solve_on(n, 0), pn_on(n, 0);
    bool any_solve = false, any_pn = false;
    for (int i = 0; i < n; ++i) {
      if (!run[i]) continue;
      HostState& h = H[i];
      const Ctl& c = G.h_ctl[i];
      h.gn2 = std::sqrt(c.grad[0]);
      h.ginf = c.grad[3];
      h.n_elem = G.S[i]->nt + (int)c.grad[2];  // tets + contact elements
      const double floor = Pi(i).grad_floor * std::sqrt(c.grad[1]);
      h.tot.final_grad_norm2 = h.gn2;
      if (!std::isfinite(h.gn2)) {
        h.status = PPN_ERR_NONFINITE;
        h.running = false;
        continue;
      }
      if (h.k == 0) h.g0 = h.gn2;
      if (Pi(i).tol_kind == 0 && (h.gn2 <= h.tol * h.g0 || h.gn2 <= floor)) {
        h.status = PPN_OK;
        h.running = false;
        continue;
      }
      if (h.k >= Pi(i).newton_max_iter) {
        h.status = PPN_ERR_NEWTON_MAXITER;
        h.running = false;
        continue;
      }
      h.cur = ppn_iter_stats{};
      h.ties_pending = 0;
      h.sel_pending.clear();
      h.cur.newton_iter = h.k;
      h.cur.grad_norm2 = h.gn2;
      h.cur.grad_norminf = h.ginf;
      h.n_proj = 0;
      h.fallback = false;
      solve_on[i] = 1;
      any_solve = true;
      h.pre = h.mode == PPN_MODE_PN || (h.mode == PPN_MODE_PDN && h.countdown > 0);
      if (h.pre) {
        pn_on[i] = 1;
        any_pn = true;
        if (h.mode == PPN_MODE_PDN) --h.countdown;
      }
    }
    if (!any_solve) return PPN_OK;
    // ---- PN: select every element and clamp before assembly
    if (any_pn) {
      for (int i = 0; i < n; ++i)
        if (pn_on[i]) G.h_desc[i].delta = -1.0;
      if ((rc = select_and_project(pn_on, true))) return rc;
      for (int i = 0; i < n; ++i)
        if (pn_on[i]) H[i].n_proj = H[i].n_elem;
    }
    // ---- assembly and first solve
    G.set_active(solve_on);
    if ((rc = G.upload_desc())) return rc;
    timed(FAM_ASSEMBLE, 0, [&] { launch_assemble<T>(G.d_desc, G.d_btiles, G.n_btiles, G.d_vtiles, G.n_vtiles, G.st); });
    if ((rc = check_launch())) return rc;
    if ((rc = solve(solve_on, 1))) return rc;
    if ((rc = G.sync_ctl())) return rc;
    if ((rc = check_errors(solve_on))) return rc;
    std::vector<char> retry(n, 0), pdn(n, 0);
    bool any_retry = false, any_pdn = false;
    for (int i = 0; i < n; ++i) {
      if (!solve_on[i]) continue;
      record_attempt(i, 0, H[i].pre ? H[i].n_elem : 0, std::numeric_limits<double>::infinity());
      if (H[i].ind && H[i].mode == PPN_MODE_PPN) {
        retry[i] = 1;
        any_retry = true;
      } else if (H[i].ind && H[i].mode == PPN_MODE_PDN && !H[i].pre) {
        pdn[i] = 1;
        any_pdn = true;
      } else if (H[i].ind) {
        H[i].fallback = true;
      }
    }
    // ---- PDN: indefinite, so project every element in place and solve again
    if (any_pdn) {
      for (int i = 0; i < n; ++i)
        if (pdn[i]) {
          G.h_desc[i].delta = -1.0;  // select every element not yet projected
          G.h_desc[i].round_id = ++G.S[i]->round_counter;
        }
      if ((rc = select_and_project(pdn, false))) return rc;
      if ((rc = update_in_place(pdn))) return rc;
      if ((rc = solve(pdn, 1))) return rc;
      if ((rc = G.sync_ctl())) return rc;
      if ((rc = check_errors(pdn))) return rc;
      for (int i = 0; i < n; ++i)
        if (pdn[i]) {
          record_attempt(i, 1, H[i].n_elem, -1.0);
          H[i].countdown = Pi(i).pdn_countdown;
          if (H[i].ind) H[i].fallback = true;  // fully projected and still indefinite (rounding)
        }
    }
    // ---- PPN retries (Algorithm 1 inner loop); a round that selects nothing new skips the
    // solve and tightens delta again, so attempts are numbered by solve
    while (any_retry) {
      for (int i = 0; i < n; ++i)
        if (retry[i]) {
          HostState& h = H[i];
          if (std::isinf(h.delta)) h.delta = Pi(i).alpha * h.ginf;
          G.h_desc[i].delta = h.delta;
          G.h_desc[i].round_id = ++G.S[i]->round_counter;
        }
      if ((rc = select_and_project(retry, false))) return rc;
      std::vector<char> resolve(n, 0);
      bool any_resolve = false;
      for (int i = 0; i < n; ++i)
        if (retry[i] && G.h_ctl[i].n_new + G.h_ctl[i].n_new_c > 0) {
          resolve[i] = 1;
          any_resolve = true;
        }
      if (any_resolve) {
        if ((rc = update_in_place(resolve))) return rc;
        if ((rc = solve(resolve, 1))) return rc;
        std::vector<int> n_new(n);
        for (int i = 0; i < n; ++i) n_new[i] = G.h_ctl[i].n_new + G.h_ctl[i].n_new_c;
        if ((rc = G.sync_ctl())) return rc;
        if ((rc = check_errors(resolve))) return rc;
        for (int i = 0; i < n; ++i)
          if (resolve[i]) record_attempt(i, H[i].cur.pcg_attempts, n_new[i], H[i].delta);  // solves so far
      }
      any_retry = false;
      for (int i = 0; i < n; ++i) {
        if (!retry[i]) continue;
        HostState& h = H[i];
        if (h.ind) {
          if (h.n_proj >= h.n_elem) {
            h.fallback = true;  // fully projected and still indefinite (rounding)
            retry[i] = 0;
          } else {
            h.delta *= Pi(i).alpha;  // tighten
            any_retry = true;
          }
        } else {
          retry[i] = 0;
        }
      }
    }
    for (int i = 0; i < n; ++i)
      if (solve_on[i] && H[i].mode == PPN_MODE_PPN) H[i].delta *= Pi(i).beta;  // relax
    // ---- fallback directions when the solve gave no usable iterate
    {
      std::vector<char> fb2(n, 0), fb3(n, 0);
      bool a2 = false, a3 = false;
      for (int i = 0; i < n; ++i) {
        if (!solve_on[i] || !H[i].fallback) continue;
        if (H[i].pcg_iters_last == 0) {
          if (H[i].precond_fail) {
            fb3[i] = 1;
            a3 = true;
            H[i].cur.fallback = 3;
          } else {
            fb2[i] = 1;
            a2 = true;
            H[i].cur.fallback = 2;
          }
        } else {
          H[i].cur.fallback = 1;
        }
      }
      if (a2 && (rc = fallback_dir(fb2, 2))) return rc;
      if (a3 && (rc = fallback_dir(fb3, 3))) return rc;
    }
    // ---- energy at gamma = 0 and directional derivative
    if ((rc = energy(solve_on, true))) return rc;
    {
      std::vector<char> fb(n, 0);
      bool afb = false;
      int kind = 2;
      for (int i = 0; i < n; ++i) {
        if (!solve_on[i]) continue;
        HostState& h = H[i];
        if (!(h.dd < 0.0)) {
          fb[i] = 1;
          afb = true;
          h.cur.fallback = h.precond_fail ? 3 : 2;
          kind = h.cur.fallback;
        }
      }
      if (afb) {
        // rare: scenes needing the fallback are handled one kind at a time
        for (int kd = 2; kd <= 3; ++kd) {
          std::vector<char> sel(n, 0);
          bool a = false;
          for (int i = 0; i < n; ++i)
            if (fb[i] && H[i].cur.fallback == kd) {
              sel[i] = 1;
              a = true;
            }
          if (a && (rc = fallback_dir(sel, kd))) return rc;
        }
        (void)kind;
        if ((rc = energy(fb, true))) return rc;
      }
    }
    // ---- intersection-based filtering: the first contact time along dx bounds the step
    std::vector<double> gamma0(n, 1.0);
    if (any_obstacles(solve_on)) {
      std::vector<char> cc(n, 0);
      for (int i = 0; i < n; ++i) cc[i] = solve_on[i] && G.S[i]->n_obst > 0;
      G.set_active(cc);
      if ((rc = G.upload_desc())) return rc;
      launch_ccd<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st);
      if ((rc = check_launch())) return rc;
      if ((rc = G.sync_ctl())) return rc;
      for (int i = 0; i < n; ++i)
        if (cc[i] && G.h_ctl[i].ccd > 0.0) gamma0[i] = std::min(1.0, Pi(i).ccd_safety / G.h_ctl[i].ccd);
    }
    // ---- backtracking line search (Armijo)
    std::vector<char> ls(n, 0);
    bool any_ls = false;
    for (int i = 0; i < n; ++i)
      if (solve_on[i]) {
        ls[i] = 1;
        any_ls = true;
        H[i].gamma = gamma0[i];
        H[i].halvings = 0;
        H[i].cur.dir_deriv = H[i].dd;
        H[i].cur.energy = H[i].E0;
      }
    std::vector<char> accept(n, 0);
    while (any_ls) {
      for (int i = 0; i < n; ++i)
        if (ls[i]) G.h_desc[i].gamma = H[i].gamma;
      if ((rc = energy(ls, false))) return rc;
      any_ls = false;
      for (int i = 0; i < n; ++i) {
        if (!ls[i]) continue;
        HostState& h = H[i];
        const double Et = G.h_ctl[i].energy[0];
        // slack: the FP64 energy sums resolve E only to a few ulps
        if (Et <= h.E0 + Pi(i).armijo_c * h.gamma * h.dd + Pi(i).ls_slack * std::fabs(h.E0)) {
          ls[i] = 0;
          accept[i] = 1;
          h.has_next = true;  // k_axpy_u forms the accepted point with the trial's own operations
          h.E_next = Et;
          h.cur.gamma = h.gamma;
          h.cur.energy_new = Et;
          h.cur.ls_halvings = h.halvings;
        } else if (h.halvings >= Pi(i).ls_max_halvings) {
          ls[i] = 0;
          h.status = PPN_ERR_LINESEARCH;
          h.running = false;
          h.cur.ls_halvings = h.halvings;
          finish_iter(i);
        } else {
          h.gamma *= 0.5;
          h.halvings += 1;
          any_ls = true;
        }
      }
    }
    // ---- position update
    bool any_acc = false;
    for (int i = 0; i < n; ++i) any_acc |= accept[i];
    if (any_acc) {
      for (int i = 0; i < n; ++i)
        if (accept[i]) G.h_desc[i].gamma = H[i].gamma;
      G.set_active(accept);
      if ((rc = G.upload_desc())) return rc;
      timed(FAM_VECTOR, 0, [&] { launch_axpy_u<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st); });
      if ((rc = check_launch())) return rc;
    }
    for (int i = 0; i < n; ++i) {
      if (!accept[i]) continue;
      HostState& h = H[i];
      finish_iter(i);
      h.k += 1;
      if (Pi(i).tol_kind == 1 && h.gamma * h.dxmax / G.S[i]->dt < h.tol) {
        h.status = PPN_OK;
        h.running = false;
      }
    }
    return PPN_OK;
  }

  // End the time step of the flagged slots: velocities and step statistics.
  ppn_status finish(const std::vector<char>& on) {
    const int n = (int)G.S.size();
    G.set_active(on);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    timed(FAM_VECTOR, 0, [&] { launch_velocity<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st); });
    if ((rc = check_launch())) return rc;
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      H[i].tot.status = H[i].status;
      H[i].tot.newton_iters = (int)G.S[i]->iters.size();
      // keep the scene's own descriptor scalars in step with the group copy
      G.S[i]->d.it_id = G.h_desc[i].it_id;
      G.S[i]->d.round_id = G.h_desc[i].round_id;
    }
    return PPN_OK;
  }

  // One time step of every scene of the group (all start and end together).
  ppn_status step(const int* modes, double tol) {
    const int n = (int)G.S.size();
    H.assign(n, HostState());
    std::vector<char> on(n, 1);
    for (int i = 0; i < n; ++i) {
      H[i].mode = modes[i];
      H[i].tol = tol;
    }
    cudaEventRecord(G.S[0]->ev_a, G.st);
    ppn_status rc = begin(on);
    if (rc) return rc;
    while (any_running())
      if ((rc = tick())) return rc;
    if ((rc = finish(on))) return rc;
    cudaEventRecord(G.S[0]->ev_b, G.st);
    PPN_CU(cudaStreamSynchronize(G.st));
    G.staging.reset();
    G.timer->collect();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, G.S[0]->ev_a, G.S[0]->ev_b);
    for (int i = 0; i < n; ++i) H[i].tot.device_ms = ms;
    return PPN_OK;
  }

  void finish_iter(int i) {
    HostState& h = H[i];
    h.cur.n_projected_total = h.n_proj;
    h.cur.delta = h.delta;
    h.cur.precond_fail = h.precond_fail;
    G.S[i]->iters.push_back(h.cur);
    h.tot.total_projections += h.n_proj;
    h.tot.total_cg_iters += h.cur.cg_iters;
    h.tot.total_attempts += h.cur.pcg_attempts;
  }

  void record_attempt(int i, int attempt, int n_new, double delta) {
    HostState& h = H[i];
    const Ctl& c = G.h_ctl[i];
    h.ind = c.pcg_ind != 0;
    h.precond_fail = c.pcg_precond_fail;
    h.pcg_iters_last = c.pcg_iters;
    h.cur.pcg_attempts += 1;
    h.cur.cg_iters += c.pcg_iters;
    ppn_attempt a;
    a.newton_iter = h.k;
    a.attempt = attempt;
    a.n_new_projected = n_new;
    a.ind = h.ind;
    a.cg_iters = c.pcg_iters;
    a.delta = delta;
    a.n_ties = h.ties_pending;
    G.S[i]->attempts.push_back(a);
    if (G.S[i]->record_sel) {
      std::sort(h.sel_pending.begin(), h.sel_pending.end());
      G.S[i]->attempt_sel.push_back(h.sel_pending);
    }
    h.ties_pending = 0;
    h.sel_pending.clear();
  }

  ppn_status check_errors(const std::vector<char>& on) {
    for (size_t i = 0; i < on.size(); ++i) {
      if (!on[i]) continue;
      if (G.h_ctl[i].error & kErrTimeout) {
        set_error("PCG grid barrier timed out");
        return PPN_ERR_TIMEOUT;
      }
    }
    if (G.h_bar->timeout) {
      const GridBar& b = *G.h_bar;
      set_error("PCG grid wait timed out (wait " + std::to_string(b.to_site) + " at CG iteration " +
                std::to_string(b.to_iter) + " in CTA " + std::to_string(b.to_cta) + ": word " +
                std::to_string(b.to_slot) + "/" + std::to_string(b.to_index) + " last seen with stamp " +
                std::to_string(b.to_seen) + ")");
      return PPN_ERR_TIMEOUT;
    }
    return PPN_OK;
  }

  bool any_obstacles(const std::vector<char>& on) const {
    for (size_t i = 0; i < on.size(); ++i)
      if (on[i] && G.S[i]->n_obst > 0) return true;
    return false;
  }

  // selection (delta in the descriptor; < 0 selects all) + clamping of the
  // newly selected elements.  pn: no host sync needed for the count.
  ppn_status select_and_project(const std::vector<char>& on, bool pn) {
    const int n = (int)on.size();
    G.set_active(on);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
      if (on[i]) PPN_CU(cudaMemsetAsync(&G.d_ctl[i].n_new, 0, 4 * sizeof(int), G.st));  // n_new, n_new_c, n_ties, n_touched
    timed(FAM_SELECT, 0, [&] {
      launch_select<T>(G.d_desc, G.d_ttiles, G.n_ttiles, G.st);
      if (any_obstacles(on)) launch_select_contact<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st);  // clamps them too
    });
    if ((rc = check_launch())) return rc;
    // PN's passes over every element: one thread per tet (throughput); a PPN round's
    // selection: the warp form (latency).  PPN_PROJECT_THREAD=1 / PPN_PROJECT_WARP=1
    // force one form (tests, measurement)
    const bool warp = project_warp_form(!pn);
    const int per = warp ? PROJW_TETS : PROJ_CTA;
    std::vector<TileRef> jt;
    if (pn) {
      for (int i = 0; i < n; ++i)
        if (on[i])
          for (int t = 0; t < (G.S[i]->nt + per - 1) / per; ++t) jt.push_back({i, t});
    } else {
      if ((rc = G.sync_ctl())) return rc;
      for (int i = 0; i < n; ++i)
        if (on[i]) {
          const int nn = G.h_ctl[i].n_new, nc = G.h_ctl[i].n_new_c;
          H[i].n_proj += nn + nc;
          H[i].cur.n_new_projected += nn + nc;
          H[i].ties_pending += G.h_ctl[i].n_ties;
          H[i].tot.n_ties += G.h_ctl[i].n_ties;
          for (int t = 0; t < (nn + per - 1) / per; ++t) jt.push_back({i, t});
          if (G.S[i]->record_sel && H[i].mode == PPN_MODE_PPN && (rc = record_selection(i, nn, nc))) return rc;
        }
    }
    if (jt.empty()) return PPN_OK;
    if ((rc = G.upload(G.d_projtiles, jt.data(), sizeof(TileRef) * jt.size()))) return rc;
    timed(FAM_PROJECT, 0, [&] { launch_project<T>(G.d_desc, G.d_projtiles, (int)jt.size(), 0, G.st, warp); });
    return check_launch();
  }

  // In-place update H += S^eT dH^e S^e of the elements the last selection projected
  // (Sec. 4.1, "Incremental Hessian updates").  A scene whose selection touches at most
  // as many blocks as it has (16 per element) updates only those blocks; otherwise every
  // block is swept (PDN's all-element rounds).  Both forms give the same bits.
  // PPN_UPDATE_SWEEP=1 always sweeps (tests).  Contact elements update their diagonal blocks.
  ppn_status update_in_place(const std::vector<char>& on) {
    const int n = (int)on.size();
    const bool force_sweep = std::getenv("PPN_UPDATE_SWEEP") != nullptr;
    std::vector<char> sweep(n, 0);
    std::vector<int> touch;  // scenes updated block by block, with their tile counts
    std::vector<int> touch_tiles;
    bool any_sweep = false;
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const long long nn = G.h_ctl[i].n_new;
      if (nn == 0) continue;
      if (!force_sweep && 16 * nn <= (long long)G.S[i]->nnzb) {
        touch.push_back(i);
        touch_tiles.push_back((int)((16 * nn + TILE - 1) / TILE));
      } else {
        sweep[i] = 1;
        any_sweep = true;
      }
    }
    // the descriptors on the device mark the scenes of the last selection active; a
    // sweep runs over every block tile of the group, so it needs its own active set
    ppn_status rc = PPN_OK;
    if (any_sweep) {
      G.set_active(sweep);
      if ((rc = G.upload_desc())) return rc;
      timed(FAM_UPDATE, 0, [&] { launch_update<T>(G.d_desc, G.d_btiles, G.n_btiles, G.st); });
      if (!touch.empty()) {
        std::vector<char> t(n, 0);
        for (int i : touch) t[i] = 1;
        G.set_active(t);
        if ((rc = G.upload_desc())) return rc;
      }
    }
    if (!touch.empty()) {
      // a scene's first block tiles in the group's table are (scene, 0), (scene, 1), ...: a
      // touched-block launch takes that range directly, so nothing is uploaded for up to
      // two scenes; more scenes share one launch over an uploaded table
      if (touch.size() <= 2) {
        for (size_t k = 0; k < touch.size(); ++k) {
          int off = 0;
          for (int j = 0; j < touch[k]; ++j) off += G.S[j]->n_btiles;
          timed(FAM_UPDATE, 0,
                [&] { launch_update_touched<T>(G.d_desc, G.d_btiles + off, touch_tiles[k], G.st); });
        }
      } else {
        std::vector<TileRef> jt;
        for (size_t k = 0; k < touch.size(); ++k)
          for (int t = 0; t < touch_tiles[k]; ++t) jt.push_back({touch[k], t});
        if ((rc = G.upload(G.d_touchtiles, jt.data(), sizeof(TileRef) * jt.size()))) return rc;
        timed(FAM_UPDATE, 0, [&] { launch_update_touched<T>(G.d_desc, G.d_touchtiles, (int)jt.size(), G.st); });
      }
    }
    if (any_obstacles(on)) {
      G.set_active(on);
      if ((rc = G.upload_desc())) return rc;
      timed(FAM_UPDATE, 0, [&] { launch_update_contact<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st); });
    }
    return check_launch();
  }

  // the elements of scene i that the last selection chose (diagnostics, on request):
  // tets from the compacted list, contact elements (n_tets + v) from their stamps
  ppn_status record_selection(int i, int nn, int nc) {
    SceneImpl<T>& s = *G.S[i];
    std::vector<int>& out = H[i].sel_pending;
    if (nn > 0) {
      const size_t at = out.size();
      out.resize(at + nn);
      PPN_CU(cudaMemcpyAsync(out.data() + at, s.d.sel_list, sizeof(int) * nn, cudaMemcpyDeviceToHost, G.st));
    }
    std::vector<int> cr, cp;
    if (nc > 0) {
      cr.resize(s.nv);
      cp.resize(s.nv);
      PPN_CU(cudaMemcpyAsync(cr.data(), s.d.cround_stamp, sizeof(int) * s.nv, cudaMemcpyDeviceToHost, G.st));
      PPN_CU(cudaMemcpyAsync(cp.data(), s.d.cproj_stamp, sizeof(int) * s.nv, cudaMemcpyDeviceToHost, G.st));
    }
    PPN_CU(cudaStreamSynchronize(G.st));
    for (int v = 0; v < (int)cr.size(); ++v)
      if (cr[v] == G.h_desc[i].round_id && cp[v] == G.h_desc[i].it_id) out.push_back(s.nt + v);
    return PPN_OK;
  }

  ppn_status fallback_dir(const std::vector<char>& on, int kind) {
    G.set_active(on);
    ppn_status rc = G.upload_desc();
    if (rc) return rc;
    timed(FAM_VECTOR, 0, [&] { launch_fallback<T>(G.d_desc, G.d_vtiles, G.n_vtiles, kind, G.st); });
    return check_launch();
  }

  // energy at u + gamma dx for the flagged scenes; at_zero also records E0, g^T dx, max|dx|.
  // At gamma = 0 a scene whose current iterate came from an accepted line-search trial of
  // this time step already has its energy (the same displacement bits, the same kernel):
  // only g^T dx and max |dx| are reduced, over the vertices.
  ppn_status energy(const std::vector<char>& on, bool at_zero) {
    const int n = (int)on.size();
    std::vector<char> full(on), quick(n, 0);
    bool any_full = false, any_quick = false;
    const bool force_full = std::getenv("PPN_ENERGY_FULL") != nullptr;  // tests: always the full pass
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      if (at_zero) G.h_desc[i].gamma = 0.0;
      if (at_zero && H[i].has_next && !force_full) {
        full[i] = 0;
        quick[i] = 1;
        any_quick = true;
      } else {
        any_full = true;
      }
    }
    ppn_status rc = PPN_OK;
    if (any_full) {
      G.set_active(full);
      if ((rc = G.upload_desc())) return rc;
      timed(FAM_ENERGY, 0, [&] { launch_energy<T>(G.d_desc, G.d_etiles, G.n_etiles, 0, G.st); });
      if ((rc = check_launch())) return rc;
    }
    if (any_quick) {
      G.set_active(quick);
      if ((rc = G.upload_desc())) return rc;
      timed(FAM_ENERGY, 0, [&] { launch_dirderiv<T>(G.d_desc, G.d_vtiles, G.n_vtiles, G.st); });
      if ((rc = check_launch())) return rc;
    }
    if ((rc = G.sync_ctl())) return rc;
    if (at_zero)
      for (int i = 0; i < n; ++i)
        if (on[i]) {
          H[i].E0 = quick[i] ? H[i].E_next : G.h_ctl[i].energy[0];
          H[i].dd = G.h_ctl[i].energy[1];
          H[i].dxmax = G.h_ctl[i].energy[2];
        }
    return PPN_OK;
  }
};

// ------------------------------------------------------------------ group cache

// positions x = X + u into a host buffer
template <typename T>
__global__ void k_positions(const double4* X, const double4* u, double* xyz, int nv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double4 a = ld_d4(X + v), b = ld_d4(u + v);
  xyz[3 * v] = a.x + b.x;
  xyz[3 * v + 1] = a.y + b.y;
  xyz[3 * v + 2] = a.z + b.z;
}

template <typename T>
__global__ void k_vel_out(const double4* w, double* xyz, int nv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double4 a = ld_d4(w + v);
  xyz[3 * v] = a.x;
  xyz[3 * v + 1] = a.y;
  xyz[3 * v + 2] = a.z;
}

template <typename T>
inline ppn_status read_positions(SceneImpl<T>& s, double* out) {
  k_positions<T><<<(s.nv + 255) / 256, 256, 0, s.stream>>>(s.d.X, s.d.u, s.d_xyz, s.nv);
  PPN_CU(cudaGetLastError());
  PPN_CU(cudaMemcpyAsync(out, s.d_xyz, sizeof(double) * 3 * s.nv, cudaMemcpyDeviceToHost, s.stream));
  PPN_CU(cudaStreamSynchronize(s.stream));
  return PPN_OK;
}

}  // namespace ppn
