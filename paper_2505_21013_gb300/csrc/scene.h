// Host-side scene objects and the lockstep Newton / PN / PPN driver.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ppn.h"
#include "common.cuh"
#include "kernels.h"

namespace ppn {

void set_error(const std::string& msg);

// Device memory of a scene or a scene group: cudaMalloc / cudaFree, or the allocator a
// caller installed with ppn_set_allocator, captured by the owner at its creation.
struct DevAllocator {
  ppn_device_alloc_fn alloc = nullptr;
  ppn_device_free_fn free = nullptr;
  void* ctx = nullptr;
};
DevAllocator current_allocator();
inline void* dev_alloc(const DevAllocator& a, size_t bytes) {
  if (!a.alloc) {
    void* p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
  }
  void* p = a.alloc(bytes, a.ctx);
  if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {  // the alignment the kernels' vector loads rely on
    a.free(p, a.ctx);
    return nullptr;
  }
  return p;
}
inline void dev_free(const DevAllocator& a, void* p) {
  if (!p) return;
  if (a.free)
    a.free(p, a.ctx);
  else
    cudaFree(p);
}

// Pinned staging arena for small host->device uploads (descriptor tables,
// tile tables).  Slots are recycled after the owning stream has been synchronized.
struct Staging {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  ~Staging();
  void* take(size_t n, cudaStream_t st);
  void reset() { off = 0; }
};

struct KernelTimer {
  bool on = false;
  struct Rec {
    int fam;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[16] = {0};
  double ms[16] = {0};
  double bytes[16] = {0};
  ~KernelTimer();
  cudaEvent_t ev();
  void begin(int fam, cudaStream_t st, double b);
  void end(cudaStream_t st);
  void collect();  // after a stream sync
  void reset();
};

enum KernelFamily {
  FAM_ELEMENT = 0,
  FAM_GRADIENT,
  FAM_ASSEMBLE,
  FAM_SELECT,
  FAM_PROJECT,
  FAM_UPDATE,
  FAM_PCG,
  FAM_ENERGY,
  FAM_VECTOR,
  FAM_COUNT
};
extern const char* kFamilyNames[FAM_COUNT];

template <typename T>
struct SceneImpl {
  // sizes and parameters
  int nv = 0, nt = 0, nnzb = 0, nmap = 0, nfixed = 0;
  int n_vtiles = 0, n_ttiles = 0, n_btiles = 0, n_ptiles = 0;
  ppn_params params;
  double dt = 0;
  std::vector<double> rest;       // host copy of rest positions (nv x 3)
  std::vector<int> fixed_list;    // caller order
  std::vector<int64_t> h_row_ptr; // pattern (host copy for probes)
  std::vector<int> h_col;
  // device memory
  DevAllocator dalloc = current_allocator();
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  SceneDev<T> d{};                // host mirror of the device descriptor
  SceneDev<T>* d_desc = nullptr;  // device descriptor (single-scene launches)
  TileRef *d_ttiles = nullptr, *d_vtiles = nullptr, *d_btiles = nullptr, *d_ptiles = nullptr,
          *d_etiles = nullptr, *d_projtiles = nullptr;
  int* d_ids = nullptr;
  GridBar* d_bar = nullptr;
  int* d_fixed_list = nullptr;
  double* d_targets = nullptr;
  const double* ext_targets = nullptr;  // device targets given by the caller for the next step
  double* d_xyz = nullptr;              // nv x 3 output staging
  ObstSet* d_obs = nullptr;             // the scene's obstacles as applied (device)
  int n_obst = 0;                       // host copy of their count
  ObstSet obs_app{}, obs_req{};         // applied and requested poses (host)
  Ctl* h_ctl = nullptr;                 // pinned
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Staging staging;
  KernelTimer timer;
  int pcg_group = 8, pcg_grid = 0;
  int last_pcg_layout = -1;  // ppn_scene_info::pcg_layout
  // counters and per-step records
  int it_counter = 0, round_counter = 0;
  std::vector<ppn_iter_stats> iters;
  std::vector<ppn_attempt> attempts;
  bool record_sel = false;                    // keep the selected elements of every attempt
  std::vector<std::vector<int>> attempt_sel;  // (ppn_set_record_selection)
  std::vector<std::vector<double>> iter_g;    // assembled gradient of every Newton iteration (same switch)
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;

  ~SceneImpl();
  ppn_status init(const double* rest_xyz, int64_t n_verts, const int32_t* tets, int64_t n_tets,
                  const ppn_material* mat, double dt, const int32_t* fixed, int64_t n_fixed,
                  const ppn_params* p);
  template <typename X>
  X* alloc(size_t n);
};

struct SceneBase;

}  // namespace ppn

struct ppn_scene {
  int precision = PPN_PREC_MIXED;
  std::unique_ptr<ppn::SceneImpl<float>> f;
  std::unique_ptr<ppn::SceneImpl<double>> d;
};
