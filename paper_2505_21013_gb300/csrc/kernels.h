// Host-side launch interface of the device kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace ppn {

constexpr int PROJ_CTA = 128;  // threads per CTA of the projection kernel (register heavy)
constexpr int PROJW_CTA = 128;  // threads per CTA of its warp form: 4 warps of 3 tets
constexpr int PROJW_TETS = 3 * PROJW_CTA / 32;  // tets per CTA of the warp form

template <typename T> void launch_element(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);
template <typename T> void launch_gradient(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);
// FP32: the warp form over n_btiles BSR-block tiles; FP64: the element-order form, off-diagonal
// blocks over the block tiles and diagonal blocks over n_vtiles vertex tiles
template <typename T>
void launch_assemble(const SceneDev<T>*, const TileRef* btiles, int n_btiles, const TileRef* vtiles, int n_vtiles,
                     cudaStream_t, int use_probe = 0);
template <typename T> void launch_update(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
// touched-block form: n tiles of TILE (selected element, corner pair) entries per scene
// (16 x the selection's count); the scene's ctl->n_touched must be zero before the launch
template <typename T> void launch_update_touched(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_select(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
// warp != 0: the warp form (tiles of PROJW_TETS selected tets), else one thread per tet (tiles of PROJ_CTA)
template <typename T> void launch_project(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t, int warp);
// the projection form for a selection round (true) or a pass over every element (false),
// unless PPN_PROJECT_THREAD=1 or PPN_PROJECT_WARP=1 fixes it
bool project_warp_form(bool selection_round);
template <typename T> void launch_energy(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);
template <typename T> void launch_predict(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
// g^T dx and max |dx| over the free vertices (vertex tiles) into ctl->energy[1], [2]
template <typename T> void launch_dirderiv(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
// contact elements (vertex tiles): selection + clamping, in-place update, first contact time
template <typename T> void launch_select_contact(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_update_contact(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_ccd(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
// smallest free-vertex distance to obstacles k0..k0+3 (ctl->gap)
template <typename T> void launch_obst_gap(const SceneDev<T>*, const TileRef*, int, int k0, cudaStream_t);
template <typename T>
void launch_apply_targets(const SceneDev<T>*, int, const int*, const double*, int, int, cudaStream_t);
template <typename T> void launch_gmax(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_axpy_u(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_velocity(const SceneDev<T>*, const TileRef*, int, cudaStream_t);
template <typename T> void launch_fallback(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);

// Grid barrier state of the cooperative PCG kernel (zeroed before each launch).
struct GridBar {
  unsigned count;      // arrivals, monotonic within a launch
  int timeout;
  unsigned to_iter;    // first timeout: the CG iteration and the wait that ran out
  int to_site;         // (1 neighbour flags, 2 reduction words, 3 halo w words, 4 progress flags; 0 not recorded)
  unsigned to_seen;    // the stamp the wait last saw, on the word it waited for
  int to_slot;         // that word's scene slot and tile (site 2) or row (site 3)
  int to_index;
  int to_cta;
};

constexpr int PCG_MAX_SCENES = 64;      // scenes per PCG launch (per-CTA scalar state in shared memory)
constexpr int XCH_MAX_CTAS_HOST = 1024;  // CTAs of one resident PCG launch
constexpr int HALO_MAX_SCENES = 8;       // scenes per launch of the halo layout (SR_HALO)
constexpr int HALO_ROW_BITS = 26;        // halo reference: slot << HALO_ROW_BITS | row

struct PcgLaunch {
  int n_tiles;           // PCG row tiles in the launch's tile table (TileRef.scene = slot)
  const TileRef* tiles;  // device, grouped by slot, slot-major and tile-ascending
  int n_scenes;          // slots taking part (<= PCG_MAX_SCENES)
  const int* scene_ids;  // device: slot -> index into the scene table
  GridBar* bar;
  int grid;              // cooperative grid size (CTAs)
  int group;             // lanes per BSR row (4 or 8)
  int use_b_from_g;      // 1: b = -g of the scene; 0: b given in r (probe)
  size_t smem_bytes;     // > 0: shared-memory-resident kernel with this dynamic size
  int smem_blocks;       // block capacity of that layout (max blocks of one CTA; k_pcg_sr: max slots)
  int sr_mode;           // single-reduction kernel: SR_RES, SR_STREAM, SR_GLOBAL or SR_HALO
  int l2_keep;           // SR_STREAM, SR_GLOBAL: 0 streamed blocks evict-first in L2, 1 at normal priority
  // SR_HALO tables, device (built by the host for this tile table and grid):
  //   halo_off[2 b], halo_off[2 b + 1]: first block and first halo row of CTA b (b <= grid)
  //   halo_col[k]: local column of the launch's k-th block (CTA order, rows ascending):
  //                own row item, or n_items + the column's index in the CTA's halo list
  //   halo_ref[h]: halo rows, slot << HALO_ROW_BITS | row, ascending per CTA
  const int* halo_off;
  const int* halo_col;
  const int* halo_ref;
  int halo_cap;          // most halo rows of one CTA
  void* zrec[HALO_MAX_SCENES];  // SR_HALO: exchange records of the slots (zeroed before the launch)
  size_t zrec_bytes[HALO_MAX_SCENES];
  unsigned launch_seq;
  unsigned long long* flags;  // single-reduction kernel: per-CTA publication and progress flags (grid words)
  int n_pword;           // stamped partial arrays to clear before the launch
  void* pword[PCG_MAX_SCENES];
  size_t pword_bytes[PCG_MAX_SCENES];
};

// dynamic shared memory of the resident PCG layout for ni rows and nb blocks
size_t pcg_smem_bytes(int ni, int nb, int fsize);
// co-resident grid of the resident PCG kernel with `smem` dynamic bytes (0: does not fit)
int pcg_smem_max_grid(int group, int device, size_t smem, int fsize);
// single-reduction FP32 PCG (pcg_sr.cu).  Layouts: BSR blocks and vectors in
// shared memory (SR_RES); vectors in shared memory, blocks streamed (SR_STREAM);
// both in global memory (SR_GLOBAL); as SR_RES plus a replicated halo, which
// removes the neighbour exchange (SR_HALO).  Shared memory for ni rows / nb
// blocks / nh halo rows, co-resident grid, launch.
constexpr int SR_RES = 0, SR_STREAM = 1, SR_GLOBAL = 2, SR_HALO = 3;
// SR_HALO keeps each row's CG state in the registers of one thread: a CTA holds at
// most one SpMV pass of rows (512 threads, two lanes per row)
constexpr int SR_HALO_MAX_ROWS = 256;
size_t pcg_sr_smem_bytes(int ni, int nb, int nh, int mode);
int pcg_sr_max_grid(int device, size_t smem, int mode);
cudaError_t launch_pcg_sr(const SceneDev<float>* scenes, const PcgLaunch& L, cudaStream_t st);
// one warp waits (at most `limit` polling rounds) for n stamped words to reach `stamp`; *out = 1 if it ran out
cudaError_t launch_wait_probe(const unsigned long long* w, int n, unsigned long long stamp, unsigned limit, int* out,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_pcg_smem(const SceneDev<T>* scenes, const PcgLaunch& L, cudaStream_t st);

// Occupancy-limited cooperative grid size for the chosen row group width.
int pcg_max_grid(int group, int device);

template <typename T>
cudaError_t launch_pcg(const SceneDev<T>* scenes, const PcgLaunch& L, cudaStream_t st);

}  // namespace ppn
