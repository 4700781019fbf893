// ppn_pcg_solve_static: the block-Jacobi PCG of the Newton solve (SolveSPD of
// Algorithm 1; Sec. 4.1 "Linear Solvers"; Sec. 5.1) on a caller's
// device-resident FP32 BSR system, with every scratch buffer taken from one
// fixed-size array in device global memory instead of allocated per call.
//
// Who needs it.  A caller that runs under a fixed device-memory budget, such as
// a serving loop that admitted its scenes against the free HBM, must not
// allocate per request. cudaMalloc can fail once the budget is spent, and
// cudaFree synchronises the whole device and stalls the other requests in
// flight.  Such a caller solves from this pre-reserved arena instead of
// creating a scene (which allocates its buffers once, at creation).
//
// Scratch.  `g_pcg_static` holds the solver descriptor, the status words, the
// grid barrier, the tile table, the diagonal-block index and the PCG vectors
// for at most PPN_PCG_STATIC_MAX_ROWS block rows (the layout is carved per
// call from the row count).  Its device address is looked up once per device
// context, at the first call in it, and cached with the context's id: a call
// after cudaDeviceReset (a new primary context, in which the array may sit
// elsewhere) looks it up again.  Larger systems are rejected with
// PPN_ERR_INVALID_ARG.
//
// Start values.  The barrier counter and the status word must be zero when the
// solve starts; every call clears them with cudaMemsetAsync.  Every other
// scratch buffer is written before it is read within a call (the tile table
// and diagonal index by the preparation kernel, r from b, z / d / P^-1 / x in
// the solver's set-up).
//
// Concurrency.  There is one arena per device, so two calls on the same device
// must not overlap: a process-wide lock serialises the host threads, and the
// call waits for its stream before returning.  Separate processes have
// separate arenas.
//
// The solver is the global-memory cooperative kernel of pcg.cu (group of four
// lanes per row), so the arithmetic is the one a scene's solve performs with
// that kernel.  Nothing here changes the scene path.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "kernels.h"
#include "scene.h"

namespace ppn {

namespace {

constexpr int kMaxRows = PPN_PCG_STATIC_MAX_ROWS;
constexpr int kMaxTiles = (kMaxRows + PCG_TILE - 1) / PCG_TILE;
constexpr int kMaxDevices = 64;
constexpr int kErrPattern = 4;  // Ctl::error bit: the caller's BSR pattern is malformed

constexpr size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// bytes of the carved layout for n rows / t tiles (see Arena)
constexpr size_t arena_bytes(size_t n, size_t t) {
  return up256(sizeof(SceneDev<float>)) + up256(sizeof(Ctl)) + up256(sizeof(GridBar)) + up256(sizeof(int)) +
         up256(sizeof(TileRef) * t) + up256(sizeof(int) * n) + 5 * up256(sizeof(float4) * n) +
         up256(sizeof(float) * 9 * n) + up256(sizeof(double) * 4 * t);
}
constexpr size_t kArenaBytes = arena_bytes(kMaxRows, kMaxTiles);

static __device__ __align__(256) unsigned char g_pcg_static[kArenaBytes];

struct Arena {
  SceneDev<float>* desc;
  Ctl* ctl;
  GridBar* bar;
  int* scene_id;
  TileRef* tiles;
  int* diag;
  float4 *r, *z, *q, *d0, *d1;
  float* Pinv;
  double* ppart;
};

Arena carve(unsigned char* base, int n, int t) {
  Arena a;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += up256(bytes);
    return p;
  };
  a.desc = (SceneDev<float>*)take(sizeof(SceneDev<float>));
  a.ctl = (Ctl*)take(sizeof(Ctl));
  a.bar = (GridBar*)take(sizeof(GridBar));
  a.scene_id = (int*)take(sizeof(int));
  a.tiles = (TileRef*)take(sizeof(TileRef) * t);
  a.diag = (int*)take(sizeof(int) * n);
  a.r = (float4*)take(sizeof(float4) * n);
  a.z = (float4*)take(sizeof(float4) * n);
  a.q = (float4*)take(sizeof(float4) * n);
  a.d0 = (float4*)take(sizeof(float4) * n);
  a.d1 = (float4*)take(sizeof(float4) * n);
  a.Pinv = (float*)take(sizeof(float) * 9 * n);
  a.ppart = (double*)take(sizeof(double) * 4 * t);
  return a;
}

struct DeviceSetup {
  unsigned char* base = nullptr;  // device address of g_pcg_static
  int grid = 0;                   // co-resident CTAs of the solver
  unsigned long long ctx = 0;     // id of the context the address belongs to (0: unknown)
};
std::mutex g_lock;
DeviceSetup g_dev[kMaxDevices];

// id of the calling thread's current context, through the driver's entry points
// (found once; 0 when the driver does not offer them, then the first lookup is kept)
unsigned long long current_context_id() {
  using GetCur = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  static bool looked = false;
  if (!looked) {  // (under g_lock)
    looked = true;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess) {
      get_cur = nullptr;
      get_id = nullptr;
      cudaGetLastError();
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Tile table and diagonal index, with a check of the caller's pattern: row
// pointers non-decreasing from 0 to nnzb, columns in range, one diagonal block
// per row.  A bad pattern sets ctl->error (nothing out of range is read).
__global__ void k_static_prep(const int* __restrict__ row_ptr, const int* __restrict__ col, int n, int nnzb,
                              int* __restrict__ diag, TileRef* __restrict__ tiles, int n_tiles, Ctl* ctl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_tiles) tiles[i] = TileRef{0, i};
  if (i >= n) return;
  const int kb = row_ptr[i], ke = row_ptr[i + 1];
  bool bad = kb < 0 || ke < kb || ke > nnzb || (i == 0 && kb != 0) || (i == n - 1 && ke != nnzb);
  int d = -1, n_diag = 0;
  if (!bad)
    for (int k = kb; k < ke; ++k) {
      const int j = col[k];
      if (j < 0 || j >= n) bad = true;
      if (j == i) {
        d = k;
        ++n_diag;
      }
    }
  diag[i] = bad ? 0 : d;
  // exactly one diagonal block: with two, the preconditioner would invert one of them
  // while the SpMV sums both
  if (bad || n_diag != 1) atomicOr(&ctl->error, kErrPattern);
}

ppn_status fail(ppn_status rc, const std::string& msg) {
  set_error(msg);
  return rc;
}

}  // namespace

}  // namespace ppn

using namespace ppn;

extern "C" {

PPN_API ppn_status ppn_pcg_solve_static(const int32_t* row_ptr, const int32_t* col, const float* val,
                                        int32_t n_rows, int32_t nnzb, const float* b, float* x, double rel_tol,
                                        int32_t max_iter, int32_t* info, void* stream) {
  if (!row_ptr || !col || !val || !b || !x)
    return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: null pointer argument");
  if (n_rows <= 0 || nnzb < n_rows)
    return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: need n_rows >= 1 and nnzb >= n_rows");
  if (n_rows > kMaxRows)
    return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: " + std::to_string(n_rows) +
                                         " block rows exceed the static scratch limit of " +
                                         std::to_string(kMaxRows) + " (solve larger systems through a scene)");
  if (!(rel_tol >= 0.0)) return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: rel_tol must be >= 0");
  const cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> guard(g_lock);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(PPN_ERR_CUDA, "ppn_pcg_solve_static: no usable current device");
  if (st) {  // the arena and the occupancy are those of the current device: the stream must be on it
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: the stream is not a valid stream");
    }
    if (sdev != dev)
      return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: the stream belongs to device " + std::to_string(sdev) +
                                           ", the current device is " + std::to_string(dev));
  }
  DeviceSetup& D = g_dev[dev];
  const unsigned long long ctx = current_context_id();
  if (!D.base || (ctx && ctx != D.ctx)) {  // first call in this context: symbol address and solver occupancy
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_static);
    if (e != cudaSuccess || !p)
      return fail(PPN_ERR_CUDA, std::string("ppn_pcg_solve_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const int grid = pcg_max_grid(4, dev);
    if (grid <= 0) return fail(PPN_ERR_CUDA, "ppn_pcg_solve_static: solver occupancy query failed");
    D.grid = grid;
    D.base = (unsigned char*)p;
    D.ctx = ctx;
  }
  const int n_tiles = (n_rows + PCG_TILE - 1) / PCG_TILE;
  const Arena A = carve(D.base, n_rows, n_tiles);

#define PPN_STATIC_CU(expr)                                                                          \
  do {                                                                                               \
    const cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                           \
      return fail(PPN_ERR_CUDA, std::string("ppn_pcg_solve_static: ") + #expr + ": " + cudaGetErrorString(e_)); \
  } while (0)

  PPN_STATIC_CU(cudaMemsetAsync(A.ctl, 0, sizeof(Ctl), st));
  PPN_STATIC_CU(cudaMemsetAsync(A.scene_id, 0, sizeof(int), st));
  const int nb = (std::max(n_rows, n_tiles) + 255) / 256;
  k_static_prep<<<nb, 256, 0, st>>>(row_ptr, col, n_rows, nnzb, A.diag, A.tiles, n_tiles, A.ctl);
  PPN_STATIC_CU(cudaGetLastError());
  Ctl c{};
  PPN_STATIC_CU(cudaMemcpyAsync(&c, A.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  PPN_STATIC_CU(cudaStreamSynchronize(st));
  if (c.error) return fail(PPN_ERR_INVALID_ARG, "ppn_pcg_solve_static: malformed BSR pattern "
                                                "(row pointers, column range or a missing diagonal block)");

  SceneDev<float> s{};
  s.nv = n_rows;
  s.nnzb = nnzb;
  s.n_ptiles = n_tiles;
  s.row_ptr = row_ptr;
  s.col = col;
  s.diag_idx = A.diag;
  s.val = const_cast<float*>(val);  // read only by the solver
  s.dx = reinterpret_cast<float4*>(x);
  s.r = A.r;
  s.z = A.z;
  s.q = A.q;
  s.d0 = A.d0;
  s.d1 = A.d1;
  s.Pinv = A.Pinv;
  s.ppart = A.ppart;
  s.ctl = A.ctl;
  s.pcg_tol2 = rel_tol * rel_tol;
  s.pcg_max_iter = max_iter > 0 ? max_iter : std::max(1000, 3 * n_rows);
  s.active = 1;
  PPN_STATIC_CU(cudaMemcpyAsync(A.desc, &s, sizeof(s), cudaMemcpyHostToDevice, st));
  PPN_STATIC_CU(cudaMemcpyAsync(A.r, b, sizeof(float4) * n_rows, cudaMemcpyDeviceToDevice, st));

  PcgLaunch L{};
  L.n_tiles = n_tiles;
  L.tiles = A.tiles;
  L.n_scenes = 1;
  L.scene_ids = A.scene_id;
  L.bar = A.bar;
  L.grid = std::min(D.grid, n_tiles);
  L.group = 4;
  L.use_b_from_g = 0;
  PPN_STATIC_CU(launch_pcg<float>(A.desc, L, st));
  GridBar bar{};
  PPN_STATIC_CU(cudaMemcpyAsync(&c, A.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  PPN_STATIC_CU(cudaMemcpyAsync(&bar, A.bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
  PPN_STATIC_CU(cudaStreamSynchronize(st));
#undef PPN_STATIC_CU
  if (bar.timeout) return fail(PPN_ERR_TIMEOUT, "ppn_pcg_solve_static: a grid-wide wait ran out");
  if (c.error & kErrNonFinite) return fail(PPN_ERR_NONFINITE, "ppn_pcg_solve_static: non-finite value in the solve");
  if (info) {
    info[0] = c.pcg_iters;
    info[1] = c.pcg_ind;
    info[2] = c.pcg_precond_fail;
    info[3] = c.pcg_hit_max;
  }
  return PPN_OK;
}

}  // extern "C"
