// Serving loop: time-step requests over resident scenes with continuous
// (iteration-level) batching.
//
// A worker thread owns the GPU work.  Its batch is a Group of up to max_batch
// scenes; every Newton iteration of the batch is one Driver::tick (one launch
// per phase over all scenes still iterating).  At each iteration boundary:
//   1. scenes whose time step ended leave the batch: velocities, positions
//      read back, the request completed;
//   2. queued requests join in the free slots, oldest first, one request per
//      scene at a time (a scene's requests run in submission order);
//   3. if the members changed, the group's tables are rebuilt in place;
//   4. joining scenes start their step (predictor, targets, delta = infinity);
//   5. one tick.
// A scene's arithmetic is the same in any batch: every kernel treats scenes
// independently and every reduction is per scene and in a fixed order.
//
// Admission: a scene is added only when the device memory of all resident
// scenes stays within hbm_fraction of the device's memory.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "driver.h"

namespace ppn {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int scene = -1;
  int mode = PPN_MODE_PPN;
  double tol = 0.0;
  std::vector<double> targets;  // empty: keep the scene's targets
  Clock::time_point t_submit, t_start, t_done;
  int batch_max = 0;
  bool started = false, done = false;
  ppn_status status = PPN_OK;
  ppn_step_stats stats{};
  std::vector<double> x;  // positions at the end of the step
};

struct Served {
  int id = -1;
  ppn_scene* h = nullptr;
  size_t bytes = 0;
  int pending = 0;        // submitted, not yet completed
  bool in_group = false;  // referenced by the worker's group tables
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace
}  // namespace ppn

using namespace ppn;

struct ppn_server {
  ppn_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0, resident = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int, std::unique_ptr<Served>> scenes;
  std::map<int64_t, std::unique_ptr<Request>> requests;
  std::deque<int64_t> fifo;  // submitted, not yet started
  int next_scene = 0;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  Clock::time_point t0, first_submit, last_done;
  bool any_submit = false;
  std::vector<double> latencies;
  int64_t submitted = 0, completed = 0, rejected = 0;
};

namespace ppn {
namespace {

template <typename T>
SceneImpl<T>* impl(ppn_scene* h);
template <>
SceneImpl<float>* impl<float>(ppn_scene* h) {
  return h->f.get();
}
template <>
SceneImpl<double>* impl<double>(ppn_scene* h) {
  return h->d.get();
}

// one slot of the running batch
template <typename T>
struct Slot {
  int scene = -1;
  SceneImpl<T>* sc = nullptr;  // stays valid: a scene with pending requests is not removed
  Request* req = nullptr;
  HostState h;
};

template <typename T>
void complete(ppn_server* S, Slot<T>& sl, ppn_status st) {
  Request* r = sl.req;
  r->status = st;
  r->stats = sl.h.tot;
  r->stats.status = st;
  r->t_done = Clock::now();
  r->stats.device_ms = ms_between(r->t_start, r->t_done);
  r->done = true;
  Served& sc = *S->scenes.at(sl.scene);
  sc.pending -= 1;
  S->completed += 1;
  S->latencies.push_back(ms_between(r->t_submit, r->t_done));
  S->last_done = r->t_done;
}

template <typename T>
void serve(ppn_server* S) {
  cudaSetDevice(S->device);
  Group<T> G;
  std::vector<Slot<T>> slots;  // group order
  for (;;) {
    std::vector<Slot<T>> joining;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !slots.empty() || !S->fifo.empty(); });
      if (slots.empty() && S->fifo.empty()) break;  // stop requested and nothing left
      // admit queued requests into free slots, oldest first, one per scene
      std::vector<int> busy;
      for (const Slot<T>& s : slots) busy.push_back(s.scene);
      for (auto it = S->fifo.begin(); it != S->fifo.end() && (int)(slots.size() + joining.size()) < S->cfg.max_batch;) {
        Request* r = S->requests.at(*it).get();
        if (std::find(busy.begin(), busy.end(), r->scene) != busy.end()) {
          ++it;
          continue;
        }
        busy.push_back(r->scene);
        Slot<T> s;
        s.scene = r->scene;
        s.sc = impl<T>(S->scenes.at(r->scene)->h);
        s.req = r;
        s.h.mode = r->mode;
        s.h.tol = r->tol;
        r->started = true;
        r->t_start = Clock::now();
        joining.push_back(s);
        it = S->fifo.erase(it);
      }
    }
    ppn_status rc = PPN_OK;
    const size_t n_old = slots.size();
    for (Slot<T>& s : joining) slots.push_back(std::move(s));
    if (slots.empty()) continue;
    // rebuild the group when its members changed
    bool changed = G.S.size() != slots.size();
    for (size_t i = 0; !changed && i < slots.size(); ++i)
      changed = G.S[i] != slots[i].sc;
    if (changed) {
      G.stash();
      std::vector<SceneImpl<T>*> members;
      for (const Slot<T>& s : slots) members.push_back(s.sc);
      rc = G.build(members);
      // a scene stays unremovable while the group tables reference it
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& kv : S->scenes) kv.second->in_group = false;
      for (const Slot<T>& s : slots) S->scenes.at(s.scene)->in_group = true;
    }
    Driver<T> D(G);
    D.H.resize(slots.size());
    for (size_t i = 0; i < slots.size(); ++i) D.H[i] = slots[i].h;
    if (rc == PPN_OK && slots.size() > n_old) {
      // requests' targets, then the start of their time steps
      std::vector<char> on(slots.size(), 0);
      for (size_t i = n_old; i < slots.size() && rc == PPN_OK; ++i) {
        on[i] = 1;
        SceneImpl<T>& sc = *G.S[i];
        const std::vector<double>& tg = slots[i].req->targets;
        if (!tg.empty() && sc.nfixed > 0) {
          if (cudaMemcpyAsync(sc.d_targets, tg.data(), sizeof(double) * tg.size(), cudaMemcpyHostToDevice,
                              sc.stream) != cudaSuccess) {
            set_error("target upload failed");
            rc = PPN_ERR_CUDA;
          }
          sc.ext_targets = nullptr;
        }
      }
      if (rc == PPN_OK) rc = D.begin(on);
    }
    if (rc == PPN_OK) rc = D.tick();
    // scenes whose step ended leave the batch
    std::vector<char> fin(slots.size(), 0);
    bool any_fin = false;
    for (size_t i = 0; i < slots.size(); ++i)
      if (rc != PPN_OK || !D.H[i].running) {
        fin[i] = 1;
        any_fin = true;
      }
    ppn_status rc_fin = PPN_OK;
    if (any_fin && rc == PPN_OK) {
      rc_fin = D.finish(fin);
      if (rc_fin == PPN_OK && cudaStreamSynchronize(G.st) != cudaSuccess) rc_fin = PPN_ERR_CUDA;
      G.staging.reset();
      for (size_t i = 0; i < slots.size() && rc_fin == PPN_OK; ++i)
        if (fin[i]) {
          Request* r = slots[i].req;
          r->x.resize((size_t)3 * G.S[i]->nv);
          rc_fin = read_positions(*G.S[i], r->x.data());
        }
    }
    for (size_t i = 0; i < slots.size(); ++i) slots[i].h = D.H[i];
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (Slot<T>& s : slots) s.req->batch_max = std::max(s.req->batch_max, (int)slots.size());
      std::vector<Slot<T>> keep;
      for (size_t i = 0; i < slots.size(); ++i) {
        if (!fin[i]) {
          keep.push_back(std::move(slots[i]));
          continue;
        }
        const ppn_status st = rc != PPN_OK ? rc : rc_fin != PPN_OK ? rc_fin : (ppn_status)slots[i].h.status;
        complete<T>(S, slots[i], st);
      }
      slots = std::move(keep);
      if (slots.empty()) {  // drop the references to finished scenes
        G.stash();
        G.S.clear();
        G.h_desc.clear();
        for (auto& kv : S->scenes) kv.second->in_group = false;
      }
    }
    S->cv_done.notify_all();
  }
}

ppn_status fail(ppn_status rc, const std::string& m) {
  set_error(m);
  return rc;
}

}  // namespace
}  // namespace ppn

extern "C" {

ppn_server_config ppn_server_default_config(void) {
  ppn_server_config c;
  c.hbm_fraction = 0.8;
  c.max_batch = 64;
  c.precision = PPN_PREC_MIXED;
  return c;
}

ppn_status ppn_server_create(const ppn_server_config* cfg, ppn_server** out) {
  if (!out) return fail(PPN_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  const ppn_server_config c = cfg ? *cfg : ppn_server_default_config();
  if (!(c.hbm_fraction > 0 && c.hbm_fraction <= 1) || c.max_batch < 1 || c.max_batch > PCG_MAX_SCENES ||
      (c.precision != PPN_PREC_FP64 && c.precision != PPN_PREC_MIXED))
    return fail(PPN_ERR_INVALID_ARG, "server config: hbm_fraction in (0,1], 1 <= max_batch <= 64, valid precision");
  auto S = std::make_unique<ppn_server>();
  S->cfg = c;
  if (cudaGetDevice(&S->device) != cudaSuccess) return fail(PPN_ERR_CUDA, "no current CUDA device");
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(PPN_ERR_CUDA, "cudaMemGetInfo failed");
  S->budget = (size_t)(c.hbm_fraction * (double)total_b);
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(PPN_ERR_CUDA, "stream creation failed");
  S->t0 = Clock::now();
  ppn_server* raw = S.get();
  if (c.precision == PPN_PREC_FP64)
    S->worker = std::thread([raw] { serve<double>(raw); });
  else
    S->worker = std::thread([raw] { serve<float>(raw); });
  *out = S.release();
  return PPN_OK;
}

void ppn_server_destroy(ppn_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& kv : S->scenes) ppn_destroy_scene(kv.second->h);
  S->scenes.clear();
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

ppn_status ppn_server_add_scene(ppn_server* S, const double* rest_xyz, int64_t n_verts, const int32_t* tets,
                                int64_t n_tets, const ppn_material* mat, double dt, const int32_t* fixed,
                                int64_t n_fixed, const ppn_params* params, int32_t* scene_id) {
  if (!S || !scene_id) return fail(PPN_ERR_INVALID_ARG, "null server or output");
  ppn_params p = params ? *params : ppn_default_params();
  if (p.precision != S->cfg.precision) return fail(PPN_ERR_INVALID_ARG, "scene precision differs from the server's");
  // the element store alone is a lower bound of a scene's footprint
  const size_t fs = S->cfg.precision == PPN_PREC_FP64 ? 8 : 4;
  const size_t lower = (size_t)n_tets * (2 * HE_STRIDE * fs + GE_STRIDE * sizeof(double));
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->resident + lower > S->budget) {
      S->rejected += 1;
      return fail(PPN_ERR_ADMISSION, "scene does not fit the server's HBM budget");
    }
  }
  ppn_scene* h = nullptr;
  ppn_status rc = ppn_create_scene(rest_xyz, n_verts, tets, n_tets, mat, dt, fixed, n_fixed, &p, &h);
  if (rc) return rc;
  if ((rc = ppn_set_stream(h, S->stream))) {
    ppn_destroy_scene(h);
    return rc;
  }
  const size_t bytes = h->f ? h->f->dev_bytes : h->d->dev_bytes;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->resident + bytes > S->budget) {
    S->rejected += 1;
    ppn_destroy_scene(h);
    return fail(PPN_ERR_ADMISSION, "scene does not fit the server's HBM budget");
  }
  auto sc = std::make_unique<Served>();
  sc->id = S->next_scene++;
  sc->h = h;
  sc->bytes = bytes;
  S->resident += bytes;
  *scene_id = sc->id;
  S->scenes.emplace(sc->id, std::move(sc));
  return PPN_OK;
}

ppn_status ppn_server_remove_scene(ppn_server* S, int32_t id) {
  if (!S) return fail(PPN_ERR_INVALID_ARG, "null server");
  ppn_scene* h = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->scenes.find(id);
    if (it == S->scenes.end()) return fail(PPN_ERR_INVALID_ARG, "unknown scene id");
    if (it->second->pending > 0 || it->second->in_group)
      return fail(PPN_ERR_INVALID_ARG, "scene has unfinished requests");
    h = it->second->h;
    S->resident -= it->second->bytes;
    S->scenes.erase(it);
  }
  ppn_destroy_scene(h);
  return PPN_OK;
}

ppn_status ppn_server_submit(ppn_server* S, int32_t id, ppn_mode mode, double tol, const double* targets,
                             int64_t* ticket) {
  if (!S || !ticket) return fail(PPN_ERR_INVALID_ARG, "null server or output");
  if (mode < PPN_MODE_NEWTON || mode > PPN_MODE_PDN || !(tol >= 0))
    return fail(PPN_ERR_INVALID_ARG, "invalid mode or tolerance");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(PPN_ERR_INVALID_ARG, "server is stopping");
    auto it = S->scenes.find(id);
    if (it == S->scenes.end()) return fail(PPN_ERR_INVALID_ARG, "unknown scene id");
    auto r = std::make_unique<Request>();
    r->ticket = S->next_ticket++;
    r->scene = id;
    r->mode = mode;
    r->tol = tol;
    const int nfix = it->second->h->f ? it->second->h->f->nfixed : it->second->h->d->nfixed;
    if (targets && nfix > 0) r->targets.assign(targets, targets + 3 * (size_t)nfix);
    r->t_submit = Clock::now();
    if (!S->any_submit) {
      S->first_submit = r->t_submit;
      S->any_submit = true;
    }
    it->second->pending += 1;
    S->submitted += 1;
    *ticket = r->ticket;
    S->fifo.push_back(r->ticket);
    S->requests.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return PPN_OK;
}

ppn_status ppn_server_poll(ppn_server* S, int64_t ticket, int wait, int* done, double* out_xyz,
                           ppn_step_stats* stats, ppn_request_times* times) {
  if (!S || !done) return fail(PPN_ERR_INVALID_ARG, "null server or output");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->requests.find(ticket);
  if (it == S->requests.end()) return fail(PPN_ERR_INVALID_ARG, "unknown or released ticket");
  Request* r = it->second.get();
  if (wait) S->cv_done.wait(lk, [&] { return r->done; });
  *done = r->done ? 1 : 0;
  if (!r->done) return PPN_OK;
  if (out_xyz && !r->x.empty()) std::copy(r->x.begin(), r->x.end(), out_xyz);
  if (stats) *stats = r->stats;
  if (times) {
    times->t_submit_ms = ms_between(S->t0, r->t_submit);
    times->t_start_ms = ms_between(S->t0, r->t_start);
    times->t_done_ms = ms_between(S->t0, r->t_done);
    times->batch_max = r->batch_max;
  }
  const ppn_status st = r->status;
  S->requests.erase(it);
  if (st != PPN_OK) set_error("request failed: " + std::string(ppn_status_string(st)));
  return st;
}

ppn_status ppn_server_get_stats(ppn_server* S, ppn_server_stats* out) {
  if (!S || !out) return fail(PPN_ERR_INVALID_ARG, "null server or output");
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->rejected_scenes = S->rejected;
  out->resident_scenes = (int)S->scenes.size();
  out->resident_bytes = (double)S->resident;
  out->budget_bytes = (double)S->budget;
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const double k = q * (double)(l.size() - 1);
    const size_t f = (size_t)k, c = std::min(l.size() - 1, f + 1);
    return l[f] + (l[c] - l[f]) * (k - (double)f);
  };
  out->p50_ms = pct(0.5);
  out->p99_ms = pct(0.99);
  const double span = S->completed > 0 ? ms_between(S->first_submit, S->last_done) : 0.0;
  out->steps_per_s = span > 0 ? 1e3 * (double)S->completed / span : 0.0;
  return PPN_OK;
}

}  // extern "C"
