// The serving loop of the C ABI (tomo_server_*): a stream of slope frames
// from several telescopes, each frame one warm-started solve of its
// telescope's plan (Sec. 5.1), batched on arrival.
//
// Threads: the caller's (admit, release, submit, poll), a worker that forms
// and enqueues launches, and a completion thread that waits for them.  One
// mutex guards the server state; device work is enqueued without it.  A
// launch is registered as in flight before the worker drops the lock, so an
// admission or a release (which waits until nothing is in flight, with the
// worker paused) never changes the batch or a telescope under a launch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tomo.h"
#include "plan_internal.h"

namespace {

using tomo::set_error;

constexpr int kMaxInFlight = 4;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Waiting {
  long long tag;
  double t_submit;
  int in_slot;
};

struct Telescope {
  int id = -1;
  tomo_plan *plan = nullptr;
  size_t n = 0, ns = 0, esz = 4;
  void *d_slopes = nullptr, *d_x = nullptr;   // the device slot
  char *h_in = nullptr;                       // pinned: queue_depth frames of slopes
  char *h_out = nullptr;                      // pinned: result_slots coefficient vectors
  std::vector<long long> out_tag;             // frame held by each result slot (-1: none)
  std::vector<char> out_writing;              // a launch is copying into the slot
  std::vector<int> free_in;
  std::list<Waiting> queue;
  int next_out = 0;
  bool busy = false;                          // a frame of this telescope is in flight
  size_t bytes = 0;                           // device bytes (plan + slot)
  // closed loop (Algorithm 4.1): the fit, the gain, two alternating command
  // buffers (a_t overwrites a_{t-2}), the reconstructed commands R s_ol and
  // the number of frames processed so far
  tomo_fit *fit = nullptr;
  double gain = 0.0;
  int fit_iters = 0;
  void *d_a[2] = {nullptr, nullptr}, *d_rec = nullptr;
  long long steps = 0;
  size_t n_out = 0;                           // elements of a result: coefficients, or commands
};

struct Launch {
  struct Frame {
    int tel;
    long long tag;
    double t_submit;
    int in_slot, out_slot;
  };
  int slot = -1;                              // stream, mask and event index
  bool enqueued = false;
  int status = TOMO_OK;
  double t_launch = 0.0;
  std::vector<Frame> frames;
};

}  // namespace

struct tomo_server {
  int device = 0;
  size_t budget = 0;
  int iters = 10, max_in_flight = 2, queue_depth = 8, result_slots = 4;

  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_idle;
  std::mutex admin_mu;                        // one admission or release at a time

  std::map<int, Telescope *> tels;            // batch order = id order
  int next_id = 0;
  tomo::Batch *batch = nullptr;
  size_t batch_bytes = 0;
  std::map<int, int> mask_index;              // telescope -> index in a launch mask
  std::vector<int> group_off;                 // per batch group: first mask index
  std::vector<const void *> pos_slopes;       // per batch position
  std::vector<void *> pos_x;
  int mask_len = 0;

  cudaStream_t streams[kMaxInFlight] = {};
  cudaEvent_t events[kMaxInFlight] = {};
  int *d_mask[kMaxInFlight] = {};
  int *h_mask[kMaxInFlight] = {};
  bool slot_busy[kMaxInFlight] = {};
  cudaStream_t admin_stream = nullptr;

  std::list<Launch> inflight;
  std::list<tomo_frame_result> results;
  int paused = 0;
  bool stop = false;
  int latest_only = 0;
  long long submitted = 0, done = 0, dropped = 0, superseded = 0, launches = 0;

  std::thread worker, completer;
};

namespace {

size_t used_bytes(const tomo_server *S) {
  size_t b = S->batch_bytes;
  for (const auto &kv : S->tels) b += kv.second->bytes;
  return b;
}

int free_slot(const tomo_server *S) {
  for (int j = 0; j < S->max_in_flight; ++j)
    if (!S->slot_busy[j]) return j;
  return -1;
}

bool ready(const tomo_server *S) {
  for (const auto &kv : S->tels)
    if (!kv.second->busy && !kv.second->queue.empty()) return true;
  return false;
}

// The telescopes of the next launch, oldest waiting frame first: every idle
// open-loop telescope with a waiting frame (one batched solve), or one
// closed-loop telescope (its own control step, so that several run on separate
// streams at once), whichever kind holds the oldest frame.
std::vector<Telescope *> next_launch(tomo_server *S) {
  std::vector<Telescope *> open;
  Telescope *loop = nullptr;
  double t_open = INFINITY;
  for (auto &kv : S->tels) {
    Telescope *t = kv.second;
    if (t->busy || t->queue.empty()) continue;
    const double ts = t->queue.front().t_submit;
    if (t->fit) {
      if (!loop || ts < loop->queue.front().t_submit) loop = t;
    } else {
      open.push_back(t);
      t_open = std::min(t_open, ts);
    }
  }
  if (loop && (open.empty() || loop->queue.front().t_submit < t_open)) return {loop};
  return open;
}

// Enqueue one launch on its stream: frame copies in, the mask, the batched
// solve, coefficient copies out, the completion event.  Runs without the
// lock; the launch is in flight, so the batch and the telescopes are fixed.
tomo_status enqueue_launch(tomo_server *S, const Launch &L) {
  tomo::NvtxRange nvtx("tomo_server launch");
  const int j = L.slot;
  cudaStream_t st = S->streams[j];
  cudaError_t e = cudaSuccess;
  std::memset(S->h_mask[j], 0, sizeof(int) * S->mask_len);
  bool open = false;
  for (const auto &f : L.frames) {
    const Telescope *t = S->tels.at(f.tel);
    if (!t->fit) {
      S->h_mask[j][S->mask_index.at(f.tel)] = 1;
      open = true;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(t->d_slopes, t->h_in + f.in_slot * t->ns * t->esz, t->ns * t->esz,
                          cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && open)
    e = cudaMemcpyAsync(S->d_mask[j], S->h_mask[j], sizeof(int) * S->mask_len, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_error(TOMO_ERR_CUDA, std::string("server copies: ") + cudaGetErrorString(e));
  if (open) {
    // the open-loop telescopes with a frame: one masked batched solve
    std::vector<const int *> active(S->group_off.size());
    for (size_t g = 0; g < active.size(); ++g) active[g] = S->d_mask[j] + S->group_off[g];
    const tomo_status ts = tomo::batch_solve(S->batch, S->pos_slopes.data(), S->pos_x.data(), active.data(),
                                             S->iters, 1, st);
    if (ts != TOMO_OK) return ts;
  }
  for (const auto &f : L.frames) {
    Telescope *t = S->tels.at(f.tel);
    const void *res = t->d_x;
    if (t->fit) {
      // closed loop: one control step, a_t into the buffer of a_{t-2}
      void *a_t = t->d_a[t->steps & 1];
      const tomo_status ts = tomo_polc_step(t->fit, t->d_slopes, t->d_x, t->d_rec, a_t, t->d_a[(t->steps + 1) & 1],
                                            a_t, t->gain, S->iters, t->fit_iters, 1, st);
      if (ts != TOMO_OK) return ts;
      ++t->steps;
      res = a_t;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(t->h_out + f.out_slot * t->n_out * t->esz, res, t->n_out * t->esz,
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(S->events[j], st);
  if (e != cudaSuccess) return set_error(TOMO_ERR_CUDA, std::string("server launch: ") + cudaGetErrorString(e));
  return TOMO_OK;
}

void worker_main(tomo_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_work.wait(lk, [&] { return S->stop || (S->paused == 0 && ready(S) && free_slot(S) >= 0); });
    if (S->stop) break;
    S->inflight.emplace_back();
    Launch &L = S->inflight.back();
    L.slot = free_slot(S);
    S->slot_busy[L.slot] = true;
    for (Telescope *t : next_launch(S)) {
      if (S->latest_only) {
        const double tnow = now_s();
        while (t->queue.size() > 1) {
          const Waiting old = t->queue.front();
          t->queue.pop_front();
          t->free_in.push_back(old.in_slot);
          S->results.push_back({t->id, TOMO_ERR_SUPERSEDED, old.tag, old.t_submit, tnow, tnow, 0, -1});
          ++S->superseded;
        }
      }
      const Waiting w = t->queue.front();
      t->queue.pop_front();
      t->busy = true;
      const int out = t->next_out;
      t->next_out = (t->next_out + 1) % S->result_slots;
      t->out_writing[out] = 1;
      L.frames.push_back({t->id, w.tag, w.t_submit, w.in_slot, out});
    }
    L.t_launch = now_s();
    lk.unlock();
    const tomo_status st = enqueue_launch(S, L);
    lk.lock();
    L.status = st;
    L.enqueued = true;
    ++S->launches;
    S->cv_done.notify_all();
  }
}

// Finish launch L (lock held): results, slots and telescopes become free.
void finish(tomo_server *S, std::list<Launch>::iterator it, int status) {
  const double t = now_s();
  const int n = static_cast<int>(it->frames.size());
  for (const auto &f : it->frames) {
    Telescope *tel = S->tels.at(f.tel);
    // a frame whose solve broke down (the plan's breakdown word, set on the device)
    const int st = (status == TOMO_OK && tomo::take_breakdown(tel->plan)) ? TOMO_ERR_BREAKDOWN : status;
    tel->busy = false;
    tel->free_in.push_back(f.in_slot);
    tel->out_writing[f.out_slot] = 0;
    tel->out_tag[f.out_slot] = st == TOMO_OK ? f.tag : -1;
    S->results.push_back({f.tel, st, f.tag, f.t_submit, it->t_launch, t, n, f.out_slot});
  }
  S->done += n;
  S->slot_busy[it->slot] = false;
  S->inflight.erase(it);
}

void completer_main(tomo_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_done.wait(lk, [&] {
      if (S->stop && S->inflight.empty()) return true;
      for (const auto &L : S->inflight)
        if (L.enqueued) return true;
      return false;
    });
    if (S->stop && S->inflight.empty()) break;
    // the oldest enqueued launch: wait for it without the lock
    auto it = S->inflight.begin();
    while (it != S->inflight.end() && !it->enqueued) ++it;
    cudaError_t e = cudaSuccess;
    if (it->status == TOMO_OK) {
      const cudaEvent_t ev = S->events[it->slot];
      lk.unlock();
      e = cudaEventSynchronize(ev);
      lk.lock();
    }
    finish(S, it, it->status != TOMO_OK ? it->status : (e == cudaSuccess ? TOMO_OK : TOMO_ERR_CUDA));
    // any other launch that is already complete
    for (auto jt = S->inflight.begin(); jt != S->inflight.end();) {
      if (!jt->enqueued) {
        ++jt;
        continue;
      }
      const cudaError_t q = jt->status == TOMO_OK ? cudaEventQuery(S->events[jt->slot]) : cudaSuccess;
      if (q == cudaErrorNotReady) {
        ++jt;
        continue;
      }
      auto cur = jt++;
      finish(S, cur, cur->status != TOMO_OK ? cur->status : (q == cudaSuccess ? TOMO_OK : TOMO_ERR_CUDA));
    }
    S->cv_work.notify_all();
    S->cv_idle.notify_all();
  }
}

// Pause the worker and wait until nothing is in flight (lock held on return).
void quiesce(tomo_server *S, std::unique_lock<std::mutex> &lk) {
  ++S->paused;
  S->cv_idle.wait(lk, [&] { return S->inflight.empty(); });
}

void resume(tomo_server *S) {
  --S->paused;
  S->cv_work.notify_all();
}

// New batch, masks and per-position pointers for the telescopes in `tels`
// (no launch in flight).  On failure nothing changes.
tomo_status rebuild(tomo_server *S, const std::map<int, Telescope *> &tels) {
  tomo::Batch *nb = nullptr;
  std::vector<tomo_plan *> plans;
  std::map<int, Telescope *> open;   // the batch holds the open-loop telescopes
  for (const auto &kv : tels)
    if (!kv.second->fit) open[kv.first] = kv.second;
  for (const auto &kv : open) plans.push_back(kv.second->plan);
  if (!plans.empty()) {
    const tomo_status st = tomo::build_batch(plans.data(), static_cast<int>(plans.size()), &nb);
    if (st != TOMO_OK) return st;
  }
  std::vector<int> ids;
  for (const auto &kv : open) ids.push_back(kv.first);
  std::map<int, int> mask_index;
  std::vector<int> group_off;
  int len = 0;
  size_t bytes = 0;
  if (nb) {
    for (const auto &g : nb->groups) {
      group_off.push_back(len);
      for (size_t slot = 0; slot < g.members.size(); ++slot) mask_index[ids[g.members[slot]]] = len + static_cast<int>(slot);
      len += static_cast<int>(g.members.size());
      bytes += g.bytes;
    }
  }
  int *dm[kMaxInFlight] = {}, *hm[kMaxInFlight] = {};
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < S->max_in_flight && e == cudaSuccess; ++j) {
    e = cudaMalloc(&dm[j], sizeof(int) * std::max(1, len));
    if (e == cudaSuccess) e = cudaHostAlloc(&hm[j], sizeof(int) * std::max(1, len), cudaHostAllocDefault);
  }
  if (e != cudaSuccess) {
    for (int j = 0; j < kMaxInFlight; ++j) {
      cudaFree(dm[j]);
      cudaFreeHost(hm[j]);
    }
    if (nb) tomo::free_batch(nb);
    return set_error(TOMO_ERR_NOMEM, std::string("server masks: ") + cudaGetErrorString(e));
  }
  if (S->batch) tomo::free_batch(S->batch);
  for (int j = 0; j < kMaxInFlight; ++j) {
    cudaFree(S->d_mask[j]);
    cudaFreeHost(S->h_mask[j]);
    S->d_mask[j] = dm[j];
    S->h_mask[j] = hm[j];
  }
  S->batch = nb;
  S->batch_bytes = bytes + static_cast<size_t>(S->max_in_flight) * sizeof(int) * std::max(1, len);
  S->mask_index = mask_index;
  S->group_off = group_off;
  S->mask_len = len;
  S->pos_slopes.clear();
  S->pos_x.clear();
  for (const auto &kv : open) {
    S->pos_slopes.push_back(kv.second->d_slopes);
    S->pos_x.push_back(kv.second->d_x);
  }
  return TOMO_OK;
}

void free_telescope(Telescope *t) {
  if (!t) return;
  if (t->fit) tomo_fit_destroy(t->fit);
  cudaFree(t->d_a[0]);
  cudaFree(t->d_a[1]);
  cudaFree(t->d_rec);
  cudaFree(t->d_slopes);
  cudaFree(t->d_x);
  cudaFreeHost(t->h_in);
  cudaFreeHost(t->h_out);
  tomo_destroy(t->plan);
  delete t;
}

}  // namespace

extern "C" {

double tomo_server_clock(void) { return now_s(); }

tomo_status tomo_server_create(size_t budget_bytes, int iters, int max_in_flight, int queue_depth,
                               int result_slots, tomo_server **out) {
  if (!out) return set_error(TOMO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (iters < 0 || iters > 100000) return set_error(TOMO_ERR_ARG, "iters out of range");
  if (max_in_flight < 1 || max_in_flight > kMaxInFlight) return set_error(TOMO_ERR_ARG, "max_in_flight must be 1..4");
  if (queue_depth < 1 || queue_depth > 256) return set_error(TOMO_ERR_ARG, "queue_depth must be 1..256");
  if (result_slots < 1 || result_slots > 256) return set_error(TOMO_ERR_ARG, "result_slots must be 1..256");
  tomo_server *S = new tomo_server();
  S->budget = budget_bytes;
  S->iters = iters;
  S->max_in_flight = max_in_flight;
  S->queue_depth = queue_depth;
  S->result_slots = result_slots;
  cudaError_t e = cudaGetDevice(&S->device);
  for (int j = 0; j < max_in_flight && e == cudaSuccess; ++j) {
    e = cudaStreamCreateWithFlags(&S->streams[j], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->events[j], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->admin_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    for (int j = 0; j < kMaxInFlight; ++j) {
      if (S->streams[j]) cudaStreamDestroy(S->streams[j]);
      if (S->events[j]) cudaEventDestroy(S->events[j]);
    }
    if (S->admin_stream) cudaStreamDestroy(S->admin_stream);
    delete S;
    return set_error(TOMO_ERR_CUDA, std::string("creating the server: ") + cudaGetErrorString(e));
  }
  S->worker = std::thread(worker_main, S);
  S->completer = std::thread(completer_main, S);
  *out = S;
  return TOMO_OK;
}

tomo_status tomo_server_admit(tomo_server *S, const tomo_geometry *g, int *telescope) {
  return tomo_server_admit_ex(S, g, nullptr, telescope);
}

tomo_status tomo_server_set_policy(tomo_server *S, int latest_only) {
  if (!S) return set_error(TOMO_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  S->latest_only = latest_only ? 1 : 0;
  return TOMO_OK;
}

tomo_status tomo_server_admit_ex(tomo_server *S, const tomo_geometry *g, const tomo_plan_options *opt,
                                 int *telescope) {
  return tomo_server_admit_loop(S, g, opt, nullptr, 0.0, 0, telescope);
}

tomo_status tomo_server_admit_loop(tomo_server *S, const tomo_geometry *g, const tomo_plan_options *opt,
                                   const tomo_fit_geometry *fit, double gain, int fit_iters, int *telescope) {
  if (!S || !g || !telescope) return set_error(TOMO_ERR_ARG, "server, geometry and telescope must not be NULL");
  if (fit && (!std::isfinite(gain) || fit_iters < 0 || fit_iters > 100000))
    return set_error(TOMO_ERR_ARG, "gain must be finite and fit_iters in 0..100000");
  std::lock_guard<std::mutex> admin(S->admin_mu);
  cudaSetDevice(S->device);
  Telescope *t = new Telescope();
  tomo_status st = tomo_plan_create_ex(g, opt, S->admin_stream, &t->plan);
  if (st != TOMO_OK) {
    delete t;
    return st;
  }
  tomo_plan_info info{};
  tomo_plan_get_info(t->plan, &info);
  t->n = static_cast<size_t>(info.n_coeffs);
  t->ns = static_cast<size_t>(info.n_slopes);
  t->esz = info.precision ? 8 : 4;
  t->n_out = t->n;
  t->bytes = tomo_plan_device_bytes(t->plan) + (t->n + t->ns) * t->esz;
  if (fit) {
    st = tomo_fit_create(t->plan, fit, &t->fit);
    if (st != TOMO_OK) {
      tomo_destroy(t->plan);
      delete t;
      return st;
    }
    tomo_fit_info fi{};
    tomo_fit_get_info(t->fit, &fi);
    t->gain = gain;
    t->fit_iters = fit_iters;
    t->n_out = static_cast<size_t>(fi.n_act);
    t->bytes += static_cast<size_t>(fi.device_bytes) + 3 * t->n_out * t->esz;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->budget && used_bytes(S) + t->bytes > S->budget) {
      const std::string msg = "admission: the telescope needs " + std::to_string(t->bytes) + " bytes; " +
                              std::to_string(used_bytes(S)) + " of " + std::to_string(S->budget) +
                              " budget bytes are in use";
      tomo_destroy(t->plan);
      delete t;
      return set_error(TOMO_ERR_NOMEM, msg);
    }
  }
  cudaError_t e = cudaMalloc(&t->d_slopes, t->ns * t->esz);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_x, t->n * t->esz);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->d_x, 0, t->n * t->esz, S->admin_stream);
  for (void **buf : {&t->d_a[0], &t->d_a[1], &t->d_rec}) {
    if (!t->fit || e != cudaSuccess) break;
    e = cudaMalloc(buf, t->n_out * t->esz);
    if (e == cudaSuccess) e = cudaMemsetAsync(*buf, 0, t->n_out * t->esz, S->admin_stream);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(&t->h_in, t->ns * t->esz * S->queue_depth, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&t->h_out, t->n_out * t->esz * S->result_slots, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->admin_stream);
  if (e != cudaSuccess) {
    free_telescope(t);
    return set_error(TOMO_ERR_NOMEM, std::string("admission: telescope slots: ") + cudaGetErrorString(e));
  }
  t->out_tag.assign(S->result_slots, -1);
  t->out_writing.assign(S->result_slots, 0);
  for (int k = 0; k < S->queue_depth; ++k) t->free_in.push_back(k);

  std::unique_lock<std::mutex> lk(S->mu);
  quiesce(S, lk);
  t->id = S->next_id;
  std::map<int, Telescope *> next = S->tels;
  next[t->id] = t;
  st = rebuild(S, next);
  if (st == TOMO_OK && S->budget && used_bytes(S) + t->bytes > S->budget) {
    rebuild(S, S->tels);   // the batch tables tipped it over: back to the previous set
    st = set_error(TOMO_ERR_NOMEM, "admission: the batch tables exceed the budget");
  }
  if (st != TOMO_OK) {
    resume(S);
    lk.unlock();
    free_telescope(t);
    return st;
  }
  S->tels = next;
  ++S->next_id;
  *telescope = t->id;
  resume(S);
  return TOMO_OK;
}

tomo_status tomo_server_release(tomo_server *S, int telescope) {
  if (!S) return set_error(TOMO_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> admin(S->admin_mu);
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tels.find(telescope);
  if (it == S->tels.end()) return set_error(TOMO_ERR_ARG, "no such telescope");
  Telescope *t = it->second;
  quiesce(S, lk);
  std::map<int, Telescope *> next = S->tels;
  next.erase(telescope);
  const tomo_status st = rebuild(S, next);
  if (st != TOMO_OK) {
    resume(S);
    return st;
  }
  S->tels = next;
  S->dropped += static_cast<long long>(t->queue.size());
  for (auto r = S->results.begin(); r != S->results.end(); ++r)
    if (r->telescope == telescope) r->result_slot = -1;
  resume(S);
  lk.unlock();
  free_telescope(t);
  return TOMO_OK;
}

tomo_status tomo_server_submit(tomo_server *S, int telescope, const void *host_slopes, long long tag) {
  if (!S || !host_slopes) return set_error(TOMO_ERR_ARG, "server and slopes must not be NULL");
  const double t0 = now_s();
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tels.find(telescope);
  if (it == S->tels.end()) return set_error(TOMO_ERR_ARG, "no such telescope");
  Telescope *t = it->second;
  if (t->free_in.empty()) return set_error(TOMO_ERR_FULL, "the telescope's frame queue is full");
  const int slot = t->free_in.back();
  t->free_in.pop_back();
  std::memcpy(t->h_in + slot * t->ns * t->esz, host_slopes, t->ns * t->esz);
  t->queue.push_back({tag, t0, slot});
  ++S->submitted;
  S->cv_work.notify_all();
  return TOMO_OK;
}

int tomo_server_poll(tomo_server *S, tomo_frame_result *out, int max) {
  if (!S || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  int k = 0;
  while (k < max && !S->results.empty()) {
    out[k++] = S->results.front();
    S->results.pop_front();
  }
  return k;
}

tomo_status tomo_server_result(tomo_server *S, int telescope, int result_slot, long long tag, void *host_out) {
  if (!S || !host_out) return set_error(TOMO_ERR_ARG, "server and output must not be NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tels.find(telescope);
  if (it == S->tels.end()) return set_error(TOMO_ERR_ARG, "no such telescope");
  Telescope *t = it->second;
  if (result_slot < 0 || result_slot >= S->result_slots) return set_error(TOMO_ERR_ARG, "result slot out of range");
  if (t->out_writing[result_slot] || t->out_tag[result_slot] != tag)
    return set_error(TOMO_ERR_ARG, "the result slot no longer holds that frame");
  std::memcpy(host_out, t->h_out + result_slot * t->n_out * t->esz, t->n_out * t->esz);
  return TOMO_OK;
}

tomo_status tomo_server_drain(tomo_server *S, double timeout_s) {
  if (!S) return set_error(TOMO_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  const bool ok = S->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return S->inflight.empty() && !ready(S) && S->done + S->dropped + S->superseded == S->submitted;
  });
  return ok ? TOMO_OK : set_error(TOMO_ERR_TIMEOUT, "drain: frames still waiting or in flight");
}

tomo_status tomo_server_get_stats(tomo_server *S, tomo_server_stats *out) {
  if (!S || !out) return set_error(TOMO_ERR_ARG, "server and output must not be NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  out->frames_submitted = S->submitted;
  out->frames_done = S->done;
  out->frames_superseded = S->superseded;
  out->launches = S->launches;
  out->bytes_in_use = static_cast<long long>(used_bytes(S));
  out->budget_bytes = static_cast<long long>(S->budget);
  out->telescopes = static_cast<int>(S->tels.size());
  out->in_flight = static_cast<int>(S->inflight.size());
  return TOMO_OK;
}

tomo_status tomo_server_get_fit(tomo_server *S, int telescope, const tomo_fit **out) {
  if (!S || !out) return set_error(TOMO_ERR_ARG, "server and out must not be NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tels.find(telescope);
  if (it == S->tels.end()) return set_error(TOMO_ERR_ARG, "no such telescope");
  *out = it->second->fit;
  return TOMO_OK;
}

tomo_status tomo_server_get_plan(tomo_server *S, int telescope, const tomo_plan **out) {
  if (!S || !out) return set_error(TOMO_ERR_ARG, "server and output must not be NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tels.find(telescope);
  if (it == S->tels.end()) return set_error(TOMO_ERR_ARG, "no such telescope");
  *out = it->second->plan;
  return TOMO_OK;
}

void tomo_server_destroy(tomo_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  if (S->worker.joinable()) S->worker.join();
  {
    std::lock_guard<std::mutex> lk(S->mu);   // launches the worker enqueued finish in the completer
  }
  S->cv_done.notify_all();
  if (S->completer.joinable()) S->completer.join();
  cudaSetDevice(S->device);
  if (S->batch) tomo::free_batch(S->batch);
  for (auto &kv : S->tels) free_telescope(kv.second);
  for (int j = 0; j < kMaxInFlight; ++j) {
    cudaFree(S->d_mask[j]);
    cudaFreeHost(S->h_mask[j]);
    if (S->streams[j]) cudaStreamDestroy(S->streams[j]);
    if (S->events[j]) cudaEventDestroy(S->events[j]);
  }
  if (S->admin_stream) cudaStreamDestroy(S->admin_stream);
  delete S;
}

}  // extern "C"
