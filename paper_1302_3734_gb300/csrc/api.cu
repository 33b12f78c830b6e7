// C ABI of the tomography library (declared in include/tomo.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tomo.h"
#include "common.h"
#include "host_plan.h"
#include "launch.h"
#include "plan_internal.h"

using namespace tomo;

namespace {

thread_local std::string g_err;
std::atomic<long long> g_launches{0};
std::mutex g_cfg_mu;
bool g_cfg_done[64] = {false};

tomo_status fail(tomo_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

}  // namespace

namespace tomo {
tomo_status set_error(tomo_status st, const std::string &msg) { return fail(st, msg); }
void count_launches(long long k) { g_launches.fetch_add(k); }
}  // namespace tomo

namespace {

tomo_status cuda_fail(cudaError_t e, const char *where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return TOMO_ERR_CUDA;
}

#define TOMO_CUDA(call, where)                      \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Arena layout helper: reserve, then resolve against the base pointer.
struct Arena {
  size_t size = 0;
  size_t take(size_t bytes) {
    size_t off = align_up(size, 256);
    size = off + bytes;
    return off;
  }
};

cudaError_t configure_device(int dev) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  if (dev >= 0 && dev < 64 && g_cfg_done[dev]) return cudaSuccess;
  cudaError_t e = configure_kernels();
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_cfg_done[dev] = true;
  return e;
}

}  // namespace

namespace {

// Launch one kernel through `fn`, bracketed by timing events when enabled.
template <typename F>
tomo_status timed(tomo_plan *p, int kind, cudaStream_t s, F fn, const char *what, int kernels = 1) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (p && p->timer.on) {
    a = p->timer.get();
    b = p->timer.get();
    cudaEventRecord(a, s);
  }
  cudaError_t e = fn();
  if (e != cudaSuccess) return cuda_fail(e, what);
  g_launches.fetch_add(kernels);
  if (p && p->timer.on) {
    cudaEventRecord(b, s);
    p->timer.recs.push_back({kind, a, b});
  }
  return TOMO_OK;
}

#define TOMO_TRY(x)                   \
  do {                                \
    tomo_status st_ = (x);            \
    if (st_ != TOMO_OK) return st_;   \
  } while (0)

// W of the grids a separate gather left in phi (src 2) or of io.in0's layers
// (src 0), with epilogue epi, for a launch set without the fused gather.
cudaError_t anal_ls(const LaunchSet &L, int src, int epi, int flags, const IoArgs &io, cudaStream_t s) {
  return L.stream ? launch_analysis_streamed(L.precision, src, epi, L.lf, flags, L.d_inst, L.ss, io, s)
                  : launch_analysis(L.precision, src, epi, L.lf, flags, L.d_inst, L.cl, L.n_cl, L.C, L.smem_a, io, s);
}
int anal_launches(const LaunchSet &L) { return L.stream ? streamed_launches(L.ss) : 1; }

// The gather of the plan's corner fields and W of the result with epilogue epi
// (0 plain into io.out0, 1 operator with p = io.in1 and q = io.out0): the fused
// kernel, or the separate gather and then the transform.
tomo_status adjoint_ls(tomo_plan *p, const LaunchSet &L, int epi, const IoArgs &io, cudaStream_t s) {
  if (!L.split)
    return timed(p, kKindAnalysis, s, [&] {
      return launch_analysis(L.precision, 1, epi, L.lf, 0, L.d_inst, L.cl, L.n_cl, L.C, L.smem_a, io, s);
    }, "analysis");
  const int tt_mode = epi == 1 ? 0 : 2;   // operator: the model term; otherwise the data alone
  TOMO_TRY(timed(p, kKindGather, s, [&] {
    return launch_gather(L.precision, tt_mode, L.d_inst, L.gi, L.n_gi, L.C, L.gather_vs, L.smem_g, io, s);
  }, "gather"));
  return timed(p, kKindAnalysis, s, [&] { return anal_ls(L, 2, epi, 0, io, s); }, "analysis", anal_launches(L));
}

// The launch sequence of one solve (Sec. 5.1): right-hand side and initial
// residual, then `iters` (P)CG iterations: synthesis, forward, (gather,)
// analysis, update.
tomo_status enqueue_solve(tomo_plan *tp, const LaunchSet &L, const void *const *slopes,
                          void *const *x, int iters, int warm, cudaStream_t s, int *n_kernels,
                          const int *active = nullptr) {
  int nk = 0;
  if (warm) {
    IoArgs io{};
    io.active = active;
    for (int i = 0; i < L.count; ++i) io.in0[i] = x[i];
    TOMO_TRY(timed(tp, kKindSynth, s, [&] { return synthesis_of(L, 0, 0, io, s); }, "synthesis (warm start)",
                   synthesis_launches(L)));
    nk += synthesis_launches(L);
  }
  {
    IoArgs io{};
    io.active = active;
    for (int i = 0; i < L.count; ++i) io.in1[i] = slopes[i];
    TOMO_TRY(timed(tp, kKindFwd, s, [&] {
      return launch_forward(L.precision, warm ? 1 : 2, L.max_layers, L.elong, L.d_inst, L.fwd, L.n_fwd, io, s);
    }, "forward (residual)"));
    ++nk;
  }
  {
    IoArgs io{};
    io.active = active;
    for (int i = 0; i < L.count; ++i) {
      io.out0[i] = x[i];
      io.in1[i] = slopes[i];   // tip/tilt-only sensors' data term
    }
    if (L.split) {
      TOMO_TRY(timed(tp, kKindGather, s, [&] {
        return launch_gather(L.precision, warm ? 1 : 2, L.d_inst, L.gi, L.n_gi, L.C, L.gather_vs, L.smem_g, io, s);
      }, "gather (residual)"));
      TOMO_TRY(timed(tp, kKindAnalysis, s, [&] { return anal_ls(L, 2, 2, warm ? kFlagWarm : 0, io, s); },
                     "analysis (residual)", anal_launches(L)));
      nk += 1 + anal_launches(L);
    } else {
      TOMO_TRY(timed(tp, kKindAnalysis, s, [&] {
        return launch_analysis(L.precision, 1, 2, L.lf, warm ? kFlagWarm : 0, L.d_inst, L.cl, L.n_cl, L.C, L.smem_a,
                               io, s);
      }, "analysis (residual)"));
      ++nk;
    }
  }
  for (int it = 0; it < iters; ++it) {
    IoArgs none{};
    none.active = active;
    TOMO_TRY(timed(tp, kKindSynth, s, [&] {
      return synthesis_of(L, 1, (it == 0 ? kFlagFirst : 0) | (it << kIterShift), none, s);
    }, "synthesis", synthesis_launches(L)));
    TOMO_TRY(timed(tp, kKindFwd, s, [&] {
      return launch_forward(L.precision, 0, L.max_layers, L.elong, L.d_inst, L.fwd, L.n_fwd, none, s);
    }, "forward"));
    if (L.split) {
      TOMO_TRY(timed(tp, kKindGather, s, [&] {
        return launch_gather(L.precision, 0, L.d_inst, L.gi, L.n_gi, L.C, L.gather_vs, L.smem_g, none, s);
      }, "gather"));
      TOMO_TRY(timed(tp, kKindAnalysis, s, [&] { return anal_ls(L, 2, 1, it << kIterShift, none, s); }, "analysis",
                     anal_launches(L)));
    } else {
      TOMO_TRY(timed(tp, kKindAnalysis, s, [&] {
        return launch_analysis(L.precision, 1, 1, L.lf, 0, L.d_inst, L.cl, L.n_cl, L.C, L.smem_a, none, s);
      }, "analysis"));
    }
    IoArgs io{};
    io.active = active;
    for (int i = 0; i < L.count; ++i) io.out0[i] = x[i];
    TOMO_TRY(timed(tp, kKindUpd, s, [&] {
      return launch_update(L.precision, it << kIterShift, L.d_inst, L.upd, L.n_upd, io, s);
    }, "update"));
    nk += synthesis_launches(L) + 2 + (L.split ? 1 + anal_launches(L) : 1);
  }
  if (n_kernels) *n_kernels = nk;
  return TOMO_OK;
}

tomo_status check_plan(const tomo_plan *p) {
  if (!p) return fail(TOMO_ERR_ARG, "plan is NULL");
  return TOMO_OK;
}

// ||r|| after a solve: the FP64 partials of the last kernel that produced r
// (the update, or the initial residual when iters == 0), summed on the host
// in the same fixed order the device uses.
tomo_status read_resnorm(tomo_plan *p, int iters, cudaStream_t s, double *out) {
  const HostPlan &H = p->hp;
  std::vector<double> part(std::max(1, H.n_part));
  double sc[kNumScalars];
  TOMO_CUDA(cudaMemcpyAsync(part.data(), p->h_inst.part, sizeof(double) * H.n_part,
                            cudaMemcpyDeviceToHost, s), "reading partials");
  TOMO_CUDA(cudaMemcpyAsync(sc, p->h_inst.scal, sizeof(sc), cudaMemcpyDeviceToHost, s), "reading scalars");
  TOMO_CUDA(cudaStreamSynchronize(s), "synchronising the solve");
  const int off = iters > 0 ? H.upd_part_off : H.cl_part_off;
  const int cnt = iters > 0 ? H.n_upd_blocks : H.n_cl_part;
  double rr = 0.0;
  for (int q = 0; q < cnt; ++q) rr += part[off + 2 * q + 1];
  *out = std::sqrt(std::max(0.0, rr));
  if (sc[kFlag] != 0.0 || !std::isfinite(rr)) {
    take_breakdown(p);   // reported here, not again by the next call
    return fail(TOMO_ERR_BREAKDOWN, "PCG breakdown: p.Ap <= 0 or not finite");
  }
  return TOMO_OK;
}

std::mutex g_batch_mu;
std::vector<Batch *> g_batches;

tomo_status get_batch(tomo_plan *const *plans, int count, Batch **out) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (Batch *b : g_batches)
    if (static_cast<int>(b->plans.size()) == count && std::equal(plans, plans + count, b->plans.begin())) {
      *out = b;
      return TOMO_OK;
    }
  if (g_batches.size() >= 32) {
    free_batch(g_batches.front());
    g_batches.erase(g_batches.begin());
  }
  DeviceGuard dg(plans[0]->device);
  Batch *b = nullptr;
  TOMO_TRY(build_batch(plans, count, &b));
  g_batches.push_back(b);
  *out = b;
  return TOMO_OK;
}

void drop_batches_of(const tomo_plan *p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batches.size();) {
    Batch *b = g_batches[i];
    if (std::find(b->plans.begin(), b->plans.end(), p) != b->plans.end()) {
      free_batch(b);
      g_batches.erase(g_batches.begin() + i);
    } else {
      ++i;
    }
  }
}

}  // namespace

namespace tomo {

tomo_status enqueue_plan_solve(tomo_plan *p, const void *slopes, void *x, int iters, int warm, cudaStream_t s,
                               int *n_kernels) {
  const void *sl[1] = {slopes};
  void *xs[1] = {x};
  return enqueue_solve(nullptr, p->ls, sl, xs, iters, warm ? 1 : 0, s, n_kernels);
}

void free_batch(Batch *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  for (auto &g : b->groups) cudaFree(g.arena);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

tomo_status build_batch(tomo_plan *const *plans, int count, Batch **out) {
  Batch *b = new Batch();
  b->plans.assign(plans, plans + count);
  b->device = plans[0]->device;
  for (int i = 0; i < count; ++i)
    if (plans[i]->device != b->device) {
      delete b;
      return fail(TOMO_ERR_ARG, "all plans of a batch must live on the same device");
    }
  // group members by launch shape
  for (int i = 0; i < count; ++i) {
    const HostPlan &H = plans[i]->hp;
    BatchGroup *g = nullptr;
    for (auto &cand : b->groups) {
      const HostPlan &H0 = plans[cand.members[0]]->hp;
      if (H0.C == H.C && H0.Lf == H.Lf && H0.precision == H.precision &&
          H0.gather_staged == H.gather_staged && H0.stream_tf == H.stream_tf &&
          H0.gather_vstage == H.gather_vstage &&
          static_cast<int>(cand.members.size()) < kMaxBatch)
        g = &cand;
    }
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
    }
    g->members.push_back(i);
  }
  for (auto &g : b->groups) {
    const int k = static_cast<int>(g.members.size());
    std::vector<InstDev> insts;
    std::vector<ClusterItem> cl;
    std::vector<FwdItem> fwd;
    std::vector<UpdItem> upd;
    std::vector<PassItem> pass[kMaxLevels + 1], coarse, gath;
    LaunchSet &L = g.ls;
    for (int slot = 0; slot < k; ++slot) {
      const tomo_plan *p = plans[g.members[slot]];
      const HostPlan &H = p->hp;
      insts.push_back(p->h_inst);
      for (auto c : H.cl_items) cl.push_back({slot, c.layer});
      for (auto f : H.fwd_items) {
        f.inst = slot;
        fwd.push_back(f);
      }
      for (auto gi : H.gather_items) {
        gi.inst = slot;
        gath.push_back(gi);
      }
      for (auto u : H.upd_items) {
        u.inst = slot;
        upd.push_back(u);
      }
      L.smem = std::max(L.smem, static_cast<size_t>(H.smem_transform));
      L.smem_a = std::max(L.smem_a, static_cast<size_t>(H.smem_analysis));
      L.max_layers = std::max(L.max_layers, H.n_layers);
      L.C = H.C;
      L.lf = H.Lf;
      L.precision = H.precision;
      L.split = H.gather_staged ? 0 : 1;
      L.smem_g = std::max(L.smem_g, static_cast<size_t>(H.smem_gather));
      L.gather_vs = H.gather_vstage;
      for (const auto &w : H.wfs) L.elong |= w.elong;
      L.stream = H.stream_tf;
      if (H.stream_tf) {
        for (int lv = 1; lv <= H.pass_kmax; ++lv)
          for (int q = 0; q < H.pass_cnt[lv]; ++q) {
            PassItem it = H.pass_items[H.pass_off[lv] + q];
            it.inst = slot;
            pass[lv].push_back(it);
          }
        for (PassItem it : H.coarse_items) {
          it.inst = slot;
          coarse.push_back(it);
        }
        L.ss.kmax = std::max(L.ss.kmax, H.pass_kmax);
        L.ss.smem_pass = std::max(L.ss.smem_pass, static_cast<size_t>(H.smem_pass));
        L.ss.smem_coarse = std::max(L.ss.smem_coarse, static_cast<size_t>(H.smem_coarse));
      }
    }
    std::vector<PassItem> passes;
    for (int lv = 1; lv <= L.ss.kmax; ++lv) {
      L.ss.off[lv] = static_cast<int>(passes.size());
      L.ss.cnt[lv] = static_cast<int>(pass[lv].size());
      passes.insert(passes.end(), pass[lv].begin(), pass[lv].end());
    }
    // the gather CTAs of all members, costliest first
    std::stable_sort(gath.begin(), gath.end(), [](const PassItem &x, const PassItem &y) { return x.slot > y.slot; });
    Arena A;
    const size_t o_i = A.take(sizeof(InstDev) * insts.size());
    const size_t o_c = A.take(sizeof(ClusterItem) * cl.size());
    const size_t o_f = A.take(sizeof(FwdItem) * fwd.size());
    const size_t o_u = A.take(sizeof(UpdItem) * upd.size());
    const size_t o_ps = A.take(sizeof(PassItem) * std::max<size_t>(1, passes.size()));
    const size_t o_co = A.take(sizeof(PassItem) * std::max<size_t>(1, coarse.size()));
    const size_t o_gi = A.take(sizeof(PassItem) * std::max<size_t>(1, gath.size()));
    const size_t bytes = align_up(A.size, 256);
    std::vector<char> img(bytes, 0);
    std::memcpy(img.data() + o_i, insts.data(), sizeof(InstDev) * insts.size());
    std::memcpy(img.data() + o_c, cl.data(), sizeof(ClusterItem) * cl.size());
    std::memcpy(img.data() + o_f, fwd.data(), sizeof(FwdItem) * fwd.size());
    std::memcpy(img.data() + o_u, upd.data(), sizeof(UpdItem) * upd.size());
    if (!passes.empty()) std::memcpy(img.data() + o_ps, passes.data(), sizeof(PassItem) * passes.size());
    if (!coarse.empty()) std::memcpy(img.data() + o_co, coarse.data(), sizeof(PassItem) * coarse.size());
    if (!gath.empty()) std::memcpy(img.data() + o_gi, gath.data(), sizeof(PassItem) * gath.size());
    cudaError_t e = cudaMalloc(&g.arena, bytes);
    g.bytes = bytes;
    if (e == cudaSuccess) e = cudaMemcpy(g.arena, img.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "uploading batch tables");
    }
    char *base = static_cast<char *>(g.arena);
    L.d_inst = reinterpret_cast<const InstDev *>(base + o_i);
    L.count = k;
    L.cl = reinterpret_cast<const ClusterItem *>(base + o_c);
    L.n_cl = static_cast<int>(cl.size());
    L.fwd = reinterpret_cast<const FwdItem *>(base + o_f);
    L.n_fwd = static_cast<int>(fwd.size());
    L.upd = reinterpret_cast<const UpdItem *>(base + o_u);
    L.n_upd = static_cast<int>(upd.size());
    L.ss.items = reinterpret_cast<const PassItem *>(base + o_ps);
    L.ss.coarse = reinterpret_cast<const PassItem *>(base + o_co);
    L.ss.n_coarse = static_cast<int>(coarse.size());
    L.gi = reinterpret_cast<const PassItem *>(base + o_gi);
    L.n_gi = static_cast<int>(gath.size());
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "creating the batch capture stream");
  }
  *out = b;
  return TOMO_OK;
}

// One solve of every instance of the batch (each group in turn); `active`
// (device, one int per batch position) lets instances sit out.
tomo_status batch_enqueue(Batch *b, const void *const *slopes, void *const *x, const int *const *active_g,
                          int iters, int warm, cudaStream_t s, int *n_kernels, tomo_plan *timing = nullptr) {
  int total = 0;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const BatchGroup &g = b->groups[gi];
    std::vector<const void *> sl(g.members.size());
    std::vector<void *> xs(g.members.size());
    for (size_t slot = 0; slot < g.members.size(); ++slot) {
      sl[slot] = slopes[g.members[slot]];
      xs[slot] = x[g.members[slot]];
    }
    int nk = 0;
    TOMO_TRY(enqueue_solve(timing, g.ls, sl.data(), xs.data(), iters, warm, s, &nk,
                           active_g ? active_g[gi] : nullptr));
    total += nk;
  }
  if (n_kernels) *n_kernels = total;
  return TOMO_OK;
}

tomo_status batch_solve(Batch *b, const void *const *slopes, void *const *x, const int *const *active_g,
                        int iters, int warm, cudaStream_t s) {
  const int count = static_cast<int>(b->plans.size());
  if (b->plans[0]->timer.on) {
    // per-kernel timing (on the first plan): every launch direct, between events
    return batch_enqueue(b, slopes, x, active_g, iters, warm, s, nullptr, b->plans[0]);
  }
  const int *key_active = active_g ? active_g[0] : nullptr;
  BatchGraph *ge = nullptr;
  for (auto &g : b->graphs)
    if (g.iters == iters && g.warm == warm && g.active == key_active &&
        std::equal(slopes, slopes + count, g.slopes.begin()) && std::equal(x, x + count, g.x.begin()))
      ge = &g;
  if (!ge) {
    if (b->graphs.size() >= 16) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      b->graphs.erase(b->graphs.begin());
    }
    cudaGraph_t graph = nullptr;
    TOMO_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin batch capture");
    int nk = 0;
    const long long before = g_launches.load();
    tomo_status st = batch_enqueue(b, slopes, x, active_g, iters, warm, b->cap, &nk);
    g_launches.store(before);
    cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
    if (st != TOMO_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "end batch capture");
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "batch graph instantiate");
    b->graphs.push_back({std::vector<const void *>(slopes, slopes + count),
                         std::vector<void *>(x, x + count), key_active, iters, warm, exec, nk});
    ge = &b->graphs.back();
  }
  TOMO_CUDA(cudaGraphLaunch(ge->exec, s), "batch graph launch");
  g_launches.fetch_add(ge->kernels);
  return TOMO_OK;
}

}  // namespace tomo

namespace tomo {

// W^-1 of a launch set: the cluster kernel, or the streamed coarse kernel and
// passes.  src 0: io.in0 coefficients; 1: the PCG direction update fused in.
cudaError_t synthesis_of(const LaunchSet &L, int src, int flags, const IoArgs &io, cudaStream_t s) {
  return L.stream ? launch_synthesis_streamed(L.precision, src, L.lf, flags, L.d_inst, L.ss, io, s)
                  : launch_synthesis(L.precision, src, L.lf, flags, L.d_inst, L.cl, L.n_cl, L.C, L.smem, io, s);
}
int synthesis_launches(const LaunchSet &L) { return L.stream ? streamed_launches(L.ss) : 1; }

}  // namespace tomo

extern "C" {

const char *tomo_version(void) { return "tomo-gb300 0.1 (sm_103a)"; }

const char *tomo_last_error(void) { return g_err.c_str(); }

long long tomo_launch_count(void) { return g_launches.load(); }

tomo_status tomo_plan_create(const tomo_geometry *g, void *cuda_stream, tomo_plan **out) {
  return tomo_plan_create_ex(g, nullptr, cuda_stream, out);
}

tomo_status tomo_plan_create_ex(const tomo_geometry *g, const tomo_plan_options *opt, void *cuda_stream,
                                tomo_plan **out) {
  if (!out) return fail(TOMO_ERR_ARG, "out is NULL");
  *out = nullptr;
  int creq = 0, treq = 0;
  if (opt) {
    for (int r : opt->reserved)
      if (r != 0) return fail(TOMO_ERR_ARG, "tomo_plan_options.reserved must be zero");
    if (opt->cluster_size < 0) return fail(TOMO_ERR_ARG, "cluster size must be >= 0");
    creq = opt->cluster_size;
    treq = opt->transforms;
  }
  tomo_plan *p = new (std::nothrow) tomo_plan();
  if (!p) return fail(TOMO_ERR_NOMEM, "host allocation failed");
  std::string err;
  tomo_status st = build_host_plan(g, &p->hp, &err, creq, treq);
  if (st != TOMO_OK) {
    delete p;
    return fail(st, err);
  }
  const HostPlan &H = p->hp;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t ce = cudaGetDevice(&p->device);
  if (ce != cudaSuccess) {
    delete p;
    return cuda_fail(ce, "cudaGetDevice");
  }
  ce = configure_device(p->device);
  if (ce != cudaSuccess) {
    delete p;
    return cuda_fail(ce, "configuring kernels");
  }
  const size_t esz = H.precision ? 8 : 4;
  p->esz = esz;
  if (forward_smem(H.n_layers, H.precision) > static_cast<size_t>(kMaxForwardSmem)) {
    delete p;
    return fail(TOMO_ERR_UNSUPPORTED, "too many layers for the forward kernel's staged tables");
  }
  for (const auto &w : H.wfs) {
    p->nc_max = std::max(p->nc_max, w.nc);
    p->max_sub2 = std::max(p->max_sub2, w.n * w.n);
  }

  // ---- arena layout: tables (uploaded) then workspace (zeroed)
  Arena A;
  const size_t o_inst = A.take(sizeof(InstDev));
  const size_t o_layers = A.take(sizeof(LayerDev) * H.layers.size());
  const size_t o_wfs = A.take(sizeof(WfsDev) * H.wfs.size());
  const size_t o_sub = A.take(sizeof(int) * H.sub_idx.size());
  const size_t o_act = A.take(H.active.size());
  const size_t o_posoff = A.take(sizeof(int) * H.pos_off.size());
  const size_t o_posi0 = A.take(sizeof(int) * H.pos_i0.size());
  const size_t o_posf = A.take(esz * H.pos_f.size());
  const size_t o_gtoff = A.take(sizeof(int) * H.gt_off.size());
  const size_t n_rec = std::max<size_t>(1, H.gt_ro.size());
  const size_t o_gtrec = A.take(esz * H.rec_stride * n_rec);
  const size_t o_gtys = A.take(sizeof(int) * n_rec);
  const size_t o_vsrun = A.take(sizeof(int4) * std::max<size_t>(1, H.vs_run.size()));
  const size_t o_stage = A.take(std::max<size_t>(16, H.stage_img.size()));
  const size_t o_eslot = A.take(sizeof(EdgeSlot) * H.edge_slots.size());
  const size_t o_gel = A.take(esz * std::max<size_t>(2, H.gel.size()));
  const size_t o_gtcols = A.take(sizeof(int2) * std::max<size_t>(1, H.gt_cols.size()));
  const size_t o_gtbrows = A.take(sizeof(int2) * std::max<size_t>(1, H.gt_brows.size()));
  const size_t o_ttseg = A.take(sizeof(int2) * H.tt_seg.size());
  const size_t o_ttnode = A.take(sizeof(int) * std::max<size_t>(1, H.tt_node.size()));
  const size_t o_ttbeg = A.take(sizeof(int) * H.tt_beg.size());
  const size_t o_ttk = A.take(sizeof(int) * std::max<size_t>(1, H.tt_k.size()));
  const size_t o_ttw = A.take(esz * std::max<size_t>(2, H.tt_w.size()));
  const size_t o_eidx = A.take(sizeof(int) * std::max<size_t>(1, H.edge_idx.size()));
  const size_t o_et = A.take(esz * std::max<size_t>(2, H.edge_t.size()));
  const size_t o_runrows = A.take(sizeof(int) * H.run_rows.size());
  const size_t o_runab = A.take(sizeof(int2) * std::max<size_t>(1, H.run_ab.size()));
  const size_t o_cl = A.take(sizeof(ClusterItem) * H.cl_items.size());
  const size_t o_fwd = A.take(sizeof(FwdItem) * H.fwd_items.size());
  const size_t o_upd = A.take(sizeof(UpdItem) * H.upd_items.size());
  const size_t o_pass = A.take(sizeof(PassItem) * std::max<size_t>(1, H.pass_items.size()));
  const size_t o_coarse = A.take(sizeof(PassItem) * std::max<size_t>(1, H.coarse_items.size()));
  const size_t o_gitem = A.take(sizeof(PassItem) * std::max<size_t>(1, H.gather_items.size()));
  const size_t tables_end = align_up(A.size, 256);
  const size_t n = static_cast<size_t>(H.n);
  const size_t o_r = A.take(esz * n);
  const size_t o_p = A.take(esz * n);
  const size_t o_q = A.take(esz * n);
  const size_t o_phi = A.take(esz * n);
  // a tap window of a sensor with fewer corners than taps reads (at zero
  // weight) up to max_taps rows and columns past its field: zero padding
  const size_t o_v = A.take(esz * (H.v_total + 32));
  const size_t o_jinv = A.take(esz * n);
  const size_t o_jdiag = A.take(sizeof(double) * n);
  const size_t o_scal = A.take(sizeof(double) * kNumScalars);
  const size_t o_part = A.take(sizeof(double) * std::max(1, H.n_part));
  // streamed transforms: the second direction buffer and the low-low scratch
  const size_t o_p2 = H.stream_tf ? A.take(esz * n) : 0;
  const size_t o_lls = H.stream_tf ? A.take(esz * std::max<long long>(1, H.lls_elems)) : 0;
  p->arena_bytes = align_up(A.size, 256);
  ce = cudaMalloc(&p->arena, p->arena_bytes);
  if (ce != cudaSuccess) {
    delete p;
    return fail(TOMO_ERR_NOMEM, std::string("cudaMalloc of the plan: ") + cudaGetErrorString(ce));
  }
  char *base = static_cast<char *>(p->arena);
  // the breakdown word: page-locked, mapped, written by the update kernel
  ce = cudaHostAlloc(reinterpret_cast<void **>(&p->bd_host), sizeof(int), cudaHostAllocMapped);
  if (ce == cudaSuccess) {
    *p->bd_host = 0;
    ce = cudaHostGetDevicePointer(reinterpret_cast<void **>(&p->h_inst.bd_word), p->bd_host, 0);
  }
  if (ce != cudaSuccess) {
    cudaFree(p->arena);
    if (p->bd_host) cudaFreeHost(p->bd_host);
    delete p;
    return fail(TOMO_ERR_NOMEM, std::string("mapped host word of the plan: ") + cudaGetErrorString(ce));
  }

  InstDev &I = p->h_inst;
  I.n = H.n;
  I.n_layers = H.n_layers;
  I.n_wfs = H.n_wfs;
  I.J = H.J;
  I.Lf = H.Lf;
  I.precond = H.precond;
  I.C = H.C;
  I.n_slopes = H.n_slopes;
  I.cl_part_off = H.cl_part_off;
  I.upd_part_off = H.upd_part_off;
  I.n_upd_blocks = H.n_upd_blocks;
  I.fwd_part_off = H.fwd_part_off;
  for (int t = 0; t < kMaxTaps; ++t) {
    I.h[t] = t < H.Lf ? H.h[t] : 0.0;
    I.g[t] = t < H.Lf ? H.g[t] : 0.0;
    I.hf[t] = static_cast<float>(I.h[t]);
    I.gf[t] = static_cast<float>(I.g[t]);
  }
  I.r = base + o_r;
  I.p = base + o_p;
  I.q = base + o_q;
  I.phi = base + o_phi;
  I.v = base + o_v;
  I.jinv = base + o_jinv;
  I.scal = reinterpret_cast<double *>(base + o_scal);
  I.part = reinterpret_cast<double *>(base + o_part);
  I.stream_tf = H.stream_tf;
  I.n_cl_part = H.n_cl_part;
  I.p2 = H.stream_tf ? base + o_p2 : nullptr;
  I.lls = H.stream_tf ? base + o_lls : nullptr;
  I.layers = reinterpret_cast<const LayerDev *>(base + o_layers);
  I.wfs = reinterpret_cast<const WfsDev *>(base + o_wfs);
  I.sub_idx = reinterpret_cast<const int *>(base + o_sub);
  I.active = reinterpret_cast<const unsigned char *>(base + o_act);
  I.pos_off = reinterpret_cast<const int *>(base + o_posoff);
  I.pos_i0 = reinterpret_cast<const int *>(base + o_posi0);
  I.pos_f = base + o_posf;
  I.gt_off = reinterpret_cast<const int *>(base + o_gtoff);
  I.gt_rec = base + o_gtrec;
  I.gt_ys = reinterpret_cast<const int *>(base + o_gtys);
  I.vs_run = reinterpret_cast<const int4 *>(base + o_vsrun);
  I.vstage = H.vstage;
  I.v_total = H.v_total;
  I.max_band_cells = static_cast<int>(H.max_band_cells);
  I.max_band_v = static_cast<int>(H.max_band_v);
  I.stage_img = base + o_stage;
  I.edge_slots = reinterpret_cast<const EdgeSlot *>(base + o_eslot);
  I.gel = H.gel.empty() ? nullptr : base + o_gel;
  I.gt_cols = reinterpret_cast<const int2 *>(base + o_gtcols);
  I.gt_brows = reinterpret_cast<const int2 *>(base + o_gtbrows);
  I.img_stride = H.img_stride;
  I.tt_seg = reinterpret_cast<const int2 *>(base + o_ttseg);
  I.tt_node = reinterpret_cast<const int *>(base + o_ttnode);
  I.tt_beg = reinterpret_cast<const int *>(base + o_ttbeg);
  I.tt_k = reinterpret_cast<const int *>(base + o_ttk);
  I.tt_w = base + o_ttw;
  I.n_tt = H.n_tt;
  I.n_edge_wfs = H.n_edge_wfs;
  I.gather_staged = H.gather_staged;
  I.n_dense = H.n_dense;
  I.max_tt_entries = H.max_tt_entries;
  I.max_taps = H.max_taps;
  I.rec_stride = H.rec_stride;
  I.edge_idx = reinterpret_cast<const int *>(base + o_eidx);
  I.edge_t = base + o_et;
  I.run_rows = reinterpret_cast<const int *>(base + o_runrows);
  I.run_ab = reinterpret_cast<const int2 *>(base + o_runab);
  p->d_inst = reinterpret_cast<InstDev *>(base + o_inst);
  p->d_jdiag = reinterpret_cast<double *>(base + o_jdiag);

  // host image of the tables
  std::vector<char> img(tables_end, 0);
  auto put = [&](size_t off, const void *src, size_t bytes) {
    if (bytes) std::memcpy(img.data() + off, src, bytes);
  };
  put(o_inst, &I, sizeof(InstDev));
  put(o_layers, H.layers.data(), sizeof(LayerDev) * H.layers.size());
  put(o_wfs, H.wfs.data(), sizeof(WfsDev) * H.wfs.size());
  put(o_sub, H.sub_idx.data(), sizeof(int) * H.sub_idx.size());
  put(o_act, H.active.data(), H.active.size());
  put(o_posoff, H.pos_off.data(), sizeof(int) * H.pos_off.size());
  put(o_posi0, H.pos_i0.data(), sizeof(int) * H.pos_i0.size());
  auto put_real = [&](size_t off, const std::vector<double> &v) {
    if (esz == 8) {
      put(off, v.data(), 8 * v.size());
    } else {
      std::vector<float> f(v.begin(), v.end());
      put(off, f.data(), 4 * f.size());
    }
  };
  put_real(o_posf, H.pos_f);
  put_real(o_et, H.edge_t);
  {
    // tap records in the plan's precision, the window offset's int bits in slot 0
    std::vector<char> rec(esz * H.rec_stride * n_rec, 0);
    for (size_t r = 0; r < H.gt_ro.size(); ++r) {
      char *dst = rec.data() + esz * H.rec_stride * r;
      std::memcpy(dst, &H.gt_ro[r], sizeof(int));
      for (int t = 0; t < H.max_taps; ++t) {
        const double w = H.gt_rw[4 * r + t];
        if (esz == 8) {
          std::memcpy(dst + 8 * (1 + t), &w, 8);
        } else {
          const float wf = static_cast<float>(w);
          std::memcpy(dst + 4 * (1 + t), &wf, 4);
        }
      }
    }
    put(o_gtrec, rec.data(), rec.size());
  }
  put(o_gtys, H.gt_ys.data(), sizeof(int) * H.gt_ys.size());
  put(o_vsrun, H.vs_run.data(), sizeof(int4) * H.vs_run.size());
  put(o_stage, H.stage_img.data(), H.stage_img.size());
  put(o_eslot, H.edge_slots.data(), sizeof(EdgeSlot) * H.edge_slots.size());
  if (!H.gel.empty()) put_real(o_gel, H.gel);
  put(o_gtcols, H.gt_cols.data(), sizeof(int2) * H.gt_cols.size());
  put(o_gtbrows, H.gt_brows.data(), sizeof(int2) * H.gt_brows.size());
  put_real(o_ttw, H.tt_w);
  put(o_gtoff, H.gt_off.data(), sizeof(int) * H.gt_off.size());
  put(o_ttseg, H.tt_seg.data(), sizeof(int2) * H.tt_seg.size());
  put(o_ttnode, H.tt_node.data(), sizeof(int) * H.tt_node.size());
  put(o_ttbeg, H.tt_beg.data(), sizeof(int) * H.tt_beg.size());
  put(o_ttk, H.tt_k.data(), sizeof(int) * H.tt_k.size());
  put(o_eidx, H.edge_idx.data(), sizeof(int) * H.edge_idx.size());
  put(o_runrows, H.run_rows.data(), sizeof(int) * H.run_rows.size());
  put(o_runab, H.run_ab.data(), sizeof(int2) * H.run_ab.size());
  put(o_cl, H.cl_items.data(), sizeof(ClusterItem) * H.cl_items.size());
  put(o_fwd, H.fwd_items.data(), sizeof(FwdItem) * H.fwd_items.size());
  put(o_upd, H.upd_items.data(), sizeof(UpdItem) * H.upd_items.size());
  put(o_pass, H.pass_items.data(), sizeof(PassItem) * H.pass_items.size());
  put(o_coarse, H.coarse_items.data(), sizeof(PassItem) * H.coarse_items.size());
  put(o_gitem, H.gather_items.data(), sizeof(PassItem) * H.gather_items.size());

  auto bail = [&](tomo_status code, const std::string &msg) {
    cudaFree(p->arena);
    cudaFreeHost(p->bd_host);
    delete p;
    return fail(code, msg);
  };
  ce = cudaMemcpyAsync(base, img.data(), tables_end, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + tables_end, 0, p->arena_bytes - tables_end, s);
  if (ce != cudaSuccess) return bail(TOMO_ERR_CUDA, std::string("uploading the plan: ") + cudaGetErrorString(ce));

  // ---- exact Jacobi diagonal (plan-time buffers in a temporary allocation)
  {
    Arena T;
    const size_t t_prof = T.take(sizeof(double) * H.profiles.size());
    const size_t t_poff = T.take(sizeof(int) * H.prof_off.size());
    const size_t t_posd = T.take(sizeof(double) * H.pos_f.size());
    void *tmp = nullptr;
    ce = cudaMalloc(&tmp, align_up(T.size, 256));
    if (ce != cudaSuccess) return bail(TOMO_ERR_NOMEM, "cudaMalloc of plan-time tables failed");
    char *tb = static_cast<char *>(tmp);
    ce = cudaMemcpyAsync(tb + t_prof, H.profiles.data(), sizeof(double) * H.profiles.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(tb + t_poff, H.prof_off.data(), sizeof(int) * H.prof_off.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(tb + t_posd, H.pos_f.data(), sizeof(double) * H.pos_f.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
      ce = launch_jacobi(p->d_inst, H.n, reinterpret_cast<double *>(tb + t_prof),
                         reinterpret_cast<int *>(tb + t_poff), reinterpret_cast<double *>(tb + t_posd),
                         p->d_jdiag, I.jinv, H.precision, p->nc_max, -1.0, s);
    if (ce == cudaSuccess) {
      g_launches.fetch_add(1);
      ce = cudaStreamSynchronize(s);
    }
    cudaFree(tmp);
    if (ce != cudaSuccess) return bail(TOMO_ERR_CUDA, std::string("Jacobi diagonal: ") + cudaGetErrorString(ce));
  }
  ce = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return bail(TOMO_ERR_CUDA, "creating the capture stream");

  LaunchSet &L = p->ls;
  L.d_inst = p->d_inst;
  L.count = 1;
  L.cl = reinterpret_cast<const ClusterItem *>(base + o_cl);
  L.n_cl = static_cast<int>(H.cl_items.size());
  L.C = H.C;
  L.smem = static_cast<size_t>(H.smem_transform);
  L.smem_a = static_cast<size_t>(H.smem_analysis);
  L.fwd = reinterpret_cast<const FwdItem *>(base + o_fwd);
  L.n_fwd = static_cast<int>(H.fwd_items.size());
  L.max_layers = H.n_layers;
  L.lf = H.Lf;
  L.upd = reinterpret_cast<const UpdItem *>(base + o_upd);
  L.n_upd = static_cast<int>(H.upd_items.size());
  L.precision = H.precision;
  L.split = H.gather_staged ? 0 : 1;
  L.smem_g = static_cast<size_t>(H.smem_gather);
  L.gather_vs = H.gather_vstage;
  L.gi = reinterpret_cast<const PassItem *>(base + o_gitem);
  L.n_gi = static_cast<int>(H.gather_items.size());
  L.elong = 0;
  for (const auto &w : H.wfs) L.elong |= w.elong;
  L.stream = H.stream_tf;
  if (H.stream_tf) {
    StreamSet &S = L.ss;
    S.items = reinterpret_cast<const PassItem *>(base + o_pass);
    S.kmax = H.pass_kmax;
    for (int k = 1; k <= H.pass_kmax; ++k) {
      S.off[k] = H.pass_off[k];
      S.cnt[k] = H.pass_cnt[k];
    }
    S.coarse = reinterpret_cast<const PassItem *>(base + o_coarse);
    S.n_coarse = static_cast<int>(H.coarse_items.size());
    S.smem_pass = static_cast<size_t>(H.smem_pass);
    S.smem_coarse = static_cast<size_t>(H.smem_coarse);
  }
  *out = p;
  g_err.clear();
  return TOMO_OK;
}

void tomo_destroy(tomo_plan *p) {
  if (!p) return;
  DeviceGuard dg(p->device);
  cudaDeviceSynchronize();
  drop_batches_of(p);
  for (auto &g : p->graphs) cudaGraphExecDestroy(g.exec);
  for (auto &r : p->timer.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : p->timer.pool) cudaEventDestroy(e);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->arena);
  if (p->bd_host) cudaFreeHost(p->bd_host);
  delete p;
}

size_t tomo_plan_device_bytes(const tomo_plan *p) { return p ? p->arena_bytes : 0; }

tomo_status tomo_plan_get_info(const tomo_plan *p, tomo_plan_info *out) {
  TOMO_TRY(check_plan(p));
  if (!out) return fail(TOMO_ERR_ARG, "out is NULL");
  const HostPlan &H = p->hp;
  out->n_coeffs = H.n;
  out->n_slopes = H.n_slopes;
  out->n_layers = H.n_layers;
  out->n_wfs = H.n_wfs;
  out->cluster_size = H.C;
  const LaunchSet &L = p->ls;
  const int adj = L.split ? 1 + anal_launches(L) : 1;
  out->kernels_per_iteration = synthesis_launches(L) + 2 + adj;
  out->kernels_per_solve_base = synthesis_launches(L) + 1 + adj;
  out->gather_separate = L.split;
  out->streamed = L.stream;
  out->device_bytes = static_cast<long long>(p->arena_bytes);
  // p-update + W^-1 (r, J^-1, p in; p, phi out), ray-trace (phi in, v out),
  // gather + W + prior (v, p in; q out), update (x, p, r, q, J^-1 in; x, r out)
  // V: corner values of the sensors with a corner field (the forward kernel writes them and
  // the gather reads them; a tip/tilt-only sensor reaches the layers through its edge list)
  const long long vec = H.precond ? 15 : 13;
  long long V = 0;
  for (const auto &w : H.wfs)
    if (w.kind != kTTOnly) V += static_cast<long long>(w.nc) * w.nc;
  out->bytes_per_iteration = (vec * H.n + 2LL * V) * static_cast<long long>(p->esz);
  out->precision = H.precision;
  out->breakdown_pending = p->bd_host ? *reinterpret_cast<volatile int *>(p->bd_host) : 0;
  return TOMO_OK;
}

tomo_status tomo_set_kernel_timing(tomo_plan *p, int enable) {
  TOMO_TRY(check_plan(p));
  p->timer.on = enable != 0;
  for (int k = 0; k < kNumKinds; ++k) {
    p->kind_ms[k] = 0.0;
    p->kind_n[k] = 0;
  }
  return TOMO_OK;
}

tomo_status tomo_get_kernel_times(tomo_plan *p, int *counts, double *ms, int n_kinds) {
  TOMO_TRY(check_plan(p));
  DeviceGuard dg(p->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "synchronising for kernel times");
  for (auto &r : p->timer.recs) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, r.a, r.b);
    p->kind_ms[r.kind] += t;
    p->kind_n[r.kind] += 1;
    p->timer.pool.push_back(r.a);
    p->timer.pool.push_back(r.b);
  }
  p->timer.recs.clear();
  for (int k = 0; k < n_kinds && k < kNumKinds; ++k) {
    if (counts) counts[k] = static_cast<int>(p->kind_n[k]);
    if (ms) ms[k] = p->kind_ms[k];
  }
  return TOMO_OK;
}

tomo_status tomo_set_launch_mode(tomo_plan *p, int use_graphs) {
  TOMO_TRY(check_plan(p));
  p->use_graphs = use_graphs ? 1 : 0;
  return TOMO_OK;
}

tomo_status tomo_solve(tomo_plan *p, const void *d_slopes, void *d_coeffs, int iters, int warm,
                       void *cuda_stream, double *out_resnorm) {
  TOMO_TRY(check_plan(p));
  if (!d_slopes || !d_coeffs) return fail(TOMO_ERR_ARG, "slopes and coefficients must be device pointers");
  if (iters < 0 || iters > 100000) return fail(TOMO_ERR_ARG, "iters out of range");
  if (take_breakdown(p))
    return fail(TOMO_ERR_BREAKDOWN, "an earlier solve of this plan broke down (p.Ap <= 0 or not finite) and "
                                    "froze its iterate; this call enqueued nothing");
  DeviceGuard dg(p->device);
  NvtxRange nvtx("tomo_solve");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  warm = warm ? 1 : 0;
  const void *sl[1] = {d_slopes};
  void *xs[1] = {d_coeffs};
  if (p->use_graphs && !p->timer.on) {
    GraphEntry *ge = nullptr;
    for (auto &g : p->graphs)
      if (g.slopes == d_slopes && g.x == d_coeffs && g.iters == iters && g.warm == warm) ge = &g;
    if (!ge) {
      if (p->graphs.size() >= 16) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
      }
      cudaGraph_t graph = nullptr;
      TOMO_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      int nk = 0;
      const long long before = g_launches.load();
      tomo_status st = enqueue_solve(nullptr, p->ls, sl, xs, iters, warm, p->cap_stream, &nk);
      g_launches.store(before);
      cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &graph);
      if (st != TOMO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
      cudaGraphExec_t exec = nullptr;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
      p->graphs.push_back({d_slopes, d_coeffs, iters, warm, exec, nk});
      ge = &p->graphs.back();
    }
    TOMO_CUDA(cudaGraphLaunch(ge->exec, s), "graph launch");
    g_launches.fetch_add(ge->kernels);
  } else {
    TOMO_TRY(enqueue_solve(p, p->ls, sl, xs, iters, warm, s, nullptr));
  }
  if (out_resnorm) {
    TOMO_TRY(read_resnorm(p, iters, s, out_resnorm));
  }
  return TOMO_OK;
}

tomo_status tomo_coeffs_to_layers(tomo_plan *p, const void *d_coeffs, void *d_layers, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_coeffs || !d_layers) return fail(TOMO_ERR_ARG, "NULL device pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const LaunchSet &L = p->ls;
  IoArgs io{};
  io.in0[0] = d_coeffs;
  io.out0[0] = d_layers;
  return timed(p, kKindSynth, s, [&] { return synthesis_of(L, 0, 0, io, s); }, "synthesis", synthesis_launches(L));
}

tomo_status tomo_layers_to_coeffs(tomo_plan *p, const void *d_layers, void *d_coeffs, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_coeffs || !d_layers) return fail(TOMO_ERR_ARG, "NULL device pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const LaunchSet &L = p->ls;
  IoArgs io{};
  io.in0[0] = d_layers;
  io.out0[0] = d_coeffs;
  return timed(p, kKindAnalysis, s, [&] { return anal_ls(L, 0, 0, 0, io, s); }, "analysis", anal_launches(L));
}

tomo_status tomo_layers_to_slopes(tomo_plan *p, const void *d_layers, void *d_slopes, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_slopes || !d_layers) return fail(TOMO_ERR_ARG, "NULL device pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  IoArgs io{};
  io.in0[0] = d_layers;
  io.out0[0] = d_slopes;
  return timed(p, kKindOther, s, [&] {
    return launch_slopes(p->ls.precision, p->d_inst, p->hp.n_wfs, p->max_sub2, io, s);
  }, "slopes");
}

tomo_status tomo_apply_normal(tomo_plan *p, const void *d_in, void *d_out, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_in || !d_out) return fail(TOMO_ERR_ARG, "NULL device pointer");
  if (d_in == d_out) return fail(TOMO_ERR_ARG, "d_in and d_out must not overlap");
  DeviceGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const LaunchSet &L = p->ls;
  IoArgs a{};
  a.in0[0] = d_in;
  TOMO_TRY(timed(p, kKindSynth, s, [&] { return synthesis_of(L, 0, 0, a, s); }, "synthesis", synthesis_launches(L)));
  IoArgs b{};
  TOMO_TRY(timed(p, kKindFwd, s, [&] { return launch_forward(L.precision, 0, L.max_layers, L.elong, L.d_inst, L.fwd, L.n_fwd, b, s); },
                 "forward"));
  IoArgs c{};
  c.in1[0] = d_in;
  c.out0[0] = d_out;
  return adjoint_ls(p, L, 1, c, s);
}

tomo_status tomo_rhs(tomo_plan *p, const void *d_slopes, void *d_out, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_slopes || !d_out) return fail(TOMO_ERR_ARG, "NULL device pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const LaunchSet &L = p->ls;
  IoArgs a{};
  a.in1[0] = d_slopes;
  TOMO_TRY(timed(p, kKindFwd, s, [&] { return launch_forward(L.precision, 2, L.max_layers, L.elong, L.d_inst, L.fwd, L.n_fwd, a, s); },
                 "forward (data)"));
  IoArgs c{};
  c.out0[0] = d_out;
  c.in1[0] = d_slopes;
  return adjoint_ls(p, L, 0, c, s);
}

tomo_status tomo_jacobi_diagonal(tomo_plan *p, double *d_out, void *cuda_stream) {
  TOMO_TRY(check_plan(p));
  if (!d_out) return fail(TOMO_ERR_ARG, "NULL device pointer");
  DeviceGuard dg(p->device);
  TOMO_CUDA(cudaMemcpyAsync(d_out, p->d_jdiag, sizeof(double) * p->hp.n, cudaMemcpyDeviceToDevice,
                            static_cast<cudaStream_t>(cuda_stream)),
            "copying the Jacobi diagonal");
  return TOMO_OK;
}

tomo_status tomo_solve_batch(tomo_plan *const *plans, const void *const *d_slopes, void *const *d_coeffs,
                             int count, int iters, int warm, void *cuda_stream) {
  if (!plans || !d_slopes || !d_coeffs || count < 0) return fail(TOMO_ERR_ARG, "NULL array or negative count");
  if (count == 0) return TOMO_OK;
  if (iters < 0 || iters > 100000) return fail(TOMO_ERR_ARG, "iters out of range");
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !d_slopes[i] || !d_coeffs[i]) return fail(TOMO_ERR_ARG, "NULL plan or buffer in the batch");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(TOMO_ERR_ARG, "a plan appears twice in one batch");
  }
  int broke = -1;
  for (int i = 0; i < count; ++i)
    if (take_breakdown(plans[i]) && broke < 0) broke = i;
  if (broke >= 0)
    return fail(TOMO_ERR_BREAKDOWN, "an earlier solve of plan " + std::to_string(broke) +
                                        " of the batch (and of any other plan whose word was set) broke down "
                                        "and froze its iterate; this call enqueued nothing");
  NvtxRange nvtx("tomo_solve_batch");
  Batch *b = nullptr;
  TOMO_TRY(get_batch(plans, count, &b));
  DeviceGuard dg(b->device);
  return batch_solve(b, d_slopes, d_coeffs, nullptr, iters, warm ? 1 : 0,
                     static_cast<cudaStream_t>(cuda_stream));
}

}  // extern "C"
