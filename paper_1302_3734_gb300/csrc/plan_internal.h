// Internal definition of the plan object shared by the C-ABI translation units.
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/tomo.h"
#include "common.h"
#include "host_plan.h"

namespace tomo {

enum Kind : int { kKindSynth = 0, kKindFwd = 1, kKindAnalysis = 2, kKindUpd = 3, kKindOther = 4, kKindGather = 5,
                  kNumKinds = 6 };

// Everything one launch sequence needs (one plan, or a batch of plans).
struct LaunchSet {
  const InstDev *d_inst = nullptr;
  int count = 0;
  const ClusterItem *cl = nullptr;
  int n_cl = 0, C = 0;
  size_t smem = 0, smem_a = 0;   // synthesis / analysis dynamic shared memory
  const FwdItem *fwd = nullptr;
  int n_fwd = 0, max_layers = 0, lf = 0;
  const UpdItem *upd = nullptr;
  int n_upd = 0;
  int precision = 0;
  int split = 0;                 // gather in its own kernel (tables not staged in shared memory)
  size_t smem_g = 0;             // its dynamic shared memory
  int gather_vs = 0;             // it stages the band rows of v in shared memory
  const PassItem *gi = nullptr;  // its CTAs' (instance, layer, band), costliest first
  int n_gi = 0;
  int elong = 0;                 // some sensor has elongated spots (k_forward variant)
  int stream = 0;                // streamed transforms (level passes over row tiles, no clusters)
  StreamSet ss;                  // their work items
};

struct Timer {
  bool on = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

struct GraphEntry {
  const void *slopes;
  void *x;
  int iters, warm;
  cudaGraphExec_t exec;
  int kernels;
};

// Record the thread-local message returned by tomo_last_error().
tomo_status set_error(tomo_status st, const std::string &msg);

// Add k kernel launches to the count tomo_launch_count() reports.
void count_launches(long long k);

// An NVTX range over the guard's lifetime (a no-op unless a profiler is attached):
// the public entry points mark their host-side enqueue work with it.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Makes `dev` the current device for the guard's lifetime.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace tomo

struct tomo_plan {
  tomo::HostPlan hp;
  int device = 0;
  size_t esz = 4;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  tomo::InstDev h_inst{};
  tomo::InstDev *d_inst = nullptr;
  double *d_jdiag = nullptr;
  tomo::LaunchSet ls;
  int nc_max = 0, max_sub2 = 0;
  cudaStream_t cap_stream = nullptr;
  int use_graphs = 1;
  std::vector<tomo::GraphEntry> graphs;
  tomo::Timer timer;
  double kind_ms[tomo::kNumKinds] = {0};
  long long kind_n[tomo::kNumKinds] = {0};
  int *bd_host = nullptr;     // breakdown word (page-locked, mapped; h_inst.bd_word on the device)
};

namespace tomo {

// Plans solved together: grouped by (cluster size, filter length, precision),
// one launch per group and phase.  Built once per distinct list of plans and
// cached; a plan's destruction drops every batch that contains it.
struct BatchGroup {
  LaunchSet ls;
  std::vector<int> members;   // position in the batch of each instance slot
  void *arena = nullptr;
  size_t bytes = 0;           // device bytes of the group's tables
};

struct BatchGraph {
  std::vector<const void *> slopes;
  std::vector<void *> x;
  const int *active;
  int iters, warm;
  cudaGraphExec_t exec;
  int kernels;
};

struct Batch {
  std::vector<tomo_plan *> plans;
  std::vector<BatchGroup> groups;
  std::vector<BatchGraph> graphs;
  cudaStream_t cap = nullptr;
  int device = 0;
};

// Build a batch of plans (all on one device); free it with free_batch.
tomo_status build_batch(tomo_plan *const *plans, int count, Batch **out);
void free_batch(Batch *b);
// One solve of every active instance of the batch on stream s, replayed from
// a graph cached per (iters, warm, active masks, slope and coefficient
// pointers).  active_g: per launch group a device array of one int per group
// slot (nonzero = solve), or NULL for all.
tomo_status batch_solve(Batch *b, const void *const *slopes, void *const *x, const int *const *active_g,
                        int iters, int warm, cudaStream_t s);

// W^-1 over a launch set (cluster or streamed kernels); src 0: io.in0
// coefficients, 1: the PCG direction update fused in.  synthesis_launches: the
// kernels one call launches.
cudaError_t synthesis_of(const LaunchSet &L, int src, int flags, const IoArgs &io, cudaStream_t s);
int synthesis_launches(const LaunchSet &L);

// Reads and clears plan p's breakdown word: true when a solve of p has broken
// down since the word was last cleared (only work that has completed on the
// device is seen).
inline bool take_breakdown(tomo_plan *p) {
  volatile int *w = p->bd_host;
  if (!w || *w == 0) return false;
  *w = 0;
  return true;
}

// Enqueue one solve of plan p on stream s, kernel by kernel (for capture into
// a caller's graph); *n_kernels receives the number of launches.
tomo_status enqueue_plan_solve(tomo_plan *p, const void *slopes, void *x, int iters, int warm, cudaStream_t s,
                               int *n_kernels);

}  // namespace tomo
