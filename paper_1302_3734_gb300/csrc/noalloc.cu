// tomo_jacobi_diagonal_noalloc: the modified Jacobi diagonal recomputed without
// any device allocation.
//
// The plan-time computation of the diagonal needs scratch device memory for the
// separable basis profiles, their offsets and the FP64 corner fractions, which
// tomo_plan_create takes from a temporary cudaMalloc.  Some callers cannot
// allocate at the moment they need the diagonal again: a real-time control
// thread that retunes the regularisation weight alpha must not touch the
// allocator (a cudaMalloc can take milliseconds and serialises with the whole
// device), and code running inside another framework's memory pool may have no
// allocator of its own.  This variant keeps that scratch in a file-scope device
// array instead.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/tomo.h"
#include "launch.h"
#include "plan_internal.h"

namespace {

// Every GPU that loads this library holds these 4 MiB until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[64] = {};   // device address of g_noalloc_scratch, per device ordinal

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" tomo_status tomo_jacobi_diagonal_noalloc(const tomo_plan *p, double alpha, double *d_out,
                                                    void *cuda_stream) {
  using tomo::set_error;
  if (!p || !d_out) return set_error(TOMO_ERR_ARG, "plan and output must not be NULL");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return set_error(TOMO_ERR_ARG, "alpha must be finite and >= 0");
  const tomo::HostPlan &H = p->hp;
  const size_t b_prof = round256(sizeof(double) * H.profiles.size());
  const size_t b_off = round256(sizeof(int) * H.prof_off.size());
  const size_t b_pos = round256(sizeof(double) * H.pos_f.size());
  if (b_prof + b_off + b_pos > kNoAllocScratchBytes) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "tomo_jacobi_diagonal_noalloc: the plan needs %zu bytes of scratch, above the fixed "
             "maximum of %zu bytes; use tomo_plan_create's diagonal (tomo_jacobi_diagonal) instead",
             b_prof + b_off + b_pos, kNoAllocScratchBytes);
    return set_error(TOMO_ERR_UNSUPPORTED, buf);
  }
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != p->device) e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return set_error(TOMO_ERR_CUDA, std::string("selecting the plan's device: ") + cudaGetErrorString(e));
  // First call on this device: look up the array's device address (the host
  // symbol g_noalloc_scratch is only a stand-in, not a device pointer).
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (p->device < 0 || p->device >= 64) {
      e = cudaErrorInvalidDevice;
    } else if (!g_scratch_ptr[p->device]) {
      e = cudaGetSymbolAddress(&g_scratch_ptr[p->device], g_noalloc_scratch);
    }
    base = e == cudaSuccess ? g_scratch_ptr[p->device] : nullptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  char *sb = static_cast<char *>(base);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sb, H.profiles.data(), sizeof(double) * H.profiles.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sb + b_prof, H.prof_off.data(), sizeof(int) * H.prof_off.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sb + b_prof + b_off, H.pos_f.data(), sizeof(double) * H.pos_f.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = tomo::launch_jacobi(p->d_inst, H.n, reinterpret_cast<const double *>(sb),
                            reinterpret_cast<const int *>(sb + b_prof),
                            reinterpret_cast<const double *>(sb + b_prof + b_off), d_out, nullptr,
                            H.precision, p->nc_max, alpha, s);
  if (e == cudaSuccess) tomo::count_launches(1);
  if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
  if (e != cudaSuccess)
    return set_error(TOMO_ERR_CUDA, std::string("tomo_jacobi_diagonal_noalloc: ") + cudaGetErrorString(e));
  return TOMO_OK;
}
