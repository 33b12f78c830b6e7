// Measurement utility: the read bandwidth of the L2 cache, the denominator of the
// L2 fractions that the benchmark reports.  Not part of the method.
#include <algorithm>
#include <string>

#include <cuda_runtime.h>

#include "../../include/tomo.h"
#include "plan_internal.h"

namespace {

constexpr int kProbeThreads = 512;

// Every pass reads the whole buffer once: in pass k, CTA b reads the slice of
// CTA (b + k) mod G, so no SM reads the same lines twice in a row; the loads
// bypass L1 (ld.global.cg), so they are served by the L2 once the buffer is
// resident there.  The sum is stored only if it takes an impossible value,
// which keeps the loads without writing anything.
__global__ void __launch_bounds__(kProbeThreads) k_l2_read(float4 *buf, long long n4, int passes) {
  const int G = gridDim.x;
  const long long per = (n4 + G - 1) / G;
  float acc = 0.0f;
  for (int k = 0; k < passes; ++k) {
    const long long s = static_cast<long long>((blockIdx.x + k) % G) * per;
    const long long e = s + per < n4 ? s + per : n4;
    long long i = s + threadIdx.x;
    for (; i + 3 * kProbeThreads < e; i += 4 * kProbeThreads) {
      const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + kProbeThreads);
      const float4 c = __ldcg(buf + i + 2 * kProbeThreads), d = __ldcg(buf + i + 3 * kProbeThreads);
      acc += (a.x + b.y) + (c.z + d.w);
    }
    for (; i < e; i += kProbeThreads) acc += __ldcg(buf + i).x;
  }
  if (acc == -1.2345e-38f) buf[blockIdx.x] = make_float4(acc, acc, acc, acc);
}

}  // namespace

extern "C" tomo_status tomo_probe_l2_read(void *d_buf, long long bytes, int passes, int reps,
                                          void *cuda_stream, double *out_gbs) {
  if (!d_buf || !out_gbs || bytes < 16 || (reinterpret_cast<uintptr_t>(d_buf) & 15) || passes < 1 || reps < 1)
    return tomo::set_error(TOMO_ERR_ARG, "tomo_probe_l2_read: a 16-byte aligned buffer of >= 16 bytes, "
                                         "passes >= 1 and reps >= 1 are required");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_read, kProbeThreads, 0);
  const long long n4 = bytes / 16;
  const int grid = std::max(1, sms * std::max(1, per_sm));
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float4 *buf = static_cast<float4 *>(d_buf);
  // one launch to bring the buffer into the L2, then the timed ones
  if (e == cudaSuccess) {
    k_l2_read<<<grid, kProbeThreads, 0, s>>>(buf, n4, 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    k_l2_read<<<grid, kProbeThreads, 0, s>>>(buf, n4, passes);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return tomo::set_error(TOMO_ERR_CUDA, std::string("tomo_probe_l2_read: ") + cudaGetErrorString(e));
  tomo::count_launches(1 + reps);
  *out_gbs = static_cast<double>(n4) * 16.0 * passes * reps / (ms * 1e-3) / 1e9;
  return TOMO_OK;
}
