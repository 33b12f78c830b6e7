// Device-side helpers shared by the kernel translation units: programmatic
// dependent launch, the inner-product accumulators and their fixed-order block
// reductions, and the launch helper.
#pragma once

#include <cuda_runtime.h>

#include "common.h"

namespace tomo {

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inner-product accumulator of one thread.  FP64 plans: a double.  FP32
// plans: an unevaluated double-float sum hi + lo (about 48 significant bits)
// on the FP32 pipes: the product of two floats enters exactly (the FMA gives
// the rounding error of a*b) and additions use Knuth's two-sum, so the error
// stays close to an FP64 accumulation while the FP64 pipe, a small fraction
// of the FP32 rate on this GPU, is left to the cross-block sums.  The _rn
// intrinsics keep the compiler from contracting the error-free steps.
template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { s += a * b; }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(hi, x);
    const float bp = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    hi = t;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  // this += o, renormalised so that |lo| <= ulp(hi) / 2
  __device__ __forceinline__ void merge(float ohi, float olo) {
    add(ohi);
    lo = __fadd_rn(lo, olo);
    const float t = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(t, hi));
    hi = t;
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Sum of (a, b) over the block; the result is returned to every thread.
// Fixed order: lane trees in each warp, then the warps' sums in warp 0.
static __device__ double2 block_sum2(Acc<double> aa, Acc<double> bb) {
  __shared__ double s_red[2][32];
  __shared__ double2 s_out;
  const double a = warp_sum(aa.s), b = warp_sum(bb.s);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[0][w] = a;
    s_red[1][w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    double x = lane < nw ? s_red[0][lane] : 0.0;
    double y = lane < nw ? s_red[1][lane] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    if (lane == 0) s_out = make_double2(x, y);
  }
  __syncthreads();
  return s_out;
}

__device__ __forceinline__ void warp_merge_down(Acc<float> &a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_down_sync(0xffffffffu, a.hi, o);
    const float l = __shfl_down_sync(0xffffffffu, a.lo, o);
    a.merge(h, l);
  }
}

static __device__ double2 block_sum2(Acc<float> a, Acc<float> b) {
  __shared__ float s_red[4][32];
  __shared__ double2 s_out;
  warp_merge_down(a);   // lane 0 holds the warp's sum
  warp_merge_down(b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[0][w] = a.hi;
    s_red[1][w] = a.lo;
    s_red[2][w] = b.hi;
    s_red[3][w] = b.lo;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    Acc<float> x, y;
    if (lane < nw) {
      x.hi = s_red[0][lane];
      x.lo = s_red[1][lane];
      y.hi = s_red[2][lane];
      y.lo = s_red[3][lane];
    }
    warp_merge_down(x);
    warp_merge_down(y);
    if (lane == 0) s_out = make_double2(x.value(), y.value());
  }
  __syncthreads();
  return s_out;
}

// The block's double-float sums of (a, b) as (a.hi, a.lo, b.hi, b.lo), valid
// in thread 0.  No barrier at the end: warp 0 may still read the scratch when
// the other warps return, so a second call needs a __syncthreads() first.
static __device__ float4 block_sum2_df(Acc<float> a, Acc<float> b) {
  __shared__ float s_red[4][32];
  warp_merge_down(a);
  warp_merge_down(b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[0][w] = a.hi;
    s_red[1][w] = a.lo;
    s_red[2][w] = b.hi;
    s_red[3][w] = b.lo;
  }
  __syncthreads();
  Acc<float> x, y;
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    if (lane < nw) {
      x.hi = s_red[0][lane];
      x.lo = s_red[1][lane];
      y.hi = s_red[2][lane];
      y.lo = s_red[3][lane];
    }
    warp_merge_down(x);
    warp_merge_down(y);
  }
  return make_float4(x.hi, x.lo, y.hi, y.lo);
}

// Fixed-order FP64 sum of component k of `count` partial pairs (stride 2),
// valid in thread 0 only: warps 0..3 take the partials w*32 + lane, + 128, ...
// (a block of fewer warps lets each take several of those four shares), each
// share's lane tree, then thread 0 adds the four in order.  Only the first
// four warps touch the FP64 pipe, a small fraction of the FP32 rate on this
// GPU, and no component is summed that the caller does not use.
static __device__ double sum_partial(const double *part, int count, int k) {
  __shared__ double s_sp[4];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int v = w; v < 4; v += nw) {
    double a = 0.0;
    for (int q = v * 32 + lane; q < count; q += 128) a += part[2 * q + k];
    a = warp_sum(a);
    if (lane == 0) s_sp[v] = a;
  }
  __syncthreads();
  return threadIdx.x == 0 ? ((s_sp[0] + s_sp[1]) + s_sp[2]) + s_sp[3] : 0.0;
}

// Every hot-path launch allows programmatic dependent launch: the kernel's
// prologue (descriptor and table loads) overlaps the previous kernel, and
// griddepcontrol.wait orders its reads of the previous kernel's results.
template <typename K, typename... Args>
cudaError_t launch_ex(K kernel, dim3 grid, int threads, int cluster, size_t smem, cudaStream_t s,
                      Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[na].val.programmaticStreamSerializationAllowed = 1;
  ++na;
  if (cluster > 0) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace tomo
