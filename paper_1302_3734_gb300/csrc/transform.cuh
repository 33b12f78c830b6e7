// Device helpers shared by the transform kernels: asynchronous copies to shared
// memory, the instance descriptor copy, the Daubechies filter taps in registers
// and the epilogue of the analysis.
#pragma once

#include <cuda_runtime.h>

#include "common.h"
#include "device_util.cuh"

#include <stdint.h>

namespace tomo {

// Asynchronous global -> shared copies (cp.async: 16 bytes through L2 only,
// or one element) and their completion for the calling thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(__cvta_generic_to_global(gmem))
               : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(__cvta_generic_to_global(gmem))
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(__cvta_generic_to_global(gmem))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy one instance descriptor into shared memory.
__device__ __forceinline__ void load_inst(InstDev *dst, const InstDev *src) {
  const int nw = sizeof(InstDev) / sizeof(int);
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

template <typename T, int LF>
struct Filt {
  T h[LF], g[LF];
  // taps 2s + parity without a runtime array index
  __device__ __forceinline__ T hs(int parity, int s) const { return parity ? h[2 * s + 1] : h[2 * s]; }
  __device__ __forceinline__ T gs(int parity, int s) const { return parity ? g[2 * s + 1] : g[2 * s]; }
  __device__ __forceinline__ void load(const InstDev &I) {
#pragma unroll
    for (int t = 0; t < LF; ++t) {
      h[t] = T(I.h[t]);
      g[t] = T(I.g[t]);
    }
  }
};

// Epilogue of the analysis for one output coefficient.
enum Epi : int { kEpiPlain = 0, kEpiOp = 1, kEpiResid = 2 };

template <typename T, int EPI>
struct Emit {
  T *out;          // plain: destination
  const T *P;      // op: direction p (global), cached copy in `cache`
  T *Q;            // op: q
  T *R, *Pn, *X;   // resid: r, p, x
  const T *jinv;
  const T *cache;
  const T *dalpha; // alpha D per level
  int off, N, precond, warm;
  Acc<T> acc0, acc1;
  // What the epilogue of (row, col) reads besides w: p (op) or x (warm
  // residual), from the cache when slot >= 0, and J^-1 (residual).  Fetched
  // ahead so that several outputs' loads are in flight together.
  struct Pre {
    T a, j;
  };
  __device__ __forceinline__ Pre fetch(int row, int col, int slot) const {
    Pre f{T(0), T(1)};
    const int idx = off + row * N + col;
    if (EPI == kEpiOp) {
      f.a = slot >= 0 ? cache[slot] : P[idx];
    } else if (EPI == kEpiResid) {
      if (warm) f.a = slot >= 0 ? cache[slot] : X[idx];
      if (precond) f.j = jinv[idx];
    }
    return f;
  }
  __device__ __forceinline__ void put(int row, int col, int level, T w, const Pre &f) {
    const int idx = off + row * N + col;
    if (EPI == kEpiPlain) {
      out[idx] = w;
    } else if (EPI == kEpiOp) {
      const T q = w + dalpha[level] * f.a;
      Q[idx] = q;
      acc0.add_prod(f.a, q);
    } else {
      T r = w;
      if (warm) r -= dalpha[level] * f.a;
      else X[idx] = T(0);
      const T z = precond ? f.j * r : r;
      R[idx] = r;
      Pn[idx] = z;
      acc0.add_prod(r, z);
      acc1.add_prod(r, r);
    }
  }
  __device__ __forceinline__ void operator()(int row, int col, int level, T w, int slot) {
    put(row, col, level, w, fetch(row, col, slot));
  }
};

// The direction p of PCG iteration `iter` (streamed plans alternate two buffers).
template <typename T>
__device__ __forceinline__ T *dir_buffer(const InstDev &I, int iter) {
  return static_cast<T *>((I.p2 && (iter & 1)) ? I.p2 : I.p);
}

}  // namespace tomo
