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

// Bulk (TMA) copies global -> shared that complete on an mbarrier: one thread
// initialises the barrier (count 1), arms it with the byte count and issues the
// copies (16-byte aligned addresses, sizes a multiple of 16); every thread then
// waits for phase 0.  The wait gives up after kMbarSpins polls (each may suspend
// the thread for a while) and returns false.
constexpr int kMbarSpins = 1 << 20;
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// arrive once, expecting `bytes` of copies (0: the phase completes now)
__device__ __forceinline__ void mbar_arm(uint64_t *bar, uint32_t bytes) {
  if (bytes == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
  else
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// global data that an earlier grid wrote, about to be read by bulk copies
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int i = 0; i < kMbarSpins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

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
  // FP32: the descriptor's FP32 copies of the taps; FP64: the taps themselves
  __device__ __forceinline__ void load(const InstDev &I) {
#pragma unroll
    for (int t = 0; t < LF; ++t) {
      if constexpr (sizeof(T) == 4) {
        h[t] = I.hf[t];
        g[t] = I.gf[t];
      } else {
        h[t] = I.h[t];
        g[t] = I.g[t];
      }
    }
  }
};

// Row analysis (x) of `rows` rows of side M = 2^lgM: the low half
// B[j][i] = sum_t h[t] X[j][(2i + t) mod M] and the high half B[j][H + i] with
// g, each sum over t = 0..LF-1 in that order, as in every other form of the
// transform (so the results are the same bits).  FP32 rows of M >= 8 give a
// thread two neighbouring output pairs from one window of LF + 2 inputs read
// as 16-byte vectors (aligned: rows start on 16 bytes and the window on a
// multiple of four, which also keeps the periodic wrap inside a vector);
// other rows take one pair per thread.
template <typename T, int LF>
__device__ __forceinline__ void row_analysis(const Filt<T, LF> &f, const T *X, T *B, int rows, int lgM, int tid,
                                             int nt) {
  const int M = 1 << lgM, H = M >> 1;
  if constexpr (sizeof(T) == 4) {
    if (lgM >= 3) {
      constexpr int NV = (LF + 5) / 4;   // vectors of a window of LF + 2 inputs
      const int lgQ = lgM - 2;
      for (int idx = tid; idx < (rows << lgQ); idx += nt) {
        const int j = idx >> lgQ, q = idx & ((1 << lgQ) - 1);
        const T *row = X + (j << lgM);
        T w[4 * NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const float4 v = *reinterpret_cast<const float4 *>(row + ((4 * q + 4 * c) & (M - 1)));
          w[4 * c] = v.x;
          w[4 * c + 1] = v.y;
          w[4 * c + 2] = v.z;
          w[4 * c + 3] = v.w;
        }
        T lo0 = T(0), hi0 = T(0), lo1 = T(0), hi1 = T(0);
#pragma unroll
        for (int t = 0; t < LF; ++t) {
          lo0 += f.h[t] * w[t];
          hi0 += f.g[t] * w[t];
          lo1 += f.h[t] * w[t + 2];
          hi1 += f.g[t] * w[t + 2];
        }
        T *b = B + (j << lgM) + 2 * q;
        *reinterpret_cast<float2 *>(b) = make_float2(lo0, lo1);
        *reinterpret_cast<float2 *>(b + H) = make_float2(hi0, hi1);
      }
      return;
    }
  }
  const int lgH = lgM - 1;
  for (int idx = tid; idx < rows * H; idx += nt) {
    const int j = idx >> lgH, i = idx & (H - 1);
    const T *row = X + j * M;
    T lo = T(0), hi = T(0);
#pragma unroll
    for (int t = 0; t < LF; ++t) {
      const T x = row[(2 * i + t) & (M - 1)];
      lo += f.h[t] * x;
      hi += f.g[t] * x;
    }
    B[j * M + i] = lo;
    B[j * M + H + i] = hi;
  }
}

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
