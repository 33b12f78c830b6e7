// Streamed transform kernels (sm_103a): the periodic 2-D Daubechies DWT and its
// inverse of layers too large for the cluster-per-layer kernels to keep more
// than one cluster per GPC resident, level by level over row tiles of the
// whole grid, with the PCG epilogue (Sec. 5.1, eq. eqn_lse) and the fused
// direction update of the cluster kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"
#include "device_util.cuh"
#include "launch.h"
#include "transform.cuh"

namespace tomo {

// ---------------------------------------------------- streamed transforms
// For layers whose transform kernels would hold one cluster per GPC at a time
// (the clusters' rows of the finest level do not fit two CTAs per SM), the
// transforms run level by level over row tiles of the whole grid instead, with
// no cluster: each CTA reads its halo rows from global memory (L2).  Levels
// 1..ks-1 are passes (one launch per level, kPassRows half-rows per CTA); the
// levels from block side N >> (ks-1) <= kCoarseMax on run in one CTA per layer.
// The arithmetic of every output (filter taps, order of the sums) is that of
// the cluster kernels.

// Epilogue setup shared by the streamed analysis kernels (as in k_analysis).
template <typename T, int EPI>
__device__ __forceinline__ void emit_setup(Emit<T, EPI> &emit, const InstDev &I, const LayerDev &L,
                                           const IoArgs &io, int inst, int flags, const T *dal) {
  emit.off = L.off;
  emit.N = L.N;
  emit.dalpha = dal;
  emit.precond = I.precond;
  emit.warm = (flags & kFlagWarm) ? 1 : 0;
  emit.jinv = static_cast<const T *>(I.jinv);
  emit.cache = nullptr;
  emit.out = static_cast<T *>(io.out0[inst]);
  emit.P = io.in1[inst] ? static_cast<const T *>(io.in1[inst]) : dir_buffer<T>(I, flags >> kIterShift);
  emit.Q = io.out0[inst] ? static_cast<T *>(io.out0[inst]) : static_cast<T *>(I.q);
  emit.R = static_cast<T *>(I.r);
  emit.Pn = static_cast<T *>(I.p);
  emit.X = static_cast<T *>(io.out0[inst]);
}

// Asynchronous copy of rows (first + j) & wrap, j < nrows, of M elements each from
// src (row stride `stride` elements) into the dense rows of dst: 16-byte copies
// when the rows are 16-byte aligned, else one element at a time.  Completed by
// cp_async_wait_all() and a barrier.
template <typename T>
__device__ __forceinline__ void stage_rows_async(T *dst, const T *src, int stride, int first, int nrows, int M,
                                                 int wrap) {
  constexpr int V = 16 / static_cast<int>(sizeof(T));
  const int lgM = __ffs(M) - 1;
  const bool vec = M >= V &&
                   ((reinterpret_cast<uintptr_t>(src) | (static_cast<size_t>(stride) * sizeof(T))) & 15) == 0;
  if (vec) {
    const int lgV = __ffs(V) - 1, lgMv = lgM - lgV, mv = M >> lgV;
    for (int idx = threadIdx.x; idx < nrows * mv; idx += blockDim.x) {
      const int j = idx >> lgMv, c = (idx & (mv - 1)) << lgV;
      cp_async16(dst + j * M + c, src + static_cast<size_t>((first + j) & wrap) * stride + c);
    }
  } else {
    for (int idx = threadIdx.x; idx < nrows * M; idx += blockDim.x) {
      const int j = idx >> lgM, x = idx & (M - 1);
      cp_async_elem(dst + idx, src + static_cast<size_t>((first + j) & wrap) * stride + x);
    }
  }
  cp_async_commit();
}

// Outputs of a column pass handled per thread at once: their epilogue inputs
// (p, or x and J^-1) are all requested before any is used.
constexpr int kEmitU = 4;

// One analysis level k over a tile: output half-rows [row0, row0 + kPassRows) of
// the level's M x M block.  SRC 0: level 1 reads io.in0's layer; SRC 2: the
// gathered grid in the plan's phi; levels > 1 read the previous low-low block.
// The low-low part goes to the scratch (or is emitted at k = J); the details
// are emitted.  One partial pair per CTA.
template <typename T, int SRC, int EPI, int LF>
__global__ void __launch_bounds__(kPassThreads) k_dwt_pass(const InstDev *__restrict__ insts,
                                                           const PassItem *__restrict__ items, IoArgs io,
                                                           int k, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ T s_dal[kMaxLevels + 1];
  pdl_trigger();
  const PassItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int J = I.J, tid = threadIdx.x, nt = blockDim.x;
  const int lgM = L.log2N - (k - 1), M = 1 << lgM, H = M >> 1;
  constexpr int NR = 2 * kPassRows + LF - 2;
  T *X = reinterpret_cast<T *>(smem_raw);
  T *B = X + NR * M;
  if (tid <= J) s_dal[tid] = T(L.dalpha[tid]);
  Filt<T, LF> f;
  f.load(I);
  Emit<T, EPI> emit;
  emit_setup<T, EPI>(emit, I, L, io, it.inst, flags, s_dal);
  const T *src = k > 1 ? static_cast<const T *>(I.lls) + L.ll_off[k - 1]
                       : (SRC == 0 ? static_cast<const T *>(io.in0[it.inst]) : static_cast<const T *>(I.phi)) + L.off;
  T *ll = k < J ? static_cast<T *>(I.lls) + L.ll_off[k] : nullptr;
  __syncthreads();
  pdl_wait();
  // input rows 2 row0 .. 2 row0 + NR - 1 (mod M)
  stage_rows_async<T>(X, src, M, 2 * it.row0, NR, M, M - 1);
  cp_async_wait_all();
  __syncthreads();
  // row pass (x)
  row_analysis<T, LF>(f, X, B, NR, lgM, tid, nt);
  __syncthreads();
  // column pass (y) and the epilogue, kEmitU outputs per thread at once
  for (int idx0 = tid; idx0 < kPassRows * M; idx0 += kEmitU * nt) {
    T lo[kEmitU], hi[kEmitU];
    typename Emit<T, EPI>::Pre fa[kEmitU], fb[kEmitU];
#pragma unroll
    for (int u = 0; u < kEmitU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < kPassRows * M) {
        const int il = idx >> lgM, x = idx & (M - 1);
        const int i = it.row0 + il;
        const T *col = B + 2 * il * M + x;
        T l = T(0), h = T(0);
#pragma unroll
        for (int t = 0; t < LF; ++t) {
          const T val = col[t * M];
          l += f.h[t] * val;
          h += f.g[t] * val;
        }
        lo[u] = l;
        hi[u] = h;
        if (x >= H || k == J) fa[u] = emit.fetch(i, x, -1);
        fb[u] = emit.fetch(H + i, x, -1);
      }
    }
#pragma unroll
    for (int u = 0; u < kEmitU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < kPassRows * M) {
        const int il = idx >> lgM, x = idx & (M - 1);
        const int i = it.row0 + il;
        if (x < H) {
          if (k == J) emit.put(i, x, J, lo[u], fa[u]);
          else ll[i * H + x] = lo[u];
        } else {
          emit.put(i, x, k, lo[u], fa[u]);
        }
        emit.put(H + i, x, k, hi[u], fb[u]);
      }
    }
  }
  if (EPI == kEpiPlain) return;
  const double2 s = block_sum2(emit.acc0, emit.acc1);
  if (tid == 0) {
    I.part[I.cl_part_off + 2 * it.slot] = s.x;
    I.part[I.cl_part_off + 2 * it.slot + 1] = s.y;
  }
}

// The coarse analysis levels ks..J of one layer in one CTA: the block of side
// N >> (ks - 1) from the scratch (or, ks = 1, the layer grid); every output emitted.
template <typename T, int SRC, int EPI, int LF>
__global__ void __launch_bounds__(kPassThreads) k_dwt_coarse(const InstDev *__restrict__ insts,
                                                             const PassItem *__restrict__ items, IoArgs io,
                                                             int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ T s_dal[kMaxLevels + 1];
  pdl_trigger();
  const PassItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int J = I.J, tid = threadIdx.x, nt = blockDim.x, ks = L.ks;
  int lgM = L.log2N - (ks - 1), M = 1 << lgM;
  T *A = reinterpret_cast<T *>(smem_raw);
  T *B = A + M * M;
  if (tid <= J) s_dal[tid] = T(L.dalpha[tid]);
  Filt<T, LF> f;
  f.load(I);
  Emit<T, EPI> emit;
  emit_setup<T, EPI>(emit, I, L, io, it.inst, flags, s_dal);
  const T *src = ks > 1 ? static_cast<const T *>(I.lls) + L.ll_off[ks - 1]
                        : (SRC == 0 ? static_cast<const T *>(io.in0[it.inst]) : static_cast<const T *>(I.phi)) + L.off;
  __syncthreads();
  pdl_wait();
  stage_rows_async<T>(A, src, M, 0, M, M, M - 1);
  cp_async_wait_all();
  __syncthreads();
  for (int k = ks; k <= J; ++k, M >>= 1, --lgM) {
    const int H = M >> 1;
    row_analysis<T, LF>(f, A, B, M, lgM, tid, nt);
    __syncthreads();
    for (int idx0 = tid; idx0 < H * M; idx0 += kEmitU * nt) {
      T lo[kEmitU], hi[kEmitU];
      typename Emit<T, EPI>::Pre fa[kEmitU], fb[kEmitU];
#pragma unroll
      for (int u = 0; u < kEmitU; ++u) {
        const int idx = idx0 + u * nt;
        if (idx < H * M) {
          const int i = idx >> lgM, x = idx & (M - 1);
          T l = T(0), h = T(0);
#pragma unroll
          for (int t = 0; t < LF; ++t) {
            const T val = B[((2 * i + t) & (M - 1)) * M + x];
            l += f.h[t] * val;
            h += f.g[t] * val;
          }
          lo[u] = l;
          hi[u] = h;
          if (!(x < H && k < J)) fa[u] = emit.fetch(i, x, -1);
          fb[u] = emit.fetch(H + i, x, -1);
        }
      }
#pragma unroll
      for (int u = 0; u < kEmitU; ++u) {
        const int idx = idx0 + u * nt;
        if (idx < H * M) {
          const int i = idx >> lgM, x = idx & (M - 1);
          if (x < H && k < J) A[i * H + x] = lo[u];
          else emit.put(i, x, (x < H) ? J : k, lo[u], fa[u]);
          emit.put(H + i, x, k, hi[u], fb[u]);
        }
      }
    }
    __syncthreads();
  }
  if (EPI == kEpiPlain) return;
  const double2 s = block_sum2(emit.acc0, emit.acc1);
  if (tid == 0) {
    I.part[I.cl_part_off + 2 * it.slot] = s.x;
    I.part[I.cl_part_off + 2 * it.slot + 1] = s.y;
  }
}

// beta = (r.z)_iter / (r.z)_(iter-1) from the update's partials, as k_synthesis
// forms it (0 at iteration 0 and after a breakdown); record: store (r.z)_iter
// and beta itself, which the level passes that follow read (stored_beta).
template <typename T>
__device__ __forceinline__ T streamed_beta(const InstDev &I, int iter, bool record) {
  __shared__ T s_b;
  const double prev = I.scal[kRz0 + ((iter + 1) & 1)];
  const double flag = I.scal[kFlag];
  const double rz = iter == 0 ? sum_partial(I.part + I.cl_part_off, I.n_cl_part, 0)
                              : sum_partial(I.part + I.upd_part_off, I.n_upd_blocks, 0);
  if (threadIdx.x == 0) {
    double beta = 0.0;
    if (iter > 0) {
      const bool stop = flag != 0.0 || !isfinite(rz) || !(prev != 0.0);
      beta = stop ? 0.0 : rz / prev;
    }
    s_b = T(beta);
    if (record) {
      I.scal[kRz0 + (iter & 1)] = rz;
      I.scal[kBeta] = beta;
    }
  }
  __syncthreads();
  return s_b;
}

// beta of the iteration in a level pass: the coarse synthesis kernel, launched
// before the passes of every streamed synthesis, formed and stored it, so the
// passes' many CTAs do not each sum the update's partials on the FP64 pipe.
template <typename T>
__device__ __forceinline__ T stored_beta(const InstDev &I) {
  __shared__ T s_b;
  if (threadIdx.x == 0) s_b = T(I.scal[kBeta]);
  __syncthreads();
  return s_b;
}

// A coefficient of the synthesis input: SRC 0 from io.in0; SRC 1 the PCG direction
// with its update p = J^-1 r + beta p (not at the first iteration), read from the
// previous iteration's buffer and, when `own`, written to this iteration's.
template <typename T, int SRC>
struct SynthCoef {
  const T *src, *Pin, *Rv, *Jv;
  T *Pout;
  T beta;
  bool first, pre;
  struct Raw {
    T p, r, j;
  };
  // the loads of coefficient idx (several are requested before any is used) ...
  __device__ __forceinline__ Raw load(size_t idx) const {
    Raw v{T(0), T(0), T(1)};
    if (SRC == 0) {
      v.p = src[idx];
    } else {
      v.p = Pin[idx];
      if (!first) {
        v.r = Rv[idx];
        if (pre) v.j = Jv[idx];
      }
    }
    return v;
  }
  // ... then its value, with the direction update (stored when owned)
  __device__ __forceinline__ T value(const Raw &v, size_t idx, bool own) const {
    if (SRC == 0 || first) return v.p;
    const T z = pre ? v.j * v.r : v.r;
    const T pn = z + beta * v.p;
    if (own) Pout[idx] = pn;
    return pn;
  }
};

// Coefficients (and low-low values) staged per thread at once by the synthesis kernels.
constexpr int kCoefU = 4;

// 16 bytes of T: the unit of the vector loads of the streamed synthesis pass.
template <typename T>
struct Vec16 {
  static constexpr int kN = 16 / static_cast<int>(sizeof(T));
  T v[kN];
  __device__ __forceinline__ void load(const T *p) { *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(p); }
  __device__ __forceinline__ void store(T *p) const { *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(v); }
};

template <typename T, int SRC>
__device__ __forceinline__ SynthCoef<T, SRC> synth_coef(const InstDev &I, const IoArgs &io, int inst, int flags,
                                                        T beta) {
  const int iter = flags >> kIterShift;
  SynthCoef<T, SRC> c;
  c.src = static_cast<const T *>(io.in0[inst]);
  c.Pin = dir_buffer<T>(I, iter > 0 ? iter - 1 : 0);
  c.Pout = dir_buffer<T>(I, iter);
  c.Rv = static_cast<const T *>(I.r);
  c.Jv = static_cast<const T *>(I.jinv);
  c.beta = beta;
  c.first = (flags & kFlagFirst) != 0;
  c.pre = I.precond != 0;
  return c;
}

// The coarse synthesis levels J..ks of one layer in one CTA: the coefficients of
// the pyramid's block of side N >> (ks - 1) (with the direction update, all owned
// here), the block synthesised level by level (rows, then columns), the result
// to the scratch (the low-low input of level ks - 1) or, ks = 1, the output grid.
// With SRC 1 this kernel records (r.z) and beta of the iteration.
template <typename T, int SRC, int LF>
__global__ void __launch_bounds__(kPassThreads) k_idwt_coarse(const InstDev *__restrict__ insts,
                                                              const PassItem *__restrict__ items, IoArgs io,
                                                              int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  pdl_trigger();
  const PassItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int J = I.J, tid = threadIdx.x, nt = blockDim.x, ks = L.ks, N = L.N;
  const int lgM0 = L.log2N - (ks - 1), M0 = 1 << lgM0;
  T *Cf = reinterpret_cast<T *>(smem_raw);   // the coefficient block, M0 x M0
  T *A = Cf + M0 * M0;                       // the current low-low block
  T *XL = A + M0 * M0;                       // row syntheses of the low-y and high-y rows
  T *XH = XL + (M0 >> 1) * M0;
  Filt<T, LF> f;
  f.load(I);
  pdl_wait();
  const T beta = SRC == 1 ? streamed_beta<T>(I, flags >> kIterShift, true) : T(0);
  const SynthCoef<T, SRC> coef = synth_coef<T, SRC>(I, io, it.inst, flags, beta);
  for (int idx0 = tid; idx0 < M0 * M0; idx0 += kCoefU * nt) {
    typename SynthCoef<T, SRC>::Raw raw[kCoefU];
#pragma unroll
    for (int u = 0; u < kCoefU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < M0 * M0)
        raw[u] = coef.load(static_cast<size_t>(L.off) + static_cast<size_t>(idx >> lgM0) * N + (idx & (M0 - 1)));
    }
#pragma unroll
    for (int u = 0; u < kCoefU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < M0 * M0)
        Cf[idx] = coef.value(raw[u], static_cast<size_t>(L.off) + static_cast<size_t>(idx >> lgM0) * N + (idx & (M0 - 1)),
                             true);
    }
  }
  __syncthreads();
  {
    const int HJ = (N >> (J - 1)) >> 1;
    for (int idx = tid; idx < HJ * HJ; idx += nt) A[idx] = Cf[(idx / HJ) * M0 + idx % HJ];
  }
  __syncthreads();
  for (int k = J; k >= ks; --k) {
    const int lgM = L.log2N - (k - 1), M = 1 << lgM, H = M >> 1;
    // row synthesis (x) of the low-y rows [LL | HL] into XL and the high-y rows [LH | HH] into XH
    const int lgH = lgM - 1;
    for (int idx = tid; idx < 2 * H * H; idx += nt) {
      const int r = idx >> lgH, m = idx & (H - 1);
      const bool high = r >= H;
      const int ii = high ? r - H : r;
      T even = T(0), odd = T(0);
#pragma unroll
      for (int s = 0; s < LF / 2; ++s) {
        const int jj = (m - s) & (H - 1);
        const T lo = high ? Cf[(H + ii) * M0 + jj] : A[ii * H + jj];
        const T hi = Cf[(high ? H + ii : ii) * M0 + H + jj];
        even += f.h[2 * s] * lo + f.g[2 * s] * hi;
        odd += f.h[2 * s + 1] * lo + f.g[2 * s + 1] * hi;
      }
      T *xr = (high ? XH : XL) + ii * M + 2 * m;
      xr[0] = even;
      xr[1] = odd;
    }
    __syncthreads();
    // column synthesis (y): the block of side M, the next level's low-low block
    for (int idx = tid; idx < H * M; idx += nt) {
      const int b = idx >> lgM, x = idx & (M - 1);
      T even = T(0), odd = T(0);
#pragma unroll
      for (int s = 0; s < LF / 2; ++s) {
        const int ii = (b - s) & (H - 1);
        const T xl = XL[ii * M + x], xh = XH[ii * M + x];
        even += f.h[2 * s] * xl + f.g[2 * s] * xh;
        odd += f.h[2 * s + 1] * xl + f.g[2 * s + 1] * xh;
      }
      A[(2 * b) * M + x] = even;
      A[(2 * b + 1) * M + x] = odd;
    }
    __syncthreads();
  }
  T *out = ks > 1 ? static_cast<T *>(I.lls) + L.ll_off[ks - 1]
                  : (io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.phi)) + L.off;
  const int stride = ks > 1 ? M0 : N;
  for (int idx = tid; idx < M0 * M0; idx += nt) out[(idx >> lgM0) * stride + (idx & (M0 - 1))] = A[idx];
}

// One synthesis level k over a tile: output rows [2 row0, 2 row0 + 2 kPassRows) of
// the level's M x M block, from the low-low block of level k (scratch) and the
// level's detail coefficients (with the direction update; the tile owns
// half-rows [row0, row0 + kPassRows) and writes their updated directions).  The
// HL = LF/2 - 1 half-rows before the tile are read too.  Output to the scratch
// (the low-low block of level k - 1) or, k = 1, the output grid.
template <typename T, int SRC, int LF>
__global__ void __launch_bounds__(kPassThreads, 2) k_idwt_pass(const InstDev *__restrict__ insts,
                                                            const PassItem *__restrict__ items, IoArgs io,
                                                            int k, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  constexpr int HL = LF / 2 - 1, NI = kPassRows + HL;
  pdl_trigger();
  const PassItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int tid = threadIdx.x, nt = blockDim.x, N = L.N;
  const int lgM = L.log2N - (k - 1), M = 1 << lgM, H = M >> 1;
  T *VL = reinterpret_cast<T *>(smem_raw);   // NI low-y rows [LL | HL], then NI high-y rows [LH | HH]
  T *VH = VL + NI * M;
  T *XL = VH + NI * M;
  T *XH = XL + NI * M;
  Filt<T, LF> f;
  f.load(I);
  const T *ll = static_cast<const T *>(I.lls) + L.ll_off[k];
  pdl_wait();
  const T beta = SRC == 1 ? stored_beta<T>(I) : T(0);
  const SynthCoef<T, SRC> coef = synth_coef<T, SRC>(I, io, it.inst, flags, beta);
  // the tile's coefficient rows: 16-byte vectors when every source is aligned (the plan's
  // buffers are; a caller's coefficient vector may not be), else kCoefU positions per
  // thread loaded before any is used
  constexpr int VN = Vec16<T>::kN;
  const bool vec = (((reinterpret_cast<uintptr_t>(SRC == 0 ? coef.src : coef.Pin) |
                      reinterpret_cast<uintptr_t>(coef.Rv) | reinterpret_cast<uintptr_t>(coef.Jv) |
                      reinterpret_cast<uintptr_t>(coef.Pout) | reinterpret_cast<uintptr_t>(ll)) & 15) == 0) &&
                   ((L.off & (VN - 1)) == 0) && H >= VN;
  if (vec) {
    const int lgMv = lgM - (__ffs(VN) - 1), mv = M / VN;
    for (int q = tid; q < NI * mv; q += nt) {
      const int j = q >> lgMv, x = (q & (mv - 1)) * VN;
      const int ii = (it.row0 - HL + j) & (H - 1);
      const bool own = j >= HL;
      const size_t lo = static_cast<size_t>(L.off) + static_cast<size_t>(ii) * N + x;
      const size_t hi = static_cast<size_t>(L.off) + static_cast<size_t>(H + ii) * N + x;
      Vec16<T> a, b, ar, br, aj, bj;
      // requests first: the low-y row's low-low values or coefficients, the high-y row's coefficients
      if (x < H) {
        a.load(ll + ii * H + x);
      } else if (SRC == 0) {
        a.load(coef.src + lo);
      } else {
        a.load(coef.Pin + lo);
        if (!coef.first) {
          ar.load(coef.Rv + lo);
          if (coef.pre) aj.load(coef.Jv + lo);
        }
      }
      if (SRC == 0) {
        b.load(coef.src + hi);
      } else {
        b.load(coef.Pin + hi);
        if (!coef.first) {
          br.load(coef.Rv + hi);
          if (coef.pre) bj.load(coef.Jv + hi);
        }
      }
      if (SRC == 1 && !coef.first) {
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          if (x >= H) a.v[e] = (coef.pre ? aj.v[e] * ar.v[e] : ar.v[e]) + coef.beta * a.v[e];
          b.v[e] = (coef.pre ? bj.v[e] * br.v[e] : br.v[e]) + coef.beta * b.v[e];
        }
        if (own) {
          if (x >= H) a.store(coef.Pout + lo);
          b.store(coef.Pout + hi);
        }
      }
      a.store(VL + j * M + x);
      b.store(VH + j * M + x);
    }
  } else
  for (int idx0 = tid; idx0 < NI * M; idx0 += kCoefU * nt) {
    typename SynthCoef<T, SRC>::Raw ra[kCoefU], rb[kCoefU];
#pragma unroll
    for (int u = 0; u < kCoefU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < NI * M) {
        const int j = idx >> lgM, x = idx & (M - 1);
        const int ii = (it.row0 - HL + j) & (H - 1);
        if (x < H) ra[u].p = ll[ii * H + x];
        else ra[u] = coef.load(static_cast<size_t>(L.off) + static_cast<size_t>(ii) * N + x);
        rb[u] = coef.load(static_cast<size_t>(L.off) + static_cast<size_t>(H + ii) * N + x);
      }
    }
#pragma unroll
    for (int u = 0; u < kCoefU; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < NI * M) {
        const int j = idx >> lgM, x = idx & (M - 1);
        const int ii = (it.row0 - HL + j) & (H - 1);
        const bool own = j >= HL;
        VL[idx] = x < H ? ra[u].p : coef.value(ra[u], static_cast<size_t>(L.off) + static_cast<size_t>(ii) * N + x, own);
        VH[idx] = coef.value(rb[u], static_cast<size_t>(L.off) + static_cast<size_t>(H + ii) * N + x, own);
      }
    }
  }
  __syncthreads();
  // row synthesis (x): outputs 2m and 2m + 1 of a row from the same taps.  VH
  // follows VL (rows NI.. are the high-y rows) and XH follows XL.
  const int lgH = lgM - 1;
  bool rows_done = false;
  if constexpr (sizeof(T) == 4 && LF <= 10) {
    if (lgH >= 2) {
      // FP32: four neighbouring m per thread from the low and high halves'
      // inputs m - 4 .. m + 3, two 16-byte vectors each (a multiple of four,
      // so a vector never straddles the periodic wrap), every output's sum in
      // the order of the scalar form below
      const int lgQ = lgH - 2;
      for (int idx = tid; idx < ((2 * NI) << lgQ); idx += nt) {
        const int r = idx >> lgQ, m0 = (idx & ((1 << lgQ) - 1)) << 2;
        const T *row = VL + r * M;
        T lo[8], hi[8];
        *reinterpret_cast<float4 *>(lo) = *reinterpret_cast<const float4 *>(row + ((m0 - 4) & (H - 1)));
        *reinterpret_cast<float4 *>(lo + 4) = *reinterpret_cast<const float4 *>(row + m0);
        *reinterpret_cast<float4 *>(hi) = *reinterpret_cast<const float4 *>(row + H + ((m0 - 4) & (H - 1)));
        *reinterpret_cast<float4 *>(hi + 4) = *reinterpret_cast<const float4 *>(row + H + m0);
        T o[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          T even = T(0), odd = T(0);
#pragma unroll
          for (int s = 0; s < LF / 2; ++s) {
            const T l = lo[4 + u - s], h = hi[4 + u - s];
            even += f.h[2 * s] * l + f.g[2 * s] * h;
            odd += f.h[2 * s + 1] * l + f.g[2 * s + 1] * h;
          }
          o[2 * u] = even;
          o[2 * u + 1] = odd;
        }
        T *x = XL + r * M + 2 * m0;
        *reinterpret_cast<float4 *>(x) = *reinterpret_cast<const float4 *>(o);
        *reinterpret_cast<float4 *>(x + 4) = *reinterpret_cast<const float4 *>(o + 4);
      }
      rows_done = true;
    }
  }
  if (!rows_done)
  for (int idx = tid; idx < 2 * NI * H; idx += nt) {
    const int r = idx >> lgH, m = idx & (H - 1);
    const T *row = VL + r * M;
    T even = T(0), odd = T(0);
#pragma unroll
    for (int s = 0; s < LF / 2; ++s) {
      const int jj = (m - s) & (H - 1);
      const T lo = row[jj], hi = row[H + jj];
      even += f.h[2 * s] * lo + f.g[2 * s] * hi;
      odd += f.h[2 * s + 1] * lo + f.g[2 * s + 1] * hi;
    }
    XL[r * M + 2 * m] = even;
    XL[r * M + 2 * m + 1] = odd;
  }
  __syncthreads();
  T *out = k > 1 ? static_cast<T *>(I.lls) + L.ll_off[k - 1]
                 : (io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.phi)) + L.off;
  const int stride = k > 1 ? M : N;
  // column synthesis (y): output rows 2b and 2b + 1 from the same half-rows
  for (int idx = tid; idx < kPassRows * M; idx += nt) {
    const int b = idx >> lgM, x = idx & (M - 1);
    const int base = b + HL;
    T even = T(0), odd = T(0);
#pragma unroll
    for (int s = 0; s < LF / 2; ++s) {
      const T xl = XL[(base - s) * M + x], xh = XH[(base - s) * M + x];
      even += f.h[2 * s] * xl + f.g[2 * s] * xh;
      odd += f.h[2 * s + 1] * xl + f.g[2 * s + 1] * xh;
    }
    T *o = out + (2 * it.row0 + 2 * b) * stride + x;
    o[0] = even;
    o[stride] = odd;
  }
}


namespace {

template <typename T, int LF>
cudaError_t synth_streamed(int src, int flags, const InstDev *insts, const StreamSet &S, const IoArgs &io,
                           cudaStream_t s) {
  const dim3 gc(S.n_coarse);
  cudaError_t e = src == 0
                      ? launch_ex(k_idwt_coarse<T, 0, LF>, gc, kPassThreads, 0, S.smem_coarse, s, insts, S.coarse, io, flags)
                      : launch_ex(k_idwt_coarse<T, 1, LF>, gc, kPassThreads, 0, S.smem_coarse, s, insts, S.coarse, io, flags);
  for (int k = S.kmax; k >= 1 && e == cudaSuccess; --k) {
    if (S.cnt[k] == 0) continue;
    const dim3 g(S.cnt[k]);
    const PassItem *it = S.items + S.off[k];
    e = src == 0 ? launch_ex(k_idwt_pass<T, 0, LF>, g, kPassThreads, 0, S.smem_pass, s, insts, it, io, k, flags)
                 : launch_ex(k_idwt_pass<T, 1, LF>, g, kPassThreads, 0, S.smem_pass, s, insts, it, io, k, flags);
  }
  return e;
}

template <typename T, int SRC, int EPI, int LF>
cudaError_t anal_streamed_e(int flags, const InstDev *insts, const StreamSet &S, const IoArgs &io, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int k = 1; k <= S.kmax && e == cudaSuccess; ++k) {
    if (S.cnt[k] == 0) continue;
    e = launch_ex(k_dwt_pass<T, SRC, EPI, LF>, dim3(S.cnt[k]), kPassThreads, 0, S.smem_pass, s, insts,
                  S.items + S.off[k], io, k, flags);
  }
  if (e == cudaSuccess)
    e = launch_ex(k_dwt_coarse<T, SRC, EPI, LF>, dim3(S.n_coarse), kPassThreads, 0, S.smem_coarse, s, insts,
                  S.coarse, io, flags);
  return e;
}

template <typename T, int LF>
cudaError_t anal_streamed(int src, int epi, int flags, const InstDev *insts, const StreamSet &S, const IoArgs &io,
                          cudaStream_t s) {
  if (src == 0) return anal_streamed_e<T, 0, kEpiPlain, LF>(flags, insts, S, io, s);
  if (epi == kEpiPlain) return anal_streamed_e<T, 2, kEpiPlain, LF>(flags, insts, S, io, s);
  if (epi == kEpiOp) return anal_streamed_e<T, 2, kEpiOp, LF>(flags, insts, S, io, s);
  return anal_streamed_e<T, 2, kEpiResid, LF>(flags, insts, S, io, s);
}

template <typename T>
cudaError_t allow_streamed_t() {
  cudaError_t e = cudaSuccess;
#define TOMO_ALLOW(K) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxTransformSmem)
#define TOMO_ALLOW_LF(LF)                                     \
  TOMO_ALLOW((k_idwt_coarse<T, 0, LF>));                      \
  TOMO_ALLOW((k_idwt_coarse<T, 1, LF>));                      \
  TOMO_ALLOW((k_idwt_pass<T, 0, LF>));                        \
  TOMO_ALLOW((k_idwt_pass<T, 1, LF>));                        \
  TOMO_ALLOW((k_dwt_pass<T, 0, kEpiPlain, LF>));              \
  TOMO_ALLOW((k_dwt_pass<T, 2, kEpiPlain, LF>));              \
  TOMO_ALLOW((k_dwt_pass<T, 2, kEpiOp, LF>));                 \
  TOMO_ALLOW((k_dwt_pass<T, 2, kEpiResid, LF>));              \
  TOMO_ALLOW((k_dwt_coarse<T, 0, kEpiPlain, LF>));            \
  TOMO_ALLOW((k_dwt_coarse<T, 2, kEpiPlain, LF>));            \
  TOMO_ALLOW((k_dwt_coarse<T, 2, kEpiOp, LF>));               \
  TOMO_ALLOW((k_dwt_coarse<T, 2, kEpiResid, LF>))
  TOMO_ALLOW_LF(2);
  TOMO_ALLOW_LF(4);
  TOMO_ALLOW_LF(6);
  TOMO_ALLOW_LF(8);
#undef TOMO_ALLOW_LF
#undef TOMO_ALLOW
  return e;
}

}  // namespace

cudaError_t configure_streamed_kernels() {
  cudaError_t e = allow_streamed_t<float>();
  if (e == cudaSuccess) e = allow_streamed_t<double>();
  return e;
}

int streamed_launches(const StreamSet &S) {
  int n = 1;
  for (int k = 1; k <= S.kmax; ++k) n += S.cnt[k] > 0 ? 1 : 0;
  return n;
}

cudaError_t launch_synthesis_streamed(int precision, int src, int lf, int flags, const InstDev *insts,
                                      const StreamSet &S, const IoArgs &io, cudaStream_t s) {
#define TOMO_S(T, LF) return synth_streamed<T, LF>(src, flags, insts, S, io, s)
  if (precision == 0) {
    switch (lf) { case 2: TOMO_S(float, 2); case 4: TOMO_S(float, 4); case 6: TOMO_S(float, 6); case 8: TOMO_S(float, 8); }
  } else {
    switch (lf) { case 2: TOMO_S(double, 2); case 4: TOMO_S(double, 4); case 6: TOMO_S(double, 6); case 8: TOMO_S(double, 8); }
  }
#undef TOMO_S
  return cudaErrorInvalidValue;
}

cudaError_t launch_analysis_streamed(int precision, int src, int epi, int lf, int flags, const InstDev *insts,
                                     const StreamSet &S, const IoArgs &io, cudaStream_t s) {
#define TOMO_A(T, LF) return anal_streamed<T, LF>(src, epi, flags, insts, S, io, s)
  if (precision == 0) {
    switch (lf) { case 2: TOMO_A(float, 2); case 4: TOMO_A(float, 4); case 6: TOMO_A(float, 6); case 8: TOMO_A(float, 8); }
  } else {
    switch (lf) { case 2: TOMO_A(double, 2); case 4: TOMO_A(double, 4); case 6: TOMO_A(double, 6); case 8: TOMO_A(double, 8); }
  }
#undef TOMO_A
  return cudaErrorInvalidValue;
}

}  // namespace tomo
