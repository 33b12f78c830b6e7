// The separate gather kernel (sm_103a): g = sum_m P_m^T v_m (Sec. 5.1, the
// transposed ray-trace) for plans whose gather tables do not fit the analysis
// kernel's shared memory, one CTA per (instance, layer, band of rows).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"
#include "device_util.cuh"
#include "launch.h"
#include "transform.cuh"
#include "adjoint.cuh"

namespace tomo {

// The gather of one CTA band (layer l, node rows [k0, k0+R0)) from the tap
// records and corner fields in global memory, into the band buffer A (shared
// memory), sensor by sensor, then the pupil-edge list.  The bilinear weights
// are separable, so each sensor's term of node (row k, column i) is
//   sum_ty wy_ty(k) * U(b0(k) + ty, i),   U(b, i) = sum_tx wx_tx(i) * v(a0(i) + tx, b),
// the same two nested sums, in the same order, as the window sum of the fused
// gather.  Pass 1 forms U for the corner rows the band's row records reach
// (gt_brows) and the columns the sensor's taps reach (gt_cols): one column
// record per thread, then independent loads of v along the corner rows.  Pass 2
// takes the node rows from U in shared memory.  Each node receives the
// sensors' terms in sensor order, as the fused gathers do.  For plans whose
// tables do not fit the analysis CTAs' shared memory; k_gather runs it.
// VS: the band rows of v that pass 1 reads are copied to shared memory V first
// (one bulk copy per sensor on the mbarrier bar, phase md for sensor md; the
// next sensor's copy runs during pass 2 of the current one); otherwise pass 1
// reads them from global memory.
constexpr int kGatherRowsU = 4;   // corner rows of a column one thread forms at once in pass 1

template <typename T, int KT, bool VS>
__device__ void gather_band_global(const InstDev &I, int l, int N, int R0, int crank, T *A, T *U, T *V, uint64_t *bar,
                                   const T *s_coef, const int *s_go, const int *s_nc, const int *s_el,
                                   const int2 *s_cols, const int2 *s_br, int *s_ry, T *s_rw, int Md) {
  constexpr int RS = TapRec<T, KT>::RS;
  constexpr int vq = 16 / static_cast<int>(sizeof(T));   // elements per 16-byte copy
  const int nt = blockDim.x, tid = threadIdx.x;
  const T *vv = static_cast<const T *>(I.v);
  const T *rec = static_cast<const T *>(I.gt_rec);
  // one thread: the bulk copy of sensor md's band rows [br.x, br.x + nb nc) of
  // v, and KT more elements (zero-weight taps when nc < KT), from the 16-byte
  // boundary at or below br.x (the plan pads v beyond its last sensor)
  auto stage = [&](int md) {
    const int2 br = s_br[md];
    const int g0 = br.x / vq * vq;
    const int nq = (br.x - g0 + br.y * s_nc[md] + KT + vq - 1) / vq;
    mbar_arm(bar, static_cast<uint32_t>(nq) * 16u);
    bulk_copy_g2s(V, vv + g0, static_cast<uint32_t>(nq) * 16u, bar);
  };
  for (int node = tid; node < R0 * N; node += nt) A[node] = T(0);
  if constexpr (VS) {
    if (tid == 0 && Md > 0) {
      fence_async_global();   // v was written by the previous kernel
      stage(0);
    }
  }
  // (every listed sensor reaches the band: nonempty columns and corner rows)
  for (int md = 0; md < Md; ++md) {
    if constexpr (VS) {
      // sensor md's rows; a copy that never completed (it does not happen with
      // valid tables) makes the solve report a breakdown
      if (!mbar_wait(bar, md & 1)) I.scal[kFlag] = 1.0;
      __syncthreads();   // pass 2 of the previous sensor is done with U
    }
    const int2 cols = s_cols[md], br = s_br[md];
    const int ncol = cols.y, nb = br.y, nc = s_nc[md], el = s_el[md];
    const T *vsrc = VS ? V + (br.x - br.x / vq * vq) : vv + br.x;
    const T *xr = rec + static_cast<size_t>(s_go[md]) * RS;
    const T *yr = rec + static_cast<size_t>(s_go[md] + N + crank * R0) * RS;
    // the band's row records: first corner row relative to the band's (-1: none) and weights
    for (int kl = tid; kl < R0; kl += nt) {
      TapRec<T, KT> y;
      y.load(yr + kl * RS);
      s_ry[kl] = y.off < 0 ? -1 : (y.off - br.x) / nc;
#pragma unroll
      for (int t = 0; t < KT; ++t) s_rw[kl * KT + t] = y.w[t];
    }
    // threads per column group: tpr threads cover the columns (tpr the power of two
    // >= the column count, at most nt), the nt / tpr groups share the rows
    int tpr = 1;
    while (tpr < ncol && tpr < nt) tpr <<= 1;
    const int groups = nt / tpr, ci = tid % tpr, rg = tid / tpr;
    // pass 1: U(b, c) for the band's corner rows b (from br.x) and columns c
    for (int c = ci; c < ncol; c += tpr) {
      const int i = (cols.x + c) & (N - 1);
      TapRec<T, KT> x;
      x.load(xr + i * RS);
      if (x.off < 0) {
        for (int bb = rg; bb < nb; bb += groups) U[bb * ncol + c] = T(0);
        continue;
      }
      const T *p0 = vsrc + x.off;
      const T *gx = el >= 0 ? static_cast<const T *>(I.gel) + br.x + x.off : nullptr;
      for (int bb0 = rg; bb0 < nb; bb0 += kGatherRowsU * groups) {
        T v[kGatherRowsU][KT];
#pragma unroll
        for (int u = 0; u < kGatherRowsU; ++u) {
          const int bb = bb0 + u * groups;
#pragma unroll
          for (int t = 0; t < KT; ++t) v[u][t] = bb < nb ? (VS ? p0[bb * nc + t] : __ldg(p0 + bb * nc + t)) : T(0);
        }
        if (el >= 0) {
          // spot elongation with tip/tilt removal: v + m_x Gx + m_y Gy
          const T mx = s_coef[2 * kMaxEdgeSlots + 2 * el], my = s_coef[2 * kMaxEdgeSlots + 2 * el + 1];
#pragma unroll
          for (int u = 0; u < kGatherRowsU; ++u) {
            const int bb = bb0 + u * groups;
            if (bb < nb)
#pragma unroll
              for (int t = 0; t < KT; ++t)
                v[u][t] += mx * __ldg(gx + bb * nc + t) + my * __ldg(gx + I.v_total + bb * nc + t);
          }
        }
#pragma unroll
        for (int u = 0; u < kGatherRowsU; ++u) {
          const int bb = bb0 + u * groups;
          if (bb >= nb) break;
          T sx = x.w[0] * v[u][0];
#pragma unroll
          for (int t = 1; t < KT; ++t) sx += x.w[t] * v[u][t];
          U[bb * ncol + c] = sx;
        }
      }
    }
    __syncthreads();
    if constexpr (VS) {
      if (tid == 0 && md + 1 < Md) stage(md + 1);   // V is free: pass 1 is done
    }
    // pass 2: the band's node rows from U
    for (int c = ci; c < ncol; c += tpr) {
      const int i = (cols.x + c) & (N - 1);
      for (int kl = rg; kl < R0; kl += groups) {
        const int b0 = s_ry[kl];
        if (b0 < 0) continue;
        const T *u = U + b0 * ncol + c;
        T acc = T(0);
#pragma unroll
        for (int t = 0; t < KT; ++t) acc += s_rw[kl * KT + t] * u[t * ncol];
        A[kl * N + i] += acc;
      }
    }
    if constexpr (!VS) __syncthreads();
  }
  if constexpr (VS) __syncthreads();
  if (I.n_edge_wfs == 0) return;
  const int2 seg = I.tt_seg[l * I.C + crank];
  gather_edges<T>(seg.y - seg.x, I.tt_node + seg.x, I.tt_beg + seg.x, I.tt_k,
                  static_cast<const T *>(I.tt_w), A, s_coef);
  __syncthreads();
}

// ------------------------------------------------------------- k_gather
// g = sum_m P_m^T v_m (Sec. 5.1, the transposed ray-trace) into the plan's phi
// buffer, one CTA per (instance, layer, band of N/C rows), the costliest bands
// first (the host orders items), for plans whose gather tables are not staged
// in the analysis kernel; k_analysis with SRC 2
// then transforms it.  phi is free here: the forward kernel that read it has
// finished (dependency wait) and the next synthesis rewrites it.
// tt_mode as in edge_coefficients; io.in1: the slopes (tip/tilt-only data).
template <typename T, bool VS>
__global__ void __launch_bounds__(kGatherThreads, sizeof(T) == 4 ? 2 : 1) k_gather(const InstDev *__restrict__ insts,
                                                           const PassItem *__restrict__ items,
                                                           IoArgs io, int C, int tt_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ T s_coef[4 * kMaxEdgeSlots];
  __shared__ int s_go[kMaxGatherSensors], s_nc[kMaxGatherSensors], s_el[kMaxGatherSensors];
  __shared__ int2 s_cols[kMaxGatherSensors], s_br[kMaxGatherSensors];
  __shared__ int s_md;
  __shared__ uint64_t s_bar;   // the staged corner rows (VS)
  pdl_trigger();
  const PassItem it = items[blockIdx.x];
  const int crank = it.row0;
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  if (threadIdx.x == 0) {
    // the dense sensors whose taps reach this band, in sensor order
    int md = 0;
    for (int m = 0; m < I.n_wfs && md < kMaxGatherSensors; ++m) {
      const WfsDev &W = I.wfs[m];
      if (W.kind == kTTOnly) continue;
      const int2 cols = I.gt_cols[m * I.n_layers + it.layer];
      const int2 br = I.gt_brows[(m * I.n_layers + it.layer) * C + crank];
      if (cols.y == 0 || br.y == 0) continue;
      s_go[md] = I.gt_off[m * I.n_layers + it.layer];
      s_nc[md] = W.nc;
      s_el[md] = (W.elong && W.kind == kRemoveTT) ? W.tt_idx : -1;
      s_cols[md] = cols;
      s_br[md] = br;
      ++md;
    }
    s_md = md;
    if (VS) mbar_init(&s_bar);
  }
  const LayerDev &L = I.layers[it.layer];
  const int N = L.N, R0 = N / C;
  T *g = static_cast<T *>(I.phi) + L.off + crank * R0 * N;
  __syncthreads();
  pdl_wait();
  if (I.n_edge_wfs > 0)
    edge_coefficients<T>(I, s_coef, tt_mode, static_cast<const T *>(io.in1[it.inst]));
  // shared memory: the band buffer, the band's row records (first row, weights),
  // the column-summed corner rows of one sensor, the staged rows of v (gather_smem_layout)
  const GatherSmem gs = gather_smem_layout(R0, N, I.max_taps, static_cast<int>(sizeof(T)), I.max_band_cells,
                                           I.max_band_v, VS);
  T *A = reinterpret_cast<T *>(smem_raw);
  int *s_ry = reinterpret_cast<int *>(smem_raw + gs.ry);
  T *s_rw = reinterpret_cast<T *>(smem_raw + gs.rw);
  T *U = reinterpret_cast<T *>(smem_raw + gs.u);
  T *V = reinterpret_cast<T *>(smem_raw + gs.v);
#define TOMO_GB(KT) gather_band_global<T, KT, VS>(I, it.layer, N, R0, crank, A, U, V, &s_bar, s_coef, s_go, s_nc, \
                                                  s_el, s_cols, s_br, s_ry, s_rw, s_md)
  if (I.max_taps <= 2) TOMO_GB(2);
  else if (I.max_taps == 3) TOMO_GB(3);
  else TOMO_GB(4);
#undef TOMO_GB
  for (int node = threadIdx.x; node < R0 * N; node += blockDim.x) g[node] = A[node];
}

template <typename T>
cudaError_t gather_t(int vstage, dim3 g, size_t smem, cudaStream_t s, const InstDev *insts, const PassItem *items,
                     const IoArgs &io, int C, int tt_mode) {
  return vstage ? launch_ex(k_gather<T, true>, g, kGatherThreads, 0, smem, s, insts, items, io, C, tt_mode)
                : launch_ex(k_gather<T, false>, g, kGatherThreads, 0, smem, s, insts, items, io, C, tt_mode);
}

cudaError_t launch_gather(int precision, int tt_mode, const InstDev *insts, const PassItem *items, int n_items,
                          int C, int vstage, size_t smem_gather, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_items);
  return precision == 0 ? gather_t<float>(vstage, g, smem_gather, s, insts, items, io, C, tt_mode)
                        : gather_t<double>(vstage, g, smem_gather, s, insts, items, io, C, tt_mode);
}

cudaError_t configure_gather_kernels() {
  cudaError_t e = cudaSuccess;
#define TOMO_CFG(K) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxTransformSmem)
  TOMO_CFG((k_gather<float, false>));
  TOMO_CFG((k_gather<float, true>));
  TOMO_CFG((k_gather<double, false>));
  TOMO_CFG((k_gather<double, true>));
#undef TOMO_CFG
  return e;
}

}  // namespace tomo
