// CUDA kernels of the wavelet-domain MAP tomography solve (sm_103a).
//
// Per PCG iteration (Sec. 5.1 of the paper) four launches cover the operator
// (W P^T Gamma^T C^-1 Gamma P W^-1 + alpha D) p and the (P)CG vector updates:
//
//   k_synthesis  beta from the r.z partials, p <- J^-1 r + beta p,
//                phi = W^-1 p                                    [cluster per layer]
//   k_forward    psi = P phi on sensor corners, Fried slopes,
//                C^-1 weighting, Gamma^T; tip/tilt sums          [tile per sensor]
//   k_analysis   g = sum_m P_m^T v_m (gather + pupil-edge list),
//                q = W g + alpha D p, p.q partials               [cluster per layer]
//   k_update     alpha from the p.q partials, x += alpha p,
//                r -= alpha q, r.J^-1 r partials                 [chunk per CTA]
//
// The periodic 2-D DWT of one layer runs inside one thread-block cluster: CTA c
// owns N/C consecutive rows; the row pass is local, and before the column pass
// each CTA copies the Lf-2 halo rows it needs from its neighbours' shared memory
// (distributed shared memory) next to its own rows.  The coarse levels (block
// side <= C) are finished by CTA 0 alone.  Each CTA loads every coefficient it
// owns in one round trip at its start (with the PCG direction update fused in).
//
// Reductions are FP64: warp shuffle -> block -> one partial per CTA; the
// consumer kernel (every CTA of it) sums the producer's partials in a fixed
// order, so no kernel waits on a "last CTA" and results do not depend on
// scheduling.  Kernels are launched with programmatic dependent launch: each
// triggers its dependents at entry and waits (griddepcontrol.wait) only before
// touching data the previous kernel wrote.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"
#include "device_util.cuh"
#include "launch.h"
#include "transform.cuh"
#include "adjoint.cuh"

namespace cg = cooperative_groups;

namespace tomo {

// ------------------------------------------------------------------ helpers

// The two halves of a cluster barrier (cluster.sync() is both): every thread
// of every CTA in the cluster alternates arrive and wait.  arrive releases the
// thread's earlier shared-memory accesses (including reads of other CTAs'
// shared memory); wait returns once all threads of the cluster have arrived.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// A forward tile's two partial sums in its 16-byte partial slot: doubles for
// FP64 plans, double-float pairs (hi, lo, hi, lo) for FP32 plans.
__device__ __forceinline__ void store_tile_partial(double *slot, Acc<double> a, Acc<double> b) {
  const double2 s = block_sum2(a, b);
  if (threadIdx.x == 0) *reinterpret_cast<double2 *>(slot) = s;
}
__device__ __forceinline__ void store_tile_partial(double *slot, Acc<float> a, Acc<float> b) {
  const float4 s = block_sum2_df(a, b);
  if (threadIdx.x == 0) *reinterpret_cast<float4 *>(slot) = s;
}


// psi at corner (a, b) of sensor m: sum over layers of the bilinear
// interpolation of phi_l at the corner's traced position (Sec. 2.1, P_m).
template <typename T>
__device__ __forceinline__ T trace_corner(const InstDev &I, int m, int nc, const T *phi, int a,
                                          int b) {
  const T *pf = static_cast<const T *>(I.pos_f);
  T acc = T(0);
  for (int l = 0; l < I.n_layers; ++l) {
    const int N = I.layers[l].N, off = I.layers[l].off;
    const int po = I.pos_off[m * I.n_layers + l];
    const int x0 = I.pos_i0[po + a], y0 = I.pos_i0[po + nc + b];
    const T fx = pf[po + a], fy = pf[po + nc + b];
    const int x1 = (x0 + 1) & (N - 1), y1 = (y0 + 1) & (N - 1);
    const T *p = phi + off;
    const T v00 = p[y0 * N + x0], v01 = p[y0 * N + x1];
    const T v10 = p[y1 * N + x0], v11 = p[y1 * N + x1];
    acc += (T(1) - fy) * ((T(1) - fx) * v00 + fx * v01) + fy * ((T(1) - fx) * v10 + fx * v11);
  }
  return acc;
}

// ------------------------------------------------------------ k_forward
// MODE 0: operator, z = Gamma P phi.  MODE 1: residual, z = s - Gamma P phi.
// MODE 2: data only, z = s (phi = 0).  Writes the corner field
// v_m = Gamma_m^T sigma^-2 z_m and, with tip/tilt removal, each tile's sums of z
// (the analysis subtracts the means on the pupil edge, Sec. 4.3 eq. widehatc).
// A tip/tilt-only sensor writes its weighted mean slopes (e_x, e_y).
// io.in0: layer grids (NULL = the plan's phi); io.in1: slopes (MODE 1, 2).
// EL: some sensor of the launch has elongated spots (Sec. 4.3); without it the
// elongation code is compiled out.
// Launched with kThreads or kFwdThreads threads.  The per-corner steps use
// every thread; the steps that feed the tile's partial sums (the slopes and
// the tip/tilt-only chunks) keep a fixed kThreads-thread mapping, so the
// partials, and every result, are bitwise the same at either block size.
constexpr int kHalo = kFwdTile + 2;

__host__ __device__ constexpr size_t fwd_table_bytes(int L, size_t esz) {
  return ((sizeof(int) * (2 * L + 2 * L * kHalo) + 15) & ~size_t(15)) + 2 * L * kHalo * esz;
}

// NT: the block size the instance is compiled for: kFwdThreads with two CTAs
// per SM for small launches, kThreads with kFwdBatchBlocks CTAs per SM (fewer
// registers) for big ones (FP32; FP64 instances keep the registers they need).
constexpr int kFwdBatchBlocks = 5;

template <typename T, int MODE, bool EL, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT == kFwdThreads ? 2 : kFwdBatchBlocks) : 1)
    k_forward(const InstDev *__restrict__ insts, const FwdItem *__restrict__ items, IoArgs io) {
  extern __shared__ __align__(16) unsigned char fsm[];
  __shared__ InstDev sI;
  __shared__ T s_psi[kHalo][kHalo + 1];
  __shared__ T s_ex[kFwdTile + 1][kFwdTile + 2];
  __shared__ T s_ey[kFwdTile + 1][kFwdTile + 2];
  pdl_trigger();
  const FwdItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const WfsDev W = I.wfs[it.wfs];
  const T *phi = io.in0[it.inst] ? static_cast<const T *>(io.in0[it.inst]) : static_cast<const T *>(I.phi);
  const T *dat = static_cast<const T *>(io.in1[it.inst]);
  const int nc = W.nc, n = W.n, tid = threadIdx.x, L = I.n_layers;

  if (it.a0 < 0) {
    // Tip/tilt-only sensor: the sum of its Fried slopes over the valid
    // subapertures is <Gamma^T 1, psi>, which lives on the pupil-edge corners;
    // one (edge corner, layer) term per thread, one FP64 partial per chunk.
    if (MODE == 2) return;   // data only: the model term is zero
    const int pair = it.tile * kThreads + tid;
    const bool on = tid < kThreads && pair < W.n_edge * L;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0, N = 1, off = 0;
    T fx = T(0), fy = T(0), tx = T(0), ty = T(0);
    if (on) {
      const int e = pair / L, l = pair - e * L;
      const int c = I.edge_idx[W.edge_off + e];
      const int a = c % nc, b = c / nc;
      const T *et = static_cast<const T *>(I.edge_t) + 2 * (W.edge_off + e);
      const T *pf = static_cast<const T *>(I.pos_f);
      const int po = I.pos_off[it.wfs * L + l];
      N = I.layers[l].N;
      off = I.layers[l].off;
      x0 = I.pos_i0[po + a];
      y0 = I.pos_i0[po + nc + b];
      fx = pf[po + a];
      fy = pf[po + nc + b];
      x1 = (x0 + 1) & (N - 1);
      y1 = (y0 + 1) & (N - 1);
      tx = et[0];
      ty = et[1];
    }
    pdl_wait();
    Acc<T> ax, ay;
    if (on) {
      const T *p = phi + off;
      const T v00 = p[y0 * N + x0], v01 = p[y0 * N + x1];
      const T v10 = p[y1 * N + x0], v11 = p[y1 * N + x1];
      const T ps = (T(1) - fy) * ((T(1) - fx) * v00 + fx * v01) + fy * ((T(1) - fx) * v10 + fx * v11);
      ax.add_prod(tx, ps);
      ay.add_prod(ty, ps);
    }
    store_tile_partial(I.part + W.part_off + 2 * it.tile, ax, ay);
    return;
  }

  // stage this tile's corner->node tables for every layer (constant data)
  int *s_N = reinterpret_cast<int *>(fsm);
  int *s_off = s_N + L;
  int *s_x0 = s_off + L;
  int *s_y0 = s_x0 + L * kHalo;
  T *s_fx = reinterpret_cast<T *>(fsm + ((sizeof(int) * (2 * L + 2 * L * kHalo) + 15) & ~size_t(15)));
  T *s_fy = s_fx + L * kHalo;
  const int a0 = it.a0, b0 = it.b0;
  {
    const T *pf = static_cast<const T *>(I.pos_f);
    for (int idx = tid; idx < L * kHalo; idx += blockDim.x) {
      const int l = idx / kHalo, u = idx - l * kHalo;
      const int po = I.pos_off[it.wfs * L + l];
      const int a = min(max(a0 - 1 + u, 0), nc - 1), b = min(max(b0 - 1 + u, 0), nc - 1);
      s_x0[idx] = I.pos_i0[po + a];
      s_fx[idx] = pf[po + a];
      s_y0[idx] = I.pos_i0[po + nc + b];
      s_fy[idx] = pf[po + nc + b];
    }
    for (int l = tid; l < L; l += blockDim.x) {
      s_N[l] = I.layers[l].N;
      s_off[l] = I.layers[l].off;
    }
  }
  __syncthreads();
  const unsigned char *act = I.active + W.act_off;
  const int *sidx = I.sub_idx + W.sub_off;
  pdl_wait();
  // 1. psi on the tile's corners plus a one-corner halo
  for (int idx = tid; idx < kHalo * kHalo; idx += blockDim.x) {
    const int u = idx % kHalo, w = idx / kHalo;
    const int a = a0 - 1 + u, b = b0 - 1 + w;
    T val = T(0);
    if (MODE != 2 && a >= 0 && b >= 0 && a < nc && b < nc && act[b * nc + a]) {
      // four layers' loads in flight at a time; the sum keeps the layer order
      for (int l0 = 0; l0 < L; l0 += 4) {
        T v00[4], v01[4], v10[4], v11[4], fx[4], fy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int l = l0 + j < L ? l0 + j : L - 1;
          const int N = s_N[l];
          const int x0 = s_x0[l * kHalo + u], y0 = s_y0[l * kHalo + w];
          fx[j] = s_fx[l * kHalo + u];
          fy[j] = s_fy[l * kHalo + w];
          const int x1 = (x0 + 1) & (N - 1), y1 = (y0 + 1) & (N - 1);
          const T *p = phi + s_off[l];
          v00[j] = p[y0 * N + x0];
          v01[j] = p[y0 * N + x1];
          v10[j] = p[y1 * N + x0];
          v11[j] = p[y1 * N + x1];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (l0 + j < L)
            val += (T(1) - fy[j]) * ((T(1) - fx[j]) * v00[j] + fx[j] * v01[j]) +
                   fy[j] * ((T(1) - fx[j]) * v10[j] + fx[j] * v11[j]);
      }
    }
    s_psi[w][u] = val;
  }
  __syncthreads();
  // 2. weighted slopes of the subapertures the tile's corners touch
  Acc<T> sx_acc, sy_acc, qx_acc, qy_acc;
  const T isg = sizeof(T) == 4 ? T(W.inv_sigma2_f) : T(W.inv_sigma2);   // no FP64 conversion in FP32
  // spot elongation: the block sigma^2 (I + tau g g^T) is inverted in closed
  // form, sigma^-2 (I - c g g^T) with c = tau / (1 + tau |g|^2)
  const bool elong = EL && W.elong != 0;
  const T el_tau = EL ? T(W.el_tau) : T(0), el_eps = EL ? T(W.el_eps) : T(0), el_d = EL ? T(W.d_sub) : T(0);
  const T el_cx = EL ? T(0.5 - 0.5 * n) * el_d - T(W.el_lx) : T(0);
  const T el_cy = EL ? T(0.5 - 0.5 * n) * el_d - T(W.el_ly) : T(0);
  const bool four = EL && tile_partials(W) == 4;
  for (int idx = tid; tid < kThreads && idx < (kFwdTile + 1) * (kFwdTile + 1); idx += kThreads) {
    const int u = idx % (kFwdTile + 1), w = idx / (kFwdTile + 1);
    const int a = a0 - 1 + u, b = b0 - 1 + w;
    T ex = T(0), ey = T(0);
    if (a >= 0 && b >= 0 && a < n && b < n) {
      const int j = sidx[b * n + a];
      if (j >= 0) {
        const T p00 = s_psi[w][u], p10 = s_psi[w][u + 1];
        const T p01 = s_psi[w + 1][u], p11 = s_psi[w + 1][u + 1];
        T sx = T(0.5) * (p10 + p11 - p00 - p01);
        T sy = T(0.5) * (p01 + p11 - p00 - p10);
        if (MODE == 1) {
          sx = dat[W.slope_off + j] - sx;
          sy = dat[W.slope_off + W.S + j] - sy;
        } else if (MODE == 2) {
          sx = dat[W.slope_off + j];
          sy = dat[W.slope_off + W.S + j];
        }
        if (elong) {
          const T gx = el_eps * (T(a) * el_d + el_cx), gy = el_eps * (T(b) * el_d + el_cy);
          const T c = el_tau / (T(1) + el_tau * (gx * gx + gy * gy));
          const T dot = c * (gx * sx + gy * sy);
          ex = isg * (sx - gx * dot);
          ey = isg * (sy - gy * dot);
        } else {
          ex = isg * sx;
          ey = isg * sy;
        }
        if (u >= 1 && w >= 1) {   // subapertures owned by this tile
          sx_acc.add(sx);
          sy_acc.add(sy);
          if (four) {
            qx_acc.add(ex);
            qy_acc.add(ey);
          }
        }
      }
    }
    s_ex[w][u] = ex;
    s_ey[w][u] = ey;
  }
  __syncthreads();
  // 3. Gamma^T: each corner gathers its four neighbouring subapertures
  T *v = static_cast<T *>(I.v) + W.v_off;
  if (tid < kFwdTile * kFwdTile) {
    const int u = tid % kFwdTile, w = tid / kFwdTile;
    const int a = a0 + u, b = b0 + w;
    if (a < nc && b < nc) {
      const T val = T(0.5) * (s_ex[w + 1][u] + s_ex[w][u] - s_ex[w + 1][u + 1] - s_ex[w][u + 1]) +
                    T(0.5) * (-s_ey[w + 1][u] + s_ey[w][u] - s_ey[w + 1][u + 1] + s_ey[w][u + 1]);
      v[b * nc + a] = val;
    }
  }
  if (W.kind != kRemoveTT) return;
  // 4. tip/tilt removal: this tile's sums of z (the consumer forms the means)
  if (four) {
    store_tile_partial(I.part + W.part_off + 4 * it.tile, sx_acc, sy_acc);
    __syncthreads();   // warp 0 has read the reduction scratch before it is reused
    store_tile_partial(I.part + W.part_off + 4 * it.tile + 2, qx_acc, qy_acc);
  } else {
    store_tile_partial(I.part + W.part_off + 2 * it.tile, sx_acc, sy_acc);
  }
}

// ------------------------------------------------------- transform helpers

// Coefficients owned by cluster rank c of one layer, and their place in the
// CTA's shared-memory cache.  Distributed levels k = 1..kd (block side
// M = N/2^(k-1) >= 2C, R = M/C rows per CTA, Rh = R/2, H = M/2): the high-x
// part of the low-y rows c*Rh + jl and the high-y rows H + c*Rh + jl; then the
// CTA's low-low rows of level J (kd == J) or, on rank 0, the coarse pyramid
// block of side C (kd < J).  Levels below cache_kc are read from global memory.
struct CoefMap {
  int N, C, J, kd, kc, crank, lgN, lgC;
  int base[kMaxLevels + 3];
  __device__ void init(int N_, int C_, int J_, int kc_, int crank_) {
    N = N_;
    C = C_;
    J = J_;
    crank = crank_;
    lgN = __ffs(N) - 1;
    lgC = __ffs(C) - 1;
    kd = 0;
    while (kd < J && (N >> kd) >= 2 * C) ++kd;
    kc = kc_ < 1 ? 1 : kc_;
    int off = 0;
    for (int k = 1; k <= kd; ++k) {
      base[k] = off;
      if (k >= kc) {
        const int M = N >> (k - 1), Rh = (M / C) >> 1;
        off += Rh * (M >> 1) + Rh * M;
      }
    }
    base[kd + 1] = off;
    if (kd == J) {
      const int M = N >> (J - 1), Rh = (M / C) >> 1;
      off += Rh * (M >> 1);
    } else if (crank == 0) {
      off += C * C;
    }
    base[kd + 2] = off;
  }
  __device__ int total() const { return base[kd + 2]; }
  // sizes of level k as log2: block side M, half H, CTA rows R, half Rh
  __device__ int lgM(int k) const { return lgN - (k - 1); }
  __device__ int hl(int k, int jl, int x) const {
    const int lh = lgM(k) - 1;
    return base[k] + (jl << lh) + (x - (1 << lh));
  }
  __device__ int lh(int k, int jl, int x) const {
    const int lm = lgM(k), lrh = lm - lgC - 1;
    return base[k] + (1 << (lrh + lm - 1)) + (jl << lm) + x;
  }
  __device__ int ll(int jl, int x) const { return base[kd + 1] + (jl << (lgM(J) - 1)) + x; }
  __device__ int coarse(int r, int c) const { return base[kd + 1] + (r << lgC) + c; }
  // pyramid position of cache slot q
  __device__ void pos(int q, int &row, int &col) const {
    if (q >= base[kd + 1]) {
      const int q2 = q - base[kd + 1];
      if (kd == J) {
        const int lh = lgM(J) - 1, lrh = lgM(J) - lgC - 1;
        row = (crank << lrh) + (q2 >> lh);
        col = q2 & ((1 << lh) - 1);
      } else {
        row = q2 >> lgC;
        col = q2 & (C - 1);
      }
      return;
    }
    int k = kd;
    while (base[k] > q) --k;
    const int lm = lgM(k), lh = lm - 1, lrh = lm - lgC - 1;
    int q2 = q - base[k];
    if (q2 < (1 << (lrh + lh))) {
      row = (crank << lrh) + (q2 >> lh);
      col = (1 << lh) + (q2 & ((1 << lh) - 1));
    } else {
      q2 -= 1 << (lrh + lh);
      row = (1 << lh) + (crank << lrh) + (q2 >> lm);
      col = q2 & ((1 << lm) - 1);
    }
  }
};

// Shared-memory copy of the gather tables of one analysis CTA (layer l, rows
// [k0, k0+R0)), laid out by stage_layout: the plan's stage image for the CTA
// (tap records, pupil-edge entries and index, run tables), one bulk copy before
// the dependency wait since the tables are constant, so the copy overlaps the
// previous kernel; after the wait, the corner rows of v that the CTA reads,
// one bulk copy per sensor.
template <typename T>
struct GatherStage {
  unsigned char *base;
  T *xr, *yr, *vs, *tw;
  int *mnc, *vpre, *vsrc, *mslot, *tk;
  const uint16_t *eb;
  int image_bytes;

  __device__ void carve(unsigned char *b, int Md, int N, int R0, const InstDev &I) {
    const StageLayout sl = stage_layout(Md, N, R0, I.rec_stride, static_cast<int>(sizeof(T)), I.max_tt_entries,
                                        I.vstage);
    base = b;
    xr = reinterpret_cast<T *>(b + sl.xr);
    yr = reinterpret_cast<T *>(b + sl.yr);
    tw = reinterpret_cast<T *>(b + sl.tw);
    vs = reinterpret_cast<T *>(b + sl.vs);
    mnc = reinterpret_cast<int *>(b + sl.mnc);
    vpre = reinterpret_cast<int *>(b + sl.vpre);
    vsrc = reinterpret_cast<int *>(b + sl.vsrc);
    mslot = reinterpret_cast<int *>(b + sl.mslot);
    tk = reinterpret_cast<int *>(b + sl.tk);
    eb = reinterpret_cast<const uint16_t *>(b + sl.eb);
    image_bytes = sl.image;
  }

  // One thread: the bulk copy of the CTA's stage image, completing on bar.
  __device__ void issue_image(const InstDev &I, int l, int crank, uint64_t *bar) const {
    const unsigned char *src = static_cast<const unsigned char *>(I.stage_img) + I.img_stride * (l * I.C + crank);
    mbar_arm(bar, static_cast<uint32_t>(image_bytes));
    if (image_bytes > 0) bulk_copy_g2s(base, src, static_cast<uint32_t>(image_bytes), bar);
  }

  // Spot elongation with tip/tilt removal: v += m_x Gx + m_y Gy over the staged
  // corner rows of those sensors (the mean slopes from edge_coefficients).
  __device__ void add_elongation(const InstDev &I, const T *s_coef) const {
    constexpr int vq = 16 / static_cast<int>(sizeof(T));
    const T *gx = static_cast<const T *>(I.gel), *gy = gx + I.v_total;
    for (int md = 0; md < I.n_dense; ++md) {
      const int k = mslot[md];
      if (k < 0) continue;
      const T mx = s_coef[2 * kMaxEdgeSlots + 2 * k], my = s_coef[2 * kMaxEdgeSlots + 2 * k + 1];
      const int e0 = vpre[md] * vq, cnt = (vpre[md + 1] - vpre[md]) * vq, g0 = vsrc[md] * vq;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) vs[e0 + i] += mx * gx[g0 + i] + my * gy[g0 + i];
    }
  }

  // One thread, after the dependency wait: the bulk copies of the CTA's
  // corner rows of v (one aligned run per sensor, written by the previous
  // kernel), completing on bar.  Needs the stage image in shared memory.
  __device__ void load_v_bulk(const InstDev &I, uint64_t *bar) const {
    const int Md = I.n_dense;
    const uint4 *src = static_cast<const uint4 *>(I.v);
    uint4 *dst = reinterpret_cast<uint4 *>(vs);
    fence_async_global();
    mbar_arm(bar, static_cast<uint32_t>(vpre[Md]) * 16u);
    for (int md = 0; md < Md; ++md) {
      const int n = vpre[md + 1] - vpre[md];
      if (n > 0) bulk_copy_g2s(dst + vpre[md], src + vsrc[md], static_cast<uint32_t>(n) * 16u, bar);
    }
  }
};

// The gather of gather_rows from the staged records and v rows, sensors inner
// with the sums in registers.  A thread takes one column and two adjacent node
// rows: they share the column's tap record, and their windows' corner rows
// overlap, so each corner row's weighted column sum sx is formed once for both
// (rows of the second window d = 0..2 rows below the first's; other offsets
// take the two windows apart).  Each node's sum has window_sum's order.
template <typename T, int KT, int D>
__device__ __forceinline__ void pair_sums(const T *h, const TapRec<T, KT> &y0, const TapRec<T, KT> &y1, T &acc0,
                                          T &acc1) {
  T s0 = T(0), s1 = T(0);
#pragma unroll
  for (int ty = 0; ty < KT; ++ty) s0 += y0.w[ty] * h[ty];
#pragma unroll
  for (int ty = 0; ty < KT; ++ty) s1 += y1.w[ty] * h[D + ty];
  acc0 += s0;
  acc1 += s1;
}

template <typename T, int KT>
__device__ void gather_rows_staged(const InstDev &I, const GatherStage<T> &st, int N, int R0,
                                   T *A, const T *s_coef) {
  constexpr int RS = TapRec<T, KT>::RS;
  const int nt = blockDim.x, tid = threadIdx.x, Md = I.n_dense, lgN = __ffs(N) - 1;
  for (int pr = tid; pr < (R0 >> 1) * N; pr += nt) {
    const int col = pr & (N - 1), k0 = (pr >> lgN) << 1;
    const T *xr = st.xr + col * RS;
    const T *yr = st.yr + k0 * RS;
    T acc0 = T(0), acc1 = T(0);
    for (int md = 0; md < Md; ++md) {
      TapRec<T, KT> x, y0, y1;
      x.load(xr + md * N * RS);
      y0.load(yr + md * R0 * RS);
      y1.load(yr + md * R0 * RS + RS);
      if (x.off < 0) continue;
      const int nc = st.mnc[md];
      const int d = (y0.off >= 0 && y1.off >= 0) ? (y1.off - y0.off) / nc : -1;
      if (d >= 0 && d <= 2 && y1.off - y0.off == d * nc) {
        // the corner rows of both windows, each row's column sum once
        T h[KT + 2];
        const T *p = st.vs + y0.off + x.off;
#pragma unroll
        for (int r = 0; r < KT + 2; ++r) {
          if (r < KT + d) {
            T v[KT];
#pragma unroll
            for (int tx = 0; tx < KT; ++tx) v[tx] = p[r * nc + tx];
            T sx = x.w[0] * v[0];
#pragma unroll
            for (int tx = 1; tx < KT; ++tx) sx += x.w[tx] * v[tx];
            h[r] = sx;
          }
        }
        if (d == 0) pair_sums<T, KT, 0>(h, y0, y1, acc0, acc1);
        else if (d == 1) pair_sums<T, KT, 1>(h, y0, y1, acc0, acc1);
        else pair_sums<T, KT, 2>(h, y0, y1, acc0, acc1);
      } else {
        if (y0.off >= 0) acc0 += window_sum<T, KT, true>(st.vs + y0.off + x.off, nc, x, y0);
        if (y1.off >= 0) acc1 += window_sum<T, KT, true>(st.vs + y1.off + x.off, nc, x, y1);
      }
    }
    if (I.n_edge_wfs > 0) {
      // the nodes' pupil-edge entries (from the dense per-node index), added after the sensors
      const int n0 = k0 * N + col, n1 = n0 + N;
      const int e0 = st.eb[n0], e1 = st.eb[n0 + 1], e2 = st.eb[n1], e3 = st.eb[n1 + 1];
      if (e1 > e0) acc0 += edge_node_sum<T>(e0, e1, st.tk, st.tw, s_coef);
      if (e3 > e2) acc1 += edge_node_sum<T>(e2, e3, st.tk, st.tw, s_coef);
    }
    A[k0 * N + col] = acc0;
    A[(k0 + 1) * N + col] = acc1;
  }
}

// ------------------------------------------------------------ k_analysis
// SRC 0: layer grids from io.in0.  SRC 1: adjoint gather from the plan's v.
// SRC 2: the gather k_gather left in the plan's phi.
// EPI plain: io.out0 = W g.  EPI op: q = W g + alpha D p with p = io.in1 (NULL:
// the plan's p), q = io.out0 (NULL: the plan's q); partial p.q per CTA.
// EPI resid: r = W g - alpha D x (x = io.out0, zeroed when cold), p = z = J^-1 r;
// partials r.z and r.r per CTA.
template <typename T, int SRC, int EPI, int LF>
__global__ void __launch_bounds__(kAnalysisThreadsMax, 1) k_analysis(const InstDev *__restrict__ insts,
                                                      const ClusterItem *__restrict__ items,
                                                      IoArgs io, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ CoefMap cm;
  __shared__ T s_coef[4 * kMaxEdgeSlots];
  __shared__ T s_dal[kMaxLevels + 1];
  __shared__ uint64_t s_bar[2];   // stage image, corner rows of v (bulk copies)
  pdl_trigger();
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const ClusterItem it = items[blockIdx.x / C];
  if (io.active && !io.active[it.inst]) return;   // the whole cluster leaves together
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int N = L.N, R0 = N / C, J = I.J, tid = threadIdx.x, nt = blockDim.x;
  T *A = reinterpret_cast<T *>(smem_raw);
  T *B = A + (R0 + kMaxTaps) * N;
  T *cb = B + (R0 + kMaxTaps) * N;
  T *cb2 = cb + C * C;
  T *cache = reinterpret_cast<T *>(smem_raw) + transform_cache_offset(N, C);
  if (tid == 0) cm.init(N, C, J, L.cache_kc, crank);
  if (tid <= J) s_dal[tid] = T(L.dalpha[tid]);
  Filt<T, LF> f;
  f.load(I);

  Emit<T, EPI> emit;
  emit.off = L.off;
  emit.N = N;
  emit.dalpha = s_dal;
  emit.precond = I.precond;
  emit.warm = (flags & kFlagWarm) ? 1 : 0;
  emit.jinv = static_cast<const T *>(I.jinv);
  emit.cache = cache;
  emit.out = static_cast<T *>(io.out0[it.inst]);
  emit.P = io.in1[it.inst] ? static_cast<const T *>(io.in1[it.inst]) : static_cast<const T *>(I.p);
  emit.Q = io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.q);
  emit.R = static_cast<T *>(I.r);
  emit.Pn = static_cast<T *>(I.p);
  emit.X = static_cast<T *>(io.out0[it.inst]);
  GatherStage<T> st;
  // SRC 1 plans stage their tables (those that cannot run k_gather, SRC 2)
  const bool staged = SRC == 1;
  bool copies_ok = true;
  if (staged) {
    const int off = transform_cache_offset(N, C) + transform_cache_size(N, C, J, L.cache_kc);
    unsigned char *sb = smem_raw + ((static_cast<size_t>(off) * sizeof(T) + 15) & ~size_t(15));
    st.carve(sb, I.n_dense, N, R0, I);
    if (tid == 0) {
      mbar_init(&s_bar[0]);
      mbar_init(&s_bar[1]);
      st.issue_image(I, it.layer, crank, &s_bar[0]);
    }
    __syncthreads();   // the barriers are initialised
    copies_ok = mbar_wait(&s_bar[0], 0);
  }
  __syncthreads();
  pdl_wait();
  // a new solve starts from the residual: clear the breakdown flag
  if (EPI == kEpiResid && it.layer == 0 && crank == 0 && tid == 0) I.scal[kFlag] = 0.0;

  // asynchronous copies: the gather's corner rows of v, then the epilogue
  // inputs (p, or x for a warm residual) of every owned coefficient into the
  // coefficient cache; both complete before the transform
  if (staged && tid == 0) st.load_v_bulk(I, &s_bar[1]);
  const bool use_cache = (EPI == kEpiOp) || (EPI == kEpiResid && emit.warm);
  if (use_cache) {
    // issued by the warps that the pupil-edge coefficients below leave idle
    // (one warp per edge slot), so the two overlap
    const int w0 = SRC == 1 ? min(I.n_edge_wfs, nt / 32 - 1) : 0, t0 = tid - 32 * w0;
    if (t0 >= 0) {
      const T *srcv = EPI == kEpiOp ? emit.P : emit.X;
      const int total = cm.total();
      for (int q = t0; q < total; q += nt - 32 * w0) {
        int row, col;
        cm.pos(q, row, col);
        cp_async_elem(cache + q, srcv + L.off + row * N + col);
      }
    }
    cp_async_commit();
  }
  // own rows [crank*R0, (crank+1)*R0) of the layer grid
  if (SRC == 0 || SRC == 2) {
    const T *src = (SRC == 0 ? static_cast<const T *>(io.in0[it.inst]) : static_cast<const T *>(I.phi)) +
                   L.off + crank * R0 * N;
    for (int idx = tid; idx < R0 * N; idx += nt) A[idx] = src[idx];
  } else {
    // the tip/tilt-only sensors' measurement term: model (operator), data
    // minus model (warm residual) or data alone (cold residual, right-hand side)
    const int tt_mode = EPI == kEpiOp ? 0 : (EPI == kEpiResid && emit.warm ? 1 : 2);
    if (I.n_edge_wfs > 0)
      edge_coefficients<T>(I, s_coef, tt_mode, static_cast<const T *>(io.in1[it.inst]));
    if (staged) {
      copies_ok = mbar_wait(&s_bar[1], 0) && copies_ok;
      // a copy that never completed (it does not happen with valid tables): the
      // solve reports a breakdown and its iterate stays as it was
      if (!copies_ok) I.scal[kFlag] = 1.0;
      __syncthreads();
      if (I.gel) {
        st.add_elongation(I, s_coef);
        __syncthreads();
      }
      if (I.max_taps <= 2) gather_rows_staged<T, 2>(I, st, N, R0, A, s_coef);
      else if (I.max_taps == 3) gather_rows_staged<T, 3>(I, st, N, R0, A, s_coef);
      else gather_rows_staged<T, 4>(I, st, N, R0, A, s_coef);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  auto slot_hl = [&](int k, int jl, int x) { return (use_cache && k >= cm.kc) ? cm.hl(k, jl, x) : -1; };
  auto slot_lh = [&](int k, int jl, int x) { return (use_cache && k >= cm.kc) ? cm.lh(k, jl, x) : -1; };

  // Distributed levels: one cluster barrier per level (row pass done) before
  // the halo rows are read from the next CTAs; the reads are released with
  // an arrive, and the matching wait comes just before this CTA next
  // overwrites B (the next level's row pass, or the end of the kernel).
  const int lgN = L.log2N, lgC = __ffs(C) - 1;
  int M = N, k = 1;
  for (; k <= J && M >= 2 * C; ++k, M >>= 1) {
    const int lgM = lgN - (k - 1), lgR = lgM - lgC;
    const int R = M >> lgC, H = M >> 1, Rh = R >> 1;
    if (k > 1) cluster_wait();
    // row pass (x): local
    row_analysis<T, LF>(f, A, B, R, lgM, tid, nt);
    cluster.sync();
    // halo: the LF-2 rows after ours (mod M) from the next CTAs
    for (int idx = tid; idx < (LF - 2) * M; idx += nt) {
      const int j = idx >> lgM, x = idx & (M - 1);
      const int r = ((crank + 1) * R + j) & (M - 1);
      B[(R + j) * M + x] = cluster.map_shared_rank(B, r >> lgR)[(r & (R - 1)) * M + x];
    }
    cluster_arrive();
    __syncthreads();
    // column pass (y), local; the epilogue inputs of kColU outputs per thread
    // are fetched before any of them is written
    constexpr int kColU = SRC == 2 ? 4 : (SRC == 1 ? 1 : 2);
    for (int idx0 = tid; idx0 < Rh * M; idx0 += kColU * nt) {
      T lo[kColU], hi[kColU];
      typename Emit<T, EPI>::Pre fa[kColU], fb[kColU];
#pragma unroll
      for (int u = 0; u < kColU; ++u) {
        const int idx = idx0 + u * nt;
        if (idx < Rh * M) {
          const int il = idx >> lgM, x = idx & (M - 1);
          const int i = crank * Rh + il;
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
          if (x >= H) fa[u] = emit.fetch(i, x, slot_hl(k, il, x));
          else if (k == J) fa[u] = emit.fetch(i, x, use_cache ? cm.ll(il, x) : -1);
          fb[u] = emit.fetch(H + i, x, slot_lh(k, il, x));
        }
      }
#pragma unroll
      for (int u = 0; u < kColU; ++u) {
        const int idx = idx0 + u * nt;
        if (idx < Rh * M) {
          const int il = idx >> lgM, x = idx & (M - 1);
          const int i = crank * Rh + il;
          if (x < H) {
            if (k == J) emit.put(i, x, J, lo[u], fa[u]);
            else A[il * H + x] = lo[u];
          } else {
            emit.put(i, x, k, lo[u], fa[u]);
          }
          emit.put(H + i, x, k, hi[u], fb[u]);
        }
      }
    }
    __syncthreads();
  }
  if (k > 1) cluster_wait();   // the next CTAs have read this CTA's halo rows
  if (k <= J) {
    // coarse levels: the remaining low-low block (side M = C) in CTA 0
    cluster.sync();   // every CTA's low-low row is written
    if (crank == 0) {
      for (int idx = tid; idx < M * M; idx += nt) {
        const int r = idx >> lgC, c = idx & (M - 1);   // M == C here
        cb[idx] = cluster.map_shared_rank(A, r)[c];   // each CTA holds one row of side M
      }
    }
    cluster.sync();
    if (crank == 0) {
      __syncthreads();
      for (; k <= J; ++k, M >>= 1) {
        const int H = M >> 1, lgMc = __ffs(M) - 1;
        row_analysis<T, LF>(f, cb, cb2, M, lgMc, tid, nt);
        __syncthreads();
        for (int idx = tid; idx < H * M; idx += nt) {
          const int i = idx >> lgMc, x = idx & (M - 1);
          T lo = T(0), hi = T(0);
#pragma unroll
          for (int t = 0; t < LF; ++t) {
            const T val = cb2[((2 * i + t) & (M - 1)) * M + x];
            lo += f.h[t] * val;
            hi += f.g[t] * val;
          }
          if (x < H && k < J) cb[i * H + x] = lo;
          else emit(i, x, (x < H) ? J : k, lo, use_cache ? cm.coarse(i, x) : -1);
          emit(H + i, x, k, hi, use_cache ? cm.coarse(H + i, x) : -1);
        }
        __syncthreads();
      }
    }
  }
  if (EPI == kEpiPlain) return;
  // one FP64 partial per CTA; the next kernel sums them
  const double2 s = block_sum2(emit.acc0, emit.acc1);
  if (tid == 0) {
    const int slot = I.cl_part_off + 2 * (it.layer * C + crank);
    I.part[slot] = s.x;
    I.part[slot + 1] = s.y;
  }
}

// ----------------------------------------------------------- k_synthesis
// SRC 0: coefficients from io.in0.  SRC 1 (PCG iteration it = flags >> 8):
// r.z of this iteration from the previous kernel's partials (the initial
// residual's for it = 0, else the update's), beta = (r.z)_it / (r.z)_(it-1),
// p <- J^-1 r + beta p written back (it = 0: p already holds J^-1 r).
// Output: io.out0 (NULL: the plan's phi).
template <typename T, int SRC, int LF>
__global__ void __launch_bounds__(kSynthThreads, 1) k_synthesis(const InstDev *__restrict__ insts,
                                                       const ClusterItem *__restrict__ items,
                                                       IoArgs io, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ CoefMap cm;
  __shared__ T s_beta;
  constexpr int HL = LF / 2 - 1;   // halo rows of the column synthesis
  pdl_trigger();
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const ClusterItem it = items[blockIdx.x / C];
  if (io.active && !io.active[it.inst]) return;   // the whole cluster leaves together
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int N = L.N, R0 = N / C, J = I.J, tid = threadIdx.x, nt = blockDim.x;
  T *buf0 = reinterpret_cast<T *>(smem_raw);
  T *buf1 = buf0 + (R0 + kMaxTaps) * N;
  T *cb = buf1 + (R0 + kMaxTaps) * N;   // low-low of the coarse stage
  T *cb2 = cb + C * C;                  // column-synthesised block
  T *cache = reinterpret_cast<T *>(smem_raw) + transform_cache_offset(N, C);
  if (tid == 0) cm.init(N, C, J, L.cache_kc, crank);
  Filt<T, LF> f;
  f.load(I);
  T *out = io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.phi);
  const T *src = static_cast<const T *>(io.in0[it.inst]);
  T *P = static_cast<T *>(I.p);
  const T *Rv = static_cast<const T *>(I.r);
  const T *Jv = static_cast<const T *>(I.jinv);
  const int iter = flags >> kIterShift;
  const bool first = (flags & kFlagFirst) != 0;
  const bool pre = I.precond != 0;
  pdl_wait();
  if (SRC == 1) {
    // r.z of this iteration; the first CTA of the instance records it
    const double prev = I.scal[kRz0 + ((iter + 1) & 1)];
    const double flag = I.scal[kFlag];
    const double rz = iter == 0 ? sum_partial(I.part + I.cl_part_off, I.n_cl_part, 0)
                                : sum_partial(I.part + I.upd_part_off, I.n_upd_blocks, 0);
    if (tid == 0) {
      double beta = 0.0;
      if (iter > 0) {
        const bool stop = flag != 0.0 || !isfinite(rz) || !(prev != 0.0);
        beta = stop ? 0.0 : rz / prev;
      }
      s_beta = T(beta);
      if (it.layer == 0 && crank == 0) I.scal[kRz0 + (iter & 1)] = rz;
    }
  }
  __syncthreads();
  const T beta = SRC == 1 ? s_beta : T(0);
  // a coefficient of an uncached level: its loads (raw), then the direction
  // update and its store (finish)
  struct Raw {
    T p, r, j;
  };
  auto raw = [&](int row, int col) -> Raw {
    const int idx = L.off + row * N + col;
    Raw v{T(0), T(0), T(1)};
    if (SRC == 0) {
      v.p = src[idx];
    } else {
      v.p = P[idx];
      if (!first) {
        v.r = Rv[idx];
        if (pre) v.j = Jv[idx];
      }
    }
    return v;
  };
  auto finish = [&](const Raw &v, int row, int col) -> T {
    if (SRC == 0 || first) return v.p;
    const T z = pre ? v.j * v.r : v.r;
    const T pn = z + beta * v.p;
    P[L.off + row * N + col] = pn;
    return pn;
  };
  // every owned coefficient of the cached levels, eight in flight per thread
  {
    const int total = cm.total();
    for (int q0 = tid; q0 < total; q0 += 8 * nt) {
      int idx[8];
      T rv[8], jv[8], pv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * nt;
        if (q < total) {
          int row, col;
          cm.pos(q, row, col);
          idx[u] = L.off + row * N + col;
          if (SRC == 0) {
            pv[u] = src[idx[u]];
          } else {
            pv[u] = P[idx[u]];
            if (!first) {
              rv[u] = Rv[idx[u]];
              jv[u] = pre ? Jv[idx[u]] : T(1);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * nt;
        if (q < total) {
          T pn = pv[u];
          if (SRC == 1 && !first) {
            const T z = pre ? jv[u] * rv[u] : rv[u];
            pn = z + beta * pv[u];
            P[idx[u]] = pn;
          }
          cache[q] = pn;
        }
      }
    }
  }
  __syncthreads();
  const int kd = cm.kd;

  T *A = buf0, *B = buf1;
  if (kd < J) {
    if (crank == 0) {
      {
        const int HJ = (N >> (J - 1)) >> 1;
        const int lgHJ = __ffs(HJ) - 1;
        for (int idx = tid; idx < HJ * HJ; idx += nt) cb[idx] = cache[cm.coarse(idx >> lgHJ, idx & (HJ - 1))];
      }
      __syncthreads();
      // rows first (x), then columns (y), as at the distributed levels and in
      // the streamed transforms, so every path gives the same bits
      const T *c3 = cache + cm.coarse(0, 0);
      for (int k = J; k > kd; --k) {
        const int M = N >> (k - 1), H = M >> 1, lgMc = __ffs(M) - 1;
        // row r < H: [LL | HL] of low-y row r; r >= H: [LH | HH] of high-y row r - H
        for (int idx = tid; idx < M * M; idx += nt) {
          const int r = idx >> lgMc, j = idx & (M - 1);
          const int q = j & 1;
          T acc = T(0);
#pragma unroll
          for (int s = 0; s < LF / 2; ++s) {
            const int t = q + 2 * s;
            const int jj = ((j - t) & (M - 1)) >> 1;
            const T lo = r < H ? cb[r * H + jj] : c3[r * C + jj];
            const T hi = c3[r * C + H + jj];
            acc += f.hs(q, s) * lo + f.gs(q, s) * hi;
          }
          cb2[r * M + j] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < M * M; idx += nt) {
          const int y = idx >> lgMc, x = idx & (M - 1);
          const int p = y & 1;
          T acc = T(0);
#pragma unroll
          for (int s = 0; s < LF / 2; ++s) {
            const int t = p + 2 * s;
            const int ii = ((y - t) & (M - 1)) >> 1;
            acc += f.hs(p, s) * cb2[ii * M + x] + f.gs(p, s) * cb2[(H + ii) * M + x];
          }
          cb[y * M + x] = acc;
        }
        __syncthreads();
      }
    }
    cluster.sync();
    // level kd: M = 2C, one low-low row per CTA
    const T *c0 = cluster.map_shared_rank(cb, 0);
    for (int j = tid; j < C; j += nt) A[j] = c0[crank * C + j];
  } else {
    const int M = N >> (J - 1), H = M >> 1, Rh = (M / C) >> 1, lgH = __ffs(H) - 1;
    for (int idx = tid; idx < Rh * H; idx += nt) A[idx] = cache[cm.ll(idx >> lgH, idx & (H - 1))];
  }
  __syncthreads();

  // Distributed levels, per level: own coefficient rows (V), their row
  // synthesis (x) into U after HL halo rows, one cluster barrier, the halo
  // rows of the previous CTAs, then the column synthesis (y) into V, which is
  // the next level's low-low block.  The halo reads are released with an
  // arrive; the matching wait comes before this CTA next overwrites U (the
  // next level's first step, or the end of the kernel).
  const int lgN = L.log2N, lgC = __ffs(C) - 1;
  T *U = A, *V = B;   // U holds the low-low block of level kd
  for (int k = kd; k >= 1; --k) {
    const int lgM = lgN - (k - 1), lgRh = lgM - lgC - 1;
    const int M = N >> (k - 1), H = M >> 1, R = M >> lgC, Rh = R >> 1;
    const bool cached = k >= cm.kc;
    if (k < kd) cluster_wait();
    // step 1: own rows, low-y (LL | HL) then high-y (LH | HH), into V; the
    // coefficients of uncached levels (with the fused direction update) are
    // loaded kRowU per thread before any is updated
    if (cached) {
      for (int idx = tid; idx < Rh * M; idx += nt) {
        const int jl = idx >> lgM, x = idx & (M - 1);
        V[jl * M + x] = x < H ? U[jl * H + x] : cache[cm.hl(k, jl, x)];
        V[(Rh + jl) * M + x] = cache[cm.lh(k, jl, x)];
      }
    } else {
      constexpr int kRowU = 4;
      for (int idx0 = tid; idx0 < Rh * M; idx0 += kRowU * nt) {
        Raw ra[kRowU], rb[kRowU];
#pragma unroll
        for (int u = 0; u < kRowU; ++u) {
          const int idx = idx0 + u * nt;
          if (idx < Rh * M) {
            const int jl = idx >> lgM, x = idx & (M - 1);
            const int i = crank * Rh + jl;
            if (x >= H) ra[u] = raw(i, x);
            rb[u] = raw(H + i, x);
          }
        }
#pragma unroll
        for (int u = 0; u < kRowU; ++u) {
          const int idx = idx0 + u * nt;
          if (idx < Rh * M) {
            const int jl = idx >> lgM, x = idx & (M - 1);
            const int i = crank * Rh + jl;
            V[jl * M + x] = x < H ? U[jl * H + x] : finish(ra[u], i, x);
            V[(Rh + jl) * M + x] = finish(rb[u], H + i, x);
          }
        }
      }
    }
    __syncthreads();
    // step 2: row synthesis (x) into U: low-y rows at XL, high-y rows at XH
    T *XL = U;                      // HL halo rows, then Rh own rows
    T *XH = U + (HL + Rh) * M;      // same layout
    for (int idx = tid; idx < 2 * Rh * M; idx += nt) {
      const int r = idx >> lgM, j = idx & (M - 1);
      const int q = j & 1;
      const T *row = V + r * M;
      T acc = T(0);
#pragma unroll
      for (int s = 0; s < LF / 2; ++s) {
        const int jj = ((j >> 1) - s) & (H - 1);
        acc += f.hs(q, s) * row[jj] + f.gs(q, s) * row[H + jj];
      }
      (r < Rh ? XL + (HL + r) * M : XH + (HL + r - Rh) * M)[j] = acc;
    }
    cluster.sync();
    // halo: the HL rows before ours (mod H) from the previous CTAs
    for (int idx = tid; idx < HL * M; idx += nt) {
      const int j = idx >> lgM, x = idx & (M - 1);
      const int ii = (crank * Rh - HL + j) & (H - 1);
      const int owner = ii >> lgRh, li = ii & (Rh - 1);
      const T *oU = cluster.map_shared_rank(U, owner);
      XL[j * M + x] = oU[(HL + li) * M + x];
      XH[j * M + x] = oU[(HL + Rh + HL + li) * M + x];
    }
    cluster_arrive();
    __syncthreads();
    // step 3: column synthesis (y) of own output rows
    for (int idx = tid; idx < R * M; idx += nt) {
      const int yl = idx >> lgM, x = idx & (M - 1);
      const int p = yl & 1;
      const int base = ((yl - p) >> 1) + HL;
      T acc = T(0);
#pragma unroll
      for (int s = 0; s < LF / 2; ++s)
        acc += f.hs(p, s) * XL[(base - s) * M + x] + f.gs(p, s) * XH[(base - s) * M + x];
      if (k == 1) out[L.off + (crank * R + yl) * N + x] = acc;
      else V[yl * M + x] = acc;
    }
    __syncthreads();
    T *tmp = U;
    U = V;
    V = tmp;
  }
  if (kd >= 1) cluster_wait();   // the next CTAs have read this CTA's halo rows
}

// -------------------------------------------------------------- k_update
// alpha = (r.z)_it / (p.Ap) from the analysis partials; x += alpha p,
// r -= alpha q, z = J^-1 r; partials r.z and r.r per CTA.  io.out0: x.
// Four consecutive elements per thread and pass (kUpdChunk = 4 * kThreads);
// a CTA makes it.chunks passes over consecutive chunks.
template <typename T>
__device__ __forceinline__ void upd_load(const T *X, const T *R, const T *P, const T *Q, const T *Jv, int precond,
                                         int n, int i0, bool vec, T *xv, T *rv, T *pv, T *qv, T *jv) {
  if (vec) {
    const float4 x4 = reinterpret_cast<const float4 *>(X)[i0 >> 2];
    const float4 r4 = reinterpret_cast<const float4 *>(R)[i0 >> 2];
    const float4 p4 = reinterpret_cast<const float4 *>(P)[i0 >> 2];
    const float4 q4 = reinterpret_cast<const float4 *>(Q)[i0 >> 2];
    const float4 j4 = precond ? reinterpret_cast<const float4 *>(Jv)[i0 >> 2] : make_float4(1.f, 1.f, 1.f, 1.f);
    xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
    rv[0] = r4.x; rv[1] = r4.y; rv[2] = r4.z; rv[3] = r4.w;
    pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
    qv[0] = q4.x; qv[1] = q4.y; qv[2] = q4.z; qv[3] = q4.w;
    jv[0] = j4.x; jv[1] = j4.y; jv[2] = j4.z; jv[3] = j4.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = i0 + u < n ? i0 + u : n - 1;
      xv[u] = X[idx];
      rv[u] = R[idx];
      pv[u] = P[idx];
      qv[u] = Q[idx];
      jv[u] = precond ? Jv[idx] : T(1);
    }
  }
}

template <typename T>
__device__ __forceinline__ void upd_store(T *X, T *R, int n, int i0, bool vec, const T *xv, const T *rv) {
  if (vec) {
    reinterpret_cast<float4 *>(X)[i0 >> 2] = make_float4(xv[0], xv[1], xv[2], xv[3]);
    reinterpret_cast<float4 *>(R)[i0 >> 2] = make_float4(rv[0], rv[1], rv[2], rv[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n) {
        X[i0 + u] = xv[u];
        R[i0 + u] = rv[u];
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(const InstDev *__restrict__ insts,
                                                    const UpdItem *__restrict__ items, IoArgs io,
                                                    int flags) {
  __shared__ T s_alpha;
  pdl_trigger();
  const UpdItem it = items[blockIdx.x];
  if (io.active && !io.active[it.inst]) return;
  const InstDev *I = insts + it.inst;
  T *X = static_cast<T *>(io.out0[it.inst]);
  T *R = static_cast<T *>(I->r);
  const int iter = flags >> kIterShift;
  const T *P = dir_buffer<T>(*I, iter);
  const T *Q = static_cast<const T *>(I->q);
  const T *Jv = static_cast<const T *>(I->jinv);
  const int precond = I->precond;
  const int n = I->n;
  pdl_wait();
  const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(R) |
                         reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(Q) |
                         reinterpret_cast<uintptr_t>(Jv)) & 15) == 0;
  // the first pass's vectors do not depend on alpha: their loads go out first
  int i0 = it.start + 4 * threadIdx.x;
  bool vec = sizeof(T) == 4 && i0 + 3 < n && aligned;
  T xv[4], rv[4], pv[4], qv[4], jv[4];
  upd_load(X, R, P, Q, Jv, precond, n, i0, vec, xv, rv, pv, qv, jv);
  {
    const double rz = I->scal[kRz0 + (iter & 1)];
    const double flag = I->scal[kFlag];
    const double pq = sum_partial(I->part + I->cl_part_off, I->n_cl_part, 0);
    if (threadIdx.x == 0) {
      // r = 0 (so p = 0 and p.Ap = 0) means the iterate is already exact: step 0
      const bool exact = (pq == 0.0 && rz == 0.0);
      const bool bad = !exact && (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz) || flag != 0.0);
      if (bad && it.blk == 0) {
        I->scal[kFlag] = 1.0;
        if (I->bd_word) *reinterpret_cast<volatile int *>(I->bd_word) = 1;
      }
      s_alpha = T((bad || exact) ? 0.0 : rz / pq);
    }
    __syncthreads();
  }
  const T alpha = s_alpha;
  // a step of zero (breakdown, or an exact iterate) leaves x and r as they are,
  // even where p or q is not finite: the iterate is frozen
  const bool step = alpha != T(0);
  Acc<T> rz, rr;
  for (int c = 0;;) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (step) {
        xv[u] += alpha * pv[u];
        rv[u] -= alpha * qv[u];
      }
      const T z = precond ? jv[u] * rv[u] : rv[u];
      if (i0 + u < n) {
        rz.add_prod(rv[u], z);
        rr.add_prod(rv[u], rv[u]);
      }
    }
    upd_store(X, R, n, i0, vec, xv, rv);
    if (++c >= it.chunks) break;
    i0 += kUpdChunk;
    vec = sizeof(T) == 4 && i0 + 3 < n && aligned;
    upd_load(X, R, P, Q, Jv, precond, n, i0, vec, xv, rv, pv, qv, jv);
  }
  const double2 s = block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    I->part[I->upd_part_off + 2 * it.blk] = s.x;
    I->part[I->upd_part_off + 2 * it.blk + 1] = s.y;
  }
}

// ---------------------------------------------------------------- k_slopes
// Noise-free measurement A phi (eq. atm_tomo): Fried slopes of every valid
// subaperture, or the two mean slopes of a tip/tilt-only sensor.
// io.in0: layers; io.out0: slopes.  grid.y = sensor.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_slopes(const InstDev *__restrict__ insts, IoArgs io) {
  __shared__ InstDev sI;
  load_inst(&sI, insts);
  const InstDev &I = sI;
  const int m = blockIdx.y;
  const WfsDev W = I.wfs[m];
  const T *phi = static_cast<const T *>(io.in0[0]);
  T *out = static_cast<T *>(io.out0[0]);
  const int nc = W.nc, n = W.n;
  if (W.kind == kTTOnly) {
    if (blockIdx.x != 0) return;
    const T *et = static_cast<const T *>(I.edge_t) + 2 * W.edge_off;
    const int *eidx = I.edge_idx + W.edge_off;
    Acc<double> ax, ay;
    for (int e = threadIdx.x; e < W.n_edge; e += blockDim.x) {
      const int c = eidx[e];
      const T ps = trace_corner<T>(I, m, nc, phi, c % nc, c / nc);
      ax.add_prod(double(et[2 * e]), double(ps));
      ay.add_prod(double(et[2 * e + 1]), double(ps));
    }
    const double2 s = block_sum2(ax, ay);
    if (threadIdx.x == 0) {
      out[W.slope_off] = T(s.x / W.S);
      out[W.slope_off + 1] = T(s.y / W.S);
    }
    return;
  }
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int a = idx % n, b = idx / n;
  const int j = I.sub_idx[W.sub_off + idx];
  if (j < 0) return;
  const T p00 = trace_corner<T>(I, m, nc, phi, a, b);
  const T p10 = trace_corner<T>(I, m, nc, phi, a + 1, b);
  const T p01 = trace_corner<T>(I, m, nc, phi, a, b + 1);
  const T p11 = trace_corner<T>(I, m, nc, phi, a + 1, b + 1);
  out[W.slope_off + j] = T(0.5) * (p10 + p11 - p00 - p01);
  out[W.slope_off + W.S + j] = T(0.5) * (p01 + p11 - p00 - p10);
}

// --------------------------------------------------------------- k_jacobi
// Modified Jacobi diagonal (Sec. 5.1), exactly, at plan time:
//   J_lambda = sum_{m LGS} sigma_m^-2 ||Gamma_m P_m w_lambda||^2 + alpha D_lambda.
// The basis function is separable, w = u(x) v(y), and so are the traced corner
// coordinates, hence P_m w = U(a) V(b) and the Fried slopes are
// sx = dU(a) mV(b), sy = mU(a) dV(b) (d: forward difference, m: two-point
// mean).  Summing their squares over the valid subapertures of row b uses
// prefix sums of dU^2 and mU^2 over the row's runs of valid subapertures.
// One warp per coefficient; FP64 throughout.
__global__ void k_jacobi(const InstDev *__restrict__ insts, const double *__restrict__ prof,
                         const int *__restrict__ prof_off, const double *__restrict__ pos_fd,
                         double *__restrict__ jdiag, void *jinv, int precision, int nc_max,
                         double alpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InstDev &I = insts[0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lam = blockIdx.x * (blockDim.x >> 5) + warp;
  double *U = reinterpret_cast<double *>(smem_raw) + warp * 4 * (nc_max + 1);
  double *V = U + (nc_max + 1);
  double *Pd = V + (nc_max + 1);
  double *Pm = Pd + (nc_max + 1);
  if (lam >= I.n) return;
  int l = 0;
  while (l + 1 < I.n_layers && I.layers[l + 1].off <= lam) ++l;
  const LayerDev &L = I.layers[l];
  const int N = L.N, J = I.J;
  const int rr = (lam - L.off) / N, cc = (lam - L.off) % N;
  const int mx = rr > cc ? rr : cc;
  int k = J;
  for (int kk = 1; kk <= J; ++kk)
    if (mx >= (N >> kk)) {
      k = kk;
      break;
    }
  const int H = (N >> (k - 1)) >> 1;
  const int kx = cc < H ? 0 : 1, px = cc < H ? cc : cc - H;
  const int ky = rr < H ? 0 : 1, py = rr < H ? rr : rr - H;
  const double *ux = prof + prof_off[(l * (J + 1) + k) * 2 + kx];
  const double *uy = prof + prof_off[(l * (J + 1) + k) * 2 + ky];
  const int sx = px << k, sy = py << k;
  double acc = 0.0;
  for (int m = 0; m < I.n_wfs; ++m) {
    const WfsDev &W = I.wfs[m];
    if (!W.is_lgs) continue;
    const int nc = W.nc, n = W.n;
    const int po = I.pos_off[m * I.n_layers + l];
    for (int a = lane; a < nc; a += 32) {
      const int x0 = I.pos_i0[po + a], y0 = I.pos_i0[po + nc + a];
      const double fx = pos_fd[po + a], fy = pos_fd[po + nc + a];
      U[a] = (1.0 - fx) * ux[(x0 - sx) & (N - 1)] + fx * ux[(x0 + 1 - sx) & (N - 1)];
      V[a] = (1.0 - fy) * uy[(y0 - sy) & (N - 1)] + fy * uy[(y0 + 1 - sy) & (N - 1)];
    }
    __syncwarp();
    if (lane == 0) {
      Pd[0] = 0.0;
      Pm[0] = 0.0;
      for (int a = 0; a < n; ++a) {
        const double d = U[a + 1] - U[a], mm = 0.5 * (U[a] + U[a + 1]);
        Pd[a + 1] = Pd[a] + d * d;
        Pm[a + 1] = Pm[a] + mm * mm;
      }
    }
    __syncwarp();
    double part = 0.0;
    const int *rows = I.run_rows + W.run_off;
    for (int b = lane; b < n; b += 32) {
      const double dv = V[b + 1] - V[b], mv = 0.5 * (V[b] + V[b + 1]);
      double sd = 0.0, sm = 0.0;
      for (int q = rows[b]; q < rows[b + 1]; ++q) {
        const int2 run = I.run_ab[q];
        sd += Pd[run.y] - Pd[run.x];
        sm += Pm[run.y] - Pm[run.x];
      }
      part += mv * mv * sd + dv * dv * sm;
    }
    acc += W.inv_sigma2 * part;
    __syncwarp();
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    // alpha < 0: the plan's own alpha D; otherwise alpha D for the given alpha
    const double Jv = acc + (alpha < 0.0 ? L.dalpha[k] : alpha * L.dprior[k]);
    jdiag[lam] = Jv;
    if (jinv) {
      if (precision) static_cast<double *>(jinv)[lam] = 1.0 / Jv;
      else static_cast<float *>(jinv)[lam] = float(1.0 / Jv);
    }
  }
}

// ------------------------------------------------------------- launchers

namespace {

template <typename K>
cudaError_t allow_cluster(K kernel) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxTransformSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

template <typename T, int LF>
cudaError_t allow_lf() {
  cudaError_t e = cudaSuccess;
#define TOMO_CFG(K) if (e == cudaSuccess) e = allow_cluster(K)
  TOMO_CFG((k_synthesis<T, 0, LF>));
  TOMO_CFG((k_synthesis<T, 1, LF>));
  TOMO_CFG((k_analysis<T, 0, kEpiPlain, LF>));
  TOMO_CFG((k_analysis<T, 1, kEpiPlain, LF>));
  TOMO_CFG((k_analysis<T, 1, kEpiOp, LF>));
  TOMO_CFG((k_analysis<T, 1, kEpiResid, LF>));
  TOMO_CFG((k_analysis<T, 2, kEpiPlain, LF>));
  TOMO_CFG((k_analysis<T, 2, kEpiOp, LF>));
  TOMO_CFG((k_analysis<T, 2, kEpiResid, LF>));
#undef TOMO_CFG
  return e;
}

template <typename T>
cudaError_t allow_type() {
  cudaError_t e = allow_lf<T, 2>();
  if (e == cudaSuccess) e = allow_lf<T, 4>();
  if (e == cudaSuccess) e = allow_lf<T, 6>();
  if (e == cudaSuccess) e = allow_lf<T, 8>();
  const void *fwd[12] = {reinterpret_cast<const void *>(k_forward<T, 0, false, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 1, false, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 2, false, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 0, true, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 1, true, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 2, true, kFwdThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 0, false, kThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 1, false, kThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 2, false, kThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 0, true, kThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 1, true, kThreads>),
                         reinterpret_cast<const void *>(k_forward<T, 2, true, kThreads>)};
  for (int i = 0; i < 12 && e == cudaSuccess; ++i)
    e = cudaFuncSetAttribute(fwd[i], cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxForwardSmem);
  return e;
}

template <typename T, int LF>
cudaError_t synth_lf(int src, int flags, const InstDev *insts, const ClusterItem *items, int n_clusters,
                     int C, size_t smem, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_clusters * C);
  // two CTAs of 256 threads per SM when their shared memory allows (two clusters per GPC),
  // else one CTA of 512
  const int nt = smem <= kTwoPerSmSmem ? kSynthThreads / 2 : kSynthThreads;
  return src ? launch_ex(k_synthesis<T, 1, LF>, g, nt, C, smem, s, insts, items, io, flags)
             : launch_ex(k_synthesis<T, 0, LF>, g, nt, C, smem, s, insts, items, io, flags);
}

template <typename T>
cudaError_t synth_t(int src, int lf, int flags, const InstDev *insts, const ClusterItem *items,
                    int n_clusters, int C, size_t smem, const IoArgs &io, cudaStream_t s) {
  switch (lf) {
    case 2: return synth_lf<T, 2>(src, flags, insts, items, n_clusters, C, smem, io, s);
    case 4: return synth_lf<T, 4>(src, flags, insts, items, n_clusters, C, smem, io, s);
    case 6: return synth_lf<T, 6>(src, flags, insts, items, n_clusters, C, smem, io, s);
    case 8: return synth_lf<T, 8>(src, flags, insts, items, n_clusters, C, smem, io, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int LF>
cudaError_t anal_lf(int src, int epi, int flags, const InstDev *insts, const ClusterItem *items,
                    int n_clusters, int C, size_t smem, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_clusters * C);
  // two CTAs of 512 threads per SM when their shared memory allows, else one of 1024
  const int nt = smem <= kTwoPerSmSmem ? kAnalysisThreads : kAnalysisThreadsMax;
#define TOMO_AN(S, E) launch_ex(k_analysis<T, S, E, LF>, g, nt, C, smem, s, insts, items, io, flags)
  if (src == 0) return TOMO_AN(0, kEpiPlain);
  if (src == 2) {
    if (epi == kEpiPlain) return TOMO_AN(2, kEpiPlain);
    if (epi == kEpiOp) return TOMO_AN(2, kEpiOp);
    return TOMO_AN(2, kEpiResid);
  }
  if (epi == kEpiPlain) return TOMO_AN(1, kEpiPlain);
  if (epi == kEpiOp) return TOMO_AN(1, kEpiOp);
  return TOMO_AN(1, kEpiResid);
#undef TOMO_AN
}

template <typename T>
cudaError_t anal_t(int src, int epi, int lf, int flags, const InstDev *insts, const ClusterItem *items,
                   int n_clusters, int C, size_t smem, const IoArgs &io, cudaStream_t s) {
  switch (lf) {
    case 2: return anal_lf<T, 2>(src, epi, flags, insts, items, n_clusters, C, smem, io, s);
    case 4: return anal_lf<T, 4>(src, epi, flags, insts, items, n_clusters, C, smem, io, s);
    case 6: return anal_lf<T, 6>(src, epi, flags, insts, items, n_clusters, C, smem, io, s);
    case 8: return anal_lf<T, 8>(src, epi, flags, insts, items, n_clusters, C, smem, io, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = allow_type<float>();
  if (e == cudaSuccess) e = allow_type<double>();
  if (e == cudaSuccess) e = configure_streamed_kernels();
  if (e == cudaSuccess) e = configure_gather_kernels();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  return e;
}

size_t forward_smem(int n_layers, int precision) {
  return fwd_table_bytes(n_layers, precision ? 8 : 4);
}

cudaError_t launch_synthesis(int precision, int src, int lf, int flags, const InstDev *insts,
                             const ClusterItem *items, int n_clusters, int C, size_t smem,
                             const IoArgs &io, cudaStream_t s) {
  return precision == 0 ? synth_t<float>(src, lf, flags, insts, items, n_clusters, C, smem, io, s)
                        : synth_t<double>(src, lf, flags, insts, items, n_clusters, C, smem, io, s);
}

cudaError_t launch_analysis(int precision, int src, int epi, int lf, int flags, const InstDev *insts,
                             const ClusterItem *items, int n_clusters, int C, size_t smem, const IoArgs &io,
                             cudaStream_t s) {
  return precision == 0 ? anal_t<float>(src, epi, lf, flags, insts, items, n_clusters, C, smem, io, s)
                        : anal_t<double>(src, epi, lf, flags, insts, items, n_clusters, C, smem, io, s);
}

template <typename T, bool EL, int NT>
cudaError_t fwd_nt(int mode, dim3 g, size_t sm, cudaStream_t s, const InstDev *insts, const FwdItem *items,
                   const IoArgs &io) {
  if (mode == 0) return launch_ex(k_forward<T, 0, EL, NT>, g, NT, 0, sm, s, insts, items, io);
  if (mode == 1) return launch_ex(k_forward<T, 1, EL, NT>, g, NT, 0, sm, s, insts, items, io);
  return launch_ex(k_forward<T, 2, EL, NT>, g, NT, 0, sm, s, insts, items, io);
}

template <typename T, bool EL>
cudaError_t fwd_t(int mode, dim3 g, int nt, size_t sm, cudaStream_t s, const InstDev *insts,
                  const FwdItem *items, const IoArgs &io) {
  return nt == kFwdThreads ? fwd_nt<T, EL, kFwdThreads>(mode, g, sm, s, insts, items, io)
                           : fwd_nt<T, EL, kThreads>(mode, g, sm, s, insts, items, io);
}

cudaError_t launch_forward(int precision, int mode, int max_layers, int elong, const InstDev *insts,
                           const FwdItem *items, int n_items, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_items);
  const int nt = n_items <= kFwdSmallLaunch ? kFwdThreads : kThreads;
  const size_t sm = forward_smem(max_layers, precision);
  if (precision == 0)
    return elong ? fwd_t<float, true>(mode, g, nt, sm, s, insts, items, io)
                 : fwd_t<float, false>(mode, g, nt, sm, s, insts, items, io);
  return elong ? fwd_t<double, true>(mode, g, nt, sm, s, insts, items, io)
               : fwd_t<double, false>(mode, g, nt, sm, s, insts, items, io);
}

cudaError_t launch_update(int precision, int flags, const InstDev *insts, const UpdItem *items,
                          int n_items, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_items);
  return precision == 0 ? launch_ex(k_update<float>, g, kThreads, 0, 0, s, insts, items, io, flags)
                        : launch_ex(k_update<double>, g, kThreads, 0, 0, s, insts, items, io, flags);
}

cudaError_t launch_slopes(int precision, const InstDev *insts, int n_wfs, int max_sub2,
                          const IoArgs &io, cudaStream_t s) {
  const dim3 g((max_sub2 + kThreads - 1) / kThreads, n_wfs);
  if (precision == 0) k_slopes<float><<<g, kThreads, 0, s>>>(insts, io);
  else k_slopes<double><<<g, kThreads, 0, s>>>(insts, io);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(const InstDev *insts, int n, const double *prof, const int *prof_off,
                          const double *pos_fd, double *jdiag, void *jinv, int precision,
                          int nc_max, double alpha, cudaStream_t s) {
  const size_t per_warp = 4 * static_cast<size_t>(nc_max + 1) * sizeof(double);
  int warps = static_cast<int>((96 * 1024) / per_warp);
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const size_t smem = per_warp * warps;
  const int blocks = (n + warps - 1) / warps;
  k_jacobi<<<blocks, warps * 32, smem, s>>>(insts, prof, prof_off, pos_fd, jdiag, jinv, precision,
                                           nc_max, alpha);
  return cudaGetLastError();
}

}  // namespace tomo
