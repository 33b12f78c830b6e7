// The fitting step (Sec. 4.1, eqs. fit_step_ideal / fit_step_min): mirror
// commands a from the reconstructed layers phi by CG on H^T H a = H^T P phi,
// tomo_reconstruct, slopes to commands in one graph, and the closed loop of
// Sec. 4.2 (Algorithm 4.1): the mirrors as the sensors see them (A_hat) and one
// pseudo-open-loop control step.
//
// H_j a (x) = sum_k a_k(x + h_k theta_j), each mirror a piecewise-bilinear
// function of its actuator grid; P_j phi (x) = sum_l phi_l(x + h_l theta_j)
// (eq. ngsproj), bilinear on the periodic layer grids; x runs over the corners
// of the valid subapertures of the aperture sampling grid.  H^T H is constant:
// it is assembled once on the host (FP64, CSR) and each CG iteration is two
// kernels:
//
//   k_fit_form     the update of the previous iteration and the new direction:
//                  a += alpha p, r -= alpha q, p = r + beta p  [actuator per thread;
//                  not in the first iteration, whose direction is r itself]
//   k_fit_iter     q = H^T H p [warp per nonempty row] and p.q, r.q, q.q, r.r
//                  partials per block; the block that takes the last ticket
//                  sums them and leaves alpha = r.r / p.q and beta of the next
//                  iteration, its r.r taken from the recurrence
//                  rr - 2 alpha r.q + alpha^2 q.q
//
// and k_fit_finish applies the last iteration's a += alpha p.
//
// The right-hand side and the initial residual stay matrix-free:
//
//   k_fit_mirror   u_j = P_j phi - H_j a on every (direction, corner)  [corner per thread]
//   k_fit_adjoint  r = sum_j H_j^T u_j as a gather over per-actuator tap
//                  windows                                          [4 threads per actuator]
//
// The tap tables (corner -> actuator and corner -> layer node, and for H^T
// each actuator's window of corners with its weights) are built in FP64 on
// the host from the same corner -> actuator taps, so the gather is the exact
// transpose of the mirror kernel.  Inner products are accumulated in a fixed
// order, so results are bitwise reproducible: for FP32 in double-float pairs
// (per thread, per block record and in the sums of the records), since FP64
// arithmetic is slow on this part.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tomo.h"
#include "common.h"
#include "device_util.cuh"
#include "launch.h"
#include "plan_internal.h"

namespace tomo {

constexpr int kFitThreads = 256;   // equals kFwdTile^2: one thread per subaperture of an A_hat tile
constexpr int kFitIterThreads = 1024;   // k_fit_iter: 32 rows per block; the last block updates with all
constexpr int kFitRmsThreads = 1024;
constexpr int kMaxDm = 4;
constexpr int kMaxFitDirs = 256;
constexpr int kFitDirBatch = 4;   // directions whose gather loads one thread issues together
constexpr int kSpmvBatch = 4;     // matrix entries whose loads one lane issues together (fit_row)

// Everything the fitting kernels read (passed by value).
struct FitDev {
  int n_dir, n_dm, nc, n_layers;
  int n_act, kw, nblk_adj, nblk_upd, n_points, n_rows;
  int dm_n[kMaxDm], dm_off[kMaxDm], w_off[kMaxDm];
  const unsigned char *act;   // nc*nc corner mask
  const int2 *lay;            // per layer (N, offset in the layer vector)
  const int *hx0, *hy0;       // [dm][dir][nc]: left / lower actuator of each corner column / row
  const void *hfx, *hfy;      //   and its fraction (T)
  const int *px0, *py0;       // [layer][dir][nc]: left / lower layer node (mod N)
  const void *pfx, *pfy;      //   and its fraction (T)
  const int *wx0, *wy0;       // per (dm, dir, actuator column / row): first corner of its window
  const void *wxw, *wyw;      //   kw weights (T), zero beyond the window
  void *u;                    // [dir][nc*nc]
  void *r, *q, *p;            // [n_act]: the CG residual, H^T H p and direction
  const void *nrm_cv;         // H^T H in CSR, its entries (column, value): int and float (8 B), or int,
                              // 0 and double (16 B)
  const int4 *nrm_desc;       // its rows (row, first entry, end, 0) by decreasing length: warp w takes
                              // desc[w]; the n_rows nonempty rows come first
  int nblk_spmv, nblk_iter;
  double *rec;                // per k_fit_iter block (32 B): p.q, r.q, q.q, r.r as FP32 pairs or FP64
  double *cg;                 // CG scalars of iteration it: alpha in cg[it & 1], beta in cg[2 + (it & 1)]
  unsigned *ticket;           // blocks of k_fit_iter done; reset by the last one
  double *flag;               // nonzero after a breakdown
  // the mirrors seen by the plan's sensors (A_hat)
  int n_ms_items;
  const int4 *ms_items;       // (sensor, first subaperture column, row, tip/tilt only): a 16x16 tile
                              // of a full sensor, or a whole tip/tilt-only sensor
  const int4 *sens;           // per sensor: slope offset, valid subapertures S, corners per side
  const int4 *sens_off;       // per sensor: first (sensor, mirror) tap entry, subaperture index table,
                              // first pupil-edge corner, pupil-edge corners
  const int *sx0, *sy0;       // per (sensor, mirror): left / lower actuator of each corner column / row
  const void *sfx, *sfy;      //   and its fraction (T)
  const int *sidx;            // per sensor n x n: slope index of each subaperture, -1 if not valid
  const int *e_idx;           // pupil-edge corners (b nc + a) of every sensor
  const void *e_t;            //   and (Gamma^T 1_x, Gamma^T 1_y) there (T pairs)
  void *s_ol;                 // pseudo-open-loop slopes (the plan's slope layout)
};

__device__ __forceinline__ float fit_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fit_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Accumulators in shared memory and in the k_fit_iter block records: an FP32
// pair (hi, lo) for FP32, an FP64 value for FP64; sums over a warp leave the
// result in lane 0.
template <typename T>
struct AccIO;
template <>
struct AccIO<float> {
  using S = float2;
  static __device__ __forceinline__ S pack(const Acc<float> &a) { return make_float2(a.hi, a.lo); }
  static __device__ __forceinline__ void add(Acc<float> &a, S v) { a.merge(v.x, v.y); }
  static __device__ __forceinline__ void add_double(Acc<float> &a, double v) {
    const float hi = __double2float_rn(v);
    a.merge(hi, __double2float_rn(v - double(hi)));
  }
  static __device__ __forceinline__ void warp(Acc<float> &a) { warp_merge_down(a); }
};
template <>
struct AccIO<double> {
  using S = double;
  static __device__ __forceinline__ S pack(const Acc<double> &a) { return a.s; }
  static __device__ __forceinline__ void add(Acc<double> &a, S v) { a.s += v; }
  static __device__ __forceinline__ void add_double(Acc<double> &a, double v) { a.s += v; }
  static __device__ __forceinline__ void warp(Acc<double> &a) { a.s = warp_sum(a.s); }
};

// One (column, value) entry of H^T H.
__device__ __forceinline__ void fit_entry(const void *cv, int e, int &c, float &w) {
  const int2 x = static_cast<const int2 *>(cv)[e];
  c = x.x;
  w = __int_as_float(x.y);
}
__device__ __forceinline__ void fit_entry(const void *cv, int e, int &c, double &w) {
  const int4 x = static_cast<const int4 *>(cv)[e];
  c = x.x;
  w = __hiloint2double(x.w, x.z);
}

// u_j = P_j phi - H_j x on every (direction, corner); phi = NULL: no layers,
// x = NULL: no mirrors.
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_fit_mirror(FitDev F, const T *__restrict__ x,
                                                           const T *__restrict__ phi) {
  pdl_trigger();
  const int j = blockIdx.y, nc = F.nc, nn = nc * nc;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nn) return;
  const bool on = F.act[c];
  const int a = c % nc, b = c / nc;
  pdl_wait();
  T val = T(0);
  if (on && phi) {
    const T *fx = static_cast<const T *>(F.pfx), *fy = static_cast<const T *>(F.pfy);
    for (int l = 0; l < F.n_layers; ++l) {
      const int2 L = F.lay[l];
      const int tx = (l * F.n_dir + j) * nc + a, ty = (l * F.n_dir + j) * nc + b;
      const int x0 = F.px0[tx], y0 = F.py0[ty];
      const int x1 = (x0 + 1) & (L.x - 1), y1 = (y0 + 1) & (L.x - 1);
      const T wx = fx[tx], wy = fy[ty];
      const T *g = phi + L.y;
      val += (T(1) - wy) * ((T(1) - wx) * g[y0 * L.x + x0] + wx * g[y0 * L.x + x1]) +
             wy * ((T(1) - wx) * g[y1 * L.x + x0] + wx * g[y1 * L.x + x1]);
    }
  }
  if (on && x) {
    const T *fx = static_cast<const T *>(F.hfx), *fy = static_cast<const T *>(F.hfy);
    T h = T(0);
#pragma unroll
    for (int k = 0; k < kMaxDm; ++k) {
      if (k >= F.n_dm) break;
      const int n = F.dm_n[k], o = F.dm_off[k];
      const int tx = (k * F.n_dir + j) * nc + a, ty = (k * F.n_dir + j) * nc + b;
      const int x0 = F.hx0[tx], y0 = F.hy0[ty];
      const T wx1 = fx[tx], wy1 = fy[ty];
      const T wx[2] = {T(1) - wx1, wx1}, wy[2] = {T(1) - wy1, wy1};
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const int iy = y0 + dy;
        if (iy < 0 || iy >= n) continue;
        T row = T(0);
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int ix = x0 + dx;
          if (ix >= 0 && ix < n) row += wx[dx] * x[o + iy * n + ix];
        }
        h += wy[dy] * row;
      }
    }
    val -= h;
  }
  static_cast<T *>(F.u)[j * nn + c] = val;
}

// sum_j H_j^T u_j for actuator `act` of mirror k (column i, row jj), over the
// directions j = g, g+4, ...; the four direction groups are then combined
// across lanes in a fixed order.
template <typename T, int KW>
__device__ __forceinline__ T fit_gather(const FitDev &F, int k, int i, int jj, int g) {
  const int n = F.dm_n[k], nc = F.nc, nn = nc * nc;
  const T *u = static_cast<const T *>(F.u);
  const T *wxw = static_cast<const T *>(F.wxw), *wyw = static_cast<const T *>(F.wyw);
  T s = T(0);
  // kFitDirBatch of this thread's directions at a time: their window starts,
  // then their weights and corners, are loaded without dependences between them
  for (int j0 = g; j0 < F.n_dir; j0 += 4 * kFitDirBatch) {
    int ex[kFitDirBatch], ey[kFitDirBatch], base[kFitDirBatch];
#pragma unroll
    for (int b = 0; b < kFitDirBatch; ++b) {
      const int j = min(j0 + 4 * b, F.n_dir - 1);
      ex[b] = F.w_off[k] + j * n + i;
      ey[b] = F.w_off[k] + j * n + jj;
      base[b] = j * nn + F.wy0[ey[b]] * nc + F.wx0[ex[b]];
    }
#pragma unroll
    for (int b = 0; b < kFitDirBatch; ++b) {
      if (j0 + 4 * b >= F.n_dir) break;
      const T *ux = u + base[b];
      T wx[KW];
#pragma unroll
      for (int t = 0; t < KW; ++t) wx[t] = wxw[ex[b] * KW + t];
      T acc = T(0);
#pragma unroll
      for (int t2 = 0; t2 < KW; ++t2) {
        T row = T(0);
#pragma unroll
        for (int t1 = 0; t1 < KW; ++t1) row += wx[t1] * ux[t2 * nc + t1];
        acc += wyw[ey[b] * KW + t2] * row;
      }
      s += acc;
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// MODE 1 (initial residual): r = H^T u.  MODE 2: out = H^T u.
template <typename T, int MODE, int KW>
__global__ void __launch_bounds__(kFitThreads) k_fit_adjoint(FitDev F, T *__restrict__ out) {
  pdl_trigger();
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = gid & 3, act = gid >> 2;
  const bool on = act < F.n_act;
  int k = 0;
  while (k + 1 < F.n_dm && act >= F.dm_off[k + 1]) ++k;
  const int loc = act - F.dm_off[k], n = F.dm_n[k];
  const int i = loc % n, jj = loc / n;
  pdl_wait();
  // idle lanes take part in the shuffles with an empty direction loop
  const T s = on ? fit_gather<T, KW>(F, k, i, jj, g) : fit_gather<T, KW>(F, 0, 0, 0, F.n_dir);
  if (on && g == 0) (MODE == 2 ? out : static_cast<T *>(F.r))[act] = s;
}

// One row of H^T H against a vector: lane sums over kSpmvBatch entries at a
// time (their columns, then their values and vector elements, are loaded
// without dependences between them), then the warp's tree.  `elem(c)` gives the
// vector element of column c.
template <typename T, typename E>
__device__ __forceinline__ T fit_row(const FitDev &F, int beg, int end, int lane, E elem) {
  T acc = T(0);
  for (int e0 = beg + lane; e0 < end; e0 += 32 * kSpmvBatch) {
    int c[kSpmvBatch];
    T w[kSpmvBatch];
#pragma unroll
    for (int b = 0; b < kSpmvBatch; ++b) {
      c[b] = -1;
      w[b] = T(0);
      if (e0 + 32 * b < end) fit_entry(F.nrm_cv, e0 + 32 * b, c[b], w[b]);
    }
#pragma unroll
    for (int b = 0; b < kSpmvBatch; ++b)
      if (c[b] >= 0) acc += w[b] * elem(c[b]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// out = H^T H x: one warp per row, the longest rows first.
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_fit_spmv(FitDev F, const T *__restrict__ x, T *__restrict__ out) {
  pdl_trigger();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= F.n_act) return;
  const int4 d = F.nrm_desc[wid];
  pdl_wait();
  const T acc = fit_row<T>(F, d.y, d.z, lane, [&](int c) { return x[c]; });
  if (lane == 0) out[d.x] = acc;
}

// The update of CG iteration it - 1 and the direction of iteration it >= 1,
// per actuator: a += alpha p (a = alpha p from a cold start when it == 1),
// r -= alpha q, p = r + beta p.  The direction of iteration 0 is the initial
// residual r itself.  alpha of it - 1 and beta of it come from the last
// k_fit_iter block.
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_fit_form(FitDev F, T *__restrict__ a, int it, int cold) {
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  if (i >= F.n_act) return;
  T *r = static_cast<T *>(F.r), *p = static_cast<T *>(F.p);
  const T al = T(F.cg[(it + 1) & 1]), beta = T(F.cg[2 + (it & 1)]);
  const T p_i = it == 1 ? r[i] : p[i], r_i = fit_fma(-al, static_cast<const T *>(F.q)[i], r[i]);
  a[i] = (cold && it == 1) ? al * p_i : fit_fma(al, p_i, a[i]);
  r[i] = r_i;
  p[i] = fit_fma(beta, p_i, r_i);
}

// q = H^T H p of CG iteration `it` over the nonempty rows, one warp per row
// with the longest rows first (actuators no sampling point reaches have empty
// rows and columns: their r, p and q stay zero).  Each block leaves a
// (p.q, r.q, q.q, r.r) record; the block that takes the last ticket sums them
// in block order and stores alpha = r.r / p.q and beta = r.r(it + 1) /
// r.r(it).  r.r(it + 1) comes from the recurrence rr - 2 alpha r.q +
// alpha^2 q.q, since the next direction needs beta before r(it + 1) exists;
// alpha takes the norm of the stored residual, so an iterate that is already
// exact (r = 0) stops moving.
template <typename T>
__global__ void __launch_bounds__(kFitIterThreads, sizeof(T) == 4 ? 2 : 1) k_fit_iter(FitDev F, int it) {
  __shared__ typename AccIO<T>::S s_v[4][kFitIterThreads / 32];
  __shared__ int s_last;
  pdl_trigger();
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool on = wid < F.n_rows;
  const int4 d = on ? F.nrm_desc[wid] : make_int4(0, 0, 0, 0);
  pdl_wait();
  const bool first = it == 0;
  const int cur = it & 1, prev = (it + 1) & 1;
  const T *p = static_cast<const T *>(first ? F.r : F.p);   // p = r in iteration 0
  T r_row = T(0), p_row = T(0);
  if (on && lane == 0) {
    r_row = static_cast<const T *>(F.r)[d.x];
    p_row = p[d.x];
  }
  const T acc = fit_row<T>(F, d.y, d.z, lane, [&](int c) { return p[c]; });
  // lane 0 of each warp holds its row's terms; sums in FP32 pairs (FP64 arithmetic is slow here)
  using IO = AccIO<T>;
  Acc<T> a0, a1, a2, a3;
  if (on && lane == 0) {
    static_cast<T *>(F.q)[d.x] = acc;
    a0.add_prod(p_row, acc);
    a1.add_prod(r_row, acc);
    a2.add_prod(acc, acc);
    a3.add_prod(r_row, r_row);
  }
  if (lane == 0) {
    s_v[0][w] = IO::pack(a0);
    s_v[1][w] = IO::pack(a1);
    s_v[2][w] = IO::pack(a2);
    s_v[3][w] = IO::pack(a3);
  }
  __syncthreads();   // the block's row stores are ordered before thread 0's release below
  const int nw = blockDim.x >> 5;
  if (w == 0) {
    Acc<T> x0, x1, x2, x3;
    if (lane < nw) {
      IO::add(x0, s_v[0][lane]);
      IO::add(x1, s_v[1][lane]);
      IO::add(x2, s_v[2][lane]);
      IO::add(x3, s_v[3][lane]);
    }
    IO::warp(x0);
    IO::warp(x1);
    IO::warp(x2);
    IO::warp(x3);
    if (lane == 0) {
      typename IO::S *rec = reinterpret_cast<typename IO::S *>(F.rec) + 4 * blockIdx.x;
      rec[0] = IO::pack(x0);
      rec[1] = IO::pack(x1);
      rec[2] = IO::pack(x2);
      rec[3] = IO::pack(x3);
      unsigned ticket;
      asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(ticket) : "l"(F.ticket) : "memory");
      s_last = ticket == gridDim.x - 1;
    }
  }
  __syncthreads();   // orders the last block's loads below after thread 0's acquire
  if (!s_last) return;
  // the last block: the blocks' records, each thread a strided subset, then
  // the warps in order; only the warps that hold some take part in the first stage
  const int nb = gridDim.x;
  Acc<T> x0, x1, x2, x3;
  if (w * 32 < nb) {
    const typename IO::S *rec = reinterpret_cast<const typename IO::S *>(F.rec);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      IO::add(x0, __ldcg(rec + 4 * b));
      IO::add(x1, __ldcg(rec + 4 * b + 1));
      IO::add(x2, __ldcg(rec + 4 * b + 2));
      IO::add(x3, __ldcg(rec + 4 * b + 3));
    }
    IO::warp(x0);
    IO::warp(x1);
    IO::warp(x2);
    IO::warp(x3);
  }
  __syncthreads();   // s_v is reused
  if (lane == 0) {
    s_v[0][w] = IO::pack(x0);
    s_v[1][w] = IO::pack(x1);
    s_v[2][w] = IO::pack(x2);
    s_v[3][w] = IO::pack(x3);
  }
  __syncthreads();
  if (w != 0) return;
  Acc<T> y0, y1, y2, y3;
  if (lane < nw) {
    IO::add(y0, s_v[0][lane]);
    IO::add(y1, s_v[1][lane]);
    IO::add(y2, s_v[2][lane]);
    IO::add(y3, s_v[3][lane]);
  }
  IO::warp(y0);
  IO::warp(y1);
  IO::warp(y2);
  IO::warp(y3);
  if (lane == 0) {
    const double s0 = y0.value(), s1 = y1.value(), s2 = y2.value();
    const double rr = y3.value();
    double alpha = 0.0;
    if (s0 == 0.0 && rr == 0.0) {
      alpha = 0.0;   // exact iterate: CG stops moving
    } else if (!(s0 > 0.0) || !isfinite(rr / s0)) {
      F.flag[0] = 1.0;
    } else {
      alpha = rr / s0;
    }
    const double rr_next = fmax(0.0, rr - 2.0 * alpha * s1 + alpha * alpha * s2);
    F.cg[cur] = alpha;
    F.cg[2 + prev] = rr != 0.0 ? rr_next / rr : 0.0;
    *F.ticket = 0u;
  }
}

// a += alpha p of the last CG iteration `it` (a = alpha p from a cold start
// when it == 0; the direction of iteration 0 is r).
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_fit_finish(FitDev F, T *__restrict__ a, int it, int cold) {
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  if (i >= F.n_act) return;
  const T al = T(F.cg[it & 1]), p_i = static_cast<const T *>(it == 0 ? F.r : F.p)[i];
  a[i] = (cold && it == 0) ? al * p_i : fit_fma(al, p_i, a[i]);
}

// r(theta_j) of the residual u_j on the sampling points: the root mean square
// after removing the mean, sqrt(mean(u^2) - mean(u)^2), one block per
// direction (the quality measure of Sec. 5.1; the Strehl ratio follows on the
// host).
template <typename T>
__global__ void __launch_bounds__(kFitRmsThreads) k_fit_rms(FitDev F, double *__restrict__ rms) {
  pdl_trigger();
  const int j = blockIdx.x, nn = F.nc * F.nc;
  const T *u = static_cast<const T *>(F.u) + static_cast<size_t>(j) * nn;
  pdl_wait();
  Acc<T> s1, s2;
  for (int c = threadIdx.x; c < nn; c += blockDim.x)
    if (F.act[c]) {
      s1.add(u[c]);
      s2.add_prod(u[c], u[c]);
    }
  const double2 v = block_sum2(s1, s2);
  if (threadIdx.x == 0) {
    const double m = v.x / F.n_points, q = v.y / F.n_points;
    rms[j] = sqrt(fmax(0.0, q - m * m));
  }
}

// sum_k a_k at corner (a, b) of a sensor whose (sensor, mirror) taps start at
// `tab`: every mirror seen like a layer at its altitude, with the cone effect
// of a laser guide star (Sec. 4.2, A_hat).
template <typename T>
__device__ __forceinline__ T sensor_mirror(const FitDev &F, const T *__restrict__ cmd, int tab, int nc, int a,
                                           int b) {
  const T *fx = static_cast<const T *>(F.sfx), *fy = static_cast<const T *>(F.sfy);
  T psi = T(0);
#pragma unroll
  for (int k = 0; k < kMaxDm; ++k) {
    if (k >= F.n_dm) break;
    const int n = F.dm_n[k], o = tab + k * nc;
    const int x0 = F.sx0[o + a], y0 = F.sy0[o + b];
    const T wx1 = fx[o + a], wy1 = fy[o + b];
    const T wx[2] = {T(1) - wx1, wx1}, wy[2] = {T(1) - wy1, wy1};
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int iy = y0 + dy;
      if (iy < 0 || iy >= n) continue;
      T row = T(0);
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int ix = x0 + dx;
        if (ix >= 0 && ix < n) row += wx[dx] * cmd[F.dm_off[k] + iy * n + ix];
      }
      psi += wy[dy] * row;
    }
  }
  return psi;
}

// out = in + scale * A_hat cmd (in = NULL: 0) in the plan's slope layout.  A
// tile item computes the mirrors on the 17 x 17 corners of its 16 x 16
// subapertures once, then their Fried slopes.  A tip/tilt-only sensor's two
// mean slopes are sum_c (Gamma^T 1)_c psi_c / S over its pupil-edge corners,
// the only corners where Gamma^T 1 is nonzero.
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_mirror_slopes(FitDev F, const T *__restrict__ cmd,
                                                              const T *__restrict__ in, T *__restrict__ out,
                                                              T scale) {
  __shared__ T s_psi[kFwdTile + 1][kFwdTile + 2];
  pdl_trigger();
  const int4 item = F.ms_items[blockIdx.x];
  const int4 sd = F.sens[item.x], so = F.sens_off[item.x];
  const int nc = sd.z, n = nc - 1;
  pdl_wait();
  if (item.w) {
    const T *et = static_cast<const T *>(F.e_t) + 2 * so.z;
    const int *ei = F.e_idx + so.z;
    Acc<T> ax, ay;
    for (int e = threadIdx.x; e < so.w; e += blockDim.x) {
      const int c = ei[e];
      const T ps = sensor_mirror(F, cmd, so.x, nc, c % nc, c / nc);
      ax.add_prod(et[2 * e], ps);
      ay.add_prod(et[2 * e + 1], ps);
    }
    const double2 v = block_sum2(ax, ay);
    if (threadIdx.x == 0) {
      out[sd.x] = (in ? in[sd.x] : T(0)) + scale * T(v.x / sd.y);
      out[sd.x + 1] = (in ? in[sd.x + 1] : T(0)) + scale * T(v.y / sd.y);
    }
    return;
  }
  const int a0 = item.y, b0 = item.z;
  for (int idx = threadIdx.x; idx < (kFwdTile + 1) * (kFwdTile + 1); idx += blockDim.x) {
    const int u = idx % (kFwdTile + 1), w = idx / (kFwdTile + 1);
    const int a = a0 + u, b = b0 + w;
    s_psi[w][u] = (a < nc && b < nc) ? sensor_mirror(F, cmd, so.x, nc, a, b) : T(0);
  }
  __syncthreads();
  const int u = threadIdx.x % kFwdTile, w = threadIdx.x / kFwdTile;
  const int a = a0 + u, b = b0 + w;
  if (a >= n || b >= n) return;
  const int j = F.sidx[so.y + b * n + a];
  if (j < 0) return;
  const T p00 = s_psi[w][u], p10 = s_psi[w][u + 1], p01 = s_psi[w + 1][u], p11 = s_psi[w + 1][u + 1];
  const T sx = T(0.5) * (p10 + p11 - p00 - p01), sy = T(0.5) * (p01 + p11 - p00 - p10);
  out[sd.x + j] = (in ? in[sd.x + j] : T(0)) + scale * sx;
  out[sd.x + sd.y + j] = (in ? in[sd.x + sd.y + j] : T(0)) + scale * sy;
}

// Algorithm 4.1, step 3 with step 2 folded in: a_t = a_{t-1} + g (R s_ol - a_{t-2}).
template <typename T>
__global__ void __launch_bounds__(kFitThreads) k_polc_update(FitDev F, const T *__restrict__ a_tm1,
                                                            const T *__restrict__ a_rec, const T *a_tm2, T *a_t,
                                                            T gain) {
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  if (i < F.n_act) a_t[i] = fit_fma(gain, a_rec[i] - a_tm2[i], a_tm1[i]);
}

// ------------------------------------------------------------------ launchers

template <typename T>
cudaError_t fit_mirror(const FitDev &F, const T *x, const T *phi, cudaStream_t s) {
  const dim3 g((F.nc * F.nc + kFitThreads - 1) / kFitThreads, F.n_dir);
  return launch_ex(k_fit_mirror<T>, g, kFitThreads, 0, 0, s, F, x, phi);
}

template <typename T>
cudaError_t fit_spmv(const FitDev &F, const T *x, T *out, cudaStream_t s) {
  return launch_ex(k_fit_spmv<T>, dim3(F.nblk_spmv), kFitThreads, 0, 0, s, F, x, out);
}

template <typename T>
cudaError_t fit_iter(const FitDev &F, int it, cudaStream_t s) {
  return launch_ex(k_fit_iter<T>, dim3(F.nblk_iter), kFitIterThreads, 0, 0, s, F, it);
}

template <typename T>
cudaError_t fit_form(const FitDev &F, T *a, int it, int cold, cudaStream_t s) {
  return launch_ex(k_fit_form<T>, dim3(F.nblk_upd), kFitThreads, 0, 0, s, F, a, it, cold);
}

template <typename T>
cudaError_t fit_finish(const FitDev &F, T *a, int it, int cold, cudaStream_t s) {
  return launch_ex(k_fit_finish<T>, dim3(F.nblk_upd), kFitThreads, 0, 0, s, F, a, it, cold);
}

template <typename T, int KW>
cudaError_t fit_adjoint_kw(int mode, const FitDev &F, T *out, cudaStream_t s) {
  const dim3 g(F.nblk_adj);
  if (mode == 1) return launch_ex(k_fit_adjoint<T, 1, KW>, g, kFitThreads, 0, 0, s, F, out);
  return launch_ex(k_fit_adjoint<T, 2, KW>, g, kFitThreads, 0, 0, s, F, out);
}

// mode 1: r = H^T u with the r.r partials; mode 2: out = H^T u.
template <typename T>
cudaError_t fit_adjoint(int mode, const FitDev &F, T *out, cudaStream_t s) {
  if (F.kw <= 2) return fit_adjoint_kw<T, 2>(mode, F, out, s);
  if (F.kw <= 4) return fit_adjoint_kw<T, 4>(mode, F, out, s);
  return fit_adjoint_kw<T, 8>(mode, F, out, s);
}

template <typename T>
cudaError_t fit_rms(const FitDev &F, double *rms, cudaStream_t s) {
  return launch_ex(k_fit_rms<T>, dim3(F.n_dir), kFitRmsThreads, 0, 0, s, F, rms);
}

template <typename T>
cudaError_t mirror_slopes(const FitDev &F, const T *cmd, const T *in, T *out, T scale, cudaStream_t s) {
  return launch_ex(k_mirror_slopes<T>, dim3(F.n_ms_items), kFitThreads, 0, 0, s, F, cmd, in, out, scale);
}

template <typename T>
cudaError_t polc_update(const FitDev &F, const T *a_tm1, const T *a_rec, const T *a_tm2, T *a_t, T gain,
                        cudaStream_t s) {
  return launch_ex(k_polc_update<T>, dim3(F.nblk_upd), kFitThreads, 0, 0, s, F, a_tm1, a_rec, a_tm2, a_t, gain);
}

}  // namespace tomo

// ---------------------------------------------------------------- the object

struct tomo_fit {
  tomo_plan *plan = nullptr;
  int device = 0, precision = 0;
  size_t esz = 4;
  tomo::FitDev F{};
  void *arena = nullptr;
  size_t arena_bytes = 0;
  void *phi = nullptr;   // layer grids of tomo_reconstruct
  long long n_active = 0, nnz = 0;
  int n_points = 0;
  cudaStream_t cap = nullptr;
  // The arguments of one graph-launched call.  kind 0: tomo_fit_solve (in =
  // layers); 1: tomo_reconstruct (in = slopes); 2: tomo_polc_step (in = slopes).
  struct Call {
    int kind;
    const void *in;
    void *x, *a;
    const void *a_tm2, *a_tm1;
    void *a_t;
    double gain;
    int iters, fit_iters, warm;
    bool operator==(const Call &o) const {
      return kind == o.kind && in == o.in && x == o.x && a == o.a && a_tm2 == o.a_tm2 && a_tm1 == o.a_tm1 &&
             a_t == o.a_t && gain == o.gain && iters == o.iters && fit_iters == o.fit_iters && warm == o.warm;
    }
  };
  struct Graph {
    Call call;
    cudaGraphExec_t exec;
    int kernels;
  };
  std::vector<Graph> graphs;
};

namespace {

using tomo::FitDev;

tomo_status fit_fail(tomo_status st, const std::string &m) { return tomo::set_error(st, m); }

tomo_status fit_cuda(cudaError_t e, const char *where) {
  return tomo::set_error(TOMO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FIT_CUDA(call, where)                          \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return fit_cuda(e_, where); \
  } while (0)

#define FIT_TRY(x)                  \
  do {                              \
    tomo_status st_ = (x);          \
    if (st_ != TOMO_OK) return st_; \
  } while (0)

// Host tables of one fit (FP64; converted to the plan's element type on upload).
struct FitTables {
  std::vector<unsigned char> act;
  std::vector<int> hx0, hy0, px0, py0, wx0, wy0;
  std::vector<double> hfx, hfy, pfx, pfy, wxw, wyw;
  std::vector<int2> lay;
  int kw = 0, n_points = 0;
  long long n_active = 0;
  // H^T H in CSR (FP64) and its rows by decreasing length
  std::vector<int> nrm_ptr, nrm_col;
  std::vector<int4> nrm_desc;
  int n_rows = 0;
  std::vector<double> nrm_val;
  // A_hat: work items, per sensor and mirror the corner taps
  std::vector<int4> ms_items, sens, sens_off;
  std::vector<int> sx0, sy0;
  std::vector<double> sfx, sfy;
};

// Left tap and fraction of coordinate g: g = i0 + f, 0 <= f < 1.
inline void tap(double g, int *i0, double *f) {
  const double fl = std::floor(g);
  *i0 = static_cast<int>(fl);
  *f = g - fl;
}

// Corner -> actuator taps of mirror k along one axis for direction offset
// `shift` (h_k theta), and each actuator's window of corners.  Returns false
// if a window is not contiguous or longer than 8.
bool mirror_axis(int nc, int n_sub, double d, const tomo_dm &m, double shift, int *i0, double *f,
                 std::vector<std::vector<std::pair<int, double>>> *win) {
  win->assign(m.n, {});
  for (int a = 0; a < nc; ++a) {
    const double g = ((a - 0.5 * n_sub) * d + shift) / m.pitch + 0.5 * (m.n - 1);
    tap(g, &i0[a], &f[a]);
    const double w[2] = {1.0 - f[a], f[a]};
    for (int t = 0; t < 2; ++t) {
      const int i = i0[a] + t;
      if (i >= 0 && i < m.n && w[t] != 0.0) (*win)[i].push_back({a, w[t]});
    }
  }
  for (const auto &v : *win) {
    if (v.size() > 8) return false;
    for (size_t t = 1; t < v.size(); ++t)
      if (v[t].first != v[t - 1].first + 1) return false;
  }
  return true;
}

tomo_status build_tables(const tomo::HostPlan &H, const tomo_fit_geometry *g, FitTables *T, std::string *err) {
  const int nc = g->n_sub + 1, ns = g->n_sub, nd = g->n_dir;
  const double d = g->d_sub;
  T->act.assign(static_cast<size_t>(nc) * nc, 0);
  for (int b = 0; b < ns; ++b)
    for (int a = 0; a < ns; ++a)
      if (g->valid[b * ns + a])
        for (int db = 0; db < 2; ++db)
          for (int da = 0; da < 2; ++da) T->act[(b + db) * nc + a + da] = 1;
  T->n_points = 0;
  for (auto v : T->act) T->n_points += v;
  if (T->n_points == 0) {
    *err = "the aperture sampling has no valid subaperture";
    return TOMO_ERR_GEOMETRY;
  }
  // mirror taps and windows
  std::vector<std::vector<std::pair<int, double>>> wins_x, wins_y;
  std::vector<std::vector<std::vector<std::pair<int, double>>>> allx, ally;   // [k*nd + j][i]
  T->hx0.resize(static_cast<size_t>(g->n_dm) * nd * nc);
  T->hy0.resize(T->hx0.size());
  T->hfx.resize(T->hx0.size());
  T->hfy.resize(T->hx0.size());
  int kw = 1;
  for (int k = 0; k < g->n_dm; ++k)
    for (int j = 0; j < nd; ++j) {
      const tomo_dm &m = g->dms[k];
      const size_t o = (static_cast<size_t>(k) * nd + j) * nc;
      if (!mirror_axis(nc, ns, d, m, m.altitude * g->theta[2 * j], &T->hx0[o], &T->hfx[o], &wins_x) ||
          !mirror_axis(nc, ns, d, m, m.altitude * g->theta[2 * j + 1], &T->hy0[o], &T->hfy[o], &wins_y)) {
        *err = "mirror " + std::to_string(k) + ": an actuator's window of sampling corners is longer than 8";
        return TOMO_ERR_UNSUPPORTED;
      }
      for (const auto &v : wins_x) kw = std::max(kw, static_cast<int>(v.size()));
      for (const auto &v : wins_y) kw = std::max(kw, static_cast<int>(v.size()));
      allx.push_back(wins_x);
      ally.push_back(wins_y);
    }
  T->kw = kw <= 2 ? 2 : (kw <= 4 ? 4 : 8);
  if (T->kw > nc) {
    *err = "the aperture sampling grid is narrower than an actuator's window";
    return TOMO_ERR_UNSUPPORTED;
  }
  // windows: start corner (shifted so the window stays inside 0..nc-1) and kw weights
  for (int k = 0; k < g->n_dm; ++k)
    for (int j = 0; j < nd; ++j)
      for (int axis = 0; axis < 2; ++axis) {
        const auto &wins = (axis == 0 ? allx : ally)[k * nd + j];
        auto &w0 = axis == 0 ? T->wx0 : T->wy0;
        auto &ww = axis == 0 ? T->wxw : T->wyw;
        for (const auto &v : wins) {
          int s = v.empty() ? 0 : v.front().first;
          const int s_eff = std::min(s, nc - T->kw);
          w0.push_back(s_eff);
          std::vector<double> w(T->kw, 0.0);
          for (size_t t = 0; t < v.size(); ++t) w[s - s_eff + t] = v[t].second;
          ww.insert(ww.end(), w.begin(), w.end());
        }
      }
  // actuators reached by a sampling point: nonzero diagonal of H^T H
  T->n_active = 0;
  for (int k = 0; k < g->n_dm; ++k) {
    const int n = g->dms[k].n;
    std::vector<unsigned char> hit(static_cast<size_t>(n) * n, 0);
    for (int j = 0; j < nd; ++j) {
      const size_t o = (static_cast<size_t>(k) * nd + j) * nc;
      for (int b = 0; b < nc; ++b)
        for (int a = 0; a < nc; ++a) {
          if (!T->act[b * nc + a]) continue;
          const double wx[2] = {1.0 - T->hfx[o + a], T->hfx[o + a]};
          const double wy[2] = {1.0 - T->hfy[o + b], T->hfy[o + b]};
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              const int ix = T->hx0[o + a] + dx, iy = T->hy0[o + b] + dy;
              if (ix >= 0 && ix < n && iy >= 0 && iy < n && wx[dx] * wy[dy] > 0.0) hit[iy * n + ix] = 1;
            }
        }
    }
    for (auto v : hit) T->n_active += v;
  }
  // H^T H: H as rows (direction, active corner) of (actuator, weight), from the
  // same taps as the mirror kernel; its columns; then each row of H^T H by
  // Gustavson's method (a sparse accumulator over the H rows touching it)
  {
    std::vector<int> dm_off(g->n_dm + 1, 0);
    for (int k = 0; k < g->n_dm; ++k) dm_off[k + 1] = dm_off[k] + g->dms[k].n * g->dms[k].n;
    const int n_act = dm_off[g->n_dm];
    std::vector<int> h_ptr{0}, h_col;
    std::vector<double> h_w;
    for (int j = 0; j < nd; ++j)
      for (int c = 0; c < nc * nc; ++c) {
        if (!T->act[c]) continue;
        const int a = c % nc, b = c / nc;
        for (int k = 0; k < g->n_dm; ++k) {
          const int n = g->dms[k].n;
          const size_t o = (static_cast<size_t>(k) * nd + j) * nc;
          const double wx[2] = {1.0 - T->hfx[o + a], T->hfx[o + a]};
          const double wy[2] = {1.0 - T->hfy[o + b], T->hfy[o + b]};
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              const int ix = T->hx0[o + a] + dx, iy = T->hy0[o + b] + dy;
              const double w = wx[dx] * wy[dy];
              if (ix < 0 || ix >= n || iy < 0 || iy >= n || w == 0.0) continue;
              h_col.push_back(dm_off[k] + iy * n + ix);
              h_w.push_back(w);
            }
        }
        h_ptr.push_back(static_cast<int>(h_col.size()));
      }
    const int n_rows = static_cast<int>(h_ptr.size()) - 1;
    std::vector<int> t_ptr(n_act + 1, 0), t_row(h_col.size());
    std::vector<double> t_w(h_col.size());
    for (int col : h_col) ++t_ptr[col + 1];
    for (int i = 0; i < n_act; ++i) t_ptr[i + 1] += t_ptr[i];
    std::vector<int> fill(t_ptr.begin(), t_ptr.end() - 1);
    for (int r = 0; r < n_rows; ++r)
      for (int e = h_ptr[r]; e < h_ptr[r + 1]; ++e) {
        const int at = fill[h_col[e]]++;
        t_row[at] = r;
        t_w[at] = h_w[e];
      }
    std::vector<double> acc(n_act, 0.0);
    std::vector<int> mark(n_act, -1), touched;
    T->nrm_ptr.assign(1, 0);
    for (int i = 0; i < n_act; ++i) {
      touched.clear();
      for (int e = t_ptr[i]; e < t_ptr[i + 1]; ++e) {
        const int r = t_row[e];
        const double wa = t_w[e];
        for (int f = h_ptr[r]; f < h_ptr[r + 1]; ++f) {
          const int col = h_col[f];
          if (mark[col] != i) {
            mark[col] = i;
            acc[col] = 0.0;
            touched.push_back(col);
          }
          acc[col] += wa * h_w[f];
        }
      }
      std::sort(touched.begin(), touched.end());
      for (int col : touched) {
        T->nrm_col.push_back(col);
        T->nrm_val.push_back(acc[col]);
      }
      if (T->nrm_col.size() > static_cast<size_t>(INT32_MAX)) {
        *err = "the fitting normal matrix has too many entries";
        return TOMO_ERR_UNSUPPORTED;
      }
      T->nrm_ptr.push_back(static_cast<int>(T->nrm_col.size()));
    }
    // rows by decreasing length, so that no late wave holds only long rows;
    // the empty rows (actuators no sampling point reaches) come last
    std::vector<int> order(n_act);
    for (int i = 0; i < n_act; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return T->nrm_ptr[a + 1] - T->nrm_ptr[a] > T->nrm_ptr[b + 1] - T->nrm_ptr[b];
    });
    T->nrm_desc.resize(n_act);
    T->n_rows = 0;
    for (int w = 0; w < n_act; ++w) {
      const int i = order[w];
      T->nrm_desc[w] = make_int4(i, T->nrm_ptr[i], T->nrm_ptr[i + 1], 0);
      if (T->nrm_ptr[i + 1] > T->nrm_ptr[i]) ++T->n_rows;
    }
  }
  // the mirrors on the plan's sensors: corner (a, b) of sensor m sees mirror k at
  // ((1 - h_k/H_m) r + theta_m h_k), cone factor 1 for a natural star
  for (int m = 0; m < H.n_wfs; ++m) {
    const tomo::WfsDev &W = H.wfs[m];
    const int n = W.n, ncm = W.nc;
    const double h_gs = H.wfs_height[m];
    const bool tt = W.kind == tomo::kTTOnly;
    T->sens.push_back({W.slope_off, W.S, ncm, tt ? 1 : 0});
    T->sens_off.push_back({static_cast<int>(T->sx0.size()), W.sub_off, W.edge_off, W.n_edge});
    if (tt) {
      T->ms_items.push_back({m, 0, 0, 1});
    } else {
      for (int b0 = 0; b0 < n; b0 += tomo::kFwdTile)
        for (int a0 = 0; a0 < n; a0 += tomo::kFwdTile) {
          bool any = false;
          for (int b = b0; b < std::min(n, b0 + tomo::kFwdTile) && !any; ++b)
            for (int a = a0; a < std::min(n, a0 + tomo::kFwdTile) && !any; ++a)
              any = H.sub_idx[W.sub_off + b * n + a] >= 0;
          if (any) T->ms_items.push_back({m, a0, b0, 0});
        }
    }
    for (int k = 0; k < g->n_dm; ++k) {
      const tomo_dm &dm = g->dms[k];
      const double cone = std::isfinite(h_gs) ? 1.0 - dm.altitude / h_gs : 1.0;
      for (int axis = 0; axis < 2; ++axis) {
        const double th = axis == 0 ? H.wfs_theta[m].x : H.wfs_theta[m].y;
        for (int a = 0; a < ncm; ++a) {
          const double r = (a - 0.5 * n) * W.d_sub;
          int i0;
          double f;
          tap((cone * r + th * dm.altitude) / dm.pitch + 0.5 * (dm.n - 1), &i0, &f);
          (axis == 0 ? T->sx0 : T->sy0).push_back(i0);
          (axis == 0 ? T->sfx : T->sfy).push_back(f);
        }
      }
    }
  }
  // layer taps (natural guide star: no cone)
  const int L = H.n_layers;
  T->px0.resize(static_cast<size_t>(L) * nd * nc);
  T->py0.resize(T->px0.size());
  T->pfx.resize(T->px0.size());
  T->pfy.resize(T->px0.size());
  for (int l = 0; l < L; ++l) {
    const int N = H.layers[l].N;
    T->lay.push_back({N, H.layers[l].off});
    for (int j = 0; j < nd; ++j)
      for (int a = 0; a < nc; ++a) {
        const size_t o = (static_cast<size_t>(l) * nd + j) * nc + a;
        const double r = (a - 0.5 * ns) * d;
        for (int axis = 0; axis < 2; ++axis) {
          const double gc = (r + g->theta[2 * j + axis] * H.layer_alt[l]) / H.layer_dx[l] + 0.5 * N;
          int i0;
          double f;
          tap(gc, &i0, &f);
          i0 = ((i0 % N) + N) % N;
          (axis == 0 ? T->px0 : T->py0)[o] = i0;
          (axis == 0 ? T->pfx : T->pfy)[o] = f;
        }
      }
  }
  return TOMO_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// The launches of one fitting solve on stream s; they are added to the launch
// count.
template <typename T>
tomo_status enqueue_fit(tomo_fit *f, const void *layers, void *a, int iters, int warm, cudaStream_t s,
                        int *nk) {
  const FitDev &F = f->F;
  T *av = static_cast<T *>(a);
  int k = 0;
  if (!warm && iters == 0) FIT_CUDA(cudaMemsetAsync(a, 0, F.n_act * sizeof(T), s), "zero start");
  FIT_CUDA(tomo::fit_mirror<T>(F, warm ? av : nullptr, static_cast<const T *>(layers), s), "fit residual");
  FIT_CUDA(tomo::fit_adjoint<T>(1, F, nullptr, s), "fit residual gather");
  k += 2;
  for (int it = 0; it < iters; ++it) {
    if (it > 0) {
      FIT_CUDA(tomo::fit_form<T>(F, av, it, warm ? 0 : 1, s), "fit CG direction");
      ++k;
    }
    FIT_CUDA(tomo::fit_iter<T>(F, it, s), "fit normal operator");
    ++k;
  }
  if (iters > 0) {
    FIT_CUDA(tomo::fit_finish<T>(F, av, iters - 1, warm ? 0 : 1, s), "fit commands");
    ++k;
  }
  tomo::count_launches(k);
  *nk = k;
  return TOMO_OK;
}

tomo_status enqueue_fit_any(tomo_fit *f, const void *layers, void *a, int iters, int warm, cudaStream_t s,
                            int *nk) {
  return f->precision == 0 ? enqueue_fit<float>(f, layers, a, iters, warm, s, nk)
                           : enqueue_fit<double>(f, layers, a, iters, warm, s, nk);
}

// The launches of one call on stream s (added to the launch count).
tomo_status enqueue_call(tomo_fit *f, const tomo_fit::Call &c, cudaStream_t s, int *nk) {
  if (c.kind == 0) return enqueue_fit_any(f, c.in, c.a, c.fit_iters, c.warm, s, nk);
  const void *slopes = c.in;
  int k0 = 0;
  if (c.kind == 2) {
    // Algorithm 4.1, step 1: s_ol = s + A_hat a_{t-2}
    if (f->precision == 0)
      FIT_CUDA(tomo::mirror_slopes<float>(f->F, static_cast<const float *>(c.a_tm2), static_cast<const float *>(c.in),
                                          static_cast<float *>(f->F.s_ol), 1.f, s), "pseudo-open-loop slopes");
    else
      FIT_CUDA(tomo::mirror_slopes<double>(f->F, static_cast<const double *>(c.a_tm2),
                                           static_cast<const double *>(c.in), static_cast<double *>(f->F.s_ol), 1.0,
                                           s), "pseudo-open-loop slopes");
    tomo::count_launches(1);
    slopes = f->F.s_ol;
    k0 = 1;
  }
  int k1 = 0, k2 = 0;
  FIT_TRY(tomo::enqueue_plan_solve(f->plan, slopes, c.x, c.iters, c.warm, s, &k1));
  // phi = W^-1 c into the fit's layer buffer
  tomo_plan *p = f->plan;
  tomo::IoArgs io{};
  io.in0[0] = c.x;
  io.out0[0] = f->phi;
  const tomo::LaunchSet &L = p->ls;
  FIT_CUDA(tomo::synthesis_of(L, 0, 0, io, s), "synthesis of the reconstructed layers");
  tomo::count_launches(tomo::synthesis_launches(L));
  FIT_TRY(enqueue_fit_any(f, f->phi, c.a, c.fit_iters, c.warm, s, &k2));
  int k3 = 0;
  if (c.kind == 2) {
    // steps 2 and 3: a_t = a_{t-1} + g (R s_ol - a_{t-2})
    if (f->precision == 0)
      FIT_CUDA(tomo::polc_update<float>(f->F, static_cast<const float *>(c.a_tm1), static_cast<const float *>(c.a),
                                        static_cast<const float *>(c.a_tm2), static_cast<float *>(c.a_t),
                                        static_cast<float>(c.gain), s), "control update");
    else
      FIT_CUDA(tomo::polc_update<double>(f->F, static_cast<const double *>(c.a_tm1), static_cast<const double *>(c.a),
                                         static_cast<const double *>(c.a_tm2), static_cast<double *>(c.a_t), c.gain,
                                         s), "control update");
    tomo::count_launches(1);
    k3 = 1;
  }
  *nk = k0 + k1 + 1 + k2 + k3;
  return TOMO_OK;
}

// Replays the call from a graph cached per argument set (captured on first use).
tomo_status run_graph(tomo_fit *f, const tomo_fit::Call &c, cudaStream_t s) {
  tomo_fit::Graph *ge = nullptr;
  for (auto &g : f->graphs)
    if (g.call == c) ge = &g;
  if (!ge) {
    if (f->graphs.size() >= 16) {
      cudaGraphExecDestroy(f->graphs.front().exec);
      f->graphs.erase(f->graphs.begin());
    }
    cudaGraph_t graph = nullptr;
    FIT_CUDA(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int nk = 0;
    const long long before = tomo_launch_count();
    tomo_status st = enqueue_call(f, c, f->cap, &nk);
    tomo::count_launches(before - tomo_launch_count());   // a capture launches nothing
    cudaError_t ce = cudaStreamEndCapture(f->cap, &graph);
    if (st != TOMO_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return fit_cuda(ce, "end capture");
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fit_cuda(ce, "graph instantiate");
    f->graphs.push_back({c, exec, nk});
    ge = &f->graphs.back();
  }
  FIT_CUDA(cudaGraphLaunch(ge->exec, s), "graph launch");
  tomo::count_launches(ge->kernels);
  return TOMO_OK;
}

// Runs a call from its graph, or launch by launch when the plan's launch mode
// says so.
tomo_status run_call(tomo_fit *f, const tomo_fit::Call &c, cudaStream_t s) {
  static const char *const kNames[] = {"tomo_fit_solve", "tomo_reconstruct", "tomo_polc_step"};
  tomo::NvtxRange nvtx(kNames[c.kind]);
  if (f->plan->use_graphs) return run_graph(f, c, s);
  int nk = 0;
  return enqueue_call(f, c, s, &nk);
}

template <typename T>
void put(std::vector<unsigned char> &img, size_t off, const std::vector<double> &v) {
  T *d = reinterpret_cast<T *>(img.data() + off);
  for (size_t i = 0; i < v.size(); ++i) d[i] = static_cast<T>(v[i]);
}

}  // namespace

extern "C" {

tomo_status tomo_fit_create(tomo_plan *p, const tomo_fit_geometry *g, tomo_fit **out) {
  if (!p || !g || !out) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (g->n_dm < 1 || g->n_dm > tomo::kMaxDm || !g->dms)
    return fit_fail(TOMO_ERR_ARG, "n_dm must be in 1..4 with a mirror array");
  if (g->n_dir < 1 || g->n_dir > tomo::kMaxFitDirs || !g->theta)
    return fit_fail(TOMO_ERR_ARG, "n_dir must be in 1..256 with a direction array");
  if (g->n_sub < 1 || g->n_sub > 1024 || !(g->d_sub > 0.0) || !std::isfinite(g->d_sub) || !g->valid)
    return fit_fail(TOMO_ERR_ARG, "n_sub must be in 1..1024, d_sub > 0 and valid not NULL");
  long long n_act = 0;
  for (int k = 0; k < g->n_dm; ++k) {
    const tomo_dm &m = g->dms[k];
    if (m.n < 2 || m.n > 4096 || !(m.pitch > 0.0) || !(m.pitch <= 4.0 * g->d_sub) || !(m.altitude >= 0.0) ||
        !std::isfinite(m.altitude))
      return fit_fail(TOMO_ERR_ARG, "mirror " + std::to_string(k) +
                                        ": n must be in 2..4096, 0 < pitch <= 4 d_sub and altitude >= 0");
    n_act += static_cast<long long>(m.n) * m.n;
  }
  for (int j = 0; j < 2 * g->n_dir; ++j)
    if (!std::isfinite(g->theta[j])) return fit_fail(TOMO_ERR_ARG, "directions must be finite");
  if (n_act > (1LL << 28)) return fit_fail(TOMO_ERR_ARG, "too many actuators");
  const tomo::HostPlan &H = p->hp;
  FitTables T;
  std::string err;
  FIT_TRY(([&] {
    tomo_status st = build_tables(H, g, &T, &err);
    return st == TOMO_OK ? st : fit_fail(st, err);
  }()));
  tomo_fit *f = new tomo_fit();
  f->plan = p;
  f->device = p->device;
  f->precision = H.precision;
  f->esz = H.precision ? 8 : 4;
  f->n_active = T.n_active;
  f->nnz = static_cast<long long>(T.nrm_col.size());
  f->n_points = T.n_points;
  FitDev &F = f->F;
  const int nc = g->n_sub + 1, nd = g->n_dir;
  F.n_dir = nd;
  F.n_dm = g->n_dm;
  F.nc = nc;
  F.n_layers = H.n_layers;
  F.n_act = static_cast<int>(n_act);
  F.kw = T.kw;
  F.n_points = T.n_points;
  F.n_ms_items = static_cast<int>(T.ms_items.size());
  F.nblk_adj = static_cast<int>((4 * n_act + tomo::kFitThreads - 1) / tomo::kFitThreads);
  F.nblk_upd = static_cast<int>((n_act + tomo::kFitThreads - 1) / tomo::kFitThreads);
  F.nblk_spmv = static_cast<int>((32 * n_act + tomo::kFitThreads - 1) / tomo::kFitThreads);
  F.n_rows = T.n_rows;
  F.nblk_iter = std::max(1, (32 * T.n_rows + tomo::kFitIterThreads - 1) / tomo::kFitIterThreads);
  int off = 0, woff = 0;
  for (int k = 0; k < g->n_dm; ++k) {
    F.dm_n[k] = g->dms[k].n;
    F.dm_off[k] = off;
    F.w_off[k] = woff;
    off += g->dms[k].n * g->dms[k].n;
    woff += nd * g->dms[k].n;
  }
  for (int k = g->n_dm; k < tomo::kMaxDm; ++k) F.dm_off[k] = off;
  // one arena: tables, then the workspace
  const size_t es = f->esz;
  struct Item { size_t *off; size_t bytes; };
  size_t o_act, o_lay, o_hx0, o_hy0, o_hfx, o_hfy, o_px0, o_py0, o_pfx, o_pfy, o_wx0, o_wy0, o_wxw, o_wyw,
      o_msi, o_sens, o_soff, o_sidx, o_eidx, o_et, o_sx0, o_sy0, o_sfx, o_sfy, o_ncv, o_nord, o_u, o_r,
      o_p, o_q, o_phi, o_sol, o_rec, o_cg, o_ticket, o_flag;
  const Item items[] = {
      {&o_act, T.act.size()},
      {&o_lay, T.lay.size() * sizeof(int2)},
      {&o_hx0, T.hx0.size() * sizeof(int)},
      {&o_hy0, T.hy0.size() * sizeof(int)},
      {&o_hfx, T.hfx.size() * es},
      {&o_hfy, T.hfy.size() * es},
      {&o_px0, T.px0.size() * sizeof(int)},
      {&o_py0, T.py0.size() * sizeof(int)},
      {&o_pfx, T.pfx.size() * es},
      {&o_pfy, T.pfy.size() * es},
      {&o_wx0, T.wx0.size() * sizeof(int)},
      {&o_wy0, T.wy0.size() * sizeof(int)},
      {&o_wxw, T.wxw.size() * es},
      {&o_wyw, T.wyw.size() * es},
      {&o_msi, T.ms_items.size() * sizeof(int4)},
      {&o_sens, T.sens.size() * sizeof(int4)},
      {&o_soff, T.sens_off.size() * sizeof(int4)},
      {&o_sidx, H.sub_idx.size() * sizeof(int)},
      {&o_eidx, H.edge_idx.size() * sizeof(int)},
      {&o_et, H.edge_t.size() * es},
      {&o_sx0, T.sx0.size() * sizeof(int)},
      {&o_sy0, T.sy0.size() * sizeof(int)},
      {&o_sfx, T.sfx.size() * es},
      {&o_sfy, T.sfy.size() * es},
      {&o_ncv, T.nrm_col.size() * 2 * es},
      {&o_nord, T.nrm_desc.size() * sizeof(int4)},
      {&o_u, static_cast<size_t>(nd) * nc * nc * es},
      {&o_r, n_act * es},
      {&o_p, n_act * es},
      {&o_q, n_act * es},
      {&o_phi, static_cast<size_t>(H.n) * es},
      {&o_sol, static_cast<size_t>(H.n_slopes) * es},
      {&o_rec, static_cast<size_t>(F.nblk_iter) * 4 * sizeof(double)},
      {&o_cg, 4 * sizeof(double)},
      {&o_ticket, sizeof(unsigned)},
      {&o_flag, sizeof(double)},
  };
  size_t total = 0;
  for (const auto &it : items) {
    *it.off = total;
    total = align256(total + it.bytes);
  }
  const size_t tables_end = o_u;
  std::vector<unsigned char> img(tables_end, 0);
  std::memcpy(img.data() + o_act, T.act.data(), T.act.size());
  std::memcpy(img.data() + o_lay, T.lay.data(), T.lay.size() * sizeof(int2));
  std::memcpy(img.data() + o_hx0, T.hx0.data(), T.hx0.size() * sizeof(int));
  std::memcpy(img.data() + o_hy0, T.hy0.data(), T.hy0.size() * sizeof(int));
  std::memcpy(img.data() + o_px0, T.px0.data(), T.px0.size() * sizeof(int));
  std::memcpy(img.data() + o_py0, T.py0.data(), T.py0.size() * sizeof(int));
  std::memcpy(img.data() + o_wx0, T.wx0.data(), T.wx0.size() * sizeof(int));
  std::memcpy(img.data() + o_wy0, T.wy0.data(), T.wy0.size() * sizeof(int));
  // (column, value) entries of H^T H
  for (size_t e = 0; e < T.nrm_col.size(); ++e) {
    unsigned char *at = img.data() + o_ncv + e * 2 * es;
    std::memcpy(at, &T.nrm_col[e], sizeof(int));
    if (f->precision) {
      const double v = T.nrm_val[e];
      std::memcpy(at + 8, &v, sizeof(double));
    } else {
      const float v = static_cast<float>(T.nrm_val[e]);
      std::memcpy(at + 4, &v, sizeof(float));
    }
  }
  std::memcpy(img.data() + o_nord, T.nrm_desc.data(), T.nrm_desc.size() * sizeof(int4));
  std::memcpy(img.data() + o_msi, T.ms_items.data(), T.ms_items.size() * sizeof(int4));
  std::memcpy(img.data() + o_sens, T.sens.data(), T.sens.size() * sizeof(int4));
  std::memcpy(img.data() + o_soff, T.sens_off.data(), T.sens_off.size() * sizeof(int4));
  std::memcpy(img.data() + o_sidx, H.sub_idx.data(), H.sub_idx.size() * sizeof(int));
  std::memcpy(img.data() + o_eidx, H.edge_idx.data(), H.edge_idx.size() * sizeof(int));
  std::memcpy(img.data() + o_sx0, T.sx0.data(), T.sx0.size() * sizeof(int));
  std::memcpy(img.data() + o_sy0, T.sy0.data(), T.sy0.size() * sizeof(int));
  const std::pair<size_t, const std::vector<double> *> reals[] = {
      {o_hfx, &T.hfx}, {o_hfy, &T.hfy}, {o_pfx, &T.pfx}, {o_pfy, &T.pfy}, {o_wxw, &T.wxw}, {o_wyw, &T.wyw},
      {o_sfx, &T.sfx}, {o_sfy, &T.sfy}, {o_et, &H.edge_t}};
  for (const auto &rv : reals) {
    if (f->precision) put<double>(img, rv.first, *rv.second);
    else put<float>(img, rv.first, *rv.second);
  }
  tomo::DeviceGuard dg(f->device);
  cudaError_t e = cudaMalloc(&f->arena, total);
  if (e != cudaSuccess) {
    delete f;
    return fit_fail(TOMO_ERR_NOMEM, std::string("device allocation of the fit: ") + cudaGetErrorString(e));
  }
  f->arena_bytes = total;
  unsigned char *base = static_cast<unsigned char *>(f->arena);
  e = cudaMemcpy(base, img.data(), tables_end, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(base + tables_end, 0, total - tables_end);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    tomo_fit_destroy(f);
    return fit_cuda(e, "uploading the fit tables");
  }
  F.act = base + o_act;
  F.lay = reinterpret_cast<const int2 *>(base + o_lay);
  F.hx0 = reinterpret_cast<const int *>(base + o_hx0);
  F.hy0 = reinterpret_cast<const int *>(base + o_hy0);
  F.hfx = base + o_hfx;
  F.hfy = base + o_hfy;
  F.px0 = reinterpret_cast<const int *>(base + o_px0);
  F.py0 = reinterpret_cast<const int *>(base + o_py0);
  F.pfx = base + o_pfx;
  F.pfy = base + o_pfy;
  F.wx0 = reinterpret_cast<const int *>(base + o_wx0);
  F.wy0 = reinterpret_cast<const int *>(base + o_wy0);
  F.wxw = base + o_wxw;
  F.wyw = base + o_wyw;
  F.ms_items = reinterpret_cast<const int4 *>(base + o_msi);
  F.sens = reinterpret_cast<const int4 *>(base + o_sens);
  F.sens_off = reinterpret_cast<const int4 *>(base + o_soff);
  F.sidx = reinterpret_cast<const int *>(base + o_sidx);
  F.e_idx = reinterpret_cast<const int *>(base + o_eidx);
  F.e_t = base + o_et;
  F.sx0 = reinterpret_cast<const int *>(base + o_sx0);
  F.sy0 = reinterpret_cast<const int *>(base + o_sy0);
  F.sfx = base + o_sfx;
  F.sfy = base + o_sfy;
  F.s_ol = base + o_sol;
  F.u = base + o_u;
  F.r = base + o_r;
  F.p = base + o_p;
  F.q = base + o_q;
  F.nrm_cv = base + o_ncv;
  F.nrm_desc = reinterpret_cast<const int4 *>(base + o_nord);
  f->phi = base + o_phi;
  F.rec = reinterpret_cast<double *>(base + o_rec);
  F.cg = reinterpret_cast<double *>(base + o_cg);
  F.ticket = reinterpret_cast<unsigned *>(base + o_ticket);
  F.flag = reinterpret_cast<double *>(base + o_flag);
  *out = f;
  return TOMO_OK;
}

tomo_status tomo_fit_get_info(const tomo_fit *f, tomo_fit_info *out) {
  if (!f || !out) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  out->n_act = f->F.n_act;
  out->n_active = f->n_active;
  out->n_points = f->n_points;
  out->n_dir = f->F.n_dir;
  out->n_dm = f->F.n_dm;
  // 2 + 2 iters launches: the first iteration has no k_fit_form, the last one is
  // followed by k_fit_finish
  out->kernels_per_iteration = 2;
  out->kernels_per_solve_base = 2;
  out->device_bytes = static_cast<long long>(f->arena_bytes);
  out->normal_nonzeros = f->nnz;
  // k_fit_form: a, p, q, r read, a, r, p written; k_fit_iter: every entry and its
  // column, a row descriptor per nonempty row, p and r read, q written
  const long long na = f->F.n_act, es = static_cast<long long>(f->esz);
  out->bytes_per_iteration = 7 * na * es + f->nnz * (es + 4) + 16LL * f->F.n_rows + 3 * na * es;
  return TOMO_OK;
}

tomo_status tomo_fit_apply_normal(tomo_fit *f, const void *d_a, void *d_out, void *cuda_stream) {
  if (!f || !d_a || !d_out) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  tomo::DeviceGuard dg(f->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (f->precision == 0)
    FIT_CUDA(tomo::fit_spmv<float>(f->F, static_cast<const float *>(d_a), static_cast<float *>(d_out), s),
             "fit normal operator");
  else
    FIT_CUDA(tomo::fit_spmv<double>(f->F, static_cast<const double *>(d_a), static_cast<double *>(d_out), s),
             "fit normal operator");
  tomo::count_launches(1);
  return TOMO_OK;
}

tomo_status tomo_fit_rhs(tomo_fit *f, const void *d_layers, void *d_out, void *cuda_stream) {
  if (!f || !d_layers || !d_out) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  tomo::DeviceGuard dg(f->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (f->precision == 0) {
    FIT_CUDA(tomo::fit_mirror<float>(f->F, nullptr, static_cast<const float *>(d_layers), s), "fit project");
    FIT_CUDA(tomo::fit_adjoint<float>(2, f->F, static_cast<float *>(d_out), s), "fit gather");
  } else {
    FIT_CUDA(tomo::fit_mirror<double>(f->F, nullptr, static_cast<const double *>(d_layers), s), "fit project");
    FIT_CUDA(tomo::fit_adjoint<double>(2, f->F, static_cast<double *>(d_out), s), "fit gather");
  }
  tomo::count_launches(2);
  return TOMO_OK;
}

tomo_status tomo_fit_residual_rms(tomo_fit *f, const void *d_layers, const void *d_a, double *d_rms,
                                  void *cuda_stream) {
  if (!f || !d_layers || !d_rms) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  tomo::DeviceGuard dg(f->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (f->precision == 0) {
    FIT_CUDA(tomo::fit_mirror<float>(f->F, static_cast<const float *>(d_a), static_cast<const float *>(d_layers), s),
             "fit residual");
    FIT_CUDA(tomo::fit_rms<float>(f->F, d_rms, s), "fit residual rms");
  } else {
    FIT_CUDA(tomo::fit_mirror<double>(f->F, static_cast<const double *>(d_a), static_cast<const double *>(d_layers),
                                      s), "fit residual");
    FIT_CUDA(tomo::fit_rms<double>(f->F, d_rms, s), "fit residual rms");
  }
  tomo::count_launches(2);
  return TOMO_OK;
}

tomo_status tomo_fit_solve(tomo_fit *f, const void *d_layers, void *d_a, int iters, int warm, void *cuda_stream) {
  if (!f || !d_layers || !d_a) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  if (iters < 0 || iters > 100000) return fit_fail(TOMO_ERR_ARG, "iters out of range");
  tomo::DeviceGuard dg(f->device);
  tomo_fit::Call c{0, d_layers, nullptr, d_a, nullptr, nullptr, nullptr, 0.0, 0, iters, warm ? 1 : 0};
  return run_call(f, c, static_cast<cudaStream_t>(cuda_stream));
}

tomo_status tomo_reconstruct(tomo_fit *f, const void *d_slopes, void *d_coeffs, void *d_a, int iters,
                             int fit_iters, int warm, void *cuda_stream) {
  if (!f || !d_slopes || !d_coeffs || !d_a) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  if (iters < 0 || iters > 100000 || fit_iters < 0 || fit_iters > 100000)
    return fit_fail(TOMO_ERR_ARG, "iters out of range");
  tomo::DeviceGuard dg(f->device);
  tomo_fit::Call c{1, d_slopes, d_coeffs, d_a, nullptr, nullptr, nullptr, 0.0, iters, fit_iters, warm ? 1 : 0};
  return run_call(f, c, static_cast<cudaStream_t>(cuda_stream));
}

tomo_status tomo_mirror_slopes(tomo_fit *f, const void *d_a, const void *d_in, void *d_out, double scale,
                               void *cuda_stream) {
  if (!f || !d_a || !d_out) return fit_fail(TOMO_ERR_ARG, "NULL argument");
  if (!std::isfinite(scale)) return fit_fail(TOMO_ERR_ARG, "scale must be finite");
  tomo::DeviceGuard dg(f->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (f->precision == 0)
    FIT_CUDA(tomo::mirror_slopes<float>(f->F, static_cast<const float *>(d_a), static_cast<const float *>(d_in),
                                        static_cast<float *>(d_out), static_cast<float>(scale), s), "mirror slopes");
  else
    FIT_CUDA(tomo::mirror_slopes<double>(f->F, static_cast<const double *>(d_a), static_cast<const double *>(d_in),
                                         static_cast<double *>(d_out), scale, s), "mirror slopes");
  tomo::count_launches(1);
  return TOMO_OK;
}

tomo_status tomo_polc_step(tomo_fit *f, const void *d_slopes, void *d_coeffs, void *d_a_rec, const void *d_a_tm2,
                           const void *d_a_tm1, void *d_a_t, double gain, int iters, int fit_iters, int warm,
                           void *cuda_stream) {
  if (!f || !d_slopes || !d_coeffs || !d_a_rec || !d_a_tm2 || !d_a_tm1 || !d_a_t)
    return fit_fail(TOMO_ERR_ARG, "NULL argument");
  if (iters < 0 || iters > 100000 || fit_iters < 0 || fit_iters > 100000)
    return fit_fail(TOMO_ERR_ARG, "iters out of range");
  if (!std::isfinite(gain)) return fit_fail(TOMO_ERR_ARG, "gain must be finite");
  if (d_a_t == d_a_tm1 || d_a_rec == d_a_tm2 || d_a_rec == d_a_tm1 || d_a_rec == d_a_t)
    return fit_fail(TOMO_ERR_ARG, "a_t may share storage with a_tm2 only; a_rec with none");
  tomo::DeviceGuard dg(f->device);
  tomo_fit::Call c{2, d_slopes, d_coeffs, d_a_rec, d_a_tm2, d_a_tm1, d_a_t, gain, iters, fit_iters, warm ? 1 : 0};
  return run_call(f, c, static_cast<cudaStream_t>(cuda_stream));
}

void tomo_fit_destroy(tomo_fit *f) {
  if (!f) return;
  tomo::DeviceGuard dg(f->device);
  for (auto &g : f->graphs) cudaGraphExecDestroy(g.exec);
  if (f->cap) cudaStreamDestroy(f->cap);
  if (f->arena) cudaFree(f->arena);
  delete f;
}

}  // extern "C"
