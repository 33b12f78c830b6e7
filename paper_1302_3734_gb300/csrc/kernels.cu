// CUDA kernels of the wavelet-domain MAP tomography solve (sm_103a).
//
// Per PCG iteration (Sec. 5.1 of the paper) four launches cover the operator
// (W P^T Gamma^T C^-1 Gamma P W^-1 + alpha D) p and the (P)CG vector updates:
//
//   k_synthesis  p <- J^-1 r + beta p (fused), phi = W^-1 p      [cluster per layer]
//   k_forward    psi = P phi on sensor corners, Fried slopes,
//                C^-1 weighting with tip/tilt removal, Gamma^T   [tile per sensor]
//   k_analysis   g = sum_m P_m^T v_m (gather), q = W g + alpha D p,
//                p.q -> alpha                                    [cluster per layer]
//   k_update     x += alpha p, r -= alpha q, r.J^-1 r -> beta     [chunk per CTA]
//
// The periodic 2-D DWT of one layer runs inside one thread-block cluster: CTA c
// owns N/C consecutive rows; the row pass is local and the column pass reads
// the Lf-2 halo rows of its neighbours through distributed shared memory.  The
// coarse levels (block side <= C) are finished by CTA 0 alone.  Reductions are
// FP64 (warp shuffle -> block -> per-CTA partial -> last CTA in a fixed order),
// so results do not depend on scheduling.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "common.h"
#include "launch.h"

namespace cg = cooperative_groups;

namespace tomo {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of (a, b) over the block; the result is returned to every thread.
__device__ double2 block_sum2(double a, double b) {
  __shared__ double s_red[2][kThreads / 32];
  __shared__ double2 s_out;
  a = warp_sum(a);
  b = warp_sum(b);
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

// Copy one instance descriptor into shared memory.
__device__ __forceinline__ void load_inst(InstDev *dst, const InstDev *src) {
  const int nw = sizeof(InstDev) / sizeof(int);
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) d[i] = s[i];
  __syncthreads();
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
// v_m = Gamma_m^T C_m^-1 z_m (C^-1 with tip/tilt removal or the tip/tilt-only
// measurement), Sec. 4.3 and the operator expansion of Sec. 5.1.
// io.in0: layer grids (NULL = the plan's phi); io.in1: slopes (MODE 1, 2).
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_forward(const InstDev *__restrict__ insts,
                                                     const FwdItem *__restrict__ items, IoArgs io) {
  __shared__ InstDev sI;
  __shared__ T s_psi[kFwdTile + 2][kFwdTile + 3];
  __shared__ T s_ex[kFwdTile + 1][kFwdTile + 2];
  __shared__ T s_ey[kFwdTile + 1][kFwdTile + 2];
  __shared__ double s_mean[2];
  __shared__ int s_last;
  const FwdItem it = items[blockIdx.x];
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const WfsDev W = I.wfs[it.wfs];
  const T *phi = io.in0[it.inst] ? static_cast<const T *>(io.in0[it.inst]) : static_cast<const T *>(I.phi);
  const T *dat = static_cast<const T *>(io.in1[it.inst]);
  T *v = static_cast<T *>(I.v) + W.v_off;
  const int nc = W.nc, n = W.n, tid = threadIdx.x;
  const T *et = static_cast<const T *>(I.edge_t) + 2 * W.edge_off;
  const int *eidx = I.edge_idx + W.edge_off;

  if (it.a0 < 0) {
    // Tip/tilt-only sensor: sum over valid subapertures of the Fried slopes
    // equals <Gamma^T 1, psi>, which lives on the pupil-edge corners only.
    double ax = 0.0, ay = 0.0;
    if (MODE != 2) {
      for (int e = tid; e < W.n_edge; e += blockDim.x) {
        const int c = eidx[e];
        const T ps = trace_corner<T>(I, it.wfs, nc, phi, c % nc, c / nc);
        ax += double(et[2 * e]) * double(ps);
        ay += double(et[2 * e + 1]) * double(ps);
      }
    }
    const double2 s = block_sum2(ax, ay);
    double zx = s.x / W.S, zy = s.y / W.S;   // model mean slopes
    if (MODE == 1) {
      zx = double(dat[W.slope_off]) - zx;
      zy = double(dat[W.slope_off + 1]) - zy;
    } else if (MODE == 2) {
      zx = double(dat[W.slope_off]);
      zy = double(dat[W.slope_off + 1]);
    }
    // C^-1 = sigma^-2 I_2 on the two means, M^T spreads w/S to every slope
    const T cx = T(W.inv_sigma2 * zx / W.S), cy = T(W.inv_sigma2 * zy / W.S);
    for (int e = tid; e < W.n_edge; e += blockDim.x) v[eidx[e]] = cx * et[2 * e] + cy * et[2 * e + 1];
    return;
  }

  const int a0 = it.a0, b0 = it.b0;
  const unsigned char *act = I.active + W.act_off;
  const int *sidx = I.sub_idx + W.sub_off;
  // 1. psi on the tile's corners plus a one-corner halo
  for (int idx = tid; idx < (kFwdTile + 2) * (kFwdTile + 2); idx += blockDim.x) {
    const int u = idx % (kFwdTile + 2), w = idx / (kFwdTile + 2);
    const int a = a0 - 1 + u, b = b0 - 1 + w;
    T val = T(0);
    if (MODE != 2 && a >= 0 && b >= 0 && a < nc && b < nc && act[b * nc + a])
      val = trace_corner<T>(I, it.wfs, nc, phi, a, b);
    s_psi[w][u] = val;
  }
  __syncthreads();
  // 2. weighted slopes of the subapertures the tile's corners touch
  double sx_acc = 0.0, sy_acc = 0.0;
  const T isg = T(W.inv_sigma2);
  for (int idx = tid; idx < (kFwdTile + 1) * (kFwdTile + 1); idx += blockDim.x) {
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
        if (u >= 1 && w >= 1) {   // subapertures owned by this tile
          sx_acc += double(sx);
          sy_acc += double(sy);
        }
        ex = isg * sx;
        ey = isg * sy;
      }
    }
    s_ex[w][u] = ex;
    s_ey[w][u] = ey;
  }
  __syncthreads();
  // 3. Gamma^T: each corner gathers its four neighbouring subapertures
  {
    const int u = tid % kFwdTile, w = tid / kFwdTile;
    const int a = a0 + u, b = b0 + w;
    if (a < nc && b < nc) {
      const T val = T(0.5) * (s_ex[w + 1][u] + s_ex[w][u] - s_ex[w + 1][u + 1] - s_ex[w][u + 1]) +
                    T(0.5) * (-s_ey[w + 1][u] + s_ey[w][u] - s_ey[w + 1][u + 1] + s_ey[w][u + 1]);
      v[b * nc + a] = val;
    }
  }
  if (W.kind != kRemoveTT) return;
  // 4. tip/tilt removal: (I - T) subtracts the mean slopes; as Gamma^T 1_x and
  //    Gamma^T 1_y live on the pupil edge, the last tile of the sensor applies
  //    the rank-2 correction there once every tile's sums are in.
  const double2 s = block_sum2(sx_acc, sy_acc);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    I.part[W.part_off + 2 * it.tile] = s.x;
    I.part[W.part_off + 2 * it.tile + 1] = s.y;
    __threadfence();
    const unsigned t = atomicAdd(I.tick + kTickFwd0 + it.wfs, 1u);
    s_last = (t == unsigned(W.n_tiles - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) {
    double Sx = 0.0, Sy = 0.0;
    for (int t = 0; t < W.n_tiles; ++t) {
      Sx += __ldcg(I.part + W.part_off + 2 * t);
      Sy += __ldcg(I.part + W.part_off + 2 * t + 1);
    }
    s_mean[0] = Sx / W.S;
    s_mean[1] = Sy / W.S;
    I.tick[kTickFwd0 + it.wfs] = 0u;
  }
  __syncthreads();
  const T cx = T(W.inv_sigma2 * s_mean[0]), cy = T(W.inv_sigma2 * s_mean[1]);
  for (int e = tid; e < W.n_edge; e += blockDim.x) {
    const int c = eidx[e];
    v[c] = __ldcg(v + c) - (cx * et[2 * e] + cy * et[2 * e + 1]);
  }
}

// ------------------------------------------------------- transform helpers

template <typename T>
struct Filt {
  T h[kMaxTaps], g[kMaxTaps];
  int L;
};

template <typename T>
__device__ __forceinline__ void load_filt(Filt<T> &f, const InstDev &I) {
  f.L = I.Lf;
#pragma unroll
  for (int t = 0; t < kMaxTaps; ++t) {
    f.h[t] = T(t < I.Lf ? I.h[t] : 0.0);
    f.g[t] = T(t < I.Lf ? I.g[t] : 0.0);
  }
}

// Adjoint ray-trace at layer node (row k, column i): g = sum_m P_m^T v_m, as a
// gather over the corners whose bilinear taps include the node.
template <typename T>
__device__ __forceinline__ T gather_node(const InstDev &I, int l, int N, int k, int i) {
  const T *pf = static_cast<const T *>(I.pos_f);
  const T *vv = static_cast<const T *>(I.v);
  T acc = T(0);
  for (int m = 0; m < I.n_wfs; ++m) {
    const WfsDev &W = I.wfs[m];
    const int nc = W.nc;
    const int po = I.pos_off[m * I.n_layers + l];
    const int ro = I.rng_off[m * I.n_layers + l];
    const int4 rx = I.rng[ro + i];
    const int4 ry = I.rng[ro + N + k];
    const T *vm = vv + W.v_off;
#pragma unroll
    for (int yr = 0; yr < 2; ++yr) {
      const int bs = yr ? ry.z : ry.x, bc = yr ? ry.w : ry.y;
      for (int b = bs; b < bs + bc; ++b) {
        const T fy = pf[po + nc + b];
        const T wy = (I.pos_i0[po + nc + b] == k) ? T(1) - fy : fy;
        T row = T(0);
#pragma unroll
        for (int xr = 0; xr < 2; ++xr) {
          const int as = xr ? rx.z : rx.x, ac = xr ? rx.w : rx.y;
          for (int a = as; a < as + ac; ++a) {
            const T fx = pf[po + a];
            const T wx = (I.pos_i0[po + a] == i) ? T(1) - fx : fx;
            row += wx * vm[b * nc + a];
          }
        }
        acc += wy * row;
      }
    }
  }
  return acc;
}

// Epilogue of the analysis for one output coefficient.
enum Epi : int { kEpiPlain = 0, kEpiOp = 1, kEpiResid = 2 };
enum Flags : int { kFlagWarm = 1, kFlagFirst = 2 };

template <typename T, int EPI>
struct Emit {
  T *out;          // plain: destination
  const T *P;      // op: direction p
  T *Q;            // op: q
  T *R, *Pn, *X;   // resid: r, p, x
  const T *jinv;
  const double *dalpha;
  int off, N, precond, warm;
  double acc0, acc1;
  __device__ __forceinline__ void operator()(int row, int col, int level, T w) {
    const int idx = off + row * N + col;
    if (EPI == kEpiPlain) {
      out[idx] = w;
    } else if (EPI == kEpiOp) {
      const T pv = P[idx];
      const T q = w + T(dalpha[level]) * pv;
      Q[idx] = q;
      acc0 += double(pv) * double(q);
    } else {
      T r = w;
      if (warm) r -= T(dalpha[level]) * X[idx];
      else X[idx] = T(0);
      const T z = precond ? jinv[idx] * r : r;
      R[idx] = r;
      Pn[idx] = z;
      acc0 += double(r) * double(z);
      acc1 += double(r) * double(r);
    }
  }
};

// ------------------------------------------------------------ k_analysis
// SRC 0: layer grids from io.in0.  SRC 1: adjoint gather from the plan's v.
// EPI plain: io.out0 = W g.  EPI op: q = W g + alpha D p with p = io.in1 (NULL:
// the plan's p), q = io.out0 (NULL: the plan's q); p.q -> alpha.
// EPI resid: r = W g - alpha D x (x = io.out0, zeroed when cold), p = z = J^-1 r,
// r.z -> rz.
template <typename T, int SRC, int EPI>
__global__ void __launch_bounds__(kThreads) k_analysis(const InstDev *__restrict__ insts,
                                                      const ClusterItem *__restrict__ items,
                                                      IoArgs io, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  __shared__ int s_last;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const ClusterItem it = items[blockIdx.x / C];
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int N = L.N, R0 = N / C, J = I.J, tid = threadIdx.x, nt = blockDim.x;
  T *A = reinterpret_cast<T *>(smem_raw);
  T *B = A + R0 * N;
  T *cb = B + R0 * N;
  T *cb2 = cb + C * C;
  Filt<T> f;
  load_filt(f, I);

  Emit<T, EPI> emit;
  emit.off = L.off;
  emit.N = N;
  emit.dalpha = L.dalpha;
  emit.precond = I.precond;
  emit.warm = (flags & kFlagWarm) ? 1 : 0;
  emit.acc0 = emit.acc1 = 0.0;
  emit.jinv = static_cast<const T *>(I.jinv);
  emit.out = static_cast<T *>(io.out0[it.inst]);
  emit.P = io.in1[it.inst] ? static_cast<const T *>(io.in1[it.inst]) : static_cast<const T *>(I.p);
  emit.Q = io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.q);
  emit.R = static_cast<T *>(I.r);
  emit.Pn = static_cast<T *>(I.p);
  emit.X = static_cast<T *>(io.out0[it.inst]);

  // own rows [crank*R0, (crank+1)*R0) of the layer grid
  if (SRC == 0) {
    const T *src = static_cast<const T *>(io.in0[it.inst]) + L.off + crank * R0 * N;
    for (int idx = tid; idx < R0 * N; idx += nt) A[idx] = src[idx];
  } else {
    for (int idx = tid; idx < R0 * N; idx += nt) {
      const int k = crank * R0 + idx / N, i = idx % N;
      A[idx] = gather_node<T>(I, it.layer, N, k, i);
    }
  }
  __syncthreads();

  int M = N, k = 1;
  for (; k <= J && M >= 2 * C; ++k, M >>= 1) {
    const int R = M / C, H = M >> 1, Rh = R >> 1;
    int lgR = 0;
    while ((1 << lgR) < R) ++lgR;
    // row pass (x): local
    for (int idx = tid; idx < R * H; idx += nt) {
      const int j = idx / H, i = idx - j * H;
      const T *row = A + j * M;
      T lo = T(0), hi = T(0);
#pragma unroll
      for (int t = 0; t < kMaxTaps; ++t) {
        if (t < f.L) {
          const T x = row[(2 * i + t) & (M - 1)];
          lo += f.h[t] * x;
          hi += f.g[t] * x;
        }
      }
      B[j * M + i] = lo;
      B[j * M + H + i] = hi;
    }
    cluster.sync();
    // column pass (y): rows 2i..2i+Lf-1 may live in the next CTAs
    for (int idx = tid; idx < Rh * M; idx += nt) {
      const int il = idx / M, x = idx - il * M;
      const int i = crank * Rh + il;
      T lo = T(0), hi = T(0);
#pragma unroll
      for (int t = 0; t < kMaxTaps; ++t) {
        if (t < f.L) {
          const int r = (2 * i + t) & (M - 1);
          const T val = cluster.map_shared_rank(B, r >> lgR)[(r & (R - 1)) * M + x];
          lo += f.h[t] * val;
          hi += f.g[t] * val;
        }
      }
      if (x < H) {
        if (k == J) emit(i, x, J, lo);
        else A[il * H + x] = lo;
      } else {
        emit(i, x, k, lo);
      }
      emit(H + i, x, k, hi);
    }
    cluster.sync();
  }
  if (k <= J) {
    // coarse levels: the remaining low-low block (side M = C) in CTA 0
    if (crank == 0) {
      for (int idx = tid; idx < M * M; idx += nt) {
        const int r = idx / M, c = idx - r * M;
        cb[idx] = cluster.map_shared_rank(A, r)[c];   // each CTA holds one row of side M
      }
    }
    cluster.sync();
    if (crank == 0) {
      __syncthreads();
      for (; k <= J; ++k, M >>= 1) {
        const int H = M >> 1;
        for (int idx = tid; idx < M * H; idx += nt) {
          const int j = idx / H, i = idx - j * H;
          T lo = T(0), hi = T(0);
#pragma unroll
          for (int t = 0; t < kMaxTaps; ++t) {
            if (t < f.L) {
              const T x = cb[j * M + ((2 * i + t) & (M - 1))];
              lo += f.h[t] * x;
              hi += f.g[t] * x;
            }
          }
          cb2[j * M + i] = lo;
          cb2[j * M + H + i] = hi;
        }
        __syncthreads();
        for (int idx = tid; idx < H * M; idx += nt) {
          const int i = idx / M, x = idx - i * M;
          T lo = T(0), hi = T(0);
#pragma unroll
          for (int t = 0; t < kMaxTaps; ++t) {
            if (t < f.L) {
              const T val = cb2[((2 * i + t) & (M - 1)) * M + x];
              lo += f.h[t] * val;
              hi += f.g[t] * val;
            }
          }
          if (x < H && k < J) cb[i * H + x] = lo;
          else emit(i, x, (x < H) ? J : k, lo);
          emit(H + i, x, k, hi);
        }
        __syncthreads();
      }
    }
  }
  if (EPI == kEpiPlain) return;

  // FP64 reduction of the epilogue dot products and the scalar step
  const double2 s = block_sum2(emit.acc0, emit.acc1);
  if (tid == 0) {
    const int slot = I.cl_part_off + 2 * (it.layer * C + crank);
    I.part[slot] = s.x;
    I.part[slot + 1] = s.y;
    __threadfence();
    const unsigned t = atomicAdd(I.tick + kTickCluster, 1u);
    s_last = (t == unsigned(I.n_layers * C - 1));
  }
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  double a0 = 0.0, a1 = 0.0;
  for (int q = 0; q < I.n_layers * C; ++q) {
    a0 += __ldcg(I.part + I.cl_part_off + 2 * q);
    a1 += __ldcg(I.part + I.cl_part_off + 2 * q + 1);
  }
  double *sc = I.scal;
  if (EPI == kEpiOp) {
    const double rz = sc[kRz];
    sc[kPq] = a0;
    // r = 0 (so p = 0 and p.Ap = 0) means the iterate is already exact: step 0
    const bool exact = (a0 == 0.0 && rz == 0.0);
    const bool bad = !exact && (!(a0 > 0.0) || !isfinite(a0) || !isfinite(rz) || sc[kFlag] != 0.0);
    if (bad) sc[kFlag] = 1.0;
    sc[kAlpha] = (bad || exact) ? 0.0 : rz / a0;
  } else {
    sc[kRz] = a0;
    sc[kRr] = a1;
    sc[kFlag] = 0.0;
    sc[kBeta] = 0.0;
  }
  I.tick[kTickCluster] = 0u;
}

// ----------------------------------------------------------- k_synthesis
// SRC 0: coefficients from io.in0.  SRC 1: p <- J^-1 r + beta p (beta ignored
// with kFlagFirst: p already holds z), written back to the plan's p.
// Output: io.out0 (NULL: the plan's phi).
template <typename T, int SRC>
__global__ void __launch_bounds__(kThreads) k_synthesis(const InstDev *__restrict__ insts,
                                                       const ClusterItem *__restrict__ items,
                                                       IoArgs io, int flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ InstDev sI;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = static_cast<int>(cluster.num_blocks());
  const int crank = static_cast<int>(cluster.block_rank());
  const ClusterItem it = items[blockIdx.x / C];
  load_inst(&sI, insts + it.inst);
  const InstDev &I = sI;
  const LayerDev &L = I.layers[it.layer];
  const int N = L.N, R0 = N / C, J = I.J, tid = threadIdx.x, nt = blockDim.x;
  T *buf0 = reinterpret_cast<T *>(smem_raw);
  T *buf1 = buf0 + R0 * N;
  T *cb = buf1 + R0 * N;   // low-low of the coarse stage
  T *cb2 = cb + C * C;     // column-synthesised block
  T *cb3 = cb2 + C * C;    // coarse pyramid (side C)
  Filt<T> f;
  load_filt(f, I);
  T *out = io.out0[it.inst] ? static_cast<T *>(io.out0[it.inst]) : static_cast<T *>(I.phi);
  const T *src = static_cast<const T *>(io.in0[it.inst]);
  T *P = static_cast<T *>(I.p);
  const T *Rv = static_cast<const T *>(I.r);
  const T *Jv = static_cast<const T *>(I.jinv);
  const T beta = T(I.scal[kBeta]);
  const bool first = (flags & kFlagFirst) != 0;
  auto coef = [&](int row, int col) -> T {
    const int idx = L.off + row * N + col;
    if (SRC == 0) return src[idx];
    if (first) return P[idx];
    const T r = Rv[idx];
    const T z = I.precond ? Jv[idx] * r : r;
    const T pn = z + beta * P[idx];
    P[idx] = pn;
    return pn;
  };
  int kd = 0;   // distributed levels 1..kd
  while (kd < J && (N >> kd) >= 2 * C) ++kd;

  T *A = buf0, *B = buf1;
  if (kd < J) {
    if (crank == 0) {
      for (int idx = tid; idx < C * C; idx += nt) cb3[idx] = coef(idx / C, idx % C);
      __syncthreads();
      {
        const int HJ = (N >> (J - 1)) >> 1;
        for (int idx = tid; idx < HJ * HJ; idx += nt) cb[idx] = cb3[(idx / HJ) * C + idx % HJ];
      }
      __syncthreads();
      for (int k = J; k > kd; --k) {
        const int M = N >> (k - 1), H = M >> 1;
        for (int idx = tid; idx < M * M; idx += nt) {
          const int y = idx / M, x = idx - y * M;
          T acc = T(0);
#pragma unroll
          for (int t = 0; t < kMaxTaps; ++t) {
            if (t < f.L && !((y - t) & 1)) {
              const int ii = ((y - t) & (M - 1)) >> 1;
              const T lo = x < H ? cb[ii * H + x] : cb3[ii * C + x];
              const T hi = cb3[(H + ii) * C + x];
              acc += f.h[t] * lo + f.g[t] * hi;
            }
          }
          cb2[y * M + x] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < M * M; idx += nt) {
          const int y = idx / M, j = idx - y * M;
          T acc = T(0);
#pragma unroll
          for (int t = 0; t < kMaxTaps; ++t) {
            if (t < f.L && !((j - t) & 1)) {
              const int jj = ((j - t) & (M - 1)) >> 1;
              acc += f.h[t] * cb2[y * M + jj] + f.g[t] * cb2[y * M + H + jj];
            }
          }
          cb[y * M + j] = acc;
        }
        __syncthreads();
      }
    }
    cluster.sync();
    // level kd: M = 2C, one low-low row per CTA
    const T *c0 = cluster.map_shared_rank(cb, 0);
    for (int j = tid; j < C; j += nt) A[j] = c0[crank * C + j];
  } else {
    const int M = N >> (J - 1), H = M >> 1, Rh = (M / C) >> 1;
    for (int idx = tid; idx < Rh * H; idx += nt) {
      const int il = idx / H, x = idx - il * H;
      A[il * H + x] = coef(crank * Rh + il, x);
    }
  }
  __syncthreads();

  for (int k = kd; k >= 1; --k) {
    const int M = N >> (k - 1), H = M >> 1, R = M / C, Rh = R >> 1;
    int lgRh = 0;
    while ((1 << lgRh) < Rh) ++lgRh;
    // step 1: own low-y rows (LL | HL) and high-y rows (LH | HH)
    for (int idx = tid; idx < Rh * M; idx += nt) {
      const int jl = idx / M, x = idx - jl * M;
      const int i = crank * Rh + jl;
      B[jl * M + x] = x < H ? A[jl * H + x] : coef(i, x);
      B[(Rh + jl) * M + x] = coef(H + i, x);
    }
    cluster.sync();
    // step 2: column synthesis of own output rows; inputs may be remote
    for (int idx = tid; idx < R * M; idx += nt) {
      const int yl = idx / M, x = idx - yl * M;
      const int y = crank * R + yl;
      T acc = T(0);
#pragma unroll
      for (int t = 0; t < kMaxTaps; ++t) {
        if (t < f.L && !((y - t) & 1)) {
          const int ii = ((y - t) & (M - 1)) >> 1;
          const T *Bo = cluster.map_shared_rank(B, ii >> lgRh);
          const int li = ii & (Rh - 1);
          acc += f.h[t] * Bo[li * M + x] + f.g[t] * Bo[(Rh + li) * M + x];
        }
      }
      A[yl * M + x] = acc;
    }
    cluster.sync();
    // step 3: row synthesis (local)
    for (int idx = tid; idx < R * M; idx += nt) {
      const int yl = idx / M, j = idx - yl * M;
      T acc = T(0);
#pragma unroll
      for (int t = 0; t < kMaxTaps; ++t) {
        if (t < f.L && !((j - t) & 1)) {
          const int jj = ((j - t) & (M - 1)) >> 1;
          acc += f.h[t] * A[yl * M + jj] + f.g[t] * A[yl * M + H + jj];
        }
      }
      if (k == 1) out[L.off + (crank * R + yl) * N + j] = acc;
      else B[yl * M + j] = acc;
    }
    __syncthreads();
    T *tmp = A;
    A = B;
    B = tmp;
  }
}

// -------------------------------------------------------------- k_update
// x += alpha p, r -= alpha q, z = J^-1 r, r.z and r.r; the last CTA forms
// beta = (r.z)_new / (r.z)_old.  io.out0: x.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(const InstDev *__restrict__ insts,
                                                    const UpdItem *__restrict__ items, IoArgs io) {
  __shared__ int s_last;
  const UpdItem it = items[blockIdx.x];
  const InstDev *I = insts + it.inst;
  const double alpha_d = I->scal[kAlpha];
  const T alpha = T(alpha_d);
  T *X = static_cast<T *>(io.out0[it.inst]);
  T *R = static_cast<T *>(I->r);
  const T *P = static_cast<const T *>(I->p);
  const T *Q = static_cast<const T *>(I->q);
  const T *Jv = static_cast<const T *>(I->jinv);
  const int precond = I->precond;
  const int end = min(it.start + kUpdChunk, I->n);
  double rz = 0.0, rr = 0.0;
  for (int idx = it.start + threadIdx.x; idx < end; idx += blockDim.x) {
    X[idx] = X[idx] + alpha * P[idx];
    const T r = R[idx] - alpha * Q[idx];
    R[idx] = r;
    const T z = precond ? Jv[idx] * r : r;
    rz += double(r) * double(z);
    rr += double(r) * double(r);
  }
  const double2 s = block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    I->part[I->upd_part_off + 2 * it.blk] = s.x;
    I->part[I->upd_part_off + 2 * it.blk + 1] = s.y;
    __threadfence();
    const unsigned t = atomicAdd(I->tick + kTickUpd, 1u);
    s_last = (t == unsigned(I->n_upd_blocks - 1));
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double a0 = 0.0, a1 = 0.0;
  for (int b = 0; b < I->n_upd_blocks; ++b) {
    a0 += __ldcg(I->part + I->upd_part_off + 2 * b);
    a1 += __ldcg(I->part + I->upd_part_off + 2 * b + 1);
  }
  double *sc = I->scal;
  const double rz_old = sc[kRz];
  if (!isfinite(a0)) sc[kFlag] = 1.0;
  const bool stop = sc[kFlag] != 0.0 || !isfinite(a0) || !(rz_old != 0.0);
  sc[kBeta] = stop ? 0.0 : a0 / rz_old;
  sc[kRz] = a0;
  sc[kRr] = a1;
  I->tick[kTickUpd] = 0u;
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
    double ax = 0.0, ay = 0.0;
    for (int e = threadIdx.x; e < W.n_edge; e += blockDim.x) {
      const int c = eidx[e];
      const T ps = trace_corner<T>(I, m, nc, phi, c % nc, c / nc);
      ax += double(et[2 * e]) * double(ps);
      ay += double(et[2 * e + 1]) * double(ps);
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
                         double *__restrict__ jdiag, void *jinv, int precision, int nc_max) {
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
    const double Jv = acc + L.dalpha[k];
    jdiag[lam] = Jv;
    if (precision) static_cast<double *>(jinv)[lam] = 1.0 / Jv;
    else static_cast<float *>(jinv)[lam] = float(1.0 / Jv);
  }
}

// ------------------------------------------------------------- launchers

namespace {

template <typename K>
cudaError_t launch_cluster(K kernel, int n_clusters, int C, size_t smem, cudaStream_t s,
                           const InstDev *insts, const ClusterItem *items, const IoArgs &io,
                           int flags) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_clusters * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, insts, items, io, flags);
}

template <typename K>
cudaError_t allow_cluster(K kernel) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxTransformSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

cudaError_t configure_kernels() {
  cudaError_t e = cudaSuccess;
#define TOMO_CFG(K) if (e == cudaSuccess) e = allow_cluster(K)
  TOMO_CFG((k_synthesis<float, 0>));
  TOMO_CFG((k_synthesis<float, 1>));
  TOMO_CFG((k_synthesis<double, 0>));
  TOMO_CFG((k_synthesis<double, 1>));
  TOMO_CFG((k_analysis<float, 0, kEpiPlain>));
  TOMO_CFG((k_analysis<float, 1, kEpiPlain>));
  TOMO_CFG((k_analysis<float, 1, kEpiOp>));
  TOMO_CFG((k_analysis<float, 1, kEpiResid>));
  TOMO_CFG((k_analysis<double, 0, kEpiPlain>));
  TOMO_CFG((k_analysis<double, 1, kEpiPlain>));
  TOMO_CFG((k_analysis<double, 1, kEpiOp>));
  TOMO_CFG((k_analysis<double, 1, kEpiResid>));
#undef TOMO_CFG
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  return e;
}

cudaError_t launch_synthesis(int precision, int src, int flags, const InstDev *insts,
                             const ClusterItem *items, int n_clusters, int C, size_t smem,
                             const IoArgs &io, cudaStream_t s) {
  if (precision == 0)
    return src ? launch_cluster(k_synthesis<float, 1>, n_clusters, C, smem, s, insts, items, io, flags)
               : launch_cluster(k_synthesis<float, 0>, n_clusters, C, smem, s, insts, items, io, flags);
  return src ? launch_cluster(k_synthesis<double, 1>, n_clusters, C, smem, s, insts, items, io, flags)
             : launch_cluster(k_synthesis<double, 0>, n_clusters, C, smem, s, insts, items, io, flags);
}

cudaError_t launch_analysis(int precision, int src, int epi, int flags, const InstDev *insts,
                            const ClusterItem *items, int n_clusters, int C, size_t smem,
                            const IoArgs &io, cudaStream_t s) {
#define TOMO_AN(T, S, E) launch_cluster(k_analysis<T, S, E>, n_clusters, C, smem, s, insts, items, io, flags)
  if (precision == 0) {
    if (src == 0) return TOMO_AN(float, 0, kEpiPlain);
    if (epi == kEpiPlain) return TOMO_AN(float, 1, kEpiPlain);
    if (epi == kEpiOp) return TOMO_AN(float, 1, kEpiOp);
    return TOMO_AN(float, 1, kEpiResid);
  }
  if (src == 0) return TOMO_AN(double, 0, kEpiPlain);
  if (epi == kEpiPlain) return TOMO_AN(double, 1, kEpiPlain);
  if (epi == kEpiOp) return TOMO_AN(double, 1, kEpiOp);
  return TOMO_AN(double, 1, kEpiResid);
#undef TOMO_AN
}

cudaError_t launch_forward(int precision, int mode, const InstDev *insts, const FwdItem *items,
                           int n_items, const IoArgs &io, cudaStream_t s) {
  const dim3 g(n_items), b(kThreads);
  if (precision == 0) {
    if (mode == 0) k_forward<float, 0><<<g, b, 0, s>>>(insts, items, io);
    else if (mode == 1) k_forward<float, 1><<<g, b, 0, s>>>(insts, items, io);
    else k_forward<float, 2><<<g, b, 0, s>>>(insts, items, io);
  } else {
    if (mode == 0) k_forward<double, 0><<<g, b, 0, s>>>(insts, items, io);
    else if (mode == 1) k_forward<double, 1><<<g, b, 0, s>>>(insts, items, io);
    else k_forward<double, 2><<<g, b, 0, s>>>(insts, items, io);
  }
  return cudaGetLastError();
}

cudaError_t launch_update(int precision, const InstDev *insts, const UpdItem *items, int n_items,
                          const IoArgs &io, cudaStream_t s) {
  if (precision == 0) k_update<float><<<n_items, kThreads, 0, s>>>(insts, items, io);
  else k_update<double><<<n_items, kThreads, 0, s>>>(insts, items, io);
  return cudaGetLastError();
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
                          int nc_max, cudaStream_t s) {
  const size_t per_warp = 4 * static_cast<size_t>(nc_max + 1) * sizeof(double);
  int warps = static_cast<int>((96 * 1024) / per_warp);
  warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
  const size_t smem = per_warp * warps;
  const int blocks = (n + warps - 1) / warps;
  k_jacobi<<<blocks, warps * 32, smem, s>>>(insts, prof, prof_off, pos_fd, jdiag, jinv, precision,
                                           nc_max);
  return cudaGetLastError();
}

}  // namespace tomo
