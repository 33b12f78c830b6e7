// Device helpers of the adjoint ray-trace P^T (Sec. 5.1), shared by the
// analysis kernel's staged gather and the separate gather kernel: the
// pupil-edge coefficients, the tap records and the pupil-edge sums.
#pragma once

#include <cuda_runtime.h>

#include "common.h"
#include "device_util.cuh"

namespace tomo {

// Coefficients of the pupil-edge terms, per edge slot, from the forward
// kernel's tile partials (one warp per slot, lanes in a fixed order):
// * tip/tilt removal: -sigma^-2 (mean z_x, mean z_y);
// * tip/tilt-only sensor: sigma^-2 z / S with z its two mean slopes: the
//   model's (tt_mode 0), data minus model (1), or the data alone (2), the data
//   read from `slopes`.
// FP32 plans sum the double-float partials and form the coefficients in
// double-float arithmetic; FP64 plans use doubles.
__device__ __forceinline__ void edge_pair(const EdgeSlot &es, int tt_mode, double a, double b,
                                          const double *slopes, double *out) {
  if (es.kind == kRemoveTT) {
    out[0] = -(a * es.tt_scale);
    out[1] = -(b * es.tt_scale);
    return;
  }
  double zx = a * es.inv_S, zy = b * es.inv_S;
  if (tt_mode == 1) {
    zx = slopes[es.slope_off] - zx;
    zy = slopes[es.slope_off + 1] - zy;
  } else if (tt_mode == 2) {
    zx = slopes[es.slope_off];
    zy = slopes[es.slope_off + 1];
  }
  out[0] = zx * es.tt_scale;
  out[1] = zy * es.tt_scale;
}

// (hi + lo) * s as a double-float (s rounded to float first)
__device__ __forceinline__ float2 df_scale(float hi, float lo, float s) {
  const float p = __fmul_rn(hi, s);
  return make_float2(p, __fadd_rn(__fmaf_rn(hi, s, -p), __fmul_rn(lo, s)));
}

__device__ __forceinline__ float edge_one(const EdgeSlot &es, int tt_mode, float hi, float lo, float data) {
  const float scale = static_cast<float>(es.tt_scale);
  if (es.kind == kRemoveTT) {
    const float2 m = df_scale(hi, lo, scale);
    return -__fadd_rn(m.x, m.y);
  }
  if (tt_mode == 2) return __fmul_rn(data, scale);
  float2 z = df_scale(hi, lo, static_cast<float>(es.inv_S));
  if (tt_mode == 1) {
    // data - z by two-sum, then the low part
    const float t = __fsub_rn(data, z.x);
    const float bp = __fsub_rn(t, data);
    const float e = __fadd_rn(__fsub_rn(data, __fsub_rn(t, bp)), __fsub_rn(-z.x, bp));
    z = make_float2(t, __fsub_rn(e, z.y));
  }
  const float2 c = df_scale(z.x, z.y, scale);
  return __fadd_rn(c.x, c.y);
}

// Tip/tilt removal under spot elongation: with m and q the means of z and of
// C_tilde^-1 z over the subapertures, (I - T) C_tilde^-1 (I - T) z =
// C_tilde^-1 z - C_tilde^-1 m - (q - M m), M = mean C_tilde_j^-1.  The forward
// kernel applied the first term; -sigma^-2 m - q + M m is constant over the
// subapertures (its Gamma^T lives on the pupil edge: this coefficient pair);
// the rest, sigma^-2 c_j g_j (g_j . m), reaches the corner field as
// m_x Gx + m_y Gy (returned in mo).
__device__ __forceinline__ void edge_elong(const EdgeSlot &es, double a, double b, double qa, double qb,
                                           double *out, double *mo) {
  const double mx = a * es.inv_S, my = b * es.inv_S, qx = qa * es.inv_S, qy = qb * es.inv_S;
  out[0] = -es.inv_sigma2 * mx - qx + (es.mb_xx * mx + es.mb_xy * my);
  out[1] = -es.inv_sigma2 * my - qy + (es.mb_xy * mx + es.mb_yy * my);
  mo[0] = mx;
  mo[1] = my;
}

// s_coef: 2 * kMaxEdgeSlots pupil-edge coefficient pairs, then per slot the
// mean slopes (m_x, m_y) that weight the elongation fields (0 without).
template <typename T>
__device__ void edge_coefficients(const InstDev &I, T *s_coef, int tt_mode, const T *slopes) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < I.n_edge_wfs; k += nw) {
    const EdgeSlot es = I.edge_slots[k];
    const bool sum = !(es.kind == kTTOnly && tt_mode == 2);
    const int stride = es.elong ? 4 : 2;   // doubles per tile
    if constexpr (sizeof(T) == 4) {
      Acc<float> a, b, qa, qb;
      if (sum)
        for (int t = lane; t < es.n_tiles; t += 32) {
          const float4 *pt = reinterpret_cast<const float4 *>(I.part + es.part_off + stride * t);
          const float4 v = pt[0];
          a.merge(v.x, v.y);
          b.merge(v.z, v.w);
          if (es.elong) {
            const float4 w = pt[1];
            qa.merge(w.x, w.y);
            qb.merge(w.z, w.w);
          }
        }
      warp_merge_down(a);
      warp_merge_down(b);
      if (es.elong) {
        warp_merge_down(qa);
        warp_merge_down(qb);
      }
      if (lane == 0) {
        if (es.elong) {
          double out[2], mo[2];
          edge_elong(es, a.value(), b.value(), qa.value(), qb.value(), out, mo);
          s_coef[2 * k] = T(out[0]);
          s_coef[2 * k + 1] = T(out[1]);
          s_coef[2 * kMaxEdgeSlots + 2 * k] = T(mo[0]);
          s_coef[2 * kMaxEdgeSlots + 2 * k + 1] = T(mo[1]);
        } else {
          const bool tt = es.kind == kTTOnly && tt_mode != 0;
          s_coef[2 * k] = edge_one(es, tt_mode, a.hi, a.lo, tt ? float(slopes[es.slope_off]) : 0.f);
          s_coef[2 * k + 1] = edge_one(es, tt_mode, b.hi, b.lo, tt ? float(slopes[es.slope_off + 1]) : 0.f);
          s_coef[2 * kMaxEdgeSlots + 2 * k] = T(0);
          s_coef[2 * kMaxEdgeSlots + 2 * k + 1] = T(0);
        }
      }
    } else {
      double a = 0.0, b = 0.0, qa = 0.0, qb = 0.0;
      if (sum)
        for (int t = lane; t < es.n_tiles; t += 32) {
          a += I.part[es.part_off + stride * t];
          b += I.part[es.part_off + stride * t + 1];
          if (es.elong) {
            qa += I.part[es.part_off + stride * t + 2];
            qb += I.part[es.part_off + stride * t + 3];
          }
        }
      a = warp_sum(a);
      b = warp_sum(b);
      if (es.elong) {
        qa = warp_sum(qa);
        qb = warp_sum(qb);
      }
      if (lane == 0) {
        double out[2], mo[2] = {0.0, 0.0};
        if (es.elong) edge_elong(es, a, b, qa, qb, out, mo);
        else edge_pair(es, tt_mode, a, b, reinterpret_cast<const double *>(slopes), out);
        s_coef[2 * k] = T(out[0]);
        s_coef[2 * k + 1] = T(out[1]);
        s_coef[2 * kMaxEdgeSlots + 2 * k] = T(mo[0]);
        s_coef[2 * kMaxEdgeSlots + 2 * k + 1] = T(mo[1]);
      }
    }
  }
  __syncthreads();
}

// One adjoint tap record: the window's first tap (an int in slot 0) and its
// KT weights, read with 16-byte vector loads.
template <typename T, int KT>
struct TapRec {
  static constexpr int RS = KT <= 3 ? 4 : 8;   // T words per record
  int off;
  T w[KT];
  __device__ __forceinline__ void load(const T *rec) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = reinterpret_cast<const float4 *>(rec)[0];
      off = __float_as_int(a.x);
      w[0] = a.y;
      w[1] = a.z;
      if constexpr (KT >= 3) w[2] = a.w;
      if constexpr (KT >= 4) w[3] = reinterpret_cast<const float4 *>(rec)[1].x;
    } else {
      const double2 a = reinterpret_cast<const double2 *>(rec)[0];
      const double2 b = reinterpret_cast<const double2 *>(rec)[1];
      off = __double2loint(a.x);
      w[0] = a.y;
      w[1] = b.x;
      if constexpr (KT >= 3) w[2] = b.y;
      if constexpr (KT >= 4) w[3] = reinterpret_cast<const double2 *>(rec)[2].x;
    }
  }
};

// (P^T v)(node) for one sensor: the KT x KT window of its corner field at p
// (row stride nc) weighted by the column weights x.w and the row weights y.w.
template <typename T, int KT, bool SHARED>
__device__ __forceinline__ T window_sum(const T *__restrict__ p, int nc, const TapRec<T, KT> &x,
                                        const TapRec<T, KT> &y) {
  T v[KT][KT];
#pragma unroll
  for (int ty = 0; ty < KT; ++ty)
#pragma unroll
    for (int tx = 0; tx < KT; ++tx) v[ty][tx] = SHARED ? p[ty * nc + tx] : __ldg(p + ty * nc + tx);
  T acc = T(0);
#pragma unroll
  for (int ty = 0; ty < KT; ++ty) {
    T sx = x.w[0] * v[ty][0];
#pragma unroll
    for (int tx = 1; tx < KT; ++tx) sx += x.w[tx] * v[ty][tx];
    acc += y.w[ty] * sx;
  }
  return acc;
}

// Pupil-edge terms of the CTA's nodes: A[node] += sum over its entries of
// (e_x t_x + e_y t_y) w (one short list per node, edge slots in s_coef).  The
// entries of a node are read kEdgeBatch at a time (independent loads, which
// matters when the lists are in global memory) and summed in list order.
constexpr int kEdgeBatch = 4;

// The pupil-edge sum of one node over its entries [e0, e1), in list order.
template <typename T>
__device__ __forceinline__ T edge_node_sum(int e0, int e1, const int *tk, const T *tw, const T *s_coef) {
  T acc = T(0);
  for (int b = e0; b < e1; b += kEdgeBatch) {
    int k[kEdgeBatch];
    T wx[kEdgeBatch], wy[kEdgeBatch];
#pragma unroll
    for (int u = 0; u < kEdgeBatch; ++u) {
      const int e = b + u < e1 ? b + u : b;
      k[u] = tk[e];
      wx[u] = tw[2 * e];
      wy[u] = tw[2 * e + 1];
    }
#pragma unroll
    for (int u = 0; u < kEdgeBatch; ++u)
      if (b + u < e1) acc += s_coef[2 * k[u]] * wx[u] + s_coef[2 * k[u] + 1] * wy[u];
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void gather_edges(int nn, const int *tn, const int *tb, const int *tk,
                                             const T *tw, T *A, const T *s_coef) {
  for (int j = threadIdx.x; j < nn; j += blockDim.x) A[tn[j]] += edge_node_sum<T>(tb[j], tb[j + 1], tk, tw, s_coef);
}

}  // namespace tomo
