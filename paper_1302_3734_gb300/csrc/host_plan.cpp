// Host-side plan construction.  Geometry conventions (Sec. 2.1 of the paper and
// the readings stated in tomo.h):
//   layer node (ix, iy) at ((ix - N/2) dx, (iy - N/2) dx);
//   sensor corner (a, b), a, b in 0..n, at ((a - n/2) d, (b - n/2) d);
//   the corner seen on layer l along guide star m is
//   (1 - h_l/H_m) r + theta_m h_l (H_m = infinity for a natural star).
#include "host_plan.h"

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>

namespace tomo {

namespace {

using cd = std::complex<double>;

double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Roots of a monic polynomial (coefficients ascending, c[deg] == 1) by the
// Weierstrass / Durand-Kerner simultaneous iteration.
std::vector<cd> poly_roots(const std::vector<double> &c) {
  const int deg = static_cast<int>(c.size()) - 1;
  std::vector<cd> z(deg);
  for (int k = 0; k < deg; ++k) z[k] = std::pow(cd(0.4, 0.9), k);
  auto eval = [&](cd x) {
    cd v(0.0, 0.0);
    for (int i = deg; i >= 0; --i) v = v * x + c[i];
    return v;
  };
  for (int it = 0; it < 500; ++it) {
    double delta = 0.0;
    for (int k = 0; k < deg; ++k) {
      cd den(1.0, 0.0);
      for (int j = 0; j < deg; ++j)
        if (j != k) den *= (z[k] - z[j]);
      cd step = eval(z[k]) / den;
      z[k] -= step;
      delta = std::max(delta, std::abs(step));
    }
    if (delta < 1e-16) break;
  }
  return z;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }

// One periodic synthesis level on x[0..M): y = [a | d] -> x.
void synth_1d(std::vector<double> *x, int M, const std::vector<double> &h,
              const std::vector<double> &g) {
  std::vector<double> out(M, 0.0);
  const int H = M / 2, L = static_cast<int>(h.size());
  for (int i = 0; i < H; ++i)
    for (int t = 0; t < L; ++t) out[(2 * i + t) % M] += h[t] * (*x)[i] + g[t] * (*x)[H + i];
  for (int i = 0; i < M; ++i) (*x)[i] = out[i];
}

}  // namespace

bool daubechies_filter(int p, std::vector<double> *h, std::string *err) {
  if (p < 1 || 2 * p > kMaxTaps) {
    *err = "wavelet_order must be in 1..4";
    return false;
  }
  // (1 + z)^p times one factor (z - z_k) per root of
  // P(y) = sum_{k<p} C(p-1+k, k) y^k, z_k the root of z^2 - (2 - 4 y_k) z + 1
  // inside the unit circle; coefficients in descending powers.
  std::vector<cd> poly{cd(1.0, 0.0)};
  auto mul = [&](cd a0, cd a1) {  // poly *= (a0 z + a1)
    std::vector<cd> r(poly.size() + 1, cd(0.0, 0.0));
    for (size_t i = 0; i < poly.size(); ++i) {
      r[i] += poly[i] * a0;
      r[i + 1] += poly[i] * a1;
    }
    poly.swap(r);
  };
  for (int i = 0; i < p; ++i) mul(1.0, 1.0);
  if (p > 1) {
    std::vector<double> c(p);
    for (int k = 0; k < p; ++k) c[k] = binom(p - 1 + k, k);
    const double lead = c[p - 1];
    for (auto &v : c) v /= lead;
    for (const cd &y : poly_roots(c)) {
      cd b = 2.0 - 4.0 * y;
      cd disc = std::sqrt(b * b - 4.0);
      cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
      mul(1.0, -(std::abs(z1) < 1.0 ? z1 : z2));
    }
  }
  h->assign(poly.size(), 0.0);
  double s = 0.0;
  for (size_t i = 0; i < poly.size(); ++i) {
    (*h)[i] = poly[i].real();
    s += (*h)[i];
  }
  for (auto &v : *h) v *= std::sqrt(2.0) / s;
  // self-check: double-shift orthonormality
  const int L = static_cast<int>(h->size());
  for (int m = 0; 2 * m < L; ++m) {
    double d = 0.0;
    for (int k = 0; k + 2 * m < L; ++k) d += (*h)[k] * (*h)[k + 2 * m];
    if (std::fabs(d - (m == 0 ? 1.0 : 0.0)) > 1e-12) {
      *err = "Daubechies factorisation failed its orthonormality check";
      return false;
    }
  }
  return true;
}

tomo_status build_host_plan(const tomo_geometry *geo, HostPlan *P, std::string *err,
                            int cluster_request, int transforms) {
  char buf[256];
  if (!geo || !geo->wfs || !geo->layers || geo->n_wfs < 1 || geo->n_layers < 1) {
    *err = "geometry, its sensor and layer arrays must be non-empty";
    return TOMO_ERR_ARG;
  }
  if (geo->precision != 0 && geo->precision != 1) { *err = "precision must be 0 or 1"; return TOMO_ERR_ARG; }
  if (geo->precond != 0 && geo->precond != 1) { *err = "precond must be 0 or 1"; return TOMO_ERR_ARG; }
  if (!(geo->alpha >= 0.0) || !std::isfinite(geo->alpha)) { *err = "alpha must be finite and >= 0"; return TOMO_ERR_ARG; }
  if (geo->levels < 1 || geo->levels > kMaxLevels) { *err = "levels out of range"; return TOMO_ERR_LEVELS; }
  if (geo->n_wfs > 4096 || geo->n_layers > 4096) { *err = "too many sensors or layers"; return TOMO_ERR_ARG; }
  if (!(geo->obstruction >= 0.0 && geo->obstruction < 1.0)) { *err = "obstruction must be in [0, 1)"; return TOMO_ERR_ARG; }

  P->n_layers = geo->n_layers;
  P->n_wfs = geo->n_wfs;
  P->J = geo->levels;
  P->precond = geo->precond;
  P->precision = geo->precision;
  P->alpha = geo->alpha;
  P->L0 = geo->L0;
  if (!daubechies_filter(geo->wavelet_order, &P->h, err)) return TOMO_ERR_ARG;
  P->Lf = static_cast<int>(P->h.size());
  P->g.resize(P->Lf);
  for (int k = 0; k < P->Lf; ++k) P->g[k] = ((k & 1) ? -1.0 : 1.0) * P->h[P->Lf - 1 - k];

  // ---------------------------------------------------------------- layers
  const int J = P->J;
  int Nmin = 1 << 30, Nmax = 0;
  P->n = 0;
  for (int l = 0; l < geo->n_layers; ++l) {
    const tomo_layer &L = geo->layers[l];
    if (!is_pow2(L.N) || L.N < 16 || L.N > 4096) {
      snprintf(buf, sizeof buf, "layer %d: N must be a power of two in [16, 4096]", l);
      *err = buf;
      return TOMO_ERR_LEVELS;
    }
    if ((L.N >> (J - 1)) < P->Lf) {
      snprintf(buf, sizeof buf, "layer %d: N/2^(levels-1) = %d is below the filter length %d", l,
               L.N >> (J - 1), P->Lf);
      *err = buf;
      return TOMO_ERR_LEVELS;
    }
    if (!(L.dx > 0.0) || !(L.prior_weight > 0.0) || !(L.altitude >= 0.0) ||
        !std::isfinite(L.altitude) || !std::isfinite(L.prior_weight)) {
      snprintf(buf, sizeof buf, "layer %d: dx, prior_weight must be > 0 and altitude >= 0", l);
      *err = buf;
      return TOMO_ERR_ARG;
    }
    LayerDev d{};
    d.N = L.N;
    d.log2N = ilog2(L.N);
    d.off = P->n;
    const double l0 = geo->L0 > 0.0 ? std::pow(geo->L0, -11.0 / 3.0) : 0.0;
    for (int k = 1; k <= J; ++k) {
      d.dprior[k] = L.prior_weight * (l0 + std::pow(std::ldexp(L.dx, k), -11.0 / 3.0));
      d.dalpha[k] = geo->alpha * d.dprior[k];
    }
    P->layers.push_back(d);
    P->layer_alt.push_back(L.altitude);
    P->layer_dx.push_back(L.dx);
    P->n += L.N * L.N;
    Nmin = std::min(Nmin, L.N);
    Nmax = std::max(Nmax, L.N);
  }
  // cluster size: every layer keeps >= 8 rows per CTA at level 1, unless the
  // caller asks for another power of two (1..16, at most N/2; streamed plans,
  // whose transforms use no cluster, up to 64 bands of the separate gather)
  P->C = std::min(16, Nmin / 8);
  if (cluster_request > 0) {
    const int cmax = transforms == 2 ? 64 : 16;
    if (cluster_request > cmax || (cluster_request & (cluster_request - 1)) || cluster_request > Nmin / 2) {
      *err = transforms == 2 ? "cluster size (gather bands) of a streamed plan must be a power of two in "
                               "[1, min(64, N/2)]"
                             : "cluster size must be a power of two in [1, min(16, N/2)]";
      return TOMO_ERR_ARG;
    }
    P->C = cluster_request;
  }
  {
    // shared memory of the transforms: row buffers, coarse buffers and the
    // coefficient cache of as many (coarse-first) levels as fit
    const long long esz = P->precision ? 8 : 4;
    const long long budget = 220LL * 1024 - 4096;   // opt-in limit minus static shared memory
    long long need = 0;
    bool cluster_fits = true;
    for (auto &d : P->layers) {
      const long long base = transform_cache_offset(d.N, P->C);
      int kc = 1;
      while (kc <= J && (base + transform_cache_size(d.N, P->C, J, kc)) * esz > budget) ++kc;
      const long long bytes = (base + transform_cache_size(d.N, P->C, J, kc)) * esz;
      cluster_fits = cluster_fits && bytes <= budget;
      d.cache_kc = kc;
      need = std::max(need, bytes);
    }
    P->smem_transform = need;
    // streamed transforms when asked, or when the cluster CTAs cannot share an SM
    // (one cluster per GPC at a time) or do not fit at all
    if (transforms < 0 || transforms > 2) {
      *err = "transforms must be 0 (choose), 1 (clusters) or 2 (streamed)";
      return TOMO_ERR_ARG;
    }
    P->stream_tf = transforms == 2 || (transforms == 0 && need > static_cast<long long>(108 * 1024));
    if (!P->stream_tf && !cluster_fits) {
      *err = "layer grids too large for the cluster transform kernels at this precision";
      return TOMO_ERR_UNSUPPORTED;
    }
    if (P->stream_tf) {
      int M0 = 1;
      for (auto &d : P->layers) {
        P->smem_pass = std::max<long long>(P->smem_pass, pass_smem_elems(d.N, P->Lf) * esz);
        d.ks = 1;
        while (d.ks <= J && (d.N >> (d.ks - 1)) > kCoarseMax) ++d.ks;
        M0 = std::max(M0, d.N >> (d.ks - 1));
        for (int k = 1; k < d.ks; ++k) {
          d.ll_off[k] = static_cast<int>(P->lls_elems);
          P->lls_elems += static_cast<long long>(d.N >> k) * (d.N >> k);
        }
        P->pass_kmax = std::max(P->pass_kmax, d.ks - 1);
      }
      P->smem_coarse = 3LL * M0 * M0 * esz;
      if (P->smem_pass > budget || P->smem_coarse > budget) {
        *err = "layer grids too large for the streamed transform kernels at this precision";
        return TOMO_ERR_UNSUPPORTED;
      }
      if (P->lls_elems > (1LL << 31) - 1) {
        *err = "layer grids too large for the streamed transforms' scratch";
        return TOMO_ERR_UNSUPPORTED;
      }
    }
  }

  // --------------------------------------------------------------- sensors
  int slope_off = 0, v_off = 0;
  P->n_lgs = 0;
  for (int m = 0; m < geo->n_wfs; ++m) {
    const tomo_wfs &W = geo->wfs[m];
    if (W.n_sub < 1 || W.n_sub > 1024 || !(W.d_sub > 0.0) || !(W.sigma > 0.0) ||
        !std::isfinite(W.theta_x) || !std::isfinite(W.theta_y)) {
      snprintf(buf, sizeof buf, "sensor %d: n_sub, d_sub, sigma or theta out of range", m);
      *err = buf;
      return TOMO_ERR_ARG;
    }
    if (W.tt_only && W.remove_tt) {
      snprintf(buf, sizeof buf, "sensor %d: tt_only and remove_tt exclude each other", m);
      *err = buf;
      return TOMO_ERR_ARG;
    }
    const int n = W.n_sub, nc = n + 1;
    const bool lgs = std::isfinite(W.height) && W.height > 0.0;
    WfsDev d{};
    d.n = n;
    d.nc = nc;
    d.kind = W.tt_only ? kTTOnly : (W.remove_tt ? kRemoveTT : kFull);
    d.is_lgs = lgs ? 1 : 0;
    d.inv_sigma2 = 1.0 / (W.sigma * W.sigma);
    d.inv_sigma2_f = static_cast<float>(d.inv_sigma2);
    if (!(W.elong_tau >= 0.0 && W.elong_tau <= 1.0) || !std::isfinite(W.elong_scale) ||
        !std::isfinite(W.llt_x) || !std::isfinite(W.llt_y)) {
      snprintf(buf, sizeof buf, "sensor %d: elong_tau must be in [0, 1] and the elongation finite", m);
      *err = buf;
      return TOMO_ERR_ARG;
    }
    d.elong = (lgs && !W.tt_only && W.elong_tau > 0.0 && W.elong_scale != 0.0) ? 1 : 0;
    d.el_tau = W.elong_tau;
    d.el_eps = W.elong_scale;
    d.el_lx = W.llt_x;
    d.el_ly = W.llt_y;
    d.d_sub = W.d_sub;
    P->n_lgs += lgs ? 1 : 0;
    // valid mask: given, or the circular pupil rule
    std::vector<unsigned char> valid(n * n);
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        if (W.valid) {
          valid[b * n + a] = W.valid[b * n + a] ? 1 : 0;
        } else {
          const double cx = (a + 0.5 - n / 2.0) * W.d_sub, cy = (b + 0.5 - n / 2.0) * W.d_sub;
          const double r = std::hypot(cx, cy);
          valid[b * n + a] = (r <= geo->D_tel / 2.0 && r >= geo->obstruction * geo->D_tel / 2.0) ? 1 : 0;
        }
      }
    d.sub_off = static_cast<int>(P->sub_idx.size());
    int S = 0;
    for (int i = 0; i < n * n; ++i) P->sub_idx.push_back(valid[i] ? S++ : -1);
    if (S == 0) {
      snprintf(buf, sizeof buf, "sensor %d has no valid subaperture", m);
      *err = buf;
      return TOMO_ERR_GEOMETRY;
    }
    d.S = S;
    d.inv_S = 1.0 / S;
    d.tt_scale = d.inv_sigma2 / S;
    auto V = [&](int a, int b) -> int {
      return (a >= 0 && b >= 0 && a < n && b < n && valid[b * n + a]) ? 1 : 0;
    };
    d.act_off = static_cast<int>(P->active.size());
    for (int b = 0; b < nc; ++b)
      for (int a = 0; a < nc; ++a)
        P->active.push_back((V(a - 1, b - 1) | V(a, b - 1) | V(a - 1, b) | V(a, b)) ? 1 : 0);
    // pupil-edge corners: Gamma^T 1_x and Gamma^T 1_y
    d.edge_off = static_cast<int>(P->edge_idx.size());
    for (int b = 0; b < nc; ++b)
      for (int a = 0; a < nc; ++a) {
        const double tx = 0.5 * (V(a - 1, b) + V(a - 1, b - 1) - V(a, b) - V(a, b - 1));
        const double ty = 0.5 * (-V(a - 1, b) + V(a - 1, b - 1) - V(a, b) + V(a, b - 1));
        if (tx != 0.0 || ty != 0.0) {
          P->edge_idx.push_back(b * nc + a);
          P->edge_t.push_back(tx);
          P->edge_t.push_back(ty);
        }
      }
    d.n_edge = static_cast<int>(P->edge_idx.size()) - d.edge_off;
    // valid runs per row (for the Jacobi diagonal)
    d.run_off = static_cast<int>(P->run_rows.size());
    for (int b = 0; b < n; ++b) {
      P->run_rows.push_back(static_cast<int>(P->run_ab.size()));
      int a = 0;
      while (a < n) {
        while (a < n && !valid[b * n + a]) ++a;
        if (a >= n) break;
        int a1 = a;
        while (a1 < n && valid[b * n + a1]) ++a1;
        P->run_ab.push_back(make_int2(a, a1));
        a = a1;
      }
    }
    P->run_rows.push_back(static_cast<int>(P->run_ab.size()));
    d.slope_off = slope_off;
    slope_off += d.kind == kTTOnly ? 2 : 2 * S;
    d.v_off = v_off;
    v_off += nc * nc;
    P->wfs.push_back(d);
    P->wfs_theta.push_back({W.theta_x, W.theta_y});
    P->wfs_height.push_back(lgs ? W.height : INFINITY);
  }
  P->n_slopes = slope_off;
  P->v_total = v_off;

  // ------------------------------------------------------ corner tables
  // Per (sensor, layer): each corner's wrapped node index and fraction along x
  // and y (forward bilinear taps), and per node and axis the window of
  // consecutive corners whose taps reach it with their weights (the transposed
  // ray-trace as a gather).
  P->pos_off.resize(P->n_wfs * P->n_layers);
  P->gt_off.assign(P->n_wfs * P->n_layers, -1);
  // edge slots: tip/tilt-only sensors first (their (e_x, e_y) live in ttc),
  // then the sensors with tip/tilt removal
  P->n_tt = 0;
  for (auto &d : P->wfs) d.tt_idx = d.kind == kTTOnly ? P->n_tt++ : -1;
  P->n_edge_wfs = P->n_tt;
  for (auto &d : P->wfs)
    if (d.kind == kRemoveTT) d.tt_idx = P->n_edge_wfs++;
  struct TTEntry { int layer, node, k; double wx, wy; };
  std::vector<TTEntry> tt_entries;
  std::vector<int> win_a0, win_n;   // per node and axis: first corner and count
  std::vector<std::array<double, kMaxTapsNode>> win_w;
  for (int m = 0; m < P->n_wfs; ++m) {
    const tomo_wfs &W = geo->wfs[m];
    const WfsDev &d = P->wfs[m];
    const bool lgs = d.is_lgs != 0;
    for (int l = 0; l < P->n_layers; ++l) {
      const tomo_layer &L = geo->layers[l];
      const int N = L.N, n = d.n, nc = d.nc;
      const double cone = lgs ? 1.0 - L.altitude / W.height : 1.0;
      if (!(cone > 0.0)) {
        snprintf(buf, sizeof buf, "layer %d lies at or above the altitude of guide star %d", l, m);
        *err = buf;
        return TOMO_ERR_GEOMETRY;
      }
      const int po = static_cast<int>(P->pos_i0.size());
      P->pos_off[m * P->n_layers + l] = po;
      std::vector<int> i0s[2];
      std::vector<double> fs[2];
      for (int axis = 0; axis < 2; ++axis) {
        const double th = axis == 0 ? W.theta_x : W.theta_y;
        for (int a = 0; a < nc; ++a) {
          const double r = (a - n / 2.0) * W.d_sub;
          double gc = (cone * r + th * L.altitude) / L.dx + N / 2.0;
          gc -= N * std::floor(gc / N);
          if (gc >= N) gc -= N;
          const double fl = std::floor(gc);
          P->pos_i0.push_back(static_cast<int>(fl));
          P->pos_f.push_back(gc - fl);
          i0s[axis].push_back(static_cast<int>(fl));
          fs[axis].push_back(gc - fl);
        }
      }
      // a footprint wider than the grid would make a node receive corners from
      // two periodic copies of the same side; reject it
      if (cone * n * W.d_sub / L.dx + 2.0 > N) {
        snprintf(buf, sizeof buf, "footprint of sensor %d on layer %d is wider than the grid", m, l);
        *err = buf;
        return TOMO_ERR_GEOMETRY;
      }
      if (d.kind == kTTOnly || d.kind == kRemoveTT) {
        // sparse adjoint of the rank-2 pupil-edge term of the sensor
        for (int e = d.edge_off; e < d.edge_off + d.n_edge; ++e) {
          const int c = P->edge_idx[e], a = c % nc, b = c / nc;
          const double tx = P->edge_t[2 * e], ty = P->edge_t[2 * e + 1];
          const int x0 = i0s[0][a], y0 = i0s[1][b], x1 = (x0 + 1) % N, y1 = (y0 + 1) % N;
          const double fx = fs[0][a], fy = fs[1][b];
          const int xs[4] = {x0, x1, x0, x1}, ys[4] = {y0, y0, y1, y1};
          const double ws[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
          for (int t = 0; t < 4; ++t)
            if (ws[t] != 0.0)
              tt_entries.push_back({l, ys[t] * N + xs[t], d.tt_idx, ws[t] * tx, ws[t] * ty});
        }
        if (d.kind == kTTOnly) continue;
      }
      // per node the consecutive run of corners whose bilinear taps reach it
      // (consecutive because the footprint is narrower than the grid)
      const int go = static_cast<int>(win_a0.size());
      P->gt_off[m * P->n_layers + l] = go;
      for (int axis = 0; axis < 2; ++axis) {
        std::vector<int> a0(N, -1), cnt(N, 0);
        std::vector<std::array<double, kMaxTapsNode>> w(N);
        for (auto &x : w) x.fill(0.0);
        auto add = [&](int i, int a, double wt) -> bool {
          if (cnt[i] == 0) a0[i] = a;
          else if (a != a0[i] + cnt[i]) return false;
          if (cnt[i] == kMaxTapsNode) return false;
          w[i][cnt[i]++] = wt;
          return true;
        };
        for (int a = 0; a < nc; ++a) {
          const int i0 = i0s[axis][a];
          const double f = fs[axis][a];
          bool ok = add(i0, a, 1.0 - f);
          if (f != 0.0) ok = ok && add((i0 + 1) % N, a, f);
          if (!ok) {
            snprintf(buf, sizeof buf,
                     "sensor %d on layer %d: more than %d corners per node (subaperture smaller "
                     "than half a layer cell)", m, l, kMaxTapsNode);
            *err = buf;
            return TOMO_ERR_UNSUPPORTED;
          }
        }
        for (int i = 0; i < N; ++i) {
          win_a0.push_back(a0[i]);
          win_n.push_back(cnt[i]);
          win_w.push_back(w[i]);
          P->max_taps = std::max(P->max_taps, cnt[i]);
        }
      }
    }
  }
  // records of KT taps (the widest run, at least 2), the window clamped to the
  // sensor's corners so that its zero-weight taps read inside the sensor's field
  {
    const int KT = std::max(2, P->max_taps);
    P->max_taps = KT;
    P->rec_stride = KT <= 3 ? 4 : 8;
    P->gt_ro.assign(win_a0.size(), -1);
    P->gt_rw.assign(4 * win_a0.size(), 0.0);
    for (int m = 0; m < P->n_wfs; ++m)
      for (int l = 0; l < P->n_layers; ++l) {
        const int go = P->gt_off[m * P->n_layers + l];
        if (go < 0) continue;
        const WfsDev &d = P->wfs[m];
        const int N = P->layers[l].N, nc = d.nc;
        for (int r = go; r < go + 2 * N; ++r) {
          if (win_n[r] == 0) continue;
          const int w0 = std::min(win_a0[r], std::max(0, nc - KT));
          for (int t = 0; t < win_n[r]; ++t) P->gt_rw[4 * r + win_a0[r] - w0 + t] = win_w[r][t];
          P->gt_ro[r] = r < go + N ? w0 : d.v_off + w0 * nc;
        }
      }
  }
  // per (sensor, layer): the columns its taps reach, one run mod N (all
  // columns when the valid records do not form one run)
  P->gt_cols.assign(static_cast<size_t>(P->n_wfs) * P->n_layers, make_int2(0, 0));
  for (int m = 0; m < P->n_wfs; ++m)
    for (int l = 0; l < P->n_layers; ++l) {
      const int go = P->gt_off[m * P->n_layers + l];
      if (go < 0) continue;
      const int N = P->layers[l].N;
      int nv = 0, c0 = -1;
      for (int i = 0; i < N; ++i) {
        const bool v = P->gt_ro[go + i] >= 0;
        nv += v ? 1 : 0;
        if (v && P->gt_ro[go + (i + N - 1) % N] < 0 && c0 < 0) c0 = i;
      }
      int2 cols = make_int2(0, nv == 0 ? 0 : N);
      if (nv > 0 && nv < N && c0 >= 0) {
        int run = 0;
        while (run < N && P->gt_ro[go + (c0 + run) % N] >= 0) ++run;
        if (run == nv) cols = make_int2(c0, nv);
      }
      P->gt_cols[m * P->n_layers + l] = cols;
    }
  // per (sensor, layer, cluster rank): the corner rows that the row records of the
  // rank's band of node rows reach, {v offset of the first row, row count}
  P->gt_brows.assign(static_cast<size_t>(P->n_wfs) * P->n_layers * P->C, make_int2(0, 0));
  P->max_band_cells = 0;
  for (int m = 0; m < P->n_wfs; ++m)
    for (int l = 0; l < P->n_layers; ++l) {
      const int go = P->gt_off[m * P->n_layers + l];
      if (go < 0) continue;
      const WfsDev &d = P->wfs[m];
      const int N = P->layers[l].N, R0 = N / P->C, KT = P->max_taps;
      for (int c = 0; c < P->C; ++c) {
        int lo = d.nc, hi = -1;
        for (int k = c * R0; k < (c + 1) * R0; ++k) {
          const int ro = P->gt_ro[go + N + k];
          if (ro < 0) continue;
          const int b0 = (ro - d.v_off) / d.nc;
          lo = std::min(lo, b0);
          hi = std::max(hi, std::min(d.nc, b0 + KT));
        }
        if (hi <= lo) continue;
        P->gt_brows[(static_cast<size_t>(m) * P->n_layers + l) * P->C + c] = make_int2(d.v_off + lo * d.nc, hi - lo);
        P->max_band_cells = std::max<long long>(P->max_band_cells,
                                                static_cast<long long>(hi - lo) * P->gt_cols[m * P->n_layers + l].y);
        // (KT more elements: a window's zero-weight taps may read past the rows when nc < KT)
        const int vq = P->precision ? 2 : 4, start = d.v_off + lo * d.nc;
        const long long run = start - start / vq * vq + static_cast<long long>(hi - lo) * d.nc + KT;
        P->max_band_v = std::max<long long>(P->max_band_v, (run + vq - 1) / vq * vq);
      }
    }
  if (P->n_edge_wfs > 64) {
    *err = "more than 64 sensors with tip/tilt removal or tip/tilt-only measurement";
    return TOMO_ERR_UNSUPPORTED;
  }
  // group the pupil-edge entries by (layer, cluster rank, node), and merge those
  // of one (node, edge slot): the slot's coefficients multiply the summed weights
  std::stable_sort(tt_entries.begin(), tt_entries.end(), [](const TTEntry &x, const TTEntry &y) {
    return x.layer != y.layer ? x.layer < y.layer : (x.node != y.node ? x.node < y.node : x.k < y.k);
  });
  {
    size_t w = 0;
    for (size_t e = 0; e < tt_entries.size(); ++e) {
      if (w > 0 && tt_entries[w - 1].layer == tt_entries[e].layer && tt_entries[w - 1].node == tt_entries[e].node &&
          tt_entries[w - 1].k == tt_entries[e].k) {
        tt_entries[w - 1].wx += tt_entries[e].wx;
        tt_entries[w - 1].wy += tt_entries[e].wy;
      } else {
        tt_entries[w++] = tt_entries[e];
      }
    }
    tt_entries.resize(w);
  }
  P->tt_seg.assign(static_cast<size_t>(P->n_layers) * P->C, make_int2(0, 0));
  {
    size_t e = 0;
    for (int l = 0; l < P->n_layers; ++l) {
      const int N = P->layers[l].N, R0 = N / P->C;
      for (int c = 0; c < P->C; ++c) {
        const int first = static_cast<int>(P->tt_node.size());
        while (e < tt_entries.size() && tt_entries[e].layer == l && tt_entries[e].node / N / R0 == c) {
          const int node = tt_entries[e].node;
          P->tt_node.push_back(node - c * R0 * N);
          P->tt_beg.push_back(static_cast<int>(P->tt_k.size()));
          while (e < tt_entries.size() && tt_entries[e].layer == l && tt_entries[e].node == node) {
            P->tt_k.push_back(tt_entries[e].k);
            P->tt_w.push_back(tt_entries[e].wx);
            P->tt_w.push_back(tt_entries[e].wy);
            ++e;
          }
        }
        P->tt_seg[l * P->C + c] = make_int2(first, static_cast<int>(P->tt_node.size()));
      }
    }
    P->tt_beg.push_back(static_cast<int>(P->tt_k.size()));
  }
  // the separate gather kernel's CTAs, one per (layer, band), costliest first so
  // that the light bands fill the end of the launch; a band's cost counts its
  // sensors' column sums and node rows, its pupil-edge entries and its grid rows
  P->gather_items.clear();
  for (int l = 0; l < P->n_layers; ++l) {
    const int N = P->layers[l].N, R0 = N / P->C;
    for (int c = 0; c < P->C; ++c) {
      long long cost = static_cast<long long>(R0) * N / 4;
      for (int m = 0; m < P->n_wfs; ++m) {
        const int2 br = P->gt_brows[(static_cast<size_t>(m) * P->n_layers + l) * P->C + c];
        const int ncol = P->gt_cols[m * P->n_layers + l].y;
        if (br.y > 0 && ncol > 0) cost += static_cast<long long>(br.y + R0) * ncol;
      }
      const int2 seg = P->tt_seg[l * P->C + c];
      cost += 4LL * (P->tt_beg[seg.y] - P->tt_beg[seg.x]);
      P->gather_items.push_back({0, l, c, static_cast<int>(std::min<long long>(cost, INT_MAX))});
    }
  }
  std::stable_sort(P->gather_items.begin(), P->gather_items.end(),
                   [](const PassItem &a, const PassItem &b) { return a.slot > b.slot; });
  // staging of the gather tables in the analysis kernel, when it fits
  P->n_dense = 0;
  for (const auto &d : P->wfs) P->n_dense += d.kind != kTTOnly ? 1 : 0;
  for (const auto &sg : P->tt_seg) {
    P->max_tt_entries = std::max(P->max_tt_entries, P->tt_beg[sg.y] - P->tt_beg[sg.x]);
  }
  // Corner rows of v that each analysis CTA's gather reads: per (layer, rank,
  // dense sensor) one run [g0, g0 + 16 nvec bytes) of v, 16-byte aligned,
  // covering every tap window of the CTA's node rows (KT rows of nc corners
  // plus KT columns of over-read when nc < KT); runs are packed in that order
  // in shared memory, and gt_ys gives each node row's window start there.
  {
    const int KT = P->max_taps, vq = P->precision ? 2 : 4;   // T elements per 16 bytes
    P->gt_ys.assign(P->gt_ro.size(), -1);
    P->vs_run.assign(static_cast<size_t>(P->n_layers) * P->C * std::max(1, P->n_dense),
                     make_int4(0, 0, 0, 0));
    P->vstage = 0;
    for (int l = 0; l < P->n_layers; ++l) {
      const int N = P->layers[l].N, R0 = N / P->C;
      for (int c = 0; c < P->C; ++c) {
        int sb = 0, md = 0;
        for (int m = 0; m < P->n_wfs; ++m) {
          const int go = P->gt_off[m * P->n_layers + l];
          if (go < 0) continue;
          const WfsDev &d = P->wfs[m];
          int lo = INT_MAX, hi = -1;
          for (int k = c * R0; k < (c + 1) * R0; ++k) {
            const int ro = P->gt_ro[go + N + k];
            if (ro < 0) continue;
            const int y0 = (ro - d.v_off) / d.nc;
            lo = std::min(lo, y0);
            hi = std::max(hi, y0 + KT - 1);
          }
          int4 run = make_int4(0, 0, sb, 0);
          if (hi >= 0) {
            const int g0 = (d.v_off + lo * d.nc) / vq * vq;
            const int g1 = (d.v_off + hi * d.nc + d.nc + KT + vq - 1) / vq * vq;
            run = make_int4(g0, (g1 - g0) / vq, sb, 0);
            for (int k = c * R0; k < (c + 1) * R0; ++k) {
              const int ro = P->gt_ro[go + N + k];
              if (ro >= 0) P->gt_ys[go + N + k] = sb + ro - g0;
            }
            sb += g1 - g0;
          }
          P->vs_run[(static_cast<size_t>(l) * P->C + c) * P->n_dense + md] = run;
          ++md;
        }
        P->vstage = std::max(P->vstage, sb);
      }
    }
  }
  {
    const int esz = P->precision ? 8 : 4;
    const long long budget = 220LL * 1024 - 4096;
    bool fits = true;
    long long need = 0;
    for (const auto &d : P->layers) {
      const long long tr = (transform_cache_offset(d.N, P->C) +
                            transform_cache_size(d.N, P->C, J, d.cache_kc)) * static_cast<long long>(esz);
      const StageLayout sl = stage_layout(P->n_dense, d.N, d.N / P->C, P->rec_stride, esz, P->max_tt_entries,
                                          P->vstage);
      const long long st = (tr + 15) / 16 * 16 + sl.total;
      fits = fits && st <= budget;
      need = std::max(need, st);
    }
    fits = fits && !P->stream_tf;   // streamed transforms take the gather from its own kernel
    fits = fits && P->max_tt_entries <= 65535;   // the image's 16-bit entry indices
    P->gather_staged = fits ? 1 : 0;
    P->smem_analysis = fits ? need : P->smem_transform;
    // the separate gather kernel: the band buffer (N/C rows of N), the band's row
    // records, one sensor's column-summed corner rows, and the staged corner rows
    // of two sensors where two CTAs per SM still fit
    long long plain = 0, staged = 0;
    for (const auto &d : P->layers) {
      plain = std::max<long long>(plain, gather_smem_layout(d.N / P->C, d.N, P->max_taps, esz, P->max_band_cells,
                                                            P->max_band_v, false).total);
      staged = std::max<long long>(staged, gather_smem_layout(d.N / P->C, d.N, P->max_taps, esz, P->max_band_cells,
                                                              P->max_band_v, true).total);
    }
    P->gather_vstage = staged <= kGatherStageSmem ? 1 : 0;
    P->smem_gather = P->gather_vstage ? staged : plain;
    if (!fits && P->smem_gather > 220LL * 1024) {
      *err = "layer grids too large for the separate gather kernel's band buffers";
      return TOMO_ERR_UNSUPPORTED;
    }
    if (!fits && P->n_dense > kMaxGatherSensors) {
      *err = "more than 64 sensors with a dense corner field on layer grids too large for the staged gather";
      return TOMO_ERR_UNSUPPORTED;
    }
  }
  // the stage images, one per analysis CTA
  if (P->gather_staged) {
    const int esz = P->precision ? 8 : 4, RS = P->rec_stride;
    long long stride = 16;
    for (const auto &d : P->layers)
      stride = std::max<long long>(stride, stage_layout(P->n_dense, d.N, d.N / P->C, RS, esz, P->max_tt_entries,
                                                        P->vstage).image);
    P->img_stride = stride;
    P->stage_img.assign(static_cast<size_t>(stride) * P->n_layers * P->C, 0);
    auto put_real = [&](unsigned char *dst, double v) {
      if (esz == 8) {
        std::memcpy(dst, &v, 8);
      } else {
        const float f = static_cast<float>(v);
        std::memcpy(dst, &f, 4);
      }
    };
    auto put_int = [&](unsigned char *dst, int v) { std::memcpy(dst, &v, 4); };
    for (int l = 0; l < P->n_layers; ++l) {
      const int N = P->layers[l].N, R0 = N / P->C;
      const StageLayout sl = stage_layout(P->n_dense, N, R0, RS, esz, P->max_tt_entries, P->vstage);
      for (int c = 0; c < P->C; ++c) {
        unsigned char *img = P->stage_img.data() + static_cast<size_t>(stride) * (l * P->C + c);
        int md = 0, vpre = 0;
        for (int m = 0; m < P->n_wfs; ++m) {
          const int go = P->gt_off[m * P->n_layers + l];
          if (go < 0) continue;
          auto put_rec = [&](unsigned char *dst, int r, int off) {
            put_int(dst, off);
            for (int t = 0; t < P->max_taps; ++t) put_real(dst + esz * (1 + t), P->gt_rw[4 * r + t]);
          };
          for (int i = 0; i < N; ++i)
            put_rec(img + sl.xr + static_cast<size_t>(esz) * RS * (md * N + i), go + i, P->gt_ro[go + i]);
          for (int k = 0; k < R0; ++k) {
            const int r = go + N + c * R0 + k;
            put_rec(img + sl.yr + static_cast<size_t>(esz) * RS * (md * R0 + k), r, P->gt_ys[r]);
          }
          const int4 run = P->vs_run[(static_cast<size_t>(l) * P->C + c) * P->n_dense + md];
          const int vq = 16 / esz;
          put_int(img + sl.mnc + 4 * md, P->wfs[m].nc);
          put_int(img + sl.vpre + 4 * md, vpre);
          put_int(img + sl.vsrc + 4 * md, run.x / vq);
          const WfsDev &dm = P->wfs[m];
          put_int(img + sl.mslot + 4 * md, (dm.elong && dm.kind == kRemoveTT) ? dm.tt_idx : -1);
          vpre += run.y;
          ++md;
        }
        put_int(img + sl.vpre + 4 * md, vpre);
        const int2 seg = P->tt_seg[l * P->C + c];
        const int nn = seg.y - seg.x, e0 = P->tt_beg[seg.x], ne = P->tt_beg[seg.y] - e0;
        for (int e = 0; e < ne; ++e) {
          put_int(img + sl.tk + 4 * e, P->tt_k[e0 + e]);
          put_real(img + sl.tw + esz * (2 * e), P->tt_w[2 * (e0 + e)]);
          put_real(img + sl.tw + esz * (2 * e + 1), P->tt_w[2 * (e0 + e) + 1]);
        }
        // per node the index of its first entry (the entries are sorted by node)
        for (int node = 0, j = 0; node <= R0 * N; ++node) {
          while (j < nn && P->tt_node[seg.x + j] < node) ++j;
          const uint16_t first = static_cast<uint16_t>(P->tt_beg[seg.x + j] - e0);
          std::memcpy(img + sl.eb + 2 * node, &first, 2);
        }
      }
    }
  }

  // -------------------------------------------------- Jacobi basis profiles
  P->prof_off.assign(static_cast<size_t>(P->n_layers) * (J + 1) * 2, 0);
  for (int l = 0; l < P->n_layers; ++l) {
    const int N = P->layers[l].N;
    for (int k = 1; k <= J; ++k)
      for (int kind = 0; kind < 2; ++kind) {
        const int M = N >> (k - 1);
        std::vector<double> x(N, 0.0);
        x[kind == 0 ? 0 : M / 2] = 1.0;
        for (int size = M; size <= N; size *= 2) synth_1d(&x, size, P->h, P->g);
        P->prof_off[(l * (J + 1) + k) * 2 + kind] = static_cast<int>(P->profiles.size());
        P->profiles.insert(P->profiles.end(), x.begin(), x.end());
      }
  }

  // --------------------------------------------------------- work tables
  int part = 0;
  P->cl_part_off = part;
  for (int l = 0; l < P->n_layers; ++l) P->cl_items.push_back({0, l});
  if (!P->stream_tf) {
    P->n_cl_part = P->n_layers * P->C;   // (dot, second dot) per analysis CTA
  } else {
    // streamed: per level the row tiles of the layers that pass through it, then one
    // coarse CTA per layer; every analysis CTA has its partial slot
    int slot = 0;
    for (int k = 1; k <= P->pass_kmax; ++k) {
      P->pass_off[k] = static_cast<int>(P->pass_items.size());
      for (int l = 0; l < P->n_layers; ++l) {
        const LayerDev &d = P->layers[l];
        if (k >= d.ks) continue;
        const int H = (d.N >> (k - 1)) >> 1;
        for (int r0 = 0; r0 < H; r0 += kPassRows) P->pass_items.push_back({0, l, r0, slot++});
      }
      P->pass_cnt[k] = static_cast<int>(P->pass_items.size()) - P->pass_off[k];
    }
    for (int l = 0; l < P->n_layers; ++l) P->coarse_items.push_back({0, l, 0, slot++});
    P->n_cl_part = slot;
  }
  part += 2 * P->n_cl_part;
  // update CTAs: consecutive chunks of kUpdChunk coefficients, at most kUpdMaxBlocks CTAs
  // (the consumers of their partials sum one partial per CTA)
  const int chunks = (P->n + kUpdChunk - 1) / kUpdChunk;
  const int per_cta = (chunks + kUpdMaxBlocks - 1) / kUpdMaxBlocks;
  P->n_upd_blocks = (chunks + per_cta - 1) / per_cta;
  P->upd_part_off = part;
  part += 2 * P->n_upd_blocks;
  for (int b = 0; b < P->n_upd_blocks; ++b)
    P->upd_items.push_back({0, b * per_cta * kUpdChunk, b, std::min(per_cta, chunks - b * per_cta)});
  P->fwd_part_off = part;
  for (int m = 0; m < P->n_wfs; ++m) {
    WfsDev &d = P->wfs[m];
    d.part_off = part;
    if (d.kind == kTTOnly) {
      // (edge corner, layer) pairs, one per thread of a chunk
      const int pairs = d.n_edge * P->n_layers;
      const int chunks = (pairs + kThreads - 1) / kThreads;
      d.n_tiles = chunks;
      for (int c = 0; c < chunks; ++c) P->fwd_items.push_back({0, m, -1, 0, c, 0, 0, 0});
      part += 2 * chunks;
      continue;
    }
    const int nt = (d.nc + kFwdTile - 1) / kFwdTile;
    int tiles = 0;
    for (int tb = 0; tb < nt; ++tb)
      for (int ta = 0; ta < nt; ++ta) {
        bool any = false;
        for (int b = tb * kFwdTile; b < std::min(d.nc, (tb + 1) * kFwdTile) && !any; ++b)
          for (int a = ta * kFwdTile; a < std::min(d.nc, (ta + 1) * kFwdTile) && !any; ++a)
            any = P->active[d.act_off + b * d.nc + a] != 0;
        if (!any) continue;
        P->fwd_items.push_back({0, m, ta * kFwdTile, tb * kFwdTile, tiles, 0, 0, 0});
        ++tiles;
      }
    d.n_tiles = tiles;
    part += tile_partials(d) * tiles;
  }
  P->n_part = part;
  P->edge_slots.assign(std::max(1, P->n_edge_wfs), EdgeSlot{});
  for (int m = 0; m < P->n_wfs; ++m) {
    const WfsDev &d = P->wfs[m];
    if (d.tt_idx < 0) continue;
    EdgeSlot e{};
    e.part_off = d.part_off;
    e.n_tiles = d.n_tiles;
    e.kind = d.kind;
    e.slope_off = d.slope_off;
    e.inv_S = d.inv_S;
    e.tt_scale = d.tt_scale;
    e.inv_sigma2 = d.inv_sigma2;
    e.elong = (d.elong && d.kind == kRemoveTT) ? 1 : 0;
    if (e.elong) {
      // M = mean over the valid subapertures of C_tilde_j^-1 = sigma^-2 (I - c_j g_j g_j^T)
      double xx = 0.0, xy = 0.0, yy = 0.0;
      for (int b = 0; b < d.n; ++b)
        for (int a = 0; a < d.n; ++a) {
          if (P->sub_idx[d.sub_off + b * d.n + a] < 0) continue;
          const double gx = d.el_eps * ((a + 0.5 - d.n / 2.0) * d.d_sub - d.el_lx);
          const double gy = d.el_eps * ((b + 0.5 - d.n / 2.0) * d.d_sub - d.el_ly);
          const double c = d.el_tau / (1.0 + d.el_tau * (gx * gx + gy * gy));
          xx += 1.0 - c * gx * gx;
          xy += -c * gx * gy;
          yy += 1.0 - c * gy * gy;
        }
      e.mb_xx = d.inv_sigma2 * xx / d.S;
      e.mb_xy = d.inv_sigma2 * xy / d.S;
      e.mb_yy = d.inv_sigma2 * yy / d.S;
    }
    P->edge_slots[d.tt_idx] = e;
  }
  // the elongation corner fields: Fried transpose of sigma^-2 c_j g_k,j g_j,
  // corner (a, b) receiving +-1/2 from the valid subapertures around it
  bool any_el = false;
  for (const auto &e : P->edge_slots) any_el = any_el || e.elong;
  P->gel.clear();
  if (any_el) {
    P->gel.assign(2 * static_cast<size_t>(P->v_total), 0.0);
    for (int m = 0; m < P->n_wfs; ++m) {
      const WfsDev &d = P->wfs[m];
      if (!(d.elong && d.kind == kRemoveTT)) continue;
      const int n = d.n, nc = d.nc;
      auto field = [&](int k, int a, int b, double *ex, double *ey) {
        *ex = *ey = 0.0;
        if (a < 0 || b < 0 || a >= n || b >= n || P->sub_idx[d.sub_off + b * n + a] < 0) return;
        const double gx = d.el_eps * ((a + 0.5 - n / 2.0) * d.d_sub - d.el_lx);
        const double gy = d.el_eps * ((b + 0.5 - n / 2.0) * d.d_sub - d.el_ly);
        const double c = d.el_tau / (1.0 + d.el_tau * (gx * gx + gy * gy));
        const double gk = k == 0 ? gx : gy;
        *ex = d.inv_sigma2 * c * gk * gx;
        *ey = d.inv_sigma2 * c * gk * gy;
      };
      for (int k = 0; k < 2; ++k)
        for (int b = 0; b < nc; ++b)
          for (int a = 0; a < nc; ++a) {
            double x00, y00, x01, y01, x10, y10, x11, y11;   // (a-1,b-1) (a-1,b) (a,b-1) (a,b)
            field(k, a - 1, b - 1, &x00, &y00);
            field(k, a - 1, b, &x01, &y01);
            field(k, a, b - 1, &x10, &y10);
            field(k, a, b, &x11, &y11);
            P->gel[k * static_cast<size_t>(P->v_total) + d.v_off + b * nc + a] =
                0.5 * (x01 + x00 - x11 - x10) + 0.5 * (-y01 + y00 - y11 + y10);
          }
    }
  }
  return TOMO_OK;
}

}  // namespace tomo
