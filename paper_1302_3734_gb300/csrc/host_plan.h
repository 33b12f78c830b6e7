// Host-side construction of a plan: validation of a tomo_geometry, the
// Daubechies filters, the pupil masks and every index table the kernels read.
#pragma once

#include <string>
#include <vector>

#include <vector_functions.h>
#include <vector_types.h>

#include "../../include/tomo.h"
#include "common.h"

namespace tomo {

struct HostPlan {
  int n_layers = 0, n_wfs = 0, J = 0, Lf = 0, precond = 0, precision = 0;
  double alpha = 0.0, L0 = 0.0;
  int n = 0, n_slopes = 0, v_total = 0, C = 0;
  int n_part = 0, cl_part_off = 0, upd_part_off = 0, fwd_part_off = 0, n_upd_blocks = 0;
  int n_lgs = 0;
  long long smem_transform = 0;   // dynamic shared memory of the synthesis kernel (bytes)
  long long smem_analysis = 0;    // dynamic shared memory of the gather + analysis kernel (bytes)
  int gather_staged = 0, n_dense = 0, max_tt_entries = 0, max_taps = 0,
      rec_stride = 0;
  std::vector<double> h, g;
  std::vector<LayerDev> layers;
  std::vector<double> layer_alt, layer_dx;   // altitude and grid spacing (m) of each layer
  std::vector<WfsDev> wfs;
  std::vector<double2> wfs_theta;          // guide-star direction (rad) of each sensor
  std::vector<double> wfs_height;          // laser guide star altitude (m); INFINITY: natural star
  std::vector<int> sub_idx;
  std::vector<unsigned char> active;
  std::vector<int> pos_off, pos_i0;
  std::vector<double> pos_f;
  // Adjoint tap windows: per (sensor, layer) N_l column records then N_l row
  // records; record r covers corners [gt_ro[r], gt_ro[r] + max_taps) of one
  // axis with weights gt_rw[4r ..] (row records add the sensor's v offset and
  // scale the corner row by nc); gt_ro = -1: no corner reaches the node.
  std::vector<int> gt_off;
  std::vector<int> gt_ro;
  std::vector<double> gt_rw;       // 4 per record, 0 beyond the window's taps
  std::vector<int> gt_ys;          // row records: window start in the CTA's staged v rows
  std::vector<int2> gt_cols;       // per (m,l): columns [x, x+y) mod N that the sensor's taps reach
  std::vector<int2> gt_brows;      // per (m,l,rank): {v offset of the band's first corner row, rows}
  long long max_band_cells = 0;    // largest (corner rows x columns) of one (sensor, layer, band)
  long long max_band_v = 0;        // largest 16-byte-aligned run of one band's corner rows of v
  int gather_vstage = 0;           // 1: the separate gather kernel stages those rows in shared memory
  long long smem_gather = 0;       // dynamic shared memory of the separate gather kernel (bytes)
  std::vector<int4> vs_run;        // per (layer, rank, dense sensor): {g0, nvec, smem offset, 0}
  int vstage = 0;                  // largest staged v (T elements) of one analysis CTA
  std::vector<unsigned char> stage_img;   // per (layer, rank) stage image, img_stride bytes apart
  long long img_stride = 0;
  std::vector<int2> tt_seg;        // per (layer, rank)
  std::vector<int> tt_node, tt_beg, tt_k;
  std::vector<double> tt_w;        // 2 per entry
  int n_tt = 0, n_edge_wfs = 0;
  std::vector<EdgeSlot> edge_slots;
  std::vector<double> gel;         // elongation corner fields (2 * v_total), empty if none
  std::vector<int> edge_idx;
  std::vector<double> edge_t;
  std::vector<int> run_rows;
  std::vector<int2> run_ab;
  // 1-D basis functions for the Jacobi diagonal: per layer, per level k (1..J),
  // per kind (0 scaling, 1 wavelet), N_l samples at position 0.
  std::vector<double> profiles;
  std::vector<int> prof_off;      // [layer * (J+1) * 2 + k * 2 + kind]
  // work tables (instance slot 0)
  std::vector<FwdItem> fwd_items;
  std::vector<ClusterItem> cl_items;
  std::vector<UpdItem> upd_items;
  // streamed transforms: pass items grouped by level (pass_off[k], pass_cnt[k],
  // k = 1..pass_kmax), one coarse item per layer, the analysis partials
  int stream_tf = 0, n_cl_part = 0, pass_kmax = 0;
  int pass_off[kMaxLevels + 1] = {0}, pass_cnt[kMaxLevels + 1] = {0};
  std::vector<PassItem> pass_items, coarse_items;
  // separate gather kernel: one CTA per (layer, band = row0), costliest first
  // (slot: the band's estimated cost)
  std::vector<PassItem> gather_items;
  long long smem_pass = 0, smem_coarse = 0, lls_elems = 0;
};

// Returns TOMO_OK or an error status with *err set.  cluster_request > 0 asks
// for that many CTAs per layer in the transform kernels (0: the default).
// transforms: 0 chooses, 1 asks for the cluster transforms, 2 for the streamed
// ones (level by level over row tiles).
tomo_status build_host_plan(const tomo_geometry *g, HostPlan *out, std::string *err,
                            int cluster_request = 0, int transforms = 0);

// Orthonormal Daubechies low-pass filter with p vanishing moments (2p taps),
// by spectral factorisation; exposed for tests through the plan only.
bool daubechies_filter(int p, std::vector<double> *h, std::string *err);

}  // namespace tomo
