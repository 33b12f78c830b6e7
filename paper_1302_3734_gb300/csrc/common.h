// Internal structures shared by the host plan builder and the CUDA kernels.
//
// One "instance" is one adaptive-optics system (one plan).  Kernels are written
// over a table of instances so that a launch can serve one plan or a batch of
// plans of uneven size; every work item of a launch names its instance.
#pragma once

#include <stdint.h>

namespace tomo {

constexpr int kMaxTaps = 8;        // Daubechies order <= 4
constexpr int kMaxLevels = 12;
constexpr int kFwdTile = 16;       // corners per side of a forward tile
constexpr int kMaxBatch = 96;      // instances per launch (kernel-argument arrays)
constexpr int kThreads = 256;      // threads per CTA of the hot kernels (transforms: below)
constexpr int kFwdThreads = 512;   // largest forward CTA; small launches use it, big batches kThreads
constexpr int kFwdSmallLaunch = 608;   // forward CTAs up to which a launch uses kFwdThreads
constexpr int kAnalysisThreads = 512;  // threads per CTA of the gather + analysis kernel when two fit an SM
constexpr int kAnalysisThreadsMax = 1024;  // ... when its shared memory leaves room for one
constexpr int kSynthThreads = 512;     // threads per CTA of the synthesis kernel (at most)
constexpr int kGatherThreads = 512;    // threads per CTA of the separate gather kernel
constexpr int kMaxGatherSensors = 64;  // dense sensors the separate gather kernel stages
constexpr int kUpdChunk = 1024;    // coefficients per pass of a vector-update CTA
constexpr int kUpdMaxBlocks = 608; // update CTAs per instance at most (four per SM of 152 SMs)
constexpr int kMaxTapsNode = 4;    // corners per axis whose bilinear taps reach one node
constexpr int kPassRows = 8;       // half-rows of a level one CTA of a streamed transform pass covers
constexpr int kPassThreads = 512;  // threads per CTA of the streamed transform kernels
constexpr int kCoarseMax = 64;     // block side up to which one CTA finishes a layer's transform

enum WfsKind : int { kFull = 0, kRemoveTT = 1, kTTOnly = 2 };

constexpr int kMaxEdgeSlots = 64;   // sensors with a pupil-edge term

// Scalar slots (double) of an instance.  r.z of iteration it lives in
// kRz0 + (it & 1): the synthesis of iteration it writes it while reading the
// other slot (r.z of iteration it-1) for beta.
enum Scalar : int {
  kRz0 = 0,
  kRz1 = 1,
  kBeta = 2,    // beta of the iteration, stored by the streamed coarse synthesis for its passes
  kFlag = 5,    // 1 after a breakdown (p.Ap <= 0 or not finite)
  kNumScalars = 8
};

// Bits of the `flags` kernel argument; the iteration index sits above them.
enum Flags : int { kFlagWarm = 1, kFlagFirst = 2, kIterShift = 8 };

struct LayerDev {
  int N, log2N;
  int off;                      // offset of this layer in the coefficient / grid vectors
  int cache_kc;                 // transforms cache the coefficients of levels >= cache_kc
  double dalpha[kMaxLevels + 1];  // alpha * D at level k (index k = 1..J)
  double dprior[kMaxLevels + 1];  // D at level k, without alpha
  // Streamed transforms: levels 1..ks-1 run as row-tile passes over the whole
  // grid, levels ks..J in one CTA per layer (block side N >> (ks - 1) <= kCoarseMax);
  // ll_off[k]: offset in the plan's scratch of the low-low block of level k
  // (side N >> k), k = 1..ks-1.
  int ks, pad_ks;
  int ll_off[kMaxLevels + 1];
};

struct WfsDev {
  int n, nc;                    // subapertures and corners per side
  int S, kind;
  int is_lgs;
  int slope_off;                // offset of this sensor in the slope vector
  int v_off;                    // offset of this sensor's corner field (nc*nc)
  int n_tiles;                  // forward tiles (partial-sum slots)
  int part_off;                 // offset of its partial sums in the instance partials (doubles)
  int n_edge, edge_off;         // pupil-edge corners where Gamma^T 1_x or Gamma^T 1_y != 0
  int sub_off;                  // offset into the subaperture-index table (n*n)
  int act_off;                  // offset into the active-corner table (nc*nc)
  int run_off;                  // offset of the per-row valid runs (n+1 row offsets)
  int tt_idx;                   // slot among the sensors with a pupil-edge correction, -1 otherwise
  float inv_sigma2_f;           // inv_sigma2 rounded to FP32 on the host (FP32 kernels read it)
  double inv_sigma2;
  double inv_S;                 // 1 / S (means of the slopes)
  double tt_scale;              // sigma^-2 / S
  // spot elongation (LGS): the subaperture's noise block sigma^2 (I + tau g g^T),
  // g = el_eps * (centre - (el_lx, el_ly)); centre = ((a + 1/2 - n/2) d, (b + 1/2 - n/2) d)
  int elong, pad_el;
  double el_tau, el_eps, el_lx, el_ly, d_sub;
};

// One sensor with a pupil-edge term (edge slot k = its tt_idx): where its
// forward partials are and how they scale into the edge coefficients.
struct EdgeSlot {
  int part_off, n_tiles, kind, slope_off;
  double inv_S, tt_scale;
  // tip/tilt removal under spot elongation: sigma^-2, and M = mean over the
  // subapertures of C_tilde_j^-1 (symmetric 2x2)
  int elong, pad;
  double inv_sigma2, mb_xx, mb_xy, mb_yy;
};

// Everything a kernel needs to know about one instance.  Pointers to element
// type T arrays are void* (T = float or double by plan precision).
struct InstDev {
  int n, n_layers, n_wfs, J;
  int Lf, precond, C, n_slopes;
  int cl_part_off, upd_part_off, n_upd_blocks, fwd_part_off;
  double h[kMaxTaps], g[kMaxTaps];
  // the same taps rounded to FP32 once on the host (round to nearest, as a
  // device conversion would): FP32 kernels read these, so no thread spends the
  // FP64 pipe, a small fraction of the FP32 rate on this GPU, converting them
  float hf[kMaxTaps], gf[kMaxTaps];
  // workspace
  void *r, *p, *q, *phi, *v, *jinv;
  double *scal, *part;
  // geometry tables
  const LayerDev *layers;
  const WfsDev *wfs;
  const int *sub_idx;           // per sensor n*n: index among the valid subapertures, or -1
  const unsigned char *active;  // per sensor nc*nc: corner of a valid subaperture
  const int *pos_off;           // per (m,l): offset of the x corner table (y table follows, nc)
  const int *pos_i0;            // wrapped integer node index of each corner coordinate
  const void *pos_f;            // fractional part (T)
  const int *gt_off;            // per (m,l): first tap record (x: N_l records, then y: N_l)
  // Tap records, rec_stride T each, 16-byte aligned: slot 0 holds the int
  // offset of the window's first tap (x: corner column; y: v_off + nc * corner
  // row; -1 when no corner reaches the node), slots 1..max_taps its weights.
  const void *gt_rec;
  const int *gt_ys;             // per row record: its window start in the staged v rows
  const int4 *vs_run;           // per (layer, rank, dense sensor): v run {g0, 16-byte words, smem offset}
  int vstage, v_total;          // staged v elements per analysis CTA; corner values of all sensors
  int max_band_cells;           // separate gather: largest column sums of one (sensor, layer, band)
  int max_band_v;               // ... and largest 16-byte-aligned run of its band rows of v (elements)
  const int2 *gt_cols;          // per (m,l): columns [x, x+y) mod N_l that the sensor's taps reach
  const int2 *gt_brows;         // per (m,l,rank): {v offset of the first corner row the band's row
                                // records reach, number of rows}
  const void *stage_img;        // per (layer, rank): the CTA's stage image (img_stride bytes apart)
  long long img_stride;
  // Pupil-edge corrections: a tip/tilt-only sensor's corner field is
  // e_x t_x + e_y t_y and tip/tilt removal subtracts sigma^-2 (m_x t_x + m_y t_y),
  // with t = Gamma^T 1 nonzero on the pupil edge only; both reach the layers
  // through this sparse list.
  const int2 *tt_seg;           // per (layer, cluster rank): [first, end) nodes with entries
  const int *tt_node;           // local node index (row-in-CTA * N + column)
  const int *tt_beg;            // entries [tt_beg[j], tt_beg[j+1]) of node j
  const int *tt_k;              // edge slot of the entry
  const void *tt_w;             // (w t_x, w t_y) of the entry (T pairs)
  int n_tt, n_edge_wfs;         // tip/tilt-only sensors; sensors with an edge slot
  const EdgeSlot *edge_slots;   // per edge slot (n_edge_wfs)
  // Tip/tilt removal under spot elongation: the corner fields
  // Gamma^T (sigma^-2 c_j g_x,j g_j) and Gamma^T (sigma^-2 c_j g_y,j g_j)
  // (c_j = tau / (1 + tau |g_j|^2)), laid out like v (Gx: v_total, then Gy),
  // whose sum weighted by the sensor's mean slopes completes its corner field.
  const void *gel;
  // Staging of the gather tables in the analysis kernel's shared memory
  // (loaded before the dependency wait); 0 = read them from global memory.
  int gather_staged, n_dense;   // flag; sensors with a dense corner field
  int max_taps, rec_stride;     // taps per window (2..4); T words per tap record (4 or 8)
  int max_tt_entries;           // largest per-CTA pupil-edge segment (entries)
  const int *edge_idx;          // corner index of each edge corner
  const void *edge_t;           // (t_x, t_y) of each edge corner (T, interleaved)
  const int *run_rows;          // per sensor (n+1): start of row b's runs in run_ab
  const int2 *run_ab;           // [a_lo, a_hi) runs of valid subapertures in a row
  // Streamed transforms (stream_tf != 0): the direction p of PCG iteration it
  // lives in p (it even) or p2 (it odd), since a pass reads the previous
  // direction of halo rows that another CTA rewrites; lls holds the low-low
  // blocks between the passes.  n_cl_part: (dot, dot) partials of the analysis
  // CTAs at cl_part_off.
  int stream_tf, n_cl_part;
  void *p2, *lls;
  // The plan's breakdown word: page-locked host memory mapped into the device
  // address space.  The update kernel sets it to 1 when a (P)CG step breaks
  // down; only the host clears it, after reporting it (NULL: not recorded).
  int *bd_word;
};

// Per-launch pointer arguments (indexed by the instance's slot in the launch).
struct IoArgs {
  const void *in0[kMaxBatch];
  const void *in1[kMaxBatch];
  void *out0[kMaxBatch];
  const int *active;            // device flags per instance slot; NULL = all active
};

#ifdef __CUDACC__
#define TOMO_HD __host__ __device__
#else
#define TOMO_HD
#endif

// Partial sums per forward tile of a sensor's slope vector: 2 (the sums of z),
// or 4 with tip/tilt removal under elongation (also the sums of C_tilde^-1 z).
TOMO_HD inline int tile_partials(const WfsDev &d) { return (d.elong && d.kind == 1) ? 4 : 2; }


// Shared-memory layout of the transform kernels (elements of T): two row
// buffers of (N/C + kMaxTaps) x N, two coarse buffers of C x C, then the
// coefficient cache.
TOMO_HD inline int transform_cache_offset(int N, int C) {
  return 2 * (N / C + kMaxTaps) * N + 2 * C * C;
}

// Elements of the coefficient cache of one CTA when levels >= kc are cached
// (the largest over the cluster's ranks: rank 0 also holds the coarse block).
TOMO_HD inline int transform_cache_size(int N, int C, int J, int kc) {
  int kd = 0;
  while (kd < J && (N >> kd) >= 2 * C) ++kd;
  int total = 0;
  for (int k = kc < 1 ? 1 : kc; k <= kd; ++k) {
    const int M = N >> (k - 1), Rh = (M / C) >> 1;
    total += Rh * (M >> 1) + Rh * M;
  }
  if (kd == J) {
    const int M = N >> (J - 1), Rh = (M / C) >> 1;
    total += Rh * (M >> 1);
  } else {
    total += C * C;
  }
  return total;
}

// Shared-memory layout of the staged gather tables of one analysis CTA
// (bytes from the stage base, 16-byte aligned): an image copied verbatim from
// the plan (per dense sensor N column and R0 row tap records, the latter with
// their window start in the staged v rows; the CTA's pupil-edge weights; the
// sensors' nc; the v run prefix and sources; each sensor's edge slot when its
// corner field takes the elongation correction, else -1; the pupil-edge entry
// slots; per node of the CTA (R0 N of them, then one more) the index of its
// first pupil-edge entry, 16-bit), then the corner rows of v the CTA reads.
struct StageLayout {
  int xr, yr, tw, mnc, vpre, vsrc, mslot, tk, eb, image, vs, total;
};
TOMO_HD inline StageLayout stage_layout(int n_dense, int N, int R0, int rec_stride, int esz, int max_entries,
                                        int vstage) {
  StageLayout L;
  L.xr = 0;
  L.yr = L.xr + n_dense * N * rec_stride * esz;
  L.tw = L.yr + n_dense * R0 * rec_stride * esz;
  L.mnc = (L.tw + 2 * max_entries * esz + 3) / 4 * 4;
  L.vpre = L.mnc + 4 * n_dense;
  L.vsrc = L.vpre + 4 * (n_dense + 1);
  L.mslot = L.vsrc + 4 * n_dense;
  L.tk = L.mslot + 4 * n_dense;
  L.eb = L.tk + 4 * max_entries;
  L.image = (L.eb + 2 * (R0 * N + 1) + 15) / 16 * 16;
  L.vs = L.image;
  L.total = L.vs + vstage * esz;
  return L;
}

// Shared-memory layout of the separate gather kernel (bytes, 16-byte aligned):
// the band buffer of R0 x N nodes, the band's row records (first corner row,
// KT weights per node row), the column-summed corner rows of one sensor (the
// plan's largest band needs `cells` elements there), then, when the kernel
// stages the corner rows it reads, `vcells` elements for one sensor's band
// rows of v.
struct GatherSmem {
  int ry, rw, u, v, total;
};
TOMO_HD inline GatherSmem gather_smem_layout(int R0, int N, int KT, int esz, long long cells, long long vcells,
                                             bool vstage) {
  GatherSmem g;
  g.ry = (R0 * N * esz + 15) / 16 * 16;
  g.rw = g.ry + (4 * R0 + 15) / 16 * 16;
  g.u = g.rw + (R0 * KT * esz + 15) / 16 * 16;
  g.v = g.u + static_cast<int>((cells * esz + 15) / 16 * 16);
  g.total = g.v + (vstage ? static_cast<int>((vcells * esz + 15) / 16 * 16) : 0);
  return g;
}
// Shared memory up to which the gather kernel stages the corner rows (two CTAs
// per SM keep fitting).
constexpr int kGatherStageSmem = 104 * 1024;

// Work items.
struct ClusterItem { int inst, layer; };
// One CTA of a streamed transform: a tile of kPassRows half-rows from row0 (a
// pass), or a whole layer's coarse levels (row0 unused); slot: its partial pair.
struct PassItem { int inst, layer, row0, slot; };

// The work of a streamed transform over one launch: pass items per level
// (items[off[k] .. off[k] + cnt[k]) for level k = 1..kmax), then one coarse
// item per layer; dynamic shared memory of the passes and of the coarse kernel.
struct StreamSet {
  const PassItem *items = nullptr;
  int off[kMaxLevels + 1] = {0}, cnt[kMaxLevels + 1] = {0};
  int kmax = 0;
  const PassItem *coarse = nullptr;
  int n_coarse = 0;
  size_t smem_pass = 0, smem_coarse = 0;
};

// Shared memory of a streamed pass at block side M (elements of T): the analysis
// stages 2 kPassRows + LF - 2 input rows and their row transforms; the synthesis
// 2 (kPassRows + LF/2 - 1) coefficient rows and their row syntheses.
TOMO_HD inline int pass_smem_elems(int M, int LF) {
  const int a = 2 * (2 * kPassRows + LF - 2) * M;
  const int s = 4 * (kPassRows + LF / 2 - 1) * M;
  return a > s ? a : s;
}
struct FwdItem { int inst, wfs, a0, b0, tile, pad0, pad1, pad2; };  // a0 < 0: tip/tilt-only sensor
struct UpdItem { int inst, start, blk, chunks; };   // chunks: passes of kUpdChunk coefficients

}  // namespace tomo
