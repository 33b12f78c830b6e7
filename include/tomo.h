/*
 * tomo.h - C ABI of the GB300 wavelet-domain MAP tomography solver.
 *
 * The library solves, for one or many adaptive-optics systems, the normal
 * equations of the MAP atmospheric-tomography problem in a wavelet basis
 * (Helin & Yudytskiy, "Wavelet methods in multi-conjugate adaptive optics",
 * Sec. 5.1, eq. eqn_lse):
 *
 *     (A~^T C^-1 A~ + alpha D) c = A~^T C^-1 s,      A~ = Gamma P W^-1,
 *
 * with W the per-layer periodic orthonormal Daubechies transform (Sec. 5.1),
 * P the guide-star ray-trace with the laser-guide-star cone effect (Sec. 2.1,
 * eq. ngsproj and the LGS projection), Gamma the Fried-geometry Shack-Hartmann
 * slope operator (eqs. SH_eq / SH_op), C the block-diagonal noise covariance
 * with LGS tip/tilt removal (Sec. 4.3, eqs. removing_tt / widehatc) and D the
 * diagonal wavelet-domain von Karman prior (Sec. 3).  The system is solved by
 * CG or by PCG with the modified Jacobi preconditioner of Sec. 5.1, for a fixed
 * number of iterations, warm-started from the previous frame.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All device pointers are CUDA device memory owned by the caller; the
 *   library never frees them.  Host pointers are read during the call only.
 * - Element type of every device array: float when the geometry's
 *   precision == 0, double when precision == 1 (tomo_jacobi_diagonal always
 *   writes double).
 * - Layer grids: layers concatenated in declaration order, each N_l x N_l,
 *   row-major with the row index = y; node (ix, iy) sits at
 *   ((ix - N/2) dx, (iy - N/2) dx) in metres; grids are periodic.
 * - Coefficients: layers concatenated, each N_l x N_l in the Mallat pyramid
 *   layout of the periodic 2-D DWT (rows = x transformed first, then columns):
 *   level k occupies the top-left block of side N/2^(k-1); its quadrants are
 *   [low-low (next level), high-x; high-y, high-high].
 * - Slopes: sensors concatenated in declaration order; a full sensor gives
 *   [sx of each valid subaperture, then sy], valid subapertures in row-major
 *   order (row = y index); a tip/tilt-only sensor gives [mean sx, mean sy].
 *   Slopes are phase differences across one subaperture (rad).
 * - Every call enqueues its work on `cuda_stream` (a cudaStream_t, NULL = the
 *   legacy default stream) and returns without waiting, unless stated.
 * - Errors: a non-zero tomo_status; tomo_last_error() gives a message
 *   (thread-local).  No C++ exception crosses this boundary.  A plan is not
 *   thread-safe: do not use one plan from two threads at once.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tomo_plan tomo_plan;     /* opaque; created and owned by the library */

typedef enum {
  TOMO_OK = 0,
  TOMO_ERR_ARG = 1,          /* a NULL pointer, a size or a flag out of range */
  TOMO_ERR_GEOMETRY = 2,     /* a footprint wider than its layer grid, no valid subaperture, ... */
  TOMO_ERR_LEVELS = 3,       /* N/2^(levels-1) < filter length, or N not a power of two */
  TOMO_ERR_NOMEM = 4,        /* device or host allocation failed */
  TOMO_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the CUDA error) */
  TOMO_ERR_TIMEOUT = 6,      /* reserved for waits with a deadline */
  TOMO_ERR_BREAKDOWN = 7,    /* p.Ap <= 0 or not finite during (P)CG: iterate frozen */
  TOMO_ERR_UNSUPPORTED = 8,  /* valid request the library does not implement (sizes beyond its tables) */
  TOMO_ERR_FULL = 9,         /* a bounded queue is full (served frames of one telescope) */
  TOMO_ERR_SUPERSEDED = 10   /* a served frame skipped because a newer one of its telescope
                                was waiting (latest-frame policy) */
} tomo_status;

/* One wavefront sensor (Sec. 2.1, Sec. 4.3). */
typedef struct {
  double theta_x, theta_y;     /* guide-star direction (rad) */
  double height;               /* laser guide star altitude H (m); INFINITY or <= 0: natural star */
  int n_sub;                   /* subapertures per side (>= 1) */
  double d_sub;                /* subaperture side (m, > 0) */
  const unsigned char *valid;  /* host, n_sub*n_sub, row = y; nonzero = valid.  NULL: the circular
                                  pupil rule (centre radius within [obstruction*D/2, D/2]) */
  double sigma;                /* noise standard deviation per slope (rad, > 0) */
  int tt_only;                 /* 1: the sensor reports only the two mean slopes (tip/tilt NGS) */
  int remove_tt;               /* 1: tip/tilt removal, C^-1 -> (I-T) C_tilde^-1 (I-T) (LGS) */
  /* Spot elongation of a laser guide star (Sec. 4.3, eq. elongation_matrix): each
   * subaperture's noise block is sigma^2 (I + tau g g^T) with g = elong_scale * (r - llt),
   * r the subaperture centre and llt the laser launch point (pupil coordinates, m), g in
   * units of the spot FWHM.  elong_tau <= 0 (or a natural star): sigma^2 I.  The modified
   * Jacobi diagonal keeps sigma^-2 I blocks (it is only the preconditioner). */
  double elong_tau;            /* tau, 0..1 */
  double elong_scale;          /* |g| per metre of distance from the launch point (1/m) */
  double llt_x, llt_y;         /* launch point (m) */
} tomo_wfs;

/* One turbulence layer (Sec. 2.1 layered model, Sec. 3 prior). */
typedef struct {
  double altitude;             /* h_l (m, >= 0) */
  double dx;                   /* grid spacing (m, > 0) */
  int N;                       /* grid side, a power of two >= 16 */
  double prior_weight;         /* 1/c_rho(h_l) of D_l (> 0) */
} tomo_layer;

typedef struct {
  double D_tel;                /* pupil diameter (m); used by the NULL-mask rule */
  double obstruction;          /* central obstruction as a radius ratio in [0, 1) */
  int n_wfs;
  const tomo_wfs *wfs;         /* host array of n_wfs */
  int n_layers;
  const tomo_layer *layers;    /* host array of n_layers */
  int wavelet_order;           /* Daubechies vanishing moments p, 1..4 (filter length 2p; 3 = paper) */
  int levels;                  /* DWT levels J >= 1 */
  double alpha;                /* regularisation weight of D (>= 0) */
  double L0;                   /* outer scale (m); <= 0 drops the L0^(-11/3) term of D */
  int precond;                 /* 0: CG, 1: modified Jacobi PCG (Sec. 5.1) */
  int precision;               /* 0: FP32 operator with FP64 dot products and scalars; 1: FP64 */
} tomo_geometry;

typedef struct {
  long long n_coeffs;          /* unknowns = sum of N_l^2 (= layer-grid elements) */
  long long n_slopes;          /* elements of the slope vector */
  int n_layers, n_wfs;
  int cluster_size;            /* CTAs per layer in the transform kernels */
  int kernels_per_iteration;   /* kernel launches per PCG iteration */
  int kernels_per_solve_base;  /* launches per solve besides the iterations (warm start) */
  long long device_bytes;      /* device memory held by the plan */
  long long bytes_per_iteration; /* algorithmic bytes of one PCG iteration: (15 n + 2 V) elements,
                                    13 n + 2 V without the preconditioner (n coefficients,
                                    V corner values of the sensors that are not tip/tilt-only,
                                    (n_sub + 1)^2 each) */
  int precision;
  int breakdown_pending;       /* 1: a solve of the plan broke down and no call has reported it yet */
  int gather_separate;         /* 1: the transposed ray-trace runs in its own kernel before the analysis */
  int streamed;                /* 1: streamed transforms (tomo_plan_options.transforms) */
} tomo_plan_info;

/* Launch shape of a plan (zero-initialise; every field 0 means the default). */
typedef struct {
  int cluster_size;            /* CTAs per layer in the transform kernels (one thread-block cluster
                                  per layer): 0 = min(16, N_min/8); else a power of two in
                                  [1, min(16, N_min/2)].  Large clusters give the lowest latency of
                                  one solve, small ones the most solves per second in big batches.
                                  Streamed plans (transforms 2) use it only as the number of row
                                  bands of the separate gather kernel, a power of two in
                                  [1, min(64, N_min/2)] */
  int transforms;              /* 0: chosen by the plan; 1: one thread-block cluster per layer and
                                  transform; 2: streamed, level by level over row tiles of every
                                  layer with no cluster (the default when a layer's cluster CTAs
                                  could not share an SM, e.g. 512^2 layers) */
  int reserved[6];             /* must be 0 */
} tomo_plan_options;

/* Build a plan: validates `g`, copies every host input, builds the index
 * tables, the prior D and the Jacobi diagonal (Sec. 5.1, computed exactly on
 * the device), and allocates the workspace.  Synchronises `cuda_stream`.
 * On success *out owns device memory until tomo_destroy. */
tomo_status tomo_plan_create(const tomo_geometry *g, void *cuda_stream, tomo_plan **out);

/* tomo_plan_create with launch options (NULL: the defaults).  TOMO_ERR_ARG for a
 * cluster size that is not allowed; TOMO_ERR_UNSUPPORTED when the layer grids do
 * not fit one CTA's shared memory at that cluster size. */
tomo_status tomo_plan_create_ex(const tomo_geometry *g, const tomo_plan_options *opt,
                                void *cuda_stream, tomo_plan **out);

/* One frame (Sec. 5.1): b = A~^T C^-1 s from d_slopes, r0 = b - (A~^T C^-1 A~ + alpha D) x0,
 * then exactly `iters` (P)CG iterations (Hestenes-Stiefel).
 * d_slopes: n_slopes elements (read).  d_coeffs: n_coeffs elements; read as x0 when
 * warm != 0 (warm restart: the previous frame's solution), ignored otherwise (x0 = 0);
 * overwritten with x.  out_resnorm: host, may be NULL; when given the call waits for
 * the stream and stores ||r|| (2-norm of the final recurrence residual), and a
 * breakdown of this solve returns TOMO_ERR_BREAKDOWN.
 * Breakdown (p.Ap <= 0 or a non-finite value, e.g. NaN slopes): the iterate is
 * frozen (x keeps its last finite value, x0 for a breakdown in the first
 * iteration) and the update kernel sets the plan's breakdown word, a mapped host
 * word that never costs a synchronisation.  Without out_resnorm the breakdown is
 * reported by the first later tomo_solve or tomo_solve_batch of the plan that is
 * called after that solve's work has completed on the device: that call returns
 * TOMO_ERR_BREAKDOWN, clears the word and enqueues nothing (call it again).
 * tomo_plan_get_info shows the word without clearing it. */
tomo_status tomo_solve(tomo_plan *p, const void *d_slopes, void *d_coeffs, int iters,
                       int warm, void *cuda_stream, double *out_resnorm);

/* `count` independent frames of `count` distinct plans that share precision and
 * precond, solved together: every phase of the iteration is one launch for all
 * of them.  plans/d_slopes/d_coeffs: host arrays of `count`; same per-plan
 * semantics as tomo_solve.  When an earlier solve of any of the plans has broken
 * down (its breakdown word is set), the call clears every set word, returns
 * TOMO_ERR_BREAKDOWN and enqueues nothing. */
tomo_status tomo_solve_batch(tomo_plan *const *plans, const void *const *d_slopes,
                             void *const *d_coeffs, int count, int iters, int warm,
                             void *cuda_stream);

/* W^-1 (synthesis): d_coeffs (n_coeffs) -> d_layers (n_coeffs).  Sec. 5.1. */
tomo_status tomo_coeffs_to_layers(tomo_plan *p, const void *d_coeffs, void *d_layers,
                                  void *cuda_stream);

/* W (analysis): d_layers (n_coeffs) -> d_coeffs (n_coeffs). */
tomo_status tomo_layers_to_coeffs(tomo_plan *p, const void *d_layers, void *d_coeffs,
                                  void *cuda_stream);

/* Noise-free measurement A phi (eq. atm_tomo): d_layers (n_coeffs) -> d_slopes (n_slopes). */
tomo_status tomo_layers_to_slopes(tomo_plan *p, const void *d_layers, void *d_slopes,
                                  void *cuda_stream);

/* Normal operator of eq. eqn_lse: d_out = (A~^T C^-1 A~ + alpha D) d_in (n_coeffs each).
 * d_in and d_out must not overlap. */
tomo_status tomo_apply_normal(tomo_plan *p, const void *d_in, void *d_out, void *cuda_stream);

/* Right-hand side of eq. eqn_lse: d_out = A~^T C^-1 d_slopes (n_coeffs). */
tomo_status tomo_rhs(tomo_plan *p, const void *d_slopes, void *d_out, void *cuda_stream);

/* The modified Jacobi diagonal J (Sec. 5.1, including alpha D): n_coeffs doubles. */
tomo_status tomo_jacobi_diagonal(tomo_plan *p, double *d_out, void *cuda_stream);

/* The modified Jacobi diagonal for regularisation weight `alpha`
 * (diag(sum over LGS of A~^T C~^-1 A~) + alpha D, n_coeffs doubles into d_out),
 * recomputed without allocating any device memory.  The paper has no
 * counterpart: this is a service for callers that cannot allocate when they
 * need the diagonal again, e.g. a real-time control thread retuning alpha,
 * which must not take the latency of cudaMalloc, or code living inside
 * another framework's memory pool.  The computation's scratch (basis
 * profiles and corner fractions of the plan) lives in a fixed 4 MiB device
 * array owned by the library; every GPU that loads the library holds it until
 * the process exits.  A plan needing more scratch than that is rejected with
 * TOMO_ERR_UNSUPPORTED and a message giving both sizes.  The first call on a
 * device looks up the array's device address; make that first call before
 * any stream capture.  Every call overwrites the whole scratch it reads (none
 * of it must start at zero), and all calls share it: calls that overlap on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  The plan itself is not modified.  Enqueued on
 * `cuda_stream`; the work reads the plan's host-side tables, so keep the plan
 * alive until that work has completed on the stream. */
tomo_status tomo_jacobi_diagonal_noalloc(const tomo_plan *p, double alpha, double *d_out,
                                         void *cuda_stream);

/* Sizes and launch facts of a plan. */
tomo_status tomo_plan_get_info(const tomo_plan *p, tomo_plan_info *out);

/* Device memory held by the plan (bytes; 0 for NULL), for admission by memory. */
size_t tomo_plan_device_bytes(const tomo_plan *p);

/* Per-kernel timing: when enabled, every launch of the plan is bracketed by CUDA
 * events; tomo_get_kernel_times returns, per kernel kind, the number of timed
 * launches and their summed milliseconds since the last reset (waits for the
 * stream).  Kinds: 0 transform-synthesis, 1 ray-trace/slopes, 2 adjoint+analysis
 * (the transform alone for plans whose gather runs separately), 3 vector update,
 * 4 other, 5 the separate gather kernel.  n_kinds = 6.  While timing is enabled on
 * the first plan of a tomo_solve_batch call, the batch's kernels are launched
 * directly (no graph) and timed on that plan. */
tomo_status tomo_set_kernel_timing(tomo_plan *p, int enable);
tomo_status tomo_get_kernel_times(tomo_plan *p, int *counts, double *ms, int n_kinds);

/* Launch mode of tomo_solve: 1 (default) captures each distinct (slopes, coeffs,
 * iters, warm) call once into a CUDA graph and replays it; 0 launches every
 * kernel directly (one launch per kernel per call, no graph). */
tomo_status tomo_set_launch_mode(tomo_plan *p, int use_graphs);

/* ------------------------------------------------------------------ fitting
 * The fitting step (Sec. 4.1, eqs. fit_step_ideal / fit_step_min): mirror
 * commands a minimising sum_j || H_j a - P_j phi ||^2 over directions theta_j,
 * solved by CG (Hestenes-Stiefel, no preconditioner) on the normal equations
 * H^T H a = H^T P phi for a fixed number of iterations, optionally from the
 * previous commands.
 *
 * - Mirror k is a square grid of n x n actuators with spacing `pitch`,
 *   conjugated to `altitude`.  Actuator (i, j) (column i = x, row j = y) sits
 *   at ((i - (n-1)/2) pitch, (j - (n-1)/2) pitch) and the mirror's shape is
 *   the piecewise-bilinear interpolation of its commands, zero beyond the
 *   outermost actuators.  H_j a (x) = sum_k a_k(x + altitude_k theta_j).
 * - The aperture is sampled at the corners of the valid subapertures of an
 *   n_sub x n_sub grid of spacing d_sub: corner (a, b) at
 *   ((a - n_sub/2) d_sub, (b - n_sub/2) d_sub), each with weight 1.
 * - P_j is the natural-guide-star ray-trace (eq. ngsproj) through the plan's
 *   layers: sum_l phi_l(x + h_l theta_j), bilinear on the periodic grids.
 * - Command vectors: the mirrors concatenated, each n x n row-major (row = y),
 *   of the plan's element type.
 * A fit refers to its plan, which must outlive it; like a plan, a fit is not
 * thread-safe.  Every call enqueues on `cuda_stream` and returns. */
typedef struct tomo_fit tomo_fit;

typedef struct {
  double altitude;             /* m, >= 0 */
  double pitch;                /* actuator spacing (m), 0 < pitch <= 4 d_sub */
  int n;                       /* actuators per side, 2..4096 */
} tomo_dm;

typedef struct {
  int n_dm;                    /* 1..4 */
  const tomo_dm *dms;          /* host array of n_dm */
  int n_dir;                   /* evaluation directions, 1..256 */
  const double *theta;         /* host [n_dir][2]: (theta_x, theta_y) in rad */
  int n_sub;                   /* aperture sampling grid, 1..1024 subapertures per side */
  double d_sub;                /* m, > 0 */
  const unsigned char *valid;  /* host, n_sub*n_sub, row = y; nonzero = valid (not NULL) */
} tomo_fit_geometry;

typedef struct {
  long long n_act;             /* elements of a command vector (sum of n^2) */
  long long n_active;          /* actuators whose support reaches a sampling point in some
                                  direction (nonzero diagonal of H^T H) */
  int n_points;                /* sampling points (corners of valid subapertures) */
  int n_dir, n_dm;
  int kernels_per_iteration;   /* launches per CG iteration */
  int kernels_per_solve_base;  /* launches per tomo_fit_solve besides the iterations */
  long long device_bytes;      /* device memory held by the fit */
  long long normal_nonzeros;   /* stored entries of H^T H */
  long long bytes_per_iteration; /* algorithmic bytes of one CG iteration: H^T H (entries and
                                    column indices, row descriptors) and the vectors r, q, p, a */
} tomo_fit_info;

/* Build a fit for plan p: validates g, builds the tap tables of H, H^T, P and
 * of the mirrors as the plan's sensors see them (A_hat, below), assembles
 * H^T H as a sparse matrix (all in FP64 on the host, stored in the plan's
 * element type) and allocates the workspace.  Synchronises the device.  On
 * success *out owns device memory until tomo_fit_destroy.  TOMO_ERR_ARG: an
 * argument out of the ranges above; TOMO_ERR_GEOMETRY: no valid subaperture;
 * TOMO_ERR_UNSUPPORTED: an actuator's window of sampling corners longer than 8
 * or than the sampling grid. */
tomo_status tomo_fit_create(tomo_plan *p, const tomo_fit_geometry *g, tomo_fit **out);

tomo_status tomo_fit_get_info(const tomo_fit *f, tomo_fit_info *out);

/* d_out = H^T H d_a (both n_act elements, device). */
tomo_status tomo_fit_apply_normal(tomo_fit *f, const void *d_a, void *d_out, void *cuda_stream);

/* d_out = H^T P phi, phi the plan's layer grids in d_layers (device). */
tomo_status tomo_fit_rhs(tomo_fit *f, const void *d_layers, void *d_out, void *cuda_stream);

/* Quality of a correction (Sec. 5.1): d_rms[j] (device, n_dir doubles) = the
 * root mean square over the sampling points of P_j phi - H_j a after removing
 * its mean, for the layers d_layers (e.g. the true atmosphere) and commands d_a
 * (NULL: no correction).  The Marechal approximation of the Strehl ratio at
 * wavelength lambda is exp(-(2 pi r / lambda)^2), r in the layers' units. */
tomo_status tomo_fit_residual_rms(tomo_fit *f, const void *d_layers, const void *d_a, double *d_rms,
                                  void *cuda_stream);

/* `iters` CG iterations on H^T H a = H^T P phi; d_a holds the starting
 * commands when warm != 0 (ignored otherwise: the start is 0) and receives the
 * result.  A p.Hp <= 0 with a nonzero residual freezes the iterate. */
tomo_status tomo_fit_solve(tomo_fit *f, const void *d_layers, void *d_a, int iters, int warm,
                           void *cuda_stream);

/* The reconstruction of one frame, slopes to mirror commands: tomo_solve of
 * the fit's plan (d_coeffs in/out, `iters` iterations), phi = W^-1 c into the
 * fit's own layer buffer, then tomo_fit_solve (d_a in/out, `fit_iters`
 * iterations); `warm` applies to both.  Replayed from one CUDA graph per
 * argument set. */
tomo_status tomo_reconstruct(tomo_fit *f, const void *d_slopes, void *d_coeffs, void *d_a, int iters,
                             int fit_iters, int warm, void *cuda_stream);

/* ------------------------------------------------------------------ closed loop
 * Pseudo-open-loop control (Sec. 4.2, Algorithm 4.1) with a delay of two
 * frames: the data s measured while the commands a_{t-2} were applied give
 *   step 1: s_ol = s + A_hat a_{t-2},
 *   step 2: Delta a = R s_ol - a_{t-2},
 *   step 3: a_t = a_{t-1} + gain Delta a,
 * with R the reconstruction of tomo_reconstruct.  A_hat maps commands to the
 * plan's slope layout: each mirror acts on the guide-star light like a layer
 * at its altitude (sensor m sees sum_k a_k((1 - h_k/H_m) r + theta_m h_k) on
 * its corners; cone factor 1 for a natural star), measured like layers are
 * (Fried slopes; the two means for a tip/tilt-only sensor). */

/* d_out = d_in + scale * A_hat d_a (d_in NULL: 0; d_in may equal d_out). */
tomo_status tomo_mirror_slopes(tomo_fit *f, const void *d_a, const void *d_in, void *d_out, double scale,
                               void *cuda_stream);

/* One control step from the residual slopes d_slopes: steps 1 to 3 above.
 * d_coeffs (tomography coefficients) and d_a_rec (R s_ol, the reconstructed
 * commands) hold the previous frame's values when warm != 0 and receive this
 * frame's; d_a_t receives a_t and may be the storage of d_a_tm2 (so two
 * command buffers can alternate); no other two of the command buffers may
 * share storage.  Replayed from one CUDA graph per argument set. */
tomo_status tomo_polc_step(tomo_fit *f, const void *d_slopes, void *d_coeffs, void *d_a_rec, const void *d_a_tm2,
                           const void *d_a_tm1, void *d_a_t, double gain, int iters, int fit_iters, int warm,
                           void *cuda_stream);

void tomo_fit_destroy(tomo_fit *f);

/* ------------------------------------------------------------------ serving
 * A request loop for a stream of slope frames from several telescopes, the
 * real-time setting of Sec. 5: every frame is one tomo_solve of its
 * telescope's plan, warm-started from that telescope's previous solution
 * (Sec. 5.1), and each telescope's frames are solved strictly in arrival
 * order.  The server owns the plans (admitted by device memory), one device
 * slot per telescope for the frame's slopes and the warm-start coefficients,
 * and two threads: a worker that launches, whenever a telescope with a
 * waiting frame is idle, one batched solve (tomo_solve_batch's kernels, from
 * a CUDA graph over all admitted plans with a per-launch mask of the
 * telescopes that have a frame) after the frames' host-to-device copies and
 * followed by the coefficients' device-to-host copies; and a completion
 * thread that timestamps finished frames.  Frames that arrive while others
 * are on the GPU go into the next launch, on the next of `max_in_flight`
 * streams, so launches overlap on the device.
 * Timestamps are seconds on the steady clock returned by tomo_server_clock(). */
typedef struct tomo_server tomo_server;

typedef struct {
  int telescope;               /* id from tomo_server_admit */
  int status;                  /* TOMO_OK; TOMO_ERR_BREAKDOWN when the frame's solve broke down (its
                                  iterate frozen, so the telescope's warm start stays finite);
                                  TOMO_ERR_SUPERSEDED; or the error of the launch that held it */
  long long tag;               /* the caller's tag from tomo_server_submit */
  double t_submit;             /* tomo_server_submit copied the frame in */
  double t_launch;             /* the launch holding the frame was enqueued */
  double t_done;               /* its result was in host memory */
  int batch_size;              /* frames in that launch */
  int result_slot;             /* where tomo_server_result finds the result */
} tomo_frame_result;

typedef struct {
  long long frames_submitted, frames_done, frames_superseded, launches;
  long long bytes_in_use;      /* plans + telescope slots + batch tables (device) */
  long long budget_bytes;
  int telescopes;              /* admitted */
  int in_flight;               /* launches on the device now */
} tomo_server_stats;

/* Create a server on the current device.  budget_bytes: device memory the
 * server may hold (0: no limit).  iters: PCG iterations per frame (>= 0).
 * max_in_flight: launches on the device at once (1..4).  queue_depth: frames
 * a telescope may have waiting before tomo_server_submit returns
 * TOMO_ERR_FULL (1..256).  result_slots: results kept per telescope for
 * tomo_server_result (1..256). */
tomo_status tomo_server_create(size_t budget_bytes, int iters, int max_in_flight, int queue_depth,
                               int result_slots, tomo_server **out);

/* Admit a telescope: builds its plan (as tomo_plan_create) and its slots if
 * they fit the budget, else TOMO_ERR_NOMEM and nothing is kept.  Waits until
 * no launch is in flight, then rebuilds the batch; frames of other telescopes
 * wait meanwhile.  *telescope: the new id (ids are never reused).  The first
 * frame starts from x0 = 0. */
tomo_status tomo_server_admit(tomo_server *s, const tomo_geometry *g, int *telescope);

/* tomo_server_admit with plan launch options (NULL: the defaults). */
tomo_status tomo_server_admit_ex(tomo_server *s, const tomo_geometry *g, const tomo_plan_options *opt,
                                 int *telescope);

/* Admit a telescope that the server runs in closed loop (Sec. 4.2, Algorithm
 * 4.1, two-frame delay): each submitted frame holds the residual slopes that
 * were measured while the commands returned two frames earlier were applied
 * (zero for the first two frames); the server runs one tomo_polc_step with
 * `gain` and `fit_iters` fitting iterations (its `iters` for the tomography),
 * and the frame's result is the commands a_t (the fit's command layout: n_act
 * elements of the plan's type).  The tomography coefficients and the
 * reconstructed commands are warm-started from the telescope's previous frame.
 * fit == NULL admits an open-loop telescope (tomo_server_admit_ex).  Frames of
 * closed-loop telescopes are not batched with others: each is its own control
 * step on the launch's stream.  Under the latest-frame policy a superseded
 * frame is also skipped by the integrator. */
tomo_status tomo_server_admit_loop(tomo_server *s, const tomo_geometry *g, const tomo_plan_options *opt,
                                   const tomo_fit_geometry *fit, double gain, int fit_iters, int *telescope);

/* Frame policy: 0 (default) solves every frame of a telescope in order; 1 solves
 * only the newest waiting frame when a launch is formed and reports the older
 * waiting ones as TOMO_ERR_SUPERSEDED (the real-time choice when the stream
 * outruns the solver: a stale frame's reconstruction is never applied). */
tomo_status tomo_server_set_policy(tomo_server *s, int latest_only);

/* Release a telescope and its memory (waits for its frame in flight; frames
 * still waiting are dropped and not reported). */
tomo_status tomo_server_release(tomo_server *s, int telescope);

/* Submit one frame: copies n_slopes elements (float, or double for precision 1
 * plans) from host memory and returns; `tag` comes back in the result.
 * TOMO_ERR_FULL: queue_depth frames of this telescope are already waiting. */
tomo_status tomo_server_submit(tomo_server *s, int telescope, const void *host_slopes, long long tag);

/* Up to `max` finished frames (oldest first) into out; returns how many. */
int tomo_server_poll(tomo_server *s, tomo_frame_result *out, int max);

/* Copy the result of a finished frame into host_out: the coefficients
 * (n_coeffs elements), or for a closed-loop telescope the commands a_t (n_act
 * elements of its fit).  TOMO_ERR_ARG if that slot already holds a later frame. */
tomo_status tomo_server_result(tomo_server *s, int telescope, int result_slot, long long tag,
                               void *host_out);

/* Wait until every submitted frame is finished (TOMO_ERR_TIMEOUT after
 * timeout_s seconds). */
tomo_status tomo_server_drain(tomo_server *s, double timeout_s);

tomo_status tomo_server_get_stats(tomo_server *s, tomo_server_stats *out);

/* The plan of an admitted telescope (owned by the server; for
 * tomo_plan_get_info and the operator calls, not for solves). */
tomo_status tomo_server_get_plan(tomo_server *s, int telescope, const tomo_plan **out);

/* The fit of a closed-loop telescope (NULL for an open-loop one), owned by the server. */
tomo_status tomo_server_get_fit(tomo_server *s, int telescope, const tomo_fit **out);

/* The steady clock of the frame timestamps (seconds). */
double tomo_server_clock(void);

/* Stop the threads, finish the frames in flight, release every plan.  NULL-safe. */
void tomo_server_destroy(tomo_server *s);

/* Measurement utility (the paper has no counterpart): the L2 read bandwidth in
 * GB/s of the current device, the denominator of the benchmark's L2 fractions.
 * d_buf: device buffer of `bytes` (16-byte aligned, small enough to stay in the
 * L2, e.g. 32 MiB), owned by the caller; its contents are read, not changed.
 * One untimed pass brings it into the L2, then `reps` launches each read it
 * `passes` times (CTAs rotate over the slices between passes, loads bypass
 * L1), timed by CUDA events on `cuda_stream`; waits for the stream. */
tomo_status tomo_probe_l2_read(void *d_buf, long long bytes, int passes, int reps, void *cuda_stream,
                               double *out_gbs);

/* Number of kernels this library has launched so far in this process. */
long long tomo_launch_count(void);

/* Thread-local message of the last failing call ("" if none). */
const char *tomo_last_error(void);

/* Release a plan and its device memory (waits for its work).  NULL-safe. */
void tomo_destroy(tomo_plan *p);

/* Library version string. */
const char *tomo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TOMO_H */
