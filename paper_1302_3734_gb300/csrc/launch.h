// Launchers of the CUDA kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.h"

namespace tomo {

constexpr int kMaxTransformSmem = 220 * 1024;   // opt-in dynamic shared memory of the transforms
constexpr int kMaxForwardSmem = 150 * 1024;     // staged corner tables of the forward kernel
constexpr size_t kTwoPerSmSmem = 108 * 1024;   // dynamic shared memory that lets two CTAs share an SM

// Dynamic shared memory of k_forward for `n_layers` layers.
size_t forward_smem(int n_layers, int precision);

// Raise the dynamic shared memory and cluster-size limits of every kernel once
// per device (before any launch, and before any stream capture).
cudaError_t configure_kernels();

// W^-1 over clusters of C CTAs per (instance, layer).  src: 0 = io.in0
// coefficients, 1 = PCG direction update fused in (flags: kFlagFirst).
cudaError_t launch_synthesis(int precision, int src, int lf, int flags, const InstDev *insts,
                             const ClusterItem *items, int n_clusters, int C, size_t smem,
                             const IoArgs &io, cudaStream_t s);

// W over clusters; src 0 = io.in0 layers, 1 = adjoint gather from v; epi 0 plain,
// 1 operator (q, p.q -> alpha), 2 residual (r, p, r.z); flags: kFlagWarm.
cudaError_t launch_analysis(int precision, int src, int epi, int lf, int flags, const InstDev *insts,
                            const ClusterItem *items, int n_clusters, int C, size_t smem,
                            const IoArgs &io, cudaStream_t s);
// The separate gather kernel alone (g = sum_m P_m^T v_m into the plan's phi),
// for plans whose gather tables are not staged; launch_analysis with src 2 then
// transforms its output.  tt_mode: 0 operator, 1 warm residual, 2 data only.
// items: one per CTA, {instance, layer, band (row0)}; C: bands per layer;
// vstage: the plans stage the band rows of v in shared memory.
cudaError_t launch_gather(int precision, int tt_mode, const InstDev *insts, const PassItem *items, int n_items,
                          int C, int vstage, size_t smem_gather, const IoArgs &io, cudaStream_t s);

// Streamed transforms (plans with stream_tf): the synthesis launches the coarse
// kernel, then the passes from the coarsest streamed level down to level 1; the
// analysis the passes from level 1 up, then the coarse kernel.  src as in
// launch_synthesis / launch_analysis (the analysis: 0 = io.in0 layers, 2 = the
// gathered grids in phi); streamed_launches: kernels one such call launches.
cudaError_t launch_synthesis_streamed(int precision, int src, int lf, int flags, const InstDev *insts,
                                      const StreamSet &S, const IoArgs &io, cudaStream_t s);
cudaError_t launch_analysis_streamed(int precision, int src, int epi, int lf, int flags, const InstDev *insts,
                                     const StreamSet &S, const IoArgs &io, cudaStream_t s);
int streamed_launches(const StreamSet &S);
cudaError_t configure_streamed_kernels();
// Shared-memory attribute of the separate gather kernel.
cudaError_t configure_gather_kernels();

// Ray-trace, Fried slopes, noise weighting, Gamma^T.  mode 0 operator, 1 residual,
// 2 data only.  elong: some sensor of the launch has elongated spots.
cudaError_t launch_forward(int precision, int mode, int max_layers, int elong, const InstDev *insts,
                           const FwdItem *items, int n_items, const IoArgs &io, cudaStream_t s);

// x, r update and the FP64 r.z partials; flags carries the iteration index.
cudaError_t launch_update(int precision, int flags, const InstDev *insts, const UpdItem *items,
                          int n_items, const IoArgs &io, cudaStream_t s);

// Noise-free measurement (single instance).
cudaError_t launch_slopes(int precision, const InstDev *insts, int n_wfs, int max_sub2,
                          const IoArgs &io, cudaStream_t s);

// Exact modified Jacobi diagonal (single instance): diag(sum_LGS A~^T C~^-1 A~)
// + alpha D into jdiag (alpha < 0: the plan's alpha), and its inverse into jinv
// unless jinv is NULL.  prof,
// prof_off, pos_fd: the plan's basis profiles and FP64 corner fractions.
cudaError_t launch_jacobi(const InstDev *insts, int n, const double *prof, const int *prof_off,
                          const double *pos_fd, double *jdiag, void *jinv, int precision,
                          int nc_max, double alpha, cudaStream_t s);

}  // namespace tomo
