// Host-side launchers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "bhac_device.cuh"

namespace bhac {

// Largest dynamic shared memory a stage kernel may request (bytes): the
// opt-in per-CTA limit of sm_103a (227 KB) less room for the kernels' static
// shared memory (the attribute plus the static size must fit the limit).
constexpr int kMaxDynSmem = 226 * 1024;
// dynamic shared memory per CTA that still lets two CTAs share an SM (228 KB
// per SM, 1 KB of it reserved per resident CTA)
constexpr int kTwoCtaSmem = 113 * 1024;

// stage kernels (stage_fp64.cu / stage_mixed.cu)
cudaError_t launch_stage_fp64(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_stage_mixed(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_cfl(const StageArgs& a, cudaStream_t st);
// resident CTAs per SM of the phased 3-D stage kernel these arguments select
int stage_occupancy_fp64(const StageArgs& a, int threads, size_t smem);
int stage_occupancy_mixed(const StageArgs& a, int threads, size_t smem);
// one pass that loads interior primitives into the ghosted arrays, sets the
// conserved state and reduces the CFL rate into a.smax_out
cudaError_t launch_load(const StageArgs& a, const double* src, double* P, float* P32, double* U, cudaStream_t st);
// split form: the cell kernel over a range of items, and the reflux pass
cudaError_t launch_cells_fp64(const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_cells_mixed(const StageArgs& a, int grid, cudaStream_t st);
cudaError_t launch_reflux_fp64(const StageArgs& a, cudaStream_t st);
cudaError_t launch_reflux_mixed(const StageArgs& a, cudaStream_t st);
// set kernel attributes ahead of a stream capture
cudaError_t prepare_stage_fp64();
cudaError_t prepare_stage_mixed();

// IMEX first stage (imex.cu): psi of the interior primitives (FP64 and, in the
// mixed form, FP32) scaled by 1 / (1 + gamma alpha kappa dt)
cudaError_t launch_imex_first_stage(const StageArgs& a, double* P, float* P32, cudaStream_t st);

// auxiliary kernels (aux.cu)
struct GhostArgs {
  const int* src;               // per (block, slot): source ghosted-cell index over all blocks,
                                // or -(node + 1) for a cross-level value
  const unsigned char* flags;   // per (block, slot): bit0 flip theta, bits 1+2d / 2+2d clamp u^d <= 0 / >= 0
  const int* tmpl;              // per slot: destination cell index inside a block
  int nslots, nblocks, ncell;
  double* P;                    // FP64 ghosted primitives (or null)
  float* P32;                   // FP32 ghosted primitives (or null)
  const double* node64;         // cross-level node values (FP64 form)
  const float* node32;          // cross-level node values (mixed form)
  unsigned int* work_reset;     // zeroed by the first thread (persistent work counter)
  unsigned long long* smax_reset;  // zeroed by the first thread when non-null
};
cudaError_t launch_ghost_fill(const GhostArgs& g, cudaStream_t st);

struct MetricArgs {
  int coords;                   // 1 KS, 2 MKS
  double spin, mass;
  double x1min, x2min, dx1, dx2;
  int N1, N2;                   // cells along x1, x2
  int axis_lo, axis_hi;         // polar axis at x2 = low / high boundary
  double rho_floor, rho_pow, p_floor, p_pow;
  double* tab_c;                // N2 x N1 x CREC
  double* tab_f1;               // N2 x (N1+1) x FREC
  double* tab_f2;               // (N2+1) x N1 x FREC
  float* tab_c32;
  float* tab_f1_32;
  float* tab_f2_32;
};
cudaError_t launch_metric_tables(const MetricArgs& m, cudaStream_t st);

// interior <-> ghosted copies and the conserved state of loaded primitives
cudaError_t launch_gather_interior(const StageArgs& a, const double* P, double* dst, cudaStream_t st);
cudaError_t launch_init_cons(const StageArgs& a, const double* P, double* U, cudaStream_t st);

}  // namespace bhac
