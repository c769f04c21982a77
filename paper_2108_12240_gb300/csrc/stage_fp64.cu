// FP64 instantiations of the stage kernel and the stand-alone CFL kernel.
#include "stage_impl.cuh"

namespace bhac {

cudaError_t launch_stage_fp64(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  return launch_stage_any<double>(a, grid, threads, smem, st);
}

cudaError_t prepare_stage_fp64() { return configure_all_t<double>(); }

cudaError_t launch_cells_fp64(const StageArgs& a, int grid, cudaStream_t st) { return launch_cells_any<double>(a, grid, st); }
cudaError_t launch_reflux_fp64(const StageArgs& a, cudaStream_t st) { return launch_reflux_any<double>(a, st); }

// grid for the per-cell reduction kernels: about eight CTAs per SM, so that
// each thread takes many cells and the warps' atomicMax on the one rate word
// stay few (one per 32 cells would be a million on the large torus, serialised
// at L2)
static int cell_grid(const StageArgs& a) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long n = (long long)a.nblocks * a.nint;
  long long g = (n + 255) / 256;
  if (g > 8LL * nsm) g = 8LL * nsm;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_cfl(const StageArgs& a, cudaStream_t st) {
  const int grid = cell_grid(a);
  if (a.ndim == 3) {
    if (a.flat) cfl_kernel<3, true><<<grid, 256, 0, st>>>(a);
    else cfl_kernel<3, false><<<grid, 256, 0, st>>>(a);
  } else {
    if (a.flat) cfl_kernel<2, true><<<grid, 256, 0, st>>>(a);
    else cfl_kernel<2, false><<<grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_load(const StageArgs& a, const double* src, double* P, float* P32, double* U, cudaStream_t st) {
  const int grid = cell_grid(a);
  if (a.ndim == 3) {
    if (a.flat) load_kernel<3, true><<<grid, 256, 0, st>>>(a, src, P, P32, U);
    else load_kernel<3, false><<<grid, 256, 0, st>>>(a, src, P, P32, U);
  } else {
    if (a.flat) load_kernel<2, true><<<grid, 256, 0, st>>>(a, src, P, P32, U);
    else load_kernel<2, false><<<grid, 256, 0, st>>>(a, src, P, P32, U);
  }
  return cudaGetLastError();
}

int stage_occupancy_fp64(const StageArgs& a, int threads, size_t smem) {
  return stage_occupancy_any<double>(a, threads, smem);
}

}  // namespace bhac
