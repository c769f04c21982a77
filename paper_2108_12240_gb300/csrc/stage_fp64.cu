// FP64 instantiations of the stage kernel and the stand-alone CFL kernel.
#include "stage_impl.cuh"

namespace bhac {

cudaError_t launch_stage_fp64(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  return launch_stage_any<double>(a, grid, threads, smem, st);
}

cudaError_t prepare_stage_fp64() { return configure_all_t<double>(); }

cudaError_t launch_cells_fp64(const StageArgs& a, int grid, cudaStream_t st) { return launch_cells_any<double>(a, grid, st); }
cudaError_t launch_reflux_fp64(const StageArgs& a, cudaStream_t st) { return launch_reflux_any<double>(a, st); }

cudaError_t launch_cfl(const StageArgs& a, cudaStream_t st) {
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long n = (long long)a.nblocks * a.nint;
  long long grid = (n + 255) / 256;
  if (grid > 8LL * nsm) grid = 8LL * nsm;
  if (grid < 1) grid = 1;
  if (a.ndim == 3) {
    if (a.flat) cfl_kernel<3, true><<<(int)grid, 256, 0, st>>>(a);
    else cfl_kernel<3, false><<<(int)grid, 256, 0, st>>>(a);
  } else {
    if (a.flat) cfl_kernel<2, true><<<(int)grid, 256, 0, st>>>(a);
    else cfl_kernel<2, false><<<(int)grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace bhac
