// Mixed-precision instantiations of the stage kernel: FP32 reconstruction,
// face fluxes, wave speeds and sources; FP64 flux differences, RK update,
// inversion and CFL.
#include "stage_impl.cuh"

namespace bhac {

cudaError_t launch_stage_mixed(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  return launch_stage_any<float>(a, grid, threads, smem, st);
}

cudaError_t prepare_stage_mixed() { return configure_all_t<float>(); }

cudaError_t launch_cells_mixed(const StageArgs& a, int grid, cudaStream_t st) { return launch_cells_any<float>(a, grid, st); }
cudaError_t launch_reflux_mixed(const StageArgs& a, cudaStream_t st) { return launch_reflux_any<float>(a, st); }

int stage_occupancy_mixed(const StageArgs& a, int threads, size_t smem) {
  return stage_occupancy_any<float>(a, threads, smem);
}

}  // namespace bhac
