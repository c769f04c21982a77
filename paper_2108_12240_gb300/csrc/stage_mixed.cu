// Mixed-precision instantiations of the stage kernel: FP32 reconstruction,
// face fluxes, wave speeds and sources; FP64 flux differences, RK update,
// inversion and CFL.
#include "stage_impl.cuh"

namespace bhac {

cudaError_t launch_stage_mixed(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  return launch_stage_any<float>(a, grid, threads, smem, st);
}

cudaError_t prepare_stage_mixed() { return configure_all_t<float>(); }

}  // namespace bhac
