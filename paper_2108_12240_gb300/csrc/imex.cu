// The first stage of the IMEX-SSP2(2,2,2) scheme (Pareschi & Russo 2005) for
// the stiff cleaning damping -alpha kappa psi: the explicit part of stage 1
// is evaluated at Y1, the implicit first stage, whose psi is
// psi_n / (1 + gamma alpha kappa dt) (gamma = 1 - 1/sqrt 2) and whose other
// variables are those of the step's start.  This pass scales psi of every
// interior cell's primitives before the stage's ghost fill; the stage kernel
// then completes the scheme cell by cell (stage_impl.cuh, cell_update).
#include "stage_impl.cuh"

namespace bhac {
namespace {

__global__ void __launch_bounds__(256) imex_first_stage_kernel(StageArgs a, double* P, float* P32) {
  const double dt = stage_dt(a);
  const long long n = (long long)a.nblocks * a.nint;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / a.nint);
    const int ci = (int)(t - (long long)b * a.nint);
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    double al = 1.0;
    if (!a.flat) {
      const LevelGeo geo = level_geo(a, a.blk[4 * b]);
      const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
      al = geo.tc[(size_t)(I2 * geo.N1 + I1) * CREC + C_AL];
    }
    const double f = 1.0 / (1.0 + a.imex_g * al * a.kappa * dt);
    const size_t o = ((size_t)b * NV + PSI) * a.ncell + cg;
    P[o] = P[o] * f;
    if (P32) P32[o] = narrow_f64(P[o]);
  }
}

}  // namespace

cudaError_t launch_imex_first_stage(const StageArgs& a, double* P, float* P32, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long n = (long long)a.nblocks * a.nint;
  long long g = (n + 255) / 256;
  if (g > 16LL * nsm) g = 16LL * nsm;
  imex_first_stage_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(a, P, P32);
  return cudaGetLastError();
}

}  // namespace bhac
