// Allocation-free CFL time step (see bhac_cfl_dt_static in the public header).
//
// Some callers cannot call cudaMalloc at all: a host whose device memory is
// entirely owned by another allocator and hands this library no arena, or a
// per-step diagnostic that must never enter an allocator (cudaMalloc can
// synchronise the device and stall the streams the time step keeps busy).  For
// them this file keeps the reduction's scratch in file-scope device arrays of
// fixed size instead of an arena: the leaf-block table and one partial maximum
// per block.  Every GPU that loads the library holds these arrays
// (BHAC_STATIC_MAX_BLOCKS x 24 bytes) until the process exits.
#include <math.h>
#include <mutex>

#include "stage_impl.cuh"

namespace bhac {
namespace {

static __device__ __align__(256) int4 g_static_blocks[BHAC_STATIC_MAX_BLOCKS];
static __device__ __align__(256) double g_static_partial[BHAC_STATIC_MAX_BLOCKS];

struct StaticGrid {
  int ndim, coords, nx[3];
  double xmin[3], dx0[3];
  double spin, mass, gam, gam_fac, ch, cfl;
};

// Kerr-Schild / modified Kerr-Schild metric at a cell centre (values only).
__device__ Met<double> centre_metric(const StaticGrid& s, double x1, double x2, double acg[3]) {
  Met<double> m = flat_metric<double>();
  acg[0] = acg[1] = acg[2] = 1.0;
  if (s.coords == BHAC_COORDS_CART) return m;
  const double r = s.coords == BHAC_COORDS_MKS ? exp(x1) : x1;
  const double th = s.coords == BHAC_COORDS_MKS ? M_PI * x2 : x2;
  const double drdx = s.coords == BHAC_COORDS_MKS ? r : 1.0;
  const double dthdx = s.coords == BHAC_COORDS_MKS ? M_PI : 1.0;
  double sn, cs;
  sincos(th, &sn, &cs);
  const double s2 = sn * sn, a = s.spin;
  const double Sigma = r * r + a * a * cs * cs;
  const double z = 2.0 * s.mass * r / Sigma;
  m.al = 1.0 / sqrt(1.0 + z);
  m.be1 = z / (1.0 + z) / drdx;
  m.g11 = (1.0 + z) * drdx * drdx;
  m.g13 = -a * s2 * (1.0 + z) * drdx;
  m.g22 = Sigma * dthdx * dthdx;
  m.g33 = s2 * (Sigma + a * a * s2 * (1.0 + z));
  const double det13 = m.g11 * m.g33 - m.g13 * m.g13;
  m.gi11 = m.g33 / det13;
  m.gi13 = -m.g13 / det13;
  m.gi33 = m.g11 / det13;
  m.gi22 = 1.0 / m.g22;
  m.sg = sqrt(m.g22 * det13);
  acg[0] = m.al * sqrt(m.gi11);
  acg[1] = m.al * sqrt(m.gi22);
  acg[2] = m.al * sqrt(m.gi33);
  return m;
}

// One CTA per block: the block's largest CFL rate into g_static_partial[b].
template <int DIM>
__global__ void __launch_bounds__(256) static_rate_kernel(StaticGrid s, const double* __restrict__ P) {
  __shared__ double red[8];
  const int b = blockIdx.x;
  const int4 bd = g_static_blocks[b];  // level, ix, iy, iz
  const int nint = s.nx[0] * s.nx[1] * s.nx[2];
  const double sc = (double)(1 << bd.x);
  double idx[3], dx[3];
  for (int k = 0; k < 3; ++k) {
    dx[k] = k < s.ndim ? s.dx0[k] / sc : s.dx0[k];
    idx[k] = 1.0 / dx[k];
  }
  double rate_max = 0.0;
  for (int c = threadIdx.x; c < nint; c += blockDim.x) {
    const int i = c % s.nx[0], j = (c / s.nx[0]) % s.nx[1];
    const double x1 = s.xmin[0] + ((double)bd.y * s.nx[0] + i + 0.5) * dx[0];
    const double x2 = s.xmin[1] + ((double)bd.z * s.nx[1] + j + 0.5) * dx[1];
    double acg[3];
    const Met<double> m = centre_metric(s, x1, x2, acg);
    double Pc[NV];
    for (int v = 0; v < NV; ++v) Pc[v] = P[((size_t)b * NV + v) * nint + c];
    rate_max = fmax(rate_max, cfl_rate_t<double, DIM>(m, acg, Pc, s.gam, s.gam_fac, s.ch, idx));
  }
  rate_max = warp_max_d(rate_max);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rate_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    g_static_partial[b] = r;
  }
}

// One CTA: dt = cfl / max over the partials of the current call.
__global__ void __launch_bounds__(256) static_dt_kernel(int nblocks, double cfl, double* dt) {
  __shared__ double red[8];
  double r = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) r = fmax(r, g_static_partial[b]);
  r = warp_max_d(r);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    *dt = cfl / m;
  }
}

// Device addresses of the two arrays, looked up once per device.
struct Symbols {
  int4* blocks = nullptr;
  double* partial = nullptr;
};
std::mutex g_sym_lock;
Symbols g_sym[64];

bool symbols_for_current_device(Symbols& out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lock(g_sym_lock);
  Symbols& s = g_sym[dev];
  if (!s.blocks) {
    void* pb = nullptr;
    void* pp = nullptr;
    if (cudaGetSymbolAddress(&pb, g_static_blocks) != cudaSuccess) return false;
    if (cudaGetSymbolAddress(&pp, g_static_partial) != cudaSuccess) return false;
    s.blocks = (int4*)pb;
    s.partial = (double*)pp;
  }
  out = s;
  return true;
}

bool valid_static(const bhac_grid_desc* d, const bhac_block_desc* b, int nb) {
  if (!d || !b || nb <= 0) return false;
  if (d->ndim < 2 || d->ndim > 3 || d->nlevels < 1 || d->nlevels > MAXLEV) return false;
  if (d->coords < 0 || d->coords > 2 || !(d->gamma_ad > 1.0) || !(d->cfl > 0.0) || !(d->ch > 0.0)) return false;
  for (int k = 0; k < 3; ++k) {
    if (d->nx[k] < 1 || d->nroot[k] < 1 || !(d->xmax[k] > d->xmin[k])) return false;
    if (k >= d->ndim && d->nx[k] != 1) return false;
  }
  for (int i = 0; i < nb; ++i) {
    if (b[i].level < 0 || b[i].level >= d->nlevels) return false;
    const int c[3] = {b[i].ix, b[i].iy, b[i].iz};
    for (int k = 0; k < 3; ++k)
      if (c[k] < 0 || c[k] >= (d->nroot[k] << (k < d->ndim ? b[i].level : 0))) return false;
  }
  return true;
}

}  // namespace
}  // namespace bhac

using namespace bhac;

extern "C" bhac_status bhac_cfl_dt_static(const bhac_grid_desc* d, const bhac_block_desc* blocks, int nblocks,
                                          const double* prims, double* dt, void* stream) {
  if (nblocks > BHAC_STATIC_MAX_BLOCKS) return BHAC_ERR_ARG;  // beyond the fixed scratch
  if (!prims || !dt || !valid_static(d, blocks, nblocks)) return BHAC_ERR_ARG;
  Symbols sym;
  if (!symbols_for_current_device(sym)) return BHAC_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  static_assert(sizeof(bhac_block_desc) == sizeof(int4), "block descriptor layout");
  if (cudaMemcpyAsync(sym.blocks, blocks, sizeof(int4) * (size_t)nblocks, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return BHAC_ERR_CUDA;
  StaticGrid s;
  s.ndim = d->ndim;
  s.coords = d->coords;
  for (int k = 0; k < 3; ++k) {
    s.nx[k] = d->nx[k];
    s.xmin[k] = d->xmin[k];
    s.dx0[k] = (d->xmax[k] - d->xmin[k]) / ((double)d->nroot[k] * d->nx[k]);
  }
  s.spin = d->spin;
  s.mass = d->mass;
  s.gam = d->gamma_ad;
  s.gam_fac = d->gamma_ad / (d->gamma_ad - 1.0);
  s.ch = d->ch;
  s.cfl = d->cfl;
  if (d->ndim == 3)
    static_rate_kernel<3><<<nblocks, 256, 0, st>>>(s, prims);
  else
    static_rate_kernel<2><<<nblocks, 256, 0, st>>>(s, prims);
  if (cudaGetLastError() != cudaSuccess) return BHAC_ERR_CUDA;
  static_dt_kernel<<<1, 256, 0, st>>>(nblocks, d->cfl, dt);
  return cudaGetLastError() == cudaSuccess ? BHAC_OK : BHAC_ERR_CUDA;
}
