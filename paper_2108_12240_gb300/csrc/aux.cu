// Auxiliary kernels: ghost-cell gather, metric tables, state set-up and read-out.
#include <math.h>

#include "launch.h"

namespace bhac {

// ----------------------------------------------------------------------------
// Ghost fill (the paper's fill_gc_srl, Sec. 4.3 / 5.1): every ghost cell of
// every block is a gather from one interior cell (same-level neighbour or the
// boundary rule's source), with the sign flips of the polar axis and the
// no-inflow clamps applied.  One thread per (block, ghost slot); the nine
// variables are moved by the same thread.  CTA rows (blockIdx.y) walk the
// blocks and the threads of a row walk one block's slots, so no thread
// divides a flat (block, slot) index.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ghost_fill_kernel(GhostArgs g) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    if (g.work_reset) *g.work_reset = 0u;
    if (g.smax_reset) *g.smax_reset = 0ull;
  }
  for (int b = blockIdx.y; b < g.nblocks; b += gridDim.y)
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.nslots; s += gridDim.x * blockDim.x) {
    const size_t t = (size_t)b * g.nslots + s;
    const int src = g.src[t];
    const size_t dout = (size_t)b * NV * g.ncell + g.tmpl[s];
    if (src < 0) {
      // value of a cross-level node (already fixed up for the boundary rules)
      const size_t nn = (size_t)(-src - 1) * NV;
      if (g.P)
        for (int q = 0; q < NV; ++q) g.P[dout + (size_t)q * g.ncell] = g.node64[nn + q];
      if (g.P32)
        for (int q = 0; q < NV; ++q) g.P32[dout + (size_t)q * g.ncell] = g.node32[nn + q];
      continue;
    }
    const unsigned f = g.flags[t];
    const int sb = src / g.ncell;
    const int sc = src - sb * g.ncell;
    const size_t so = (size_t)sb * NV * g.ncell + sc;
    if (g.P) {
      double v[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] = g.P[so + (size_t)q * g.ncell];
      if (f & 1u) {
        v[U2] = -v[U2];
        v[B2] = -v[B2];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if ((f >> (1 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] > 0.0 ? 0.0 : v[U1 + d];
        if ((f >> (2 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] < 0.0 ? 0.0 : v[U1 + d];
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) g.P[dout + (size_t)q * g.ncell] = v[q];
    }
    if (g.P32) {
      float v[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] = g.P32[so + (size_t)q * g.ncell];
      if (f & 1u) {
        v[U2] = -v[U2];
        v[B2] = -v[B2];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if ((f >> (1 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] > 0.f ? 0.f : v[U1 + d];
        if ((f >> (2 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] < 0.f ? 0.f : v[U1 + d];
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) g.P32[dout + (size_t)q * g.ncell] = v[q];
    }
  }
}

static int grid_for(long long n, int threads) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long g = (n + threads - 1) / threads;
  const long long cap = 16LL * nsm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_ghost_fill(const GhostArgs& g, cudaStream_t st) {
  // x: the CTAs covering one block's slots; y: blocks (a CTA row loops over
  // blocks beyond the grid's y limit)
  const int gx = g.nslots > 0 ? (g.nslots + 255) / 256 : 1;
  const int gy = g.nblocks < 1 ? 1 : (g.nblocks < 65535 ? g.nblocks : 65535);
  ghost_fill_kernel<<<dim3(gx, gy), 256, 0, st>>>(g);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Metric tables.  Kerr-Schild (mass M, spin a) in (r, th, ph) or modified KS
// (x1 = ln r, x2 = th / pi, ph):
//   Sigma = r^2 + a^2 cos^2 th, z = 2 M r / Sigma,
//   gamma_rr = 1 + z, gamma_rph = -a sin^2 th (1 + z), gamma_thth = Sigma,
//   gamma_phph = sin^2 th (Sigma + a^2 sin^2 th (1 + z)),
//   alpha = (1 + z)^(-1/2), beta^r = z / (1 + z),
// with first derivatives along x1 and x2 carried by forward-mode dual numbers.
// ----------------------------------------------------------------------------
struct Dual {
  double v, a, b;  // value, d/dx1, d/dx2
};
__device__ __forceinline__ Dual mk(double v, double a = 0.0, double b = 0.0) { return Dual{v, a, b}; }
__device__ __forceinline__ Dual operator+(Dual x, Dual y) { return Dual{x.v + y.v, x.a + y.a, x.b + y.b}; }
__device__ __forceinline__ Dual operator-(Dual x, Dual y) { return Dual{x.v - y.v, x.a - y.a, x.b - y.b}; }
__device__ __forceinline__ Dual operator-(Dual x) { return Dual{-x.v, -x.a, -x.b}; }
__device__ __forceinline__ Dual operator*(Dual x, Dual y) {
  return Dual{x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b};
}
__device__ __forceinline__ Dual operator*(double s, Dual x) { return Dual{s * x.v, s * x.a, s * x.b}; }
__device__ __forceinline__ Dual operator+(double s, Dual x) { return Dual{s + x.v, x.a, x.b}; }
__device__ __forceinline__ Dual operator/(Dual x, Dual y) {
  const double q = x.v / y.v;
  return Dual{q, (x.a - q * y.a) / y.v, (x.b - q * y.b) / y.v};
}
__device__ __forceinline__ Dual dsqrt(Dual x) {
  const double s = sqrt(x.v);
  return Dual{s, 0.5 * x.a / s, 0.5 * x.b / s};
}
__device__ __forceinline__ Dual dsin(Dual x) {
  double s, c;
  sincos(x.v, &s, &c);
  return Dual{s, c * x.a, c * x.b};
}
__device__ __forceinline__ Dual dcos(Dual x) {
  double s, c;
  sincos(x.v, &s, &c);
  return Dual{c, -s * x.a, -s * x.b};
}
__device__ __forceinline__ Dual dexp(Dual x) {
  const double e = exp(x.v);
  return Dual{e, e * x.a, e * x.b};
}

struct KSCode {
  Dual al, be1, g11, g13, g22, g33;
  double r;
};

__device__ KSCode ks_code(const MetricArgs& M, double x1, double x2) {
  Dual X1 = mk(x1, 1.0, 0.0), X2 = mk(x2, 0.0, 1.0);
  Dual r, th, drdx, dthdx;
  if (M.coords == 2) {
    r = dexp(X1);
    th = M_PI * X2;
    drdx = r;
    dthdx = mk(M_PI);
  } else {
    r = X1;
    th = X2;
    drdx = mk(1.0);
    dthdx = mk(1.0);
  }
  const double a = M.spin;
  Dual s = dsin(th), c = dcos(th);
  Dual s2 = s * s;
  Dual Sigma = r * r + (a * a) * (c * c);
  Dual z = (2.0 * M.mass) * (r / Sigma);
  Dual opz = 1.0 + z;
  KSCode k;
  k.al = mk(1.0) / dsqrt(opz);
  k.be1 = (z / opz) / drdx;
  k.g11 = opz * drdx * drdx;
  k.g13 = (-a) * (s2 * opz) * drdx;
  k.g22 = Sigma * dthdx * dthdx;
  k.g33 = s2 * (Sigma + (a * a) * (s2 * opz));
  k.r = r.v;
  return k;
}

// Writes the inverse-metric block and sqrt(gamma) of a KS-structured metric.
__device__ __forceinline__ void ks_inverse(double g11, double g13, double g22, double g33, double& gi11,
                                           double& gi13, double& gi22, double& gi33, double& sg) {
  const double det13 = g11 * g33 - g13 * g13;
  gi11 = g33 / det13;
  gi13 = -g13 / det13;
  gi33 = g11 / det13;
  gi22 = 1.0 / g22;
  sg = sqrt(g22 * det13);
}

__global__ void metric_centre_kernel(MetricArgs M) {
  const int n = M.N1 * M.N2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i1 = t % M.N1, i2 = t / M.N1;
    const double x1 = M.x1min + (i1 + 0.5) * M.dx1, x2 = M.x2min + (i2 + 0.5) * M.dx2;
    KSCode k = ks_code(M, x1, x2);
    double* rec = M.tab_c + (size_t)t * CREC;
    double gi11, gi13, gi22, gi33, sg;
    ks_inverse(k.g11.v, k.g13.v, k.g22.v, k.g33.v, gi11, gi13, gi22, gi33, sg);
    rec[C_AL] = k.al.v;
    rec[C_BE1] = k.be1.v;
    rec[C_G11] = k.g11.v;
    rec[C_G13] = k.g13.v;
    rec[C_G22] = k.g22.v;
    rec[C_G33] = k.g33.v;
    rec[C_GI11] = gi11;
    rec[C_GI13] = gi13;
    rec[C_GI22] = gi22;
    rec[C_GI33] = gi33;
    rec[C_SG] = sg;
    rec[C_ISG] = 1.0 / sg;
    rec[C_ACG1] = k.al.v * sqrt(gi11);
    rec[C_ACG2] = k.al.v * sqrt(gi22);
    rec[C_ACG3] = k.al.v * sqrt(gi33);
    rec[C_RHOFL] = M.rho_floor * pow(k.r, M.rho_pow);
    rec[C_PFL] = M.p_floor * pow(k.r, M.p_pow);
    rec[C_DAL1] = k.al.a;
    rec[C_DAL2] = k.al.b;
    rec[C_DBE1_1] = k.be1.a;
    rec[C_DBE1_2] = k.be1.b;
    rec[C_DG11_1] = k.g11.a;
    rec[C_DG11_2] = k.g11.b;
    rec[C_DG13_1] = k.g13.a;
    rec[C_DG13_2] = k.g13.b;
    rec[C_DG22_1] = k.g22.a;
    rec[C_DG22_2] = k.g22.b;
    rec[C_DG33_1] = k.g33.a;
    rec[C_DG33_2] = k.g33.b;
    for (int q = C_DG33_2 + 1; q < CREC; ++q) rec[q] = 0.0;
    float* r32 = M.tab_c32 + (size_t)t * CREC;
    for (int q = 0; q < CREC; ++q) r32[q] = (float)rec[q];
  }
}

__device__ void face_record(const MetricArgs& M, double x1, double x2, int dir, bool axis, double* rec,
                            float* r32) {
  if (axis) {
    for (int q = 0; q < FREC; ++q) {
      rec[q] = 0.0;
      r32[q] = 0.f;
    }
    return;
  }
  KSCode k = ks_code(M, x1, x2);
  double gi11, gi13, gi22, gi33, sg;
  ks_inverse(k.g11.v, k.g13.v, k.g22.v, k.g33.v, gi11, gi13, gi22, gi33, sg);
  rec[F_AL] = k.al.v;
  rec[F_BE1] = k.be1.v;
  rec[F_G11] = k.g11.v;
  rec[F_G13] = k.g13.v;
  rec[F_G22] = k.g22.v;
  rec[F_G33] = k.g33.v;
  rec[F_GI11] = gi11;
  rec[F_GI13] = gi13;
  rec[F_GI22] = gi22;
  rec[F_GI33] = gi33;
  rec[F_SG] = sg;
  rec[F_ACG] = k.al.v * sqrt(dir == 0 ? gi11 : gi22);
  for (int q = 0; q < FREC; ++q) r32[q] = (float)rec[q];
}

__global__ void metric_face_kernel(MetricArgs M) {
  const int n1 = (M.N1 + 1) * M.N2, n2 = M.N1 * (M.N2 + 1);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2; t += gridDim.x * blockDim.x) {
    if (t < n1) {
      const int i1 = t % (M.N1 + 1), i2 = t / (M.N1 + 1);
      face_record(M, M.x1min + i1 * M.dx1, M.x2min + (i2 + 0.5) * M.dx2, 0, false, M.tab_f1 + (size_t)t * FREC,
                  M.tab_f1_32 + (size_t)t * FREC);
    } else {
      const int u = t - n1;
      const int i1 = u % M.N1, i2 = u / M.N1;
      const bool axis = (i2 == 0 && M.axis_lo) || (i2 == M.N2 && M.axis_hi);
      face_record(M, M.x1min + (i1 + 0.5) * M.dx1, M.x2min + i2 * M.dx2, 1, axis, M.tab_f2 + (size_t)u * FREC,
                  M.tab_f2_32 + (size_t)u * FREC);
    }
  }
}

cudaError_t launch_metric_tables(const MetricArgs& M, cudaStream_t st) {
  metric_centre_kernel<<<grid_for((long long)M.N1 * M.N2, 128), 128, 0, st>>>(M);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  metric_face_kernel<<<grid_for((long long)(M.N1 + 1) * M.N2 + (long long)M.N1 * (M.N2 + 1), 128), 128, 0, st>>>(M);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Interior <-> ghosted copies and the conserved state of given primitives.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void interior_coords(const StageArgs& a, long long t, int& b, int& ci, int& cg, int& i,
                                                int& j) {
  b = (int)(t / a.nint);
  ci = (int)(t - (long long)b * a.nint);
  i = ci % a.nx;
  j = (ci / a.nx) % a.ny;
  const int k = ci / (a.nx * a.ny);
  cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
}

__global__ void gather_kernel(StageArgs a, const double* __restrict__ P, double* dst) {
  const long long n = (long long)a.nblocks * a.nint;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int b, ci, cg, i, j;
    interior_coords(a, t, b, ci, cg, i, j);
    for (int v = 0; v < NV; ++v) dst[((size_t)b * NV + v) * a.nint + ci] = P[((size_t)b * NV + v) * a.ncell + cg];
  }
}

__global__ void init_cons_kernel(StageArgs a, const double* __restrict__ P, double* U) {
  const long long n = (long long)a.nblocks * a.nint;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int b, ci, cg, i, j;
    interior_coords(a, t, b, ci, cg, i, j);
    double Pc[NV], Uc[NV];
    for (int v = 0; v < NV; ++v) Pc[v] = P[((size_t)b * NV + v) * a.ncell + cg];
    Met<double> m = flat_metric<double>();
    double sg = 1.0;
    if (!a.flat) {
      const LevelGeo geo = level_geo(a, a.blk[4 * b]);
      const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
      const double* rec = geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC;
      m = load_centre_metric<double>(rec);
      sg = rec[C_SG];
    }
    Derived<double> s;
    derive(m, Pc, a.gam_fac, s);
    cons_of(Pc, s, Uc);
    for (int v = 0; v < NV; ++v) U[((size_t)b * NV + v) * a.nint + ci] = sg * Uc[v];
  }
}

cudaError_t launch_gather_interior(const StageArgs& a, const double* P, double* dst, cudaStream_t st) {
  gather_kernel<<<grid_for((long long)a.nblocks * a.nint, 256), 256, 0, st>>>(a, P, dst);
  return cudaGetLastError();
}

cudaError_t launch_init_cons(const StageArgs& a, const double* P, double* U, cudaStream_t st) {
  init_cons_kernel<<<grid_for((long long)a.nblocks * a.nint, 256), 256, 0, st>>>(a, P, U);
  return cudaGetLastError();
}

}  // namespace bhac
