// Operation count of one zone-stage, for the roofline (a measurement utility,
// not part of the method).  The stage kernel's own formulas (reconstruction,
// Riemann solve, sources, RK combination, inversion, CFL rate) are templates
// on the scalar type; here they run on the host with a counting scalar over
// cells sampled from the live state, so branch paths and Newton iteration
// counts are those of the actual workload.
//
// Counting convention: +, -, * = 1 flop each (a fused multiply-add is a
// multiply and an add: 2), / = 1, sqrt = 1, 1/sqrt = 1; compares, min/max,
// negation, selects and conversions = 0.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <random>
#include <type_traits>
#include <vector>

// The counting type is host-only; the host-device physics templates are only
// instantiated with it on the host.
#pragma nv_diag_suppress 20011
#pragma nv_diag_suppress 20014
#include "ctx.h"
#include "stage_impl.cuh"

namespace bhac {
namespace count {

struct Tally {
  double flops = 0, special = 0;  // special: divisions, square roots, reciprocal square roots
};
static Tally g_tally[2];  // [0] FP64, [1] FP32
static bool g_on = true;

template <int P>
struct Num {
  using V = typename std::conditional<P == 64, double, float>::type;
  V v;
  Num() : v(0) {}
  Num(double x) : v((V)x) {}
  Num(float x) : v((V)x) {}
  Num(int x) : v((V)x) {}
  static void op(int n = 1) {
    if (g_on) g_tally[P == 64 ? 0 : 1].flops += n;
  }
  static void sp() {
    if (g_on) {
      g_tally[P == 64 ? 0 : 1].flops += 1;
      g_tally[P == 64 ? 0 : 1].special += 1;
    }
  }
};

template <int P> Num<P> operator+(Num<P> a, Num<P> b) { Num<P>::op(); Num<P> r; r.v = a.v + b.v; return r; }
template <int P> Num<P> operator-(Num<P> a, Num<P> b) { Num<P>::op(); Num<P> r; r.v = a.v - b.v; return r; }
template <int P> Num<P> operator*(Num<P> a, Num<P> b) { Num<P>::op(); Num<P> r; r.v = a.v * b.v; return r; }
template <int P> Num<P> operator/(Num<P> a, Num<P> b) { Num<P>::sp(); Num<P> r; r.v = a.v / b.v; return r; }
template <int P> Num<P> operator-(Num<P> a) { Num<P> r; r.v = -a.v; return r; }
template <int P> bool operator<(Num<P> a, Num<P> b) { return a.v < b.v; }
template <int P> bool operator>(Num<P> a, Num<P> b) { return a.v > b.v; }
template <int P> bool operator<=(Num<P> a, Num<P> b) { return a.v <= b.v; }
template <int P> bool operator>=(Num<P> a, Num<P> b) { return a.v >= b.v; }

template <int P> Num<P> rsqrt_t(Num<P> x) { Num<P>::sp(); Num<P> r; r.v = (typename Num<P>::V)1 / std::sqrt(x.v); return r; }
template <int P> Num<P> sqrt_t(Num<P> x) { Num<P>::sp(); Num<P> r; r.v = std::sqrt(x.v); return r; }
template <int P> Num<P> rcp_t(Num<P> x) { Num<P>::sp(); Num<P> r; r.v = (typename Num<P>::V)1 / x.v; return r; }
template <int P> Num<P> abs_t(Num<P> x) { Num<P> r; r.v = std::fabs(x.v); return r; }
template <int P> bool finite_t(Num<P> x) { return std::isfinite(x.v); }
template <int P> double to_double(Num<P> x) { return (double)x.v; }

using N64 = Num<64>;
using N32 = Num<32>;

}  // namespace count
}  // namespace bhac

using namespace bhac;
using namespace bhac::count;

namespace {

struct HostState {
  int nbs;                      // sampled blocks
  std::vector<int> ids;         // their block indices
  std::vector<double> P;        // nbs x NV x ncell (FP64 ghosted)
  std::vector<float> P32;       // nbs x NV x ncell (FP32 ghosted, mixed form)
  std::vector<double> U;        // nbs x NV x nint
  std::vector<double> tc, tf1, tf2;
  std::vector<float> tc32, tf132, tf232;
};

template <typename T, typename S>
void load_stencil(const StageArgs& a, const S* Pb, int d, int ig, int jg, int kg, T PL[NV], T PR[NV]) {
  const int sd = d == 0 ? 1 : (d == 1 ? a.Nx : a.Nx * a.Ny);
  const int c0 = (kg * a.Ny + jg) * a.Nx + ig;
  // the face states are the high edge of the low cell and the low edge of
  // the high cell; the kernel reconstructs each cell's edges once per
  // direction, so only the high cell's (the sampled cell's) are counted
  const bool on = g_on;
  for (int v = 0; v < NV; ++v) {
    const S* p = Pb + (size_t)v * a.ncell + c0;
    T l0, r0, l1, r1;
    g_on = false;
    recon_edges(a.recon, T(p[-3 * sd]), T(p[-2 * sd]), T(p[-sd]), T(p[0]), T(p[sd]), l0, r0);
    g_on = on;
    recon_edges(a.recon, T(p[-2 * sd]), T(p[-sd]), T(p[0]), T(p[sd]), T(p[2 * sd]), l1, r1);
    PL[v] = r0;
    PR[v] = l1;
  }
  if (!(PL[RHO] > T(0)) || !(PL[PRS] > T(0)) || !(PR[RHO] > T(0)) || !(PR[PRS] > T(0))) {
    for (int v = 0; v < NV; ++v) {
      const S* p = Pb + (size_t)v * a.ncell + c0;
      PL[v] = T(p[-sd]);
      PR[v] = T(p[0]);
    }
  }
}

// Flux through the face of direction d whose high-side cell is (ig, jg, kg).
// tc, tf1, tf2 are the tables of the block's level, N1 x N2 cells.
template <typename T, typename S, typename R>
void face(const StageArgs& a, const S* Pb, const R* tc, const R* tf1, const R* tf2, int N1, int N2, int d, int ig,
          int jg, int kg, int I1, int I2, double out[NV]) {
  T PL[NV], PR[NV], F[NV];
  if (!a.flat && d == 1 && ((I2 == 0 && a.axis_lo1) || (I2 == N2 && a.axis_hi1))) {
    for (int v = 0; v < NV; ++v) out[v] = 0.0;
    return;
  }
  load_stencil<T, S>(a, Pb, d, ig, jg, kg, PL, PR);
  Met<T> m = flat_metric<T>();
  T acg = T(1);
  if (!a.flat) {
    const R* rec = d == 0 ? tf1 + (size_t)(I2 * (N1 + 1) + I1) * FREC
                          : (d == 1 ? tf2 + (size_t)(I2 * N1 + I1) * FREC : tc + (size_t)(I2 * N1 + I1) * CREC);
    m = load_face_metric<T>(rec);
    acg = T(d == 2 ? rec[C_ACG3] : rec[F_ACG]);
  }
  riemann_flux(m, acg, PL, PR, d, a.riemann, T(a.gam), T(a.gam_fac), T(a.ch), F);
  for (int v = 0; v < NV; ++v) out[v] = to_double(F[v]);
}

// One cell through both stages' arithmetic; faces are counted once per
// direction (the low face), as the kernel evaluates each face once.
template <typename T, typename S, typename R>
void cell(const StageArgs& a, const HostState& h, int sb, int i, int j, int k, double dt, int stage) {
  const int bidx = h.ids[sb];
  const S* Pb;
  const R *tc, *tf1, *tf2;
  if (std::is_same<S, float>::value) {
    Pb = (const S*)(h.P32.data() + (size_t)sb * NV * a.ncell);
    tc = (const R*)h.tc32.data();
    tf1 = (const R*)h.tf132.data();
    tf2 = (const R*)h.tf232.data();
  } else {
    Pb = (const S*)(h.P.data() + (size_t)sb * NV * a.ncell);
    tc = (const R*)h.tc.data();
    tf1 = (const R*)h.tf1.data();
    tf2 = (const R*)h.tf2.data();
  }
  // the block's refinement level: its metric tables, extents and spacing
  const int L = a.blk[4 * bidx];
  const int N1 = a.N1l[L], N2 = a.N2l[L];
  tc += (size_t)a.toff_c[L] * CREC;
  tf1 += (size_t)a.toff_f1[L] * FREC;
  tf2 += (size_t)a.toff_f2[L] * FREC;
  const double lsc = (double)(1 << L);
  const double idx[3] = {a.idx[0] * lsc, a.idx[1] * lsc, a.ndim == 3 ? a.idx[2] * lsc : a.idx[2]};
  const int ig = i + a.gx, jg = j + a.gy, kg = k + a.gz;
  const int I1 = a.blk[4 * bidx + 1] * a.nx + i, I2 = a.blk[4 * bidx + 2] * a.ny + j;
  double Flo[3][NV], Fhi[3][NV];
  for (int d = 0; d < a.ndim; ++d) {
    g_on = true;
    face<T, S, R>(a, Pb, tc, tf1, tf2, N1, N2, d, ig, jg, kg, I1, I2, Flo[d]);
    g_on = false;
    face<T, S, R>(a, Pb, tc, tf1, tf2, N1, N2, d, ig + (d == 0), jg + (d == 1), kg + (d == 2), I1 + (d == 0),
                  I2 + (d == 1), Fhi[d]);
  }
  g_on = true;
  // flux divergence in the flux arithmetic T, as the kernel forms it
  T rdiv[NV];
  N64 rhs[NV];
  for (int v = 0; v < NV; ++v) {
    T r = -(T(Fhi[0][v]) - T(Flo[0][v])) * T(idx[0]);
    r = r - (T(Fhi[1][v]) - T(Flo[1][v])) * T(idx[1]);
    if (a.ndim == 3) r = r - (T(Fhi[2][v]) - T(Flo[2][v])) * T(idx[2]);
    rdiv[v] = r;
  }
  const int cg = (kg * a.Ny + jg) * a.Nx + ig;
  T Pc[NV];
  for (int v = 0; v < NV; ++v) Pc[v] = T(Pb[(size_t)v * a.ncell + cg]);
  double sg = 1.0, isg = 1.0, rho_fl = a.rho_fl_c, p_fl = a.p_fl_c;
  const double* crec = a.flat ? nullptr : h.tc.data() + ((size_t)a.toff_c[L] + (size_t)I2 * N1 + I1) * CREC;
  if (a.flat) {
    rdiv[PSI] = rdiv[PSI] - T(a.kappa) * Pc[PSI];
    for (int v = 0; v < NV; ++v) rhs[v] = N64(to_double(rdiv[v]));
  } else {
    const R* rec = tc + (size_t)(I2 * N1 + I1) * CREC;
    Met<T> m = load_centre_metric<T>(rec);
    Derived<T> s;
    T Uc[NV], S_[NV];
    derive(m, Pc, T(a.gam_fac), s);
    cons_of(Pc, s, Uc);
    sources_of(m, rec, Pc, s, Uc, T(a.kappa), T(a.ch * a.ch), S_);
    sg = crec[C_SG];
    isg = crec[C_ISG];
    rho_fl = crec[C_RHOFL];
    p_fl = crec[C_PFL];
    if (std::is_same<T, N64>::value) {
      for (int v = 0; v < NV; ++v) rhs[v] = N64(to_double(rdiv[v])) + N64(sg) * N64(to_double(S_[v]));
    } else {
      for (int v = 0; v < NV; ++v) rhs[v] = N64(to_double(rdiv[v] + T(sg) * S_[v]));
    }
  }
  // RK combination (the stage-2 form also uses the stage-1 state; the
  // operation count does not depend on its value)
  const double* Ub = h.U.data() + (size_t)sb * NV * a.nint;
  const int ci = (k * a.ny + j) * a.nx + i;
  N64 U[NV];
  for (int v = 0; v < NV; ++v) {
    const N64 un = N64(Ub[(size_t)v * a.nint + ci]);
    U[v] = stage == 1 ? un + N64(dt) * rhs[v] : N64(0.5) * un + N64(0.5) * (un + N64(dt) * rhs[v]);
  }
  Met<N64> md = a.flat ? flat_metric<N64>() : load_centre_metric<N64>(crec);
  N64 Uu[NV], Pg[NV], Pn[NV];
  const double* Pd = h.P.data() + (size_t)sb * NV * a.ncell + cg;
  for (int v = 0; v < NV; ++v) {
    Uu[v] = U[v] * N64(isg);
    Pg[v] = N64(Pd[(size_t)v * a.ncell]);
  }
  // the mixed form starts Newton from the FP32 previous primitives and
  // rebuilds a floored cell's D, S_i, tau in FP32 (as finish_cell does)
  const bool mixed = std::is_same<T, N32>::value;
  const float* crec32 =
      (a.flat || !mixed) ? nullptr : h.tc32.data() + ((size_t)a.toff_c[L] + (size_t)I2 * N1 + I1) * CREC;
  Met<N32> m32 = crec32 ? load_centre_metric<N32>(crec32) : flat_metric<N32>();
  N64 Z0, v20;
  if (mixed) {
    const float* P3 = h.P32.data() + (size_t)sb * NV * a.ncell + cg;
    N32 Pg32[NV];
    for (int v = 0; v < NV; ++v) Pg32[v] = N32(P3[(size_t)v * a.ncell]);
    N32 z, w;
    c2p_guess<N32>(m32, Pg32, N32(a.gam_fac_f), z, w);
    Z0 = N64((double)z.v);
    v20 = N64((double)w.v);
  } else {
    c2p_guess<N64>(md, Pg, N64(a.gam_fac), Z0, v20);
  }
  const int st = con2prim_t<N64>(md, Uu, Pg, 1, Z0, v20, N64(rho_fl), N64(p_fl), a.c2p_gf, a.wmax, a.c2p_v2max,
                                 a.c2p_tol, a.c2p_maxit, a.c2p_nk, Pn);
  if (st >= 2) {
    if (mixed) {
      N32 P32[NV], Uc[NV];
      for (int v = 0; v < NV; ++v) P32[v] = N32((float)Pn[v].v);
      Derived<N32> s;
      derive(m32, P32, N32(a.gam_fac_f), s);
      cons_of(P32, s, Uc);
      const N32 sg32 = N32(a.flat ? 1.0f : crec32[C_SG]);
      for (int v = CD; v <= CTAU; ++v) U[v] = N64((double)(sg32 * Uc[v]).v);
    } else {
      Derived<N64> s;
      derive(md, Pn, N64(a.gam_fac), s);
      cons_of(Pn, s, Uu);
      for (int v = 0; v < NV; ++v) U[v] = N64(sg) * Uu[v];
    }
  }
  if (stage == 2) {
    N64 acg[3] = {N64(1.0), N64(1.0), N64(1.0)};
    if (!a.flat) {
      acg[0] = N64(crec[C_ACG1]);
      acg[1] = N64(crec[C_ACG2]);
      acg[2] = N64(crec[C_ACG3]);
    }
    if (a.ndim == 3)
      (void)cfl_rate_t<N64, 3>(md, acg, Pn, a.gam, a.gam_fac, a.ch, idx);
    else
      (void)cfl_rate_t<N64, 2>(md, acg, Pn, a.gam, a.gam_fac, a.ch, idx);
  }
}

template <typename V>
cudaError_t fetch(std::vector<V>& out, const V* src, size_t n, cudaStream_t st) {
  out.resize(n);
  if (n == 0) return cudaSuccess;
  return cudaMemcpyAsync(out.data(), src, n * sizeof(V), cudaMemcpyDeviceToHost, st);
}

}  // namespace

extern "C" bhac_status bhac_count_flops(bhac_ctx* c, double dt, int nsamples, unsigned seed, double out[6]) {
  if (!c || !out || nsamples < 1 || !(dt > 0.0)) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  bhac_status s = ghost_fill(c, c->cur, false);
  if (s != BHAC_OK) return s;
  StageArgs a = base_args(c);
  a.blk = c->blk.data();  // host copy
  HostState h;
  std::mt19937 rng(seed);
  h.nbs = c->nb < 4 ? c->nb : 4;
  for (int q = 0; q < h.nbs; ++q) h.ids.push_back((int)(rng() % (unsigned)c->nb));
  h.P.resize((size_t)h.nbs * NV * c->ncell);
  h.U.resize((size_t)h.nbs * NV * c->nint);
  if (c->mixed) h.P32.resize((size_t)h.nbs * NV * c->ncell);
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < h.nbs && e == cudaSuccess; ++q) {
    const int b = h.ids[q];
    e = cudaMemcpyAsync(h.P.data() + (size_t)q * NV * c->ncell, c->P[c->cur] + (size_t)b * NV * c->ncell,
                        sizeof(double) * NV * c->ncell, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && c->mixed)
      e = cudaMemcpyAsync(h.P32.data() + (size_t)q * NV * c->ncell, c->P32[c->cur] + (size_t)b * NV * c->ncell,
                          sizeof(float) * NV * c->ncell, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.U.data() + (size_t)q * NV * c->nint, c->U[c->ucur] + (size_t)b * NV * c->nint,
                          sizeof(double) * NV * c->nint, cudaMemcpyDeviceToHost, c->st);
  }
  if (!c->flat && e == cudaSuccess) {
    // every level's tables (levels follow one another in each table)
    const StageArgs t = base_args(c);
    const int Lt = t.nlev - 1;
    const size_t nc = (size_t)t.toff_c[Lt] + (size_t)t.N1l[Lt] * t.N2l[Lt];
    const size_t nf1 = (size_t)t.toff_f1[Lt] + (size_t)(t.N1l[Lt] + 1) * t.N2l[Lt];
    const size_t nf2 = (size_t)t.toff_f2[Lt] + (size_t)t.N1l[Lt] * (t.N2l[Lt] + 1);
    e = fetch(h.tc, c->tab_c, nc * CREC, c->st);
    if (e == cudaSuccess) e = fetch(h.tf1, c->tab_f1, nf1 * FREC, c->st);
    if (e == cudaSuccess) e = fetch(h.tf2, c->tab_f2, nf2 * FREC, c->st);
    if (e == cudaSuccess) e = fetch(h.tc32, c->tab_c32, nc * CREC, c->st);
    if (e == cudaSuccess) e = fetch(h.tf132, c->tab_f1_32, nf1 * FREC, c->st);
    if (e == cudaSuccess) e = fetch(h.tf232, c->tab_f2_32, nf2 * FREC, c->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  g_tally[0] = Tally();
  g_tally[1] = Tally();
  for (int n = 0; n < nsamples; ++n) {
    const int sb = (int)(rng() % (unsigned)h.nbs);
    const int i = (int)(rng() % (unsigned)a.nx), j = (int)(rng() % (unsigned)a.ny), k = (int)(rng() % (unsigned)a.nz);
    for (int stage = 1; stage <= 2; ++stage) {
      if (c->mixed)
        cell<N32, float, float>(a, h, sb, i, j, k, dt, stage);
      else
        cell<N64, double, double>(a, h, sb, i, j, k, dt, stage);
    }
  }
  g_on = true;
  const double per = 1.0 / (2.0 * nsamples);  // per zone-stage
  out[0] = g_tally[0].flops * per;
  out[1] = g_tally[1].flops * per;
  out[2] = g_tally[0].special * per;
  out[3] = g_tally[1].special * per;
  out[4] = (double)nsamples;
  out[5] = (double)h.nbs;
  return BHAC_OK;
}
