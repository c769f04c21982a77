// Device-side data layout and point-wise GRMHD for the GB300 stage kernels.
//
// Equations: ideal GRMHD in 3+1 ("Valencia") conservative form with GLM
// divergence cleaning, the covariant finite-volume scheme of the paper's
// Sec. 2.  The spatial metric is restricted to the Kerr-Schild structure
// (gamma_12 = gamma_23 = 0, beta = (beta^1, 0, 0), phi-independent), which
// covers Minkowski Cartesian, Kerr-Schild and modified Kerr-Schild exactly and
// lets every contraction skip its structural zeros.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define BHAC_HD __host__ __device__ __forceinline__

namespace bhac {

constexpr int NV = 9;
constexpr int MAXLEV = 4;  // refinement levels supported
// primitive slots
constexpr int RHO = 0, PRS = 1, U1 = 2, U2 = 3, U3 = 4, B1 = 5, B2 = 6, B3 = 7, PSI = 8;
// conserved slots
constexpr int CD = 0, CS1 = 1, CS2 = 2, CS3 = 3, CTAU = 4;

// Metric tables: cell-centre records (CREC doubles) and face records (FREC).
constexpr int CREC = 32, FREC = 12;
enum CRec {
  C_AL = 0, C_BE1, C_G11, C_G13, C_G22, C_G33, C_GI11, C_GI13, C_GI22, C_GI33, C_SG, C_ISG,
  C_ACG1, C_ACG2, C_ACG3, C_RHOFL, C_PFL,
  C_DAL1, C_DAL2, C_DBE1_1, C_DBE1_2, C_DG11_1, C_DG11_2, C_DG13_1, C_DG13_2, C_DG22_1, C_DG22_2,
  C_DG33_1, C_DG33_2
};
enum FRec { F_AL = 0, F_BE1, F_G11, F_G13, F_G22, F_G33, F_GI11, F_GI13, F_GI22, F_GI33, F_SG, F_ACG };

// Everything a stage kernel needs, passed by value.
struct StageArgs {
  int ndim;
  int nx, ny, nz;        // interior cells per block
  int gx, gy, gz;        // ghosts per side
  int Nx, Ny, Nz;        // ghosted extents
  int ncell, nint;       // ghosted / interior cells per block
  int tx, ty, ntx, nty;  // CTA column tile and tiles per block
  int nblocks, nitems;
  int nzp;               // z parts per (block, tile) item of the phased 3-D kernel (1: whole columns)
  int persistent;
  int minb;              // register bound of the 3-D stage kernel: 1 or 2 CTAs per SM
  int pwarps;            // 3-D: warps that produce face fluxes while the others update cells (0: phased)
  const int* blk;        // nblocks x 4: level, bx, by, bz
  const int* order;      // visiting order of the blocks (items run through it)
  double idx[3];         // 1/dx at level 0 per dimension
  double dxl0[3];        // dx at level 0
  int N1g, N2g;          // level-0 global cells along x1 and x2 (table extents)
  int axis_lo1, axis_hi1;  // polar axis at the low/high x2 boundary
  int flat;
  int recon, riemann;
  double gam, gam_fac, ch, kappa, cfl;
  float gam_f, gam_fac_f, ch_f, kappa_f, ch2_f;  // FP32 copies for the mixed form's flux arithmetic
  double c2p_tol;
  int c2p_maxit;
  double c2p_gf, c2p_v2max;  // (Gamma - 1)/Gamma and 1 - 1/W_max^2
  int split;                 // face kernel stores the stage right-hand side; a cell kernel finishes
  void* R;                   // that right-hand side, T per (block, var, interior cell)
  int item0, item1;          // (block, tile) items of this launch, in the visiting order
  int imex;                  // the cleaning damping is the implicit part of IMEX-SSP2(2,2,2)
  int c2p_nk;                // primary inversion: Jacobian-free Newton-Krylov (else analytic Newton)
  double imex_g;             // its gamma = 1 - 1/sqrt(2)
  double wmax, rho_fl_c, p_fl_c;  // constant floors (flat coordinates)
  // state
  const double* P_in;    // FP64 primitives, ghosted
  double* P_out;
  const float* P32_in;   // FP32 primitives, ghosted (mixed precision)
  float* P32_out;
  const double* Un;      // conserved at the start of the step
  const double* U1;      // conserved after stage 1
  double* Uout;
  const double* tab_c;   // cell-centre metric records, N2g x N1g
  const double* tab_f1;  // x1-face records, N2g x (N1g+1)
  const double* tab_f2;  // x2-face records, (N2g+1) x N1g
  const float* tab_c32;
  const float* tab_f1_32;
  const float* tab_f2_32;
  int stage;
  double dt_host;        // > 0: use it; else cfl / smax
  double* dt_dev;
  unsigned long long* smax_in;   // bits of the max CFL rate read by stage 1
  unsigned long long* smax_out;  // accumulated by stage 2 (and the CFL kernel)
  unsigned long long* counts;    // 4 inversion outcome counters
  unsigned char* status;         // per interior cell: inversion outcome of this stage
  unsigned int* work;            // persistent work counter
  // refinement levels: table offsets (records) and extents per level
  int nlev;
  long long toff_c[MAXLEV], toff_f1[MAXLEV], toff_f2[MAXLEV];
  int N1l[MAXLEV], N2l[MAXLEV];
  // coarse-fine faces: per block, bit 2d+s marks a face bordering finer blocks
  // (its adjacent cells are finished by the reflux pass); per block x 6 the
  // element offset of the face's flux register, or -1
  const unsigned char* cf;
  const long long* regoff;
  double* reg;
  const struct RefluxCell* rcells;
  const struct RefluxTerm* rterms;
  int nrcells;
};

// Geometry of one refinement level as seen by a kernel.
struct LevelGeo {
  const double* tc;
  const double* tf1;
  const double* tf2;
  const float* tc32;
  const float* tf1_32;
  const float* tf2_32;
  int N1, N2;
  double idx[3];
  float idx_f[3];
};

__host__ __device__ __forceinline__ LevelGeo level_geo(const StageArgs& a, int L) {
  LevelGeo g;
  g.tc = a.tab_c ? a.tab_c + a.toff_c[L] * CREC : nullptr;
  g.tf1 = a.tab_f1 ? a.tab_f1 + a.toff_f1[L] * FREC : nullptr;
  g.tf2 = a.tab_f2 ? a.tab_f2 + a.toff_f2[L] * FREC : nullptr;
  g.tc32 = a.tab_c32 ? a.tab_c32 + a.toff_c[L] * CREC : nullptr;
  g.tf1_32 = a.tab_f1_32 ? a.tab_f1_32 + a.toff_f1[L] * FREC : nullptr;
  g.tf2_32 = a.tab_f2_32 ? a.tab_f2_32 + a.toff_f2[L] * FREC : nullptr;
  g.N1 = a.N1l[L];
  g.N2 = a.N2l[L];
  const double s = (double)(1 << L);
  g.idx[0] = a.idx[0] * s;
  g.idx[1] = a.idx[1] * s;
  g.idx[2] = a.ndim == 3 ? a.idx[2] * s : a.idx[2];
  for (int d = 0; d < 3; ++d) g.idx_f[d] = (float)g.idx[d];
  return g;
}

// The kernel-argument scalar in the flux arithmetic T: the double for the
// FP64 form, the float copy for the mixed form (no conversion per use).
template <typename T>
__host__ __device__ __forceinline__ T pick(double d, float f);
template <>
__host__ __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__host__ __device__ __forceinline__ float pick<float>(double, float f) { return f; }

template <typename T>
struct Met {
  T al, be1, g11, g13, g22, g33, gi11, gi13, gi22, gi33, sg;
};

template <typename T>
BHAC_HD Met<T> flat_metric() {
  Met<T> m;
  m.al = T(1); m.be1 = T(0);
  m.g11 = T(1); m.g13 = T(0); m.g22 = T(1); m.g33 = T(1);
  m.gi11 = T(1); m.gi13 = T(0); m.gi22 = T(1); m.gi33 = T(1);
  m.sg = T(1);
  return m;
}

template <typename T, typename R>
BHAC_HD Met<T> load_face_metric(const R* __restrict__ rec) {
  Met<T> m;
  m.al = T(rec[F_AL]); m.be1 = T(rec[F_BE1]);
  m.g11 = T(rec[F_G11]); m.g13 = T(rec[F_G13]); m.g22 = T(rec[F_G22]); m.g33 = T(rec[F_G33]);
  m.gi11 = T(rec[F_GI11]); m.gi13 = T(rec[F_GI13]); m.gi22 = T(rec[F_GI22]); m.gi33 = T(rec[F_GI33]);
  m.sg = T(rec[F_SG]);
  return m;
}

template <typename T, typename R>
BHAC_HD Met<T> load_centre_metric(const R* __restrict__ rec) {
  Met<T> m;
  m.al = T(rec[C_AL]); m.be1 = T(rec[C_BE1]);
  m.g11 = T(rec[C_G11]); m.g13 = T(rec[C_G13]); m.g22 = T(rec[C_G22]); m.g33 = T(rec[C_G33]);
  m.gi11 = T(rec[C_GI11]); m.gi13 = T(rec[C_GI13]); m.gi22 = T(rec[C_GI22]); m.gi33 = T(rec[C_GI33]);
  m.sg = T(rec[C_SG]);
  return m;
}

// Scalar helpers.  The double/float overloads are the device arithmetic; the
// flop counter provides overloads for its counting type.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double abs_t(double x) { return fabs(x); }
__device__ __forceinline__ float abs_t(float x) { return fabsf(x); }
// exponent field not all ones (integer test, off the FP64 unit)
__device__ __forceinline__ bool finite_t(double x) {
  return ((unsigned)__double2hiint(x) & 0x7FF00000u) != 0x7FF00000u;
}
// FP32 <-> FP64 conversions by integer bit operations.  The FP64 unit
// executes conversion instructions at the cost of an FP64 FMA; rearranging
// the bits on the integer pipes gives the same IEEE results.  Widening is
// exact: a normal float's exponent is rebiased (+896) and its 23-bit
// significand placed at the top of the 52-bit one; narrowing rounds the
// 52-bit significand to 23 bits to nearest, ties to even (round bit = bit 28
// of the low word, sticky = bits 0..27), a carry out of the significand
// incrementing the exponent and reaching +-inf past the largest float.
// Zeros are handled in place; subnormal, overflowing, infinite and NaN
// operands take the hardware conversion.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}
__device__ __forceinline__ float narrow_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned E = (hi >> 20) & 0x7FFu;
  if (E - 897u < 254u) {  // the float exponent E - 896 is in [1, 254]
    unsigned r = (hi & 0x80000000u) | ((E - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rb = (lo >> 28) & 1u;
    const unsigned sticky = (lo & 0x0FFFFFFFu) != 0u ? 1u : 0u;
    r += rb & (sticky | (r & 1u));
    return __uint_as_float(r);
  }
  if (((hi & 0x7FFFFFFFu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return __double2float_rn(x);
}
// FP64 reciprocal, reciprocal square root and square root on the FP64 unit's
// budget.  GB300 runs an IEEE FP64 division or square root at about a tenth of
// its fused-multiply-add rate, and the inversion and the wave speeds take
// several per cell.  Here the FP32 hardware approximation (PTX rcp.approx /
// rsqrt.approx, on the special-function unit) of the operand rounded down to
// 20 significand bits seeds one step of a third-order (Householder) iteration
// in FP64 fused multiply-adds:
//   1/x:       e = 1 - x y,    y <- y (1 + e + e^2)          (error e0^3)
//   x^(-1/2):  e = 1 - x y^2,  y <- y (1 + e/2 + 3 e^2/8)    (error 5/2 e0^3)
// With |e0| < 2^-19 the iteration error is below 2^-57, so the result is the
// exact value up to the rounding of the last operations: within one unit in the
// last place for 1/x and x^(-1/2), 1.5 for sqrt x = x x^(-1/2)
// (bhac_check_bit_ops measures each against the IEEE operations on 2^24
// operands).  Operands whose binary exponent lies outside [-120, 120) (where
// the FP32 seed would leave the normal range), zeros, negatives (for the
// square roots), infinities and NaNs take the IEEE operation.
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx_f32(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// the FP32 value of a double whose biased exponent E is in [903, 1143),
// significand truncated to its top 20 bits (hi: the double's high word)
__device__ __forceinline__ float seed_of(unsigned hi, unsigned E) {
  return __uint_as_float((hi & 0x80000000u) | ((E - 896u) << 23) | ((hi & 0xFFFFFu) << 3));
}
// exact widening of a normal float (integer pipes)
__device__ __forceinline__ double widen_normal(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned hi = (u & 0x80000000u) | ((((u >> 23) & 0xFFu) + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ bool seed_range(unsigned hi, unsigned& E) {
  E = (hi >> 20) & 0x7FFu;
  return E - 903u < 240u;
}
__device__ __forceinline__ double rcp_t(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  unsigned E;
  if (!seed_range(hi, E)) return 1.0 / x;
  const double y = widen_normal(rcp_approx_f32(seed_of(hi, E)));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ double rsqrt_pos(double x, unsigned hi, unsigned E) {
  const double y = widen_normal(rsqrt_approx_f32(seed_of(hi, E)));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}
__device__ __forceinline__ double rsqrt_t(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  unsigned E;
  if ((hi >> 31) || !seed_range(hi, E)) return rsqrt(x);
  return rsqrt_pos(x, hi, E);
}
__device__ __forceinline__ double sqrt_t(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  unsigned E;
  if ((hi >> 31) || !seed_range(hi, E)) return sqrt(x);
  return x * rsqrt_pos(x, hi, E);
}
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return widen_f32(x); }

// Ordered selections.  On GB300 an FP64 compare occupies the SM's FP64 unit
// exactly like an FP64 fused multiply-add (two lanes per clock per SM), while
// 64-bit integer compares and selects run on the integer pipes at tens of
// lanes per clock.  The double overloads therefore compare an
// order-preserving integer image of the operands: okey maps -0 and +0 to 0
// and every other finite or infinite double so that okey(x) < okey(y)
// exactly when x < y; every compare below also returns false when an
// operand is NaN, so each decision is the IEEE compare's for all inputs.
// The NaN exclusions are integer compares too (on the keys or the bits), on
// the lightly used ALU pipe.  The generic templates (float, and the flop
// counter's counting type) are the plain compares.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? (long long)(0x8000000000000000ULL - (unsigned long long)b) : b;
}
constexpr unsigned long long kExpAll = 0x7FF0000000000000ULL;  // bits of +inf
template <typename T>
BHAC_HD bool lt_t(T a, T b) { return a < b; }
template <typename T>
BHAC_HD bool gt0_t(T x) { return x > T(0); }
template <typename T>
BHAC_HD bool le0_t(T x) { return x <= T(0); }
template <typename T>
BHAC_HD bool lt_abs_t(T a, T b) { return abs_t(a) < abs_t(b); }
// NaN keys lie outside [okey(-inf), okey(+inf)]: with ka < kb, a NaN operand
// can only be a negative NaN a (ka below okey(-inf)) or a positive NaN b (kb
// above okey(+inf)), so two range compares on the keys make a < b IEEE for
// all inputs.  (A bit-mask NaN test here is recognised by the compiler and
// lowered onto the FP64 unit.)
constexpr long long kKeyPosInf = 0x7FF0000000000000LL, kKeyNegInf = -0x7FF0000000000000LL;
BHAC_HD bool lt_t(double a, double b) {
#ifdef __CUDA_ARCH__
  const long long ka = okey(a), kb = okey(b);
  return ka < kb && ka >= kKeyNegInf && kb <= kKeyPosInf;
#else
  return a < b;
#endif
}
BHAC_HD bool gt0_t(double x) {
#ifdef __CUDA_ARCH__
  // positive finite or +inf: bits in [1, kExpAll]
  return (unsigned long long)__double_as_longlong(x) - 1ULL < kExpAll;
#else
  return x > 0.0;
#endif
}
BHAC_HD bool le0_t(double x) {
#ifdef __CUDA_ARCH__
  // +0, or sign bit set and not NaN
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return b == 0ULL || ((b >> 63) && (b & 0x7FFFFFFFFFFFFFFFULL) <= kExpAll);
#else
  return x <= 0.0;
#endif
}
// a <= b and x < 0 (the inversion's safeguards and convergence test)
template <typename T>
BHAC_HD bool le_x(T a, T b) { return a <= b; }
template <typename T>
BHAC_HD bool lt0_x(T x) { return x < T(0); }
BHAC_HD bool le_x(double a, double b) {
#ifdef __CUDA_ARCH__
  const long long ka = okey(a), kb = okey(b);
  return ka <= kb && ka >= kKeyNegInf && kb <= kKeyPosInf;
#else
  return a <= b;
#endif
}
BHAC_HD bool lt0_x(double x) {
#ifdef __CUDA_ARCH__
  // sign bit set, magnitude in (0, +inf]
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) && (b & 0x7FFFFFFFFFFFFFFFULL) - 1ULL < kExpAll;
#else
  return x < 0.0;
#endif
}

BHAC_HD bool lt_abs_t(double a, double b) {
#ifdef __CUDA_ARCH__
  const unsigned long long m = 0x7FFFFFFFFFFFFFFFULL;
  const unsigned long long x = (unsigned long long)__double_as_longlong(a) & m;
  const unsigned long long y = (unsigned long long)__double_as_longlong(b) & m;
  return x < y && y <= kExpAll;
#else
  return fabs(a) < fabs(b);
#endif
}

template <typename T>
BHAC_HD T sel3(int d, T a, T b, T c) {
  return d == 0 ? a : (d == 1 ? b : c);
}

// Derived quantities of a primitive state under a metric.
template <typename T>
struct Derived {
  T ul1, ul2, ul3, Bl1, Bl2, Bl3;
  T iW, W, iW2, v1, v2, v3, vl1, vl2, vl3, vsq;
  T Bsq, Bv, b2, rhoh, ptot;
};

template <typename T>
BHAC_HD void derive(const Met<T>& m, const T* P, T gam_fac, Derived<T>& s) {
  const T u1 = P[U1], u2 = P[U2], u3 = P[U3], B1_ = P[B1], B2_ = P[B2], B3_ = P[B3];
  s.ul1 = m.g11 * u1 + m.g13 * u3;
  s.ul2 = m.g22 * u2;
  s.ul3 = m.g13 * u1 + m.g33 * u3;
  s.Bl1 = m.g11 * B1_ + m.g13 * B3_;
  s.Bl2 = m.g22 * B2_;
  s.Bl3 = m.g13 * B1_ + m.g33 * B3_;
  const T usq = u1 * s.ul1 + u2 * s.ul2 + u3 * s.ul3;
  const T W2 = T(1) + usq;
  s.iW = rsqrt_t(W2);
  s.W = W2 * s.iW;
  s.iW2 = s.iW * s.iW;
  s.v1 = u1 * s.iW; s.v2 = u2 * s.iW; s.v3 = u3 * s.iW;
  s.vl1 = s.ul1 * s.iW; s.vl2 = s.ul2 * s.iW; s.vl3 = s.ul3 * s.iW;
  s.vsq = usq * s.iW2;
  s.Bsq = B1_ * s.Bl1 + B2_ * s.Bl2 + B3_ * s.Bl3;
  s.Bv = B1_ * s.vl1 + B2_ * s.vl2 + B3_ * s.vl3;
  s.b2 = s.Bsq * s.iW2 + s.Bv * s.Bv;
  s.rhoh = P[RHO] + gam_fac * P[PRS];
  s.ptot = P[PRS] + T(0.5) * s.b2;
}

// D = rho W, S_j = (rho h W^2 + B^2) v_j - (B.v) B_j, tau = rho h W^2 - p + B^2 - b^2/2 - D.
template <typename T>
BHAC_HD void cons_of(const T* P, const Derived<T>& s, T* U) {
  const T Z = s.rhoh * s.W * s.W;
  U[CD] = P[RHO] * s.W;
  const T ZB = Z + s.Bsq;
  U[CS1] = ZB * s.vl1 - s.Bv * s.Bl1;
  U[CS2] = ZB * s.vl2 - s.Bv * s.Bl2;
  U[CS3] = ZB * s.vl3 - s.Bv * s.Bl3;
  U[CTAU] = Z - P[PRS] + s.Bsq - T(0.5) * s.b2 - U[CD];
  U[B1] = P[B1]; U[B2] = P[B2]; U[B3] = P[B3];
  U[PSI] = P[PSI];
}

// Fluxes along d (undensitized):
//   F(D) = D (alpha v^d - beta^d), F(S_j) = alpha W^d_j - beta^d S_j,
//   W^d_j = S_j v^d + p_tot delta^d_j - B^d B_j / W^2 - (B.v) B^d v_j,
//   F(tau) = alpha (S^d - D v^d) - beta^d tau,
//   F(B^j) = (alpha v^d - beta^d) B^j - (alpha v^j - beta^j) B^d + alpha gamma^dj psi,
//   F(psi) = alpha ch^2 B^d - beta^d psi.
template <typename T>
BHAC_HD void flux_of(const Met<T>& m, const T* P, const Derived<T>& s, const T* U, int d,
                                        T ch2, T* F) {
  const T vd = sel3(d, s.v1, s.v2, s.v3);
  const T Bd = sel3(d, P[B1], P[B2], P[B3]);
  const T bed = d == 0 ? m.be1 : T(0);
  const T gid1 = sel3(d, m.gi11, T(0), m.gi13);
  const T gid2 = d == 1 ? m.gi22 : T(0);
  const T gid3 = sel3(d, m.gi13, T(0), m.gi33);
  const T al = m.al;
  F[CD] = U[CD] * (al * vd - bed);
  const T BdiW2 = Bd * s.iW2, BvBd = s.Bv * Bd;
  F[CS1] = al * (U[CS1] * vd - BdiW2 * s.Bl1 - BvBd * s.vl1 + (d == 0 ? s.ptot : T(0))) - bed * U[CS1];
  F[CS2] = al * (U[CS2] * vd - BdiW2 * s.Bl2 - BvBd * s.vl2 + (d == 1 ? s.ptot : T(0))) - bed * U[CS2];
  F[CS3] = al * (U[CS3] * vd - BdiW2 * s.Bl3 - BvBd * s.vl3 + (d == 2 ? s.ptot : T(0))) - bed * U[CS3];
  const T Sd = gid1 * U[CS1] + gid2 * U[CS2] + gid3 * U[CS3];
  F[CTAU] = al * (Sd - U[CD] * vd) - bed * U[CTAU];
  const T Vd = al * vd - bed;
  const T alpsi = al * P[PSI];
  F[B1] = Vd * P[B1] - (al * s.v1 - m.be1) * Bd + alpsi * gid1;
  F[B2] = Vd * P[B2] - (al * s.v2) * Bd + alpsi * gid2;
  F[B3] = Vd * P[B3] - (al * s.v3) * Bd + alpsi * gid3;
  F[PSI] = al * ch2 * Bd - bed * P[PSI];
}

// Fast-magnetosonic bound in the Eulerian frame (Del Zanna et al. 2007):
// a^2 = cs^2 + ca^2 - cs^2 ca^2, boosted by v and shifted by beta.  With
// cs^2 = Gamma p / (rho h) and ca^2 = b^2 / (rho h + b^2) this is
// a^2 = G / E, G = Gamma p + b^2, E = rho h + b^2, so with R = E - v^2 G
//   lambda = alpha [v^d (E - G) +- sqrt(G (1 - v^2) (gamma^dd R - v^d v^d (E - G)))] / R - beta^d,
// one reciprocal and one square root per state.
template <typename T>
BHAC_HD void speeds_of(const Met<T>& m, const T* P, const Derived<T>& s, int d, T gam, T& lm, T& lp) {
  const T E = s.rhoh + s.b2;
  const T G = gam * P[PRS] + s.b2;
  const T R = E - s.vsq * G;
  const T EG = E - G;
  const T vd = sel3(d, s.v1, s.v2, s.v3);
  const T gidd = sel3(d, m.gi11, m.gi22, m.gi33);
  T disc = G * (T(1) - s.vsq) * (gidd * R - vd * vd * EG);
  disc = gt0_t(disc) ? disc : T(0);
  const T sq = sqrt_t(disc);
  const T ir = rcp_t(R);
  const T bed = d == 0 ? m.be1 : T(0);
  const T c = vd * EG;
  lp = m.al * (c + sq) * ir - bed;
  lm = m.al * (c - sq) * ir - bed;
}

// ----------------------------------------------------------------------------
// Reconstruction (per variable).  PPM: Colella & Woodward 1984 interface value
// 7/12 (a_k + a_k+1) - 1/12 (a_k-1 + a_k+2) clipped to [a_k, a_k+1], then the
// CW84 monotonicity constraints per cell.  Minmod: limited linear slopes.
// ----------------------------------------------------------------------------
template <typename T>
BHAC_HD T ppm_iface(T am1, T a0, T a1, T a2) {
  T v = T(7.0 / 12.0) * (a0 + a1) - T(1.0 / 12.0) * (am1 + a2);
  const bool o = lt_t(a0, a1);
  const T lo = o ? a0 : a1, hi = o ? a1 : a0;
  v = lt_t(v, lo) ? lo : v;
  v = lt_t(hi, v) ? hi : v;
  return v;
}

template <typename T>
BHAC_HD void ppm_limit(T a, T& aL, T& aR) {
  if (le0_t((aR - a) * (a - aL))) {
    aL = a;
    aR = a;
  } else {
    const T d = aR - aL;
    const T m6 = T(6) * (a - T(0.5) * (aL + aR));
    if (lt_t(d * d, d * m6)) aL = T(3) * a - T(2) * aR;
    if (lt_t(d * m6, -d * d)) aR = T(3) * a - T(2) * aL;
  }
}

template <typename T>
BHAC_HD T minmod_t(T a, T b) {
  if (le0_t(a * b)) return T(0);
  return lt_abs_t(a, b) ? a : b;
}

// Both edges of one cell from its five-point stencil s_m2..s2 (cells c-2..c+2):
// aL at the cell's low face, aR at its high face.  The same formulas as
// recon_var evaluates per face, so a face's states from two cells' edges are
// bit-identical to recon_var's.
template <typename T>
BHAC_HD void recon_edges(int recon, T s_m2, T s_m1, T s0, T s1, T s2, T& aL, T& aR) {
  if (recon == 0) {
    aL = ppm_iface(s_m2, s_m1, s0, s1);
    aR = ppm_iface(s_m1, s0, s1, s2);
    ppm_limit(s0, aL, aR);
  } else {
    const T mm = minmod_t(s0 - s_m1, s1 - s0);
    aL = s0 - T(0.5) * mm;
    aR = s0 + T(0.5) * mm;
  }
}

template <typename T>
BHAC_HD void recon_var(int recon, T a0, T a1, T a2, T a3, T a4, T a5, T& L, T& R) {
  if (recon == 0) {
    T l2 = ppm_iface(a0, a1, a2, a3);
    T r2 = ppm_iface(a1, a2, a3, a4);
    T l3 = r2;
    T r3 = ppm_iface(a2, a3, a4, a5);
    ppm_limit(a2, l2, r2);
    ppm_limit(a3, l3, r3);
    L = r2;
    R = l3;
  } else {
    L = a2 + T(0.5) * minmod_t(a2 - a1, a3 - a2);
    R = a3 - T(0.5) * minmod_t(a3 - a2, a4 - a3);
  }
}

}  // namespace bhac
