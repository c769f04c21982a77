// The fused RK-stage kernel: reconstruction, HLL/TVDLF face fluxes, geometric
// and GLM sources, the SSP-RK2 stage combination, the Newton conserved-to-
// primitive inversion with its backup and floors, and (stage 2) the per-cell
// CFL rate reduced into one device word.  Included by stage_fp64.cu and
// stage_mixed.cu, which instantiate it for FP64 and FP32 flux arithmetic.
//
// Work decomposition: one CTA owns a column of tx x ty cells of one block and
// marches through its nz planes.  Per plane it reconstructs each cell's edges
// once per direction into shared memory, computes every x-, y- and (top)
// z-face flux of the column once from them, then updates each cell; the
// z-face flux at the top of a plane is carried over as the bottom of the
// next, so no interior face flux is evaluated twice.
#pragma once

#include "amr.h"
#include "bhac_device.cuh"
#include "launch.h"

namespace bhac {

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ----------------------------------------------------------------------------
// Geometric + GLM sources for a stationary, phi-independent metric of
// Kerr-Schild structure (derivatives along x1 and x2 only):
//   S(S_j) = 1/2 alpha W^ik d_j gamma_ik + S_i d_j beta^i - E d_j alpha
//   S(tau) = 1/2 W^ik beta^j d_j gamma_ik + W^j_i d_j beta^i - S^j d_j alpha
//   S(psi) = -alpha kappa psi - psi d_i beta^i + ch^2 B^i d_i alpha
// ----------------------------------------------------------------------------
template <typename T, typename R>
BHAC_HD void sources_of(const Met<T>& m, const R* __restrict__ rec, const T* P,
                                           const Derived<T>& s, const T* U, T kappa, T ch2, T* S) {
  const T dal1 = T(rec[C_DAL1]), dal2 = T(rec[C_DAL2]);
  const T db11 = T(rec[C_DBE1_1]), db12 = T(rec[C_DBE1_2]);
  const T Su1 = m.gi11 * U[CS1] + m.gi13 * U[CS3];
  const T Su2 = m.gi22 * U[CS2];
  const T Su3 = m.gi13 * U[CS1] + m.gi33 * U[CS3];
  const T B1_ = P[B1], B2_ = P[B2], B3_ = P[B3];
  const T BvB1 = s.Bv * B1_, BvB2 = s.Bv * B2_, BvB3 = s.Bv * B3_;
  const T W11 = Su1 * s.v1 + s.ptot * m.gi11 - B1_ * B1_ * s.iW2 - BvB1 * s.v1;
  const T W13 = Su3 * s.v1 + s.ptot * m.gi13 - B1_ * B3_ * s.iW2 - BvB1 * s.v3;
  const T W22 = Su2 * s.v2 + s.ptot * m.gi22 - B2_ * B2_ * s.iW2 - BvB2 * s.v2;
  const T W33 = Su3 * s.v3 + s.ptot * m.gi33 - B3_ * B3_ * s.iW2 - BvB3 * s.v3;
  const T G1 = W11 * T(rec[C_DG11_1]) + T(2) * W13 * T(rec[C_DG13_1]) + W22 * T(rec[C_DG22_1]) +
               W33 * T(rec[C_DG33_1]);
  const T G2 = W11 * T(rec[C_DG11_2]) + T(2) * W13 * T(rec[C_DG13_2]) + W22 * T(rec[C_DG22_2]) +
               W33 * T(rec[C_DG33_2]);
  const T E = U[CTAU] + U[CD];
  S[CD] = T(0);
  S[CS1] = T(0.5) * m.al * G1 + U[CS1] * db11 - E * dal1;
  S[CS2] = T(0.5) * m.al * G2 + U[CS1] * db12 - E * dal2;
  S[CS3] = T(0);
  const T Wm11 = U[CS1] * s.v1 + s.ptot - B1_ * s.Bl1 * s.iW2 - BvB1 * s.vl1;  // W^1_1
  const T Wm21 = U[CS1] * s.v2 - B2_ * s.Bl1 * s.iW2 - BvB2 * s.vl1;           // W^2_1
  S[CTAU] = T(0.5) * m.be1 * G1 + Wm11 * db11 + Wm21 * db12 - (Su1 * dal1 + Su2 * dal2);
  S[B1] = T(0); S[B2] = T(0); S[B3] = T(0);
  S[PSI] = -m.al * kappa * P[PSI] - P[PSI] * db11 + ch2 * (B1_ * dal1 + B2_ * dal2);
}

// ----------------------------------------------------------------------------
// Conserved -> primitive inversion (FP64).  Two-dimensional Newton-Raphson in
// (Z = rho h W^2, v^2) on the momentum and energy equations (Noble et al.
// 2006), started from the previous primitives; converged when the step
// |dZ| <= tol Z (quadratic convergence: that iterate is accurate to
// round-off).  Backup: bisection on Z of the
// one-dimensional energy residual over a bracket grown from the guess.  Last
// resort: previous primitives (status 3).  Then floors (status 2).
// ----------------------------------------------------------------------------
template <typename T>
struct C2PQ {
  T D, E, S2, Bsq, BS;
};

template <typename T>
BHAC_HD T c2p_v2(const C2PQ<T>& q, T Z) {
  const T iZ = T(1.0) / Z;
  const T num = q.S2 + q.BS * q.BS * (T(2.0) * Z + q.Bsq) * iZ * iZ;
  const T ZB = Z + q.Bsq;
  return num / (ZB * ZB);
}

template <typename T>
BHAC_HD T c2p_f1d(const C2PQ<T>& q, T gf, T v2max, T Z) {
  T v2 = c2p_v2(q, Z);
  v2 = v2 > v2max ? v2max : v2;
  v2 = v2 < T(0.0) ? T(0.0) : v2;
  const T pr = gf * (Z * (T(1.0) - v2) - q.D * sqrt_t(T(1.0) - v2));
  return Z - pr + T(0.5) * q.Bsq * (T(1.0) + v2) - T(0.5) * q.BS * q.BS / (Z * Z) - q.E;
}

// A product rounded on its own: the inversion's steps (dZ, dv^2) come out of
// either solver as finished values, so the update Z + dZ is the same addition
// whichever solver a kernel carries (no fused multiply-add across the choice).
template <typename T>
BHAC_HD T mul_rn(T a, T b) {
  return a * b;
}
template <>
BHAC_HD double mul_rn<double>(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}

// Momentum and energy residuals of the two-dimensional system in (Z, v^2):
//   F1 = (Z + B^2)^2 v^2 - (B.S)^2 (2 Z + B^2) / Z^2 - S^2,
//   F2 = Z - p + B^2 (1 + v^2)/2 - (B.S)^2 / (2 Z^2) - E.
template <typename T>
BHAC_HD void c2p_residual_t(const C2PQ<T>& q, T gf, T Z, T v2, T& F1, T& F2) {
  const T omv = T(1.0) - v2;
  const T sq = omv * rsqrt_t(omv);
  const T pr = gf * (Z * omv - q.D * sq);
  const T iZ = rcp_t(Z);
  const T iZ2 = iZ * iZ;
  const T BS2 = q.BS * q.BS;
  const T ZB = Z + q.Bsq;
  F1 = ZB * ZB * v2 - BS2 * (T(2.0) * Z + q.Bsq) * iZ2 - q.S2;
  F2 = Z - pr + T(0.5) * q.Bsq * (T(1.0) + v2) - T(0.5) * BS2 * iZ2 - q.E;
}

// One Jacobian-free Newton-Krylov step at (Z, v^2): the system scaled by rows
// 1/(Z + B^2)^2 and 1/Z, unknowns (dZ/Z, dv^2); GMRES, whose Krylov space is
// the plane after two vectors, on products of the Jacobian with unit vectors
// taken as forward differences with step 2^-26 (backward where the forward
// point would leave 0 <= v^2 < 1).  Writes the step (dZ, dv^2).
template <typename T>
BHAC_HD void c2p_nk_step_t(const C2PQ<T>& q, T gf, T Z, T v2, T& dZ, T& dv2) {
  const T eps = T(1.4901161193847656e-08), ieps = T(67108864.0);  // 2^-26, 2^26
  const T ZB = Z + q.Bsq;
  const T rs0 = rcp_t(ZB * ZB), rs1 = rcp_t(Z);
  T F1, F2;
  c2p_residual_t(q, gf, Z, v2, F1, F2);
  const T G1 = rs0 * F1, G2 = rs1 * F2;
  const T beta = sqrt_t(G1 * G1 + G2 * G2);
  dZ = T(0.0);
  dv2 = T(0.0);
  if (!gt0_t(beta)) return;
  const T ib = rcp_t(beta);
  const T a1 = -G1 * ib, a2 = -G2 * ib;  // first basis vector
  // J a by a one-sided difference
  T sgn = T(1.0);
  {
    const T w = v2 + eps * a2;
    if (lt0_x(w) || le_x(T(1.0), w)) sgn = T(-1.0);
  }
  T P1, P2;
  c2p_residual_t(q, gf, Z + sgn * eps * a1 * Z, v2 + sgn * eps * a2, P1, P2);
  T j1 = (rs0 * P1 - G1) * (sgn * ieps), j2 = (rs1 * P2 - G2) * (sgn * ieps);
  const T h11 = j1 * a1 + j2 * a2;
  j1 = j1 - h11 * a1;
  j2 = j2 - h11 * a2;
  const T h21 = sqrt_t(j1 * j1 + j2 * j2);
  if (!lt_t(T(1e-14) * abs_t(h11), h21)) {  // a spans an invariant direction
    const T y = beta * rcp_t(h11);
    dZ = mul_rn(Z, y * a1);
    dv2 = mul_rn(y, a2);
    return;
  }
  const T i21 = rcp_t(h21);
  const T b1 = j1 * i21, b2 = j2 * i21;  // second basis vector
  sgn = T(1.0);
  {
    const T w = v2 + eps * b2;
    if (lt0_x(w) || le_x(T(1.0), w)) sgn = T(-1.0);
  }
  c2p_residual_t(q, gf, Z + sgn * eps * b1 * Z, v2 + sgn * eps * b2, P1, P2);
  T k1 = (rs0 * P1 - G1) * (sgn * ieps), k2 = (rs1 * P2 - G2) * (sgn * ieps);
  const T h12 = k1 * a1 + k2 * a2;
  k1 = k1 - h12 * a1;
  k2 = k2 - h12 * a2;
  const T h22 = k1 * b1 + k2 * b2;
  // min |beta e1 - H y| for the 2 x 2 Hessenberg H: a Givens rotation, then
  // back substitution
  const T r = sqrt_t(h11 * h11 + h21 * h21);
  const T ir = rcp_t(r);
  const T c = h11 * ir, sn = h21 * ir;
  const T R12 = c * h12 + sn * h22;
  const T R22 = -sn * h12 + c * h22;
  const T y1 = (-sn * beta) * rcp_t(R22);
  const T y0 = (c * beta - R12 * y1) * ir;
  dZ = mul_rn(Z, y0 * a1 + y1 * b1);
  dv2 = mul_rn(y0, a2) + mul_rn(y1, b2);
}

// Newton starting point from the previous primitives Pg: Z = (rho + Gamma/(Gamma - 1) p) W^2
// and v^2 = u^2 / W^2 with W^2 = 1 + u^2.
template <typename T>
BHAC_HD void c2p_guess(const Met<T>& m, const T* Pg, T gam_fac, T& Z0, T& v2) {
  const T gu1 = m.g11 * Pg[U1] + m.g13 * Pg[U3];
  const T gu2 = m.g22 * Pg[U2];
  const T gu3 = m.g13 * Pg[U1] + m.g33 * Pg[U3];
  const T usq = Pg[U1] * gu1 + Pg[U2] * gu2 + Pg[U3] * gu3;
  Z0 = (Pg[RHO] + gam_fac * Pg[PRS]) * (T(1.0) + usq);
  v2 = usq * rcp_t(T(1.0) + usq);
}

// U undensitized; (Z0g, v2g) the starting point (c2p_guess); Pg the previous
// primitives, variable v at Pg[v ps], read only when every solver fails;
// writes P; returns the status.  gf_d = (Gamma - 1)/Gamma and
// v2max_d = 1 - 1/W_max^2 come precomputed.
// NKM: the primary solver, 0 analytic Newton, 1 Newton-Krylov, 2 chosen at run
// time by nk (kernels that pick the solver at compile time carry no code of the
// other one).
template <typename T, int NKM = 2>
BHAC_HD int con2prim_t(const Met<T>& m, const T* U, const T* Pg, size_t ps, T Z0g, T v2g, T rho_fl, T p_fl,
                       double gf_d, double wmax_d, double v2max_d, double tol, int maxit, int nk, T* P) {
  const T gf = T(gf_d);
  const T wmax = T(wmax_d);
  const T v2max = T(v2max_d);
  C2PQ<T> q;
  q.D = U[CD];
  q.E = U[CTAU] + U[CD];
  const T Su1 = m.gi11 * U[CS1] + m.gi13 * U[CS3];
  const T Su2 = m.gi22 * U[CS2];
  const T Su3 = m.gi13 * U[CS1] + m.gi33 * U[CS3];
  const T Bl1 = m.g11 * U[B1] + m.g13 * U[B3];
  const T Bl2 = m.g22 * U[B2];
  const T Bl3 = m.g13 * U[B1] + m.g33 * U[B3];
  q.S2 = Su1 * U[CS1] + Su2 * U[CS2] + Su3 * U[CS3];
  q.Bsq = U[B1] * Bl1 + U[B2] * Bl2 + U[B3] * Bl3;
  q.BS = U[B1] * U[CS1] + U[B2] * U[CS2] + U[B3] * U[CS3];
  bool fin = true;
  for (int v = 0; v < NV; ++v) fin = fin && finite_t(U[v]);
  int status = 0;
  bool solved = false;
  T Z = T(0.0), v2 = T(0.0);
  T W = T(0.0), sq = T(0.0);  // 1/sqrt(1 - v^2) and sqrt(1 - v^2) of the accepted solution
  if (fin && gt0_t(q.D) && gt0_t(q.E)) {
    const T Z0 = (gt0_t(Z0g) && finite_t(Z0g)) ? Z0g : q.E;
    Z = Z0;
    v2 = v2g;
    const T BS2 = q.BS * q.BS;
    for (int it = 0; it < maxit; ++it) {
      T dZ, dv2;
      if (NKM == 1 || (NKM == 2 && nk)) {
        c2p_nk_step_t(q, gf, Z, v2, dZ, dv2);
      } else {
        const T omv = T(1.0) - v2;
        const T isq = rsqrt_t(omv);
        const T sq = omv * isq;
        const T pr = gf * (Z * omv - q.D * sq);
        const T iZ = rcp_t(Z);
        const T iZ2 = iZ * iZ;
        const T ZB = Z + q.Bsq;
        const T f1 = ZB * ZB * v2 - BS2 * (T(2.0) * Z + q.Bsq) * iZ2 - q.S2;
        const T f2 = Z - pr + T(0.5) * q.Bsq * (T(1.0) + v2) - T(0.5) * BS2 * iZ2 - q.E;
        const T j11 = T(2.0) * ZB * v2 + T(2.0) * BS2 * ZB * iZ2 * iZ;
        const T j12 = ZB * ZB;
        const T j21 = T(1.0) - gf * omv + BS2 * iZ2 * iZ;
        const T j22 = -gf * (-Z + T(0.5) * q.D * isq) + T(0.5) * q.Bsq;
        const T idet = rcp_t(j11 * j22 - j12 * j21);
        dZ = mul_rn(-f1 * j22 + f2 * j12, idet);
        dv2 = mul_rn(-f2 * j11 + f1 * j21, idet);
      }
      T Zn = Z + dZ, v2n = v2 + dv2;
      if (!gt0_t(Zn)) Zn = T(0.5) * Z;
      if (lt0_x(v2n)) v2n = T(0.5) * v2;
      if (le_x(T(1.0), v2n)) v2n = T(0.5) * (v2 + T(1.0));
      const bool conv = le_x(abs_t(Zn - Z), T(tol) * Zn);
      Z = Zn;
      v2 = v2n;
      if (!finite_t(Z) || !finite_t(v2)) break;
      if (conv) {
        solved = true;
        break;
      }
    }
    if (solved && !(le_x(T(0.0), v2) && lt_t(v2, T(1.0)) && gt0_t(Z))) solved = false;
    // the recovered density D sqrt(1 - v^2) must be positive; sqrt(1 - v^2)
    // is formed as (1 - v^2) / sqrt(1 - v^2), the factor the recovery uses
    if (solved) {
      W = rsqrt_t(T(1.0) - v2);
      sq = (T(1.0) - v2) * W;
      if (!gt0_t(q.D * sq)) solved = false;
    }
    if (!solved) {
      T lo = Z0, hi = Z0;
      int k = 0;
      while (c2p_f1d(q, gf, v2max, lo) > T(0.0) && k < 200) {
        lo = lo * T(0.5);
        ++k;
      }
      k = 0;
      while (c2p_f1d(q, gf, v2max, hi) < T(0.0) && k < 200) {
        hi = hi * T(2.0);
        ++k;
      }
      if (c2p_f1d(q, gf, v2max, lo) <= T(0.0) && c2p_f1d(q, gf, v2max, hi) >= T(0.0)) {
        for (int it = 0; it < 200 && hi - lo > T(4e-16) * hi; ++it) {
          const T mid = T(0.5) * (lo + hi);
          if (c2p_f1d(q, gf, v2max, mid) > T(0.0))
            hi = mid;
          else
            lo = mid;
        }
        Z = T(0.5) * (lo + hi);
        v2 = c2p_v2(q, Z);
        v2 = v2 > v2max ? v2max : v2;
        v2 = v2 < T(0.0) ? T(0.0) : v2;
        if (finite_t(Z) && Z > T(0.0)) {
          solved = true;
          status = 1;
          W = rsqrt_t(T(1.0) - v2);
          sq = (T(1.0) - v2) * W;
        }
      }
    }
  }
  if (solved) {
    // W = 1/sqrt(1 - v^2) and sqrt(1 - v^2) came from one reciprocal square
    // root; 1/Z and 1/(Z + B^2) from one reciprocal of their product
    const T omv = T(1.0) - v2;
    const T ZB = Z + q.Bsq;
    const T r = rcp_t(Z * ZB);
    P[RHO] = q.D * sq;
    P[PRS] = gf * (Z * omv - q.D * sq);
    const T c = W * Z * r;
    const T bz = q.BS * ZB * r;
    P[U1] = c * (Su1 + bz * U[B1]);
    P[U2] = c * (Su2 + bz * U[B2]);
    P[U3] = c * (Su3 + bz * U[B3]);
  } else {
    status = 3;
    P[RHO] = Pg[RHO * ps];
    P[PRS] = Pg[PRS * ps];
    P[U1] = Pg[U1 * ps];
    P[U2] = Pg[U2 * ps];
    P[U3] = Pg[U3 * ps];
  }
  P[B1] = U[B1];
  P[B2] = U[B2];
  P[B3] = U[B3];
  P[PSI] = U[PSI];
  bool fl = false;
  if (!le_x(rho_fl, P[RHO])) {
    P[RHO] = rho_fl;
    fl = true;
  }
  if (!le_x(p_fl, P[PRS])) {
    P[PRS] = p_fl;
    fl = true;
  }
  const T gu1 = m.g11 * P[U1] + m.g13 * P[U3];
  const T gu2 = m.g22 * P[U2];
  const T gu3 = m.g13 * P[U1] + m.g33 * P[U3];
  const T usq = P[U1] * gu1 + P[U2] * gu2 + P[U3] * gu3;
  if (lt_t(wmax * wmax, T(1.0) + usq)) {
    const T sc = sqrt_t((wmax * wmax - T(1.0)) / usq);
    P[U1] = P[U1] * sc;
    P[U2] = P[U2] * sc;
    P[U3] = P[U3] * sc;
    fl = true;
  }
  if (status == 3) return 3;
  return fl ? 2 : status;
}

template <int NKM>
static __device__ __forceinline__ int con2prim(const Met<double>& m, const double* U, const double* Pg, size_t ps,
                                            double Z0, double v20, double rho_fl, double p_fl, const StageArgs& a,
                                            double* P) {
  return con2prim_t<double, NKM>(m, U, Pg, ps, Z0, v20, rho_fl, p_fl, a.c2p_gf, a.wmax, a.c2p_v2max, a.c2p_tol,
                                 a.c2p_maxit, a.c2p_nk, P);
}

// CFL rate of one cell: sum over active d of c_d / dx_d, where c_d is the
// largest of |lambda+-| and ch alpha sqrt(gamma^dd) + |beta^d|.
template <typename T, int DIM>
BHAC_HD T cfl_rate_t(const Met<T>& m, const T* acg, const T* P, double gam, double gam_fac, double ch,
                     const double* idx) {
  if (ch >= 1.0) {
    // The fast-magnetosonic bound boosts a comoving speed a < 1 and so never
    // leaves the light cone: with ch >= 1 the cleaning speed is the largest.
    T rate = T(0.0);
    for (int d = 0; d < DIM; ++d) rate = rate + (T(ch) * acg[d] + (d == 0 ? abs_t(m.be1) : T(0.0))) * T(idx[d]);
    return rate;
  }
  Derived<T> s;
  derive(m, P, T(gam_fac), s);
  T rate = T(0.0);
  for (int d = 0; d < DIM; ++d) {
    T lm, lp;
    speeds_of(m, P, s, d, T(gam), lm, lp);
    const T alp = abs_t(lp), alm = abs_t(lm);
    T c = alp > alm ? alp : alm;
    const T cg = T(ch) * acg[d] + (d == 0 ? abs_t(m.be1) : T(0.0));
    c = cg > c ? cg : c;
    rate = rate + c * T(idx[d]);
  }
  return rate;
}

// ----------------------------------------------------------------------------
// Riemann solve at one face: states PL, PR (already reconstructed), face
// metric m, GLM speed factor acg = alpha sqrt(gamma^dd).  HLL or TVDLF; the
// GLM pair (normal B, psi) uses signal speeds no smaller than
// +-ch alpha sqrt(gamma^dd) - beta^d.  Writes the flux densitized by sqrt(gamma).
// ----------------------------------------------------------------------------
template <typename T>
BHAC_HD void riemann_flux(const Met<T>& m, T acg, const T* PL, const T* PR, int d, int riemann, T gam, T gam_fac,
                          T ch, T* out) {
  const T ch2 = ch * ch;
  Derived<T> sL, sR;
  derive(m, PL, gam_fac, sL);
  derive(m, PR, gam_fac, sR);
  T lmL, lpL, lmR, lpR;
  speeds_of(m, PL, sL, d, gam, lmL, lpL);
  speeds_of(m, PR, sR, d, gam, lmR, lpR);
  const T bed = d == 0 ? m.be1 : T(0);
  const T lgp = acg * ch - bed, lgm = -acg * ch - bed;
  T acc[NV];
  T U[NV], F[NV];
  if (riemann == 0) {
    T lp = T(0), lm = T(0);
    lp = lt_t(lp, lpL) ? lpL : lp;
    lp = lt_t(lp, lpR) ? lpR : lp;
    lm = lt_t(lmL, lm) ? lmL : lm;
    lm = lt_t(lmR, lm) ? lmR : lm;
    const T lpg = lt_t(lp, lgp) ? lgp : lp, lmg = lt_t(lgm, lm) ? lgm : lm;
    const T wh = lp - lm, wg = lpg - lmg;
    const bool okh = gt0_t(wh), okg = gt0_t(wg);
    // both fan widths' reciprocals from one division
    const T r = okh && okg ? rcp_t(wh * wg) : T(0);
    const T ih = okh ? (okg ? wg * r : rcp_t(wh)) : T(0);
    const T ihg = okg ? (okh ? wh * r : rcp_t(wg)) : T(0);
    cons_of(PL, sL, U);
    flux_of(m, PL, sL, U, d, ch2, F);
    T FL[NV];
    for (int v = 0; v < NV; ++v) {
      const bool g = (v == PSI) || (v == B1 + d);
      const T p = g ? lpg : lp, q = g ? lmg : lm;
      acc[v] = p * (F[v] - q * U[v]);
      FL[v] = F[v];
    }
    cons_of(PR, sR, U);
    flux_of(m, PR, sR, U, d, ch2, F);
    for (int v = 0; v < NV; ++v) {
      const bool g = (v == PSI) || (v == B1 + d);
      const T p = g ? lpg : lp, q = g ? lmg : lm, ihv = g ? ihg : ih;
      // a degenerate fan (no signal speed at all) falls back to the mean flux
      out[v] = m.sg * ((g ? okg : okh) ? (acc[v] - q * (F[v] - p * U[v])) * ihv : T(0.5) * (FL[v] + F[v]));
    }
  } else {
    const T alpL = abs_t(lpL), almL = abs_t(lmL), alpR = abs_t(lpR), almR = abs_t(lmR);
    T c = alpL;
    c = lt_t(c, almL) ? almL : c;
    c = lt_t(c, alpR) ? alpR : c;
    c = lt_t(c, almR) ? almR : c;
    const T agp = abs_t(lgp), agm = abs_t(lgm);
    T cg = c;
    cg = lt_t(cg, agp) ? agp : cg;
    cg = lt_t(cg, agm) ? agm : cg;
    cons_of(PL, sL, U);
    flux_of(m, PL, sL, U, d, ch2, F);
    for (int v = 0; v < NV; ++v) {
      const bool g = (v == PSI) || (v == B1 + d);
      acc[v] = F[v] + (g ? cg : c) * U[v];
    }
    cons_of(PR, sR, U);
    flux_of(m, PR, sR, U, d, ch2, F);
    for (int v = 0; v < NV; ++v) {
      const bool g = (v == PSI) || (v == B1 + d);
      out[v] = m.sg * (T(0.5) * (acc[v] + F[v]) - T(0.5) * (g ? cg : c) * U[v]);
    }
  }
}

// ----------------------------------------------------------------------------
// Face fluxes, densitized by the face sqrt(gamma).  (ig, jg, kg): ghosted
// coordinates of the cell on the high side of the face; (I1, I2): level-global
// table indices of the face.
// ----------------------------------------------------------------------------
// Axis faces carry no flux (sqrt(gamma) = 0 there).
template <bool FLAT>
__device__ __forceinline__ bool axis_face(const StageArgs& a, const LevelGeo& geo, int d, int I2) {
  return !FLAT && d == 1 && ((I2 == 0 && a.axis_lo1) || (I2 == geo.N2 && a.axis_hi1));
}

// Reconstructed states with a non-positive density or pressure fall back to
// the two adjacent cell values (first order).  c0: ghosted index of the high cell.
template <typename T>
__device__ __forceinline__ void positivity_fallback(const StageArgs& a, const T* __restrict__ Pb, int sd, int c0,
                                                    T PL[NV], T PR[NV]) {
  if (!gt0_t(PL[RHO]) || !gt0_t(PL[PRS]) || !gt0_t(PR[RHO]) || !gt0_t(PR[PRS])) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* p = Pb + (size_t)v * a.ncell + c0;
      PL[v] = p[-sd];
      PR[v] = p[0];
    }
  }
}

// Face metric and Riemann solve of the states PL, PR.
template <typename T, bool FLAT>
__device__ __forceinline__ void face_solve(const StageArgs& a, const LevelGeo& geo, int d, int I1, int I2,
                                           const T PL[NV], const T PR[NV], T* out, int ostride) {
  Met<T> m;
  T acg;
  if (FLAT) {
    m = flat_metric<T>();
    acg = T(1);
  } else if (sizeof(T) == 8) {
    const double* rec = d == 0 ? geo.tf1 + (size_t)(I2 * (geo.N1 + 1) + I1) * FREC
                               : (d == 1 ? geo.tf2 + (size_t)(I2 * geo.N1 + I1) * FREC
                                         : geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC);
    m = load_face_metric<T>(rec);
    acg = T(d == 2 ? rec[C_ACG3] : rec[F_ACG]);
  } else {
    const float* rec = d == 0 ? geo.tf1_32 + (size_t)(I2 * (geo.N1 + 1) + I1) * FREC
                              : (d == 1 ? geo.tf2_32 + (size_t)(I2 * geo.N1 + I1) * FREC
                                        : geo.tc32 + (size_t)(I2 * geo.N1 + I1) * CREC);
    m = load_face_metric<T>(rec);
    acg = T(d == 2 ? rec[C_ACG3] : rec[F_ACG]);
  }
  T F[NV];
  riemann_flux(m, acg, PL, PR, d, a.riemann, pick<T>(a.gam, a.gam_f), pick<T>(a.gam_fac, a.gam_fac_f),
               pick<T>(a.ch, a.ch_f), F);
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v * ostride] = F[v];
}

// One face flux from the six-point stencil across the face (the
// warp-specialised kernel's per-face form).
template <typename T, bool FLAT>
__device__ __forceinline__ void face_flux(const StageArgs& a, const LevelGeo& geo, const T* __restrict__ Pb, int d,
                                          int ig, int jg, int kg, int I1, int I2, T* out, int ostride) {
  const int sd = d == 0 ? 1 : (d == 1 ? a.Nx : a.Nx * a.Ny);
  const int c0 = (kg * a.Ny + jg) * a.Nx + ig;
  if (axis_face<FLAT>(a, geo, d, I2)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * ostride] = T(0);
    return;
  }
  T PL[NV], PR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T* p = Pb + (size_t)v * a.ncell + c0;
    const T s0 = p[-3 * sd], s1 = p[-2 * sd], s2 = p[-sd], s3 = p[0], s4 = p[sd], s5 = p[2 * sd];
    recon_var(a.recon, s0, s1, s2, s3, s4, s5, PL[v], PR[v]);
  }
  positivity_fallback(a, Pb, sd, c0, PL, PR);
  face_solve<T, FLAT>(a, geo, d, I1, I2, PL, PR, out, ostride);
}

// Both reconstructed edges along d of the cell at ghosted index c, all
// variables: aL (low face) to L[v * sl], aR (high face) to R[v * sr].
template <typename T>
__device__ __forceinline__ void cell_edges(const StageArgs& a, const T* __restrict__ Pb, int sd, int c, T* L, int sl,
                                           T* R, int sr) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T* p = Pb + (size_t)v * a.ncell + c;
    T l, r;
    recon_edges(a.recon, p[-2 * sd], p[-sd], p[0], p[sd], p[2 * sd], l, r);
    L[v * sl] = l;
    R[v * sr] = r;
  }
}

// A face flux from the two adjacent cells' edges: the low cell's aR (eL,
// stride es) and the high cell's aL (eR).
template <typename T, bool FLAT>
__device__ __forceinline__ void edge_face(const StageArgs& a, const LevelGeo& geo, const T* __restrict__ Pb, int d,
                                          int ig, int jg, int kg, int I1, int I2, const T* eL, const T* eR, int es,
                                          T* out, int ostride) {
  if (axis_face<FLAT>(a, geo, d, I2)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * ostride] = T(0);
    return;
  }
  const int sd = d == 0 ? 1 : (d == 1 ? a.Nx : a.Nx * a.Ny);
  const int c0 = (kg * a.Ny + jg) * a.Nx + ig;
  T PL[NV], PR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    PL[v] = eL[v * es];
    PR[v] = eR[v * es];
  }
  positivity_fallback(a, Pb, sd, c0, PL, PR);
  face_solve<T, FLAT>(a, geo, d, I1, I2, PL, PR, out, ostride);
}

// Copies a block-boundary face flux into the face's register (faces between
// refinement levels only).  fc: index of the face cell in the register, over
// the two transverse dimensions in ascending order.
template <typename T>
__device__ __forceinline__ void to_register(const StageArgs& a, int b, int d, int side, int fc, const T* F,
                                            int stride) {
  const long long off = a.regoff[b * 6 + 2 * d + side];
  if (off < 0) return;
  const int ncf = d == 0 ? a.ny * a.nz : (d == 1 ? a.nx * a.nz : a.nx * a.ny);
#pragma unroll
  for (int v = 0; v < NV; ++v) a.reg[off + (long long)v * ncf + fc] = to_double(F[v * stride]);
}

// Inversion, floors, outputs, counters and (stage 2) the CFL rate of a cell
// whose stage conserved state U (densitized) is final.  The Newton iteration,
// floors and CFL rate are FP64 in both forms.  In the mixed form (T = float)
// the Newton starting point comes from the FP32 previous primitives (G32;
// callers that hold their own FP64 starting point pass G32 = false) and a
// floored cell's D, S_i, tau are rebuilt in FP32.
template <typename T, int DIM, bool FLAT, bool G32 = (sizeof(T) == 4), int NKM = 2>
__device__ __forceinline__ void finish_cell(const StageArgs& a, const LevelGeo& geo, int b, int ci, int cg, int I1,
                                            int I2, double U[NV], unsigned cnt[4], double& rate_max) {
  const double* crec = FLAT ? nullptr : geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC;
  const float* crec32 = (FLAT || sizeof(T) == 8) ? nullptr : geo.tc32 + (size_t)(I2 * geo.N1 + I1) * CREC;
  const double sg = FLAT ? 1.0 : crec[C_SG];
  const double isg = FLAT ? 1.0 : crec[C_ISG];
  const double rho_fl = FLAT ? a.rho_fl_c : crec[C_RHOFL];
  const double p_fl = FLAT ? a.p_fl_c : crec[C_PFL];
  Met<double> md = FLAT ? flat_metric<double>() : load_centre_metric<double>(crec);
  Met<float> m32;
  if (sizeof(T) == 4) m32 = FLAT ? flat_metric<float>() : load_centre_metric<float>(crec32);
  double Uu[NV], Pn[NV];
  const double* Pd = a.P_in + (size_t)b * NV * a.ncell + cg;
#pragma unroll
  for (int v = 0; v < NV; ++v) Uu[v] = U[v] * isg;
  int st;
  if (G32) {
    // mixed form: the Newton starting point from the FP32 previous primitives
    // (a starting point needs no FP64); the FP64 ones are read only if every
    // solver fails
    const float* P3 = a.P32_in + (size_t)b * NV * a.ncell + cg;
    float Pg32[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      Pg32[v] = (v == RHO || v == PRS || v == U1 || v == U2 || v == U3) ? P3[(size_t)v * a.ncell] : 0.0f;
    float z0, w0;
    c2p_guess<float>(m32, Pg32, a.gam_fac_f, z0, w0);
    st = con2prim<NKM>(md, Uu, Pd, (size_t)a.ncell, widen_f32(z0), widen_f32(w0), rho_fl, p_fl, a, Pn);
  } else {
    double Pg[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Pg[v] = Pd[(size_t)v * a.ncell];
    double z0, w0;
    c2p_guess<double>(md, Pg, a.gam_fac, z0, w0);
    st = con2prim<NKM>(md, Uu, Pg, 1, z0, w0, rho_fl, p_fl, a, Pn);
  }
  cnt[st] += 1u;
  a.status[(size_t)b * a.nint + ci] = (unsigned char)st;
  float P32[NV];
  if (sizeof(T) == 4) {
#pragma unroll
    for (int v = 0; v < NV; ++v) P32[v] = narrow_f64(Pn[v]);
  }
  if (st >= 2) {
    if (sizeof(T) == 4) {
      // mixed form: the floored state's D, S_i, tau in FP32 (the field and psi
      // are left as they are); FP64 form: every conserved variable in FP64
      Derived<float> s;
      derive(m32, P32, a.gam_fac_f, s);
      float Uc[NV];
      cons_of(P32, s, Uc);
      const float sg32 = FLAT ? 1.0f : crec32[C_SG];
#pragma unroll
      for (int v = CD; v <= CTAU; ++v) U[v] = widen_f32(sg32 * Uc[v]);
    } else {
      Derived<double> s;
      derive(md, Pn, a.gam_fac, s);
      cons_of(Pn, s, Uu);
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = sg * Uu[v];
    }
  }
  const size_t ub = (size_t)b * NV * a.nint + ci;
  double* Po = a.P_out + (size_t)b * NV * a.ncell + cg;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    a.Uout[ub + (size_t)v * a.nint] = U[v];
    Po[(size_t)v * a.ncell] = Pn[v];
  }
  if (sizeof(T) == 4) {
    float* P3o = a.P32_out + (size_t)b * NV * a.ncell + cg;
#pragma unroll
    for (int v = 0; v < NV; ++v) P3o[(size_t)v * a.ncell] = P32[v];
  }
  if (a.stage == 2) {
    double acg[3] = {1.0, 1.0, 1.0};
    if (!FLAT) {
      acg[0] = crec[C_ACG1];
      acg[1] = crec[C_ACG2];
      acg[2] = crec[C_ACG3];
    }
    rate_max = fmax(rate_max, cfl_rate_t<double, DIM>(md, acg, Pn, a.gam, a.gam_fac, a.ch, geo.idx));
  }
}

__device__ __forceinline__ double stage_dt(const StageArgs& a) {
  if (a.dt_host > 0.0) return a.dt_host;
  if (a.stage == 1) return a.cfl / __longlong_as_double((long long)*a.smax_in);
  return *a.dt_dev;
}

__device__ __forceinline__ void reduce_outputs(const StageArgs& a, const unsigned cnt[4], double rate_max) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const unsigned tot = __reduce_add_sync(0xffffffffu, cnt[s]);
    if (lane == 0 && tot) atomicAdd(a.counts + s, (unsigned long long)tot);
  }
  if (a.stage == 2) {
    const double w = warp_max_d(rate_max);
    if (lane == 0) atomicMax(a.smax_out, (unsigned long long)__double_as_longlong(w));
  }
}

template <typename T, int DIM, bool FLAT, int NKM = 2>
__device__ __forceinline__ void rk_finish(const StageArgs& a, const LevelGeo& geo, int b, int ci, int cg, int I1, int I2,
                                          int bi, int bj, int k, const double rhs[NV], double dt, unsigned cfb,
                                          unsigned cnt[4], double& rate_max);

// Divergence of the face fluxes staged in shared memory, sources, RK stage
// combination and (unless the reflux pass owns the cell) the inversion of cell
// c of plane k in the tile at (x0, y0) of block b.
template <typename T, int DIM, bool FLAT, bool SPLIT, int NKM = 2>
__device__ __forceinline__ void cell_update(const StageArgs& a, const LevelGeo& geo, const T* __restrict__ Pb, int b,
                                            int x0, int y0, int k, int c, const T* Fx, const T* Fy, const T* Fz0,
                                            const T* Fz1, double dt, unsigned cfb, unsigned cnt[4],
                                            double& rate_max) {
  const int tx = a.tx, ty = a.ty;
  const int sFx = ty * (tx + 1), sFy = (ty + 1) * tx, sFz = tx * ty;
  const int kg = k + a.gz;
  const int I1b = a.blk[4 * b + 1] * a.nx + x0, I2b = a.blk[4 * b + 2] * a.ny + y0;
  const int i = c % tx, j = c / tx;
  const int ig = i + x0 + a.gx, jg = j + y0 + a.gy;
  const int cg = (kg * a.Ny + jg) * a.Nx + ig;
  const int ci = (k * a.ny + (j + y0)) * a.nx + (i + x0);
  const int I1 = I1b + i, I2 = I2b + j;
  // flux divergence in the flux arithmetic T (FP32 in the mixed form, whose
  // face fluxes carry FP32 rounding already), then widened once per variable
  T rdiv[NV];
  const T ix = pick<T>(geo.idx[0], geo.idx_f[0]), iy = pick<T>(geo.idx[1], geo.idx_f[1]),
          iz = pick<T>(geo.idx[2], geo.idx_f[2]);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T r = -(Fx[v * sFx + j * (tx + 1) + i + 1] - Fx[v * sFx + j * (tx + 1) + i]) * ix;
    r = r - (Fy[v * sFy + (j + 1) * tx + i] - Fy[v * sFy + j * tx + i]) * iy;
    if (DIM == 3) r = r - (Fz1[v * sFz + c] - Fz0[v * sFz + c]) * iz;
    rdiv[v] = r;
  }
  double rhs[NV];
  // explicit damping rate of the cleaning source (with IMEX it is implicit)
  const double kap_x = a.imex ? 0.0 : a.kappa;
  const float kap_xf = a.imex ? 0.f : a.kappa_f;
  // sources from the cell's primitives
  {
    T Pc[NV], Uc[NV], S[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Pc[v] = Pb[(size_t)v * a.ncell + cg];
    if (FLAT) {
      rdiv[PSI] = rdiv[PSI] - pick<T>(kap_x, kap_xf) * Pc[PSI];
#pragma unroll
      for (int v = 0; v < NV; ++v) rhs[v] = to_double(rdiv[v]);
    } else {
      const double* crec = geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC;
      Met<T> m;
      if (sizeof(T) == 8) {
        m = load_centre_metric<T>(crec);
      } else {
        m = load_centre_metric<T>(geo.tc32 + (size_t)(I2 * geo.N1 + I1) * CREC);
      }
      Derived<T> s;
      derive(m, Pc, pick<T>(a.gam_fac, a.gam_fac_f), s);
      cons_of(Pc, s, Uc);
      if (sizeof(T) == 8)
        sources_of(m, crec, Pc, s, Uc, pick<T>(kap_x, kap_xf), pick<T>(a.ch * a.ch, a.ch2_f), S);
      else
        sources_of(m, geo.tc32 + (size_t)(I2 * geo.N1 + I1) * CREC, Pc, s, Uc, pick<T>(kap_x, kap_xf),
                   pick<T>(a.ch * a.ch, a.ch2_f),
                   S);
      if (sizeof(T) == 8) {
        const double sg = crec[C_SG];
#pragma unroll
        for (int v = 0; v < NV; ++v) rhs[v] = to_double(rdiv[v]) + sg * to_double(S[v]);
      } else {
        const T sg = T(geo.tc32[(size_t)(I2 * geo.N1 + I1) * CREC + C_SG]);
#pragma unroll
        for (int v = 0; v < NV; ++v) rhs[v] = to_double(rdiv[v] + sg * S[v]);
      }
    }
  }
  if (SPLIT) {  // the cell kernel completes the stage from the stored right-hand side
    T* R = reinterpret_cast<T*>(a.R) + (size_t)b * NV * a.nint + ci;
#pragma unroll
    for (int v = 0; v < NV; ++v) R[(size_t)v * a.nint] = sizeof(T) == 4 ? (T)narrow_f64(rhs[v]) : (T)rhs[v];
    return;
  }
  rk_finish<T, DIM, FLAT, NKM>(a, geo, b, ci, cg, I1, I2, x0 + i, y0 + j, k, rhs, dt, cfb, cnt, rate_max);
}

// RK combination (and the IMEX damping), then the inversion, floors, outputs
// and CFL rate of cell (bi, bj, k) of block b, given the stage right-hand side.
template <typename T, int DIM, bool FLAT, int NKM>
__device__ __forceinline__ void rk_finish(const StageArgs& a, const LevelGeo& geo, int b, int ci, int cg, int I1, int I2,
                                          int bi, int bj, int k, const double rhs[NV], double dt, unsigned cfb,
                                          unsigned cnt[4], double& rate_max) {
  const size_t ub = (size_t)b * NV * a.nint + ci;
  double U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double un = a.Un[ub + (size_t)v * a.nint];
    if (a.stage == 1)
      U[v] = un + dt * rhs[v];
    else
      U[v] = 0.5 * un + 0.5 * (a.U1[ub + (size_t)v * a.nint] + dt * rhs[v]);
  }
  if (a.imex) {
    // IMEX-SSP2(2,2,2) for the damping -lam psi (lam = alpha kappa, z = lam dt):
    // Y1 = psi_n/(1 + g z); stage 1: Y2 = (psi_n + dt F(Y1) - (1 - 2g) z Y1)/(1 + g z);
    // stage 2: psi = psi_n/2 + (Y2 + dt F(Y2))/2 - z (1 - g) Y2 / 2 - g z Y1
    const double al = FLAT ? 1.0 : geo.tc[(size_t)(I2 * geo.N1 + I1) * CREC + C_AL];
    const double z = al * a.kappa * dt, g = a.imex_g;
    const double un = a.Un[ub + (size_t)PSI * a.nint];
    const double y1 = un / (1.0 + g * z);
    if (a.stage == 1) {
      U[PSI] = (un + dt * rhs[PSI] - (1.0 - 2.0 * g) * z * y1) / (1.0 + g * z);
    } else {
      const double u1 = a.U1[ub + (size_t)PSI * a.nint];
      U[PSI] = 0.5 * un + 0.5 * (u1 + dt * rhs[PSI]) - 0.5 * z * (1.0 - g) * u1 - g * z * y1;
    }
  }
  // cells next to a face bordering finer blocks are finished by the reflux pass
  const bool later = cfb && (((cfb & 1u) && bi == 0) || ((cfb & 2u) && bi == a.nx - 1) ||
                             ((cfb & 4u) && bj == 0) || ((cfb & 8u) && bj == a.ny - 1) ||
                             ((cfb & 16u) && k == 0) || ((cfb & 32u) && k == a.nz - 1));
  if (later) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a.Uout[ub + (size_t)v * a.nint] = U[v];
  } else {
    finish_cell<T, DIM, FLAT, (sizeof(T) == 4), NKM>(a, geo, b, ci, cg, I1, I2, U, cnt, rate_max);
  }
}

// ----------------------------------------------------------------------------
// The stage kernel.  T: flux arithmetic (double: FP64 form; float: mixed form).
// Every block of every level is an item of the same launch.
//
// Per plane k of the CTA's column, three phases separated by CTA barriers:
//  R  every cell's two reconstructed edges along x (the tile plus one cell on
//     each x side) and along y (plus one cell on each y side) into shared
//     memory; in 3-D each z column also reconstructs its cell of plane k+1,
//     solves the z face between planes k and k+1 from that cell's low edge
//     and plane k's high edge (kept in shared memory from the previous
//     plane), and keeps plane k+1's high edge for the next plane;
//  F  the x and y face fluxes from the edges of the two adjacent cells;
//  C  the cell updates.
// Each cell's edges are reconstructed once per direction (up to the one-cell
// tile halo) instead of once for each of its two faces; the face states are
// the same numbers as a per-face reconstruction's.
//
// Shared memory (T): Fx, Fy, [Fz0, Fz1, EzR in 3-D], ExL, ExR, EyL, EyR.
//
// MINB: the register bound (resident CTAs per SM) in its last digit; + 10: the
// face kernel of the split form (no inversion code); + 100: the Newton-Krylov
// inversion in place of the analytic Newton step.
// ----------------------------------------------------------------------------
template <typename T, int DIM, bool FLAT, int MINB>
__global__ void __launch_bounds__(256, MINB % 10) stage_kernel(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tx = a.tx, ty = a.ty;
  const int sFx = ty * (tx + 1), sFy = (ty + 1) * tx, sFz = tx * ty;
  const int nex = (tx + 2) * ty, ney = tx * (ty + 2);
  T* Fx = reinterpret_cast<T*>(smem_raw);
  T* Fy = Fx + NV * sFx;
  T* Fza = Fy + NV * sFy;
  T* Fzb = Fza + (DIM == 3 ? NV * sFz : 0);
  T* EzR = Fzb + (DIM == 3 ? NV * sFz : 0);
  T* ExL = EzR + (DIM == 3 ? NV * sFz : 0);
  T* ExR = ExL + NV * nex;
  T* EyL = ExR + NV * nex;
  T* EyR = EyL + NV * ney;
  __shared__ int s_item;

  const double dt = stage_dt(a);
  if (a.stage == 1 && blockIdx.x == 0 && threadIdx.x == 0) *a.dt_dev = dt;

  const T* Pb_all = sizeof(T) == 8 ? reinterpret_cast<const T*>(a.P_in) : reinterpret_cast<const T*>(a.P32_in);
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const int ntile = a.ntx * a.nty;
  const int sy = a.Nx, sz = a.Nx * a.Ny;
  const int nzc = DIM == 3 ? sFz : 0;

  int item = a.persistent ? -1 : (int)blockIdx.x + a.item0;
  for (;;) {
    if (a.persistent) {
      __syncthreads();
      if (threadIdx.x == 0) s_item = a.item0 + (int)atomicAdd(a.work, 1u);
      __syncthreads();
      item = s_item;
    }
    if (item >= a.item1) break;
    // item = (visiting-order block, tile, z part); a part runs planes [kbeg, kend)
    const int zp = item % a.nzp, it2 = item / a.nzp;
    const int ord = it2 / ntile;
    const int b = a.order[ord];
    const int tile = it2 - ord * ntile;
    const int kbeg = zp * (a.nz / a.nzp), kend = kbeg + a.nz / a.nzp;
    const int x0 = (tile % a.ntx) * tx, y0 = (tile / a.ntx) * ty;
    const int L = a.blk[4 * b];
    const LevelGeo geo = level_geo(a, L);
    const int bx = a.blk[4 * b + 1], by = a.blk[4 * b + 2];
    const int I1b = bx * a.nx + x0, I2b = by * a.ny + y0;
    const T* Pb = Pb_all + (size_t)b * NV * a.ncell;
    const unsigned cfb = a.nlev > 1 ? a.cf[b] : 0u;
    const bool regs = a.nlev > 1;
    T* Fz0 = Fza;
    T* Fz1 = Fzb;
    if (DIM == 3) {
      // bottom face of plane kbeg from the high edge of plane kbeg - 1 and the
      // low edge of plane kbeg; plane kbeg's high edge is kept for the face
      // above it (the same arithmetic as the face carried up from below)
      for (int t = threadIdx.x; t < sFz; t += blockDim.x) {
        const int i = t % tx, j = t / tx;
        const int ig = i + x0 + a.gx, jg = j + y0 + a.gy;
        const int c0 = ((kbeg + a.gz) * a.Ny + jg) * a.Nx + ig;
        T PL[NV], PR[NV], tmp[NV];
        if (axis_face<FLAT>(a, geo, 2, I2b + j)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) Fz0[v * sFz + t] = T(0);
        } else {
          cell_edges(a, Pb, sz, c0 - sz, tmp, 1, PL, 1);
          cell_edges(a, Pb, sz, c0, PR, 1, EzR + t, sFz);
          positivity_fallback(a, Pb, sz, c0, PL, PR);
          face_solve<T, FLAT>(a, geo, 2, I1b + i, I2b + j, PL, PR, Fz0 + t, sFz);
        }
        if (regs && kbeg == 0) to_register(a, b, 2, 0, (j + y0) * a.nx + i + x0, Fz0 + t, sFz);
      }
    }
    for (int k = kbeg; k < kend; ++k) {
      const int kg = k + a.gz;
      // R: edges (and the z face above plane k)
      for (int t = threadIdx.x; t < nzc + nex + ney; t += blockDim.x) {
        if (t < nzc) {
          const int i = t % tx, j = t / tx;
          const int ig = i + x0 + a.gx, jg = j + y0 + a.gy;
          const int c1 = ((kg + 1) * a.Ny + jg) * a.Nx + ig;
          T PL[NV], PR[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) PL[v] = EzR[v * sFz + t];
          cell_edges(a, Pb, sz, c1, PR, 1, EzR + t, sFz);
          positivity_fallback(a, Pb, sz, c1, PL, PR);
          face_solve<T, FLAT>(a, geo, 2, I1b + i, I2b + j, PL, PR, Fz1 + t, sFz);
          if (regs && k + 1 == a.nz) to_register(a, b, 2, 1, (j + y0) * a.nx + i + x0, Fz1 + t, sFz);
        } else if (t < nzc + nex) {
          const int u = t - nzc;
          const int i = u % (tx + 2) - 1, j = u / (tx + 2);
          const int c = (kg * a.Ny + j + y0 + a.gy) * a.Nx + i + x0 + a.gx;
          cell_edges(a, Pb, 1, c, ExL + u, nex, ExR + u, nex);
        } else {
          const int u = t - nzc - nex;
          const int i = u % tx, j = u / tx - 1;
          const int c = (kg * a.Ny + j + y0 + a.gy) * a.Nx + i + x0 + a.gx;
          cell_edges(a, Pb, sy, c, EyL + u, ney, EyR + u, ney);
        }
      }
      __syncthreads();
      // F: x and y faces
      for (int t = threadIdx.x; t < sFx + sFy; t += blockDim.x) {
        if (t < sFx) {
          const int i = t % (tx + 1), j = t / (tx + 1);
          const int e = j * (tx + 2) + i;  // edge slot of the low cell
          edge_face<T, FLAT>(a, geo, Pb, 0, i + x0 + a.gx, j + y0 + a.gy, kg, I1b + i, I2b + j, ExR + e, ExL + e + 1,
                             nex, Fx + t, sFx);
          if (regs && (x0 + i == 0 || x0 + i == a.nx))
            to_register(a, b, 0, x0 + i == 0 ? 0 : 1, k * a.ny + j + y0, Fx + t, sFx);
        } else {
          const int u = t - sFx;
          const int i = u % tx, j = u / tx;
          edge_face<T, FLAT>(a, geo, Pb, 1, i + x0 + a.gx, j + y0 + a.gy, kg, I1b + i, I2b + j, EyR + u,
                             EyL + u + tx, ney, Fy + u, sFy);
          if (regs && (y0 + j == 0 || y0 + j == a.ny))
            to_register(a, b, 1, y0 + j == 0 ? 0 : 1, k * a.nx + i + x0, Fy + u, sFy);
        }
      }
      __syncthreads();
      // C: cell updates
      for (int c = threadIdx.x; c < sFz; c += blockDim.x)
        cell_update<T, DIM, FLAT, (MINB % 100 >= 10), (MINB >= 100 ? 1 : 0)>(a, geo, Pb, b, x0, y0, k, c, Fx, Fy, Fz0,
                                                                          Fz1, dt, cfb, cnt, rate_max);
      __syncthreads();
      T* tmp = Fz0;
      Fz0 = Fz1;
      Fz1 = tmp;
    }
    if (!a.persistent) break;
  }
  reduce_outputs(a, cnt, rate_max);
}

// ----------------------------------------------------------------------------
// Warp-specialised form of the 3-D stage kernel.  The first pwarps warps
// (producers) compute the face fluxes of plane k+1 while the other warps
// (consumers) update the cells of plane k, so the FP64 work of the cell
// updates is not interrupted by the face phase.  Face fluxes are double
// buffered (x and y faces per plane parity, z faces in three slots: plane k
// reads faces k and k+1 while plane k+1's producer writes face k+2); named
// barriers FULL[parity] (producers -> consumers) and EMPTY[parity]
// (consumers -> producers) hand the buffers over.  It reconstructs per face
// (recon_var), gives each role only part of the CTA's warps, and measured
// slower than the phased kernel on the tori; it is selected only by an
// explicit producer-warp count in bhac_set_launch.
// ----------------------------------------------------------------------------
// Named barriers (ids 1..4; 0 is __syncthreads).  Producer and consumer roles
// are whole warps; each warp reconverges before the barrier instruction.
__device__ __forceinline__ void named_sync(int id, int n) {
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  __syncwarp();
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
constexpr int BAR_FULL = 1, BAR_EMPTY = 3;

template <typename T, bool FLAT>
__device__ __forceinline__ void produce_plane(const StageArgs& a, const LevelGeo& geo, const T* __restrict__ Pb, int b,
                                              int x0, int y0, int k, bool bottom, T* Fx, T* Fy, T* Fzlo, T* Fzhi,
                                              int ptid, int nprod) {
  const int tx = a.tx, ty = a.ty;
  const int sFx = ty * (tx + 1), sFy = (ty + 1) * tx, sFz = tx * ty;
  const int I1b = a.blk[4 * b + 1] * a.nx + x0, I2b = a.blk[4 * b + 2] * a.ny + y0;
  const bool regs = a.nlev > 1;
  const int kg = k + a.gz;
  const int nb = bottom ? sFz : 0;
  const int n = nb + sFx + sFy + sFz;
  for (int t = ptid; t < n; t += nprod) {
    if (t < nb) {
      const int i = t % tx, j = t / tx;
      face_flux<T, FLAT>(a, geo, Pb, 2, i + x0 + a.gx, j + y0 + a.gy, kg, I1b + i, I2b + j, Fzlo + t, sFz);
      if (regs) to_register(a, b, 2, 0, (j + y0) * a.nx + i + x0, Fzlo + t, sFz);
      continue;
    }
    const int u0 = t - nb;
    if (u0 < sFx) {
      const int i = u0 % (tx + 1), j = u0 / (tx + 1);
      face_flux<T, FLAT>(a, geo, Pb, 0, i + x0 + a.gx, j + y0 + a.gy, kg, I1b + i, I2b + j, Fx + u0, sFx);
      if (regs && (x0 + i == 0 || x0 + i == a.nx)) to_register(a, b, 0, x0 + i == 0 ? 0 : 1, k * a.ny + j + y0, Fx + u0, sFx);
    } else if (u0 < sFx + sFy) {
      const int u = u0 - sFx;
      const int i = u % tx, j = u / tx;
      face_flux<T, FLAT>(a, geo, Pb, 1, i + x0 + a.gx, j + y0 + a.gy, kg, I1b + i, I2b + j, Fy + u, sFy);
      if (regs && (y0 + j == 0 || y0 + j == a.ny)) to_register(a, b, 1, y0 + j == 0 ? 0 : 1, k * a.nx + i + x0, Fy + u, sFy);
    } else {
      const int u = u0 - sFx - sFy;
      const int i = u % tx, j = u / tx;
      face_flux<T, FLAT>(a, geo, Pb, 2, i + x0 + a.gx, j + y0 + a.gy, kg + 1, I1b + i, I2b + j, Fzhi + u, sFz);
      if (regs && k + 1 == a.nz) to_register(a, b, 2, 1, (j + y0) * a.nx + i + x0, Fzhi + u, sFz);
    }
  }
}

template <typename T, bool FLAT, int MINB>
__global__ void __launch_bounds__(256, MINB) stage_kernel_ws(StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tx = a.tx, ty = a.ty;
  const int sFx = ty * (tx + 1), sFy = (ty + 1) * tx, sFz = tx * ty;
  T* base = reinterpret_cast<T*>(smem_raw);
  T* FxB[2] = {base, base + NV * sFx};
  T* FyB[2] = {base + 2 * NV * sFx, base + 2 * NV * sFx + NV * sFy};
  T* FzB[3];
  for (int q = 0; q < 3; ++q) FzB[q] = base + 2 * NV * (sFx + sFy) + q * NV * sFz;
  __shared__ int s_item;

  const double dt = stage_dt(a);
  if (a.stage == 1 && blockIdx.x == 0 && threadIdx.x == 0) *a.dt_dev = dt;
  const T* Pb_all = sizeof(T) == 8 ? reinterpret_cast<const T*>(a.P_in) : reinterpret_cast<const T*>(a.P32_in);
  const int nthr = blockDim.x, nprod = a.pwarps * 32, ncons = nthr - nprod;
  const bool producer = (int)threadIdx.x < nprod;
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const int ntile = a.ntx * a.nty;
  int item = a.persistent ? -1 : (int)blockIdx.x;
  for (;;) {
    if (a.persistent) {
      __syncthreads();
      if (threadIdx.x == 0) s_item = (int)atomicAdd(a.work, 1u);
      __syncthreads();
      item = s_item;
    }
    if (item >= a.nitems) break;
    const int ord = item / ntile;
    const int b = a.order[ord];
    const int tile = item - ord * ntile;
    const int x0 = (tile % a.ntx) * tx, y0 = (tile / a.ntx) * ty;
    const LevelGeo geo = level_geo(a, a.blk[4 * b]);
    const T* Pb = Pb_all + (size_t)b * NV * a.ncell;
    const unsigned cfb = a.nlev > 1 ? a.cf[b] : 0u;
    if (producer) {
      for (int k = 0; k < a.nz; ++k) {
        const int par = k & 1;
        if (k >= 2) named_sync(BAR_EMPTY + par, nthr);
        produce_plane<T, FLAT>(a, geo, Pb, b, x0, y0, k, k == 0, FxB[par], FyB[par], FzB[k % 3], FzB[(k + 1) % 3],
                               threadIdx.x, nprod);
        __threadfence_block();
        named_arrive(BAR_FULL + par, nthr);
      }
      // take the consumers' last releases so every barrier starts the next item clean
      for (int k = a.nz - 2 < 0 ? 0 : a.nz - 2; k < a.nz; ++k) named_sync(BAR_EMPTY + (k & 1), nthr);
    } else {
      for (int k = 0; k < a.nz; ++k) {
        const int par = k & 1;
        named_sync(BAR_FULL + par, nthr);
        for (int c = threadIdx.x - nprod; c < sFz; c += ncons)
          cell_update<T, 3, FLAT, false>(a, geo, Pb, b, x0, y0, k, c, FxB[par], FyB[par], FzB[k % 3], FzB[(k + 1) % 3], dt,
                                  cfb, cnt, rate_max);
        __threadfence_block();
        named_arrive(BAR_EMPTY + par, nthr);
      }
    }
    if (!a.persistent) break;
  }
  reduce_outputs(a, cnt, rate_max);
}

// Split form, second kernel: one thread per interior cell of the items
// [item0, item1): the stage right-hand side the face kernel stored, then
// rk_finish (the same arithmetic as the fused kernel).
template <typename T, int DIM, bool FLAT>
__global__ void __launch_bounds__(256) cell_kernel(StageArgs a) {
  const double dt = stage_dt(a);
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const int tx = a.tx, ty = a.ty, ntile = a.ntx * a.nty;
  const long long per = (long long)tx * ty * a.nz;
  const long long n = (long long)(a.item1 - a.item0) * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int item = a.item0 + (int)(t / per);
    const int rem = (int)(t - (long long)(item - a.item0) * per);
    const int k = rem / (tx * ty), c = rem - k * tx * ty;
    const int i = c % tx, j = c / tx;
    const int ord = item / ntile;
    const int b = a.order[ord];
    const int tile = item - ord * ntile;
    const int bi = (tile % a.ntx) * tx + i, bj = (tile / a.ntx) * ty + j;
    const int ci = (k * a.ny + bj) * a.nx + bi;
    const int cg = ((k + a.gz) * a.Ny + (bj + a.gy)) * a.Nx + (bi + a.gx);
    const LevelGeo geo = level_geo(a, a.blk[4 * b]);
    const int I1 = a.blk[4 * b + 1] * a.nx + bi, I2 = a.blk[4 * b + 2] * a.ny + bj;
    const unsigned cfb = a.nlev > 1 ? a.cf[b] : 0u;
    const T* R = reinterpret_cast<const T*>(a.R) + (size_t)b * NV * a.nint + ci;
    double rhs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) rhs[v] = to_double(R[(size_t)v * a.nint]);
    rk_finish<T, DIM, FLAT>(a, geo, b, ci, cg, I1, I2, bi, bj, k, rhs, dt, cfb, cnt, rate_max);
  }
  reduce_outputs(a, cnt, rate_max);
}

template <typename T, int DIM, bool FLAT>
static cudaError_t launch_cells_t(const StageArgs& a, int grid, cudaStream_t st) {
  cell_kernel<T, DIM, FLAT><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cells_any(const StageArgs& a, int grid, cudaStream_t st) {
  if (a.ndim == 3) return a.flat ? launch_cells_t<T, 3, true>(a, grid, st) : launch_cells_t<T, 3, false>(a, grid, st);
  return a.flat ? launch_cells_t<T, 2, true>(a, grid, st) : launch_cells_t<T, 2, false>(a, grid, st);
}

// Coarse-fine flux correction: each listed coarse cell trades the coarse flux
// through a face bordering finer blocks for the mean of the fine fluxes that
// cover it (U += f dt (F_fine - F_coarse) / dx, sign by side, f = 1 in stage 1
// and 1/2 in stage 2), then is inverted like every other cell.
template <typename T, int DIM, bool FLAT>
__global__ void __launch_bounds__(128) reflux_kernel(StageArgs a) {
  const double dt = stage_dt(a);
  const double f = a.stage == 1 ? 1.0 : 0.5;
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const int n = a.nrcells;
  const int nthreads = gridDim.x * blockDim.x;
  const int rounds = (n + nthreads - 1) / nthreads;
  for (int r = 0; r < rounds; ++r) {
    const int t = r * nthreads + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) continue;
    const RefluxCell rc = a.rcells[t];
    const LevelGeo geo = level_geo(a, rc.level);
    const size_t ub = (size_t)rc.b * NV * a.nint + rc.ci;
    double U[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = a.Uout[ub + (size_t)v * a.nint];
    for (int q = 0; q < rc.nterm; ++q) {
      const RefluxTerm T_ = a.rterms[rc.term0 + q];
      const double w = f * dt * geo.idx[T_.d] * (double)T_.sign;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double acc = 0.0;
        for (int m = 0; m < T_.nfine; ++m) acc += a.reg[T_.fine[m] + (long long)v * T_.fstride];
        const double Ff = acc / T_.nfine;
        const double Fc = a.reg[T_.coarse + (long long)v * T_.cstride];
        // the IMEX first stage divides the explicit increment of psi by 1 + g z
        const double wv = (v == PSI && a.imex && a.stage == 1)
                              ? w / (1.0 + a.imex_g * geo.tc[(size_t)(rc.I2 * geo.N1 + rc.I1) * CREC + C_AL] * a.kappa * dt)
                              : w;
        U[v] += wv * (Ff - Fc);
      }
    }
    finish_cell<T, DIM, FLAT>(a, geo, rc.b, rc.ci, rc.cg, rc.I1, rc.I2, U, cnt, rate_max);
  }
  reduce_outputs(a, cnt, rate_max);
}

// Stand-alone CFL rate reduction over interior cells (FP64 primitives); a
// grid-stride loop over (block, cell) with 32-bit index arithmetic (the
// library's grids hold fewer than 2^31 interior cells).
template <int DIM, bool FLAT>
__global__ void __launch_bounds__(256) cfl_kernel(StageArgs a) {
  double rate_max = 0.0;
  const unsigned n = (unsigned)a.nblocks * (unsigned)a.nint;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)a.nint);
    const int ci = (int)(t - (unsigned)b * (unsigned)a.nint);
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    const LevelGeo geo = level_geo(a, a.blk[4 * b]);
    double P[NV];
    const double* Pd = a.P_in + (size_t)b * NV * a.ncell + cg;
#pragma unroll
    for (int v = 0; v < NV; ++v) P[v] = Pd[(size_t)v * a.ncell];
    Met<double> m = flat_metric<double>();
    double acg[3] = {1.0, 1.0, 1.0};
    if (!FLAT) {
      const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
      const double* crec = geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC;
      m = load_centre_metric<double>(crec);
      acg[0] = crec[C_ACG1];
      acg[1] = crec[C_ACG2];
      acg[2] = crec[C_ACG3];
    }
    rate_max = fmax(rate_max, cfl_rate_t<double, DIM>(m, acg, P, a.gam, a.gam_fac, a.ch, geo.idx));
  }
  const double w = warp_max_d(rate_max);
  if ((threadIdx.x & 31u) == 0) atomicMax(a.smax_out, (unsigned long long)__double_as_longlong(w));
}

// Loading a state in one pass: the interior primitives src ([block][var][cell],
// FP64) go to the ghosted FP64 array P and (mixed form) its FP32 copy P32; the
// densitized conserved state U follows from them, and the CFL rate of the
// loaded primitives is reduced into smax_out (the same per-cell rate as
// cfl_kernel's).  Same loop as cfl_kernel.
template <int DIM, bool FLAT>
__global__ void __launch_bounds__(256) load_kernel(StageArgs a, const double* __restrict__ src, double* P, float* P32,
                                                   double* U) {
  double rate_max = 0.0;
  const unsigned n = (unsigned)a.nblocks * (unsigned)a.nint;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)a.nint);
    const int ci = (int)(t - (unsigned)b * (unsigned)a.nint);
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    const LevelGeo geo = level_geo(a, a.blk[4 * b]);
    double Pc[NV], Uc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Pc[v] = src[((size_t)b * NV + v) * a.nint + ci];
      P[((size_t)b * NV + v) * a.ncell + cg] = Pc[v];
      if (P32) P32[((size_t)b * NV + v) * a.ncell + cg] = narrow_f64(Pc[v]);
    }
    Met<double> m = flat_metric<double>();
    double sg = 1.0;
    double acg[3] = {1.0, 1.0, 1.0};
    if (!FLAT) {
      const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
      const double* rec = geo.tc + (size_t)(I2 * geo.N1 + I1) * CREC;
      m = load_centre_metric<double>(rec);
      sg = rec[C_SG];
      acg[0] = rec[C_ACG1];
      acg[1] = rec[C_ACG2];
      acg[2] = rec[C_ACG3];
    }
    Derived<double> s;
    derive(m, Pc, a.gam_fac, s);
    cons_of(Pc, s, Uc);
#pragma unroll
    for (int v = 0; v < NV; ++v) U[((size_t)b * NV + v) * a.nint + ci] = sg * Uc[v];
    rate_max = fmax(rate_max, cfl_rate_t<double, DIM>(m, acg, Pc, a.gam, a.gam_fac, a.ch, geo.idx));
  }
  const double w = warp_max_d(rate_max);
  if ((threadIdx.x & 31u) == 0) atomicMax(a.smax_out, (unsigned long long)__double_as_longlong(w));
}

// Raises a kernel's dynamic shared-memory limit to kMaxDynSmem, or to what
// the device's opt-in limit leaves beside the kernel's static shared memory
// if that is less.
template <typename K>
static cudaError_t raise_smem_limit(K kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  int lim = optin - (int)fa.sharedSizeBytes;
  lim = lim < kMaxDynSmem ? lim : kMaxDynSmem;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <typename T, int DIM, bool FLAT, int MINB>
static cudaError_t configure_stage_t() {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = raise_smem_limit(stage_kernel<T, DIM, FLAT, MINB>);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return cudaSuccess;
}

template <typename T, bool FLAT, int MINB>
static cudaError_t configure_ws_t() {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = raise_smem_limit(stage_kernel_ws<T, FLAT, MINB>);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t configure_all_t() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = configure_stage_t<T, 2, true, 1>();
  if (e == cudaSuccess) e = configure_stage_t<T, 2, false, 1>();
  if (e == cudaSuccess) e = configure_stage_t<T, 3, true, 1>();
  if (e == cudaSuccess) e = configure_stage_t<T, 3, false, 1>();
  if (e == cudaSuccess) e = configure_stage_t<T, 3, true, 2>();
  if (e == cudaSuccess) e = configure_stage_t<T, 3, false, 2>();
  if (e == cudaSuccess) e = configure_ws_t<T, true, 1>();
  if (e == cudaSuccess) e = configure_ws_t<T, false, 1>();
  if (e == cudaSuccess) e = configure_ws_t<T, true, 2>();
  if (e == cudaSuccess) e = configure_ws_t<T, false, 2>();
  return e;
}

template <typename T, int DIM, bool FLAT>
static cudaError_t launch_reflux_t(const StageArgs& a, cudaStream_t st);

template <typename T, int DIM, bool FLAT, int MINB>
static cudaError_t launch_stage_t(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  cudaError_t e;
  if constexpr (DIM == 3 && MINB < 10) {
    if (a.pwarps > 0) {
      e = configure_ws_t<T, FLAT, MINB>();
      if (e != cudaSuccess) return e;
      stage_kernel_ws<T, FLAT, MINB><<<grid, threads, smem, st>>>(a);
      e = cudaGetLastError();
      if (e != cudaSuccess || a.nrcells == 0 || a.split) return e;
      return launch_reflux_t<T, DIM, FLAT>(a, st);
    }
  }
  {
    e = configure_stage_t<T, DIM, FLAT, MINB>();
    if (e != cudaSuccess) return e;
    stage_kernel<T, DIM, FLAT, MINB><<<grid, threads, smem, st>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || a.nrcells == 0 || a.split) return e;
  return launch_reflux_t<T, DIM, FLAT>(a, st);
}

template <typename T, int DIM, bool FLAT>
static cudaError_t launch_reflux_t(const StageArgs& a, cudaStream_t st) {
  int g = (a.nrcells + 127) / 128;
  reflux_kernel<T, DIM, FLAT><<<g, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_reflux_any(const StageArgs& a, cudaStream_t st) {
  if (a.nrcells == 0) return cudaSuccess;
  if (a.ndim == 3) return a.flat ? launch_reflux_t<T, 3, true>(a, st) : launch_reflux_t<T, 3, false>(a, st);
  return a.flat ? launch_reflux_t<T, 2, true>(a, st) : launch_reflux_t<T, 2, false>(a, st);
}

// Resident CTAs per SM of the phased 3-D kernel that launch_stage_any would
// launch for these arguments (non-split), at this CTA size and shared memory.
template <typename T, bool FLAT, int MINB>
static int occupancy_t(int threads, size_t smem) {
  if (configure_stage_t<T, 3, FLAT, MINB>() != cudaSuccess) return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<T, 3, FLAT, MINB>, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

template <typename T>
static int stage_occupancy_any(const StageArgs& a, int threads, size_t smem) {
  if (a.c2p_nk)
    return a.minb >= 2 ? (a.flat ? occupancy_t<T, true, 102>(threads, smem) : occupancy_t<T, false, 102>(threads, smem))
                       : (a.flat ? occupancy_t<T, true, 101>(threads, smem) : occupancy_t<T, false, 101>(threads, smem));
  return a.minb >= 2 ? (a.flat ? occupancy_t<T, true, 2>(threads, smem) : occupancy_t<T, false, 2>(threads, smem))
                     : (a.flat ? occupancy_t<T, true, 1>(threads, smem) : occupancy_t<T, false, 1>(threads, smem));
}

// 3-D kernels exist with one or two resident CTAs per SM as the register
// bound; 2-D grids use the one-CTA form.
template <typename T>
static cudaError_t launch_stage_any(const StageArgs& a, int grid, int threads, size_t smem, cudaStream_t st) {
  if (a.split) {
    if (a.ndim == 3) {
      if (a.minb == 3)
        return a.flat ? launch_stage_t<T, 3, true, 13>(a, grid, threads, smem, st)
                      : launch_stage_t<T, 3, false, 13>(a, grid, threads, smem, st);
      if (a.minb == 2)
        return a.flat ? launch_stage_t<T, 3, true, 12>(a, grid, threads, smem, st)
                      : launch_stage_t<T, 3, false, 12>(a, grid, threads, smem, st);
      return a.flat ? launch_stage_t<T, 3, true, 11>(a, grid, threads, smem, st)
                    : launch_stage_t<T, 3, false, 11>(a, grid, threads, smem, st);
    }
    return a.flat ? launch_stage_t<T, 2, true, 11>(a, grid, threads, smem, st)
                  : launch_stage_t<T, 2, false, 11>(a, grid, threads, smem, st);
  }
  if (a.c2p_nk && a.pwarps == 0) {  // the Newton-Krylov inversion compiled in
    if (a.ndim == 3) {
      if (a.minb >= 2)
        return a.flat ? launch_stage_t<T, 3, true, 102>(a, grid, threads, smem, st)
                      : launch_stage_t<T, 3, false, 102>(a, grid, threads, smem, st);
      return a.flat ? launch_stage_t<T, 3, true, 101>(a, grid, threads, smem, st)
                    : launch_stage_t<T, 3, false, 101>(a, grid, threads, smem, st);
    }
    return a.flat ? launch_stage_t<T, 2, true, 101>(a, grid, threads, smem, st)
                  : launch_stage_t<T, 2, false, 101>(a, grid, threads, smem, st);
  }
  if (a.ndim == 3) {
    if (a.minb >= 2)
      return a.flat ? launch_stage_t<T, 3, true, 2>(a, grid, threads, smem, st)
                    : launch_stage_t<T, 3, false, 2>(a, grid, threads, smem, st);
    return a.flat ? launch_stage_t<T, 3, true, 1>(a, grid, threads, smem, st)
                  : launch_stage_t<T, 3, false, 1>(a, grid, threads, smem, st);
  }
  return a.flat ? launch_stage_t<T, 2, true, 1>(a, grid, threads, smem, st)
                : launch_stage_t<T, 2, false, 1>(a, grid, threads, smem, st);
}

}  // namespace bhac
