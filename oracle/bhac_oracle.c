/*
 * Plain FP64 CPU oracle for the per-block finite-volume GRMHD update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * It follows the method of the paper's Sec. 2 ("Code overview"): a
 * shock-capturing finite-volume scheme on a block grid with ghost cells,
 * covariant coordinates, a second-order two-stage time stepper, PPM (or
 * minmod) reconstruction, and a Newton (or Jacobian-free Newton-Krylov)
 * conserved-to-primitive inversion with backup strategies.  The concrete equations are the standard 3+1 ("Valencia")
 * ideal GRMHD system with GLM divergence cleaning; each function names the
 * published form it writes out.  The code favours obviousness over speed:
 * metric quantities are re-evaluated at every point, nothing is fused.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps x86 and Arm results identical).
 */
#include "bhac_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Metric                                                                    */
/* ------------------------------------------------------------------------ */

/* Kerr-Schild spatial metric, lapse and shift (mass M, spin a) in code
 * coordinates, written for complex arguments so that derivatives follow from
 * the complex-step method (Squire & Trapp 1998): d f/dx = Im f(x + i h) / h.
 *   Sigma = r^2 + a^2 cos^2 th, z = 2 M r / Sigma
 *   gamma_rr = 1 + z, gamma_rph = -a sin^2 th (1 + z), gamma_thth = Sigma,
 *   gamma_phph = sin^2 th (Sigma + a^2 sin^2 th (1 + z)),
 *   alpha = 1/sqrt(1 + z), beta^r = z/(1 + z).
 * Modified KS: r = exp(x1), th = pi x2, ph = x3 (diagonal Jacobian). */
static void ks_metric_c(const or_params* p, const cplx x[3], cplx* alpha, cplx beta[3], cplx g[3][3]) {
  cplx r, th, drdx, dthdx;
  const double a = p->spin, M = p->mass;
  if (p->coords == OR_MKS) {
    r = cexp(x[0]);
    th = M_PI * x[1];
    drdx = r;
    dthdx = M_PI;
  } else {
    r = x[0];
    th = x[1];
    drdx = 1.0;
    dthdx = 1.0;
  }
  cplx s = csin(th), c = ccos(th);
  cplx Sigma = r * r + a * a * c * c;
  cplx z = 2.0 * M * r / Sigma;
  cplx grr = 1.0 + z;
  cplx grp = -a * s * s * (1.0 + z);
  cplx gtt = Sigma;
  cplx gpp = s * s * (Sigma + a * a * s * s * (1.0 + z));
  *alpha = 1.0 / csqrt(1.0 + z);
  beta[0] = z / (1.0 + z) / drdx;
  beta[1] = 0.0;
  beta[2] = 0.0;
  g[0][0] = grr * drdx * drdx;
  g[0][1] = 0.0;
  g[0][2] = grp * drdx;
  g[1][1] = gtt * dthdx * dthdx;
  g[1][2] = 0.0;
  g[2][2] = gpp;
  g[1][0] = g[0][1];
  g[2][0] = g[0][2];
  g[2][1] = g[1][2];
}

static double det3(const double g[3][3]) {
  return g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) - g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
         g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
}

/* Inverse by cofactors: gi = adj(g) / det(g). */
static void inv3(const double g[3][3], double gi[3][3]) {
  double d = det3(g);
  gi[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / d;
  gi[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / d;
  gi[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / d;
  gi[1][0] = (g[1][2] * g[2][0] - g[1][0] * g[2][2]) / d;
  gi[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / d;
  gi[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / d;
  gi[2][0] = (g[1][0] * g[2][1] - g[1][1] * g[2][0]) / d;
  gi[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / d;
  gi[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / d;
}

void or_metric_at(const or_params* p, const double x[3], int with_derivs, or_metric* m) {
  memset(m, 0, sizeof(*m));
  if (p->coords == OR_CART) {
    m->alpha = 1.0;
    for (int i = 0; i < 3; ++i) m->g[i][i] = m->gi[i][i] = 1.0;
    m->sqrtg = 1.0;
    return;
  }
  cplx xc[3] = {x[0], x[1], x[2]};
  cplx al, be[3], g[3][3];
  ks_metric_c(p, xc, &al, be, g);
  m->alpha = creal(al);
  for (int i = 0; i < 3; ++i) {
    m->beta[i] = creal(be[i]);
    for (int j = 0; j < 3; ++j) m->g[i][j] = creal(g[i][j]);
  }
  double d = det3(m->g);
  m->sqrtg = d > 0.0 ? sqrt(d) : 0.0;
  if (d > 0.0) inv3(m->g, m->gi);
  if (!with_derivs) return;
  const double h = 1e-30;
  for (int k = 0; k < 3; ++k) {
    cplx xp[3] = {x[0], x[1], x[2]};
    xp[k] += I * h;
    ks_metric_c(p, xp, &al, be, g);
    m->da[k] = cimag(al) / h;
    for (int i = 0; i < 3; ++i) {
      m->db[k][i] = cimag(be[i]) / h;
      for (int j = 0; j < 3; ++j) m->dg[k][i][j] = cimag(g[i][j]) / h;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Point-wise GRMHD (3+1 Valencia form; Anton et al. 2006, Del Zanna et al.  */
/* 2007; GLM after Dedner et al. 2002)                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rho, p, u[3], B[3], psi;
  double ul[3], u2, W, v[3], vl[3], v2;
  double Bl[3], B2, Bv, b2, rhoh, ptot;
} state;

static void make_state(const or_params* pp, const or_metric* m, const double P[OR_NV], state* s) {
  s->rho = P[OR_RHO];
  s->p = P[OR_P];
  for (int i = 0; i < 3; ++i) {
    s->u[i] = P[OR_U1 + i];
    s->B[i] = P[OR_B1 + i];
  }
  s->psi = P[OR_PSI];
  s->u2 = 0.0;
  s->B2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    s->ul[i] = 0.0;
    s->Bl[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
      s->ul[i] += m->g[i][j] * s->u[j];
      s->Bl[i] += m->g[i][j] * s->B[j];
    }
  }
  for (int i = 0; i < 3; ++i) {
    s->u2 += s->u[i] * s->ul[i];
    s->B2 += s->B[i] * s->Bl[i];
  }
  s->W = sqrt(1.0 + s->u2);
  s->Bv = 0.0;
  for (int i = 0; i < 3; ++i) {
    s->v[i] = s->u[i] / s->W;
    s->vl[i] = s->ul[i] / s->W;
    s->Bv += s->B[i] * s->vl[i];
  }
  s->v2 = s->u2 / (s->W * s->W);
  s->b2 = s->B2 / (s->W * s->W) + s->Bv * s->Bv;
  s->rhoh = s->rho + pp->gamma_ad / (pp->gamma_ad - 1.0) * s->p;
  s->ptot = s->p + 0.5 * s->b2;
}

/* D = rho W, S_j = (rho h W^2 + B^2) v_j - (B.v) B_j,
 * tau = rho h W^2 - p + B^2 - (B^2/W^2 + (B.v)^2)/2 - D. */
static void cons_of_state(const state* s, double U[OR_NV]) {
  double Z = s->rhoh * s->W * s->W;
  U[OR_D] = s->rho * s->W;
  for (int j = 0; j < 3; ++j) U[OR_S1 + j] = (Z + s->B2) * s->vl[j] - s->Bv * s->Bl[j];
  U[OR_TAU] = Z - s->p + s->B2 - 0.5 * s->b2 - U[OR_D];
  for (int j = 0; j < 3; ++j) U[OR_B1 + j] = s->B[j];
  U[OR_PSI] = s->psi;
}

void or_prim2con(const or_params* p, const or_metric* m, const double P[OR_NV], double U[OR_NV]) {
  state s;
  make_state(p, m, P, &s);
  cons_of_state(&s, U);
}

/* Mixed-index stress W^i_j = S_j v^i + p_tot delta^i_j - B^i B_j / W^2 - (B.v) B^i v_j. */
static double stress(const state* s, const double U[OR_NV], int i, int j) {
  double w = U[OR_S1 + j] * s->v[i] - s->B[i] * s->Bl[j] / (s->W * s->W) - s->Bv * s->B[i] * s->vl[j];
  if (i == j) w += s->ptot;
  return w;
}

/* Fluxes along direction i (undensitized):
 *   F(D)    = D (alpha v^i - beta^i)
 *   F(S_j)  = alpha W^i_j - beta^i S_j
 *   F(tau)  = alpha (S^i - D v^i) - beta^i tau
 *   F(B^j)  = (alpha v^i - beta^i) B^j - (alpha v^j - beta^j) B^i + alpha gamma^ij psi
 *   F(psi)  = alpha ch^2 B^i - beta^i psi */
static void flux_of_state(const or_params* p, const or_metric* m, const state* s, const double U[OR_NV], int i,
                          double F[OR_NV]) {
  const double al = m->alpha;
  F[OR_D] = U[OR_D] * (al * s->v[i] - m->beta[i]);
  for (int j = 0; j < 3; ++j) F[OR_S1 + j] = al * stress(s, U, i, j) - m->beta[i] * U[OR_S1 + j];
  double Si = 0.0;
  for (int j = 0; j < 3; ++j) Si += m->gi[i][j] * U[OR_S1 + j];
  F[OR_TAU] = al * (Si - U[OR_D] * s->v[i]) - m->beta[i] * U[OR_TAU];
  for (int j = 0; j < 3; ++j)
    F[OR_B1 + j] = (al * s->v[i] - m->beta[i]) * s->B[j] - (al * s->v[j] - m->beta[j]) * s->B[i] +
                   al * m->gi[i][j] * s->psi;
  F[OR_PSI] = al * p->ch * p->ch * s->B[i] - m->beta[i] * s->psi;
}

void or_flux(const or_params* p, const or_metric* m, const double P[OR_NV], int dir, double F[OR_NV]) {
  state s;
  double U[OR_NV];
  make_state(p, m, P, &s);
  cons_of_state(&s, U);
  flux_of_state(p, m, &s, U, dir, F);
}

/* Fast-magnetosonic speed bound (Del Zanna et al. 2007): in the fluid frame
 * a^2 = cs^2 + ca^2 - cs^2 ca^2, with cs^2 = Gamma p / (rho h) and
 * ca^2 = b^2 / (rho h + b^2); boosted to the Eulerian frame and shifted:
 *   lam = alpha/(1 - v^2 a^2) [v^i (1 - a^2) +- sqrt(a^2 (1 - v^2)
 *         (gamma^ii (1 - v^2 a^2) - v^i v^i (1 - a^2)))] - beta^i. */
static void speeds_of_state(const or_params* p, const or_metric* m, const state* s, int i, double* lm,
                            double* lp) {
  double cs2 = p->gamma_ad * s->p / s->rhoh;
  double ca2 = s->b2 / (s->rhoh + s->b2);
  double a2 = cs2 + ca2 - cs2 * ca2;
  double vi = s->v[i];
  double disc = a2 * (1.0 - s->v2) * (m->gi[i][i] * (1.0 - s->v2 * a2) - vi * vi * (1.0 - a2));
  if (disc < 0.0) disc = 0.0;
  double sq = sqrt(disc);
  double den = 1.0 - s->v2 * a2;
  *lp = m->alpha * (vi * (1.0 - a2) + sq) / den - m->beta[i];
  *lm = m->alpha * (vi * (1.0 - a2) - sq) / den - m->beta[i];
}

void or_wavespeeds(const or_params* p, const or_metric* m, const double P[OR_NV], int dir, double* lm,
                   double* lp) {
  state s;
  make_state(p, m, P, &s);
  speeds_of_state(p, m, &s, dir, lm, lp);
}

/* Geometric sources for a stationary metric (E = tau + D):
 *   S(S_j) = 1/2 alpha W^ik d_j gamma_ik + S_i d_j beta^i - E d_j alpha
 *   S(tau) = 1/2 W^ik beta^j d_j gamma_ik + W^j_i d_j beta^i - S^j d_j alpha
 *   S(psi) = -alpha kappa psi - psi d_i beta^i + ch^2 B^i d_i alpha
 *   S(D) = S(B^j) = 0. */
void or_sources(const or_params* p, const or_metric* m, const double P[OR_NV], double S[OR_NV]) {
  state s;
  double U[OR_NV], Wmix[3][3], Wup[3][3], Sup[3];
  make_state(p, m, P, &s);
  cons_of_state(&s, U);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Wmix[i][j] = stress(&s, U, i, j); /* W^i_j */
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      Wup[i][k] = 0.0;
      for (int l = 0; l < 3; ++l) Wup[i][k] += Wmix[i][l] * m->gi[l][k];
    }
  for (int i = 0; i < 3; ++i) {
    Sup[i] = 0.0;
    for (int j = 0; j < 3; ++j) Sup[i] += m->gi[i][j] * U[OR_S1 + j];
  }
  double E = U[OR_TAU] + U[OR_D];
  for (int v = 0; v < OR_NV; ++v) S[v] = 0.0;
  for (int j = 0; j < 3; ++j) {
    double a = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) a += 0.5 * m->alpha * Wup[i][k] * m->dg[j][i][k];
    for (int i = 0; i < 3; ++i) a += U[OR_S1 + i] * m->db[j][i];
    a -= E * m->da[j];
    S[OR_S1 + j] = a;
  }
  double t = 0.0;
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) t += 0.5 * Wup[i][k] * m->beta[j] * m->dg[j][i][k];
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) t += Wmix[j][i] * m->db[j][i];
  for (int j = 0; j < 3; ++j) t -= Sup[j] * m->da[j];
  S[OR_TAU] = t;
  double divb = m->db[0][0] + m->db[1][1] + m->db[2][2];
  double damp = p->imex ? 0.0 : p->kappa; /* with IMEX the damping is the implicit part */
  double ps = -m->alpha * damp * s.psi - s.psi * divb;
  for (int i = 0; i < 3; ++i) ps += p->ch * p->ch * s.B[i] * m->da[i];
  S[OR_PSI] = ps;
}

/* ------------------------------------------------------------------------ */
/* Conserved -> primitive inversion                                           */
/* ------------------------------------------------------------------------ */

/* Invariants of the conserved state used by the inversion. */
typedef struct {
  double D, E, S2, B2, BS, Sup[3], Bl[3];
} c2p_in;

/* Ideal-gas pressure as a function of Z = rho h W^2 and v^2:
 *   p = (Gamma-1)/Gamma (Z (1 - v^2) - D sqrt(1 - v^2)). */
static double c2p_pressure(double gam, double D, double Z, double v2) {
  return (gam - 1.0) / gam * (Z * (1.0 - v2) - D * sqrt(1.0 - v2));
}

/* v^2 implied by the momentum equation at a given Z:
 *   S^2 = (Z + B^2)^2 v^2 - (B.S)^2 (2 Z + B^2) / Z^2. */
static double c2p_v2_of_Z(const c2p_in* q, double Z) {
  double num = q->S2 + q->BS * q->BS * (2.0 * Z + q->B2) / (Z * Z);
  return num / ((Z + q->B2) * (Z + q->B2));
}

/* Energy residual of the one-dimensional formulation (v^2 clamped to [0, v2max]):
 *   f(Z) = Z - p + B^2 (1 + v^2)/2 - (B.S)^2/(2 Z^2) - E. */
static double c2p_f1d(const c2p_in* q, double gam, double v2max, double Z) {
  double v2 = c2p_v2_of_Z(q, Z);
  if (v2 > v2max) v2 = v2max;
  if (v2 < 0.0) v2 = 0.0;
  return Z - c2p_pressure(gam, q->D, Z, v2) + 0.5 * q->B2 * (1.0 + v2) - 0.5 * q->BS * q->BS / (Z * Z) - q->E;
}

static int finite9(const double* x) {
  for (int i = 0; i < OR_NV; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* Momentum and energy residuals of the two-dimensional system in (Z, v^2):
 *   F1 = (Z + B^2)^2 v^2 - (B.S)^2 (2 Z + B^2) / Z^2 - S^2,
 *   F2 = Z - p + B^2 (1 + v^2)/2 - (B.S)^2 / (2 Z^2) - E. */
static void c2p_residual(const c2p_in* q, double gf, double Z, double v2, double F[2]) {
  double sq = sqrt(1.0 - v2);
  double pr = gf * (Z * (1.0 - v2) - q->D * sq);
  double BS2 = q->BS * q->BS;
  F[0] = (Z + q->B2) * (Z + q->B2) * v2 - BS2 * (2.0 * Z + q->B2) / (Z * Z) - q->S2;
  F[1] = Z - pr + 0.5 * q->B2 * (1.0 + v2) - 0.5 * BS2 / (Z * Z) - q->E;
}

/* One Jacobian-free Newton-Krylov step for the residuals above, at (Z, v^2).
 * The system is scaled: rows by 1/(Z + B^2)^2 and 1/Z, the unknowns are
 * (dZ / Z, dv^2).  The Newton equation J s = -F is solved by GMRES, whose
 * Krylov space is the whole plane after two vectors, so two Arnoldi steps give
 * its solution; each product of J with a unit vector u is the forward
 * difference (G(x + eps u) - G(x)) / eps with eps = sqrt(machine epsilon),
 * taken backwards when the forward point would leave 0 <= v^2 < 1.  Returns
 * the step (dZ, dv^2). */
static void c2p_nk_step(const c2p_in* q, double gf, double Z, double v2, double* dZ, double* dv2) {
  const double eps = 1.4901161193847656e-08; /* 2^-26 */
  double rs[2] = {1.0 / ((Z + q->B2) * (Z + q->B2)), 1.0 / Z};
  double F[2], G0[2];
  c2p_residual(q, gf, Z, v2, F);
  G0[0] = rs[0] * F[0];
  G0[1] = rs[1] * F[1];
  double beta = sqrt(G0[0] * G0[0] + G0[1] * G0[1]);
  *dZ = 0.0;
  *dv2 = 0.0;
  if (!(beta > 0.0)) return;
  double V[2][2], Jv[2];
  V[0][0] = -G0[0] / beta;
  V[0][1] = -G0[1] / beta;
  double H[2][2] = {{0.0, 0.0}, {0.0, 0.0}}; /* H[row][col] of the Arnoldi relation */
  int m = 2;
  for (int k = 0; k < 2; ++k) {
    /* Jv = J V[k] by a one-sided difference */
    double h = eps;
    double w = v2 + h * V[k][1];
    if (w < 0.0 || w >= 1.0) h = -eps;
    double Fp[2];
    c2p_residual(q, gf, Z + h * V[k][0] * Z, v2 + h * V[k][1], Fp);
    Jv[0] = (rs[0] * Fp[0] - G0[0]) / h;
    Jv[1] = (rs[1] * Fp[1] - G0[1]) / h;
    /* modified Gram-Schmidt against the earlier basis vectors */
    for (int i = 0; i <= k; ++i) {
      H[i][k] = Jv[0] * V[i][0] + Jv[1] * V[i][1];
      Jv[0] -= H[i][k] * V[i][0];
      Jv[1] -= H[i][k] * V[i][1];
    }
    if (k == 0) {
      double h21 = sqrt(Jv[0] * Jv[0] + Jv[1] * Jv[1]);
      H[1][0] = h21;
      if (!(h21 > 1e-14 * fabs(H[0][0]))) { /* V[0] spans an invariant direction */
        m = 1;
        break;
      }
      V[1][0] = Jv[0] / h21;
      V[1][1] = Jv[1] / h21;
    }
  }
  double y[2];
  if (m == 1) {
    y[0] = beta / H[0][0];
    y[1] = 0.0;
  } else {
    /* least squares min |beta e1 - H y| for the 2 x 2 Hessenberg H (exact in
     * the plane): one Givens rotation, then back substitution */
    double r = sqrt(H[0][0] * H[0][0] + H[1][0] * H[1][0]);
    double c = H[0][0] / r, sn = H[1][0] / r;
    double R12 = c * H[0][1] + sn * H[1][1];
    double R22 = -sn * H[0][1] + c * H[1][1];
    double g0 = c * beta, g1 = -sn * beta;
    y[1] = g1 / R22;
    y[0] = (g0 - R12 * y[1]) / r;
  }
  double s0 = y[0] * V[0][0] + y[1] * (m == 2 ? V[1][0] : 0.0);
  double s1 = y[0] * V[0][1] + y[1] * (m == 2 ? V[1][1] : 0.0);
  *dZ = Z * s0;
  *dv2 = s1;
}

/* Primary solver: two-dimensional Newton-Raphson in (Z, v^2) on the momentum
 * and energy equations (the "2D" scheme of Noble et al. 2006), or with
 * p->c2p_nk the Jacobian-free Newton-Krylov step above in its place, started
 * from the previous primitives; stop when the step |dZ| <= tol Z (the
 * iteration converges quadratically, so that iterate is accurate to
 * round-off).
 * Backup: bracketed bisection on Z of the one-dimensional energy residual.
 * Last resort: keep the previous primitives (status 3).  Floors last. */
int or_con2prim(const or_params* p, const or_metric* m, const double U[OR_NV], const double Pg[OR_NV],
                double r_floor, double P[OR_NV]) {
  const double gam = p->gamma_ad, gf = (gam - 1.0) / gam;
  const double v2max = 1.0 - 1.0 / (p->w_max * p->w_max);
  c2p_in q;
  q.D = U[OR_D];
  q.E = U[OR_TAU] + U[OR_D];
  for (int i = 0; i < 3; ++i) {
    q.Sup[i] = 0.0;
    q.Bl[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
      q.Sup[i] += m->gi[i][j] * U[OR_S1 + j];
      q.Bl[i] += m->g[i][j] * U[OR_B1 + j];
    }
  }
  q.S2 = q.B2 = q.BS = 0.0;
  for (int i = 0; i < 3; ++i) {
    q.S2 += q.Sup[i] * U[OR_S1 + i];
    q.B2 += U[OR_B1 + i] * q.Bl[i];
    q.BS += U[OR_B1 + i] * U[OR_S1 + i];
  }
  int status = 0;
  double Z = 0.0, v2 = 0.0;
  int solved = 0;
  if (finite9(U) && q.D > 0.0 && q.E > 0.0) {
    /* initial guess from the previous primitives */
    double ul[3], u2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      ul[i] = 0.0;
      for (int j = 0; j < 3; ++j) ul[i] += m->g[i][j] * Pg[OR_U1 + j];
    }
    for (int i = 0; i < 3; ++i) u2 += Pg[OR_U1 + i] * ul[i];
    Z = (Pg[OR_RHO] + gam / (gam - 1.0) * Pg[OR_P]) * (1.0 + u2);
    v2 = u2 / (1.0 + u2);
    if (!(Z > 0.0) || !isfinite(Z)) Z = q.E;
    for (int it = 0; it < p->c2p_maxit; ++it) {
      double dZ, dv2;
      if (p->c2p_nk) {
        c2p_nk_step(&q, gf, Z, v2, &dZ, &dv2);
      } else {
        double sq = sqrt(1.0 - v2);
        double pr = gf * (Z * (1.0 - v2) - q.D * sq);
        double BS2 = q.BS * q.BS;
        double f1 = (Z + q.B2) * (Z + q.B2) * v2 - BS2 * (2.0 * Z + q.B2) / (Z * Z) - q.S2;
        double f2 = Z - pr + 0.5 * q.B2 * (1.0 + v2) - 0.5 * BS2 / (Z * Z) - q.E;
        double j11 = 2.0 * (Z + q.B2) * v2 + 2.0 * BS2 * (Z + q.B2) / (Z * Z * Z);
        double j12 = (Z + q.B2) * (Z + q.B2);
        double dpdZ = gf * (1.0 - v2);
        double dpdv2 = gf * (-Z + 0.5 * q.D / sq);
        double j21 = 1.0 - dpdZ + BS2 / (Z * Z * Z);
        double j22 = -dpdv2 + 0.5 * q.B2;
        double det = j11 * j22 - j12 * j21;
        dZ = (-f1 * j22 + f2 * j12) / det;
        dv2 = (-f2 * j11 + f1 * j21) / det;
      }
      double Zn = Z + dZ, v2n = v2 + dv2;
      if (!(Zn > 0.0)) Zn = 0.5 * Z;
      if (v2n < 0.0) v2n = 0.5 * v2;
      if (v2n >= 1.0) v2n = 0.5 * (v2 + 1.0);
      int conv = fabs(Zn - Z) <= p->c2p_tol * Zn;
      Z = Zn;
      v2 = v2n;
      if (!isfinite(Z) || !isfinite(v2)) break;
      if (conv) {
        solved = 1;
        break;
      }
    }
    if (solved && !(v2 >= 0.0 && v2 < 1.0 && Z > 0.0)) solved = 0;
    if (solved) {
      double W = 1.0 / sqrt(1.0 - v2);
      if (!(q.D / W > 0.0)) solved = 0;
    }
    if (!solved) {
      /* backup: bisection on the bracketed one-dimensional residual */
      double Z0 = (Pg[OR_RHO] + gam / (gam - 1.0) * Pg[OR_P]) * (1.0 + u2);
      if (!(Z0 > 0.0) || !isfinite(Z0)) Z0 = q.E;
      double lo = Z0, hi = Z0;
      int k = 0;
      while (c2p_f1d(&q, gam, v2max, lo) > 0.0 && k < 200) {
        lo *= 0.5;
        ++k;
      }
      k = 0;
      while (c2p_f1d(&q, gam, v2max, hi) < 0.0 && k < 200) {
        hi *= 2.0;
        ++k;
      }
      if (c2p_f1d(&q, gam, v2max, lo) <= 0.0 && c2p_f1d(&q, gam, v2max, hi) >= 0.0) {
        for (int it = 0; it < 200 && hi - lo > 4e-16 * hi; ++it) {
          double mid = 0.5 * (lo + hi);
          if (c2p_f1d(&q, gam, v2max, mid) > 0.0)
            hi = mid;
          else
            lo = mid;
        }
        Z = 0.5 * (lo + hi);
        v2 = c2p_v2_of_Z(&q, Z);
        if (v2 > v2max) v2 = v2max;
        if (v2 < 0.0) v2 = 0.0;
        if (isfinite(Z) && Z > 0.0) {
          solved = 1;
          status = 1;
        }
      }
    }
  }
  if (solved) {
    double W = 1.0 / sqrt(1.0 - v2);
    P[OR_RHO] = q.D / W;
    P[OR_P] = c2p_pressure(gam, q.D, Z, v2);
    for (int i = 0; i < 3; ++i) P[OR_U1 + i] = W * (q.Sup[i] + q.BS / Z * U[OR_B1 + i]) / (Z + q.B2);
  } else {
    status = 3;
    P[OR_RHO] = Pg[OR_RHO];
    P[OR_P] = Pg[OR_P];
    for (int i = 0; i < 3; ++i) P[OR_U1 + i] = Pg[OR_U1 + i];
  }
  for (int i = 0; i < 3; ++i) P[OR_B1 + i] = U[OR_B1 + i];
  P[OR_PSI] = U[OR_PSI];
  /* floors: rho >= rho_fl r^k1, p >= p_fl r^k2, W <= W_max */
  int fl = 0;
  double rfl = p->rho_floor * pow(r_floor, p->rho_floor_pow);
  double pfl = p->p_floor * pow(r_floor, p->p_floor_pow);
  if (!(P[OR_RHO] >= rfl)) {
    P[OR_RHO] = rfl;
    fl = 1;
  }
  if (!(P[OR_P] >= pfl)) {
    P[OR_P] = pfl;
    fl = 1;
  }
  double u2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) u2 += m->g[i][j] * P[OR_U1 + i] * P[OR_U1 + j];
  if (1.0 + u2 > p->w_max * p->w_max) {
    double s = sqrt((p->w_max * p->w_max - 1.0) / u2);
    for (int i = 0; i < 3; ++i) P[OR_U1 + i] *= s;
    fl = 1;
  }
  if (status == 3) return 3;
  if (fl) return 2;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction and numerical flux                                          */
/* ------------------------------------------------------------------------ */

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* PPM interface value (Colella & Woodward 1984): fourth-order estimate
 * 7/12 (a_k + a_k+1) - 1/12 (a_k-1 + a_k+2), clipped between a_k and a_k+1. */
static double ppm_iface(double am1, double a0, double a1, double a2) {
  double v = 7.0 / 12.0 * (a0 + a1) - 1.0 / 12.0 * (am1 + a2);
  double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
  if (v < lo) v = lo;
  if (v > hi) v = hi;
  return v;
}

/* CW84 monotonicity constraints on the parabola of a cell with mean a and
 * edge values (aL, aR): flatten at a local extremum, otherwise pull the
 * far edge in so the parabola does not overshoot. */
static void ppm_limit(double a, double* aL, double* aR) {
  if ((*aR - a) * (a - *aL) <= 0.0) {
    *aL = a;
    *aR = a;
    return;
  }
  double d = *aR - *aL;
  double m6 = 6.0 * (a - 0.5 * (*aL + *aR));
  if (d * m6 > d * d) *aL = 3.0 * a - 2.0 * (*aR);
  if (-d * d > d * m6) *aR = 3.0 * a - 2.0 * (*aL);
}

/* Face states from stencil cells 0..5 (the face lies between cells 2 and 3).
 * If either state has rho <= 0 or p <= 0 the face falls back to first order. */
void or_reconstruct(const or_params* p, const double st[6][OR_NV], double PL[OR_NV], double PR[OR_NV]) {
  for (int v = 0; v < OR_NV; ++v) {
    double a0 = st[0][v], a1 = st[1][v], a2 = st[2][v], a3 = st[3][v], a4 = st[4][v], a5 = st[5][v];
    if (p->recon == 0) {
      /* cell 2 (left of the face) and cell 3 (right of the face) */
      double l2 = ppm_iface(a0, a1, a2, a3), r2 = ppm_iface(a1, a2, a3, a4);
      double l3 = ppm_iface(a1, a2, a3, a4), r3 = ppm_iface(a2, a3, a4, a5);
      ppm_limit(a2, &l2, &r2);
      ppm_limit(a3, &l3, &r3);
      PL[v] = r2;
      PR[v] = l3;
    } else {
      PL[v] = a2 + 0.5 * minmod(a2 - a1, a3 - a2);
      PR[v] = a3 - 0.5 * minmod(a3 - a2, a4 - a3);
    }
  }
  if (!(PL[OR_RHO] > 0.0) || !(PL[OR_P] > 0.0) || !(PR[OR_RHO] > 0.0) || !(PR[OR_P] > 0.0)) {
    for (int v = 0; v < OR_NV; ++v) {
      PL[v] = st[2][v];
      PR[v] = st[3][v];
    }
  }
}

/* HLL (Harten, Lax & van Leer 1983) or TVDLF (Rusanov) flux, densitized by
 * the face sqrt(gamma).  The GLM pair (normal B, psi) uses signal speeds no
 * smaller than its own characteristic speeds +-alpha ch sqrt(gamma^ii) - beta^i. */
void or_face_flux(const or_params* p, const or_metric* m, const double PL[OR_NV], const double PR[OR_NV],
                  int dir, double F[OR_NV]) {
  state sL, sR;
  double UL[OR_NV], UR[OR_NV], FL[OR_NV], FR[OR_NV];
  double lmL, lpL, lmR, lpR;
  make_state(p, m, PL, &sL);
  make_state(p, m, PR, &sR);
  cons_of_state(&sL, UL);
  cons_of_state(&sR, UR);
  flux_of_state(p, m, &sL, UL, dir, FL);
  flux_of_state(p, m, &sR, UR, dir, FR);
  speeds_of_state(p, m, &sL, dir, &lmL, &lpL);
  speeds_of_state(p, m, &sR, dir, &lmR, &lpR);
  double cg = m->alpha * p->ch * sqrt(m->gi[dir][dir]);
  double lgp = cg - m->beta[dir], lgm = -cg - m->beta[dir];
  for (int v = 0; v < OR_NV; ++v) {
    int glm = (v == OR_PSI) || (v == OR_B1 + dir);
    double f;
    if (p->riemann == 0) {
      double lp = 0.0, lm = 0.0;
      if (lpL > lp) lp = lpL;
      if (lpR > lp) lp = lpR;
      if (lmL < lm) lm = lmL;
      if (lmR < lm) lm = lmR;
      if (glm) {
        if (lgp > lp) lp = lgp;
        if (lgm < lm) lm = lgm;
      }
      if (lp - lm > 0.0)
        f = (lp * FL[v] - lm * FR[v] + lp * lm * (UR[v] - UL[v])) / (lp - lm);
      else
        f = 0.5 * (FL[v] + FR[v]);
    } else {
      double c = fabs(lpL);
      if (fabs(lmL) > c) c = fabs(lmL);
      if (fabs(lpR) > c) c = fabs(lpR);
      if (fabs(lmR) > c) c = fabs(lmR);
      if (glm) {
        if (fabs(lgp) > c) c = fabs(lgp);
        if (fabs(lgm) > c) c = fabs(lgm);
      }
      f = 0.5 * (FL[v] + FR[v]) - 0.5 * c * (UR[v] - UL[v]);
    }
    F[v] = m->sqrtg * f;
  }
}

/* ------------------------------------------------------------------------ */
/* Block grid                                                                 */
/* ------------------------------------------------------------------------ */

struct or_ctx {
  or_params p;
  int nb;
  int* blk;        /* nb x 4 : level, ix, iy, iz */
  int gd[3];       /* ghosts per dimension */
  int N[3];        /* ghosted extent per dimension */
  int ncell;       /* ghosted cells per block */
  int nint;        /* interior cells per block */
  double* prim;    /* nb x NV x ghosted */
  double* ucur;    /* nb x NV x interior, densitized */
  double* un;      /* conserved at the start of the step */
  double* flux[3]; /* nb x NV x face-array per direction */
  int* lut[8];     /* per level: block id at block coordinates, -1 if not a leaf */
  long long counts[4];
  unsigned char* status; /* nb x interior: inversion outcome of the last stage */
  /* constrained transport: per active direction d, the face field Phi^d and the
   * fluxes through the faces normal to d, over the block's faces plus a ring
   * of one face across in every active transverse direction */
  int fe[3][3];          /* extents of the direction-d face arrays */
  int fo[3][3];          /* position of local index 0 inside them */
  double* fc[3];         /* Phi^d = sqrt(gamma) B^d at face centres */
  double* fcn[3];        /* Phi^d at the start of the step */
  double* xf[3];         /* fluxes through those faces, NV per face, densitized */
};

static long lut_size(const or_ctx* c, int L) {
  long n = 1;
  for (int d = 0; d < 3; ++d) n *= (long)c->p.nroot[d] << (d < c->p.ndim ? L : 0);
  return n;
}

static int lut_get(const or_ctx* c, int L, const long bc[3]) {
  if (L < 0 || L >= c->p.nlevels) return -1;
  long nbd[3];
  for (int d = 0; d < 3; ++d) {
    nbd[d] = (long)c->p.nroot[d] << (d < c->p.ndim ? L : 0);
    if (bc[d] < 0 || bc[d] >= nbd[d]) return -1;
  }
  return c->lut[L][(bc[2] * nbd[1] + bc[1]) * nbd[0] + bc[0]];
}

static size_t pidx(const or_ctx* c, int b, int v, int i, int j, int k) {
  return ((((size_t)b * OR_NV + v) * c->N[2] + k) * c->N[1] + j) * c->N[0] + i;
}

static size_t uidx(const or_ctx* c, int b, int v, int i, int j, int k) {
  return ((((size_t)b * OR_NV + v) * c->p.nx[2] + k) * c->p.nx[1] + j) * c->p.nx[0] + i;
}

static double dxl(const or_ctx* c, int d, int L) {
  int scale = d < c->p.ndim ? (1 << L) : 1;
  return (c->p.xmax[d] - c->p.xmin[d]) / ((double)c->p.nroot[d] * c->p.nx[d] * scale);
}

/* coordinate of cell-centre (off = 0.5) or low face (off = 0) of global index G at level L */
static double coord(const or_ctx* c, int d, int L, long G, double off) {
  return c->p.xmin[d] + ((double)G + off) * dxl(c, d, L);
}

static double floor_radius(const or_params* p, const double x[3]) {
  if (p->coords == OR_KS) return x[0];
  if (p->coords == OR_MKS) return exp(x[0]);
  return 1.0;
}

or_ctx* or_create(const or_params* p, int nblocks, const int* blocks) {
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->p = *p;
  c->nb = nblocks;
  c->blk = (int*)malloc(sizeof(int) * 4 * nblocks);
  memcpy(c->blk, blocks, sizeof(int) * 4 * nblocks);
  c->ncell = 1;
  c->nint = 1;
  for (int d = 0; d < 3; ++d) {
    c->gd[d] = d < p->ndim ? p->ng : 0;
    c->N[d] = p->nx[d] + 2 * c->gd[d];
    c->ncell *= c->N[d];
    c->nint *= p->nx[d];
  }
  c->prim = (double*)calloc((size_t)nblocks * OR_NV * c->ncell, sizeof(double));
  c->ucur = (double*)calloc((size_t)nblocks * OR_NV * c->nint, sizeof(double));
  c->un = (double*)calloc((size_t)nblocks * OR_NV * c->nint, sizeof(double));
  c->status = (unsigned char*)calloc((size_t)nblocks * c->nint, 1);
  for (int d = 0; d < p->ndim; ++d) {
    size_t nf = (size_t)c->nint / p->nx[d] * (p->nx[d] + 1);
    c->flux[d] = (double*)calloc((size_t)nblocks * OR_NV * nf, sizeof(double));
  }
  if (p->ct) {
    /* psi is not evolved: no cleaning speed, no damping */
    c->p.ch = 0.0;
    c->p.kappa = 0.0;
    for (int d = 0; d < p->ndim; ++d) {
      size_t n = (size_t)nblocks;
      for (int e = 0; e < 3; ++e) {
        int across = e != d && e < p->ndim;
        c->fe[d][e] = e == d ? p->nx[e] + 1 : p->nx[e] + (across ? 2 : 0);
        c->fo[d][e] = across ? 1 : 0;
        n *= c->fe[d][e];
      }
      c->fc[d] = (double*)calloc(n, sizeof(double));
      c->fcn[d] = (double*)calloc(n, sizeof(double));
      c->xf[d] = (double*)calloc(n * OR_NV, sizeof(double));
    }
  }
  for (int L = 0; L < p->nlevels && L < 8; ++L) {
    long n = lut_size(c, L);
    c->lut[L] = (int*)malloc(sizeof(int) * n);
    for (long i = 0; i < n; ++i) c->lut[L][i] = -1;
  }
  for (int b = 0; b < nblocks; ++b) {
    int L = blocks[4 * b];
    long nbd[3];
    for (int d = 0; d < 3; ++d) nbd[d] = (long)p->nroot[d] << (d < p->ndim ? L : 0);
    c->lut[L][((long)blocks[4 * b + 3] * nbd[1] + blocks[4 * b + 2]) * nbd[0] + blocks[4 * b + 1]] = b;
  }
  return c;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->blk);
  free(c->prim);
  free(c->ucur);
  free(c->un);
  free(c->status);
  for (int d = 0; d < 3; ++d) {
    free(c->flux[d]);
    free(c->fc[d]);
    free(c->fcn[d]);
    free(c->xf[d]);
  }
  for (int L = 0; L < 8; ++L) free(c->lut[L]);
  free(c);
}

int or_ghosted_cells(const or_ctx* c) { return c->ncell; }

static void cell_centre(const or_ctx* c, int b, int i, int j, int k, double x[3]) {
  int L = c->blk[4 * b];
  int loc[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) x[d] = coord(c, d, L, (long)c->blk[4 * b + 1 + d] * c->p.nx[d] + loc[d], 0.5);
}

void or_set_prims(or_ctx* c, const double* prims) {
  const int* nx = c->p.nx;
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < nx[2]; ++k)
      for (int j = 0; j < nx[1]; ++j)
        for (int i = 0; i < nx[0]; ++i) {
          double P[OR_NV], U[OR_NV], x[3];
          or_metric m;
          for (int v = 0; v < OR_NV; ++v) {
            P[v] = prims[uidx(c, b, v, i, j, k)];
            c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])] = P[v];
          }
          cell_centre(c, b, i, j, k, x);
          or_metric_at(&c->p, x, 0, &m);
          or_prim2con(&c->p, &m, P, U);
          for (int v = 0; v < OR_NV; ++v) c->ucur[uidx(c, b, v, i, j, k)] = m.sqrtg * U[v];
        }
}

void or_get_prims(const or_ctx* c, double* prims) {
  const int* nx = c->p.nx;
  for (int b = 0; b < c->nb; ++b)
    for (int v = 0; v < OR_NV; ++v)
      for (int k = 0; k < nx[2]; ++k)
        for (int j = 0; j < nx[1]; ++j)
          for (int i = 0; i < nx[0]; ++i)
            prims[uidx(c, b, v, i, j, k)] = c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])];
}

void or_get_prims_ghosted(const or_ctx* c, double* prims) {
  memcpy(prims, c->prim, sizeof(double) * (size_t)c->nb * OR_NV * c->ncell);
}

void or_get_cons(const or_ctx* c, double* cons) {
  memcpy(cons, c->ucur, sizeof(double) * (size_t)c->nb * OR_NV * c->nint);
}

void or_c2p_status(const or_ctx* c, unsigned char* status) {
  memcpy(status, c->status, (size_t)c->nb * c->nint);
}

void or_c2p_counts(const or_ctx* c, long long counts[4]) {
  for (int i = 0; i < 4; ++i) counts[i] = c->counts[i];
}

/* ---- ghost cells ---- */

/* Maps a level-L global index that may lie outside the root domain back
 * inside it according to the boundary kinds.  Returns the sign flips and
 * clamps to apply to the fetched primitives:
 *   periodic : wrap;  outflow : copy the nearest interior cell;
 *   no-inflow: outflow, then u^d <= 0 at the low and >= 0 at the high side;
 *   polar axis (theta): mirror in theta, flip u^theta and B^theta, and in 3-D
 *   take the cell at phi + pi. */
typedef struct {
  int flip;       /* theta components flip sign */
  int clamp[3];   /* -1: u^d <= 0, +1: u^d >= 0, 0: none */
} bcfix;

static void apply_bc(const or_ctx* c, int L, long G[3], bcfix* fx) {
  fx->flip = 0;
  for (int d = 0; d < 3; ++d) fx->clamp[d] = 0;
  for (int d = 0; d < c->p.ndim; ++d) {
    long N = (long)c->p.nroot[d] * c->p.nx[d] << L;
    for (int side = 0; side < 2; ++side) {
      int out = side == 0 ? G[d] < 0 : G[d] >= N;
      if (!out) continue;
      int kind = c->p.bc[d][side];
      if (kind == OR_BC_PERIODIC) {
        G[d] = ((G[d] % N) + N) % N;
      } else if (kind == OR_BC_OUTFLOW || kind == OR_BC_NOINFLOW) {
        G[d] = side == 0 ? 0 : N - 1;
        if (kind == OR_BC_NOINFLOW) fx->clamp[d] = side == 0 ? -1 : 1;
      } else if (kind == OR_BC_AXIS) {
        G[d] = side == 0 ? -1 - G[d] : 2 * N - 1 - G[d];
        fx->flip ^= 1;
        if (c->p.ndim == 3) {
          long Nph = (long)c->p.nroot[2] * c->p.nx[2] << L;
          G[2] = (((G[2] + Nph / 2) % Nph) + Nph) % Nph;
        }
      }
    }
  }
  /* the axis shift can move phi out of range only if phi is periodic */
  if (c->p.ndim == 3) {
    long Nph = (long)c->p.nroot[2] * c->p.nx[2] << L;
    if (c->p.bc[2][0] == OR_BC_PERIODIC) G[2] = ((G[2] % Nph) + Nph) % Nph;
  }
}

static void fix_values(const bcfix* fx, double P[OR_NV]) {
  if (fx->flip) {
    P[OR_U2] = -P[OR_U2];
    P[OR_B2] = -P[OR_B2];
  }
  for (int d = 0; d < 3; ++d) {
    if (fx->clamp[d] < 0 && P[OR_U1 + d] > 0.0) P[OR_U1 + d] = 0.0;
    if (fx->clamp[d] > 0 && P[OR_U1 + d] < 0.0) P[OR_U1 + d] = 0.0;
  }
}

/* Primitives of cell G (level-L global index, any position) from the leaf
 * blocks: a copy where a level-L leaf holds the cell; a minmod-limited linear
 * prolongation from the coarser leaf; or the mean of the 2^ndim finer cells
 * (restriction) where finer leaves hold it. */
static void cell_value(const or_ctx* c, int L, const long Gin[3], double P[OR_NV]) {
  long G[3] = {Gin[0], Gin[1], Gin[2]};
  bcfix fx;
  apply_bc(c, L, G, &fx);
  long bc[3];
  for (int d = 0; d < 3; ++d) bc[d] = G[d] / c->p.nx[d];
  int b = lut_get(c, L, bc);
  if (b >= 0) {
    for (int v = 0; v < OR_NV; ++v)
      P[v] = c->prim[pidx(c, b, v, (int)(G[0] % c->p.nx[0]) + c->gd[0], (int)(G[1] % c->p.nx[1]) + c->gd[1],
                          (int)(G[2] % c->p.nx[2]) + c->gd[2])];
  } else {
    /* is a coarser leaf covering this cell? */
    int coarse = 0;
    for (int Lc = L - 1; Lc >= 0; --Lc) {
      long bcc[3];
      for (int d = 0; d < 3; ++d) bcc[d] = (d < c->p.ndim ? G[d] >> (L - Lc) : G[d]) / c->p.nx[d];
      if (lut_get(c, Lc, bcc) >= 0) {
        coarse = 1;
        break;
      }
    }
    if (coarse && L > 0) {
      long C[3];
      for (int d = 0; d < 3; ++d) C[d] = d < c->p.ndim ? G[d] >> 1 : G[d];
      double Pc[OR_NV];
      cell_value(c, L - 1, C, Pc);
      for (int v = 0; v < OR_NV; ++v) P[v] = Pc[v];
      for (int d = 0; d < c->p.ndim; ++d) {
        long Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
        Cm[d] -= 1;
        Cp[d] += 1;
        double Pm[OR_NV], Pp[OR_NV];
        cell_value(c, L - 1, Cm, Pm);
        cell_value(c, L - 1, Cp, Pp);
        double off = (G[d] & 1) ? 0.25 : -0.25;
        for (int v = 0; v < OR_NV; ++v) P[v] += off * minmod(Pc[v] - Pm[v], Pp[v] - Pc[v]);
      }
    } else {
      int nch = 1 << c->p.ndim;
      for (int v = 0; v < OR_NV; ++v) P[v] = 0.0;
      for (int ch = 0; ch < nch; ++ch) {
        long F[3] = {G[0], G[1], G[2]};
        for (int d = 0; d < c->p.ndim; ++d) F[d] = 2 * G[d] + ((ch >> d) & 1);
        double Pf[OR_NV];
        cell_value(c, L + 1, F, Pf);
        for (int v = 0; v < OR_NV; ++v) P[v] += Pf[v];
      }
      for (int v = 0; v < OR_NV; ++v) P[v] /= nch;
    }
  }
  fix_values(&fx, P);
}

static void fill_block_ghosts(or_ctx* c, int b) {
  int L = c->blk[4 * b];
  for (int k = 0; k < c->N[2]; ++k)
    for (int j = 0; j < c->N[1]; ++j)
      for (int i = 0; i < c->N[0]; ++i) {
        int loc[3] = {i - c->gd[0], j - c->gd[1], k - c->gd[2]};
        int inside = 1;
        for (int d = 0; d < 3; ++d)
          if (loc[d] < 0 || loc[d] >= c->p.nx[d]) inside = 0;
        if (inside) continue;
        long G[3];
        for (int d = 0; d < 3; ++d) G[d] = (long)c->blk[4 * b + 1 + d] * c->p.nx[d] + loc[d];
        double P[OR_NV];
        cell_value(c, L, G, P);
        for (int v = 0; v < OR_NV; ++v) c->prim[pidx(c, b, v, i, j, k)] = P[v];
      }
}

void or_fill_ghosts(or_ctx* c) {
  /* ghosts read only interior cells, so blocks are independent */
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < c->nb; ++b) fill_block_ghosts(c, b);
}

/* ---- CFL ---- */

/* dt = C / max over interior cells of sum_d c_d / dx_d, with c_d the largest
 * of |lambda+-| and the GLM speeds alpha ch sqrt(gamma^dd) + |beta^d|. */
double or_cfl_dt(or_ctx* c) {
  double smax = 0.0;
#pragma omp parallel for schedule(dynamic) reduction(max : smax)
  for (int b = 0; b < c->nb; ++b) {
    int L = c->blk[4 * b];
    for (int k = 0; k < c->p.nx[2]; ++k)
      for (int j = 0; j < c->p.nx[1]; ++j)
        for (int i = 0; i < c->p.nx[0]; ++i) {
          double x[3], P[OR_NV];
          or_metric m;
          cell_centre(c, b, i, j, k, x);
          or_metric_at(&c->p, x, 0, &m);
          for (int v = 0; v < OR_NV; ++v) P[v] = c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])];
          double s = 0.0;
          for (int d = 0; d < c->p.ndim; ++d) {
            double lm, lp;
            or_wavespeeds(&c->p, &m, P, d, &lm, &lp);
            double cd = fabs(lp) > fabs(lm) ? fabs(lp) : fabs(lm);
            double cg = m.alpha * c->p.ch * sqrt(m.gi[d][d]) + fabs(m.beta[d]);
            if (cg > cd) cd = cg;
            s += cd / dxl(c, d, L);
          }
          if (s > smax) smax = s;
        }
  }
  return c->p.cfl / smax;
}

/* ---- constrained transport ---- */

/* Staggered-mesh constrained transport: the field normal to each face is
 * evolved as Phi^d = sqrt(gamma) B^d at the face centre, by the induction
 * equation in integral form, d_t Phi = -curl E, with the electric field at
 * cell edges.  The face fluxes of B already are E up to sign:
 *   F^2(B^1) = -F^1(B^2) = E_3,  F^3(B^2) = -F^2(B^3) = E_1,
 *   F^1(B^3) = -F^3(B^1) = E_2    (E = -(alpha v - beta) x B, densitized),
 * so the EMF at an edge is the mean of the four upwinded (HLL/TVDLF) face
 * fluxes around it (the flux-interpolated constrained transport of Balsara &
 * Spicer 1999).  Because the face update is a discrete curl, the discrete
 * divergence sum_d (Phi^d_high - Phi^d_low) / dx_d of every cell keeps its
 * initial value to round-off.  At a face the normal field in both reconstructed
 * states is Phi^d / sqrt(gamma) of the face itself.  Cell-centred
 * sqrt(gamma) B^d = (Phi^d_low + Phi^d_high) / 2.  A block owns its faces
 * 0..nx_d along d; the ring of faces one cell outside it across (needed by the
 * EMFs at the block's edges) is filled from the neighbours like ghost cells, so
 * both blocks sharing a face compute the same EMFs and keep the same value.
 * Across refinement levels a ring face takes the coarse face it lies on, or
 * the mean of the two faces of the coarse cell it cuts, or the mean of the
 * finer faces on it; the coarse flux through a face on a level boundary is the
 * mean of the finer fluxes (as for the cell-centred variables), and an edge
 * that a finer leaf touches takes the mean of the finer EMFs along it, so the
 * coarse copy of such a face changes by the mean of the changes of the finer
 * faces covering it, and every cell's divergence stays at round-off. */

static size_t fcx(const or_ctx* c, int d, int b, int i, int j, int k) {
  const int* e = c->fe[d];
  const int* o = c->fo[d];
  return (((size_t)b * e[2] + (k + o[2])) * e[1] + (j + o[1])) * e[0] + (i + o[0]);
}

static size_t xfx(const or_ctx* c, int d, int b, int v, int i, int j, int k) {
  const int* e = c->fe[d];
  const int* o = c->fo[d];
  return ((((size_t)b * OR_NV + v) * e[2] + (k + o[2])) * e[1] + (j + o[1])) * e[0] + (i + o[0]);
}

/* cells along d at level L across the root domain */
static long ncell_l(const or_ctx* c, int d, int L) {
  return ((long)c->p.nroot[d] * c->p.nx[d]) << (d < c->p.ndim ? L : 0);
}

/* Level-L cell G (global index inside the root domain): 0 if a level-L leaf
 * holds it, -1 if a coarser leaf covers it, +1 if finer leaves cover it. */
static int cover_of(const or_ctx* c, int L, const long G[3]) {
  long bc[3];
  for (int d = 0; d < 3; ++d) bc[d] = G[d] / c->p.nx[d];
  if (lut_get(c, L, bc) >= 0) return 0;
  for (int Lc = L - 1; Lc >= 0; --Lc) {
    for (int d = 0; d < 3; ++d) bc[d] = (d < c->p.ndim ? G[d] >> (L - Lc) : G[d]) / c->p.nx[d];
    if (lut_get(c, Lc, bc) >= 0) return -1;
  }
  return 1;
}

/* Phi^d of face G at level L (a face index along d, cell indices across, inside
 * the root domain): the face of the level-L leaf that holds it (the block above
 * it along d, else the one below); where a coarser leaf covers it, the coarse
 * face it lies on (even G_d) or the mean of the two faces of the coarse cell it
 * cuts (odd G_d); where finer leaves cover it, the mean of the 2^(ndim-1)
 * finer faces on it.  Only owned faces are read. */
static double ct_face_value(const or_ctx* c, int d, int L, const long G[3]) {
  const int* nx = c->p.nx;
  const long Nd = ncell_l(c, d, L);
  long bc[3];
  int lf[3];
  for (int e = 0; e < 3; ++e)
    if (e != d) {
      bc[e] = G[e] / nx[e];
      lf[e] = (int)(G[e] % nx[e]);
    }
  for (int above = 1; above >= 0; --above) {
    const long cell = above ? G[d] : G[d] - 1;
    if (cell < 0 || cell >= Nd) continue;
    bc[d] = cell / nx[d];
    lf[d] = (int)(G[d] - bc[d] * nx[d]);
    const int b = lut_get(c, L, bc);
    if (b >= 0) return c->fc[d][fcx(c, d, b, lf[0], lf[1], lf[2])];
  }
  long cell[3] = {G[0], G[1], G[2]};
  if (cell[d] >= Nd) cell[d] = Nd - 1;
  const int cov = cover_of(c, L, cell);
  if (cov < 0 && L > 0) {
    long H[3];
    for (int e = 0; e < 3; ++e) H[e] = e < c->p.ndim ? G[e] >> 1 : G[e];
    if (!(G[d] & 1)) return ct_face_value(c, d, L - 1, H);
    long H1[3] = {H[0], H[1], H[2]};
    H1[d] += 1;
    return 0.5 * (ct_face_value(c, d, L - 1, H) + ct_face_value(c, d, L - 1, H1));
  }
  if (cov <= 0 || L + 1 >= c->p.nlevels) return 0.0; /* no leaf: an inconsistent grid */
  int t[2], nt = 0;
  for (int e = 0; e < c->p.ndim; ++e)
    if (e != d) t[nt++] = e;
  double s = 0.0;
  for (int q = 0; q < (1 << nt); ++q) {
    long F[3] = {G[0], G[1], G[2]};
    F[d] = 2 * G[d];
    for (int u = 0; u < nt; ++u) F[t[u]] = 2 * G[t[u]] + ((q >> u) & 1);
    s += ct_face_value(c, d, L + 1, F);
  }
  return s / (1 << nt);
}

/* The ring faces of every block: the boundary rules across the face (periodic
 * wrap, outflow / no-inflow copy of the nearest face, polar axis mirror in
 * theta and phi + pi in 3-D), then the face's value at the block's level
 * (zero where no face exists). */
static void ct_fill_face_ring(or_ctx* c) {
  const int* nx = c->p.nx;
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < c->nb; ++b) {
    const int L = c->blk[4 * b];
    for (int d = 0; d < c->p.ndim; ++d) {
      const int* e = c->fe[d];
      const int* o = c->fo[d];
      long N[3];
      for (int t = 0; t < 3; ++t) N[t] = ncell_l(c, t, L);
      for (int k = -o[2]; k < e[2] - o[2]; ++k)
        for (int j = -o[1]; j < e[1] - o[1]; ++j)
          for (int i = -o[0]; i < e[0] - o[0]; ++i) {
            int f[3] = {i, j, k}, ring = 0;
            for (int t = 0; t < 3; ++t)
              if (t != d && (f[t] < 0 || f[t] >= nx[t])) ring = 1;
            if (!ring) continue;
            long G[3];
            for (int t = 0; t < 3; ++t) G[t] = (long)c->blk[4 * b + 1 + t] * nx[t] + f[t];
            for (int t = 0; t < c->p.ndim; ++t) {
              if (t == d) continue;
              for (int side = 0; side < 2; ++side) {
                int out = side == 0 ? G[t] < 0 : G[t] >= N[t];
                if (!out) continue;
                int kind = c->p.bc[t][side];
                if (kind == OR_BC_PERIODIC) {
                  G[t] = ((G[t] % N[t]) + N[t]) % N[t];
                } else if (kind == OR_BC_OUTFLOW || kind == OR_BC_NOINFLOW) {
                  G[t] = side == 0 ? 0 : N[t] - 1;
                } else if (kind == OR_BC_AXIS) {
                  G[t] = side == 0 ? -1 - G[t] : 2 * N[t] - 1 - G[t];
                  if (c->p.ndim == 3) G[2] = ((G[2] + N[2] / 2) % N[2] + N[2]) % N[2];
                }
              }
            }
            if (c->p.ndim == 3 && d != 2 && c->p.bc[2][0] == OR_BC_PERIODIC) G[2] = ((G[2] % N[2]) + N[2]) % N[2];
            int inside = 1;
            for (int t = 0; t < 3; ++t)
              if (G[t] < 0 || G[t] > N[t] || (t != d && G[t] == N[t])) inside = 0;
            c->fc[d][fcx(c, d, b, i, j, k)] = inside ? ct_face_value(c, d, L, G) : 0.0;
          }
    }
  }
}

/* Fluxes through every face of direction d of block b and its ring. */
static void ct_block_xfluxes(or_ctx* c, int b, int d) {
  int L = c->blk[4 * b];
  const int* e = c->fe[d];
  const int* o = c->fo[d];
  long Nd = ncell_l(c, d, L);
  for (int k = -o[2]; k < e[2] - o[2]; ++k)
    for (int j = -o[1]; j < e[1] - o[1]; ++j)
      for (int i = -o[0]; i < e[0] - o[0]; ++i) {
        int f[3] = {i, j, k};
        double x[3], F[OR_NV];
        long G[3];
        for (int t = 0; t < 3; ++t) {
          G[t] = (long)c->blk[4 * b + 1 + t] * c->p.nx[t] + f[t];
          x[t] = coord(c, t, L, G[t], t == d ? 0.0 : 0.5);
        }
        int axis = (G[d] == 0 && c->p.bc[d][0] == OR_BC_AXIS) || (G[d] == Nd && c->p.bc[d][1] == OR_BC_AXIS);
        if (axis) {
          for (int v = 0; v < OR_NV; ++v) F[v] = 0.0;
        } else {
          double st[6][OR_NV], PL[OR_NV], PR[OR_NV];
          for (int s = 0; s < 6; ++s) {
            int g[3] = {i + c->gd[0], j + c->gd[1], k + c->gd[2]};
            g[d] += s - 3;
            for (int v = 0; v < OR_NV; ++v) st[s][v] = c->prim[pidx(c, b, v, g[0], g[1], g[2])];
          }
          or_reconstruct(&c->p, (const double(*)[OR_NV])st, PL, PR);
          or_metric m;
          or_metric_at(&c->p, x, 0, &m);
          double Bn = c->fc[d][fcx(c, d, b, i, j, k)] / m.sqrtg;
          PL[OR_B1 + d] = Bn;
          PR[OR_B1 + d] = Bn;
          or_face_flux(&c->p, &m, PL, PR, d, F);
        }
        for (int v = 0; v < OR_NV; ++v) c->xf[d][xfx(c, d, b, v, i, j, k)] = F[v];
      }
}

/* Edge EMFs of block b: E_3 at the edge (i-1/2, j-1/2) of cell layer k, E_1
 * at (j-1/2, k-1/2) of column i, E_2 at (k-1/2, i-1/2) of row j, each the
 * mean of the four face fluxes around the edge. */
static double ct_emf3(const or_ctx* c, int b, int i, int j, int k) {
  return 0.25 * (c->xf[1][xfx(c, 1, b, OR_B1, i, j, k)] + c->xf[1][xfx(c, 1, b, OR_B1, i - 1, j, k)] -
                 c->xf[0][xfx(c, 0, b, OR_B2, i, j, k)] - c->xf[0][xfx(c, 0, b, OR_B2, i, j - 1, k)]);
}
static double ct_emf1(const or_ctx* c, int b, int i, int j, int k) {
  return 0.25 * (c->xf[2][xfx(c, 2, b, OR_B2, i, j, k)] + c->xf[2][xfx(c, 2, b, OR_B2, i, j - 1, k)] -
                 c->xf[1][xfx(c, 1, b, OR_B3, i, j, k)] - c->xf[1][xfx(c, 1, b, OR_B3, i, j, k - 1)]);
}
static double ct_emf2(const or_ctx* c, int b, int i, int j, int k) {
  return 0.25 * (c->xf[0][xfx(c, 0, b, OR_B3, i, j, k)] + c->xf[0][xfx(c, 0, b, OR_B3, i, j, k - 1)] -
                 c->xf[2][xfx(c, 2, b, OR_B1, i, j, k)] - c->xf[2][xfx(c, 2, b, OR_B1, i - 1, j, k)]);
}

static double ct_emf_block(const or_ctx* c, int a, int b, int i, int j, int k) {
  return a == 0 ? ct_emf1(c, b, i, j, k) : (a == 1 ? ct_emf2(c, b, i, j, k) : ct_emf3(c, b, i, j, k));
}

/* The level-L cell q (0..3) around the edge along a at G (a cell index along
 * a, face indices across): across each active transverse direction the cell
 * below (bit 0) or above (bit 1) the edge; periodic wrap; 0 where it leaves
 * the root domain across another boundary. */
static int ct_edge_cell(const or_ctx* c, int a, int L, const long G[3], int q, long C[3], int s[3]) {
  int u = 0;
  for (int e = 0; e < 3; ++e) {
    C[e] = G[e];
    s[e] = 0;
    if (e == a || e >= c->p.ndim) continue;
    s[e] = (q >> u++) & 1;
    C[e] = G[e] - 1 + s[e];
    const long N = ncell_l(c, e, L);
    if (C[e] < 0 || C[e] >= N) {
      if (c->p.bc[e][C[e] < 0 ? 0 : 1] != OR_BC_PERIODIC) return 0;
      C[e] = ((C[e] % N) + N) % N;
    }
  }
  return 1;
}

/* E_a (a = 0, 1, 2: E_1, E_2, E_3) at the edge of block b with local index
 * (i, j, k) in the layout of ct_emf1/2/3: the block's own mean of four face
 * fluxes, except where a finer leaf touches the edge.  There it is the mean
 * of the finer EMFs along the edge (two segments when a is active, else one),
 * each taken from a finer leaf holding a cell around that segment; then every
 * coarse face around the edge changes by the mean of the changes of the finer
 * faces covering it, and the coarse and fine copies of a face on a level
 * boundary keep the same flux through it (EMF correction). */
static double ct_emf(const or_ctx* c, int a, int b, int i, int j, int k) {
  if (c->p.nlevels == 1) return ct_emf_block(c, a, b, i, j, k);
  const int L = c->blk[4 * b];
  const int* nx = c->p.nx;
  const int loc[3] = {i, j, k};
  long G[3], C[3];
  int s[3];
  for (int e = 0; e < 3; ++e) G[e] = (long)c->blk[4 * b + 1 + e] * nx[e] + loc[e];
  int finer = 0;
  for (int q = 0; q < 4 && !finer; ++q)
    if (ct_edge_cell(c, a, L, G, q, C, s) && cover_of(c, L, C) > 0) finer = 1;
  if (!finer || L + 1 >= c->p.nlevels) return ct_emf_block(c, a, b, i, j, k);
  const int na = a < c->p.ndim ? 2 : 1;
  double sum = 0.0;
  int n = 0;
  for (int t = 0; t < na; ++t) {
    long F[3];
    for (int e = 0; e < 3; ++e) F[e] = e >= c->p.ndim ? G[e] : 2 * G[e] + (e == a ? t : 0);
    for (int q = 0; q < 4; ++q) {
      if (!ct_edge_cell(c, a, L + 1, F, q, C, s)) continue;
      long bc[3];
      for (int e = 0; e < 3; ++e) bc[e] = C[e] / nx[e];
      const int bf = lut_get(c, L + 1, bc);
      if (bf < 0) continue;
      int lf[3];
      for (int e = 0; e < 3; ++e) lf[e] = (int)(C[e] - bc[e] * nx[e]) + (e != a && e < c->p.ndim && !s[e] ? 1 : 0);
      sum += ct_emf_block(c, a, bf, lf[0], lf[1], lf[2]);
      ++n;
      break;
    }
  }
  return n == na ? sum / na : ct_emf_block(c, a, b, i, j, k);
}

/* d_t Phi = -curl E on the owned faces of block b, then the stage combination
 * (stage 1: Phi1 = Phin + dt R; stage 2: Phi = Phin/2 + (Phi1 + dt R)/2).
 * Faces on the polar axis (sqrt(gamma) = 0) stay zero. */
static void ct_update_faces(or_ctx* c, int b, int stage, double dt) {
  int L = c->blk[4 * b];
  const int* nx = c->p.nx;
  int three = c->p.ndim == 3;
  double dx[3];
  for (int t = 0; t < 3; ++t) dx[t] = dxl(c, t, L);
  for (int d = 0; d < c->p.ndim; ++d) {
    long Nd = ncell_l(c, d, L);
    int n[3] = {nx[0], nx[1], nx[2]};
    n[d] += 1;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          size_t q = fcx(c, d, b, i, j, k);
          int f[3] = {i, j, k};
          long Gd = (long)c->blk[4 * b + 1 + d] * nx[d] + f[d];
          if (d == 1 && ((Gd == 0 && c->p.bc[1][0] == OR_BC_AXIS) || (Gd == Nd && c->p.bc[1][1] == OR_BC_AXIS))) {
            c->fc[d][q] = 0.0;
            if (stage == 1) c->fcn[d][q] = 0.0;
            continue;
          }
          double R;
          if (d == 0) {
            R = -(ct_emf(c, 2, b, i, j + 1, k) - ct_emf(c, 2, b, i, j, k)) / dx[1];
            if (three) R += (ct_emf(c, 1, b, i, j, k + 1) - ct_emf(c, 1, b, i, j, k)) / dx[2];
          } else if (d == 1) {
            R = (ct_emf(c, 2, b, i + 1, j, k) - ct_emf(c, 2, b, i, j, k)) / dx[0];
            if (three) R -= (ct_emf(c, 0, b, i, j, k + 1) - ct_emf(c, 0, b, i, j, k)) / dx[2];
          } else {
            R = -(ct_emf(c, 1, b, i + 1, j, k) - ct_emf(c, 1, b, i, j, k)) / dx[0] +
                (ct_emf(c, 0, b, i, j + 1, k) - ct_emf(c, 0, b, i, j, k)) / dx[1];
          }
          if (stage == 1) {
            c->fcn[d][q] = c->fc[d][q];
            c->fc[d][q] = c->fcn[d][q] + dt * R;
          } else {
            c->fc[d][q] = 0.5 * c->fcn[d][q] + 0.5 * (c->fc[d][q] + dt * R);
          }
        }
  }
}

long or_face_count(const or_ctx* c) {
  long n = 0;
  for (int d = 0; d < c->p.ndim; ++d) {
    long m = c->nb;
    for (int t = 0; t < 3; ++t) m *= c->p.nx[t] + (t == d ? 1 : 0);
    n += m;
  }
  return n;
}

/* owned faces in [block][d][k][j][i] order */
static void ct_copy_faces(or_ctx* c, double* io, int to_ctx) {
  const int* nx = c->p.nx;
  size_t q = 0;
  for (int b = 0; b < c->nb; ++b)
    for (int d = 0; d < c->p.ndim; ++d) {
      int n[3] = {nx[0], nx[1], nx[2]};
      n[d] += 1;
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i, ++q) {
            if (to_ctx)
              c->fc[d][fcx(c, d, b, i, j, k)] = io[q];
            else
              io[q] = c->fc[d][fcx(c, d, b, i, j, k)];
          }
    }
}

void or_set_faces(or_ctx* c, const double* faces) {
  ct_copy_faces(c, (double*)faces, 1);
  const int* nx = c->p.nx;
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < nx[2]; ++k)
      for (int j = 0; j < nx[1]; ++j)
        for (int i = 0; i < nx[0]; ++i) {
          double x[3], P[OR_NV], U[OR_NV];
          or_metric m;
          cell_centre(c, b, i, j, k, x);
          or_metric_at(&c->p, x, 0, &m);
          int g[3] = {i + c->gd[0], j + c->gd[1], k + c->gd[2]};
          for (int v = 0; v < OR_NV; ++v) P[v] = c->prim[pidx(c, b, v, g[0], g[1], g[2])];
          for (int d = 0; d < c->p.ndim; ++d) {
            int hi[3] = {i, j, k};
            hi[d] += 1;
            double Bd = 0.5 * (c->fc[d][fcx(c, d, b, i, j, k)] + c->fc[d][fcx(c, d, b, hi[0], hi[1], hi[2])]);
            P[OR_B1 + d] = Bd / m.sqrtg;
          }
          P[OR_PSI] = 0.0;
          or_prim2con(&c->p, &m, P, U);
          for (int v = 0; v < OR_NV; ++v) {
            c->prim[pidx(c, b, v, g[0], g[1], g[2])] = P[v];
            c->ucur[uidx(c, b, v, i, j, k)] = m.sqrtg * U[v];
          }
        }
}

void or_get_faces(const or_ctx* c, double* faces) { ct_copy_faces((or_ctx*)c, faces, 0); }

void or_ct_ring_faces(or_ctx* c, int d, double* out) {
  ct_fill_face_ring(c);
  size_t n = (size_t)c->nb * c->fe[d][0] * c->fe[d][1] * c->fe[d][2];
  memcpy(out, c->fc[d], sizeof(double) * n);
}

/* ---- one Runge-Kutta stage ---- */

static size_t fidx(const or_ctx* c, int d, int b, int v, int i, int j, int k) {
  int n[3] = {c->p.nx[0], c->p.nx[1], c->p.nx[2]};
  n[d] += 1;
  return ((((size_t)b * OR_NV + v) * n[2] + k) * n[1] + j) * n[0] + i;
}

/* Face fluxes of block b in direction d, for faces 0..nx_d (face f lies
 * between interior cells f-1 and f). */
static void block_fluxes(or_ctx* c, int b, int d) {
  int L = c->blk[4 * b];
  int n[3] = {c->p.nx[0], c->p.nx[1], c->p.nx[2]};
  n[d] += 1;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int f[3] = {i, j, k};
        double x[3];
        long G[3];
        for (int e = 0; e < 3; ++e) {
          G[e] = (long)c->blk[4 * b + 1 + e] * c->p.nx[e] + f[e];
          x[e] = coord(c, e, L, G[e], e == d ? 0.0 : 0.5);
        }
        double F[OR_NV];
        long Nd = (long)c->p.nroot[d] * c->p.nx[d] << L;
        int axis = (G[d] == 0 && c->p.bc[d][0] == OR_BC_AXIS) || (G[d] == Nd && c->p.bc[d][1] == OR_BC_AXIS);
        if (axis) {
          for (int v = 0; v < OR_NV; ++v) F[v] = 0.0;
        } else {
          double st[6][OR_NV], PL[OR_NV], PR[OR_NV];
          for (int s = 0; s < 6; ++s) {
            int g[3] = {i + c->gd[0], j + c->gd[1], k + c->gd[2]};
            g[d] += s - 3;
            for (int v = 0; v < OR_NV; ++v) st[s][v] = c->prim[pidx(c, b, v, g[0], g[1], g[2])];
          }
          or_reconstruct(&c->p, (const double(*)[OR_NV])st, PL, PR);
          or_metric m;
          or_metric_at(&c->p, x, 0, &m);
          or_face_flux(&c->p, &m, PL, PR, d, F);
        }
        for (int v = 0; v < OR_NV; ++v) c->flux[d][fidx(c, d, b, v, i, j, k)] = F[v];
      }
}

/* Flux of variable v through face (i, j, k) of direction d of block b: the
 * face-flux arrays, or with constrained transport the ring-extended ones. */
static double* flux_slot(or_ctx* c, int d, int b, int v, int i, int j, int k) {
  return c->p.ct ? &c->xf[d][xfx(c, d, b, v, i, j, k)] : &c->flux[d][fidx(c, d, b, v, i, j, k)];
}

/* Coarse-fine flux correction: at a face where the neighbour is one level
 * finer, the coarse flux becomes the mean of the 2^(ndim-1) fine fluxes that
 * cover it, so the fluxes leaving and entering each level agree exactly. */
static void reflux_block(or_ctx* c, int b) {
  int L = c->blk[4 * b];
  for (int d = 0; d < c->p.ndim; ++d)
    for (int side = 0; side < 2; ++side) {
      long nb_[3];
      for (int e = 0; e < 3; ++e) nb_[e] = c->blk[4 * b + 1 + e];
      nb_[d] += side == 0 ? -1 : 1;
      long nbd = (long)c->p.nroot[d] << L;
      if (nb_[d] < 0 || nb_[d] >= nbd) {
        if (c->p.bc[d][side] != OR_BC_PERIODIC) continue;
        nb_[d] = (nb_[d] + nbd) % nbd;
      }
      if (lut_get(c, L, nb_) >= 0) continue; /* same level */
      /* finer neighbour? check the child block touching this face */
      long chb[3];
      for (int e = 0; e < 3; ++e) chb[e] = e < c->p.ndim ? 2 * nb_[e] : nb_[e];
      if (side == 0) chb[d] += 1;
      if (lut_get(c, L + 1, chb) < 0) continue;
      int n[3] = {c->p.nx[0], c->p.nx[1], c->p.nx[2]};
      int fcoarse = side == 0 ? 0 : n[d];
      int ffine = side == 0 ? n[d] : 0;
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int a = 0; a < n[t1]; ++a)
        for (int bb = 0; bb < n[t2]; ++bb) {
          /* global coarse transverse index -> fine block and local indices */
          double acc[OR_NV] = {0};
          int cnt = 0;
          for (int s1 = 0; s1 < (t1 < c->p.ndim ? 2 : 1); ++s1)
            for (int s2 = 0; s2 < (t2 < c->p.ndim ? 2 : 1); ++s2) {
              long Gf[3];
              Gf[d] = 0;
              long gc1 = (long)c->blk[4 * b + 1 + t1] * n[t1] + a;
              long gc2 = (long)c->blk[4 * b + 1 + t2] * n[t2] + bb;
              Gf[t1] = t1 < c->p.ndim ? 2 * gc1 + s1 : gc1;
              Gf[t2] = t2 < c->p.ndim ? 2 * gc2 + s2 : gc2;
              long fb[3];
              fb[d] = chb[d];
              fb[t1] = Gf[t1] / n[t1];
              fb[t2] = Gf[t2] / n[t2];
              int bf = lut_get(c, L + 1, fb);
              if (bf < 0) continue;
              int li[3];
              li[d] = ffine;
              li[t1] = (int)(Gf[t1] % n[t1]);
              li[t2] = (int)(Gf[t2] % n[t2]);
              for (int v = 0; v < OR_NV; ++v) acc[v] += *flux_slot(c, d, bf, v, li[0], li[1], li[2]);
              ++cnt;
            }
          if (cnt == 0) continue;
          int lc[3];
          lc[d] = fcoarse;
          lc[t1] = a;
          lc[t2] = bb;
          for (int v = 0; v < OR_NV; ++v) *flux_slot(c, d, b, v, lc[0], lc[1], lc[2]) = acc[v] / cnt;
        }
    }
}

/* L = -sum_d (F_d(+) - F_d(-)) / dx_d + sqrt(gamma) S, then the SSP-RK2 stage
 * (Shu & Osher 1988): stage 1  U1 = Un + dt L(Pn);
 * stage 2  U = 1/2 Un + 1/2 (U1 + dt L(P1)); then the inversion per cell. */
/* flux through face (i, j, k) of direction d of block b (the ring-extended
 * arrays in constrained transport) */
static double face_flux_at(const or_ctx* c, int d, int b, int v, int i, int j, int k) {
  return c->p.ct ? c->xf[d][xfx(c, d, b, v, i, j, k)] : c->flux[d][fidx(c, d, b, v, i, j, k)];
}

static void update_block(or_ctx* c, int b, int stage, double dt, long long cnt[4]) {
  int L = c->blk[4 * b];
  const int* nx = c->p.nx;
  for (int k = 0; k < nx[2]; ++k)
    for (int j = 0; j < nx[1]; ++j)
      for (int i = 0; i < nx[0]; ++i) {
        double x[3], P[OR_NV], S[OR_NV], rhs[OR_NV], U[OR_NV], Pn[OR_NV];
        or_metric m;
        cell_centre(c, b, i, j, k, x);
        or_metric_at(&c->p, x, 1, &m);
        for (int v = 0; v < OR_NV; ++v) P[v] = c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])];
        or_sources(&c->p, &m, P, S);
        for (int v = 0; v < OR_NV; ++v) rhs[v] = 0.0;
        for (int d = 0; d < c->p.ndim; ++d) {
          int ip[3] = {i, j, k};
          ip[d] += 1;
          double dx = dxl(c, d, L);
          for (int v = 0; v < OR_NV; ++v)
            rhs[v] += -(face_flux_at(c, d, b, v, ip[0], ip[1], ip[2]) - face_flux_at(c, d, b, v, i, j, k)) / dx;
        }
        for (int v = 0; v < OR_NV; ++v) rhs[v] += m.sqrtg * S[v];
        for (int v = 0; v < OR_NV; ++v) {
          size_t u = uidx(c, b, v, i, j, k);
          if (stage == 1) {
            c->un[u] = c->ucur[u];
            U[v] = c->un[u] + dt * rhs[v];
          } else {
            U[v] = 0.5 * c->un[u] + 0.5 * (c->ucur[u] + dt * rhs[v]);
          }
        }
        if (c->p.imex && !c->p.ct) {
          /* IMEX-SSP2(2,2,2) (Pareschi & Russo 2005; gamma = 1 - 1/sqrt 2) for
           * the stiff damping S(psi) = -lam psi, lam = alpha kappa, with the
           * explicit SSP-RK2 part above:
           *   Y1 = psi_n / (1 + gamma z),  z = lam dt     (stage 1's fluxes see Y1)
           *   Y2 = (psi_n + dt F(Y1) - (1 - 2 gamma) z Y1) / (1 + gamma z)
           *   psi = psi_n + dt/2 (F(Y1) + F(Y2)) - z/2 (Y1 + Y2),
           * written with U1 = Y2 and the stage-2 explicit combination. */
          const double g = 1.0 - 1.0 / sqrt(2.0);
          const double z = m.alpha * c->p.kappa * dt;
          size_t u = uidx(c, b, OR_PSI, i, j, k);
          double y1 = c->un[u] / (1.0 + g * z);
          if (stage == 1)
            U[OR_PSI] = (c->un[u] + dt * rhs[OR_PSI] - (1.0 - 2.0 * g) * z * y1) / (1.0 + g * z);
          else
            U[OR_PSI] = 0.5 * c->un[u] + 0.5 * (c->ucur[u] + dt * rhs[OR_PSI]) - 0.5 * z * (1.0 - g) * c->ucur[u] -
                        g * z * y1;
        }
        if (c->p.ct) {
          /* the field along active directions is the mean of the updated faces */
          for (int d = 0; d < c->p.ndim; ++d) {
            int hi[3] = {i, j, k};
            hi[d] += 1;
            U[OR_B1 + d] = 0.5 * (c->fc[d][fcx(c, d, b, i, j, k)] + c->fc[d][fcx(c, d, b, hi[0], hi[1], hi[2])]);
          }
          U[OR_PSI] = 0.0;
        }
        double Uu[OR_NV];
        for (int v = 0; v < OR_NV; ++v) Uu[v] = U[v] / m.sqrtg;
        int st = or_con2prim(&c->p, &m, Uu, P, floor_radius(&c->p, x), Pn);
        cnt[st] += 1;
        c->status[(size_t)b * c->nint + ((size_t)k * c->p.nx[1] + j) * c->p.nx[0] + i] = (unsigned char)st;
        if (st >= 2) {
          or_prim2con(&c->p, &m, Pn, Uu);
          for (int v = 0; v < OR_NV; ++v) U[v] = m.sqrtg * Uu[v];
        }
        for (int v = 0; v < OR_NV; ++v) c->ucur[uidx(c, b, v, i, j, k)] = U[v];
        /* the new primitives may only be written once every flux of this
         * block is final; fluxes were computed before this pass */
        for (int v = 0; v < OR_NV; ++v) c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])] = Pn[v];
      }
}

/* IMEX stage 1: the fluxes are evaluated at Y1, whose psi is
 * psi_n / (1 + gamma alpha kappa dt) (the implicit first stage); the other
 * primitives are those of U_n. */
static void imex_first_stage_psi(or_ctx* c, double dt) {
  const double g = 1.0 - 1.0 / sqrt(2.0);
  const int* nx = c->p.nx;
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < nx[2]; ++k)
      for (int j = 0; j < nx[1]; ++j)
        for (int i = 0; i < nx[0]; ++i) {
          double x[3];
          or_metric m;
          cell_centre(c, b, i, j, k, x);
          or_metric_at(&c->p, x, 0, &m);
          size_t q = pidx(c, b, OR_PSI, i + c->gd[0], j + c->gd[1], k + c->gd[2]);
          c->prim[q] = c->prim[q] / (1.0 + g * m.alpha * c->p.kappa * dt);
        }
}

void or_stage_blocks(or_ctx* c, int stage, double dt, int nsel, const int* sel) {
  if (c->p.imex && !c->p.ct && stage == 1) imex_first_stage_psi(c, dt);
  or_fill_ghosts(c);
  if (c->p.ct) {
    /* constrained transport: ring faces, ring-extended fluxes (of every block
     * when levels differ: the corrections read the finer neighbours'), the
     * coarse-fine flux correction, the face update with the EMF correction,
     * then the cells */
    ct_fill_face_ring(c);
    int allx = c->p.nlevels > 1;
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < (allx ? c->nb : nsel); ++q)
      for (int d = 0; d < c->p.ndim; ++d) ct_block_xfluxes(c, allx ? q : sel[q], d);
    if (allx) {
#pragma omp parallel for schedule(dynamic)
      for (int q = 0; q < nsel; ++q) reflux_block(c, sel[q]);
    }
    long long tot[4] = {0, 0, 0, 0};
#pragma omp parallel
    {
      long long cnt[4] = {0, 0, 0, 0};
#pragma omp for schedule(dynamic)
      for (int q = 0; q < nsel; ++q) {
        ct_update_faces(c, sel[q], stage, dt);
        update_block(c, sel[q], stage, dt, cnt);
      }
#pragma omp critical
      for (int s = 0; s < 4; ++s) tot[s] += cnt[s];
    }
    for (int s = 0; s < 4; ++s) c->counts[s] += tot[s];
    return;
  }
  int all = c->p.nlevels > 1; /* refluxing needs the fine neighbours' fluxes */
#pragma omp parallel for schedule(dynamic)
  for (int q = 0; q < (all ? c->nb : nsel); ++q) {
    int b = all ? q : sel[q];
    for (int d = 0; d < c->p.ndim; ++d) block_fluxes(c, b, d);
  }
  if (c->p.nlevels > 1) {
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < nsel; ++q) reflux_block(c, sel[q]);
  }
  long long tot[4] = {0, 0, 0, 0};
#pragma omp parallel
  {
    long long cnt[4] = {0, 0, 0, 0};
#pragma omp for schedule(dynamic)
    for (int q = 0; q < nsel; ++q) update_block(c, sel[q], stage, dt, cnt);
#pragma omp critical
    for (int s = 0; s < 4; ++s) tot[s] += cnt[s];
  }
  for (int s = 0; s < 4; ++s) c->counts[s] += tot[s];
}

void or_stage(or_ctx* c, int stage, double dt) {
  int* sel = (int*)malloc(sizeof(int) * c->nb);
  for (int b = 0; b < c->nb; ++b) sel[b] = b;
  or_stage_blocks(c, stage, dt, c->nb, sel);
  free(sel);
}

void or_step(or_ctx* c, double dt) {
  or_stage(c, 1, dt);
  or_stage(c, 2, dt);
}

/* ------------------------------------------------------------------------ */
/* AMR regridding                                                             */
/* ------------------------------------------------------------------------ */

/* Loehner (1987) estimator: the second difference of the density normalised
 * by its first differences plus a noise filter eps times the local values,
 * combined over the active directions. */
void or_estimate(or_ctx* c, double eps, double* block_err) {
  or_fill_ghosts(c);
  const int* nx = c->p.nx;
  for (int b = 0; b < c->nb; ++b) {
    double emax = 0.0;
    for (int k = 0; k < nx[2]; ++k)
      for (int j = 0; j < nx[1]; ++j)
        for (int i = 0; i < nx[0]; ++i) {
          int g[3] = {i + c->gd[0], j + c->gd[1], k + c->gd[2]};
          double num2 = 0.0, den2 = 0.0;
          double u0 = c->prim[pidx(c, b, OR_RHO, g[0], g[1], g[2])];
          for (int d = 0; d < c->p.ndim; ++d) {
            int lo[3] = {g[0], g[1], g[2]}, hi[3] = {g[0], g[1], g[2]};
            lo[d] -= 1;
            hi[d] += 1;
            double um = c->prim[pidx(c, b, OR_RHO, lo[0], lo[1], lo[2])];
            double up = c->prim[pidx(c, b, OR_RHO, hi[0], hi[1], hi[2])];
            double n = up - 2.0 * u0 + um;
            double dd = fabs(up - u0) + fabs(u0 - um) + eps * (fabs(up) + 2.0 * fabs(u0) + fabs(um));
            num2 += n * n;
            den2 += dd * dd;
          }
          double e = den2 > 0.0 ? sqrt(num2 / den2) : 0.0;
          if (e > emax) emax = e;
        }
    block_err[b] = emax;
  }
}

/* The leaf set as one flag array per level over the block lattice. */
typedef struct {
  int ndim, nlev, nx[3], bc[3][2];
  long nbl[8][3];
  unsigned char* leaf[8];
} rg_tree;

static long rg_idx(const rg_tree* t, int L, const long c[3]) {
  return (c[2] * t->nbl[L][1] + c[1]) * t->nbl[L][0] + c[0];
}

static int rg_in(const rg_tree* t, int L, const long c[3]) {
  if (L < 0 || L >= t->nlev) return 0;
  for (int k = 0; k < 3; ++k)
    if (c[k] < 0 || c[k] >= t->nbl[L][k]) return 0;
  return 1;
}

static int rg_leaf(const rg_tree* t, int L, const long c[3]) { return rg_in(t, L, c) && t->leaf[L][rg_idx(t, L, c)]; }

/* level of the leaf covering the block region (L, c), or L + 1 if finer
 * leaves subdivide it */
static int rg_cover(const rg_tree* t, int L, const long c[3]) {
  for (int Lc = L; Lc >= 0; --Lc) {
    long a[3];
    for (int k = 0; k < 3; ++k) a[k] = k < t->ndim ? c[k] >> (L - Lc) : c[k];
    if (rg_leaf(t, Lc, a)) return Lc;
  }
  return L + 1;
}

/* block regions at level L across offset dl from c, after the boundary rules
 * (none beyond an outflow boundary; through the polar axis the mirrored row at
 * phi + pi, whose cells can span two blocks) */
static int rg_neighbours(const rg_tree* t, int L, const long c[3], const int dl[3], long out[2][3]) {
  long n[3];
  int axis = 0;
  for (int k = 0; k < 3; ++k) n[k] = c[k] + dl[k];
  for (int k = 0; k < t->ndim; ++k) {
    long N = t->nbl[L][k];
    if (n[k] >= 0 && n[k] < N) continue;
    int side = n[k] < 0 ? 0 : 1, kind = t->bc[k][side];
    if (kind == OR_BC_PERIODIC) {
      n[k] = ((n[k] % N) + N) % N;
    } else if (kind == OR_BC_AXIS) {
      n[k] = side == 0 ? -1 - n[k] : 2 * N - 1 - n[k];
      axis = 1;
    } else {
      return 0;
    }
  }
  for (int k = 0; k < 3; ++k) out[0][k] = n[k];
  if (!axis || t->ndim != 3) return 1;
  long nz = t->nx[2], Nc = t->nbl[L][2] * nz, half = Nc / 2;
  long first = ((n[2] * nz + half) % Nc) / nz, last = (((n[2] + 1) * nz - 1 + half) % Nc) / nz;
  out[0][2] = first;
  if (last == first) return 1;
  for (int k = 0; k < 3; ++k) out[1][k] = n[k];
  out[1][2] = last;
  return 2;
}

static void rg_split(rg_tree* t, int L, const long c[3]) {
  t->leaf[L][rg_idx(t, L, c)] = 0;
  for (int s = 0; s < (1 << t->ndim); ++s) {
    long ch[3] = {c[0], c[1], c[2]};
    for (int k = 0; k < t->ndim; ++k) ch[k] = 2 * c[k] + ((s >> k) & 1);
    t->leaf[L + 1][rg_idx(t, L + 1, ch)] = 1;
  }
}

/* offsets dl in {-1, 0, 1}^ndim \ {0}, enumerated in a fixed order */
static int rg_offsets(int ndim, int dl[26][3]) {
  int n = 0;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int e = -1; e <= 1; ++e) {
        if (ndim < 3 && e != 0) continue;
        if (a == 0 && b == 0 && e == 0) continue;
        dl[n][0] = a;
        dl[n][1] = b;
        dl[n][2] = e;
        ++n;
      }
  return n;
}

/* whether the region (L, r), subdivided, holds leaves finer than L + 1 */
static int rg_deeper(const rg_tree* t, int L, const long r[3]) {
  for (int s = 0; s < (1 << t->ndim); ++s) {
    long ch[3] = {r[0], r[1], r[2]};
    for (int k = 0; k < t->ndim; ++k) ch[k] = 2 * r[k] + ((s >> k) & 1);
    if (rg_cover(t, L + 1, ch) == L + 2) return 1;
  }
  return 0;
}

int or_regrid_plan(const or_params* p, int nb, const int* blocks, const double* block_err, double tol_refine,
                   double tol_coarsen, int max_level, int cap, int* new_blocks) {
  rg_tree t;
  memset(&t, 0, sizeof(t));
  t.ndim = p->ndim;
  t.nlev = max_level + 1;
  for (int L = 0; L < nb; ++L)
    if (blocks[4 * L] + 1 > t.nlev) t.nlev = blocks[4 * L] + 1;
  if (t.nlev > 8) return -1;
  for (int k = 0; k < 3; ++k) {
    t.nx[k] = p->nx[k];
    t.bc[k][0] = p->bc[k][0];
    t.bc[k][1] = p->bc[k][1];
  }
  int* orig[8];
  for (int L = 0; L < t.nlev; ++L) {
    long n = 1;
    for (int k = 0; k < 3; ++k) {
      t.nbl[L][k] = (long)p->nroot[k] << (k < p->ndim ? L : 0);
      n *= t.nbl[L][k];
    }
    t.leaf[L] = (unsigned char*)calloc(n, 1);
    orig[L] = (int*)malloc(sizeof(int) * n);
    for (long q = 0; q < n; ++q) orig[L][q] = -1;
  }
  for (int b = 0; b < nb; ++b) {
    long c[3] = {blocks[4 * b + 1], blocks[4 * b + 2], blocks[4 * b + 3]};
    t.leaf[blocks[4 * b]][rg_idx(&t, blocks[4 * b], c)] = 1;
    orig[blocks[4 * b]][rg_idx(&t, blocks[4 * b], c)] = b;
  }
  /* refinement requests */
  for (int b = 0; b < nb; ++b) {
    int L = blocks[4 * b];
    long c[3] = {blocks[4 * b + 1], blocks[4 * b + 2], blocks[4 * b + 3]};
    if (L < max_level && block_err[b] > tol_refine) rg_split(&t, L, c);
  }
  /* 2:1 balance by refinement, to a fixed point */
  int dl[26][3];
  int nd = rg_offsets(p->ndim, dl);
  for (;;) {
    int changed = 0;
    for (int L = 0; L < t.nlev; ++L) {
      long n = t.nbl[L][0] * t.nbl[L][1] * t.nbl[L][2];
      unsigned char* mark = (unsigned char*)calloc(n, 1);
      unsigned char* markc[8] = {0};
      for (int Lc = 0; Lc < L; ++Lc) markc[Lc] = (unsigned char*)calloc(t.nbl[Lc][0] * t.nbl[Lc][1] * t.nbl[Lc][2], 1);
      for (long q = 0; q < n; ++q) {
        if (!t.leaf[L][q]) continue;
        long c[3] = {q % t.nbl[L][0], (q / t.nbl[L][0]) % t.nbl[L][1], q / (t.nbl[L][0] * t.nbl[L][1])};
        for (int o = 0; o < nd; ++o) {
          long r[2][3];
          int nr = rg_neighbours(&t, L, c, dl[o], r);
          for (int m = 0; m < nr; ++m) {
            int st = rg_cover(&t, L, r[m]);
            if (st < L - 1) {
              long a[3];
              for (int k = 0; k < 3; ++k) a[k] = k < t.ndim ? r[m][k] >> (L - st) : r[m][k];
              markc[st][rg_idx(&t, st, a)] = 1;
            } else if (st == L + 1 && L + 1 < t.nlev && rg_deeper(&t, L, r[m])) {
              mark[q] = 1;
            }
          }
        }
      }
      for (long q = 0; q < n; ++q)
        if (mark[q] && L + 1 < t.nlev) {
          long c[3] = {q % t.nbl[L][0], (q / t.nbl[L][0]) % t.nbl[L][1], q / (t.nbl[L][0] * t.nbl[L][1])};
          rg_split(&t, L, c);
          changed = 1;
        }
      for (int Lc = 0; Lc < L; ++Lc) {
        long m = t.nbl[Lc][0] * t.nbl[Lc][1] * t.nbl[Lc][2];
        for (long q = 0; q < m; ++q)
          if (markc[Lc][q] && t.leaf[Lc][q]) {
            long c[3] = {q % t.nbl[Lc][0], (q / t.nbl[Lc][0]) % t.nbl[Lc][1], q / (t.nbl[Lc][0] * t.nbl[Lc][1])};
            rg_split(&t, Lc, c);
            changed = 1;
          }
        free(markc[Lc]);
      }
      free(mark);
    }
    if (!changed) break;
  }
  /* coarsening: complete sibling groups of original leaves below tol_coarsen,
   * where the parent keeps the balance (checked against the refined set) */
  int ngroups = 0;
  long(*groups)[4] = (long(*)[4])malloc(sizeof(long[4]) * (size_t)(nb + 1));
  for (int L = 1; L < t.nlev; ++L) {
    long n = t.nbl[L - 1][0] * t.nbl[L - 1][1] * t.nbl[L - 1][2];
    for (long q = 0; q < n; ++q) {
      long pc[3] = {q % t.nbl[L - 1][0], (q / t.nbl[L - 1][0]) % t.nbl[L - 1][1],
                    q / (t.nbl[L - 1][0] * t.nbl[L - 1][1])};
      int ok = 1;
      for (int s = 0; s < (1 << t.ndim) && ok; ++s) {
        long ch[3] = {pc[0], pc[1], pc[2]};
        for (int k = 0; k < t.ndim; ++k) ch[k] = 2 * pc[k] + ((s >> k) & 1);
        int ob = rg_in(&t, L, ch) ? orig[L][rg_idx(&t, L, ch)] : -1;
        if (ob < 0 || !rg_leaf(&t, L, ch) || !(block_err[ob] < tol_coarsen)) ok = 0;
      }
      for (int o = 0; o < nd && ok; ++o) {
        long r[2][3];
        int nr = rg_neighbours(&t, L - 1, pc, dl[o], r);
        for (int m = 0; m < nr && ok; ++m) {
          int st = rg_cover(&t, L - 1, r[m]);
          if (st < L - 2 || (st == L && rg_deeper(&t, L - 1, r[m]))) ok = 0;
        }
      }
      if (ok) {
        groups[ngroups][0] = L - 1;
        for (int k = 0; k < 3; ++k) groups[ngroups][1 + k] = pc[k];
        ++ngroups;
      }
    }
  }
  for (int g = 0; g < ngroups; ++g) {
    int Lp = (int)groups[g][0];
    long pc[3] = {groups[g][1], groups[g][2], groups[g][3]};
    for (int s = 0; s < (1 << t.ndim); ++s) {
      long ch[3] = {pc[0], pc[1], pc[2]};
      for (int k = 0; k < t.ndim; ++k) ch[k] = 2 * pc[k] + ((s >> k) & 1);
      t.leaf[Lp + 1][rg_idx(&t, Lp + 1, ch)] = 0;
    }
    t.leaf[Lp][rg_idx(&t, Lp, pc)] = 1;
  }
  free(groups);
  /* output in (level, iz, iy, ix) order */
  int count = 0;
  for (int L = 0; L < t.nlev; ++L) {
    long n = t.nbl[L][0] * t.nbl[L][1] * t.nbl[L][2];
    for (long q = 0; q < n; ++q)
      if (t.leaf[L][q]) {
        if (count < cap) {
          new_blocks[4 * count] = L;
          new_blocks[4 * count + 1] = (int)(q % t.nbl[L][0]);
          new_blocks[4 * count + 2] = (int)((q / t.nbl[L][0]) % t.nbl[L][1]);
          new_blocks[4 * count + 3] = (int)(q / (t.nbl[L][0] * t.nbl[L][1]));
        }
        ++count;
      }
    free(t.leaf[L]);
    free(orig[L]);
  }
  return count <= cap ? count : -1;
}

/* Conservative transfer of the densitized state to a new leaf list, then the
 * inversion of every new cell. */
/* ---- regridding with constrained transport: the face fields ---- */

/* Phi^d of face F (level-L global index, a face index along d) held by an old
 * level-L leaf: the block above it along d, else the one below, after the
 * periodic wrap along d; 0 if no old level-L leaf holds it. */
static int rg_old_face(const or_ctx* old, int d, int L, const long Fin[3], double* out) {
  const int* nx = old->p.nx;
  long F[3] = {Fin[0], Fin[1], Fin[2]};
  const long Nd = ncell_l(old, d, L);
  for (int above = 1; above >= 0; --above) {
    long cell = above ? F[d] : F[d] - 1;
    if (cell < 0 || cell >= Nd) {
      if (old->p.bc[d][cell < 0 ? 0 : 1] != OR_BC_PERIODIC) continue;
      cell = ((cell % Nd) + Nd) % Nd;
    }
    long bc[3];
    int lf[3];
    for (int e = 0; e < 3; ++e) {
      long g = e == d ? cell : F[e];
      bc[e] = g / nx[e];
      lf[e] = (int)(g - bc[e] * nx[e]);
    }
    lf[d] += above ? 0 : 1;
    int b = lut_get(old, L, bc);
    if (b >= 0) {
      *out = old->fc[d][fcx(old, d, b, lf[0], lf[1], lf[2])];
      return 1;
    }
  }
  return 0;
}

/* Solves the symmetric system M y = r (n unknowns, M positive semi-definite
 * with the constants as its null space) with y_0 = 0, by Gaussian elimination
 * on the remaining n - 1 equations. */
static void rg_solve_fixed0(int n, double M[8][8], const double r[8], double y[8]) {
  double a[8][9];
  for (int i = 1; i < n; ++i) {
    for (int j = 1; j < n; ++j) a[i - 1][j - 1] = M[i][j];
    a[i - 1][n - 1] = r[i];
  }
  const int m = n - 1;
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int i = col + 1; i < m; ++i)
      if (fabs(a[i][col]) > fabs(a[piv][col])) piv = i;
    for (int j = 0; j <= m; ++j) {
      double t = a[col][j];
      a[col][j] = a[piv][j];
      a[piv][j] = t;
    }
    for (int i = col + 1; i < m; ++i) {
      double f = a[i][col] / a[col][col];
      for (int j = col; j <= m; ++j) a[i][j] -= f * a[col][j];
    }
  }
  y[0] = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    double t = a[i][m];
    for (int j = i + 1; j < m; ++j) t -= a[i][j] * y[j + 1];
    y[i + 1] = t / a[i][i];
  }
}

/* The face fields of new block b (level L) of c from the old grid (kind 0:
 * kept as old block ob, 1: refined from old parent ob, 2: coarsened from its
 * old children):
 *  - kept: a copy;
 *  - otherwise a face on the block's boundary held by an old leaf of level L
 *    across it takes that leaf's value (the same face before the regrid);
 *  - coarsened: the mean of the 2^(ndim-1) old finer faces on each face;
 *  - refined, faces on the planes of the parent's faces: the parent face plus
 *    +-1/4 of its minmod-limited differences to the neighbouring parent faces
 *    across (within the parent block; at its edge the one difference there
 *    is), so the finer faces keep the parent face's flux;
 *  - refined, faces inside a parent cell: first the mean of the two outer
 *    finer faces of that cell at the same position across, then the change of
 *    least Euclidean norm that makes all 2^ndim finer cells of the parent cell
 *    divergence-free (the outer faces already carry the parent cell's
 *    divergence, zero). */
static void rg_transfer_faces(const or_ctx* old, or_ctx* c, int b, int kind, int ob) {
  const int* nx = c->p.nx;
  const int nd = c->p.ndim;
  const int L = c->blk[4 * b];
  const long bo[3] = {c->blk[4 * b + 1], c->blk[4 * b + 2], c->blk[4 * b + 3]};
  for (int d = 0; d < nd; ++d) {
    int n[3] = {nx[0], nx[1], nx[2]};
    n[d] += 1;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          const int f[3] = {i, j, k};
          double *dst = &c->fc[d][fcx(c, d, b, i, j, k)], v;
          if (kind == 0) {
            *dst = old->fc[d][fcx(old, d, ob, i, j, k)];
            continue;
          }
          long G[3];
          for (int e = 0; e < 3; ++e) G[e] = bo[e] * nx[e] + f[e];
          if ((f[d] == 0 || f[d] == nx[d]) && rg_old_face(old, d, L, G, &v)) {
            *dst = v;
            continue;
          }
          if (kind == 2) {
            int t[2], nt = 0;
            for (int e = 0; e < nd; ++e)
              if (e != d) t[nt++] = e;
            double sum = 0.0;
            for (int q = 0; q < (1 << nt); ++q) {
              long F[3] = {G[0], G[1], G[2]};
              F[d] = 2 * G[d];
              for (int u = 0; u < nt; ++u) F[t[u]] = 2 * G[t[u]] + ((q >> u) & 1);
              double w = 0.0;
              rg_old_face(old, d, L + 1, F, &w);
              sum += w;
            }
            *dst = sum / (1 << nt);
            continue;
          }
          if (G[d] & 1) continue; /* inside a parent cell: below */
          int pl[3];
          for (int e = 0; e < 3; ++e) pl[e] = (int)((e < nd ? G[e] >> 1 : G[e]) - (e < nd ? bo[e] >> 1 : bo[e]) * nx[e]);
          const double Pc = old->fc[d][fcx(old, d, ob, pl[0], pl[1], pl[2])];
          double val = Pc;
          for (int e = 0; e < nd; ++e) {
            if (e == d) continue;
            int lo[3] = {pl[0], pl[1], pl[2]}, hi[3] = {pl[0], pl[1], pl[2]};
            lo[e] -= 1;
            hi[e] += 1;
            double dl = 0.0, dh = 0.0;
            int hl = pl[e] > 0, hh = pl[e] < nx[e] - 1;
            if (hl) dl = Pc - old->fc[d][fcx(old, d, ob, lo[0], lo[1], lo[2])];
            if (hh) dh = old->fc[d][fcx(old, d, ob, hi[0], hi[1], hi[2])] - Pc;
            double slope = hl && hh ? minmod(dl, dh) : (hl ? dl : dh);
            val += ((G[e] & 1) ? 0.25 : -0.25) * slope;
          }
          *dst = val;
        }
  }
  if (kind != 1) return;
  /* faces inside the parent cells */
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = dxl(c, d, L);
  const int ncell = 1 << nd;
  int ca[3] = {1, 1, 1};
  for (int d = 0; d < nd; ++d) ca[d] = nx[d] / 2;
  for (int pk = 0; pk < ca[2]; ++pk)
    for (int pj = 0; pj < ca[1]; ++pj)
      for (int pi = 0; pi < ca[0]; ++pi) {
        const int base[3] = {2 * pi, 2 * pj, nd == 3 ? 2 * pk : 0};
        /* unknowns: for each d, the faces at base_d + 1 of the cells a with a_d = 0 */
        int nu = 0, ud[12], ua[12];
        for (int d = 0; d < nd; ++d)
          for (int a = 0; a < ncell; ++a)
            if (!((a >> d) & 1)) {
              ud[nu] = d;
              ua[nu] = a;
              ++nu;
            }
        double x0[12], A[8][12], r[8];
        for (int q = 0; q < nu; ++q) {
          const int d = ud[q], a = ua[q];
          int lo[3], hi[3];
          for (int e = 0; e < 3; ++e) lo[e] = hi[e] = base[e] + (e < nd ? (a >> e) & 1 : 0);
          hi[d] = base[d] + 2; /* the outer high face of the cell above */
          lo[d] = base[d];     /* the outer low face of the cell below */
          x0[q] = 0.5 * (c->fc[d][fcx(c, d, b, lo[0], lo[1], lo[2])] + c->fc[d][fcx(c, d, b, hi[0], hi[1], hi[2])]);
        }
        for (int a = 0; a < ncell; ++a) {
          for (int q = 0; q < nu; ++q) A[a][q] = 0.0;
          r[a] = 0.0;
        }
        /* divergence of each finer cell with the first values */
        for (int a = 0; a < ncell; ++a)
          for (int d = 0; d < nd; ++d) {
            int cl[3];
            for (int e = 0; e < 3; ++e) cl[e] = base[e] + (e < nd ? (a >> e) & 1 : 0);
            double lo, hi;
            if (!((a >> d) & 1)) {
              int lf[3] = {cl[0], cl[1], cl[2]};
              lo = c->fc[d][fcx(c, d, b, lf[0], lf[1], lf[2])];
              int q = 0;
              while (!(ud[q] == d && ua[q] == a)) ++q;
              hi = x0[q];
              A[a][q] += 1.0 / h[d];
            } else {
              int hf[3] = {cl[0], cl[1], cl[2]};
              hf[d] += 1;
              hi = c->fc[d][fcx(c, d, b, hf[0], hf[1], hf[2])];
              int q = 0;
              while (!(ud[q] == d && ua[q] == (a & ~(1 << d)))) ++q;
              lo = x0[q];
              A[a][q] -= 1.0 / h[d];
            }
            r[a] += (hi - lo) / h[d];
          }
        /* least-norm change dx with A dx = -r: dx = -A^T y, (A A^T) y = r */
        double M[8][8], y[8];
        for (int p = 0; p < ncell; ++p)
          for (int q = 0; q < ncell; ++q) {
            M[p][q] = 0.0;
            for (int u = 0; u < nu; ++u) M[p][q] += A[p][u] * A[q][u];
          }
        rg_solve_fixed0(ncell, M, r, y);
        for (int q = 0; q < nu; ++q) {
          double at_y = 0.0;
          for (int a = 0; a < ncell; ++a) at_y += A[a][q] * y[a];
          const int d = ud[q], a = ua[q];
          int fl[3];
          for (int e = 0; e < 3; ++e) fl[e] = base[e] + (e < nd ? (a >> e) & 1 : 0);
          fl[d] = base[d] + 1;
          c->fc[d][fcx(c, d, b, fl[0], fl[1], fl[2])] = x0[q] - at_y;
        }
      }
}

void or_regrid_transfer(const or_ctx* old, or_ctx* c) {
  const int* nx = c->p.nx;
  const int nd = c->p.ndim, nch = 1 << nd;
  long long cnt[4] = {0, 0, 0, 0};
  if (c->p.ct) {
    /* constrained transport: the face fields first (the cells' field is their mean) */
    for (int b = 0; b < c->nb; ++b) {
      int L = c->blk[4 * b];
      long bc[3] = {c->blk[4 * b + 1], c->blk[4 * b + 2], c->blk[4 * b + 3]}, pb[3];
      for (int k = 0; k < 3; ++k) pb[k] = k < nd ? bc[k] >> 1 : bc[k];
      int ob = lut_get(old, L, bc), kind = 0;
      if (ob < 0) {
        ob = L > 0 ? lut_get(old, L - 1, pb) : -1;
        kind = ob >= 0 ? 1 : 2;
      }
      rg_transfer_faces(old, c, b, kind, ob);
    }
  }
  for (int b = 0; b < c->nb; ++b) {
    int L = c->blk[4 * b];
    long bc[3] = {c->blk[4 * b + 1], c->blk[4 * b + 2], c->blk[4 * b + 3]};
    int kind, ob = lut_get(old, L, bc);
    long pb[3];
    for (int k = 0; k < 3; ++k) pb[k] = k < nd ? bc[k] >> 1 : bc[k];
    if (ob >= 0) {
      kind = 0;
    } else if (L > 0 && (ob = lut_get(old, L - 1, pb)) >= 0) {
      kind = 1;
    } else {
      kind = 2;
    }
    for (int k = 0; k < nx[2]; ++k)
      for (int j = 0; j < nx[1]; ++j)
        for (int i = 0; i < nx[0]; ++i) {
          int loc[3] = {i, j, k};
          long G[3];
          for (int e = 0; e < 3; ++e) G[e] = bc[e] * nx[e] + loc[e];
          double U[OR_NV], Pg[OR_NV];
          if (kind == 0) {
            for (int v = 0; v < OR_NV; ++v) {
              U[v] = old->ucur[uidx(old, ob, v, i, j, k)];
              Pg[v] = old->prim[pidx(old, ob, v, i + old->gd[0], j + old->gd[1], k + old->gd[2])];
            }
          } else if (kind == 1) {
            /* the parent cell, and minmod slopes within the parent block */
            int pl[3];
            for (int e = 0; e < 3; ++e) pl[e] = (int)((e < nd ? G[e] >> 1 : G[e]) - pb[e] * nx[e]);
            for (int v = 0; v < OR_NV; ++v) {
              double Uc = old->ucur[uidx(old, ob, v, pl[0], pl[1], pl[2])];
              double u = Uc;
              for (int d = 0; d < nd; ++d) {
                double s = 0.0;
                if (pl[d] > 0 && pl[d] < nx[d] - 1) {
                  int lo[3] = {pl[0], pl[1], pl[2]}, hi[3] = {pl[0], pl[1], pl[2]};
                  lo[d] -= 1;
                  hi[d] += 1;
                  double Um = old->ucur[uidx(old, ob, v, lo[0], lo[1], lo[2])];
                  double Up = old->ucur[uidx(old, ob, v, hi[0], hi[1], hi[2])];
                  s = minmod(Uc - Um, Up - Uc);
                }
                u += ((G[d] & 1) ? 0.25 : -0.25) * s;
              }
              U[v] = u;
              Pg[v] = old->prim[pidx(old, ob, v, pl[0] + old->gd[0], pl[1] + old->gd[1], pl[2] + old->gd[2])];
            }
          } else {
            /* the mean of the 2^d finer cells */
            for (int v = 0; v < OR_NV; ++v) U[v] = Pg[v] = 0.0;
            for (int s = 0; s < nch; ++s) {
              long F[3], fb[3];
              int fl[3];
              for (int e = 0; e < 3; ++e) {
                F[e] = e < nd ? 2 * G[e] + ((s >> e) & 1) : G[e];
                fb[e] = F[e] / nx[e];
                fl[e] = (int)(F[e] - fb[e] * nx[e]);
              }
              int fbi = lut_get(old, L + 1, fb);
              for (int v = 0; v < OR_NV; ++v) {
                U[v] += old->ucur[uidx(old, fbi, v, fl[0], fl[1], fl[2])];
                Pg[v] += old->prim[pidx(old, fbi, v, fl[0] + old->gd[0], fl[1] + old->gd[1], fl[2] + old->gd[2])];
              }
            }
            for (int v = 0; v < OR_NV; ++v) {
              U[v] /= nch;
              Pg[v] /= nch;
            }
          }
          if (c->p.ct) {
            for (int d = 0; d < nd; ++d) {
              int hi[3] = {i, j, k};
              hi[d] += 1;
              U[OR_B1 + d] = 0.5 * (c->fc[d][fcx(c, d, b, i, j, k)] + c->fc[d][fcx(c, d, b, hi[0], hi[1], hi[2])]);
            }
            U[OR_PSI] = 0.0;
          }
          double x[3], Uu[OR_NV], Pn[OR_NV];
          or_metric m;
          cell_centre(c, b, i, j, k, x);
          or_metric_at(&c->p, x, 0, &m);
          for (int v = 0; v < OR_NV; ++v) Uu[v] = U[v] / m.sqrtg;
          int st = or_con2prim(&c->p, &m, Uu, Pg, floor_radius(&c->p, x), Pn);
          cnt[st] += 1;
          c->status[(size_t)b * c->nint + ((size_t)k * nx[1] + j) * nx[0] + i] = (unsigned char)st;
          if (st >= 2) {
            or_prim2con(&c->p, &m, Pn, Uu);
            for (int v = 0; v < OR_NV; ++v) U[v] = m.sqrtg * Uu[v];
          }
          for (int v = 0; v < OR_NV; ++v) {
            c->ucur[uidx(c, b, v, i, j, k)] = U[v];
            c->prim[pidx(c, b, v, i + c->gd[0], j + c->gd[1], k + c->gd[2])] = Pn[v];
          }
        }
  }
  for (int s = 0; s < 4; ++s) c->counts[s] += cnt[s];
}
