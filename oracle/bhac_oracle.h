/*
 * Plain FP64 CPU oracle for the per-block finite-volume GRMHD update
 * (test infrastructure only: tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it; the product path never links it).
 *
 * The paper (Sec. 2, "Code overview") states the method only in words: a
 * high-resolution shock-capturing finite-volume scheme on block-based AMR, in
 * any covariant coordinate system, with second-order time stepping, PPM
 * reconstruction, and Newton-Raphson conserved-to-primitive inversion with
 * backup strategies.  Everything concrete below (3+1 "Valencia" GRMHD
 * equations, HLL/TVDLF, GLM cleaning, SSP-RK2, Kerr-Schild metric, floors) is
 * the standard published form of those ingredients, restated here step by step
 * in the order the method applies them; every reading of a point the paper
 * leaves open is listed in the design notes of the repository.
 *
 * Every function here is pinned by the tests against facts outside the
 * oracle (closed forms, the covariant formulation, invariants, brute force,
 * convergence to exact solutions).  The GLM source's metric terms are a
 * reading (the paper gives no cleaning equations), pinned against the
 * covariant damped cleaning equation plus the one term the reading adds.  The
 * SRMHD shock tube is a configuration with no printed reference solution in
 * the paper: its stored profile is a regression record written by the oracle,
 * not a pin; the functions it exercises are each pinned.
 *
 * Conventions
 *   primitive order : rho, p, u^1, u^2, u^3, B^1, B^2, B^3, psi
 *                     (u^i = W v^i, contravariant code-coordinate components)
 *   conserved order : D, S_1, S_2, S_3, tau, B^1, B^2, B^3, psi
 *                     (stored densitized by sqrt(gamma) inside the grid)
 *   arrays          : [block][var][k][j][i], i fastest; interior only unless
 *                     the name says "ghosted".
 */
#ifndef BHAC_ORACLE_H
#define BHAC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NV 9

enum { OR_RHO = 0, OR_P = 1, OR_U1 = 2, OR_U2 = 3, OR_U3 = 4, OR_B1 = 5, OR_B2 = 6, OR_B3 = 7, OR_PSI = 8 };
enum { OR_D = 0, OR_S1 = 1, OR_S2 = 2, OR_S3 = 3, OR_TAU = 4 };

/* coordinate systems */
enum { OR_CART = 0, OR_KS = 1, OR_MKS = 2 };
/* boundary kinds per face of the root domain */
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_AXIS = 2, OR_BC_NOINFLOW = 3 };

typedef struct {
  int ndim;              /* 1..3 active dimensions */
  int nx[3];             /* interior cells per block per dimension (1 if inactive) */
  int ng;                /* ghost cells per side in active dimensions (3) */
  int nroot[3];          /* level-0 blocks per dimension */
  int nlevels;           /* refinement levels present (1 = uniform) */
  double xmin[3], xmax[3];
  int coords;            /* OR_CART, OR_KS (r, theta, phi) or OR_MKS (ln r, theta/pi, phi) */
  double spin, mass;     /* Kerr parameter a and mass M (M = 0 gives flat curvilinear space) */
  int bc[3][2];          /* boundary kind at [dim][low/high] */
  int recon;             /* 0 PPM, 1 minmod */
  int riemann;           /* 0 HLL, 1 TVDLF */
  double gamma_ad;       /* ideal-gas adiabatic index */
  double cfl;            /* Courant number */
  double ch, kappa;      /* GLM cleaning speed and damping rate */
  double c2p_tol;        /* Newton stopping tolerance on |dZ|/Z */
  int c2p_maxit;         /* Newton iteration cap */
  double rho_floor, rho_floor_pow, p_floor, p_floor_pow, w_max;
  int ct;                /* 0: GLM cleaning; 1: staggered-mesh constrained transport
                            (any level structure whose touching leaves differ by at most
                            one level; psi is not evolved, ch and kappa are ignored) */
  int imex;              /* 0: the cleaning damping -alpha kappa psi is an explicit source;
                            1: it is the implicit part of IMEX-SSP2(2,2,2) */
  int c2p_nk;            /* primary inversion: 0 Newton-Raphson with the analytic Jacobian,
                            1 Jacobian-free Newton-Krylov (GMRES on difference quotients) */
} or_params;

/* Spatial metric at a point plus its first derivatives along the code
 * coordinates: da[k] = d_k alpha, db[k][i] = d_k beta^i, dg[k][i][j] = d_k gamma_ij. */
typedef struct {
  double alpha, beta[3], g[3][3], gi[3][3], sqrtg;
  double da[3], db[3][3], dg[3][3][3];
} or_metric;

/* ---- point-wise physics (undensitized quantities) ---- */
void or_metric_at(const or_params* p, const double x[3], int with_derivs, or_metric* m);
void or_prim2con(const or_params* p, const or_metric* m, const double P[OR_NV], double U[OR_NV]);
void or_flux(const or_params* p, const or_metric* m, const double P[OR_NV], int dir, double F[OR_NV]);
void or_wavespeeds(const or_params* p, const or_metric* m, const double P[OR_NV], int dir,
                   double* lam_minus, double* lam_plus);
void or_sources(const or_params* p, const or_metric* m, const double P[OR_NV], double S[OR_NV]);
/* Returns status 0 ok, 1 fallback solver used, 2 floors applied, 3 failed (guess kept).
 * r_floor is the radius used by the floor profiles. */
int or_con2prim(const or_params* p, const or_metric* m, const double U[OR_NV],
                const double Pguess[OR_NV], double r_floor, double P[OR_NV]);
/* Face states of all variables at the face between stencil cells 2 and 3 of st[6][OR_NV]. */
void or_reconstruct(const or_params* p, const double st[6][OR_NV], double PL[OR_NV], double PR[OR_NV]);
/* Densitized numerical flux (HLL or TVDLF) through a face with metric m. */
void or_face_flux(const or_params* p, const or_metric* m, const double PL[OR_NV],
                  const double PR[OR_NV], int dir, double F[OR_NV]);

/* ---- the block grid ---- */
typedef struct or_ctx or_ctx;
/* blocks: nblocks x {level, ix, iy, iz}; only leaf blocks are listed. */
or_ctx* or_create(const or_params* p, int nblocks, const int* blocks);
void or_destroy(or_ctx* c);
/* Loads interior primitives (floors are not applied) and sets U from them. */
void or_set_prims(or_ctx* c, const double* prims);
void or_get_prims(const or_ctx* c, double* prims);
void or_get_prims_ghosted(const or_ctx* c, double* prims);
void or_get_cons(const or_ctx* c, double* cons);          /* densitized, interior */
void or_fill_ghosts(or_ctx* c);
double or_cfl_dt(or_ctx* c);
/* One Runge-Kutta stage (1 or 2) over every leaf block, or over a list of blocks. */
void or_stage(or_ctx* c, int stage, double dt);
void or_stage_blocks(or_ctx* c, int stage, double dt, int nsel, const int* sel);
void or_step(or_ctx* c, double dt);
void or_c2p_counts(const or_ctx* c, long long counts[4]);
/* per interior cell ([block][k][j][i]): inversion outcome of the last stage */
void or_c2p_status(const or_ctx* c, unsigned char* status);
int or_ghosted_cells(const or_ctx* c);                    /* per block, with ghosts */

/* ---- constrained transport (params.ct = 1) ----
 * The evolved field is Phi^d = sqrt(gamma) B^d at the centre of each face
 * normal to an active direction d.  Owned faces of a block: index 0..nx_d
 * along d, the block's cells across; layout [block][d][k][j][i] over the
 * active d in order, each over (nx_d + 1) x (cells across), i fastest.
 * or_set_faces replaces B^d of the loaded state by the face averages
 * (sqrt(gamma) B^d = (Phi^d_low + Phi^d_high) / 2) and recomputes U. */
long or_face_count(const or_ctx* c);                      /* owned faces, all blocks */
void or_set_faces(or_ctx* c, const double* faces);
void or_get_faces(const or_ctx* c, double* faces);
/* Fills the ring faces (the faces one cell outside each block, across) from
 * the owned ones and copies Phi^d over every block's ring-extended face array,
 * [block][k][j][i] with extents nx_e + 2 across in active directions e, nx_d + 1
 * along d (the ring at local index -1 and nx_e); a test accessor. */
void or_ct_ring_faces(or_ctx* c, int d, double* out);

/* ---- AMR regridding ----
 * or_estimate: Loehner's error estimator on the density of every interior cell
 * (ghosts filled first), E = sqrt(sum_d N_d^2 / sum_d D_d^2) with
 * N_d = u_+ - 2 u_0 + u_-, D_d = |u_+ - u_0| + |u_0 - u_-| + eps (|u_+| + 2|u_0| + |u_-|),
 * maximum per block into block_err[nb].
 * or_regrid_plan: the new leaf list from the old one and the block errors:
 * refine a leaf with err > tol_refine below max_level, balance 2:1 across
 * faces, edges and corners (boundary rules included) by refining coarser
 * neighbours, then coarsen every complete sibling group whose members all
 * have err < tol_coarsen where the parent keeps the 2:1 balance.  Output
 * sorted by (level, iz, iy, ix); returns the count, or -1 if cap is too small.
 * or_regrid_transfer: conservative transfer of the densitized conserved state
 * from `old` to `fresh` (same parameters, new leaf list): a kept block is
 * copied, a refined one prolonged (each child cell the parent value plus
 * minmod-limited slopes times +-1/4, slopes within the parent block only),
 * a coarsened one restricted (the mean of its 2^d children); then every cell
 * is inverted (guess: the parent's or the children's mean primitives) with
 * floors, as after a stage.  With constrained transport the face fields are
 * transferred first (kept: copied; a face on a changed block's boundary held
 * by an old leaf of the same level: that value; coarsened: the mean of the
 * finer faces; refined: parent faces split with +-1/4 of their limited
 * differences across, faces inside a parent cell from the least-norm
 * divergence-free completion) and the cells' field is the mean of their
 * faces.  Refinement needs nx even in the active directions. */
void or_estimate(or_ctx* c, double eps, double* block_err);
int or_regrid_plan(const or_params* p, int nb, const int* blocks, const double* block_err, double tol_refine,
                   double tol_coarsen, int max_level, int cap, int* new_blocks);
void or_regrid_transfer(const or_ctx* old, or_ctx* fresh);

#ifdef __cplusplus
}
#endif
#endif
