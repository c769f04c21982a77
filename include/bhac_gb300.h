/*
 * bhac_gb300.h - C ABI of the GB300 (sm_103a) per-block finite-volume GRMHD update.
 *
 * The library advances ideal GRMHD on a grid of equal-sized blocks with ghost
 * cells, the data-parallel core of the method in Sec. 2 of the paper ("Code
 * overview"): a shock-capturing finite-volume scheme on block-based AMR in a
 * covariant coordinate system, second-order two-stage time stepping, PPM (or
 * minmod) reconstruction and a Newton conserved-to-primitive inversion with
 * backup strategies.  The ghost-cell fill between blocks of the same level is
 * the kernel the paper singles out (Sec. 4.3, the roofline figure; Sec. 5.1).
 *
 * Conventions shared by every entry point
 *   - primitive variables, in this order: rho, p, u^1, u^2, u^3, B^1, B^2, B^3, psi
 *     (u^i = W v^i in contravariant code-coordinate components; psi is the GLM
 *     cleaning scalar);
 *   - conserved variables, in this order: D, S_1, S_2, S_3, tau, B^1, B^2, B^3, psi,
 *     each multiplied by sqrt(gamma) of its cell;
 *   - host/device arrays of cell data are [block][var][k][j][i] over the interior
 *     cells of every block, i fastest, FP64, in the block order given at init;
 *   - every call is asynchronous on the stream given at init, except calls that
 *     return values through host pointers, which synchronise that stream;
 *   - errors are returned as bhac_status; nothing traps, aborts or exits.
 *
 * Ownership: device memory belongs to the caller, who passes one arena of at
 * least bhac_query_sizes() bytes at init (e.g. the data pointer of a torch
 * uint8 tensor).  The library never allocates or frees device memory.  The
 * context itself (host memory) is owned by the library until bhac_destroy().
 * A context is not thread-safe.
 */
#ifndef BHAC_GB300_H
#define BHAC_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bhac_ctx bhac_ctx;

typedef enum {
  BHAC_OK = 0,
  BHAC_ERR_ARG = 1,      /* invalid argument or descriptor */
  BHAC_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  BHAC_ERR_NOMEM = 3,    /* the arena is smaller than bhac_query_sizes(), or a device allocation failed */
  BHAC_ERR_STATE = 4,    /* call out of order (e.g. step before set_prims) */
  BHAC_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
  BHAC_WARN_C2P = 6      /* some cells failed the inversion and kept their previous state */
} bhac_status;

enum { BHAC_COORDS_CART = 0, BHAC_COORDS_KS = 1, BHAC_COORDS_MKS = 2 };
enum { BHAC_BC_PERIODIC = 0, BHAC_BC_OUTFLOW = 1, BHAC_BC_AXIS = 2, BHAC_BC_NOINFLOW = 3 };
enum { BHAC_RECON_PPM = 0, BHAC_RECON_MINMOD = 1 };
enum { BHAC_RIEMANN_HLL = 0, BHAC_RIEMANN_TVDLF = 1 };
enum { BHAC_PREC_FP64 = 0, BHAC_PREC_MIXED = 1 };
enum { BHAC_DIVB_GLM = 0, BHAC_DIVB_CT = 1 };
enum { BHAC_C2P_NEWTON = 0, BHAC_C2P_NK = 1 };

/* Grid and scheme description, copied at init. */
typedef struct {
  int ndim;              /* 2 or 3 active dimensions */
  int nx[3];             /* interior cells per block per dimension (1 if inactive) */
  int nghost;            /* ghost cells per side in active dimensions; must be 3 */
  int nroot[3];          /* level-0 blocks per dimension */
  int nlevels;           /* refinement levels (1 = uniform grid) */
  double xmin[3], xmax[3];
  int coords;            /* BHAC_COORDS_*: Cartesian Minkowski, Kerr-Schild (r, th, ph) or
                            modified KS (x1 = ln r, x2 = th/pi, x3 = ph) */
  double spin, mass;     /* Kerr a and M (M = 0: flat space in those coordinates) */
  int bc[3][2];          /* BHAC_BC_* at [dimension][low, high] */
  int recon;             /* BHAC_RECON_* */
  int riemann;           /* BHAC_RIEMANN_* */
  int precision;         /* BHAC_PREC_FP64, or BHAC_PREC_MIXED: FP32 reconstruction,
                            fluxes and sources summed into FP64 conserved state;
                            FP64 Newton inversion started from the FP32 previous
                            primitives; a floored cell's D, S_i, tau rebuilt in FP32 */
  double gamma_ad;       /* ideal-gas index */
  double cfl;            /* Courant number */
  double ch, kappa;      /* GLM cleaning speed and damping rate */
  double c2p_tol;        /* Newton stops at the first step with |dZ| <= c2p_tol Z */
  int c2p_maxit;         /* Newton iteration cap */
  double rho_floor, rho_floor_pow, p_floor, p_floor_pow, w_max;
                         /* floors rho >= rho_floor r^rho_floor_pow, p >= p_floor r^p_floor_pow,
                            W <= w_max; r = 1 in Cartesian coordinates */
  int divb;              /* BHAC_DIVB_GLM: GLM cleaning (psi evolved with ch, kappa);
                            BHAC_DIVB_CT: staggered-mesh constrained transport of face
                            fields (psi stays 0, ch and kappa are ignored; with
                            refinement levels, leaves touching across a face, edge or
                            corner must differ by at most one level, else
                            BHAC_ERR_ARG).  In the mixed form the face states and
                            fluxes are FP32; the EMFs, the face update and the face
                            field stay FP64, so div B stays at FP64 round-off */
  int imex;              /* 0: the cleaning damping -alpha kappa psi is an explicit source
                            of both stages; 1: it is the implicit part of the IMEX-SSP2(2,2,2)
                            scheme (Pareschi & Russo 2005) whose explicit part is the SSP-RK2
                            step, so any kappa dt is stable (Sec. 2: implicit/explicit time
                            stepping for stiff sources).  Ignored with constrained transport. */
  int c2p_solver;        /* primary conserved-to-primitive solver (Sec. 2: Newton-Raphson and
                            Newton-Krylov solvers with backups): BHAC_C2P_NEWTON, 2-D
                            Newton-Raphson with the analytic Jacobian; BHAC_C2P_NK,
                            Jacobian-free Newton-Krylov (GMRES on difference quotients of the
                            same residuals).  Both stop at |dZ| <= c2p_tol Z and share the
                            bisection backup and the floors. */
} bhac_grid_desc;

/* One leaf block: refinement level and integer block coordinates at that level. */
typedef struct {
  int level, ix, iy, iz;
} bhac_block_desc;

/* Device bytes the arena must hold for this grid (tables, state, ghost maps).
 * Returns BHAC_ERR_ARG for an invalid description.
 * Source: Sec. 2 (the block-based grid whose blocks carry ghost cells); sizing
 * the caller-owned arena has no counterpart in the paper, whose Fortran code
 * allocates its own blocks. */
bhac_status bhac_query_sizes(const bhac_grid_desc* desc, const bhac_block_desc* blocks, int nblocks,
                             size_t* device_bytes_out);

/* Source: Sec. 2 (leaf blocks of a block-based tree grid, each with its ghost
 * cells); the ghost maps built here are the device form of the ghost-cell
 * exchange of Sec. 4.3 (fill_gc_srl) and Sec. 5.1.
 *
 * Creates a context on the current CUDA device.  `device_arena` must be a device
 * pointer to >= bhac_query_sizes() bytes, 256-byte aligned; it stays owned by
 * the caller and must outlive the context.  `cuda_stream` is a cudaStream_t (or
 * NULL for the legacy default stream).  Builds the ghost-cell maps on the host
 * (same-level copies and the physical boundary rules) and uploads them. */
bhac_status bhac_init_grid(bhac_ctx** out, const bhac_grid_desc* desc, const bhac_block_desc* blocks,
                           int nblocks, void* device_arena, size_t arena_bytes, void* cuda_stream);

/* Source: Sec. 2 (the scheme works in general covariant coordinates); the paper names no
 * metric, so the Kerr-Schild / modified Kerr-Schild forms (x1 = ln r,
 * theta = pi x2, no polar squeeze) are the hot-path reading of the torus set-ups.
 *
 * Evaluates the metric tables on the device in FP64: lapse, shift, spatial
 * metric, its inverse, sqrt(gamma), their first derivatives along x1 and x2
 * (forward-mode dual numbers) and the floor profiles, at cell centres and at
 * x1- and x2-faces.  The metric must be phi-independent.  `kind` and `spin_a`,
 * `mass` override the descriptor's coords/spin/mass; `mks_params` is reserved
 * and may be NULL. */
bhac_status bhac_set_metric(bhac_ctx* ctx, int kind, double spin_a, double mass, const double* mks_params);

/* Source: Sec. 2 (the scheme evolves integrated conserved variables and
 * recovers primitives from them); this is the inverse map, primitives to
 * conserved, used to load a state.  The paper has no entry point of its own.
 *
 * Loads interior primitives ([block][var][k][j][i], FP64; host pointer if
 * on_device == 0, device pointer otherwise) and sets the conserved state from
 * them.  Floors are not applied. */
bhac_status bhac_set_prims(bhac_ctx* ctx, const double* prims, int on_device);

/* Source: Sec. 4.3 (fill_gc_srl, the same-level ghost-cell fill the roofline
 * analysis singles out) and Sec. 5.1 (the ghost-cell exchange whose serial
 * region was the main bottleneck); cross-level values by restriction and
 * prolongation follow the block-based AMR of Sec. 2.  The physical boundary
 * rules (axis, no-inflow) are the hot-path reading: the paper is silent.
 *
 * Fills every ghost cell from the owning block (same level) or the boundary
 * rule: periodic wrap; outflow copy; no-inflow (outflow, then u^d clamped so
 * that nothing enters); polar axis (mirror in theta, flip u^theta and B^theta,
 * and take the cell at phi + pi in 3-D). */
bhac_status bhac_fill_ghosts(bhac_ctx* ctx);

/* Source: Sec. 2 (explicit high-resolution shock-capturing scheme, hence a
 * Courant limit); the paper gives no CFL formula, so the "maxsum" form below is
 * the hot-path reading (one rate per cell summed over directions).
 *
 * Computes dt = cfl / max over interior cells of sum_d c_d/dx_d (c_d: largest of
 * the fast-magnetosonic speeds and the GLM speeds along d) into device memory;
 * also returns it through dt_host when non-NULL (synchronises the stream).
 * Right after a load (bhac_set_prims, bhac_set_prims_host_async), or a
 * previous bhac_cfl_dt with no stage in between, the rate is already on the
 * device and no kernel runs. */
bhac_status bhac_cfl_dt(bhac_ctx* ctx, double* dt_host_or_null);

/* Source: Sec. 2 (second-order time stepping of a finite-volume scheme with PPM
 * reconstruction and Newton-Raphson inversion with backup strategies) and
 * Sec. 4.2 (one cell-update = one cell through one sub-step of the two-step
 * integrator).  The stepper (SSP-RK2), the Riemann solvers, the GLM cleaning and
 * the inversion's formulation are the hot-path readings of that paragraph.
 *
 * One SSP-RK2 step (two stages) of size dt: ghost fill, stage 1, ghost fill,
 * stage 2; each stage reconstructs, computes HLL/TVDLF face fluxes, adds the
 * geometric and GLM sources, updates the conserved state and inverts it to
 * primitives.  dt <= 0 uses the device dt of the last CFL evaluation (the step
 * itself refreshes it from its final primitives), so steps can be captured in
 * a CUDA graph with no host round trip. */
bhac_status bhac_step(bhac_ctx* ctx, double dt);

/* One RK stage (1 or 2) with its preceding ghost fill (Sec. 4.2: a sub-step). */
bhac_status bhac_stage(bhac_ctx* ctx, int stage, double dt);

/* Replaces the conserved state that bhac_set_prims derived from the
 * primitives by `cons` (densitized, [block][var][k][j][i] interior, as
 * bhac_get_cons returns it).  Call after bhac_set_prims.  Restoring both
 * primitives and conserved variables of a saved state resumes a run bit for
 * bit (the conserved state is not re-derived from the primitives).  Host
 * copies synchronise the stream. */
bhac_status bhac_set_cons(bhac_ctx* ctx, const double* cons, int on_device);

/* Copies interior primitives (or densitized conserved variables) out, same
 * layout as bhac_set_prims; host copies synchronise the stream.
 * Source: Sec. 2 (primitive and integrated conserved variables of the scheme);
 * reading state back has no counterpart in the paper. */
bhac_status bhac_get_prims(bhac_ctx* ctx, double* out, int on_device);
bhac_status bhac_get_cons(bhac_ctx* ctx, double* out, int on_device);

/* Constrained transport (divb = BHAC_DIVB_CT).  Source: Sec. 2 (staggered-mesh
 * constrained transport in covariant coordinates); the edge electric field is
 * the hot-path reading: the mean of the four upwinded (HLL/TVDLF) face fluxes
 * of B around each edge, the face update the discrete curl, so each cell's
 * sum_d (Phi^d_high - Phi^d_low) / dx_d keeps its initial value to round-off.
 *
 * The evolved field is Phi^d = sqrt(gamma) B^d at the centre of every face
 * normal to an active direction d.  Layout: for each block, for each active d
 * in order, the block's faces 0..nx_d along d and its cells across, [k][j][i],
 * i fastest (a face on a block boundary appears in both blocks, with equal
 * values).  bhac_set_faces loads them (host pointer if on_device == 0, device
 * pointer otherwise; host copies synchronise the stream) after bhac_set_prims,
 * replaces the cell field of the primitives by the face means
 * (sqrt(gamma) B^d = (Phi^d_low + Phi^d_high) / 2), sets psi = 0 and recomputes
 * the conserved state; a step before it returns BHAC_ERR_STATE.
 * bhac_get_faces reads them back in the same layout.  BHAC_ERR_STATE for a
 * grid in the cleaning form.
 *
 * Across refinement levels (Sec. 2 pairs the scheme with block-based tree
 * AMR; the transfer rules are the hot-path reading): a face one cell outside a
 * block takes the face of the leaf at the block's level, else the coarser face
 * it lies on or the mean of the two faces of the coarser cell it cuts, else
 * the mean of the finer faces on it; the coarse flux through a face on a level
 * boundary is the mean of the finer fluxes; an edge that a finer leaf touches
 * takes the mean of the finer EMFs along it.  A coarse face on a level boundary
 * then changes by the mean of the changes of the finer faces covering it, so a
 * loaded state whose coarse faces there are the mean of the finer ones keeps
 * that to round-off, with every cell's divergence. */
bhac_status bhac_set_faces(bhac_ctx* ctx, const double* faces, int on_device);
bhac_status bhac_get_faces(bhac_ctx* ctx, double* faces, int on_device);

/* AMR regridding.  Source: Sec. 2 (block-based tree AMR) and Sec. 7 (extending
 * the work to AMR runs); the paper names no refinement criterion, so the
 * estimator is the reading: Loehner's normalised second difference of the
 * density, E = sqrt(sum_d N_d^2 / sum_d D_d^2) over the active directions with
 * N_d = u_+ - 2 u_0 + u_- and D_d = |u_+ - u_0| + |u_0 - u_-| + eps (|u_+| + 2|u_0| + |u_-|),
 * the default of the MPI-AMRVAC toolkit BHAC is built on.
 *
 * bhac_estimate: fills the ghost cells and writes the largest E of each block's
 * interior cells to the host array block_err[nblocks] (block order of the
 * context); synchronises the stream.  (Mixed form: on the FP32 primitives.)
 *
 * bhac_regrid_plan (host only): the new leaf list.  Leaves with
 * block_err > tol_refine below max_level (< desc->nlevels) are split; then
 * coarser leaves are split until every pair of leaves touching across a face,
 * an edge or a corner (through periodic and polar-axis boundaries too) differs
 * by at most one level, a leaf next to a block region holding leaves two or
 * more levels finer counting as touching them; then every complete group of
 * 2^ndim sibling leaves of the input, each with block_err < tol_coarsen, whose
 * parent would keep that balance, is merged into the parent.  Output in
 * (level, iz, iy, ix) order into out[cap]; *nout is the count
 * (BHAC_ERR_NOMEM if it exceeds cap; BHAC_ERR_ARG for an invalid list).
 *
 * bhac_regrid_transfer: moves the state of `old` to `fresh`, a context made by
 * bhac_init_grid + bhac_set_metric with the same descriptor and the planned
 * leaves (each new leaf kept, one level finer or one level coarser than
 * leaves of `old`).  The densitized conserved state is copied, prolonged
 * (parent value plus minmod-limited slopes within the parent block, zero at
 * its faces, times +-1/4 per direction) or restricted (mean of the 2^ndim
 * children), so its volume integrals are unchanged; every new cell is then
 * inverted with floors (guess: the parent's or the children's mean
 * primitives) as after a stage.  Asynchronous on fresh's stream, which first
 * waits for the work enqueued on old's; `old` may be destroyed once fresh's
 * stream has passed the call.  Both contexts use the same div B control.  With
 * constrained transport (the loaded faces of `old` required, BHAC_ERR_STATE
 * otherwise; nx even in every active direction, BHAC_ERR_ARG otherwise) the
 * face fields go first: a kept block's are copied; a changed block's face on
 * its boundary that an old leaf of the same level held keeps that value; a
 * coarsened block's faces are the mean of the old finer faces on them; a
 * refined block's faces on its parent's face planes are the parent face plus
 * +-1/4 of its minmod-limited differences to the parent faces beside it
 * (within the parent block, one-sided at its edge), keeping the parent face's
 * flux, and the faces inside a parent cell are the mean of the two outer
 * faces at the same place plus the least-norm change that makes the finer
 * cells divergence-free; then the cells' field is the mean of their faces.
 * Reading of the hot path (the paper names no transfer rule). */
bhac_status bhac_estimate(bhac_ctx* ctx, double eps, double* block_err);
bhac_status bhac_regrid_plan(const bhac_grid_desc* desc, const bhac_block_desc* blocks, int nblocks,
                             const double* block_err, double tol_refine, double tol_coarsen, int max_level,
                             bhac_block_desc* out, int cap, int* nout);
bhac_status bhac_regrid_transfer(const bhac_ctx* old_ctx, bhac_ctx* fresh_ctx);

/* Pipelined host transfers, for a host-side loop that feeds every step its
 * primitives from host memory and reads every result back while the kernels of
 * the neighbouring steps run.  The context owns two copy streams, one per
 * direction, and the arena two staging buffers of the interior primitives
 * (bhac_query_sizes counts them); the host link carries both directions at
 * once.
 *
 * bhac_set_prims_host_async: copies interior primitives ([block][var][k][j][i],
 * FP64) from page-locked host memory into the input staging buffer on the
 * host-to-device copy stream, as soon as the previous load has consumed that
 * buffer; the context's stream then waits for the copy and loads it as
 * bhac_set_prims does (one kernel: ghosted primitives, conserved state and
 * the CFL rate of the loaded primitives).  Returns once
 * enqueued; `host_prims` must stay unchanged until a later bhac_host_fence()
 * has been followed by a synchronisation of the context's stream.
 *
 * bhac_get_prims_host_async: gathers the current interior primitives into the
 * output staging buffer on the context's stream, after the previous read-back
 * has drained it, then copies them to page-locked `host_prims` on the
 * device-to-host copy stream.  Returns once enqueued.
 *
 * bhac_host_fence: orders the copy streams and the context's stream both ways:
 * transfers enqueued after the fence start after the work enqueued on the
 * stream before it, and work enqueued on the stream after the fence starts
 * after every transfer enqueued before it.  Synchronising the stream after a
 * fence therefore waits for all transfers.
 *
 * Pageable host memory is rejected (BHAC_ERR_ARG).  These calls order work
 * across the context's copy streams with events; they are not meant for a
 * stream that is being captured (bhac_graph_capture records steps only). */
bhac_status bhac_set_prims_host_async(bhac_ctx* ctx, const double* host_prims);
bhac_status bhac_get_prims_host_async(bhac_ctx* ctx, double* host_prims);
bhac_status bhac_host_fence(bhac_ctx* ctx);

/* Per interior cell, the inversion outcome of the last stage run (0 Newton
 * converged, 1 backup solver, 2 floors applied, 3 failed and kept the
 * previous primitives), one byte per cell, [block][k][j][i].  Host copies
 * synchronise the stream. */
bhac_status bhac_get_c2p_status(bhac_ctx* ctx, unsigned char* out, int on_device);

/* The current FP64 primitive state including ghost cells, [block][var][k][j][i]
 * over the ghosted extents (nx + 2 nghost per active dimension), e.g. after
 * bhac_fill_ghosts to check the fill.  FP64 form only (BHAC_ERR_STATE for the
 * mixed form, whose fills write the FP32 copy).  Host copies synchronise the
 * stream. */
bhac_status bhac_get_prims_ghosted(bhac_ctx* ctx, double* out, int on_device);

/* Source: Sec. 2 (Newton-Raphson inversion backed by fall-back solvers); the
 * outcome classes are the hot-path reading of those fall-backs.
 *
 * Inversion outcome counts accumulated since init, per cell and stage:
 * [0] Newton converged, [1] backup solver used, [2] floors applied,
 * [3] failed (previous primitives kept).  Synchronises the stream. */
bhac_status bhac_get_diagnostics(bhac_ctx* ctx, long long counts[4]);

/* Kernel launches one bhac_step makes on the context's stream: per stage one
 * cross-level node pass per dependency depth (AMR grids), the ghost gather,
 * the stage kernel and, where levels meet, the reflux kernel; with constrained
 * transport the ghost gather (and node passes), the ring-face copy, the
 * face-flux, face-update and cell kernels, and with refinement levels also
 * the ring-face means, the coarse-fine flux correction, the edge EMFs and
 * their correction; with IMEX one more pass before stage 1. */
bhac_status bhac_launches_per_step(const bhac_ctx* ctx, int* launches);

/* Kernel launch shape of the stage kernel: tile of tx x ty cells per CTA column
 * (must divide the block), threads per CTA (a multiple of 32, at most 256),
 * persistent = k > 0 for k CTAs per SM pulling (block, tile) items from a device
 * work counter (0: one CTA per item), and min_ctas = 1, 2 or 3: the register
 * bound the 3-D kernel is compiled for (2 trades a few spilled registers for two
 * resident CTAs per SM; 3 applies to the face kernel of the split form, see
 * bhac_set_split, and means 2 for the fused kernel), and producer_warps = p > 0 (3-D only, p * 32 < threads)
 * for the warp-specialised form: p warps compute the next plane's face fluxes
 * while the others update the current plane's cells (0: the phased form).
 * tx, ty, threads, min_ctas = 0 keep the current setting.  Results do not
 * depend on the launch shape.  The default after bhac_init_grid: 256 threads,
 * one CTA per item, and the largest of the tiles 32x16, 16x16, 16x8, 8x8
 * that divides the block and fits the shared-memory limit; in the 3-D mixed
 * form the largest of them up to 16x16 that leaves room for two CTAs per SM,
 * with min_ctas = 2. */
bhac_status bhac_set_launch(bhac_ctx* ctx, int tx, int ty, int threads, int persistent, int min_ctas,
                            int producer_warps);

/* Split form of the stage (a measured alternative to the fused kernel, off by
 * default; chunks = 0 restores the fused form).  chunks = n > 0 runs each stage
 * as n chunks of (block, tile) items: a face kernel (reconstruction, Riemann
 * fluxes, flux divergence and sources, compiled without the inversion code)
 * stores the stage right-hand side in a buffer of one value per (block,
 * variable, interior cell) in the form's flux type (FP32 for the mixed form,
 * FP64 otherwise); a cell kernel on a second stream then applies the RK
 * combination, inversion, floors and CFL rate of that chunk, overlapping the
 * next chunk's face kernel.  Same arithmetic as the fused kernel, so results
 * are identical bit for bit.  Source: the per-cell update of Sec. 2 (flux
 * divergence, sources, two-stage RK and inversion), reorganised into two
 * kernels.  First use allocates the second stream, its events and the
 * buffer (BHAC_ERR_NOMEM if the device has no room).  BHAC_ERR_ARG: chunks
 * outside [0, 32], or chunks > 0 with constrained transport or a
 * warp-specialised launch shape.  Not for graph capture (bhac_graph_capture
 * returns BHAC_ERR_STATE while chunks > 0). */
bhac_status bhac_set_split(bhac_ctx* ctx, int chunks);

/* Z parts of the stage kernel's work items (3-D grids, the phased kernel):
 * parts = p > 0 splits each (block, tile) column of cells into p runs of
 * nz/p planes, each a work item of its own (every part recomputes the z faces
 * at its bottom, the same numbers as the face carried up from below, so the
 * results do not depend on p); parts = 0 (the default) lets the library
 * choose: whole columns unless splitting fills the GPU's resident CTA slots
 * markedly better (grids with few columns).  Source: the per-block update of
 * Sec. 2; the paper's blocks are the work units, this only cuts them finer.
 * BHAC_ERR_ARG: parts < 0, or parts > 0 on a 2-D grid or not dividing nz.
 * bhac_zsplit_in_force returns the parts the last stage used (0 before any
 * stage since the last launch-shape change; always 1 on 2-D grids, with the
 * split form and with the warp-specialised kernel). */
bhac_status bhac_set_zsplit(bhac_ctx* ctx, int parts);
int bhac_zsplit_in_force(const bhac_ctx* ctx);

/* Records `nsteps` steps with the device time step (bhac_step(ctx, 0.0)) into a
 * CUDA graph on the context's stream and instantiates it; bhac_graph_launch()
 * then replays all of them with one launch.  The stream must be a created
 * (non-legacy-default) stream; the CFL must have been evaluated (bhac_cfl_dt or
 * a previous step).  Buffer roles return to their starting state after every
 * step, so replays continue the evolution.  Capturing again replaces the graph. */
bhac_status bhac_graph_capture(bhac_ctx* ctx, int nsteps);
bhac_status bhac_graph_launch(bhac_ctx* ctx);

/* Measurement utility for the roofline (the paper has no counterpart): counts
 * the floating-point operations one zone-stage costs with the library's own
 * formulas (reconstruction, Riemann solve, sources, RK combination, inversion
 * and, averaged over the two stages, the CFL rate), by running them on the
 * host with a counting scalar over `nsamples` interior cells of the current
 * state drawn with `seed` (their Newton iteration counts are the real ones;
 * the stage is taken of size dt > 0).  Convention: + - * / sqrt 1/sqrt = 1 flop,
 * a fused multiply-add = 2, compares/min/max/selects = 0.  out[0], out[1]:
 * FP64 and FP32 flops per zone-stage; out[2], out[3]: of which divisions and
 * (reciprocal) square roots; out[4]: samples; out[5]: blocks sampled.  Fills
 * the ghost cells of the current state and synchronises the stream. */
bhac_status bhac_count_flops(bhac_ctx* ctx, double dt, int nsamples, unsigned seed, double out[6]);

/* Self-check utility (the paper has no counterpart).  The stage kernels
 * replace FP64 compares and FP32<->FP64 conversions by integer bit operations
 * (GB300 runs those FP64-unit instructions at the cost of an FP64 FMA), and
 * FP64 reciprocals and square roots by an FP32 hardware seed refined with
 * fused multiply-adds.  This runs each replacement beside the hardware or IEEE
 * operation on `n` operand pairs generated on the device from `seed` (random
 * bit patterns; doubles in and around the float range; round-to-nearest ties;
 * neighbours one ulp apart; zeros, subnormals, infinities, NaNs) and writes the
 * number of disagreements per operation to out[11]: [0] a < b, [1] x > 0,
 * [2] x <= 0, [3] |a| < |b|, [4] a <= b and x < 0 (all IEEE, NaN operands
 * included), [5] isfinite, [6] double -> float (bitwise; NaN as NaN),
 * [7] float -> double; and the operands whose result lies farther than the
 * bound from the reference: [8] 1/x more than 1 ulp from the IEEE reciprocal,
 * [9] x^(-1/2) more than 2 ulp from CUDA's rsqrt, [10] sqrt x more than 2 ulp
 * from the IEEE square root (special values must match exactly).
 * n in [1, 1<<26].  Synchronous (default stream); the counters are a
 * file-scope device array, so concurrent calls race on them. */
bhac_status bhac_check_bit_ops(long long n, unsigned seed, long long out[11]);

/* Self-check utility of the host-built constrained-transport maps (no device
 * work; the paper has no counterpart): for a constrained-transport descriptor
 * and its leaves, applies the ring-face maps bhac_init_grid would build to
 * `owned` (host, every block's owned faces in the bhac_set_faces layout) and
 * writes every block's ring-extended face arrays to `ring` (host): per block,
 * per active d, extents nx_e + 2 across active directions (local index -1 at
 * position 0) and nx_d + 1 along d, i fastest; zero where nothing maps.
 * BHAC_ERR_ARG for an invalid descriptor or a grid the maps reject. */
bhac_status bhac_ct_ring_faces_host(const bhac_grid_desc* desc, const bhac_block_desc* blocks, int nblocks,
                                    const double* owned, double* ring);

/* Measurement utility for the roofline (the paper has no counterpart): the
 * arithmetic throughput of the current device, each figure from one kernel that
 * keeps 8 CTAs of 256 threads per SM busy with 8 independent chains per
 * thread, timed with CUDA events on `cuda_stream` after one warm-up launch.
 * out[0] FP64 flops/s of fused multiply-adds (2 flops each), out[1] the same for
 * FP32, out[2] FP64 IEEE divisions/s, out[3] FP64 IEEE square roots/s,
 * out[4] FP64 reciprocal square roots/s, out[5] SM count, out[6] CTAs,
 * out[7] threads per CTA.  `iters` (1 .. 2^20) sets the FP64 chain length
 * (FP32: 16x; the special functions: 1/8).  Synchronises the stream; writes
 * only a file-scope device word, never in practice. */
bhac_status bhac_measure_peaks(int iters, void* cuda_stream, double out[8]);

/* Allocation-free CFL time step, for callers that cannot allocate device memory
 * (no counterpart in the paper: it exists only because of how some callers run).
 * Such callers include hosts whose device memory is entirely owned by another
 * allocator and that therefore hand this library no arena, and per-step
 * diagnostics that must never enter an allocator because cudaMalloc can
 * synchronise the device and stall the streams that the step keeps busy.
 *
 * Computes dt = cfl / max over interior cells of sum_d c_d / dx_d (the same
 * rate as bhac_cfl_dt) for the FP64 interior primitives `prims` (device pointer,
 * [block][var][k][j][i] as in bhac_set_prims) of the leaf blocks `blocks`, and
 * writes it to the device word `dt`; no context, no arena.  The scratch (a copy
 * of the block table and one partial maximum per block) is a pair of file-scope
 * device arrays of this library sized for BHAC_STATIC_MAX_BLOCKS blocks (24 bytes
 * each, 384 KiB in all), held by every GPU that loads the library until the
 * process exits.  More blocks than that: BHAC_ERR_ARG, nothing launched.
 *
 * The first call on a device looks up the arrays' device addresses
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call reuses the same arrays and leaves its
 * contents there; each call writes every partial it reads, so nothing has to be
 * cleared between calls.  Calls whose kernels overlap on the GPU (other streams,
 * other threads) race on the arrays: serialise them.  Asynchronous on `stream`.
 * The block table `blocks` is copied to the device on `stream`: from pageable
 * host memory that copy is complete when the call returns, but from page-locked
 * memory it is asynchronous, so such a table must stay unchanged until the
 * stream has reached the call (e.g. until the stream is synchronised). */
#define BHAC_STATIC_MAX_BLOCKS 16384
bhac_status bhac_cfl_dt_static(const bhac_grid_desc* desc, const bhac_block_desc* blocks, int nblocks,
                               const double* prims, double* dt, void* cuda_stream);

/* Releases the context (host memory only; the arena stays the caller's). */
void bhac_destroy(bhac_ctx* ctx);

const char* bhac_status_string(bhac_status status);

#ifdef __cplusplus
}
#endif
#endif
