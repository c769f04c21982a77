// The C ABI (include/bhac_gb300.h): context, arena carving, ghost maps, and the
// launch sequence of a step.  No device memory is allocated here: every
// device array is a slice of the caller's arena.
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ctx.h"

using namespace bhac;

namespace {
// NVTX range around an ABI call, so profilers (ncu --nvtx, nsys) can group
// its kernels; a no-op when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace


namespace {

struct Layout {
  size_t off_blk, off_order, off_src, off_flags, off_tmpl, off_tc, off_tf1, off_tf2, off_tc32, off_tf1_32, off_tf2_32;
  size_t off_P[2], off_P32[2], off_U[2], off_scratch, off_scratch_out, off_status, off_small;
  size_t off_nodes, off_ops, off_nodeval, off_cf, off_regoff, off_reg, off_rcells, off_rterms;
  size_t off_phi[2], off_xf, off_te_c, off_te_f1, off_te_f2, off_te_c32, off_te_f1_32, off_te_f2_32, off_ring[2];
  size_t off_ringm[2], off_emf, off_xr[3], off_ef[2];
  size_t total;
  long long toff_c[MAXLEV], toff_f1[MAXLEV], toff_f2[MAXLEV];
  long long teo_c[MAXLEV], teo_f1[MAXLEV], teo_f2[MAXLEV];
};

// The constrained-transport maps of a grid: the ring-face copies (every grid)
// and, with refinement levels, the means and the coarse-fine corrections.
struct CtMaps {
  std::vector<long long> ring_dst, ring_src;
  CtLevelMaps lv;
  bool ok;
};

CtMaps build_ct_maps(const bhac_grid_desc* d, const bhac_block_desc* b, int nb) {
  CtMaps m;
  m.ok = true;
  m.lv.ok = true;
  if (d->divb != BHAC_DIVB_CT) return m;
  if (d->nlevels == 1) {
    m.ok = ct_ring_map(d, b, nb, ct_geom(d), m.ring_dst, m.ring_src);
  } else {
    m.lv = ct_level_maps(d, b, nb, ct_geom(d));
    m.ok = m.lv.ok;
    m.ring_dst.swap(m.lv.copy_dst);
    m.ring_src.swap(m.lv.copy_src);
  }
  return m;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool valid_desc(const bhac_grid_desc* d, const bhac_block_desc* b, int nb) {
  if (!d || !b || nb <= 0) return false;
  if (d->ndim < 2 || d->ndim > 3 || d->nghost != 3) return false;
  for (int k = 0; k < 3; ++k) {
    if (d->nx[k] < 1 || d->nroot[k] < 1) return false;
    if (k >= d->ndim && d->nx[k] != 1) return false;
    if (k < d->ndim && d->nx[k] < 3) return false;
    for (int s = 0; s < 2; ++s)
      if (d->bc[k][s] < 0 || d->bc[k][s] > 3) return false;
    if (!(d->xmax[k] > d->xmin[k])) return false;
  }
  if (d->nlevels < 1 || d->nlevels > MAXLEV) return false;
  if (d->coords < 0 || d->coords > 2) return false;
  if (d->precision < 0 || d->precision > 1) return false;
  if (d->recon < 0 || d->recon > 1 || d->riemann < 0 || d->riemann > 1) return false;
  if (!(d->gamma_ad > 1.0) || !(d->cfl > 0.0) || !(d->ch > 0.0) || d->c2p_maxit < 1) return false;
  if (!(d->w_max > 1.0)) return false;
  if (d->divb < 0 || d->divb > 1) return false;
  // the face and edge kernels' 32-bit indices: blocks x ring-extended faces
  // and blocks x edges < 2^31
  if (d->divb == BHAC_DIVB_CT && ((long long)nb * ct_geom(d).nfb >= (1LL << 31) ||
                                  (long long)nb * ct_geom(d).nEb >= (1LL << 31)))
    return false;
  if (d->imex < 0 || d->imex > 1) return false;
  if (d->c2p_solver != BHAC_C2P_NEWTON && d->c2p_solver != BHAC_C2P_NK) return false;
  // the axis rule is for x2 (theta) only; phi must be periodic with an even cell count in 3-D
  for (int k = 0; k < 3; ++k)
    for (int s = 0; s < 2; ++s)
      if (d->bc[k][s] == BHAC_BC_AXIS && k != 1) return false;
  if ((d->bc[1][0] == BHAC_BC_AXIS || d->bc[1][1] == BHAC_BC_AXIS) && d->ndim == 3 &&
      (d->bc[2][0] != BHAC_BC_PERIODIC || (d->nroot[2] * d->nx[2]) % 2))
    return false;
  for (int i = 0; i < nb; ++i) {
    if (b[i].level < 0 || b[i].level >= d->nlevels) return false;
    const int c[3] = {b[i].ix, b[i].iy, b[i].iz};
    for (int k = 0; k < 3; ++k)
      if (c[k] < 0 || c[k] >= (d->nroot[k] << (k < d->ndim ? b[i].level : 0))) return false;
  }
  // cell indices must fit the 32-bit ghost map
  long long nc = 1;
  for (int k = 0; k < 3; ++k) nc *= d->nx[k] + (k < d->ndim ? 6 : 0);
  if (nc * nb >= (1LL << 31)) return false;
  return true;
}

void geometry(const bhac_grid_desc* d, int g[3], int N[3], int& ncell, int& nint, int& nslots) {
  ncell = 1;
  nint = 1;
  for (int k = 0; k < 3; ++k) {
    g[k] = k < d->ndim ? d->nghost : 0;
    N[k] = d->nx[k] + 2 * g[k];
    ncell *= N[k];
    nint *= d->nx[k];
  }
  nslots = ncell - nint;
}

Layout layout(const bhac_grid_desc* d, int nb, const HostMaps& M, const CtMaps& C) {
  int g[3], N[3], ncell, nint, nslots;
  geometry(d, g, N, ncell, nint, nslots);
  const bool flat = d->coords == BHAC_COORDS_CART;
  const bool mixed = d->precision == BHAC_PREC_MIXED;
  Layout L;
  long long nc = 0, nf1 = 0, nf2 = 0;
  for (int l = 0; l < MAXLEV; ++l) {
    L.toff_c[l] = nc;
    L.toff_f1[l] = nf1;
    L.toff_f2[l] = nf2;
    if (l < d->nlevels && !flat) {
      const long long N1 = (long long)d->nroot[0] * d->nx[0] << l, N2 = (long long)d->nroot[1] * d->nx[1] << l;
      nc += N1 * N2;
      nf1 += (N1 + 1) * N2;
      nf2 += N1 * (N2 + 1);
    }
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.off_blk = take(sizeof(int) * 4 * nb);
  L.off_order = take(sizeof(int) * nb);
  L.off_src = take(sizeof(int) * (size_t)nb * nslots);
  L.off_flags = take((size_t)nb * nslots);
  L.off_tmpl = take(sizeof(int) * (size_t)nslots);
  L.off_tc = take(sizeof(double) * CREC * nc);
  L.off_tf1 = take(sizeof(double) * FREC * nf1);
  L.off_tf2 = take(sizeof(double) * FREC * nf2);
  L.off_tc32 = take(sizeof(float) * CREC * nc);
  L.off_tf1_32 = take(sizeof(float) * FREC * nf1);
  L.off_tf2_32 = take(sizeof(float) * FREC * nf2);
  for (int s = 0; s < 2; ++s) L.off_P[s] = take(sizeof(double) * NV * (size_t)nb * ncell);
  for (int s = 0; s < 2; ++s) L.off_P32[s] = take(mixed ? sizeof(float) * NV * (size_t)nb * ncell : 0);
  for (int s = 0; s < 2; ++s) L.off_U[s] = take(sizeof(double) * NV * (size_t)nb * nint);
  L.off_scratch = take(sizeof(double) * NV * (size_t)nb * nint);
  L.off_scratch_out = take(sizeof(double) * NV * (size_t)nb * nint);
  L.off_status = take((size_t)nb * nint);
  L.off_small = take(256);
  L.off_nodes = take(sizeof(GhostNode) * M.nodes.size());
  L.off_ops = take(sizeof(long long) * M.ops.size());
  L.off_nodeval = take((mixed ? sizeof(float) : sizeof(double)) * NV * M.nodes.size());
  L.off_cf = take((size_t)nb);
  L.off_regoff = take(sizeof(long long) * 6 * (size_t)nb);
  L.off_reg = take(sizeof(double) * (size_t)M.reg_elems);
  L.off_rcells = take(sizeof(RefluxCell) * M.rcells.size());
  L.off_rterms = take(sizeof(RefluxTerm) * M.rterms.size());
  // constrained transport: face fields, fluxes, extended metric tables, ring map
  const bool ct = d->divb == BHAC_DIVB_CT;
  const CtGeom cg = ct_geom(d);
  const size_t nfaces = ct ? (size_t)nb * cg.nfb : 0;
  for (int s = 0; s < 2; ++s) L.off_phi[s] = take(sizeof(double) * nfaces);
  L.off_xf = take(sizeof(double) * NV * nfaces);
  size_t ec = 0, ef1 = 0, ef2 = 0;
  for (int l = 0; l < MAXLEV; ++l) {
    L.teo_c[l] = (long long)ec;
    L.teo_f1[l] = (long long)ef1;
    L.teo_f2[l] = (long long)ef2;
    if (ct && !flat && l < d->nlevels) {
      const size_t n1 = ((size_t)d->nroot[0] * d->nx[0]) << l, n2 = ((size_t)d->nroot[1] * d->nx[1]) << l;
      ec += (n1 + 2) * (n2 + 2);
      ef1 += (n1 + 3) * (n2 + 2);
      ef2 += (n1 + 2) * (n2 + 3);
    }
  }
  L.off_te_c = take(sizeof(double) * CREC * ec);
  L.off_te_f1 = take(sizeof(double) * FREC * ef1);
  L.off_te_f2 = take(sizeof(double) * FREC * ef2);
  L.off_te_c32 = take(sizeof(float) * CREC * ec);
  L.off_te_f1_32 = take(sizeof(float) * FREC * ef1);
  L.off_te_f2_32 = take(sizeof(float) * FREC * ef2);
  for (int s = 0; s < 2; ++s) L.off_ring[s] = take(sizeof(long long) * C.ring_dst.size());
  L.off_ringm[0] = take(sizeof(long long) * C.lv.mean_dst.size());
  L.off_ringm[1] = take(sizeof(long long) * C.lv.mean_src.size());
  const bool levels = ct && d->nlevels > 1;
  L.off_emf = take(sizeof(double) * (levels ? (size_t)nb * cg.nEb : 0));
  L.off_xr[0] = take(sizeof(long long) * C.lv.xr_dst.size());
  L.off_xr[1] = take(sizeof(long long) * C.lv.xr_src.size());
  L.off_xr[2] = take(sizeof(int) * C.lv.xr_d.size());
  L.off_ef[0] = take(sizeof(long long) * C.lv.ef_dst.size());
  L.off_ef[1] = take(sizeof(long long) * C.lv.ef_src.size());
  L.total = o;
  return L;
}

bhac_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BHAC_OK : BHAC_ERR_CUDA; }

}  // namespace

StageArgs base_args(const bhac_ctx* c) {
  StageArgs a;
  memset(&a, 0, sizeof(a));
  const bhac_grid_desc& d = c->d;
  a.ndim = d.ndim;
  a.nx = d.nx[0];
  a.ny = d.nx[1];
  a.nz = d.nx[2];
  a.gx = c->g[0];
  a.gy = c->g[1];
  a.gz = c->g[2];
  a.Nx = c->N[0];
  a.Ny = c->N[1];
  a.Nz = c->N[2];
  a.ncell = c->ncell;
  a.nint = c->nint;
  a.tx = c->tx;
  a.ty = c->ty;
  a.ntx = d.nx[0] / c->tx;
  a.nty = d.nx[1] / c->ty;
  a.nblocks = c->nb;
  a.nitems = c->nb * a.ntx * a.nty;
  a.nzp = 1;
  a.item0 = 0;
  a.item1 = a.nitems;
  a.split = 0;
  a.R = c->Rbuf;
  a.persistent = c->persistent;
  a.minb = c->minb;
  a.pwarps = c->pwarps;
  a.blk = c->d_blk;
  a.order = c->d_order;
  for (int k = 0; k < 3; ++k) {
    a.dxl0[k] = (d.xmax[k] - d.xmin[k]) / ((double)d.nroot[k] * d.nx[k]);
    a.idx[k] = 1.0 / a.dxl0[k];
  }
  a.N1g = c->N1g;
  a.N2g = c->N2g;
  a.axis_lo1 = d.bc[1][0] == BHAC_BC_AXIS;
  a.axis_hi1 = d.bc[1][1] == BHAC_BC_AXIS;
  a.flat = c->flat;
  a.recon = d.recon;
  a.riemann = d.riemann;
  a.gam = d.gamma_ad;
  a.gam_fac = d.gamma_ad / (d.gamma_ad - 1.0);
  // constrained transport does not evolve psi: no cleaning speed, no damping
  a.ch = c->ct ? 0.0 : d.ch;
  a.kappa = c->ct ? 0.0 : d.kappa;
  a.gam_f = (float)a.gam;
  a.gam_fac_f = (float)a.gam_fac;
  a.ch_f = (float)a.ch;
  a.kappa_f = (float)a.kappa;
  a.ch2_f = (float)(a.ch * a.ch);
  a.cfl = d.cfl;
  a.c2p_tol = d.c2p_tol;
  a.c2p_maxit = d.c2p_maxit;
  a.wmax = d.w_max;
  a.imex = d.imex && !c->ct;
  a.c2p_nk = d.c2p_solver == BHAC_C2P_NK;
  a.imex_g = 1.0 - 1.0 / sqrt(2.0);
  a.c2p_gf = (d.gamma_ad - 1.0) / d.gamma_ad;
  a.c2p_v2max = 1.0 - 1.0 / (d.w_max * d.w_max);
  a.rho_fl_c = d.rho_floor;
  a.p_fl_c = d.p_floor;
  a.tab_c = c->tab_c;
  a.tab_f1 = c->tab_f1;
  a.tab_f2 = c->tab_f2;
  a.tab_c32 = c->tab_c32;
  a.tab_f1_32 = c->tab_f1_32;
  a.tab_f2_32 = c->tab_f2_32;
  a.dt_dev = c->dt_dev;
  a.smax_in = c->smax;
  a.smax_out = c->smax;
  a.counts = c->counts;
  a.status = c->d_status;
  a.work = c->work;
  a.nlev = c->d.nlevels;
  for (int l = 0; l < MAXLEV; ++l) {
    a.toff_c[l] = c->toff_c[l];
    a.toff_f1[l] = c->toff_f1[l];
    a.toff_f2[l] = c->toff_f2[l];
    a.N1l[l] = c->N1g << l;
    a.N2l[l] = c->N2g << l;
  }
  a.cf = c->d_cf;
  a.regoff = c->d_regoff;
  a.reg = c->d_reg;
  a.rcells = c->d_rcells;
  a.rterms = c->d_rterms;
  a.nrcells = c->nrcells;
  return a;
}

// Shared memory of the stage kernel: face fluxes of one plane (x, y and two
// z-face planes), or in the warp-specialised form two planes of x and y faces
// and three z-face planes.
size_t stage_smem(const bhac_ctx* c, int tx, int ty, int pwarps) {
  const size_t tsz = c->mixed ? sizeof(float) : sizeof(double);
  const size_t sFx = (size_t)ty * (tx + 1), sFy = (size_t)(ty + 1) * tx, sFz = (size_t)tx * ty;
  if (c->d.ndim == 3 && pwarps > 0) return NV * (2 * sFx + 2 * sFy + 3 * sFz) * tsz;
  // phased form: face fluxes, edges along x and y (tile plus halo), and in
  // 3-D two z-face planes and the carried z edges
  const size_t nex = (size_t)(tx + 2) * ty, ney = (size_t)tx * (ty + 2);
  size_t n = sFx + sFy + 2 * nex + 2 * ney;
  if (c->d.ndim == 3) n += 3 * sFz;
  return NV * n * tsz;
}

bhac_status ghost_fill(bhac_ctx* c, int buf, bool zero_smax) {
  for (size_t dep = 1; dep < c->depth_start.size(); ++dep) {
    NodeArgs n;
    n.nodes = c->d_nodes;
    n.ops = c->d_ops;
    n.first = c->depth_start[dep - 1];
    n.count = c->depth_start[dep] - c->depth_start[dep - 1];
    n.nnodes = c->nnodes;
    n.ncell = c->ncell;
    n.P = c->mixed ? nullptr : c->P[buf];
    n.P32 = c->mixed ? c->P32[buf] : nullptr;
    n.out = c->d_node64;
    n.out32 = c->d_node32;
    if (launch_ghost_nodes(n, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  }
  GhostArgs g;
  g.node64 = c->d_node64;
  g.node32 = c->d_node32;
  g.src = c->d_src;
  g.flags = c->d_flags;
  g.tmpl = c->d_tmpl;
  g.nslots = c->nslots;
  g.nblocks = c->nb;
  g.ncell = c->ncell;
  g.P = c->mixed ? nullptr : c->P[buf];
  g.P32 = c->mixed ? c->P32[buf] : nullptr;
  g.work_reset = c->work;
  g.smax_reset = zero_smax ? c->smax : nullptr;
  return cuda_status(launch_ghost_fill(g, c->st));
}

namespace {

// Z parts per (block, tile) column of the phased 3-D stage kernel.  A fixed
// choice (bhac_set_zsplit) is used as given.  Otherwise: among the parts that
// divide nz and leave at least 4 planes, the one that minimises the modelled
// time, rounds of items over the resident CTA slots times the planes of an
// item plus a quarter plane for the z faces it recomputes at its bottom.
// Whole columns are kept unless splitting fills the GPU's slots markedly
// better (small grids: 432 columns of 16^3 on 152 SMs).
int choose_nzp(const bhac_ctx* c, const StageArgs& a, size_t smem) {
  const int nz = c->d.nx[2];
  if (c->zsplit > 0) return c->zsplit;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = c->persistent ? c->persistent
                                   : (c->mixed ? stage_occupancy_mixed(a, c->threads, smem)
                                               : stage_occupancy_fp64(a, c->threads, smem));
  const long long slots = (long long)(nsm > 0 ? nsm : 1) * (per_sm > 0 ? per_sm : 1);
  const long long items = (long long)a.nitems;
  int best = 1;
  const double cost1 = (double)((items + slots - 1) / slots) * ((double)nz + 0.25);
  double best_cost = cost1;
  for (int p = 2; p <= nz; p *= 2) {
    if (nz % p || nz / p < 4) break;
    const long long n = items * p;
    const double cost = (double)((n + slots - 1) / slots) * ((double)(nz / p) + 0.25);
    if (cost < 0.95 * cost1 && cost < best_cost) {
      best = p;
      best_cost = cost;
    }
  }
  return best;
}

bhac_status run_stage(bhac_ctx* c, int stage, double dt) {
  StageArgs a = base_args(c);
  const int in = c->cur, out = 1 - c->cur;
  a.stage = stage;
  a.dt_host = dt;
  a.P_in = c->P[in];
  a.P_out = c->P[out];
  a.P32_in = c->P32[in];
  a.P32_out = c->P32[out];
  if (stage == 1) {
    a.Un = c->U[c->ucur];
    a.U1 = nullptr;
    a.Uout = c->U[1 - c->ucur];
  } else {
    a.Un = c->U[1 - c->ucur];  // conserved at the start of the step
    a.U1 = c->U[c->ucur];      // after stage 1
    a.Uout = c->U[1 - c->ucur];
  }
  const size_t smem = stage_smem(c, c->tx, c->ty, c->pwarps);
  if (c->split <= 0 && c->pwarps == 0 && c->d.ndim == 3) {
    // the phased kernel's items may be z parts of (block, tile) columns
    if (c->nzp_eff <= 0) c->nzp_eff = choose_nzp(c, a, smem);
    a.nzp = c->nzp_eff;
    a.nitems *= a.nzp;
    a.item1 = a.nitems;
  } else {
    c->nzp_eff = 1;  // whole columns (2-D grids, the split form, the warp-specialised kernel)
  }
  int grid = a.nitems;
  if (c->persistent) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    grid = nsm * c->persistent;
  }
  cudaError_t e = cudaSuccess;
  if (c->split <= 0) {
    e = c->mixed ? launch_stage_mixed(a, grid, c->threads, smem, c->st)
                 : launch_stage_fp64(a, grid, c->threads, smem, c->st);
  } else {
    // split form: chunk q's face kernel on st, its cell kernel on st2 after it;
    // the face kernel of chunk q + 1 overlaps the cell kernel of chunk q
    const int nch = c->split;
    a.split = 1;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaMemsetAsync(c->work, 0, sizeof(unsigned int) * 32, c->st);  // one counter per chunk
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, c->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st2, c->ev_fork, 0);
    for (int q = 0; q < nch && e == cudaSuccess; ++q) {
      StageArgs f = a;
      f.item0 = (int)((long long)a.nitems * q / nch);
      f.item1 = (int)((long long)a.nitems * (q + 1) / nch);
      f.work = c->work + q;
      const int g = c->persistent ? grid : f.item1 - f.item0;
      e = c->mixed ? launch_stage_mixed(f, g, c->threads, smem, c->st) : launch_stage_fp64(f, g, c->threads, smem, c->st);
      if (e == cudaSuccess) e = cudaEventRecord(c->ev_chunk[q], c->st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st2, c->ev_chunk[q], 0);
      const long long cells = (long long)(f.item1 - f.item0) * c->tx * c->ty * c->d.nx[2];
      long long cg = (cells + 255) / 256;
      if (cg > 8LL * nsm) cg = 8LL * nsm;
      if (e == cudaSuccess)
        e = c->mixed ? launch_cells_mixed(f, (int)(cg < 1 ? 1 : cg), c->st2) : launch_cells_fp64(f, (int)(cg < 1 ? 1 : cg), c->st2);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join2, c->st2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, c->ev_join2, 0);
    if (e == cudaSuccess) e = c->mixed ? launch_reflux_mixed(a, c->st) : launch_reflux_fp64(a, c->st);
  }
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  c->cur = out;
  c->ucur = 1 - c->ucur;
  return BHAC_OK;
}

// Arguments of the constrained-transport kernels for the current buffers.
CtArgs ct_args(const bhac_ctx* c) {
  CtArgs t;
  t.g = c->ctg;
  t.phi_in = c->phi[c->pcur];
  t.phi_out = c->phi[1 - c->pcur];
  t.phi_n = c->phi[1 - c->pcur];
  t.xf = c->xf;
  t.te_c = c->te_c;
  t.te_f1 = c->te_f1;
  t.te_f2 = c->te_f2;
  t.te_c32 = c->te_c32;
  t.te_f1_32 = c->te_f1_32;
  t.te_f2_32 = c->te_f2_32;
  for (int l = 0; l < MAXLEV; ++l) {
    t.teo_c[l] = c->teo_c[l];
    t.teo_f1[l] = c->teo_f1[l];
    t.teo_f2[l] = c->teo_f2[l];
  }
  t.axis_lo = c->d.bc[1][0] == BHAC_BC_AXIS;
  t.axis_hi = c->d.bc[1][1] == BHAC_BC_AXIS;
  t.amr = c->d.nlevels > 1;
  t.emf = c->emf;
  t.xr_dst = c->xr_dst;
  t.xr_src = c->xr_src;
  t.xr_d = c->xr_d;
  t.nxr = c->nxr;
  t.ef_dst = c->ef_dst;
  t.ef_src = c->ef_src;
  t.nef = c->nef;
  return t;
}

// One constrained-transport stage after the ghost fill: ring faces, face
// fluxes, face update, cells.  Face buffers: stage 1 reads the step's start
// (pcur) and writes the other; stage 2 reads that one and writes the start
// buffer (Phi = Phi_n / 2 + (Phi_1 + dt R) / 2 in place), so the roles are
// back where they were after every step.
bhac_status run_stage_ct(bhac_ctx* c, int stage, double dt) {
  StageArgs a = base_args(c);
  const int in = c->cur, out = 1 - c->cur;
  a.stage = stage;
  a.dt_host = dt;
  a.P_in = c->P[in];
  a.P_out = c->P[out];
  a.P32_in = c->P32[in];
  a.P32_out = c->P32[out];
  if (stage == 1) {
    a.Un = c->U[c->ucur];
    a.U1 = nullptr;
    a.Uout = c->U[1 - c->ucur];
  } else {
    a.Un = c->U[1 - c->ucur];
    a.U1 = c->U[c->ucur];
    a.Uout = c->U[1 - c->ucur];
  }
  CtArgs t = ct_args(c);
  if (launch_ct_ring(c->ring_dst, c->ring_src, c->nring, c->phi[c->pcur], c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  if (launch_ct_ring_mean(c->ringm_dst, c->ringm_src, c->nringm, c->phi[c->pcur], c->st) != cudaSuccess)
    return BHAC_ERR_CUDA;
  if (launch_ct_stage(a, t, c->mixed, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  c->cur = out;
  c->ucur = 1 - c->ucur;
  c->pcur = 1 - c->pcur;
  return BHAC_OK;
}

}  // namespace

extern "C" {

const char* bhac_status_string(bhac_status s) {
  switch (s) {
    case BHAC_OK: return "ok";
    case BHAC_ERR_ARG: return "invalid argument";
    case BHAC_ERR_CUDA: return "CUDA error";
    case BHAC_ERR_NOMEM: return "arena too small or device allocation failed";
    case BHAC_ERR_STATE: return "call out of order";
    case BHAC_ERR_TIMEOUT: return "device wait timed out";
    case BHAC_WARN_C2P: return "inversion failures";
  }
  return "unknown status";
}

bhac_status bhac_query_sizes(const bhac_grid_desc* d, const bhac_block_desc* b, int nb, size_t* out) {
  if (!out || !valid_desc(d, b, nb)) return BHAC_ERR_ARG;
  int g[3], N[3], ncell, nint, nslots;
  geometry(d, g, N, ncell, nint, nslots);
  const HostMaps M = build_maps(d, b, nb, g, N, ncell);
  if (!M.ok) return BHAC_ERR_ARG;
  const CtMaps C = build_ct_maps(d, b, nb);
  if (!C.ok) return BHAC_ERR_ARG;
  *out = layout(d, nb, M, C).total;
  return BHAC_OK;
}

bhac_status bhac_init_grid(bhac_ctx** out, const bhac_grid_desc* d, const bhac_block_desc* b, int nb,
                           void* arena, size_t arena_bytes, void* stream) {
  if (!out || !valid_desc(d, b, nb) || !arena || ((uintptr_t)arena & 255)) return BHAC_ERR_ARG;
  int g[3], N[3], ncell, nint, nslots;
  geometry(d, g, N, ncell, nint, nslots);
  const HostMaps M = build_maps(d, b, nb, g, N, ncell);
  if (!M.ok) return BHAC_ERR_ARG;  // a boundary rule or a level points at a missing block
  const CtMaps C = build_ct_maps(d, b, nb);
  if (!C.ok) return BHAC_ERR_ARG;  // a ring face or a correction points at a missing block
  const Layout L = layout(d, nb, M, C);
  if (arena_bytes < L.total) return BHAC_ERR_NOMEM;
  bhac_ctx* c = new bhac_ctx();
  c->d = *d;
  c->nb = nb;
  c->st = (cudaStream_t)stream;
  geometry(d, c->g, c->N, c->ncell, c->nint, c->nslots);
  c->N1g = d->nroot[0] * d->nx[0];
  c->N2g = d->nroot[1] * d->nx[1];
  c->flat = d->coords == BHAC_COORDS_CART;
  c->mixed = d->precision == BHAC_PREC_MIXED;
  c->arena = (char*)arena;
  c->arena_bytes = arena_bytes;
  c->d_blk = (int*)(c->arena + L.off_blk);
  c->d_order = (int*)(c->arena + L.off_order);
  c->d_src = (int*)(c->arena + L.off_src);
  c->d_flags = (unsigned char*)(c->arena + L.off_flags);
  c->d_tmpl = (int*)(c->arena + L.off_tmpl);
  c->tab_c = (double*)(c->arena + L.off_tc);
  c->tab_f1 = (double*)(c->arena + L.off_tf1);
  c->tab_f2 = (double*)(c->arena + L.off_tf2);
  c->tab_c32 = (float*)(c->arena + L.off_tc32);
  c->tab_f1_32 = (float*)(c->arena + L.off_tf1_32);
  c->tab_f2_32 = (float*)(c->arena + L.off_tf2_32);
  for (int l = 0; l < MAXLEV; ++l) {
    c->toff_c[l] = L.toff_c[l];
    c->toff_f1[l] = L.toff_f1[l];
    c->toff_f2[l] = L.toff_f2[l];
  }
  for (int s = 0; s < 2; ++s) {
    c->P[s] = (double*)(c->arena + L.off_P[s]);
    c->P32[s] = c->mixed ? (float*)(c->arena + L.off_P32[s]) : nullptr;
    c->U[s] = (double*)(c->arena + L.off_U[s]);
  }
  c->scratch = (double*)(c->arena + L.off_scratch);
  c->scratch_out = (double*)(c->arena + L.off_scratch_out);
  c->d_status = (unsigned char*)(c->arena + L.off_status);
  c->Rbuf = nullptr;
  c->split = 0;
  c->zsplit = 0;
  c->nzp_eff = 0;
  c->st2 = nullptr;
  c->ev_fork = c->ev_join2 = nullptr;
  for (int q = 0; q < 32; ++q) c->ev_chunk[q] = nullptr;
  char* small = c->arena + L.off_small;
  c->dt_dev = (double*)small;
  c->smax = (unsigned long long*)(small + 8);
  c->counts = (unsigned long long*)(small + 16);
  c->work = (unsigned int*)(small + 48);
  c->nnodes = (int)M.nodes.size();
  c->depth_start = M.depth_start;
  c->d_nodes = (GhostNode*)(c->arena + L.off_nodes);
  c->d_ops = (long long*)(c->arena + L.off_ops);
  c->d_node64 = c->mixed ? nullptr : (double*)(c->arena + L.off_nodeval);
  c->d_node32 = c->mixed ? (float*)(c->arena + L.off_nodeval) : nullptr;
  c->d_cf = (unsigned char*)(c->arena + L.off_cf);
  c->d_regoff = (long long*)(c->arena + L.off_regoff);
  c->d_reg = (double*)(c->arena + L.off_reg);
  c->d_rcells = (RefluxCell*)(c->arena + L.off_rcells);
  c->d_rterms = (RefluxTerm*)(c->arena + L.off_rterms);
  c->nrcells = (int)M.rcells.size();
  c->ct = d->divb == BHAC_DIVB_CT;
  c->faces_ok = false;
  c->ctg = ct_geom(d);
  for (int s = 0; s < 2; ++s) c->phi[s] = (double*)(c->arena + L.off_phi[s]);
  c->pcur = 0;
  c->xf = (double*)(c->arena + L.off_xf);
  c->te_c = (double*)(c->arena + L.off_te_c);
  c->te_f1 = (double*)(c->arena + L.off_te_f1);
  c->te_f2 = (double*)(c->arena + L.off_te_f2);
  c->te_c32 = (float*)(c->arena + L.off_te_c32);
  c->te_f1_32 = (float*)(c->arena + L.off_te_f1_32);
  c->te_f2_32 = (float*)(c->arena + L.off_te_f2_32);
  for (int l = 0; l < MAXLEV; ++l) {
    c->teo_c[l] = L.teo_c[l];
    c->teo_f1[l] = L.teo_f1[l];
    c->teo_f2[l] = L.teo_f2[l];
  }
  c->ring_dst = (long long*)(c->arena + L.off_ring[0]);
  c->ring_src = (long long*)(c->arena + L.off_ring[1]);
  c->nring = (long long)C.ring_dst.size();
  c->ringm_dst = (long long*)(c->arena + L.off_ringm[0]);
  c->ringm_src = (long long*)(c->arena + L.off_ringm[1]);
  c->nringm = (long long)C.lv.mean_dst.size();
  c->emf = (double*)(c->arena + L.off_emf);
  c->xr_dst = (long long*)(c->arena + L.off_xr[0]);
  c->xr_src = (long long*)(c->arena + L.off_xr[1]);
  c->xr_d = (int*)(c->arena + L.off_xr[2]);
  c->nxr = (long long)C.lv.xr_dst.size();
  c->ef_dst = (long long*)(c->arena + L.off_ef[0]);
  c->ef_src = (long long*)(c->arena + L.off_ef[1]);
  c->nef = (long long)C.lv.ef_dst.size();
  c->cur = 0;
  c->ucur = 0;
  c->threads = 256;
  // default launch shape: the largest of these tiles that divides the block
  // and fits the shared-memory limit, else the whole block face.  The 3-D
  // mixed form takes the largest tile of at most 16 x 16 whose workspace lets
  // two CTAs share an SM, with the two-CTA register bound: the fastest shape
  // family on every 3-D grid the autotuner has timed.
  c->minb = 1;
  {
    static const int tiles[][2] = {{32, 16}, {16, 16}, {16, 8}, {8, 8}};
    c->tx = d->nx[0];
    c->ty = d->nx[1];
    const bool two_ctas = d->ndim == 3 && c->mixed;
    for (const auto& t : tiles) {
      if (two_ctas && t[0] * t[1] > 256) continue;
      const size_t limit = two_ctas ? (size_t)kTwoCtaSmem : (size_t)kMaxDynSmem;
      if (d->nx[0] % t[0] == 0 && d->nx[1] % t[1] == 0 && stage_smem(c, t[0], t[1], 0) <= limit) {
        c->tx = t[0];
        c->ty = t[1];
        if (two_ctas) c->minb = 2;
        break;
      }
    }
  }
  c->persistent = 0;
  c->pwarps = 0;
  c->graph = nullptr;
  c->graph_steps = 0;
  c->cp_in = c->cp_out = nullptr;
  c->ev_h2d = c->ev_scat = c->ev_gath = c->ev_d2h = c->ev_fence = c->ev_join_in = c->ev_join_out = nullptr;
  c->blk.resize(4 * nb);
  for (int i = 0; i < nb; ++i) {
    c->blk[4 * i] = b[i].level;
    c->blk[4 * i + 1] = b[i].ix;
    c->blk[4 * i + 2] = b[i].iy;
    c->blk[4 * i + 3] = b[i].iz;
  }
  // visiting order: finest level first, then by x2 and x1 with x3 fastest, so
  // the CTAs in flight share the phi-independent metric records in L2
  std::vector<int> order(nb);
  for (int i = 0; i < nb; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
    const int* x = &c->blk[4 * p];
    const int* y = &c->blk[4 * q];
    if (x[0] != y[0]) return x[0] > y[0];
    if (x[2] != y[2]) return x[2] < y[2];
    if (x[1] != y[1]) return x[1] < y[1];
    return x[3] < y[3];
  });
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->st) : cudaSuccess;
  };
  cudaError_t e = up(c->d_blk, c->blk.data(), sizeof(int) * 4 * nb);
  if (e == cudaSuccess) e = up(c->d_order, order.data(), sizeof(int) * nb);
  if (e == cudaSuccess) e = up(c->d_src, M.src.data(), sizeof(int) * M.src.size());
  if (e == cudaSuccess) e = up(c->d_flags, M.flags.data(), M.flags.size());
  if (e == cudaSuccess) e = up(c->d_tmpl, M.tmpl.data(), sizeof(int) * M.tmpl.size());
  if (e == cudaSuccess) e = up(c->d_nodes, M.nodes.data(), sizeof(GhostNode) * M.nodes.size());
  if (e == cudaSuccess) e = up(c->d_ops, M.ops.data(), sizeof(long long) * M.ops.size());
  if (e == cudaSuccess) e = up(c->d_cf, M.cf.data(), M.cf.size());
  if (e == cudaSuccess) e = up(c->d_regoff, M.regoff.data(), sizeof(long long) * M.regoff.size());
  if (e == cudaSuccess) e = up(c->d_rcells, M.rcells.data(), sizeof(RefluxCell) * M.rcells.size());
  if (e == cudaSuccess) e = up(c->d_rterms, M.rterms.data(), sizeof(RefluxTerm) * M.rterms.size());
  if (e == cudaSuccess) e = up(c->ring_dst, C.ring_dst.data(), sizeof(long long) * C.ring_dst.size());
  if (e == cudaSuccess) e = up(c->ring_src, C.ring_src.data(), sizeof(long long) * C.ring_src.size());
  if (e == cudaSuccess) e = up(c->ringm_dst, C.lv.mean_dst.data(), sizeof(long long) * C.lv.mean_dst.size());
  if (e == cudaSuccess) e = up(c->ringm_src, C.lv.mean_src.data(), sizeof(long long) * C.lv.mean_src.size());
  if (e == cudaSuccess) e = up(c->xr_dst, C.lv.xr_dst.data(), sizeof(long long) * C.lv.xr_dst.size());
  if (e == cudaSuccess) e = up(c->xr_src, C.lv.xr_src.data(), sizeof(long long) * C.lv.xr_src.size());
  if (e == cudaSuccess) e = up(c->xr_d, C.lv.xr_d.data(), sizeof(int) * C.lv.xr_d.size());
  if (e == cudaSuccess) e = up(c->ef_dst, C.lv.ef_dst.data(), sizeof(long long) * C.lv.ef_dst.size());
  if (e == cudaSuccess) e = up(c->ef_src, C.lv.ef_src.data(), sizeof(long long) * C.lv.ef_src.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(small, 0, 256, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // the host maps die here
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&c->ev_h2d, &c->ev_scat, &c->ev_gath, &c->ev_d2h, &c->ev_fence, &c->ev_join_in,
                          &c->ev_join_out})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    bhac_destroy(c);
    return BHAC_ERR_CUDA;
  }
  c->metric_ok = c->flat;
  *out = c;
  return BHAC_OK;
}

bhac_status bhac_set_metric(bhac_ctx* c, int kind, double spin, double mass, const double* mks_params) {
  (void)mks_params;
  if (!c) return BHAC_ERR_ARG;
  if (kind == BHAC_COORDS_CART) {
    if (!c->flat) return BHAC_ERR_ARG;
    c->metric_ok = true;
    return BHAC_OK;
  }
  if (c->flat || kind != c->d.coords) return BHAC_ERR_ARG;
  c->d.spin = spin;
  c->d.mass = mass;
  for (int l = 0; l < c->d.nlevels; ++l) {
    MetricArgs M;
    M.coords = kind;
    M.spin = spin;
    M.mass = mass;
    M.x1min = c->d.xmin[0];
    M.x2min = c->d.xmin[1];
    M.N1 = c->N1g << l;
    M.N2 = c->N2g << l;
    M.dx1 = (c->d.xmax[0] - c->d.xmin[0]) / M.N1;
    M.dx2 = (c->d.xmax[1] - c->d.xmin[1]) / M.N2;
    M.axis_lo = c->d.bc[1][0] == BHAC_BC_AXIS;
    M.axis_hi = c->d.bc[1][1] == BHAC_BC_AXIS;
    M.rho_floor = c->d.rho_floor;
    M.rho_pow = c->d.rho_floor_pow;
    M.p_floor = c->d.p_floor;
    M.p_pow = c->d.p_floor_pow;
    M.tab_c = c->tab_c + c->toff_c[l] * CREC;
    M.tab_f1 = c->tab_f1 + c->toff_f1[l] * FREC;
    M.tab_f2 = c->tab_f2 + c->toff_f2[l] * FREC;
    M.tab_c32 = c->tab_c32 + c->toff_c[l] * CREC;
    M.tab_f1_32 = c->tab_f1_32 + c->toff_f1[l] * FREC;
    M.tab_f2_32 = c->tab_f2_32 + c->toff_f2[l] * FREC;
    if (launch_metric_tables(M, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  }
  for (int l = 0; c->ct && l < c->d.nlevels; ++l) {
    // the same tables of every level on its grid extended by one cell on each
    // side in x1 and x2, for the faces around each block (a face beyond the
    // polar axis sees the mirrored metric, which depends on sin^2 and cos^2 of
    // theta only)
    MetricArgs M;
    M.coords = kind;
    M.spin = spin;
    M.mass = mass;
    M.dx1 = (c->d.xmax[0] - c->d.xmin[0]) / (c->N1g << l);
    M.dx2 = (c->d.xmax[1] - c->d.xmin[1]) / (c->N2g << l);
    M.x1min = c->d.xmin[0] - M.dx1;
    M.x2min = c->d.xmin[1] - M.dx2;
    M.N1 = (c->N1g << l) + 2;
    M.N2 = (c->N2g << l) + 2;
    M.axis_lo = M.axis_hi = 0;
    M.rho_floor = c->d.rho_floor;
    M.rho_pow = c->d.rho_floor_pow;
    M.p_floor = c->d.p_floor;
    M.p_pow = c->d.p_floor_pow;
    M.tab_c = c->te_c + c->teo_c[l] * CREC;
    M.tab_f1 = c->te_f1 + c->teo_f1[l] * FREC;
    M.tab_f2 = c->te_f2 + c->teo_f2[l] * FREC;
    M.tab_c32 = c->te_c32 + c->teo_c[l] * CREC;
    M.tab_f1_32 = c->te_f1_32 + c->teo_f1[l] * FREC;
    M.tab_f2_32 = c->te_f2_32 + c->teo_f2[l] * FREC;
    if (launch_metric_tables(M, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  }
  c->metric_ok = true;
  return BHAC_OK;
}

bhac_status bhac_set_prims(bhac_ctx* c, const double* prims, int on_device) {
  if (!c || !prims) return BHAC_ERR_ARG;
  if (!c->metric_ok) return BHAC_ERR_STATE;
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->nint;
  const double* src = prims;
  if (!on_device) {
    if (cudaMemcpyAsync(c->scratch, prims, bytes, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return BHAC_ERR_CUDA;
    src = c->scratch;
  }
  c->cur = 0;
  c->ucur = 0;
  StageArgs a = base_args(c);
  // one pass: ghosted primitives, conserved state and the CFL rate
  cudaError_t e = cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long), c->st);
  if (e == cudaSuccess) e = launch_load(a, src, c->P[0], c->P32[0], c->U[0], c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, (size_t)c->nb * c->nint, c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  c->prims_ok = true;
  c->cfl_ok = false;
  c->cfl_fresh = true;
  c->faces_ok = false;
  c->pcur = 0;
  return BHAC_OK;
}

bhac_status bhac_set_cons(bhac_ctx* c, const double* cons, int on_device) {
  if (!c || !cons) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->nint;
  cudaError_t e = cudaMemcpyAsync(c->U[c->ucur], cons, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  return cuda_status(e);
}

// Host memory the copy engines can read and write without staging.
static bool page_locked(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

bhac_status bhac_set_prims_host_async(bhac_ctx* c, const double* host_prims) {
  if (!c || !host_prims) return BHAC_ERR_ARG;
  if (!c->metric_ok) return BHAC_ERR_STATE;
  if (!page_locked(host_prims)) return BHAC_ERR_ARG;
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->nint;
  // the copy starts once the previous load has consumed the staging buffer
  cudaError_t e = cudaStreamWaitEvent(c->cp_in, c->ev_scat, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->scratch, host_prims, bytes, cudaMemcpyHostToDevice, c->cp_in);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_h2d, c->cp_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, c->ev_h2d, 0);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  c->cur = 0;
  c->ucur = 0;
  StageArgs a = base_args(c);
  // one pass: ghosted primitives, conserved state and the CFL rate; then the
  // staging buffer is free for the next load
  e = cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long), c->st);
  if (e == cudaSuccess) e = launch_load(a, c->scratch, c->P[0], c->P32[0], c->U[0], c->st);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_scat, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, (size_t)c->nb * c->nint, c->st);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  c->prims_ok = true;
  c->cfl_ok = false;
  c->cfl_fresh = true;
  c->faces_ok = false;
  c->pcur = 0;
  return BHAC_OK;
}

bhac_status bhac_get_prims_host_async(bhac_ctx* c, double* host_prims) {
  if (!c || !host_prims) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  if (!page_locked(host_prims)) return BHAC_ERR_ARG;
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->nint;
  StageArgs a = base_args(c);
  // the gather waits until the previous read-back has drained the staging buffer
  cudaError_t e = cudaStreamWaitEvent(c->st, c->ev_d2h, 0);
  if (e == cudaSuccess) e = launch_gather_interior(a, c->P[c->cur], c->scratch_out, c->st);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_gath, c->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cp_out, c->ev_gath, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_prims, c->scratch_out, bytes, cudaMemcpyDeviceToHost, c->cp_out);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_d2h, c->cp_out);
  return cuda_status(e);
}

bhac_status bhac_host_fence(bhac_ctx* c) {
  if (!c) return BHAC_ERR_ARG;
  cudaError_t e = cudaEventRecord(c->ev_fence, c->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cp_in, c->ev_fence, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->cp_out, c->ev_fence, 0);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join_in, c->cp_in);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join_out, c->cp_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, c->ev_join_in, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, c->ev_join_out, 0);
  return cuda_status(e);
}

bhac_status bhac_fill_ghosts(bhac_ctx* c) {
  NvtxRange range("bhac_fill_ghosts");
  if (!c) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  return ghost_fill(c, c->cur, false);
}

bhac_status bhac_cfl_dt(bhac_ctx* c, double* dt_host) {
  NvtxRange range("bhac_cfl_dt");
  if (!c) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  if (!c->cfl_fresh) {
    // (a load leaves the rate of the loaded primitives in smax already)
    if (cudaMemsetAsync(c->smax, 0, sizeof(unsigned long long), c->st) != cudaSuccess) return BHAC_ERR_CUDA;
    StageArgs a = base_args(c);
    a.P_in = c->P[c->cur];
    if (launch_cfl(a, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
    c->cfl_fresh = true;
  }
  c->cfl_ok = true;
  if (dt_host) {
    unsigned long long bits = 0;
    if (cudaMemcpyAsync(&bits, c->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess)
      return BHAC_ERR_CUDA;
    double smax;
    memcpy(&smax, &bits, sizeof(smax));
    *dt_host = c->d.cfl / smax;
  }
  return BHAC_OK;
}

bhac_status bhac_stage(bhac_ctx* c, int stage, double dt) {
  NvtxRange range(stage == 1 ? "bhac_stage 1" : "bhac_stage 2");
  if (!c || (stage != 1 && stage != 2)) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  if (stage == 1 && !(dt > 0.0) && !c->cfl_ok) return BHAC_ERR_STATE;
  if (c->ct && !c->faces_ok) return BHAC_ERR_STATE;
  c->cfl_fresh = false;  // the stage changes the primitives (stage 2 leaves their rate in smax)
  if (stage == 1 && c->d.imex && !c->ct) {
    // the IMEX first stage: the fluxes of stage 1 see psi of Y1
    StageArgs a = base_args(c);
    a.stage = 1;
    a.dt_host = dt;
    a.P_in = c->P[c->cur];
    a.P32_in = c->P32[c->cur];
    if (launch_imex_first_stage(a, c->P[c->cur], c->P32[c->cur], c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  }
  bhac_status s = ghost_fill(c, c->cur, stage == 2);
  if (s != BHAC_OK) return s;
  s = c->ct ? run_stage_ct(c, stage, dt) : run_stage(c, stage, dt);
  if (s == BHAC_OK && stage == 2) c->cfl_ok = true;
  return s;
}

bhac_status bhac_launches_per_step(const bhac_ctx* c, int* out) {
  if (!c || !out) return BHAC_ERR_ARG;
  int per_fill = 1;  // the ghost gather
  for (size_t dep = 1; dep < c->depth_start.size(); ++dep)
    if (c->depth_start[dep] > c->depth_start[dep - 1]) ++per_fill;  // one cross-level node pass per depth
  // constrained transport: + ring copy, face fluxes, face update, cells; with
  // refinement levels + ring means, flux correction, EMFs, EMF correction
  const int levels = c->ct && c->d.nlevels > 1 ? 1 + (c->nxr > 0) + (c->nef > 0) : 0;
  const int per_stage = c->ct ? per_fill + 4 + (c->nringm > 0) + levels
                              : per_fill + 1 + (c->nrcells > 0 ? 1 : 0);  // + stage kernel (+ reflux)
  *out = 2 * per_stage + (c->d.imex && !c->ct ? 1 : 0);  // + the IMEX first-stage pass
  return BHAC_OK;
}

bhac_status bhac_step(bhac_ctx* c, double dt) {
  bhac_status s = bhac_stage(c, 1, dt);
  if (s != BHAC_OK) return s;
  return bhac_stage(c, 2, dt);
}

static bhac_status copy_out(bhac_ctx* c, const double* dev_src, double* out, int on_device) {
  const size_t bytes = sizeof(double) * NV * (size_t)c->nb * c->nint;
  cudaError_t e = cudaMemcpyAsync(out, dev_src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  return cuda_status(e);
}

bhac_status bhac_get_prims(bhac_ctx* c, double* out, int on_device) {
  if (!c || !out) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  StageArgs a = base_args(c);
  if (on_device) return cuda_status(launch_gather_interior(a, c->P[c->cur], out, c->st));
  // the output staging buffer, once an asynchronous read-back still copying from it is done
  if (c->ev_d2h && cudaStreamWaitEvent(c->st, c->ev_d2h, 0) != cudaSuccess) return BHAC_ERR_CUDA;
  if (launch_gather_interior(a, c->P[c->cur], c->scratch_out, c->st) != cudaSuccess) return BHAC_ERR_CUDA;
  return copy_out(c, c->scratch_out, out, 0);
}

bhac_status bhac_get_cons(bhac_ctx* c, double* out, int on_device) {
  if (!c || !out) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  return copy_out(c, c->U[c->ucur], out, on_device);
}

bhac_status bhac_get_diagnostics(bhac_ctx* c, long long counts[4]) {
  if (!c || !counts) return BHAC_ERR_ARG;
  unsigned long long h[4];
  if (cudaMemcpyAsync(h, c->counts, sizeof(h), cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return BHAC_ERR_CUDA;
  for (int i = 0; i < 4; ++i) counts[i] = (long long)h[i];
  return h[3] ? BHAC_WARN_C2P : BHAC_OK;
}

bhac_status bhac_get_c2p_status(bhac_ctx* c, unsigned char* out, int on_device) {
  if (!c || !out) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(out, c->d_status, (size_t)c->nb * c->nint,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  return cuda_status(e);
}

bhac_status bhac_set_launch(bhac_ctx* c, int tx, int ty, int threads, int persistent, int min_ctas,
                            int producer_warps) {
  if (!c || min_ctas < 0 || min_ctas > 3 || producer_warps < 0) return BHAC_ERR_ARG;
  if (producer_warps > 0 && (c->d.ndim != 3 || producer_warps * 32 >= (threads > 0 ? threads : c->threads)))
    return BHAC_ERR_ARG;
  const int ntx = tx > 0 ? tx : c->tx, nty = ty > 0 ? ty : c->ty, nth = threads > 0 ? threads : c->threads;
  if (c->d.nx[0] % ntx || c->d.nx[1] % nty || nth % 32 || nth > 256 || persistent < 0 || persistent > 8)
    return BHAC_ERR_ARG;
  const size_t smem = stage_smem(c, ntx, nty, producer_warps);
  if (smem > (size_t)kMaxDynSmem) return BHAC_ERR_ARG;
  if (min_ctas > 0) c->minb = min_ctas;
  c->pwarps = producer_warps;
  c->tx = ntx;
  c->ty = nty;
  c->threads = nth;
  c->persistent = persistent;
  c->nzp_eff = 0;
  return BHAC_OK;
}

bhac_status bhac_set_split(bhac_ctx* c, int chunks) {
  if (!c || chunks < 0 || chunks > 32) return BHAC_ERR_ARG;
  if (chunks > 0 && (c->pwarps > 0 || c->ct)) return BHAC_ERR_ARG;
  if (chunks > 0 && !c->Rbuf) {
    // the second stream, its events and the right-hand-side buffer are made
    // on first use: the fused form needs none of them
    cudaError_t e = cudaSuccess;
    if (!c->st2) e = cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&c->ev_fork, &c->ev_join2})
      if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (int q = 0; q < 32 && e == cudaSuccess; ++q)
      if (!c->ev_chunk[q]) e = cudaEventCreateWithFlags(&c->ev_chunk[q], cudaEventDisableTiming);
    const size_t bytes = (c->mixed ? sizeof(float) : sizeof(double)) * NV * (size_t)c->nb * c->nint;
    if (e == cudaSuccess) e = cudaMalloc(&c->Rbuf, bytes);
    if (e == cudaErrorMemoryAllocation) {
      c->Rbuf = nullptr;
      cudaGetLastError();
      return BHAC_ERR_NOMEM;
    }
    if (e != cudaSuccess) return BHAC_ERR_CUDA;
  }
  c->split = chunks;
  c->nzp_eff = 0;
  return BHAC_OK;
}

bhac_status bhac_set_zsplit(bhac_ctx* c, int parts) {
  if (!c || parts < 0) return BHAC_ERR_ARG;
  if (parts > 0 && (c->d.ndim != 3 || c->d.nx[2] % parts)) return BHAC_ERR_ARG;
  c->zsplit = parts;
  c->nzp_eff = 0;
  return BHAC_OK;
}

int bhac_zsplit_in_force(const bhac_ctx* c) { return c ? c->nzp_eff : -1; }

bhac_status bhac_graph_capture(bhac_ctx* c, int nsteps) {
  if (!c || nsteps < 1) return BHAC_ERR_ARG;
  if (c->split > 0) return BHAC_ERR_STATE;  // the split form runs on two streams
  if (!c->prims_ok || !c->cfl_ok) return BHAC_ERR_STATE;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if ((c->mixed ? prepare_stage_mixed() : prepare_stage_fp64()) != cudaSuccess) return BHAC_ERR_CUDA;
  if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BHAC_ERR_CUDA;
  const int cur = c->cur, ucur = c->ucur, pcur = c->pcur;
  bhac_status s = BHAC_OK;
  for (int k = 0; k < nsteps && s == BHAC_OK; ++k) s = bhac_step(c, 0.0);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  c->cur = cur;  // buffer roles return to the same state after every step
  c->ucur = ucur;
  c->pcur = pcur;
  if (s != BHAC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return s != BHAC_OK ? s : BHAC_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return BHAC_ERR_CUDA;
  }
  c->graph_steps = nsteps;
  return BHAC_OK;
}

bhac_status bhac_graph_launch(bhac_ctx* c) {
  if (!c) return BHAC_ERR_ARG;
  if (!c->graph) return BHAC_ERR_STATE;
  c->cfl_fresh = false;
  return cuda_status(cudaGraphLaunch(c->graph, c->st));
}

bhac_status bhac_set_faces(bhac_ctx* c, const double* faces, int on_device) {
  if (!c || !faces) return BHAC_ERR_ARG;
  if (!c->ct || !c->prims_ok) return BHAC_ERR_STATE;
  const size_t n = (size_t)c->nb * c->ctg.nown_b;
  const double* src = faces;
  double* stage_buf = c->xf;  // the flux array is free between stages: it stages a host load
  if (!on_device) {
    if (cudaMemcpyAsync(stage_buf, faces, sizeof(double) * n, cudaMemcpyHostToDevice, c->st) != cudaSuccess)
      return BHAC_ERR_CUDA;
    src = stage_buf;
  }
  c->pcur = 0;
  StageArgs a = base_args(c);
  CtArgs t = ct_args(c);
  cudaError_t e = launch_ct_copy_faces(a, c->ctg, src, c->phi[0], 1, c->st);
  // the cell field of the loaded primitives from the faces, then U
  if (e == cudaSuccess) e = launch_ct_cell_field(a, t, c->P[c->cur], c->mixed ? c->P32[c->cur] : nullptr, c->st);
  if (e == cudaSuccess) e = launch_init_cons(a, c->P[c->cur], c->U[c->ucur], c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  c->faces_ok = true;
  c->cfl_ok = false;
  c->cfl_fresh = false;  // the cell field now comes from the faces
  return BHAC_OK;
}

bhac_status bhac_get_faces(bhac_ctx* c, double* out, int on_device) {
  if (!c || !out) return BHAC_ERR_ARG;
  if (!c->ct || !c->faces_ok) return BHAC_ERR_STATE;
  const size_t n = (size_t)c->nb * c->ctg.nown_b;
  StageArgs a = base_args(c);
  double* dst = on_device ? out : c->xf;
  cudaError_t e = launch_ct_copy_faces(a, c->ctg, c->phi[c->pcur], dst, 0, c->st);
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dst, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->st);
  return cuda_status(e);
}

void bhac_destroy(bhac_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (cudaStream_t s : {c->cp_in, c->cp_out})
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  for (cudaEvent_t e : {c->ev_h2d, c->ev_scat, c->ev_gath, c->ev_d2h, c->ev_fence, c->ev_join_in, c->ev_join_out,
                        c->ev_fork, c->ev_join2})
    if (e) cudaEventDestroy(e);
  for (int q = 0; q < 32; ++q)
    if (c->ev_chunk[q]) cudaEventDestroy(c->ev_chunk[q]);
  if (c->st2) {
    cudaStreamSynchronize(c->st2);
    cudaStreamDestroy(c->st2);
  }
  if (c->Rbuf) cudaFree(c->Rbuf);
  delete c;
}

}  // extern "C"
