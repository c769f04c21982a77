// The library context (host memory), shared by the translation units that
// implement the C ABI.
#pragma once

#include <vector>

#include "../../include/bhac_gb300.h"
#include "amr.h"
#include "ct.h"
#include "launch.h"

struct bhac_ctx {
  // descriptor, blocks and stream
  bhac_grid_desc d;
  int nb;
  std::vector<int> blk;  // nb x 4
  cudaStream_t st;
  // geometry
  int g[3], N[3], ncell, nint, nslots;
  int N1g, N2g;
  bool flat, mixed;
  // arena slices
  char* arena;
  size_t arena_bytes;
  int* d_blk;
  int* d_order;
  int* d_src;
  unsigned char* d_flags;
  int* d_tmpl;
  double *tab_c, *tab_f1, *tab_f2;
  float *tab_c32, *tab_f1_32, *tab_f2_32;
  double* P[2];
  float* P32[2];
  double* U[2];
  double* scratch;      // interior primitives: host loads (input staging)
  double* scratch_out;  // interior primitives: host read-backs (output staging)
  double* dt_dev;
  unsigned long long* smax;
  unsigned long long* counts;
  unsigned char* d_status;   // per interior cell: inversion outcome of the last stage
  unsigned int* work;
  // state
  int cur;       // primitive buffer holding the current state
  int ucur;      // conserved buffer holding the current state
  bool metric_ok, prims_ok, cfl_ok;
  bool cfl_fresh;  // smax holds the CFL rate of the current primitives (set by loads and bhac_cfl_dt)
  // launch shape
  int tx, ty, threads, persistent, minb, pwarps;
  // refinement levels: metric-table record offsets per level
  long long toff_c[bhac::MAXLEV], toff_f1[bhac::MAXLEV], toff_f2[bhac::MAXLEV];
  // cross-level ghost nodes (evaluated depth by depth) and flux correction
  int nnodes;
  std::vector<int> depth_start;
  bhac::GhostNode* d_nodes;
  long long* d_ops;
  double* d_node64;
  float* d_node32;
  unsigned char* d_cf;
  long long* d_regoff;
  double* d_reg;
  bhac::RefluxCell* d_rcells;
  bhac::RefluxTerm* d_rterms;
  int nrcells;
  // constrained transport: face fields in ring layout (two buffers, pcur the
  // current state's), ring-extended face fluxes, the metric records of every
  // level on its grid extended by one cell in x1 and x2 (teo_*: each level's
  // first record), and the ring-face maps (copies; means of 2 or 4 faces
  // across levels); with refinement levels also the edge EMFs and the maps of
  // the coarse-fine flux and EMF corrections
  bool ct, faces_ok;
  bhac::CtGeom ctg;
  double* phi[2];
  int pcur;
  double* xf;
  double *te_c, *te_f1, *te_f2;
  float *te_c32, *te_f1_32, *te_f2_32;
  long long teo_c[bhac::MAXLEV], teo_f1[bhac::MAXLEV], teo_f2[bhac::MAXLEV];
  long long *ring_dst, *ring_src, *ringm_dst, *ringm_src;
  long long nring, nringm;
  double* emf;
  long long *xr_dst, *xr_src, *ef_dst, *ef_src;
  int* xr_d;
  long long nxr, nef;
  // split form: chunks of items, the face kernel on st and the cell kernel on
  // st2, chunk by chunk; R holds the stage right-hand side
  int split;
  // z parts per (block, tile) item of the phased 3-D kernel: zsplit as set
  // (0: chosen by the library), nzp_eff the count in force (0: not yet chosen)
  int zsplit, nzp_eff;
  cudaStream_t st2;
  cudaEvent_t ev_chunk[32], ev_fork, ev_join2;
  double* Rbuf;
  // captured steps
  cudaGraphExec_t graph;
  int graph_steps;
  // pipelined host transfers: one copy stream per direction and the events
  // that order them with the context's stream
  cudaStream_t cp_in, cp_out;
  cudaEvent_t ev_h2d, ev_scat, ev_gath, ev_d2h, ev_fence, ev_join_in, ev_join_out;
};

// Shared helpers of the ABI units (api.cu).
bhac::StageArgs base_args(const bhac_ctx* c);
bhac_status ghost_fill(bhac_ctx* c, int buf, bool zero_smax);
size_t stage_smem(const bhac_ctx* c, int tx, int ty, int pwarps);
