// Staggered-mesh constrained transport: face-field and edge-EMF layouts, the
// host-built maps of the ring faces (and, across refinement levels, of the
// coarse-fine flux and EMF corrections), and the kernel launchers (ct.cu).
#pragma once

#include <vector>

#include "../../include/bhac_gb300.h"
#include "bhac_device.cuh"

namespace bhac {

// Per block, for each active direction d: the face field Phi^d = sqrt(gamma) B^d
// (and the NV fluxes) on the faces normal to d, over the block's own faces
// (index 0..nx_d along d, the block's cells across) plus a ring of one face
// across in every active transverse direction.  fe[d][e]: extent along e;
// fo[d][e]: where local index 0 sits inside it; foff[d]: first face of
// direction d inside one block's record; nfb: faces per block.
// Edge EMFs (refinement levels only): E_a on the block's edges along a, the
// block's cells along a and its faces 0..nx_e across (ee[a][e] extents, eoff[a]
// the first edge of direction a in one block's record, nEb edges per block;
// in 2-D only E_3).
struct CtGeom {
  int ndim, nx[3];
  int fe[3][3], fo[3][3];
  long long foff[3], nfd[3], nfb;
  long long own_off[3], nown_d[3], nown_b;  // owned faces only (the public layout)
  int ee[3][3];
  long long eoff[3], nEb;
};

CtGeom ct_geom(const bhac_grid_desc* d);

// Index of face (d; i, j, k) of a block in its ring-layout record (i, j, k
// local: along d 0..nx_d, across -1..nx_e in active directions).
__host__ __device__ __forceinline__ long long ring_index(const CtGeom& g, int d, int i, int j, int k) {
  return g.foff[d] + ((long long)(k + g.fo[d][2]) * g.fe[d][1] + (j + g.fo[d][1])) * g.fe[d][0] + (i + g.fo[d][0]);
}

// Direction and local index of owned face r of a block (the public order:
// d, then k, j, i with i fastest).
__host__ __device__ __forceinline__ void owned_face(const CtGeom& g, int r, int& d, int& i, int& j, int& k) {
  d = (g.ndim == 3 && r >= g.own_off[2]) ? 2 : (r >= g.own_off[1] ? 1 : 0);
  const int q = r - (int)g.own_off[d];
  const int n0 = g.nx[0] + (d == 0), n1 = g.nx[1] + (d == 1);
  i = q % n0;
  j = (q / n0) % n1;
  k = q / (n0 * n1);
}

// Ring faces: for every block and ring slot, the Phi index it copies (a face
// owned by the neighbour across, after the boundary rules).  Returns false if a
// rule points at a missing block.
bool ct_ring_map(const bhac_grid_desc* d, const bhac_block_desc* b, int nb, const CtGeom& g,
                 std::vector<long long>& dst, std::vector<long long>& src);

// Grids with refinement levels.  Ring faces: a copy of the face of the leaf at
// the block's level (copy_*), else the mean of 2 or 4 faces (mean_*, 4 sources
// per entry, -1 padded): the two faces of the coarser cell a face cuts, or the
// finer faces on it (a face lying on a coarser face copies it).  Fluxes
// (xr_*): a coarse face on a level boundary gets the mean of the finer faces'
// fluxes (sources and destination are the flux index of variable 0, xr_d the
// direction; 4 sources, -1 padded).  EMFs (ef_*): an edge that a finer leaf
// touches gets the mean of the finer EMFs along it (2 sources, -1 padded).
// ok is false if a boundary rule or a level points at a missing block, or the
// levels of neighbouring leaves differ by more than one.
struct CtLevelMaps {
  std::vector<long long> copy_dst, copy_src, mean_dst, mean_src;
  std::vector<long long> xr_dst, xr_src, ef_dst, ef_src;
  std::vector<int> xr_d;
  bool ok;
};
CtLevelMaps ct_level_maps(const bhac_grid_desc* d, const bhac_block_desc* b, int nb, const CtGeom& g);

struct CtArgs {
  CtGeom g;
  const double* phi_in;   // Phi of the stage's input state, ring filled
  double* phi_out;        // Phi written by the face update
  const double* phi_n;    // Phi at the start of the step (stage 2)
  double* xf;             // fluxes [block][d][var][face], ring-extended
  const double* te_c;     // metric records on the grid extended by one cell each side in x1, x2
  const double* te_f1;
  const double* te_f2;
  const float* te_c32;    // their FP32 copies (mixed form)
  const float* te_f1_32;
  const float* te_f2_32;
  long long teo_c[MAXLEV], teo_f1[MAXLEV], teo_f2[MAXLEV];  // each level's first record in them
  int axis_lo, axis_hi;   // polar axis at the low / high x2 boundary
  // refinement levels: edge EMFs [block][edge], the flux and EMF corrections
  int amr;
  double* emf;
  const long long* xr_dst;
  const long long* xr_src;
  const int* xr_d;
  long long nxr;
  const long long* ef_dst;
  const long long* ef_src;
  long long nef;
};

cudaError_t launch_ct_ring(const long long* dst, const long long* src, long long n, double* phi, cudaStream_t st);
// ring faces that average 2 or 4 owned faces (4 sources per entry, -1 padded)
cudaError_t launch_ct_ring_mean(const long long* dst, const long long* src, long long n, double* phi,
                                cudaStream_t st);
// mixed: FP32 face fluxes and cell sources (the mixed form); else FP64
cudaError_t launch_ct_stage(const StageArgs& a, const CtArgs& c, bool mixed, cudaStream_t st);
// B^d of the interior cells of P (and of its FP32 copy P32 when not null) from
// the faces, psi = 0 (after a face load)
cudaError_t launch_ct_cell_field(const StageArgs& a, const CtArgs& c, double* P, float* P32, cudaStream_t st);
// owned faces <-> the ring layout
cudaError_t launch_ct_copy_faces(const StageArgs& a, const CtGeom& g, const double* src, double* dst, int to_ring,
                                 cudaStream_t st);

}  // namespace bhac
