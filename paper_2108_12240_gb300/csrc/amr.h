// Ghost maps and coarse-fine flux-correction tables for block grids with
// several refinement levels (host construction, device layout).
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/bhac_gb300.h"
#include "bhac_device.cuh"

namespace bhac {

// Operand of a ghost node: an interior cell (with boundary fix-up flags) or
// the output of another node.
constexpr long long OP_NODE = 1LL << 62;
__host__ __device__ __forceinline__ long long op_cell(long long cell, unsigned flags) {
  return cell | ((long long)flags << 32);
}
__host__ __device__ __forceinline__ long long op_node(long long node) { return node | OP_NODE; }

enum NodeType { NODE_RESTRICT = 1, NODE_PROLONG = 2 };

// x: type | flags << 8 | parity << 16 (bit d: fine cell is the upper child along d),
// y: first operand, z: operand count.
struct GhostNode {
  int x, y, z, w;
};

// One coarse cell next to a face whose neighbour is finer, with up to three
// corrections (one per direction it touches).
struct RefluxTerm {
  long long coarse;      // register element of the coarse face flux (variable 0)
  long long fine[4];     // register elements of the covering fine face fluxes (variable 0)
  int cstride, fstride;  // variable strides of the two registers
  int nfine, d, sign, pad;
};
struct RefluxCell {
  int b, ci, cg, level;
  int I1, I2, term0, nterm;
};

struct HostMaps {
  std::vector<int> tmpl;               // ghost slot -> cell inside a block
  std::vector<int> src;                // per (block, slot): >= 0 cell, < 0 -(node + 1)
  std::vector<unsigned char> flags;    // per (block, slot) for cell sources
  std::vector<GhostNode> nodes;        // sorted by depth
  std::vector<long long> ops;
  std::vector<int> depth_start;        // nodes of depth k: [depth_start[k-1], depth_start[k])
  std::vector<unsigned char> cf;       // per block: bit 2d+s set if face (d, s) borders finer blocks
  std::vector<long long> regoff;       // per block x 6: register element offset, or -1
  long long reg_elems = 0;
  std::vector<RefluxCell> rcells;
  std::vector<RefluxTerm> rterms;
  bool ok = true;
};

// Builds every map of a grid (same-level copies, boundary rules, cross-level
// nodes, flux registers).  g/N/ncell: ghost widths, ghosted extents, cells per block.
HostMaps build_maps(const bhac_grid_desc* d, const bhac_block_desc* b, int nb, const int g[3], const int N[3],
                    int ncell);

struct NodeArgs {
  const GhostNode* nodes;
  const long long* ops;
  int first, count, nnodes, ncell;
  const double* P;
  const float* P32;
  double* out;        // nnodes x NV
  float* out32;
};
cudaError_t launch_ghost_nodes(const NodeArgs& n, cudaStream_t st);

}  // namespace bhac
