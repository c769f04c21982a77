// Ghost maps for block grids with several refinement levels, and the tables
// of the coarse-fine flux correction (block-based AMR, paper Sec. 2).
//
// A ghost cell's value is defined by the level-L global index it stands for,
// after the boundary rules: a copy where a level-L leaf holds the cell; a
// minmod-limited linear prolongation from level L-1 where a coarser leaf
// holds it; the mean of the 2^ndim level-(L+1) cells where finer leaves hold
// it.  Operands of a prolongation or a restriction may themselves be
// prolongations or restrictions (e.g. the coarse neighbour of a coarse cell
// lies inside the refined region), so the host expands the definition once
// into a DAG of nodes over interior cells; the device evaluates the nodes in
// order of depth and the ghost gather reads either a cell or a node.
#include <string.h>

#include <algorithm>
#include <unordered_map>

#include "amr.h"
#include "launch.h"

namespace bhac {

namespace {

struct Builder {
  const bhac_grid_desc* d;
  int nb, g[3], N[3], ncell, nlev;
  std::vector<std::vector<int>> lut;  // per level: block id at block coordinates
  std::vector<GhostNode> nodes;        // creation order
  std::vector<int> depth;              // per node
  std::vector<std::vector<long long>> nops;  // per node operand list
  std::unordered_map<unsigned long long, long long> memo;
  bool ok = true;

  long long extent(int k, int L) const { return (long long)d->nroot[k] * d->nx[k] << (k < d->ndim ? L : 0); }
  long long nblk(int k, int L) const { return (long long)d->nroot[k] << (k < d->ndim ? L : 0); }

  int lookup(int L, const long long bc[3]) const {
    if (L < 0 || L >= nlev) return -1;
    for (int k = 0; k < 3; ++k)
      if (bc[k] < 0 || bc[k] >= nblk(k, L)) return -1;
    return lut[L][(size_t)((bc[2] * nblk(1, L) + bc[1]) * nblk(0, L) + bc[0])];
  }

  // boundary rules at level L (same as the level-0 rules with extents scaled)
  bool rules(int L, long long G[3], unsigned& flags) const {
    flags = 0;
    for (int k = 0; k < d->ndim; ++k) {
      const long long Nk = extent(k, L);
      for (int side = 0; side < 2; ++side) {
        const bool out = side == 0 ? G[k] < 0 : G[k] >= Nk;
        if (!out) continue;
        const int kind = d->bc[k][side];
        if (kind == BHAC_BC_PERIODIC) {
          G[k] = ((G[k] % Nk) + Nk) % Nk;
        } else if (kind == BHAC_BC_OUTFLOW || kind == BHAC_BC_NOINFLOW) {
          G[k] = side == 0 ? 0 : Nk - 1;
          if (kind == BHAC_BC_NOINFLOW) flags |= 1u << (side == 0 ? 1 + 2 * k : 2 + 2 * k);
        } else {
          G[k] = side == 0 ? -1 - G[k] : 2 * Nk - 1 - G[k];
          flags ^= 1u;
          if (d->ndim == 3) G[2] += extent(2, L) / 2;
        }
      }
    }
    if (d->ndim == 3 && d->bc[2][0] == BHAC_BC_PERIODIC) {
      const long long N2 = extent(2, L);
      G[2] = ((G[2] % N2) + N2) % N2;
    }
    for (int k = 0; k < 3; ++k)
      if (G[k] < 0 || G[k] >= extent(k, L)) return false;
    return true;
  }

  int depth_of(long long op) const { return (op & OP_NODE) ? depth[(size_t)(op & 0xffffffffLL)] : 0; }

  long long add_node(int type, unsigned flags, unsigned parity, std::vector<long long>&& ops) {
    int dep = 0;
    for (long long o : ops) dep = std::max(dep, depth_of(o));
    GhostNode n;
    n.x = type | (int)(flags << 8) | (int)(parity << 16);
    n.y = 0;
    n.z = (int)ops.size();
    n.w = 0;
    nodes.push_back(n);
    depth.push_back(dep + 1);
    nops.push_back(std::move(ops));
    return op_node((long long)nodes.size() - 1);
  }

  long long value_of(int L, const long long Gin[3]) {
    long long G[3] = {Gin[0], Gin[1], Gin[2]};
    unsigned fl = 0;
    long long res = 0;
    if (!rules(L, G, fl)) {
      ok = false;
      return 0;
    }
    long long bc[3];
    for (int k = 0; k < 3; ++k) bc[k] = G[k] / d->nx[k];
    const int b = lookup(L, bc);
    if (b >= 0) {
      // a cell of a leaf at this level (most ghost slots): no memo needed
      const long long li = G[0] % d->nx[0] + g[0], lj = G[1] % d->nx[1] + g[1], lk = G[2] % d->nx[2] + g[2];
      return op_cell((long long)b * ncell + (lk * N[1] + lj) * N[0] + li, fl);
    }
    const unsigned long long key = ((unsigned long long)L << 60) |
                                   ((unsigned long long)(Gin[0] + 64) & 0xfffffULL) |
                                   (((unsigned long long)(Gin[1] + 64) & 0xfffffULL) << 20) |
                                   (((unsigned long long)(Gin[2] + 64) & 0xfffffULL) << 40);
    auto it = memo.find(key);
    if (it != memo.end()) return it->second;
    bool coarse = false;
    for (int Lc = L - 1; Lc >= 0 && !coarse; --Lc) {
      long long bcc[3];
      for (int k = 0; k < 3; ++k) bcc[k] = (k < d->ndim ? G[k] >> (L - Lc) : G[k]) / d->nx[k];
      coarse = lookup(Lc, bcc) >= 0;
    }
    if (coarse && L > 0) {
      long long C[3];
      for (int k = 0; k < 3; ++k) C[k] = k < d->ndim ? G[k] >> 1 : G[k];
      std::vector<long long> ops;
      ops.push_back(value_of(L - 1, C));
      unsigned parity = 0;
      for (int k = 0; k < d->ndim; ++k) {
        long long Cm[3] = {C[0], C[1], C[2]}, Cp[3] = {C[0], C[1], C[2]};
        Cm[k] -= 1;
        Cp[k] += 1;
        ops.push_back(value_of(L - 1, Cm));
        ops.push_back(value_of(L - 1, Cp));
        if (G[k] & 1) parity |= 1u << k;
      }
      res = add_node(NODE_PROLONG, fl, parity, std::move(ops));
    } else if (L + 1 < nlev) {
      std::vector<long long> ops;
      const int nch = 1 << d->ndim;
      for (int ch = 0; ch < nch; ++ch) {
        long long F[3] = {G[0], G[1], G[2]};
        for (int k = 0; k < d->ndim; ++k) F[k] = 2 * G[k] + ((ch >> k) & 1);
        ops.push_back(value_of(L + 1, F));
      }
      res = add_node(NODE_RESTRICT, fl, 0u, std::move(ops));
    } else {
      ok = false;  // nothing holds this cell
    }
    if (res & OP_NODE) memo[key] = res;
    return res;
  }
};

}  // namespace

HostMaps build_maps(const bhac_grid_desc* d, const bhac_block_desc* blocks, int nb, const int g[3], const int N[3],
                    int ncell) {
  HostMaps M;
  Builder B;
  B.d = d;
  B.nb = nb;
  B.ncell = ncell;
  B.nlev = d->nlevels;
  for (int k = 0; k < 3; ++k) {
    B.g[k] = g[k];
    B.N[k] = N[k];
  }
  B.lut.resize(B.nlev);
  for (int L = 0; L < B.nlev; ++L) B.lut[L].assign((size_t)(B.nblk(0, L) * B.nblk(1, L) * B.nblk(2, L)), -1);
  for (int i = 0; i < nb; ++i) {
    const int L = blocks[i].level;
    B.lut[L][(size_t)(((long long)blocks[i].iz * B.nblk(1, L) + blocks[i].iy) * B.nblk(0, L) + blocks[i].ix)] = i;
  }
  // ghost slots of a block, in (k, j, i) order
  for (int k = 0; k < N[2]; ++k)
    for (int j = 0; j < N[1]; ++j)
      for (int i = 0; i < N[0]; ++i) {
        const bool in = i >= g[0] && i < g[0] + d->nx[0] && j >= g[1] && j < g[1] + d->nx[1] && k >= g[2] &&
                        k < g[2] + d->nx[2];
        if (!in) M.tmpl.push_back((k * N[1] + j) * N[0] + i);
      }
  const int nslots = (int)M.tmpl.size();
  std::vector<long long> gsrc((size_t)nb * nslots);
  for (int bi = 0; bi < nb && B.ok; ++bi) {
    const int L = blocks[bi].level;
    const int bc[3] = {blocks[bi].ix, blocks[bi].iy, blocks[bi].iz};
    for (int s = 0; s < nslots && B.ok; ++s) {
      const int cell = M.tmpl[s];
      const int loc[3] = {cell % N[0] - g[0], (cell / N[0]) % N[1] - g[1], cell / (N[0] * N[1]) - g[2]};
      long long G[3];
      for (int k = 0; k < 3; ++k) G[k] = (long long)bc[k] * d->nx[k] + loc[k];
      gsrc[(size_t)bi * nslots + s] = B.value_of(L, G);
    }
  }
  if (!B.ok) {
    M.ok = false;
    return M;
  }
  // order nodes by depth and remap
  const int nn = (int)B.nodes.size();
  int maxd = 0;
  for (int i = 0; i < nn; ++i) maxd = std::max(maxd, B.depth[i]);
  std::vector<int> order(nn), newidx(nn);
  for (int i = 0; i < nn; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B.depth[a] < B.depth[b]; });
  for (int i = 0; i < nn; ++i) newidx[order[i]] = i;
  M.depth_start.assign(maxd + 1, 0);
  auto remap = [&](long long op) {
    return (op & OP_NODE) ? op_node(newidx[(size_t)(op & 0xffffffffLL)]) : op;
  };
  for (int r = 0; r < nn; ++r) {
    const int i = order[r];
    GhostNode n = B.nodes[i];
    n.y = (int)M.ops.size();
    for (long long o : B.nops[i]) M.ops.push_back(remap(o));
    M.nodes.push_back(n);
  }
  for (int dep = 1; dep <= maxd; ++dep) {
    int c = 0;
    for (int i = 0; i < nn; ++i) c += B.depth[i] < dep;
    M.depth_start[dep - 1] = c;
  }
  M.depth_start[maxd] = nn;
  M.src.resize(gsrc.size());
  M.flags.resize(gsrc.size());
  for (size_t t = 0; t < gsrc.size(); ++t) {
    const long long op = remap(gsrc[t]);
    if (op & OP_NODE) {
      M.src[t] = -(int)(op & 0xffffffffLL) - 1;
      M.flags[t] = 0;
    } else {
      M.src[t] = (int)(op & 0xffffffffLL);
      M.flags[t] = (unsigned char)((op >> 32) & 0xff);
    }
  }

  // flux registers at faces between levels, and the coarse cells to correct
  M.cf.assign(nb, 0);
  M.regoff.assign((size_t)nb * 6, -1);
  auto ncf = [&](int dd) {
    int n = 1;
    for (int k = 0; k < 3; ++k)
      if (k != dd) n *= d->nx[k];
    return n;
  };
  std::vector<int> side_kind((size_t)nb * 6, 0);  // 1 fine side, 2 coarse side
  for (int bi = 0; bi < nb; ++bi) {
    const int L = blocks[bi].level;
    const long long c[3] = {blocks[bi].ix, blocks[bi].iy, blocks[bi].iz};
    for (int dd = 0; dd < d->ndim; ++dd)
      for (int s = 0; s < 2; ++s) {
        long long nbc[3] = {c[0], c[1], c[2]};
        nbc[dd] += s ? 1 : -1;
        const long long nbd = B.nblk(dd, L);
        if (nbc[dd] < 0 || nbc[dd] >= nbd) {
          if (d->bc[dd][s] != BHAC_BC_PERIODIC) continue;
          nbc[dd] = (nbc[dd] + nbd) % nbd;
        }
        if (B.lookup(L, nbc) >= 0) continue;
        int kind = 0;
        if (L > 0) {
          long long pc[3];
          for (int k = 0; k < 3; ++k) pc[k] = k < d->ndim ? nbc[k] >> 1 : nbc[k];
          if (B.lookup(L - 1, pc) >= 0) kind = 1;
        }
        if (!kind) {
          long long ch[3];
          for (int k = 0; k < 3; ++k) ch[k] = k < d->ndim ? 2 * nbc[k] : nbc[k];
          if (s == 0) ch[dd] += 1;
          if (B.lookup(L + 1, ch) >= 0) kind = 2;
        }
        if (!kind) continue;
        side_kind[(size_t)bi * 6 + 2 * dd + s] = kind;
        M.regoff[(size_t)bi * 6 + 2 * dd + s] = M.reg_elems;
        M.reg_elems += (long long)NV * ncf(dd);
        if (kind == 2) M.cf[bi] |= (unsigned char)(1u << (2 * dd + s));
      }
  }
  // corrections, cell by cell (a cell at an edge gets one term per face)
  std::unordered_map<long long, int> cell_of;
  std::vector<std::vector<RefluxTerm>> terms;
  for (int bi = 0; bi < nb; ++bi) {
    if (!M.cf[bi]) continue;
    const int L = blocks[bi].level;
    const long long c[3] = {blocks[bi].ix, blocks[bi].iy, blocks[bi].iz};
    for (int dd = 0; dd < d->ndim; ++dd)
      for (int s = 0; s < 2; ++s) {
        if (side_kind[(size_t)bi * 6 + 2 * dd + s] != 2) continue;
        long long nbc[3] = {c[0], c[1], c[2]};
        nbc[dd] += s ? 1 : -1;
        const long long nbd = B.nblk(dd, L);
        nbc[dd] = (nbc[dd] + nbd) % nbd;
        long long chb[3];
        for (int k = 0; k < 3; ++k) chb[k] = k < d->ndim ? 2 * nbc[k] : nbc[k];
        if (s == 0) chb[dd] += 1;
        const int t1 = (dd + 1) % 3, t2 = (dd + 2) % 3;  // the oracle's summation order
        const int lo = dd == 0 ? 1 : 0, hi = dd == 2 ? 1 : 2;  // register layout: transverse dims ascending
        for (int a1 = 0; a1 < d->nx[t1]; ++a1)
          for (int a2 = 0; a2 < d->nx[t2]; ++a2) {
            int loc[3];
            loc[dd] = s ? d->nx[dd] - 1 : 0;
            loc[t1] = a1;
            loc[t2] = a2;
            RefluxTerm T;
            memset(&T, 0, sizeof(T));
            T.d = dd;
            T.sign = s == 0 ? 1 : -1;
            T.cstride = ncf(dd);
            T.fstride = ncf(dd);
            T.coarse = M.regoff[(size_t)bi * 6 + 2 * dd + s] + (long long)loc[hi] * d->nx[lo] + loc[lo];
            int cnt = 0;
            for (int s1 = 0; s1 < (t1 < d->ndim ? 2 : 1); ++s1)
              for (int s2 = 0; s2 < (t2 < d->ndim ? 2 : 1); ++s2) {
                long long Gf[3];
                const long long gc1 = c[t1] * d->nx[t1] + a1, gc2 = c[t2] * d->nx[t2] + a2;
                Gf[t1] = t1 < d->ndim ? 2 * gc1 + s1 : gc1;
                Gf[t2] = t2 < d->ndim ? 2 * gc2 + s2 : gc2;
                long long fb[3];
                fb[dd] = chb[dd];
                fb[t1] = Gf[t1] / d->nx[t1];
                fb[t2] = Gf[t2] / d->nx[t2];
                const int bf = B.lookup(L + 1, fb);
                if (bf < 0) continue;
                int fl[3];
                fl[dd] = 0;
                fl[t1] = (int)(Gf[t1] % d->nx[t1]);
                fl[t2] = (int)(Gf[t2] % d->nx[t2]);
                const long long ro = M.regoff[(size_t)bf * 6 + 2 * dd + (1 - s)];
                if (ro < 0) {
                  M.ok = false;
                  return M;
                }
                T.fine[cnt++] = ro + (long long)fl[hi] * d->nx[lo] + fl[lo];
              }
            T.nfine = cnt;
            if (cnt == 0) continue;
            const long long key = (long long)bi * ncell + ((loc[2] + g[2]) * N[1] + loc[1] + g[1]) * N[0] + loc[0] + g[0];
            auto it = cell_of.find(key);
            int id;
            if (it == cell_of.end()) {
              id = (int)M.rcells.size();
              cell_of[key] = id;
              RefluxCell rc;
              rc.b = bi;
              rc.ci = (loc[2] * d->nx[1] + loc[1]) * d->nx[0] + loc[0];
              rc.cg = ((loc[2] + g[2]) * N[1] + loc[1] + g[1]) * N[0] + loc[0] + g[0];
              rc.level = L;
              rc.I1 = (int)(c[0] * d->nx[0] + loc[0]);
              rc.I2 = (int)(c[1] * d->nx[1] + loc[1]);
              rc.term0 = 0;
              rc.nterm = 0;
              M.rcells.push_back(rc);
              terms.emplace_back();
            } else {
              id = it->second;
            }
            terms[id].push_back(T);
          }
      }
  }
  for (size_t i = 0; i < M.rcells.size(); ++i) {
    M.rcells[i].term0 = (int)M.rterms.size();
    M.rcells[i].nterm = (int)terms[i].size();
    for (const RefluxTerm& T : terms[i]) M.rterms.push_back(T);
  }
  return M;
}

// ----------------------------------------------------------------------------
// Node evaluation: restriction = mean of the operands in order; prolongation =
// centre + sum over d of (+-1/4) minmod(centre - minus_d, plus_d - centre);
// then the node's own boundary fix-ups.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void fetch_op(long long op, const T* P, const T* out, int ncell, T v[NV]) {
  if (op & OP_NODE) {
    const T* s = out + (size_t)(op & 0xffffffffLL) * NV;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = s[q];
    return;
  }
  const int cell = (int)(op & 0xffffffffLL);
  const unsigned f = (unsigned)((op >> 32) & 0xff);
  const int sb = cell / ncell, sc = cell - sb * ncell;
  const T* s = P + (size_t)sb * NV * ncell + sc;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = s[(size_t)q * ncell];
  if (f & 1u) {
    v[U2] = -v[U2];
    v[B2] = -v[B2];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if ((f >> (1 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] > T(0) ? T(0) : v[U1 + d];
    if ((f >> (2 + 2 * d)) & 1u) v[U1 + d] = v[U1 + d] < T(0) ? T(0) : v[U1 + d];
  }
}

template <typename T>
__global__ void __launch_bounds__(128) ghost_node_kernel(const GhostNode* __restrict__ nodes,
                                                         const long long* __restrict__ ops, int first, int count,
                                                         int ncell, const T* __restrict__ P, T* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const int i = first + t;
    const GhostNode n = nodes[i];
    const int type = n.x & 0xff;
    const unsigned f = (unsigned)(n.x >> 8) & 0xffu, parity = (unsigned)(n.x >> 16) & 0xffu;
    T acc[NV], v[NV];
    if (type == NODE_RESTRICT) {
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] = T(0);
      for (int o = 0; o < n.z; ++o) {
        fetch_op<T>(ops[n.y + o], P, out, ncell, v);
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += v[q];
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) acc[q] /= T(n.z);
    } else {
      fetch_op<T>(ops[n.y], P, out, ncell, acc);
      T c[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) c[q] = acc[q];
      const int ndim = (n.z - 1) / 2;
      for (int d = 0; d < ndim; ++d) {
        T m[NV], p[NV];
        fetch_op<T>(ops[n.y + 1 + 2 * d], P, out, ncell, m);
        fetch_op<T>(ops[n.y + 2 + 2 * d], P, out, ncell, p);
        const T off = ((parity >> d) & 1u) ? T(0.25) : T(-0.25);
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] += off * minmod_t(c[q] - m[q], p[q] - c[q]);
      }
    }
    if (f & 1u) {
      acc[U2] = -acc[U2];
      acc[B2] = -acc[B2];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if ((f >> (1 + 2 * d)) & 1u) acc[U1 + d] = acc[U1 + d] > T(0) ? T(0) : acc[U1 + d];
      if ((f >> (2 + 2 * d)) & 1u) acc[U1 + d] = acc[U1 + d] < T(0) ? T(0) : acc[U1 + d];
    }
    T* o = out + (size_t)i * NV;
#pragma unroll
    for (int q = 0; q < NV; ++q) o[q] = acc[q];
  }
}

cudaError_t launch_ghost_nodes(const NodeArgs& n, cudaStream_t st) {
  if (n.count <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int grid = (n.count + 127) / 128;
  if (grid > 32 * nsm) grid = 32 * nsm;
  if (n.P32)
    ghost_node_kernel<float><<<grid, 128, 0, st>>>(n.nodes, n.ops, n.first, n.count, n.ncell, n.P32, n.out32);
  else
    ghost_node_kernel<double><<<grid, 128, 0, st>>>(n.nodes, n.ops, n.first, n.count, n.ncell, n.P, n.out);
  return cudaGetLastError();
}

}  // namespace bhac
