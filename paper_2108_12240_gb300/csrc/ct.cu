// Staggered-mesh constrained transport (the div B control of the method's
// Sec. 2), in the FP64 form or the mixed form (T = float: the
// face states and fluxes in FP32 from the FP32 primitives, the fluxes stored,
// the EMFs, the face update and the face field in FP64, so the discrete
// divergence stays at FP64 round-off; the cell sources in FP32 and the
// inversion as in the mixed stage kernel).
//
// Evolved field: Phi^d = sqrt(gamma) B^d at the centre of every face normal to
// an active direction d.  A stage runs, after the usual ghost-cell fill:
//   ring   the faces one cell outside each block (across, in every active
//          transverse direction) copied from the neighbour that owns them;
//   flux   every face of the block and its ring: PPM/minmod states from the
//          ghosted primitives, the normal field of both states set to the
//          face's own Phi^d / sqrt(gamma), HLL/TVDLF flux (densitized);
//   faces  d_t Phi = -curl E on the block's faces, the edge EMF the mean of
//          the four face fluxes of B around the edge (E_3 = F^2(B^1) =
//          -F^1(B^2), and cyclically), then the RK stage combination;
//   cells  flux divergence, sources and RK combination of D, S_i, tau (and of
//          B^3 in 2-D), cell field sqrt(gamma) B^d = (Phi^d_low + Phi^d_high)/2,
//          then the inversion, floors and CFL rate of the stage kernel.
// Both blocks sharing a face compute its update from identical inputs (their
// ghost cells and ring faces hold the same values), so their copies agree and
// the discrete divergence sum_d dPhi^d/dx_d of every cell stays at round-off.
// Across refinement levels a ring face is a copy, or the mean of the two faces
// of the coarser cell it cuts, or of the finer faces on it; after the fluxes,
// a coarse face on a level boundary takes the mean of the finer fluxes, every
// edge EMF is stored, and an edge that a finer leaf touches takes the mean of
// the finer EMFs along it before the face update (host-built maps), so the
// coarse copy of a level-boundary face changes by the mean of the changes of
// the finer faces covering it.
// psi is not evolved (zero), and no cleaning speed enters the fluxes.
#include <algorithm>
#include <thread>

#include "ct.h"
#include "stage_impl.cuh"

namespace bhac {

CtGeom ct_geom(const bhac_grid_desc* d) {
  CtGeom g;
  g.ndim = d->ndim;
  for (int e = 0; e < 3; ++e) g.nx[e] = d->nx[e];
  long long off = 0, own = 0;
  for (int dd = 0; dd < 3; ++dd) {
    long long nf = 1, no = 1;
    for (int e = 0; e < 3; ++e) {
      const bool across = e != dd && e < d->ndim;
      g.fe[dd][e] = e == dd ? d->nx[e] + 1 : d->nx[e] + (across ? 2 : 0);
      g.fo[dd][e] = across ? 1 : 0;
      nf *= g.fe[dd][e];
      no *= d->nx[e] + (e == dd ? 1 : 0);
    }
    if (dd >= d->ndim) nf = no = 0;
    g.foff[dd] = off;
    g.nfd[dd] = nf;
    off += nf;
    g.own_off[dd] = own;
    g.nown_d[dd] = no;
    own += no;
  }
  g.nfb = off;
  g.nown_b = own;
  long long eo = 0;
  for (int a = 0; a < 3; ++a) {
    const bool active = d->ndim == 3 || a == 2;
    long long n = active ? 1 : 0;
    for (int e = 0; e < 3; ++e) {
      g.ee[a][e] = e == a ? d->nx[e] : d->nx[e] + (e < d->ndim ? 1 : 0);
      n *= g.ee[a][e];
    }
    g.eoff[a] = eo;
    eo += n;
  }
  g.nEb = eo;
  return g;
}


bool ct_ring_map(const bhac_grid_desc* desc, const bhac_block_desc* blocks, int nb, const CtGeom& g,
                 std::vector<long long>& dst, std::vector<long long>& src) {
  const int* nr = desc->nroot;
  std::vector<int> lut((size_t)nr[0] * nr[1] * nr[2], -1);
  for (int b = 0; b < nb; ++b) lut[((size_t)blocks[b].iz * nr[1] + blocks[b].iy) * nr[0] + blocks[b].ix] = b;
  long long N[3];
  for (int e = 0; e < 3; ++e) N[e] = (long long)nr[e] * desc->nx[e];
  dst.clear();
  src.clear();
  for (int b = 0; b < nb; ++b) {
    const int bc[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    for (int d = 0; d < desc->ndim; ++d)
      for (int k = -g.fo[d][2]; k < g.fe[d][2] - g.fo[d][2]; ++k)
        for (int j = -g.fo[d][1]; j < g.fe[d][1] - g.fo[d][1]; ++j)
          for (int i = -g.fo[d][0]; i < g.fe[d][0] - g.fo[d][0]; ++i) {
            const int f[3] = {i, j, k};
            bool ring = false;
            for (int e = 0; e < 3; ++e)
              if (e != d && (f[e] < 0 || f[e] >= desc->nx[e])) ring = true;
            if (!ring) continue;
            long long G[3];
            for (int e = 0; e < 3; ++e) G[e] = (long long)bc[e] * desc->nx[e] + f[e];
            // boundary rules across the face (the along-d index is a face index and stays)
            for (int e = 0; e < desc->ndim; ++e) {
              if (e == d) continue;
              const int side = G[e] < 0 ? 0 : (G[e] >= N[e] ? 1 : -1);
              if (side < 0) continue;
              const int kind = desc->bc[e][side];
              if (kind == BHAC_BC_PERIODIC) {
                G[e] = ((G[e] % N[e]) + N[e]) % N[e];
              } else if (kind == BHAC_BC_OUTFLOW || kind == BHAC_BC_NOINFLOW) {
                G[e] = side == 0 ? 0 : N[e] - 1;
              } else {  // polar axis (x2): mirror, and phi + pi in 3-D
                G[e] = side == 0 ? -1 - G[e] : 2 * N[e] - 1 - G[e];
                if (desc->ndim == 3) G[2] = ((G[2] + N[2] / 2) % N[2] + N[2]) % N[2];
              }
            }
            if (desc->ndim == 3 && d != 2 && desc->bc[2][0] == BHAC_BC_PERIODIC) G[2] = ((G[2] % N[2]) + N[2]) % N[2];
            int ob[3], lf[3];
            for (int e = 0; e < 3; ++e) {
              if (G[e] < 0 || G[e] > N[e] || (e != d && G[e] == N[e])) return false;
              ob[e] = (int)(G[e] / desc->nx[e]);
              if (e == d && ob[e] >= nr[e]) ob[e] = nr[e] - 1;
              lf[e] = (int)(G[e] - (long long)ob[e] * desc->nx[e]);
            }
            const int o = lut[((size_t)ob[2] * nr[1] + ob[1]) * nr[0] + ob[0]];
            if (o < 0) return false;
            dst.push_back((long long)b * g.nfb + ring_index(g, d, i, j, k));
            src.push_back((long long)o * g.nfb + ring_index(g, d, lf[0], lf[1], lf[2]));
          }
  }
  return true;
}

namespace {

// Leaf blocks by (level, block coordinates): one dense table per level.
struct LeafFinder {
  std::vector<std::vector<int>> lut;
  void build(const bhac_grid_desc* d, const bhac_block_desc* blocks, int nb) {
    lut.resize(d->nlevels);
    for (int L = 0; L < d->nlevels; ++L) {
      size_t n = 1;
      for (int e = 0; e < 3; ++e) n *= (size_t)d->nroot[e] << (e < d->ndim ? L : 0);
      lut[L].assign(n, -1);
    }
    for (int b = 0; b < nb; ++b) {
      const int L = blocks[b].level;
      const size_t n0 = (size_t)d->nroot[0] << L, n1 = (size_t)d->nroot[1] << L;
      lut[L][((size_t)blocks[b].iz * n1 + blocks[b].iy) * n0 + blocks[b].ix] = b;
    }
  }
  int get(const bhac_grid_desc* d, int L, const long long bc[3]) const {
    if (L < 0 || L >= d->nlevels) return -1;
    long long n[3];
    for (int e = 0; e < 3; ++e) {
      n[e] = (long long)d->nroot[e] << (e < d->ndim ? L : 0);
      if (bc[e] < 0 || bc[e] >= n[e]) return -1;
    }
    return lut[L][(size_t)((bc[2] * n[1] + bc[1]) * n[0] + bc[0])];
  }
};

struct LevelCtx {
  const bhac_grid_desc* d;
  const CtGeom* g;
  LeafFinder leaves;
  long long ncell(int e, int L) const { return ((long long)d->nroot[e] * d->nx[e]) << (e < d->ndim ? L : 0); }
  // 0: a level-L leaf holds cell G; -1: a coarser leaf covers it; +1: finer leaves do
  int cover(int L, const long long G[3]) const {
    long long bc[3];
    for (int e = 0; e < 3; ++e) bc[e] = G[e] / d->nx[e];
    if (leaves.get(d, L, bc) >= 0) return 0;
    for (int Lc = L - 1; Lc >= 0; --Lc) {
      for (int e = 0; e < 3; ++e) bc[e] = (e < d->ndim ? G[e] >> (L - Lc) : G[e]) / d->nx[e];
      if (leaves.get(d, Lc, bc) >= 0) return -1;
    }
    return 1;
  }
  // Phi indices (ring layout, whole arena) whose mean is face G of direction dd
  // at level L (a face index along dd, cell indices across, inside the domain):
  // the face of the level-L leaf above it along dd, else below; the coarse face
  // it lies on or the two faces of the coarse cell it cuts; the finer faces on
  // it.  Returns the count (1, 2 or 4), 0 if the levels do not resolve it.
  int face_sources(int dd, int L, const long long G[3], long long src[4]) const {
    const long long Nd = ncell(dd, L);
    long long bc[3];
    int lf[3];
    for (int e = 0; e < 3; ++e)
      if (e != dd) {
        bc[e] = G[e] / d->nx[e];
        lf[e] = (int)(G[e] % d->nx[e]);
      }
    for (int above = 1; above >= 0; --above) {
      const long long cell = above ? G[dd] : G[dd] - 1;
      if (cell < 0 || cell >= Nd) continue;
      bc[dd] = cell / d->nx[dd];
      lf[dd] = (int)(G[dd] - bc[dd] * d->nx[dd]);
      const int b = leaves.get(d, L, bc);
      if (b >= 0) {
        src[0] = (long long)b * g->nfb + ring_index(*g, dd, lf[0], lf[1], lf[2]);
        return 1;
      }
    }
    long long cell[3] = {G[0], G[1], G[2]};
    if (cell[dd] >= Nd) cell[dd] = Nd - 1;
    const int cov = cover(L, cell);
    if (cov < 0 && L > 0) {
      long long H[3], H1[3];
      for (int e = 0; e < 3; ++e) H[e] = H1[e] = e < d->ndim ? G[e] >> 1 : G[e];
      if (!(G[dd] & 1)) return face_sources(dd, L - 1, H, src) == 1 ? 1 : 0;
      H1[dd] += 1;
      long long s1[4];
      if (face_sources(dd, L - 1, H, src) != 1 || face_sources(dd, L - 1, H1, s1) != 1) return 0;
      src[1] = s1[0];
      return 2;
    }
    if (cov <= 0 || L + 1 >= d->nlevels) return 0;
    int t[2], nt = 0;
    for (int e = 0; e < d->ndim; ++e)
      if (e != dd) t[nt++] = e;
    for (int q = 0; q < (1 << nt); ++q) {
      long long F[3] = {G[0], G[1], G[2]}, s1[4];
      F[dd] = 2 * G[dd];
      for (int u = 0; u < nt; ++u) F[t[u]] = 2 * G[t[u]] + ((q >> u) & 1);
      if (face_sources(dd, L + 1, F, s1) != 1) return 0;
      src[q] = s1[0];
    }
    return 1 << nt;
  }
  // cell q (0..3) around the edge along a at G (level L): across each active
  // transverse direction below (bit 0) or above (bit 1); periodic wrap; false
  // where it leaves the domain across another boundary
  bool edge_cell(int a, int L, const long long G[3], int q, long long C[3], int s[3]) const {
    int u = 0;
    for (int e = 0; e < 3; ++e) {
      C[e] = G[e];
      s[e] = 0;
      if (e == a || e >= d->ndim) continue;
      s[e] = (q >> u++) & 1;
      C[e] = G[e] - 1 + s[e];
      const long long N = ncell(e, L);
      if (C[e] < 0 || C[e] >= N) {
        if (d->bc[e][C[e] < 0 ? 0 : 1] != BHAC_BC_PERIODIC) return false;
        C[e] = ((C[e] % N) + N) % N;
      }
    }
    return true;
  }
};


// flux of variable v through face (d; i, j, k) of block b
__device__ __forceinline__ double xf_at(const CtArgs& c, int b, int d, int v, int i, int j, int k) {
  return c.xf[(long long)b * NV * c.g.nfb + NV * c.g.foff[d] + v * c.g.nfd[d] + (ring_index(c.g, d, i, j, k) - c.g.foff[d])];
}

__global__ void __launch_bounds__(256) ct_ring_kernel(const long long* __restrict__ dst, const long long* __restrict__ src,
                                                      long long n, double* phi) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    phi[dst[t]] = phi[src[t]];
}

__global__ void __launch_bounds__(256) ct_ring_mean_kernel(const long long* __restrict__ dst,
                                                           const long long* __restrict__ src, long long n,
                                                           double* phi) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    int m = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long o = src[4 * t + q];
      if (o >= 0) {
        s += phi[o];
        ++m;
      }
    }
    phi[dst[t]] = s / m;
  }
}

// Coarse fluxes on level boundaries: the mean of the finer faces' fluxes, every variable.
__global__ void __launch_bounds__(256) ct_reflux_kernel(CtArgs c) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < c.nxr;
       t += (long long)gridDim.x * blockDim.x) {
    const long long stride = c.g.nfd[c.xr_d[t]];
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      int m = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long o = c.xr_src[4 * t + q];
        if (o >= 0) {
          s += c.xf[o + v * stride];
          ++m;
        }
      }
      c.xf[c.xr_dst[t] + v * stride] = s / m;
    }
  }
}

__device__ __forceinline__ double to_t(double x, double) { return x; }
__device__ __forceinline__ float to_t(double x, float) { return narrow_f64(x); }

// Flux through face (D; i, j, k) of block b (D a compile-time direction, so
// the states stay in registers), q its index among the direction's faces; T
// the flux arithmetic (double: FP64 form; float: mixed form).
template <typename T, int D, bool FLAT>
__device__ __forceinline__ void ct_one_face(const StageArgs& a, const CtArgs& c, int b, int i, int j, int k,
                                            long long q) {
  const int L = a.blk[4 * b];
  const int G1 = a.blk[4 * b + 1] * a.nx + i, G2 = a.blk[4 * b + 2] * a.ny + j;
  const int N1 = a.N1l[L];
  T F[NV];
  const bool axis = !FLAT && D == 1 && ((G2 == 0 && c.axis_lo) || (G2 == a.N2l[L] && c.axis_hi));
  if (axis) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = T(0.0);
  } else {
    const int sd = D == 0 ? 1 : (D == 1 ? a.Nx : a.Nx * a.Ny);
    const int c0 = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);  // the cell above the face
    const T* Pb = (sizeof(T) == 8 ? reinterpret_cast<const T*>(a.P_in) : reinterpret_cast<const T*>(a.P32_in)) +
                  (size_t)b * NV * a.ncell;
    T PL[NV], PR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* p = Pb + (size_t)v * a.ncell + c0;
      recon_var(a.recon, p[-3 * sd], p[-2 * sd], p[-sd], p[0], p[sd], p[2 * sd], PL[v], PR[v]);
    }
    positivity_fallback(a, Pb, sd, c0, PL, PR);
    Met<T> m;
    T acg = T(1.0);
    if (FLAT) {
      m = flat_metric<T>();
    } else if (D == 0) {
      const size_t r = ((size_t)c.teo_f1[L] + (size_t)(G2 + 1) * (N1 + 3) + (G1 + 1)) * FREC;
      if (sizeof(T) == 8) {
        m = load_face_metric<T>(c.te_f1 + r);
        acg = T(c.te_f1[r + F_ACG]);
      } else {
        m = load_face_metric<T>(c.te_f1_32 + r);
        acg = T(c.te_f1_32[r + F_ACG]);
      }
    } else if (D == 1) {
      const size_t r = ((size_t)c.teo_f2[L] + (size_t)(G2 + 1) * (N1 + 2) + (G1 + 1)) * FREC;
      if (sizeof(T) == 8) {
        m = load_face_metric<T>(c.te_f2 + r);
        acg = T(c.te_f2[r + F_ACG]);
      } else {
        m = load_face_metric<T>(c.te_f2_32 + r);
        acg = T(c.te_f2_32[r + F_ACG]);
      }
    } else {
      const size_t r = ((size_t)c.teo_c[L] + (size_t)(G2 + 1) * (N1 + 2) + (G1 + 1)) * CREC;
      if (sizeof(T) == 8) {
        m = load_centre_metric<T>(c.te_c + r);
        acg = T(c.te_c[r + C_ACG3]);
      } else {
        m = load_centre_metric<T>(c.te_c32 + r);
        acg = T(c.te_c32[r + C_ACG3]);
      }
    }
    const T Bn = to_t(c.phi_in[(long long)b * c.g.nfb + ring_index(c.g, D, i, j, k)], T(0)) / m.sg;
    PL[B1 + D] = Bn;
    PR[B1 + D] = Bn;
    riemann_flux(m, acg, PL, PR, D, a.riemann, pick<T>(a.gam, a.gam_f), pick<T>(a.gam_fac, a.gam_fac_f), T(0.0), F);
  }
  const long long o = (long long)b * NV * c.g.nfb + NV * c.g.foff[D] + q;
#pragma unroll
  for (int v = 0; v < NV; ++v) c.xf[o + v * c.g.nfd[D]] = to_double(F[v]);
}

// Fluxes through every face of every block and its ring, one thread per face.
template <typename T, bool FLAT>
__global__ void __launch_bounds__(256) ct_flux_kernel(StageArgs a, CtArgs c) {
  // 32-bit index arithmetic: bhac_init_grid keeps blocks x ring-extended faces below 2^31
  const unsigned n = (unsigned)a.nblocks * (unsigned)c.g.nfb;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)c.g.nfb);
    const int r = (int)(t - (unsigned)b * (unsigned)c.g.nfb);
    const int d = (c.g.ndim == 3 && r >= c.g.foff[2]) ? 2 : (r >= c.g.foff[1] ? 1 : 0);
    const int q = r - (int)c.g.foff[d];
    const int e0 = c.g.fe[d][0], e1 = c.g.fe[d][1];
    const int i = q % e0 - c.g.fo[d][0];
    const int j = (q / e0) % e1 - c.g.fo[d][1];
    const int k = q / (e0 * e1) - c.g.fo[d][2];
    if (d == 0)
      ct_one_face<T, 0, FLAT>(a, c, b, i, j, k, q);
    else if (d == 1)
      ct_one_face<T, 1, FLAT>(a, c, b, i, j, k, q);
    else
      ct_one_face<T, 2, FLAT>(a, c, b, i, j, k, q);
  }
}

// Edge EMFs: E_3 at (i-1/2, j-1/2) of cell layer k, E_1 at (j-1/2, k-1/2) of
// column i, E_2 at (k-1/2, i-1/2) of row j.
__device__ __forceinline__ double emf3(const CtArgs& c, int b, int i, int j, int k) {
  return 0.25 * (xf_at(c, b, 1, B1, i, j, k) + xf_at(c, b, 1, B1, i - 1, j, k) - xf_at(c, b, 0, B2, i, j, k) -
                 xf_at(c, b, 0, B2, i, j - 1, k));
}
__device__ __forceinline__ double emf1(const CtArgs& c, int b, int i, int j, int k) {
  return 0.25 * (xf_at(c, b, 2, B2, i, j, k) + xf_at(c, b, 2, B2, i, j - 1, k) - xf_at(c, b, 1, B3, i, j, k) -
                 xf_at(c, b, 1, B3, i, j, k - 1));
}
__device__ __forceinline__ double emf2(const CtArgs& c, int b, int i, int j, int k) {
  return 0.25 * (xf_at(c, b, 0, B3, i, j, k) + xf_at(c, b, 0, B3, i, j, k - 1) - xf_at(c, b, 2, B1, i, j, k) -
                 xf_at(c, b, 2, B1, i - 1, j, k));
}


// d_t Phi = -curl E and the stage combination, one thread per owned face.
template <int DIM>
__global__ void __launch_bounds__(256) ct_face_kernel(StageArgs a, CtArgs c) {
  const double dt = stage_dt(a);
  const unsigned n = (unsigned)a.nblocks * (unsigned)c.g.nown_b;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)c.g.nown_b);
    int d, i, j, k;
    owned_face(c.g, (int)(t - (unsigned)b * (unsigned)c.g.nown_b), d, i, j, k);
    const long long o = (long long)b * c.g.nfb + ring_index(c.g, d, i, j, k);
    const int G2 = a.blk[4 * b + 2] * a.ny + j;
    if (!a.flat && d == 1 && ((G2 == 0 && c.axis_lo) || (G2 == a.N2g && c.axis_hi))) {
      c.phi_out[o] = 0.0;  // sqrt(gamma) = 0 on the axis
      continue;
    }
    double R;
    if (d == 0) {
      R = -(emf3(c, b, i, j + 1, k) - emf3(c, b, i, j, k)) * a.idx[1];
      if (DIM == 3) R += (emf2(c, b, i, j, k + 1) - emf2(c, b, i, j, k)) * a.idx[2];
    } else if (d == 1) {
      R = (emf3(c, b, i + 1, j, k) - emf3(c, b, i, j, k)) * a.idx[0];
      if (DIM == 3) R -= (emf1(c, b, i, j, k + 1) - emf1(c, b, i, j, k)) * a.idx[2];
    } else {
      R = -(emf2(c, b, i + 1, j, k) - emf2(c, b, i, j, k)) * a.idx[0] +
          (emf1(c, b, i, j + 1, k) - emf1(c, b, i, j, k)) * a.idx[1];
    }
    if (a.stage == 1)
      c.phi_out[o] = c.phi_in[o] + dt * R;
    else
      c.phi_out[o] = 0.5 * c.phi_n[o] + 0.5 * (c.phi_in[o] + dt * R);
  }
}

// Every edge EMF of every block into c.emf (grids with refinement levels).
__global__ void __launch_bounds__(256) ct_emf_kernel(StageArgs a, CtArgs c) {
  const unsigned n = (unsigned)a.nblocks * (unsigned)c.g.nEb;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)c.g.nEb);
    const int r = (int)(t - (unsigned)b * (unsigned)c.g.nEb);
    const int e = r >= c.g.eoff[2] ? 2 : (r >= c.g.eoff[1] ? 1 : 0);
    const int q = r - (int)c.g.eoff[e];
    const int i = q % c.g.ee[e][0], j = (q / c.g.ee[e][0]) % c.g.ee[e][1], k = q / (c.g.ee[e][0] * c.g.ee[e][1]);
    c.emf[t] = e == 0 ? emf1(c, b, i, j, k) : (e == 1 ? emf2(c, b, i, j, k) : emf3(c, b, i, j, k));
  }
}

// Edges that a finer leaf touches: the mean of the finer EMFs along them (the
// finer entries are never corrected themselves, so the order does not matter).
__global__ void __launch_bounds__(256) ct_emf_fix_kernel(CtArgs c) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < c.nef;
       t += (long long)gridDim.x * blockDim.x) {
    const long long s1 = c.ef_src[2 * t + 1];
    const double e0 = c.emf[c.ef_src[2 * t]];
    c.emf[c.ef_dst[t]] = s1 >= 0 ? (e0 + c.emf[s1]) / 2.0 : e0;
  }
}

__device__ __forceinline__ double emf_at(const CtArgs& c, int b, int e, int i, int j, int k) {
  return c.emf[(long long)b * c.g.nEb + c.g.eoff[e] + ((long long)k * c.g.ee[e][1] + j) * c.g.ee[e][0] + i];
}

// d_t Phi = -curl E from the stored (corrected) EMFs with the block's level
// spacing, and the stage combination, one thread per owned face.
template <int DIM>
__global__ void __launch_bounds__(256) ct_face_level_kernel(StageArgs a, CtArgs c) {
  const double dt = stage_dt(a);
  const unsigned n = (unsigned)a.nblocks * (unsigned)c.g.nown_b;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)c.g.nown_b);
    int d, i, j, k;
    owned_face(c.g, (int)(t - (unsigned)b * (unsigned)c.g.nown_b), d, i, j, k);
    const long long o = (long long)b * c.g.nfb + ring_index(c.g, d, i, j, k);
    const int L = a.blk[4 * b];
    const int G2 = a.blk[4 * b + 2] * a.ny + j;
    if (!a.flat && d == 1 && ((G2 == 0 && c.axis_lo) || (G2 == a.N2l[L] && c.axis_hi))) {
      c.phi_out[o] = 0.0;  // sqrt(gamma) = 0 on the axis
      continue;
    }
    const double s = (double)(1 << L);
    const double ix = a.idx[0] * s, iy = a.idx[1] * s, iz = DIM == 3 ? a.idx[2] * s : a.idx[2];
    double R;
    if (d == 0) {
      R = -(emf_at(c, b, 2, i, j + 1, k) - emf_at(c, b, 2, i, j, k)) * iy;
      if (DIM == 3) R += (emf_at(c, b, 1, i, j, k + 1) - emf_at(c, b, 1, i, j, k)) * iz;
    } else if (d == 1) {
      R = (emf_at(c, b, 2, i + 1, j, k) - emf_at(c, b, 2, i, j, k)) * ix;
      if (DIM == 3) R -= (emf_at(c, b, 0, i, j, k + 1) - emf_at(c, b, 0, i, j, k)) * iz;
    } else {
      R = -(emf_at(c, b, 1, i + 1, j, k) - emf_at(c, b, 1, i, j, k)) * ix +
          (emf_at(c, b, 0, i, j + 1, k) - emf_at(c, b, 0, i, j, k)) * iy;
    }
    if (a.stage == 1)
      c.phi_out[o] = c.phi_in[o] + dt * R;
    else
      c.phi_out[o] = 0.5 * c.phi_n[o] + 0.5 * (c.phi_in[o] + dt * R);
  }
}

// Flux divergence, sources, RK combination, the cell field from the updated
// faces, then the stage kernel's inversion, floors, outputs and CFL rate.  T:
// the arithmetic of the sources (float in the mixed form, from the FP32
// primitives and metric records).  Two CTAs per SM as the register bound (a
// few spilled values; the mixed form's stage 2.5% faster than at one CTA).
template <typename T, int DIM, bool FLAT>
__global__ void __launch_bounds__(256, 2) ct_cell_kernel(StageArgs a, CtArgs c) {
  const double dt = stage_dt(a);
  if (a.stage == 1 && blockIdx.x == 0 && threadIdx.x == 0) *a.dt_dev = dt;
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const unsigned n = (unsigned)a.nblocks * (unsigned)a.nint;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)a.nint);
    const LevelGeo geo = level_geo(a, a.blk[4 * b]);
    const int ci = (int)(t - (unsigned)b * (unsigned)a.nint);
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
    double rhs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) rhs[v] = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int ih = i + (d == 0), jh = j + (d == 1), kh = k + (d == 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) rhs[v] += -(xf_at(c, b, d, v, ih, jh, kh) - xf_at(c, b, d, v, i, j, k)) * geo.idx[d];
    }
    if (!FLAT) {
      const T* crec = (sizeof(T) == 8 ? reinterpret_cast<const T*>(geo.tc) : reinterpret_cast<const T*>(geo.tc32)) +
                      (size_t)(I2 * geo.N1 + I1) * CREC;
      const T* Pin = sizeof(T) == 8 ? reinterpret_cast<const T*>(a.P_in) : reinterpret_cast<const T*>(a.P32_in);
      T Pc[NV], Uc[NV], S[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Pc[v] = Pin[(size_t)b * NV * a.ncell + (size_t)v * a.ncell + cg];
      const Met<T> m = load_centre_metric<T>(crec);
      Derived<T> s;
      derive(m, Pc, pick<T>(a.gam_fac, a.gam_fac_f), s);
      cons_of(Pc, s, Uc);
      sources_of(m, crec, Pc, s, Uc, T(0.0), T(0.0), S);
      const T sg = crec[C_SG];
#pragma unroll
      for (int v = 0; v < NV; ++v) rhs[v] += to_double(sg * S[v]);
    }
    const size_t ub = (size_t)b * NV * a.nint + ci;
    double U[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double un = a.Un[ub + (size_t)v * a.nint];
      U[v] = a.stage == 1 ? un + dt * rhs[v] : 0.5 * un + 0.5 * (a.U1[ub + (size_t)v * a.nint] + dt * rhs[v]);
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const long long lo = (long long)b * c.g.nfb + ring_index(c.g, d, i, j, k);
      const long long hi = (long long)b * c.g.nfb + ring_index(c.g, d, i + (d == 0), j + (d == 1), k + (d == 2));
      U[B1 + d] = 0.5 * (c.phi_out[lo] + c.phi_out[hi]);
    }
    U[PSI] = 0.0;
    finish_cell<T, DIM, FLAT>(a, geo, b, ci, cg, I1, I2, U, cnt, rate_max);
  }
  reduce_outputs(a, cnt, rate_max);
}

// The cell field of the loaded state from its faces.
template <int DIM>
__global__ void __launch_bounds__(256) ct_cell_field_kernel(StageArgs a, CtArgs c, double* P, float* P32) {
  const long long n = (long long)a.nblocks * a.nint;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / a.nint);
    const int ci = (int)(t - (long long)b * a.nint);
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    double sg = 1.0;
    if (!a.flat) {
      const int L = a.blk[4 * b];
      const int I1 = a.blk[4 * b + 1] * a.nx + i, I2 = a.blk[4 * b + 2] * a.ny + j;
      sg = a.tab_c[((size_t)a.toff_c[L] + (size_t)I2 * a.N1l[L] + I1) * CREC + C_SG];
    }
    double* Pc = P + (size_t)b * NV * a.ncell + cg;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const long long lo = (long long)b * c.g.nfb + ring_index(c.g, d, i, j, k);
      const long long hi = (long long)b * c.g.nfb + ring_index(c.g, d, i + (d == 0), j + (d == 1), k + (d == 2));
      Pc[(size_t)(B1 + d) * a.ncell] = 0.5 * (c.phi_in[lo] + c.phi_in[hi]) / sg;
      if (P32) P32[(size_t)b * NV * a.ncell + cg + (size_t)(B1 + d) * a.ncell] = narrow_f64(Pc[(size_t)(B1 + d) * a.ncell]);
    }
    Pc[(size_t)PSI * a.ncell] = 0.0;
    if (P32) P32[(size_t)b * NV * a.ncell + cg + (size_t)PSI * a.ncell] = 0.0f;
  }
}

__global__ void __launch_bounds__(256) ct_copy_kernel(int nblocks, CtGeom g, const double* __restrict__ src, double* dst,
                                                      int to_ring) {
  const long long n = (long long)nblocks * g.nown_b;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / g.nown_b);
    int d, i, j, k;
    owned_face(g, (int)(t - (long long)b * g.nown_b), d, i, j, k);
    const long long o = (long long)b * g.nfb + ring_index(g, d, i, j, k);
    if (to_ring)
      dst[o] = src[t];
    else
      dst[t] = src[o];
  }
}

int grid_of(long long n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long g = (n + 255) / 256;
  const long long cap = 32LL * nsm;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

CtLevelMaps ct_level_maps(const bhac_grid_desc* d, const bhac_block_desc* blocks, int nb, const CtGeom& g) {
  CtLevelMaps M;
  M.ok = false;
  LevelCtx X;
  X.d = d;
  X.g = &g;
  X.leaves.build(d, blocks, nb);
  const int* nx = d->nx;
  // ring faces: the boundary rules across (at the block's level), then the
  // sources; blocks in contiguous ranges on host threads, joined in order
  struct RingOut {
    std::vector<long long> copy_dst, copy_src, mean_dst, mean_src;
    bool ok = true;
  };
  auto ring_block = [&](int b, RingOut& R) {
    const int L = blocks[b].level;
    const long long bo[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    long long N[3];
    for (int e = 0; e < 3; ++e) N[e] = X.ncell(e, L);
    for (int dd = 0; dd < d->ndim; ++dd)
      for (int k = -g.fo[dd][2]; k < g.fe[dd][2] - g.fo[dd][2]; ++k)
        for (int j = -g.fo[dd][1]; j < g.fe[dd][1] - g.fo[dd][1]; ++j)
          for (int i = -g.fo[dd][0]; i < g.fe[dd][0] - g.fo[dd][0]; ++i) {
            const int f[3] = {i, j, k};
            bool ring = false;
            for (int e = 0; e < 3; ++e)
              if (e != dd && (f[e] < 0 || f[e] >= nx[e])) ring = true;
            if (!ring) continue;
            long long G[3];
            for (int e = 0; e < 3; ++e) G[e] = bo[e] * nx[e] + f[e];
            for (int e = 0; e < d->ndim; ++e) {
              if (e == dd) continue;
              const int side = G[e] < 0 ? 0 : (G[e] >= N[e] ? 1 : -1);
              if (side < 0) continue;
              const int kind = d->bc[e][side];
              if (kind == BHAC_BC_PERIODIC) {
                G[e] = ((G[e] % N[e]) + N[e]) % N[e];
              } else if (kind == BHAC_BC_OUTFLOW || kind == BHAC_BC_NOINFLOW) {
                G[e] = side == 0 ? 0 : N[e] - 1;
              } else {  // polar axis (x2): mirror, and phi + pi in 3-D
                G[e] = side == 0 ? -1 - G[e] : 2 * N[e] - 1 - G[e];
                if (d->ndim == 3) G[2] = ((G[2] + N[2] / 2) % N[2] + N[2]) % N[2];
              }
            }
            if (d->ndim == 3 && dd != 2 && d->bc[2][0] == BHAC_BC_PERIODIC) G[2] = ((G[2] % N[2]) + N[2]) % N[2];
            for (int e = 0; e < 3; ++e)
              if (G[e] < 0 || G[e] > N[e] || (e != dd && G[e] == N[e])) {
                R.ok = false;
                return;
              }
            long long src[4];
            const int n = X.face_sources(dd, L, G, src);
            if (n == 0) {
              R.ok = false;
              return;
            }
            const long long dst = (long long)b * g.nfb + ring_index(g, dd, i, j, k);
            if (n == 1) {
              R.copy_dst.push_back(dst);
              R.copy_src.push_back(src[0]);
            } else {
              R.mean_dst.push_back(dst);
              for (int q = 0; q < 4; ++q) R.mean_src.push_back(q < n ? src[q] : -1);
            }
          }
  };
  {
    const int nt = std::max(1, std::min(16, std::min(nb / 64, (int)std::thread::hardware_concurrency())));
    std::vector<RingOut> part(nt);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
      pool.emplace_back([&, t] {
        for (int b = (int)((long long)nb * t / nt); b < (int)((long long)nb * (t + 1) / nt) && part[t].ok; ++b)
          ring_block(b, part[t]);
      });
    for (auto& th : pool) th.join();
    for (const RingOut& R : part) {
      if (!R.ok) return M;
      M.copy_dst.insert(M.copy_dst.end(), R.copy_dst.begin(), R.copy_dst.end());
      M.copy_src.insert(M.copy_src.end(), R.copy_src.begin(), R.copy_src.end());
      M.mean_dst.insert(M.mean_dst.end(), R.mean_dst.begin(), R.mean_dst.end());
      M.mean_src.insert(M.mean_src.end(), R.mean_src.begin(), R.mean_src.end());
    }
  }
  // coarse fluxes on level boundaries: the mean of the finer ones (the finer
  // faces in the order: first transverse direction (d + 1) % 3 outer, (d + 2) % 3 inner)
  auto xf_index = [&](int b, int dd, int i, int j, int k) {
    return (long long)b * NV * g.nfb + NV * g.foff[dd] + (ring_index(g, dd, i, j, k) - g.foff[dd]);
  };
  for (int b = 0; b < nb; ++b) {
    const int L = blocks[b].level;
    const long long bo[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    for (int dd = 0; dd < d->ndim; ++dd)
      for (int side = 0; side < 2; ++side) {
        long long nbc[3] = {bo[0], bo[1], bo[2]};
        nbc[dd] += side == 0 ? -1 : 1;
        const long long nbd = (long long)d->nroot[dd] << L;
        if (nbc[dd] < 0 || nbc[dd] >= nbd) {
          if (d->bc[dd][side] != BHAC_BC_PERIODIC) continue;
          nbc[dd] = (nbc[dd] + nbd) % nbd;
        }
        if (X.leaves.get(d, L, nbc) >= 0) continue;
        long long chb[3];
        for (int e = 0; e < 3; ++e) chb[e] = e < d->ndim ? 2 * nbc[e] : nbc[e];
        if (side == 0) chb[dd] += 1;
        if (X.leaves.get(d, L + 1, chb) < 0) continue;
        const int t1 = (dd + 1) % 3, t2 = (dd + 2) % 3;
        const int fcoarse = side == 0 ? 0 : nx[dd], ffine = side == 0 ? nx[dd] : 0;
        for (int a = 0; a < nx[t1]; ++a)
          for (int bb = 0; bb < nx[t2]; ++bb) {
            long long src[4] = {-1, -1, -1, -1};
            int cnt = 0;
            for (int s1 = 0; s1 < (t1 < d->ndim ? 2 : 1); ++s1)
              for (int s2 = 0; s2 < (t2 < d->ndim ? 2 : 1); ++s2) {
                const long long gc1 = bo[t1] * nx[t1] + a, gc2 = bo[t2] * nx[t2] + bb;
                const long long Gf1 = t1 < d->ndim ? 2 * gc1 + s1 : gc1, Gf2 = t2 < d->ndim ? 2 * gc2 + s2 : gc2;
                long long fb[3];
                fb[dd] = chb[dd];
                fb[t1] = Gf1 / nx[t1];
                fb[t2] = Gf2 / nx[t2];
                const int bf = X.leaves.get(d, L + 1, fb);
                if (bf < 0) continue;
                int li[3];
                li[dd] = ffine;
                li[t1] = (int)(Gf1 % nx[t1]);
                li[t2] = (int)(Gf2 % nx[t2]);
                src[cnt++] = xf_index(bf, dd, li[0], li[1], li[2]);
              }
            if (cnt == 0) continue;
            int lc[3];
            lc[dd] = fcoarse;
            lc[t1] = a;
            lc[t2] = bb;
            M.xr_dst.push_back(xf_index(b, dd, lc[0], lc[1], lc[2]));
            for (int q = 0; q < 4; ++q) M.xr_src.push_back(src[q]);
            M.xr_d.push_back(dd);
          }
      }
  }
  // EMFs of edges that a finer leaf touches: the mean of the finer EMFs along them
  for (int b = 0; b < nb; ++b) {
    const int L = blocks[b].level;
    const long long bo[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    for (int a = 0; a < 3; ++a) {
      if (!(d->ndim == 3 || a == 2)) continue;
      const int* ee = g.ee[a];
      for (int k = 0; k < ee[2]; ++k)
        for (int j = 0; j < ee[1]; ++j)
          for (int i = 0; i < ee[0]; ++i) {
            const int loc[3] = {i, j, k};
            bool inner = true;  // all four cells around the edge are the block's own
            for (int e = 0; e < d->ndim; ++e)
              if (e != a && (loc[e] == 0 || loc[e] == nx[e])) inner = false;
            if (inner) continue;
            long long G[3], C[3];
            int sgn[3];
            for (int e = 0; e < 3; ++e) G[e] = bo[e] * nx[e] + loc[e];
            bool finer = false;
            for (int q = 0; q < 4 && !finer; ++q)
              if (X.edge_cell(a, L, G, q, C, sgn) && X.cover(L, C) > 0) finer = true;
            if (!finer || L + 1 >= d->nlevels) continue;
            const int na = a < d->ndim ? 2 : 1;
            long long src[2] = {-1, -1};
            int n = 0;
            for (int t = 0; t < na; ++t) {
              long long F[3];
              for (int e = 0; e < 3; ++e) F[e] = e >= d->ndim ? G[e] : 2 * G[e] + (e == a ? t : 0);
              for (int q = 0; q < 4; ++q) {
                if (!X.edge_cell(a, L + 1, F, q, C, sgn)) continue;
                long long bc[3];
                for (int e = 0; e < 3; ++e) bc[e] = C[e] / nx[e];
                const int bf = X.leaves.get(d, L + 1, bc);
                if (bf < 0) continue;
                int lf[3];
                for (int e = 0; e < 3; ++e)
                  lf[e] = (int)(C[e] - bc[e] * nx[e]) + (e != a && e < d->ndim && !sgn[e] ? 1 : 0);
                src[n++] = (long long)bf * g.nEb + g.eoff[a] + ((long long)lf[2] * g.ee[a][1] + lf[1]) * g.ee[a][0] + lf[0];
                break;
              }
            }
            if (n != na) continue;
            M.ef_dst.push_back((long long)b * g.nEb + g.eoff[a] + ((long long)k * ee[1] + j) * ee[0] + i);
            M.ef_src.push_back(src[0]);
            M.ef_src.push_back(src[1]);
          }
    }
  }
  M.ok = true;
  return M;
}

}  // namespace bhac

// Host self-check of the constrained-transport ring maps (test utility).
extern "C" bhac_status bhac_ct_ring_faces_host(const bhac_grid_desc* d, const bhac_block_desc* b, int nb,
                                               const double* owned, double* ring) {
  using namespace bhac;
  if (!d || !b || !owned || !ring || nb <= 0 || d->divb != BHAC_DIVB_CT || d->ndim < 2 || d->ndim > 3 ||
      d->nlevels < 1 || d->nlevels > MAXLEV)
    return BHAC_ERR_ARG;
  const CtGeom g = ct_geom(d);
  std::vector<long long> cd, cs, md, ms;
  if (d->nlevels == 1) {
    if (!ct_ring_map(d, b, nb, g, cd, cs)) return BHAC_ERR_ARG;
  } else {
    CtLevelMaps M = ct_level_maps(d, b, nb, g);
    if (!M.ok) return BHAC_ERR_ARG;
    cd.swap(M.copy_dst);
    cs.swap(M.copy_src);
    md.swap(M.mean_dst);
    ms.swap(M.mean_src);
  }
  for (long long t = 0; t < (long long)nb * g.nfb; ++t) ring[t] = 0.0;
  for (int q = 0; q < nb; ++q)
    for (long long r = 0; r < g.nown_b; ++r) {
      int dd, i, j, k;
      owned_face(g, (int)r, dd, i, j, k);
      ring[(long long)q * g.nfb + ring_index(g, dd, i, j, k)] = owned[(long long)q * g.nown_b + r];
    }
  for (size_t t = 0; t < cd.size(); ++t) ring[cd[t]] = ring[cs[t]];
  for (size_t t = 0; t < md.size(); ++t) {
    double s = 0.0;
    int m = 0;
    for (int q = 0; q < 4; ++q)
      if (ms[4 * t + q] >= 0) {
        s += ring[ms[4 * t + q]];
        ++m;
      }
    ring[md[t]] = s / m;
  }
  return BHAC_OK;
}

namespace bhac {

cudaError_t launch_ct_ring(const long long* dst, const long long* src, long long n, double* phi, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ct_ring_kernel<<<grid_of(n), 256, 0, st>>>(dst, src, n, phi);
  return cudaGetLastError();
}

cudaError_t launch_ct_ring_mean(const long long* dst, const long long* src, long long n, double* phi,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ct_ring_mean_kernel<<<grid_of(n), 256, 0, st>>>(dst, src, n, phi);
  return cudaGetLastError();
}

cudaError_t launch_ct_stage(const StageArgs& a, const CtArgs& c, bool mixed, cudaStream_t st) {
  const long long nf = (long long)a.nblocks * c.g.nfb, no = (long long)a.nblocks * c.g.nown_b,
                  nc = (long long)a.nblocks * a.nint;
  if (mixed) {
    if (a.flat)
      ct_flux_kernel<float, true><<<grid_of(nf), 256, 0, st>>>(a, c);
    else
      ct_flux_kernel<float, false><<<grid_of(nf), 256, 0, st>>>(a, c);
  } else {
    if (a.flat)
      ct_flux_kernel<double, true><<<grid_of(nf), 256, 0, st>>>(a, c);
    else
      ct_flux_kernel<double, false><<<grid_of(nf), 256, 0, st>>>(a, c);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c.amr) {
    // refinement levels: coarse fluxes corrected, every EMF stored and the
    // touched coarse ones corrected, then the face update from them
    if (c.nxr > 0) ct_reflux_kernel<<<grid_of(c.nxr), 256, 0, st>>>(c);
    ct_emf_kernel<<<grid_of((long long)a.nblocks * c.g.nEb), 256, 0, st>>>(a, c);
    if (c.nef > 0) ct_emf_fix_kernel<<<grid_of(c.nef), 256, 0, st>>>(c);
    if (a.ndim == 3)
      ct_face_level_kernel<3><<<grid_of(no), 256, 0, st>>>(a, c);
    else
      ct_face_level_kernel<2><<<grid_of(no), 256, 0, st>>>(a, c);
  } else if (a.ndim == 3) {
    ct_face_kernel<3><<<grid_of(no), 256, 0, st>>>(a, c);
  } else {
    ct_face_kernel<2><<<grid_of(no), 256, 0, st>>>(a, c);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mixed) {
    if (a.ndim == 3)
      a.flat ? ct_cell_kernel<float, 3, true><<<grid_of(nc), 256, 0, st>>>(a, c)
             : ct_cell_kernel<float, 3, false><<<grid_of(nc), 256, 0, st>>>(a, c);
    else
      a.flat ? ct_cell_kernel<float, 2, true><<<grid_of(nc), 256, 0, st>>>(a, c)
             : ct_cell_kernel<float, 2, false><<<grid_of(nc), 256, 0, st>>>(a, c);
  } else {
    if (a.ndim == 3)
      a.flat ? ct_cell_kernel<double, 3, true><<<grid_of(nc), 256, 0, st>>>(a, c)
             : ct_cell_kernel<double, 3, false><<<grid_of(nc), 256, 0, st>>>(a, c);
    else
      a.flat ? ct_cell_kernel<double, 2, true><<<grid_of(nc), 256, 0, st>>>(a, c)
             : ct_cell_kernel<double, 2, false><<<grid_of(nc), 256, 0, st>>>(a, c);
  }
  return cudaGetLastError();
}

cudaError_t launch_ct_cell_field(const StageArgs& a, const CtArgs& c, double* P, float* P32, cudaStream_t st) {
  const long long nc = (long long)a.nblocks * a.nint;
  if (a.ndim == 3)
    ct_cell_field_kernel<3><<<grid_of(nc), 256, 0, st>>>(a, c, P, P32);
  else
    ct_cell_field_kernel<2><<<grid_of(nc), 256, 0, st>>>(a, c, P, P32);
  return cudaGetLastError();
}

cudaError_t launch_ct_copy_faces(const StageArgs& a, const CtGeom& g, const double* src, double* dst, int to_ring,
                                 cudaStream_t st) {
  ct_copy_kernel<<<grid_of((long long)a.nblocks * g.nown_b), 256, 0, st>>>(a.nblocks, g, src, dst, to_ring);
  return cudaGetLastError();
}

}  // namespace bhac
