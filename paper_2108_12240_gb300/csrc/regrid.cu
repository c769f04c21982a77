// AMR regridding of the block grid (the paper's Sec. 2 block-based tree AMR,
// and its closing outlook on AMR runs): a refinement estimator on the device,
// the new leaf list on the host (thresholds, 2:1 balance, sibling-group
// coarsening), and the conservative transfer of the state to a context built
// for the new leaves, on the device.
//
// Estimator: Loehner's normalised second difference of the density (the
// default of the MPI-AMRVAC toolkit the method is built on), combined over
// the active directions, E = sqrt(sum_d N_d^2 / sum_d D_d^2),
//   N_d = u_+ - 2 u_0 + u_-,  D_d = |u_+ - u_0| + |u_0 - u_-| + eps (|u_+| + 2|u_0| + |u_-|),
// maximum per block.  Transfer of the densitized conserved state: a kept block
// is copied; a new child takes its parent cell's value plus minmod-limited
// slopes (within the parent block; zero at its faces) times +-1/4; a new parent
// takes the mean of its 2^d children.  Sums of sqrt(gamma) U dV are unchanged.
// Every new cell is then inverted with floors, as after a stage.
//
// With constrained transport the face fields are transferred first: a kept
// block's faces are copied; a changed block's face on its boundary that an old
// leaf of the same level held keeps that value; a coarsened block's faces are
// the mean of the old finer faces on them; a refined block's faces on the
// planes of its parent's faces are the parent face plus +-1/4 of its
// minmod-limited differences to the neighbouring parent faces across (within
// the parent; one-sided at its edge), which keeps the parent face's flux, and
// the faces inside a parent cell complete the 2^d finer cells divergence-free
// with the least change from the mean of the two outer faces at the same
// place: the change is -A^T y with A the finer cells' divergence operator and
// y solving (A A^T) y = r (r the divergences before the change); A A^T is the
// weighted Laplacian of the cube graph of the finer cells, whose eigenvectors
// are the Walsh functions, so y comes in closed form.  The cells' field is
// then the mean of their faces.
#include <algorithm>
#include <array>
#include <map>
#include <vector>

#include "ct.h"
#include "ctx.h"
#include "stage_impl.cuh"

namespace bhac {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) estimate_kernel(StageArgs a, const T* __restrict__ P, double eps, double* out) {
  __shared__ double red[8];
  const int b = blockIdx.x;
  const T* Pr = P + (size_t)b * NV * a.ncell;  // density is variable 0
  const int sd[3] = {1, a.Nx, a.Nx * a.Ny};
  double emax = 0.0;
  for (int ci = threadIdx.x; ci < a.nint; ci += blockDim.x) {
    const int i = ci % a.nx, j = (ci / a.nx) % a.ny, k = ci / (a.nx * a.ny);
    const int cg = ((k + a.gz) * a.Ny + (j + a.gy)) * a.Nx + (i + a.gx);
    const double u0 = (double)Pr[cg];
    double num2 = 0.0, den2 = 0.0;
    for (int d = 0; d < a.ndim; ++d) {
      const double um = (double)Pr[cg - sd[d]], up = (double)Pr[cg + sd[d]];
      const double n = up - 2.0 * u0 + um;
      const double dd = fabs(up - u0) + fabs(u0 - um) + eps * (fabs(up) + 2.0 * fabs(u0) + fabs(um));
      num2 += n * n;
      den2 += dd * dd;
    }
    const double e = den2 > 0.0 ? sqrt(num2 / den2) : 0.0;
    emax = fmax(emax, e);
  }
  emax = warp_max_d(emax);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    out[b] = m;
  }
}

// Per new block: [0] kind (0 copy, 1 prolong, 2 restrict), [1] the old block
// (copy, prolong), [2 + s] the old child whose offset bits along the active
// dimensions are s (restrict), [10 + 2 d + side] the old leaf of the block's
// level across its low (side 0) / high (side 1) face normal to d, or -1.
constexpr int kMapStride = 16;

struct TransferArgs {
  const int* map;
  const double* U_old;   // densitized, interior, old blocks
  const double* P_old;   // ghosted FP64 primitives of the old blocks
  const double* phi;     // constrained transport: the new face fields (else null)
  CtGeom g;
};

// The face fields of every new block except those inside refined parents'
// cells, one thread per owned face.
template <int DIM>
__global__ void __launch_bounds__(256) face_transfer_kernel(StageArgs a, const int* __restrict__ map, CtGeom g,
                                                           const double* __restrict__ phi_old, double* phi) {
  const unsigned n = (unsigned)a.nblocks * (unsigned)g.nown_b;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / (unsigned)g.nown_b);
    int d, f[3];
    owned_face(g, (int)(t - (unsigned)b * (unsigned)g.nown_b), d, f[0], f[1], f[2]);
    const int* m = map + (size_t)b * kMapStride;
    const int nxd[3] = {a.nx, a.ny, a.nz};
    const int bc[3] = {a.blk[4 * b + 1], a.blk[4 * b + 2], a.blk[4 * b + 3]};
    double* dst = phi + (long long)b * g.nfb + ring_index(g, d, f[0], f[1], f[2]);
    if (m[0] == 0) {
      *dst = phi_old[(long long)m[1] * g.nfb + ring_index(g, d, f[0], f[1], f[2])];
      continue;
    }
    if (f[d] == 0 || f[d] == nxd[d]) {
      const int across = m[10 + 2 * d + (f[d] == 0 ? 0 : 1)];
      if (across >= 0) {
        int o[3] = {f[0], f[1], f[2]};
        o[d] = f[d] == 0 ? nxd[d] : 0;
        *dst = phi_old[(long long)across * g.nfb + ring_index(g, d, o[0], o[1], o[2])];
        continue;
      }
    }
    int G[3];
    for (int e = 0; e < 3; ++e) G[e] = bc[e] * nxd[e] + f[e];
    if (m[0] == 2) {
      // the mean of the old finer faces on it, first transverse direction the low bit
      int tr[2], nt = 0;
      for (int e = 0; e < DIM; ++e)
        if (e != d) tr[nt++] = e;
      double sum = 0.0;
      for (int q = 0; q < (1 << nt); ++q) {
        int F[3] = {G[0], G[1], G[2]}, lf[3], slot = 0;
        F[d] = 2 * G[d];
        for (int u = 0; u < nt; ++u) F[tr[u]] = 2 * G[tr[u]] + ((q >> u) & 1);
        for (int e = 0; e < 3; ++e) {
          if (e >= DIM) {
            lf[e] = F[e] - bc[e] * nxd[e];
            continue;
          }
          int off = (F[e] - 2 * bc[e] * nxd[e]) / nxd[e];
          if (off > 1) off = 1;  // the child's high face
          lf[e] = F[e] - (2 * bc[e] + off) * nxd[e];
          slot |= off << e;
        }
        sum += phi_old[(long long)m[2 + slot] * g.nfb + ring_index(g, d, lf[0], lf[1], lf[2])];
      }
      *dst = sum / (1 << nt);
      continue;
    }
    if (G[d] & 1) continue;  // inside a parent cell: the next kernel
    int pl[3];
    for (int e = 0; e < 3; ++e) pl[e] = e < DIM ? (G[e] >> 1) - (bc[e] >> 1) * nxd[e] : f[e];
    const double* P = phi_old + (long long)m[1] * g.nfb;
    const double pc = P[ring_index(g, d, pl[0], pl[1], pl[2])];
    double val = pc;
    for (int e = 0; e < DIM; ++e) {
      if (e == d) continue;
      int lo[3] = {pl[0], pl[1], pl[2]}, hi[3] = {pl[0], pl[1], pl[2]};
      lo[e] -= 1;
      hi[e] += 1;
      const bool hl = pl[e] > 0, hh = pl[e] < nxd[e] - 1;
      const double dl = hl ? pc - P[ring_index(g, d, lo[0], lo[1], lo[2])] : 0.0;
      const double dh = hh ? P[ring_index(g, d, hi[0], hi[1], hi[2])] - pc : 0.0;
      const double slope = hl && hh ? minmod_t(dl, dh) : (hl ? dl : dh);
      val += ((G[e] & 1) ? 0.25 : -0.25) * slope;
    }
    *dst = val;
  }
}

// The faces inside the parent cells of refined blocks: one thread per parent
// cell (blocks of other kinds skip), the least-norm divergence-free completion.
template <int DIM>
__global__ void __launch_bounds__(256) face_interior_kernel(StageArgs a, const int* __restrict__ map, CtGeom g,
                                                           double* phi) {
  constexpr int NC = 1 << DIM;
  const int hx = a.nx / 2, hy = a.ny / 2, hz = DIM == 3 ? a.nz / 2 : 1;
  const unsigned per = (unsigned)hx * hy * hz;
  const unsigned n = (unsigned)a.nblocks * per;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    if (map[(size_t)b * kMapStride] != 1) continue;
    const int q = (int)(t - (unsigned)b * per);
    const int base[3] = {2 * (q % hx), 2 * ((q / hx) % hy), DIM == 3 ? 2 * (q / (hx * hy)) : 0};
    const int L = a.blk[4 * b];
    double ih[3], w[3];
    for (int d = 0; d < 3; ++d) {
      ih[d] = d < DIM ? a.idx[d] * (double)(1 << L) : 0.0;
      w[d] = ih[d] * ih[d];
    }
    double* P = phi + (long long)b * g.nfb;
    // the first values: the mean of the two outer faces at the same place
    double x0[DIM][NC], lo[DIM][NC], hi[DIM][NC];
    for (int d = 0; d < DIM; ++d)
      for (int c = 0; c < NC; ++c) {
        int cl[3];
        for (int e = 0; e < 3; ++e) cl[e] = base[e] + (e < DIM ? (c >> e) & 1 : 0);
        int fl[3] = {cl[0], cl[1], cl[2]}, fh[3] = {cl[0], cl[1], cl[2]};
        fl[d] = base[d];
        fh[d] = base[d] + 2;
        lo[d][c] = P[ring_index(g, d, fl[0], fl[1], fl[2])];
        hi[d][c] = P[ring_index(g, d, fh[0], fh[1], fh[2])];
        x0[d][c] = 0.5 * (lo[d][c] + hi[d][c]);  // used for c with bit d clear
      }
    // divergence of each finer cell with the first values
    double r[NC];
    for (int c = 0; c < NC; ++c) {
      double s = 0.0;
      for (int d = 0; d < DIM; ++d) {
        const int c0 = c & ~(1 << d);
        s += ((c >> d) & 1) ? (hi[d][c] - x0[d][c0]) * ih[d] : (x0[d][c0] - lo[d][c]) * ih[d];
      }
      r[c] = s;
    }
    // y = sum over the Walsh functions chi_s, s != 0, of <chi_s, r> / (NC lambda_s) chi_s,
    // lambda_s = 2 sum_{d in s} 1/h_d^2
    double y[NC];
    for (int c = 0; c < NC; ++c) y[c] = 0.0;
    for (int sw = 1; sw < NC; ++sw) {
      double proj = 0.0, lam = 0.0;
      for (int c = 0; c < NC; ++c) proj += (__popc(sw & c) & 1) ? -r[c] : r[c];
      for (int d = 0; d < DIM; ++d)
        if ((sw >> d) & 1) lam += 2.0 * w[d];
      const double coef = proj / (NC * lam);
      for (int c = 0; c < NC; ++c) y[c] += (__popc(sw & c) & 1) ? -coef : coef;
    }
    for (int d = 0; d < DIM; ++d)
      for (int c = 0; c < NC; ++c) {
        if ((c >> d) & 1) continue;
        int fl[3];
        for (int e = 0; e < 3; ++e) fl[e] = base[e] + (e < DIM ? (c >> e) & 1 : 0);
        fl[d] = base[d] + 1;
        P[ring_index(g, d, fl[0], fl[1], fl[2])] = x0[d][c] + (y[c | (1 << d)] - y[c]) * ih[d];
      }
  }
}

template <typename T, int DIM, bool FLAT>
__global__ void __launch_bounds__(256) transfer_kernel(StageArgs a, TransferArgs r) {
  unsigned cnt[4] = {0u, 0u, 0u, 0u};
  double rate_max = 0.0;
  const int nch = 1 << DIM;
  const long long n = (long long)a.nblocks * a.nint;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / a.nint);
    const int ci = (int)(t - (long long)b * a.nint);
    const int loc[3] = {ci % a.nx, (ci / a.nx) % a.ny, ci / (a.nx * a.ny)};
    const int nxd[3] = {a.nx, a.ny, a.nz};
    const int cg = ((loc[2] + a.gz) * a.Ny + (loc[1] + a.gy)) * a.Nx + (loc[0] + a.gx);
    const int L = a.blk[4 * b];
    const int bc[3] = {a.blk[4 * b + 1], a.blk[4 * b + 2], a.blk[4 * b + 3]};
    const int* m = r.map + (size_t)b * kMapStride;
    const int kind = m[0];
    double U[NV], Pg[NV];
    if (kind == 0) {
      const int ob = m[1];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        U[v] = r.U_old[((size_t)ob * NV + v) * a.nint + ci];
        Pg[v] = r.P_old[((size_t)ob * NV + v) * a.ncell + cg];
      }
    } else if (kind == 1) {
      const int ob = m[1];
      int pl[3], G[3];
      for (int e = 0; e < 3; ++e) {
        G[e] = bc[e] * nxd[e] + loc[e];
        pl[e] = e < DIM ? (G[e] >> 1) - (bc[e] >> 1) * nxd[e] : loc[e];
      }
      const int pint = (pl[2] * a.ny + pl[1]) * a.nx + pl[0];
      const int pg = ((pl[2] + a.gz) * a.Ny + (pl[1] + a.gy)) * a.Nx + (pl[0] + a.gx);
      const int si[3] = {1, a.nx, a.nx * a.ny};
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double* Uo = r.U_old + ((size_t)ob * NV + v) * a.nint;
        const double Uc = Uo[pint];
        double u = Uc;
        for (int d = 0; d < DIM; ++d) {
          double s = 0.0;
          if (pl[d] > 0 && pl[d] < nxd[d] - 1) s = minmod_t(Uc - Uo[pint - si[d]], Uo[pint + si[d]] - Uc);
          u += ((G[d] & 1) ? 0.25 : -0.25) * s;
        }
        U[v] = u;
        Pg[v] = r.P_old[((size_t)ob * NV + v) * a.ncell + pg];
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = Pg[v] = 0.0;
      for (int s = 0; s < nch; ++s) {
        int fl[3], slot = 0;
        for (int e = 0; e < 3; ++e) {
          const int G = bc[e] * nxd[e] + loc[e];
          const int F = e < DIM ? 2 * G + ((s >> e) & 1) : G;
          const int fb = F / nxd[e];
          fl[e] = F - fb * nxd[e];
          if (e < DIM) slot |= (fb - 2 * bc[e]) << e;
        }
        const int ob = m[2 + slot];
        const int fint = (fl[2] * a.ny + fl[1]) * a.nx + fl[0];
        const int fg = ((fl[2] + a.gz) * a.Ny + (fl[1] + a.gy)) * a.Nx + (fl[0] + a.gx);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          U[v] += r.U_old[((size_t)ob * NV + v) * a.nint + fint];
          Pg[v] += r.P_old[((size_t)ob * NV + v) * a.ncell + fg];
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        U[v] /= nch;
        Pg[v] /= nch;
      }
    }
    if (r.phi) {
      // constrained transport: the cell field is the mean of the new faces
      const double* P = r.phi + (long long)b * r.g.nfb;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        int h[3] = {loc[0], loc[1], loc[2]};
        h[d] += 1;
        U[B1 + d] = 0.5 * (P[ring_index(r.g, d, loc[0], loc[1], loc[2])] + P[ring_index(r.g, d, h[0], h[1], h[2])]);
      }
      U[PSI] = 0.0;
    }
    // the guess goes where finish_cell reads the previous primitives
    double* Pin = const_cast<double*>(a.P_in) + (size_t)b * NV * a.ncell + cg;
#pragma unroll
    for (int v = 0; v < NV; ++v) Pin[(size_t)v * a.ncell] = Pg[v];
    const LevelGeo geo = level_geo(a, L);
    const int I1 = bc[0] * a.nx + loc[0], I2 = bc[1] * a.ny + loc[1];
    finish_cell<T, DIM, FLAT, false>(a, geo, b, ci, cg, I1, I2, U, cnt, rate_max);
  }
  reduce_outputs(a, cnt, rate_max);
}

int transfer_grid(long long n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long g = (n + 255) / 256;
  if (g > 32LL * nsm) g = 32LL * nsm;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_face_transfer(const StageArgs& a, const int* map, const CtGeom& g, const double* phi_old,
                                 double* phi, cudaStream_t st) {
  const long long nf = (long long)a.nblocks * g.nown_b;
  const long long nc = (long long)a.nblocks * (a.nx / 2) * (a.ny / 2) * (a.ndim == 3 ? a.nz / 2 : 1);
  if (a.ndim == 3) {
    face_transfer_kernel<3><<<transfer_grid(nf), 256, 0, st>>>(a, map, g, phi_old, phi);
    face_interior_kernel<3><<<transfer_grid(nc), 256, 0, st>>>(a, map, g, phi);
  } else {
    face_transfer_kernel<2><<<transfer_grid(nf), 256, 0, st>>>(a, map, g, phi_old, phi);
    face_interior_kernel<2><<<transfer_grid(nc), 256, 0, st>>>(a, map, g, phi);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transfer_t(const StageArgs& a, const TransferArgs& r, cudaStream_t st) {
  const int grid = transfer_grid((long long)a.nblocks * a.nint);
  if (a.ndim == 3)
    a.flat ? transfer_kernel<T, 3, true><<<grid, 256, 0, st>>>(a, r) : transfer_kernel<T, 3, false><<<grid, 256, 0, st>>>(a, r);
  else
    a.flat ? transfer_kernel<T, 2, true><<<grid, 256, 0, st>>>(a, r) : transfer_kernel<T, 2, false><<<grid, 256, 0, st>>>(a, r);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The plan (host).  Leaves are kept per level as flags over that level's block
// lattice; a block region (L, c) is "covered" by the leaf at the coarsest level
// containing it, or is subdivided.
// ---------------------------------------------------------------------------
struct Forest {
  int ndim, nlev, nx[3], bc[3][2];
  long long n[8][3];
  std::vector<unsigned char> leaf[8];
  long long index(int L, const long long c[3]) const { return (c[2] * n[L][1] + c[1]) * n[L][0] + c[0]; }
  bool inside(int L, const long long c[3]) const {
    if (L < 0 || L >= nlev) return false;
    for (int k = 0; k < 3; ++k)
      if (c[k] < 0 || c[k] >= n[L][k]) return false;
    return true;
  }
  bool is_leaf(int L, const long long c[3]) const { return inside(L, c) && leaf[L][index(L, c)]; }
  // level of the covering leaf, or L + 1 if the region is subdivided
  int cover(int L, const long long c[3]) const {
    for (int l = L; l >= 0; --l) {
      long long a[3];
      for (int k = 0; k < 3; ++k) a[k] = k < ndim ? c[k] >> (L - l) : c[k];
      if (is_leaf(l, a)) return l;
    }
    return L + 1;
  }
  // whether any child of the subdivided region (L, r) is itself subdivided
  bool deeper(int L, const long long r[3]) const {
    for (int s = 0; s < (1 << ndim); ++s) {
      long long ch[3] = {r[0], r[1], r[2]};
      for (int k = 0; k < ndim; ++k) ch[k] = 2 * r[k] + ((s >> k) & 1);
      if (cover(L + 1, ch) == L + 2) return true;
    }
    return false;
  }
  void split(int L, const long long c[3]) {
    leaf[L][index(L, c)] = 0;
    for (int s = 0; s < (1 << ndim); ++s) {
      long long ch[3] = {c[0], c[1], c[2]};
      for (int k = 0; k < ndim; ++k) ch[k] = 2 * c[k] + ((s >> k) & 1);
      leaf[L + 1][index(L + 1, ch)] = 1;
    }
  }
  // regions at level L across offset dl from c, after the boundary rules
  int across(int L, const long long c[3], const int dl[3], long long out[2][3]) const {
    long long p[3];
    bool axis = false;
    for (int k = 0; k < 3; ++k) p[k] = c[k] + dl[k];
    for (int k = 0; k < ndim; ++k) {
      const long long N = n[L][k];
      if (p[k] >= 0 && p[k] < N) continue;
      const int side = p[k] < 0 ? 0 : 1, kind = bc[k][side];
      if (kind == BHAC_BC_PERIODIC) {
        p[k] = ((p[k] % N) + N) % N;
      } else if (kind == BHAC_BC_AXIS) {
        p[k] = side == 0 ? -1 - p[k] : 2 * N - 1 - p[k];
        axis = true;
      } else {
        return 0;
      }
    }
    for (int k = 0; k < 3; ++k) out[0][k] = p[k];
    if (!axis || ndim != 3) return 1;
    // through the axis at phi + pi: the block's cells, shifted by half the
    // cells around, lie in one or two blocks
    const long long nz = nx[2], cells = n[L][2] * nz, half = cells / 2;
    const long long b0 = ((p[2] * nz + half) % cells) / nz, b1 = (((p[2] + 1) * nz - 1 + half) % cells) / nz;
    out[0][2] = b0;
    if (b1 == b0) return 1;
    for (int k = 0; k < 3; ++k) out[1][k] = p[k];
    out[1][2] = b1;
    return 2;
  }
};

void unindex(const Forest& f, int L, long long q, long long c[3]) {
  c[0] = q % f.n[L][0];
  c[1] = (q / f.n[L][0]) % f.n[L][1];
  c[2] = q / (f.n[L][0] * f.n[L][1]);
}

}  // namespace
}  // namespace bhac

using namespace bhac;

extern "C" bhac_status bhac_estimate(bhac_ctx* c, double eps, double* block_err) {
  if (!c || !block_err || !(eps >= 0.0)) return BHAC_ERR_ARG;
  if (!c->prims_ok) return BHAC_ERR_STATE;
  if (ghost_fill(c, c->cur, false) != BHAC_OK) return BHAC_ERR_CUDA;
  StageArgs a = base_args(c);
  double* d_out = c->scratch_out;  // the output staging array is free between read-backs
  if (c->ev_d2h && cudaStreamWaitEvent(c->st, c->ev_d2h, 0) != cudaSuccess) return BHAC_ERR_CUDA;
  if (c->mixed)
    estimate_kernel<float><<<c->nb, 256, 0, c->st>>>(a, c->P32[c->cur], eps, d_out);
  else
    estimate_kernel<double><<<c->nb, 256, 0, c->st>>>(a, c->P[c->cur], eps, d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(block_err, d_out, sizeof(double) * c->nb, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  return e == cudaSuccess ? BHAC_OK : BHAC_ERR_CUDA;
}

extern "C" bhac_status bhac_regrid_plan(const bhac_grid_desc* d, const bhac_block_desc* blocks, int nb,
                                        const double* block_err, double tol_refine, double tol_coarsen, int max_level,
                                        bhac_block_desc* out, int cap, int* nout) {
  if (!d || !blocks || nb <= 0 || !block_err || !out || !nout || cap < 0) return BHAC_ERR_ARG;
  if (d->ndim < 2 || d->ndim > 3 || max_level < 0 || max_level >= d->nlevels || d->nlevels > 8) return BHAC_ERR_ARG;
  Forest f;
  f.ndim = d->ndim;
  f.nlev = d->nlevels;
  for (int k = 0; k < 3; ++k) {
    f.nx[k] = d->nx[k];
    f.bc[k][0] = d->bc[k][0];
    f.bc[k][1] = d->bc[k][1];
  }
  std::vector<int> orig[8];
  for (int L = 0; L < f.nlev; ++L) {
    long long cells = 1;
    for (int k = 0; k < 3; ++k) {
      f.n[L][k] = (long long)d->nroot[k] << (k < d->ndim ? L : 0);
      cells *= f.n[L][k];
    }
    f.leaf[L].assign(cells, 0);
    orig[L].assign(cells, -1);
  }
  for (int b = 0; b < nb; ++b) {
    const long long c[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    const int L = blocks[b].level;
    if (!f.inside(L, c) || f.leaf[L][f.index(L, c)]) return BHAC_ERR_ARG;
    f.leaf[L][f.index(L, c)] = 1;
    orig[L][f.index(L, c)] = b;
  }
  for (int b = 0; b < nb; ++b) {
    const long long c[3] = {blocks[b].ix, blocks[b].iy, blocks[b].iz};
    if (blocks[b].level < max_level && block_err[b] > tol_refine) f.split(blocks[b].level, c);
  }
  // neighbour offsets, fixed order
  std::vector<std::array<int, 3>> offs;
  for (int a = -1; a <= 1; ++a)
    for (int bb = -1; bb <= 1; ++bb)
      for (int e = -1; e <= 1; ++e)
        if (!(a == 0 && bb == 0 && e == 0) && (d->ndim == 3 || e == 0)) offs.push_back({a, bb, e});
  // balance 2:1 by refining, to a fixed point
  for (bool changed = true; changed;) {
    changed = false;
    for (int L = 0; L < f.nlev; ++L) {
      std::vector<unsigned char> here(f.leaf[L].size(), 0);
      std::vector<std::vector<unsigned char>> coarser(L);
      for (int l = 0; l < L; ++l) coarser[l].assign(f.leaf[l].size(), 0);
      for (long long q = 0; q < (long long)f.leaf[L].size(); ++q) {
        if (!f.leaf[L][q]) continue;
        long long c[3];
        unindex(f, L, q, c);
        for (const auto& o : offs) {
          long long r[2][3];
          const int nr = f.across(L, c, o.data(), r);
          for (int m = 0; m < nr; ++m) {
            const int st = f.cover(L, r[m]);
            if (st < L - 1) {
              long long a[3];
              for (int k = 0; k < 3; ++k) a[k] = k < f.ndim ? r[m][k] >> (L - st) : r[m][k];
              coarser[st][f.index(st, a)] = 1;
            } else if (st == L + 1 && L + 1 < f.nlev && f.deeper(L, r[m])) {
              here[q] = 1;
            }
          }
        }
      }
      for (long long q = 0; q < (long long)here.size(); ++q)
        if (here[q] && L + 1 < f.nlev) {
          long long c[3];
          unindex(f, L, q, c);
          f.split(L, c);
          changed = true;
        }
      for (int l = 0; l < L; ++l)
        for (long long q = 0; q < (long long)coarser[l].size(); ++q)
          if (coarser[l][q] && f.leaf[l][q]) {
            long long c[3];
            unindex(f, l, q, c);
            f.split(l, c);
            changed = true;
          }
    }
  }
  // coarsen complete groups of original leaves below tol_coarsen whose parent
  // keeps the balance (decided on the refined forest, then applied together)
  std::vector<std::pair<int, long long>> merge;
  for (int L = 1; L < f.nlev; ++L)
    for (long long q = 0; q < (long long)f.leaf[L - 1].size(); ++q) {
      long long p[3];
      unindex(f, L - 1, q, p);
      bool ok = true;
      for (int s = 0; s < (1 << f.ndim) && ok; ++s) {
        long long ch[3] = {p[0], p[1], p[2]};
        for (int k = 0; k < f.ndim; ++k) ch[k] = 2 * p[k] + ((s >> k) & 1);
        const int ob = f.inside(L, ch) ? orig[L][f.index(L, ch)] : -1;
        if (ob < 0 || !f.is_leaf(L, ch) || !(block_err[ob] < tol_coarsen)) ok = false;
      }
      for (size_t o = 0; o < offs.size() && ok; ++o) {
        long long r[2][3];
        const int nr = f.across(L - 1, p, offs[o].data(), r);
        for (int m = 0; m < nr && ok; ++m) {
          const int st = f.cover(L - 1, r[m]);
          if (st < L - 2 || (st == L && f.deeper(L - 1, r[m]))) ok = false;
        }
      }
      if (ok) merge.push_back({L - 1, q});
    }
  for (const auto& g : merge) {
    long long p[3];
    unindex(f, g.first, g.second, p);
    for (int s = 0; s < (1 << f.ndim); ++s) {
      long long ch[3] = {p[0], p[1], p[2]};
      for (int k = 0; k < f.ndim; ++k) ch[k] = 2 * p[k] + ((s >> k) & 1);
      f.leaf[g.first + 1][f.index(g.first + 1, ch)] = 0;
    }
    f.leaf[g.first][g.second] = 1;
  }
  int count = 0;
  for (int L = 0; L < f.nlev; ++L)
    for (long long q = 0; q < (long long)f.leaf[L].size(); ++q)
      if (f.leaf[L][q]) {
        if (count < cap) {
          long long c[3];
          unindex(f, L, q, c);
          out[count].level = L;
          out[count].ix = (int)c[0];
          out[count].iy = (int)c[1];
          out[count].iz = (int)c[2];
        }
        ++count;
      }
  *nout = count;
  return count <= cap ? BHAC_OK : BHAC_ERR_NOMEM;
}

extern "C" bhac_status bhac_regrid_transfer(const bhac_ctx* old, bhac_ctx* fresh) {
  if (!old || !fresh || old == fresh) return BHAC_ERR_ARG;
  const bhac_grid_desc &a = old->d, &b = fresh->d;
  if (a.ndim != b.ndim || a.precision != b.precision || a.coords != b.coords || a.divb != b.divb)
    return BHAC_ERR_ARG;
  const bool ct = a.divb == BHAC_DIVB_CT;
  for (int k = 0; k < 3; ++k) {
    if (a.nx[k] != b.nx[k] || a.nroot[k] != b.nroot[k]) return BHAC_ERR_ARG;
    if (ct && k < a.ndim && (a.nx[k] & 1)) return BHAC_ERR_ARG;  // parent cells split inside a block
  }
  if (!old->prims_ok || !fresh->metric_ok || (ct && !old->faces_ok)) return BHAC_ERR_STATE;
  // which old blocks feed each new one
  std::map<std::array<int, 4>, int> where;
  for (int n = 0; n < old->nb; ++n)
    where[{old->blk[4 * n], old->blk[4 * n + 1], old->blk[4 * n + 2], old->blk[4 * n + 3]}] = n;
  std::vector<int> map((size_t)fresh->nb * kMapStride, -1);
  const int nd = b.ndim;
  for (int n = 0; n < fresh->nb; ++n) {
    const int L = fresh->blk[4 * n];
    const int c[3] = {fresh->blk[4 * n + 1], fresh->blk[4 * n + 2], fresh->blk[4 * n + 3]};
    int* m = &map[(size_t)n * kMapStride];
    auto it = where.find({L, c[0], c[1], c[2]});
    if (it != where.end()) {
      m[0] = 0;
      m[1] = it->second;
      continue;
    }
    // the old leaves of this level across each face (periodic wrap)
    for (int d = 0; d < nd; ++d)
      for (int side = 0; side < 2; ++side) {
        int q[3] = {c[0], c[1], c[2]};
        const int nbd = b.nroot[d] << L;
        q[d] += side ? 1 : -1;
        if (q[d] < 0 || q[d] >= nbd) {
          if (b.bc[d][side] != BHAC_BC_PERIODIC) continue;
          q[d] = (q[d] + nbd) % nbd;
        }
        auto jt = where.find({L, q[0], q[1], q[2]});
        if (jt != where.end()) m[10 + 2 * d + side] = jt->second;
      }
    const int p[3] = {c[0] >> 1, c[1] >> 1, nd == 3 ? c[2] >> 1 : c[2]};
    if (L > 0 && (it = where.find({L - 1, p[0], p[1], p[2]})) != where.end()) {
      m[0] = 1;
      m[1] = it->second;
      continue;
    }
    m[0] = 2;
    for (int s = 0; s < (1 << nd); ++s) {
      const int ch[3] = {2 * c[0] + (s & 1), 2 * c[1] + ((s >> 1) & 1), nd == 3 ? 2 * c[2] + ((s >> 2) & 1) : c[2]};
      auto jt = where.find({L + 1, ch[0], ch[1], ch[2]});
      if (jt == where.end()) return BHAC_ERR_ARG;  // neither kept, refined nor coarsened by one level
      m[2 + s] = jt->second;
    }
  }
  // the map rides in the fresh context's input staging array
  int* d_map = reinterpret_cast<int*>(fresh->scratch);
  cudaError_t e = cudaStreamWaitEvent(fresh->st, fresh->ev_scat, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_map, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice, fresh->st);
  // the old state must be complete on its own stream before the fresh one reads it
  cudaEvent_t ready = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, old->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(fresh->st, ready, 0);
  if (ready) cudaEventDestroy(ready);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  StageArgs s = base_args(fresh);
  s.stage = 1;
  s.dt_host = 1.0;  // no time step is taken; keeps stage 1's dt off the CFL word
  s.P_in = fresh->P[1];
  s.P_out = fresh->P[0];
  s.P32_out = fresh->P32[0];
  s.Uout = fresh->U[0];
  TransferArgs r;
  r.map = d_map;
  r.U_old = old->U[old->ucur];
  r.P_old = old->P[old->cur];
  r.phi = ct ? fresh->phi[0] : nullptr;
  r.g = fresh->ctg;
  if (ct) e = launch_face_transfer(s, d_map, fresh->ctg, old->phi[old->pcur], fresh->phi[0], fresh->st);
  if (e == cudaSuccess)
    e = fresh->mixed ? launch_transfer_t<float>(s, r, fresh->st) : launch_transfer_t<double>(s, r, fresh->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fresh->work, 0, sizeof(unsigned int), fresh->st);
  if (e != cudaSuccess) return BHAC_ERR_CUDA;
  fresh->cur = 0;
  fresh->ucur = 0;
  fresh->prims_ok = true;
  fresh->cfl_ok = false;
  if (ct) {
    fresh->pcur = 0;
    fresh->faces_ok = true;
  }
  return BHAC_OK;
}
