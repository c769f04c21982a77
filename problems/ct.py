"""Face-centred magnetic fields for constrained transport.

The evolved field is Phi^d = sqrt(gamma) B^d at the centre of every face
normal to an active direction d.  Layout of a face array (both the oracle's
and the library's): for each block, for each active d in order, the block's
owned faces 0..nx_d along d and its cells across, [k][j][i] with i fastest.

A divergence-free start comes from a vector potential at cell edges:
  Phi^1 = d_2 A_3 - d_3 A_2,  Phi^2 = d_3 A_1 - d_1 A_3,  Phi^3 = d_1 A_2 - d_2 A_1
by differences of the edge values (A_3 on edges along x3, A_1 along x1, A_2
along x2), so the discrete divergence of every cell vanishes to round-off.
On a grid with refinement levels each block uses its own level's spacing.
A potential component that does not depend on its own coordinate (A_1 free
of x1, and so on) has exact edge integrals, so a coarse face on a level
boundary then equals the mean of the finer faces covering it.
These are set-ups and diagnostics; the update arithmetic lives in the
oracle and in the library, not here."""
from __future__ import annotations

import math

import numpy as np

from . import Grid

__all__ = ["face_shapes", "face_count", "split_faces", "join_faces", "faces_from_potential",
           "face_divergence", "shock_tube_faces", "alfven_wave_faces", "random_potential_faces",
           "fm_torus_faces"]


def face_shapes(grid: Grid):
    """Per active direction d: (nz, ny, nx) of one block's face array, +1 along d."""
    out = []
    for d in range(grid.ndim):
        n = [grid.nx[2], grid.nx[1], grid.nx[0]]
        n[2 - d] += 1
        out.append(tuple(n))
    return out


def face_count(grid: Grid) -> int:
    return grid.nb * sum(int(np.prod(s)) for s in face_shapes(grid))


def split_faces(grid: Grid, flat: np.ndarray):
    """Flat face array -> list over d of (nb, nz', ny', nx') arrays."""
    shapes = face_shapes(grid)
    per = [int(np.prod(s)) for s in shapes]
    blk = np.asarray(flat).reshape(grid.nb, sum(per))
    out, o = [], 0
    for s, n in zip(shapes, per):
        out.append(blk[:, o:o + n].reshape((grid.nb,) + s))
        o += n
    return out


def join_faces(grid: Grid, parts) -> np.ndarray:
    return np.concatenate([p.reshape(grid.nb, -1) for p in parts], axis=1).ravel()


def _dx(grid):
    """Per direction, the spacing of every block at its level, shape (nb, 1, 1, 1)."""
    lev = grid.blocks[:, 0].astype(np.int64)
    out = []
    for d in range(3):
        scale = 2.0 ** lev if d < grid.ndim else np.ones(grid.nb)
        out.append(((grid.xmax[d] - grid.xmin[d]) / (grid.nroot[d] * grid.nx[d]) / scale).reshape(-1, 1, 1, 1))
    return out


def _coords(grid, face_dims, centre_dims):
    """Per block, coordinates (x1, x2, x3) on a lattice that is face-located
    (index 0..n) in face_dims and cell-centred (0..n-1) elsewhere; each array
    (nb, nz', ny', nx')."""
    dx = _dx(grid)
    axes = []
    for d in range(3):
        n = grid.nx[d] + (1 if d in face_dims else 0)
        off = 0.0 if d in face_dims else 0.5
        g = grid.blocks[:, 1 + d].astype(np.int64)[:, None] * grid.nx[d] + np.arange(n)[None, :]
        axes.append(grid.xmin[d] + (g + off) * dx[d].reshape(-1, 1))
    nb = grid.nb
    X1 = axes[0][:, None, None, :]
    X2 = axes[1][:, None, :, None]
    X3 = axes[2][:, :, None, None]
    shape = (nb, X3.shape[1], X2.shape[2], X1.shape[3])
    return (np.broadcast_to(X1, shape), np.broadcast_to(X2, shape), np.broadcast_to(X3, shape))


def faces_from_potential(grid: Grid, A1=None, A2=None, A3=None) -> np.ndarray:
    """Phi from edge values of a vector potential (callables of (x1, x2, x3)
    arrays; None for a zero component)."""
    dx = _dx(grid)
    three = grid.ndim == 3

    def edge(fn, face_dims):
        x = _coords(grid, face_dims, ())
        return np.zeros(x[0].shape) if fn is None else fn(*x)

    a3 = edge(A3, (0, 1))                       # (nb, nz, ny+1, nx+1)
    p1 = (a3[:, :, 1:, :] - a3[:, :, :-1, :]) / dx[1]
    p2 = -(a3[:, :, :, 1:] - a3[:, :, :, :-1]) / dx[0]
    parts = [p1, p2]
    if three:
        a1 = edge(A1, (1, 2))                   # (nb, nz+1, ny+1, nx)
        a2 = edge(A2, (0, 2))                   # (nb, nz+1, ny, nx+1)
        parts[0] = p1 - (a2[:, 1:, :, :] - a2[:, :-1, :, :]) / dx[2]
        parts[1] = p2 + (a1[:, 1:, :, :] - a1[:, :-1, :, :]) / dx[2]
        p3 = (a2[:, :, :, 1:] - a2[:, :, :, :-1]) / dx[0] - (a1[:, :, 1:, :] - a1[:, :, :-1, :]) / dx[1]
        parts.append(p3)
    return join_faces(grid, parts)


def face_divergence(grid: Grid, faces) -> np.ndarray:
    """Discrete divergence sum_d (Phi^d_high - Phi^d_low) / dx_d of every
    interior cell, (nb, nz, ny, nx)."""
    dx = _dx(grid)
    parts = split_faces(grid, faces)
    div = np.zeros((grid.nb, grid.nx[2], grid.nx[1], grid.nx[0]))
    for d, p in enumerate(parts):
        ax = 3 - d
        hi = np.take(p, np.arange(1, p.shape[ax]), axis=ax)
        lo = np.take(p, np.arange(0, p.shape[ax] - 1), axis=ax)
        div += (hi - lo) / dx[d]
    return div


def shock_tube_faces(grid: Grid) -> np.ndarray:
    """The shock tube's field as faces: Phi^1 = B^x = 0.5, Phi^2 = B^y of the
    cell column (+1 left of x = 0.5, -1 right), uniform in y."""
    return faces_from_potential(grid, A3=lambda x1, x2, x3: 0.5 * x2 - np.where(
        x1 <= 0.5 + 1e-12, x1, 1.0 - x1))


def alfven_wave_faces(grid: Grid, b0: float = 1.0, eta: float = 1.0) -> np.ndarray:
    """The circularly polarised Alfven wave's field along x as faces:
    A_3 = b0 y - eta b0 sin(2 pi x) / (2 pi) (and in 3-D A_2 = eta b0 cos(2 pi x) / (2 pi)),
    so Phi^1 = b0 and Phi^2, Phi^3 are the face averages of eta b0 cos, sin."""
    k = 2.0 * math.pi
    A3 = lambda x1, x2, x3: b0 * x2 - eta * b0 * np.sin(k * x1) / k
    A2 = (lambda x1, x2, x3: -eta * b0 * np.cos(k * x1) / k) if grid.ndim == 3 else None
    return faces_from_potential(grid, A2=A2, A3=A3)


def random_potential_faces(grid: Grid, seed: int = 7, amp: float = 0.5) -> np.ndarray:
    """A smooth random periodic field: each component of A a sum of a few
    periodic modes of the unit box with seeded amplitudes and phases."""
    rng = np.random.default_rng(seed)

    def comp():
        modes = [(rng.integers(1, 3, size=3), rng.uniform(0.2, 1.0), rng.uniform(0, 2 * np.pi)) for _ in range(3)]

        def f(x1, x2, x3):
            out = np.zeros_like(x1)
            for kv, a, ph in modes:
                arg = 2 * np.pi * (kv[0] * x1 + kv[1] * x2 + (kv[2] * x3 if grid.ndim == 3 else 0.0)) + ph
                out += amp * a * np.sin(arg) / (2 * np.pi)
            return out
        return f

    return faces_from_potential(grid, A1=comp(), A2=comp(), A3=comp())


def fm_torus_faces(grid: Grid, P: np.ndarray, r_in: float = 6.0, r_pmax: float = 12.0) -> np.ndarray:
    """The torus's poloidal loop as faces: Phi^1 = d_2 A_phi, Phi^2 = -d_1 A_phi
    from A_phi = max(rho/rho_max - 0.2, 0) at the cell corners, scaled like the
    cell-centred field of P (fm_torus_prims normalises it to beta)."""
    from .torus import _loop_field, _torus_rho_p_uphi, fm_constants, fm_lnh
    a, gam = grid.spin, grid.gamma_ad
    ell, lnh_in = fm_constants(a, r_in, r_pmax)
    hmax = math.exp(float(fm_lnh(r_pmax, math.pi / 2, a, ell)) - lnh_in)
    K = (hmax - 1.0) * (gam - 1.0) / gam
    g2 = grid.with_(nx=(grid.nx[0], grid.nx[1], 1)) if grid.ndim == 3 else grid
    B1u, _ = _loop_field(g2, a, gam, ell, lnh_in, K, r_in)
    scale = float(np.abs(P[:, 5]).max() / np.abs(B1u).max()) if np.abs(B1u).max() > 0 else 0.0

    def aphi(x1, x2, x3):
        r, th = np.exp(x1), np.pi * x2
        inside, rho, _, _, _ = _torus_rho_p_uphi(r, th, a, gam, ell, lnh_in, K)
        rho = np.where(inside & (r >= r_in), rho, 0.0)
        return scale * np.maximum(rho - 0.2, 0.0)

    return faces_from_potential(grid, A3=aphi)


def own_potential_free(grid: Grid, seed: int = 7, amp: float = 0.5):
    """A smooth random periodic potential whose component A_d does not depend
    on x_d (exact edge integrals at every level): three callables or None."""
    rng = np.random.default_rng(seed)

    def comp(own):
        modes = []
        for _ in range(3):
            kv = rng.integers(1, 3, size=3)
            kv[own] = 0
            if grid.ndim == 2:
                kv[2] = 0
            modes.append((kv, rng.uniform(0.2, 1.0), rng.uniform(0, 2 * np.pi)))

        def f(x1, x2, x3):
            out = np.zeros_like(x1)
            for kv, a, ph in modes:
                out += amp * a * np.sin(2 * np.pi * (kv[0] * x1 + kv[1] * x2 + kv[2] * x3) + ph) / (2 * np.pi)
            return out
        return f

    if grid.ndim == 2:
        return None, None, comp(2)
    return comp(0), comp(1), comp(2)


def _face_table(grid: Grid, faces):
    """{(level, d, G1, G2, G3): Phi} over every block's owned faces (global
    level indices: a face index along d, cell indices across)."""
    out = {}
    for d, p in enumerate(split_faces(grid, faces)):
        nb, n3, n2, n1 = p.shape
        k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
        for b in range(grid.nb):
            lev, bx, by, bz = (int(v) for v in grid.blocks[b])
            G1, G2, G3 = bx * grid.nx[0] + i, by * grid.nx[1] + j, bz * grid.nx[2] + k
            for g1, g2, g3, v in zip(G1.ravel(), G2.ravel(), G3.ravel(), p[b].ravel()):
                out[(lev, d, int(g1), int(g2), int(g3))] = float(v)
    return out


def level_face_mismatch(grid: Grid, faces) -> float:
    """Largest |Phi of a coarse face - mean of the finer faces covering it| over
    the faces that lie on a level boundary (0.0 on a uniform grid)."""
    tab = _face_table(grid, faces)
    worst = 0.0
    for (lev, d, g1, g2, g3), v in tab.items():
        G = [g1, g2, g3]
        fine = []
        trans = [e for e in range(grid.ndim) if e != d]
        for q in range(1 << len(trans)):
            F = [2 * G[e] if e < grid.ndim else G[e] for e in range(3)]
            for u, e in enumerate(trans):
                F[e] += (q >> u) & 1
            key = (lev + 1, d, F[0], F[1], F[2])
            if key in tab:
                fine.append(tab[key])
        if len(fine) == 1 << len(trans):
            worst = max(worst, abs(v - sum(fine) / len(fine)))
    return worst


def plane_fluxes(grid: Grid, faces, d: int):
    """Magnetic flux sum Phi^d * (face area) through each plane x_d = const at
    the level-0 face positions (the finest faces available over each part of
    the plane), as a list over the planes."""
    tab = _face_table(grid, faces)
    dx0 = [(grid.xmax[e] - grid.xmin[e]) / (grid.nroot[e] * grid.nx[e]) for e in range(3)]
    N0 = grid.nroot[d] * grid.nx[d]
    out = []
    for G0 in range(N0):
        total = 0.0
        for (lev, dd, g1, g2, g3), v in tab.items():
            G = (g1, g2, g3)
            if dd != d or G[d] != G0 * 2 ** lev:
                continue
            # a face counts where no finer face covers it
            trans = [e for e in range(grid.ndim) if e != d]
            F = [2 * G[e] if e < grid.ndim else G[e] for e in range(3)]
            if (lev + 1, d, F[0], F[1], F[2]) in tab:
                continue
            area = 1.0
            for e in range(3):
                if e != d:
                    area *= dx0[e] / (2 ** lev if e < grid.ndim else 1)
            total += v * area
        out.append(total)
    return out
