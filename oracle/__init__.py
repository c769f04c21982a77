"""Python access to the plain FP64 CPU oracle (ctypes).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the product package never
does.  The oracle is written in C (``bhac_oracle.c``) and follows the method of
the paper's Sec. 2 step by step; see the C file for the equations.

The grid description is read from a ``problems.Grid`` object (a plain record of
sizes and parameters shared with the CUDA path's tests); nothing else is shared.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bhac_oracle.c")
_HDR = os.path.join(_HERE, "bhac_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NV = 9
COORDS = {"cart": 0, "ks": 1, "mks": 2}
BCS = {"periodic": 0, "outflow": 1, "axis": 2, "noinflow": 3}
RECON = {"ppm": 0, "minmod": 1}
RIEMANN = {"hll": 0, "tvdlf": 1}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, FP contraction off so
    x86 and Arm give identical results)."""
    with _lock:
        stale = not os.path.exists(_LIB) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class OrParams(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_int * 3), ("ng", C.c_int), ("nroot", C.c_int * 3),
        ("nlevels", C.c_int), ("xmin", C.c_double * 3), ("xmax", C.c_double * 3),
        ("coords", C.c_int), ("spin", C.c_double), ("mass", C.c_double),
        ("bc", (C.c_int * 2) * 3), ("recon", C.c_int), ("riemann", C.c_int),
        ("gamma_ad", C.c_double), ("cfl", C.c_double), ("ch", C.c_double), ("kappa", C.c_double),
        ("c2p_tol", C.c_double), ("c2p_maxit", C.c_int),
        ("rho_floor", C.c_double), ("rho_floor_pow", C.c_double), ("p_floor", C.c_double),
        ("p_floor_pow", C.c_double), ("w_max", C.c_double), ("ct", C.c_int), ("imex", C.c_int),
        ("c2p_nk", C.c_int),
    ]


_DP = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_IP = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_LP = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
METRIC_LEN = 62  # alpha, beta[3], g[9], gi[9], sqrtg, da[3], db[9], dg[27]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER(OrParams)
        L.or_metric_at.argtypes = [P, _DP, C.c_int, _DP]
        L.or_prim2con.argtypes = [P, _DP, _DP, _DP]
        L.or_flux.argtypes = [P, _DP, _DP, C.c_int, _DP]
        L.or_wavespeeds.argtypes = [P, _DP, _DP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_sources.argtypes = [P, _DP, _DP, _DP]
        L.or_con2prim.argtypes = [P, _DP, _DP, _DP, C.c_double, _DP]
        L.or_con2prim.restype = C.c_int
        L.or_reconstruct.argtypes = [P, _DP, _DP, _DP]
        L.or_face_flux.argtypes = [P, _DP, _DP, _DP, C.c_int, _DP]
        L.or_create.argtypes = [P, C.c_int, _IP]
        L.or_create.restype = C.c_void_p
        L.or_destroy.argtypes = [C.c_void_p]
        for name in ("or_set_prims", "or_get_prims", "or_get_prims_ghosted", "or_get_cons"):
            getattr(L, name).argtypes = [C.c_void_p, _DP]
        L.or_fill_ghosts.argtypes = [C.c_void_p]
        L.or_cfl_dt.argtypes = [C.c_void_p]
        L.or_cfl_dt.restype = C.c_double
        L.or_stage.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.or_stage_blocks.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, _IP]
        L.or_step.argtypes = [C.c_void_p, C.c_double]
        L.or_c2p_counts.argtypes = [C.c_void_p, _LP]
        L.or_c2p_status.argtypes = [C.c_void_p, C.c_void_p]
        L.or_ghosted_cells.argtypes = [C.c_void_p]
        L.or_ghosted_cells.restype = C.c_int
        L.or_estimate.argtypes = [C.c_void_p, C.c_double, _DP]
        L.or_regrid_plan.argtypes = [C.POINTER(OrParams), C.c_int, _IP, _DP, C.c_double, C.c_double, C.c_int,
                                     C.c_int, _IP]
        L.or_regrid_plan.restype = C.c_int
        L.or_regrid_transfer.argtypes = [C.c_void_p, C.c_void_p]
        L.or_face_count.argtypes = [C.c_void_p]
        L.or_face_count.restype = C.c_long
        L.or_set_faces.argtypes = [C.c_void_p, _DP]
        L.or_get_faces.argtypes = [C.c_void_p, _DP]
        L.or_ct_ring_faces.argtypes = [C.c_void_p, C.c_int, _DP]
        _lib = L
    return _lib


def params_of(grid) -> OrParams:
    """Fill the C parameter record from a problems.Grid."""
    p = OrParams()
    p.ndim = grid.ndim
    for d in range(3):
        p.nx[d] = grid.nx[d]
        p.nroot[d] = grid.nroot[d]
        p.xmin[d] = grid.xmin[d]
        p.xmax[d] = grid.xmax[d]
        p.bc[d][0] = BCS[grid.bc[d][0]]
        p.bc[d][1] = BCS[grid.bc[d][1]]
    p.ng = grid.ng
    p.nlevels = grid.nlevels
    p.coords = COORDS[grid.coords]
    p.spin = grid.spin
    p.mass = grid.mass
    p.recon = RECON[grid.recon]
    p.riemann = RIEMANN[grid.riemann]
    p.gamma_ad = grid.gamma_ad
    p.cfl = grid.cfl
    p.ch = grid.ch
    p.kappa = grid.kappa
    p.c2p_tol = grid.c2p_tol
    p.c2p_maxit = grid.c2p_maxit
    p.rho_floor = grid.rho_floor
    p.rho_floor_pow = grid.rho_floor_pow
    p.p_floor = grid.p_floor
    p.p_floor_pow = grid.p_floor_pow
    p.w_max = grid.w_max
    p.ct = 1 if getattr(grid, "divb", "glm") == "ct" else 0
    p.imex = 1 if getattr(grid, "imex", False) else 0
    p.c2p_nk = 1 if getattr(grid, "c2p", "newton") == "nk" else 0
    return p


class Metric:
    """Unpacked or_metric record."""

    def __init__(self, a: np.ndarray):
        self.raw = a
        self.alpha = a[0]
        self.beta = a[1:4]
        self.g = a[4:13].reshape(3, 3)
        self.gi = a[13:22].reshape(3, 3)
        self.sqrtg = a[22]
        self.da = a[23:26]
        self.db = a[26:35].reshape(3, 3)   # db[k][i] = d_k beta^i
        self.dg = a[35:62].reshape(3, 3, 3)  # dg[k][i][j] = d_k gamma_ij


class Point:
    """Point-wise oracle physics for one parameter set."""

    def __init__(self, grid):
        self.p = params_of(grid)
        self.L = lib()

    def metric(self, x, derivs=True) -> Metric:
        out = np.zeros(METRIC_LEN)
        self.L.or_metric_at(C.byref(self.p), np.ascontiguousarray(x, dtype=np.float64), int(derivs), out)
        return Metric(out)

    def prim2con(self, m: Metric, P):
        U = np.zeros(NV)
        self.L.or_prim2con(C.byref(self.p), m.raw, np.ascontiguousarray(P, np.float64), U)
        return U

    def flux(self, m: Metric, P, d):
        F = np.zeros(NV)
        self.L.or_flux(C.byref(self.p), m.raw, np.ascontiguousarray(P, np.float64), d, F)
        return F

    def wavespeeds(self, m: Metric, P, d):
        lm, lp = C.c_double(), C.c_double()
        self.L.or_wavespeeds(C.byref(self.p), m.raw, np.ascontiguousarray(P, np.float64), d,
                             C.byref(lm), C.byref(lp))
        return lm.value, lp.value

    def sources(self, m: Metric, P):
        S = np.zeros(NV)
        self.L.or_sources(C.byref(self.p), m.raw, np.ascontiguousarray(P, np.float64), S)
        return S

    def con2prim(self, m: Metric, U, Pguess, r_floor=1.0):
        P = np.zeros(NV)
        st = self.L.or_con2prim(C.byref(self.p), m.raw, np.ascontiguousarray(U, np.float64),
                                np.ascontiguousarray(Pguess, np.float64), r_floor, P)
        return P, st

    def reconstruct(self, stencil):
        st = np.ascontiguousarray(stencil, np.float64).reshape(6, NV)
        PL, PR = np.zeros(NV), np.zeros(NV)
        self.L.or_reconstruct(C.byref(self.p), st, PL, PR)
        return PL, PR

    def face_flux(self, m: Metric, PL, PR, d):
        F = np.zeros(NV)
        self.L.or_face_flux(C.byref(self.p), m.raw, np.ascontiguousarray(PL, np.float64),
                            np.ascontiguousarray(PR, np.float64), d, F)
        return F


class Oracle:
    """The block grid, stepped by the oracle."""

    def __init__(self, grid):
        self.grid = grid
        self.p = params_of(grid)
        self.L = lib()
        blocks = np.ascontiguousarray(grid.blocks, dtype=np.int32).reshape(-1, 4)
        self.nb = blocks.shape[0]
        self.ctx = self.L.or_create(C.byref(self.p), self.nb, blocks)
        self.shape = (self.nb, NV, grid.nx[2], grid.nx[1], grid.nx[0])

    def __del__(self):
        if getattr(self, "ctx", None):
            self.L.or_destroy(self.ctx)
            self.ctx = None

    def set_prims(self, prims):
        a = np.ascontiguousarray(prims, dtype=np.float64)
        assert a.size == int(np.prod(self.shape))
        self.L.or_set_prims(self.ctx, a)

    def prims(self):
        out = np.zeros(self.shape)
        self.L.or_get_prims(self.ctx, out)
        return out

    def prims_ghosted(self):
        n = self.L.or_ghosted_cells(self.ctx)
        out = np.zeros(self.nb * NV * n)
        self.L.or_get_prims_ghosted(self.ctx, out)
        g = self.grid
        gd = [g.ng if d < g.ndim else 0 for d in range(3)]
        return out.reshape(self.nb, NV, g.nx[2] + 2 * gd[2], g.nx[1] + 2 * gd[1], g.nx[0] + 2 * gd[0])

    def cons(self):
        out = np.zeros(self.shape)
        self.L.or_get_cons(self.ctx, out)
        return out

    def fill_ghosts(self):
        self.L.or_fill_ghosts(self.ctx)

    def cfl_dt(self) -> float:
        return self.L.or_cfl_dt(self.ctx)

    def stage(self, stage: int, dt: float, blocks=None):
        if blocks is None:
            self.L.or_stage(self.ctx, stage, dt)
        else:
            sel = np.ascontiguousarray(blocks, dtype=np.int32)
            self.L.or_stage_blocks(self.ctx, stage, dt, sel.size, sel)

    def step(self, dt: float):
        self.L.or_step(self.ctx, dt)

    def c2p_status(self):
        """Per interior cell (blocks, nz, ny, nx): the last stage's inversion outcome."""
        g = self.grid
        out = np.zeros((self.nb, g.nx[2], g.nx[1], g.nx[0]), dtype=np.uint8)
        self.L.or_c2p_status(self.ctx, out.ctypes.data)
        return out

    def set_faces(self, faces):
        """Face fields Phi^d = sqrt(gamma) B^d (constrained transport), owned
        faces in [block][d][k][j][i] order (problems.face_layout)."""
        a = np.ascontiguousarray(faces, dtype=np.float64)
        assert a.size == self.L.or_face_count(self.ctx)
        self.L.or_set_faces(self.ctx, a)

    def faces(self):
        out = np.zeros(self.L.or_face_count(self.ctx))
        self.L.or_get_faces(self.ctx, out)
        return out

    def ring_faces(self, d):
        """Phi^d over every block's faces and the ring one cell outside it
        (filled from the owned faces), shape (nb, nz', ny', nx') with local
        index -1 at position 0 across active directions."""
        g = self.grid
        ext = [g.nx[e] + (1 if e == d else (2 if e < g.ndim else 0)) for e in range(3)]
        out = np.zeros(self.nb * ext[0] * ext[1] * ext[2])
        self.L.or_ct_ring_faces(self.ctx, d, out)
        return out.reshape(self.nb, ext[2], ext[1], ext[0])

    def estimate(self, eps=0.01):
        """Loehner's estimator on the density, maximum per block."""
        out = np.zeros(self.nb)
        self.L.or_estimate(self.ctx, eps, out)
        return out

    def regrid_plan(self, block_err, tol_refine, tol_coarsen, max_level):
        """The new leaf list, (n, 4) int32 rows (level, ix, iy, iz)."""
        blocks = np.ascontiguousarray(self.grid.blocks, dtype=np.int32).reshape(-1, 4)
        err = np.ascontiguousarray(block_err, dtype=np.float64)
        cap = 64 * self.nb + 64
        out = np.zeros(4 * cap, dtype=np.int32)
        n = self.L.or_regrid_plan(C.byref(self.p), self.nb, blocks, err, tol_refine, tol_coarsen, max_level, cap, out)
        assert n >= 0
        return out[:4 * n].reshape(n, 4)

    def regridded(self, new_blocks):
        """A new oracle grid with the leaf list new_blocks, its state the
        conservative transfer of this one's."""
        fresh = Oracle(self.grid.with_(blocks=np.asarray(new_blocks, dtype=np.int32)))
        self.L.or_regrid_transfer(self.ctx, fresh.ctx)
        return fresh

    def c2p_counts(self):
        out = np.zeros(4, dtype=np.int64)
        self.L.or_c2p_counts(self.ctx, out)
        return out
