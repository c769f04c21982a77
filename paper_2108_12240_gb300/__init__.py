"""GB300 (sm_103a) per-block finite-volume GRMHD update behind a C ABI.

The functions ``bhac_*`` below are a thin ctypes binding of
``include/bhac_gb300.h`` (same names, argument marshalling only); every step
of the update runs in the library's CUDA kernels.  ``Solver`` bundles the
calls for a ``problems.Grid``-like record, with the device arena and stream
taken from PyTorch.  There is no CPU fallback: if the library cannot be
loaded, importing this package raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build, stale

__all__ = [
    "GridDesc", "BlockDesc", "Solver", "BhacError", "lib", "status_string",
    "bhac_query_sizes", "bhac_init_grid", "bhac_set_metric", "bhac_set_prims", "bhac_fill_ghosts",
    "bhac_cfl_dt", "bhac_step", "bhac_stage", "bhac_get_prims", "bhac_get_cons", "bhac_get_diagnostics",
    "bhac_set_launch", "bhac_count_flops", "bhac_graph_capture", "bhac_graph_launch", "bhac_cfl_dt_static", "bhac_destroy",
    "bhac_status_string", "bhac_check_bit_ops", "bhac_ct_ring_faces_host", "bhac_launches_per_step", "bhac_get_prims_ghosted",
    "bhac_get_c2p_status", "bhac_set_cons", "bhac_set_prims_host_async", "bhac_get_prims_host_async",
    "bhac_host_fence", "bhac_measure_peaks", "bhac_set_faces", "bhac_get_faces",
    "bhac_estimate", "bhac_regrid_plan", "bhac_regrid_transfer", "bhac_set_split", "bhac_set_zsplit",
    "bhac_zsplit_in_force",
]

NV = 9
COORDS = {"cart": 0, "ks": 1, "mks": 2}
BCS = {"periodic": 0, "outflow": 1, "axis": 2, "noinflow": 3}
RECON = {"ppm": 0, "minmod": 1}
RIEMANN = {"hll": 0, "tvdlf": 1}
PREC = {"fp64": 0, "mixed": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "arena too small or device allocation failed", 4: "call out of order",
          5: "device wait timed out", 6: "inversion failures"}


class GridDesc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_int * 3), ("nghost", C.c_int), ("nroot", C.c_int * 3),
        ("nlevels", C.c_int), ("xmin", C.c_double * 3), ("xmax", C.c_double * 3), ("coords", C.c_int),
        ("spin", C.c_double), ("mass", C.c_double), ("bc", (C.c_int * 2) * 3), ("recon", C.c_int),
        ("riemann", C.c_int), ("precision", C.c_int), ("gamma_ad", C.c_double), ("cfl", C.c_double),
        ("ch", C.c_double), ("kappa", C.c_double), ("c2p_tol", C.c_double), ("c2p_maxit", C.c_int),
        ("rho_floor", C.c_double), ("rho_floor_pow", C.c_double), ("p_floor", C.c_double),
        ("p_floor_pow", C.c_double), ("w_max", C.c_double), ("divb", C.c_int), ("imex", C.c_int),
        ("c2p_solver", C.c_int),
    ]


class BlockDesc(C.Structure):
    _fields_ = [("level", C.c_int), ("ix", C.c_int), ("iy", C.c_int), ("iz", C.c_int)]


class BhacError(RuntimeError):
    def __init__(self, where: str, status: int):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


_lib = None


def lib():
    """Loads libbhac_gb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = build() if (stale() and os.environ.get("BHAC_NO_BUILD") is None) else LIB
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing; run paper_2108_12240_gb300.build.build()")
        L = C.CDLL(path)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        G, B = C.POINTER(GridDesc), C.POINTER(BlockDesc)
        sig = {
            "bhac_query_sizes": ([G, B, i, C.POINTER(sz)], i),
            "bhac_init_grid": ([C.POINTER(vp), G, B, i, vp, sz, vp], i),
            "bhac_set_metric": ([vp, i, d, d, vp], i),
            "bhac_set_prims": ([vp, vp, i], i),
            "bhac_fill_ghosts": ([vp], i),
            "bhac_cfl_dt": ([vp, C.POINTER(d)], i),
            "bhac_step": ([vp, d], i),
            "bhac_stage": ([vp, i, d], i),
            "bhac_get_prims": ([vp, vp, i], i),
            "bhac_get_cons": ([vp, vp, i], i),
            "bhac_get_diagnostics": ([vp, C.POINTER(C.c_longlong)], i),
            "bhac_set_launch": ([vp, i, i, i, i, i, i], i),
            "bhac_set_split": ([vp, i], i),
            "bhac_set_zsplit": ([vp, i], i),
            "bhac_zsplit_in_force": ([vp], i),
            "bhac_count_flops": ([vp, d, i, C.c_uint, C.POINTER(d)], i),
            "bhac_graph_capture": ([vp, i], i),
            "bhac_graph_launch": ([vp], i),
            "bhac_cfl_dt_static": ([G, B, i, vp, vp, vp], i),
            "bhac_check_bit_ops": ([C.c_longlong, C.c_uint, C.POINTER(C.c_longlong)], i),
            "bhac_ct_ring_faces_host": ([G, B, i, vp, vp], i),
            "bhac_launches_per_step": ([vp, C.POINTER(i)], i),
            "bhac_get_prims_ghosted": ([vp, vp, i], i),
            "bhac_get_c2p_status": ([vp, vp, i], i),
            "bhac_set_cons": ([vp, vp, i], i),
            "bhac_set_prims_host_async": ([vp, vp], i),
            "bhac_get_prims_host_async": ([vp, vp], i),
            "bhac_host_fence": ([vp], i),
            "bhac_measure_peaks": ([i, vp, C.POINTER(d)], i),
            "bhac_set_faces": ([vp, vp, i], i),
            "bhac_estimate": ([vp, d, C.POINTER(d)], i),
            "bhac_regrid_plan": ([G, B, i, C.POINTER(d), d, d, i, B, i, C.POINTER(i)], i),
            "bhac_regrid_transfer": ([vp, vp], i),
            "bhac_get_faces": ([vp, vp, i], i),
            "bhac_destroy": ([vp], None),
            "bhac_status_string": ([i], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(where, st):
    if st not in (0, 6):
        raise BhacError(where, st)
    return st


def status_string(st: int) -> str:
    return lib().bhac_status_string(st).decode()


# ---- the C ABI, one Python function per entry point ----

def bhac_query_sizes(desc: GridDesc, blocks) -> int:
    n = C.c_size_t()
    _check("bhac_query_sizes", lib().bhac_query_sizes(C.byref(desc), blocks, len(blocks), C.byref(n)))
    return n.value


def bhac_init_grid(desc: GridDesc, blocks, arena_ptr: int, arena_bytes: int, stream_ptr: int):
    ctx = C.c_void_p()
    _check("bhac_init_grid", lib().bhac_init_grid(C.byref(ctx), C.byref(desc), blocks, len(blocks),
                                                  C.c_void_p(arena_ptr), arena_bytes, C.c_void_p(stream_ptr)))
    return ctx


def bhac_set_metric(ctx, kind: int, spin: float, mass: float):
    return _check("bhac_set_metric", lib().bhac_set_metric(ctx, kind, spin, mass, None))


def bhac_set_prims(ctx, ptr: int, on_device: bool):
    return _check("bhac_set_prims", lib().bhac_set_prims(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_fill_ghosts(ctx):
    return _check("bhac_fill_ghosts", lib().bhac_fill_ghosts(ctx))


def bhac_cfl_dt(ctx, want_host: bool = True):
    dt = C.c_double(0.0)
    _check("bhac_cfl_dt", lib().bhac_cfl_dt(ctx, C.byref(dt) if want_host else None))
    return dt.value if want_host else None


def bhac_step(ctx, dt: float):
    return _check("bhac_step", lib().bhac_step(ctx, dt))


def bhac_stage(ctx, stage: int, dt: float):
    return _check("bhac_stage", lib().bhac_stage(ctx, stage, dt))


def bhac_get_prims(ctx, ptr: int, on_device: bool):
    return _check("bhac_get_prims", lib().bhac_get_prims(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_get_cons(ctx, ptr: int, on_device: bool):
    return _check("bhac_get_cons", lib().bhac_get_cons(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_get_c2p_status(ctx, ptr: int, on_device: bool):
    _check("bhac_get_c2p_status", lib().bhac_get_c2p_status(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_set_cons(ctx, ptr: int, on_device: bool):
    _check("bhac_set_cons", lib().bhac_set_cons(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_set_prims_host_async(ctx, ptr: int):
    _check("bhac_set_prims_host_async", lib().bhac_set_prims_host_async(ctx, C.c_void_p(ptr)))


def bhac_get_prims_host_async(ctx, ptr: int):
    _check("bhac_get_prims_host_async", lib().bhac_get_prims_host_async(ctx, C.c_void_p(ptr)))


def bhac_host_fence(ctx):
    _check("bhac_host_fence", lib().bhac_host_fence(ctx))


def bhac_estimate(ctx, eps: float, nblocks: int) -> np.ndarray:
    out = np.zeros(nblocks)
    _check("bhac_estimate", lib().bhac_estimate(ctx, eps, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def bhac_regrid_plan(desc: GridDesc, blocks, block_err, tol_refine: float, tol_coarsen: float, max_level: int):
    """The new leaf list as an (n, 4) int32 array of (level, ix, iy, iz)."""
    err = np.ascontiguousarray(block_err, dtype=np.float64)
    cap = 64 * len(blocks) + 64
    out = (BlockDesc * cap)()
    n = C.c_int(0)
    _check("bhac_regrid_plan", lib().bhac_regrid_plan(C.byref(desc), blocks, len(blocks),
                                                      err.ctypes.data_as(C.POINTER(C.c_double)), tol_refine,
                                                      tol_coarsen, max_level, out, cap, C.byref(n)))
    return np.array([(out[k].level, out[k].ix, out[k].iy, out[k].iz) for k in range(n.value)],
                    dtype=np.int32).reshape(-1, 4)


def bhac_regrid_transfer(old_ctx, fresh_ctx):
    _check("bhac_regrid_transfer", lib().bhac_regrid_transfer(old_ctx, fresh_ctx))


def bhac_set_faces(ctx, ptr: int, on_device: bool):
    _check("bhac_set_faces", lib().bhac_set_faces(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_get_faces(ctx, ptr: int, on_device: bool):
    _check("bhac_get_faces", lib().bhac_get_faces(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_get_prims_ghosted(ctx, ptr: int, on_device: bool):
    _check("bhac_get_prims_ghosted", lib().bhac_get_prims_ghosted(ctx, C.c_void_p(ptr), int(on_device)))


def bhac_get_diagnostics(ctx):
    out = (C.c_longlong * 4)()
    st = _check("bhac_get_diagnostics", lib().bhac_get_diagnostics(ctx, out))
    return np.array(list(out), dtype=np.int64), st


def bhac_set_launch(ctx, tx=0, ty=0, threads=0, persistent=0, min_ctas=0, producer_warps=0):
    return _check("bhac_set_launch", lib().bhac_set_launch(ctx, tx, ty, threads, persistent, min_ctas,
                                                           producer_warps))


def bhac_set_split(ctx, chunks: int):
    return _check("bhac_set_split", lib().bhac_set_split(ctx, chunks))


def bhac_set_zsplit(ctx, parts: int):
    return _check("bhac_set_zsplit", lib().bhac_set_zsplit(ctx, parts))


def bhac_zsplit_in_force(ctx) -> int:
    return int(lib().bhac_zsplit_in_force(ctx))


def bhac_count_flops(ctx, dt: float, nsamples: int = 2000, seed: int = 1):
    out = (C.c_double * 6)()
    _check("bhac_count_flops", lib().bhac_count_flops(ctx, dt, nsamples, seed, out))
    return {"fp64_flops": out[0], "fp32_flops": out[1], "fp64_special": out[2], "fp32_special": out[3],
            "samples": int(out[4]), "blocks": int(out[5])}


def bhac_check_bit_ops(n: int, seed: int = 1):
    """Disagreement counts of the integer-pipe compares and conversions with
    the hardware instructions, and of the FP64 reciprocal and square roots
    beyond their ulp bounds (see the header for the eleven checks)."""
    out = (C.c_longlong * 11)()
    _check("bhac_check_bit_ops", lib().bhac_check_bit_ops(n, seed, out))
    return list(out)


def bhac_ct_ring_faces_host(grid, owned):
    """The library's ring-face maps applied on the host to the owned faces of
    a constrained-transport grid: per active d, (nb, nz', ny', nx') arrays
    with the ring one face outside each block (no device work)."""
    d = desc_of(grid)
    blocks = blocks_of(grid)
    owned = np.ascontiguousarray(owned, dtype=np.float64)
    ext = [[grid.nx[e] + (1 if e == dd else (2 if e < grid.ndim else 0)) for e in range(3)] for dd in range(grid.ndim)]
    per = [int(np.prod(x)) for x in ext]
    out = np.zeros(grid.nb * sum(per))
    _check("bhac_ct_ring_faces_host", lib().bhac_ct_ring_faces_host(
        C.byref(d), blocks, grid.nb, owned.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p)))
    blk = out.reshape(grid.nb, sum(per))
    res, o = [], 0
    for x, n in zip(ext, per):
        res.append(blk[:, o:o + n].reshape(grid.nb, x[2], x[1], x[0]))
        o += n
    return res


def bhac_measure_peaks(iters: int = 1 << 14, stream_ptr: int = 0):
    """Arithmetic throughput of the current device (see the header)."""
    out = (C.c_double * 8)()
    _check("bhac_measure_peaks", lib().bhac_measure_peaks(iters, C.c_void_p(stream_ptr), out))
    return {"fp64_flops": out[0], "fp32_flops": out[1], "fp64_div": out[2], "fp64_sqrt": out[3],
            "fp64_rsqrt": out[4], "sms": int(out[5]), "ctas": int(out[6]), "threads": int(out[7])}


def bhac_launches_per_step(ctx) -> int:
    n = C.c_int(0)
    _check("bhac_launches_per_step", lib().bhac_launches_per_step(ctx, C.byref(n)))
    return n.value


def bhac_graph_capture(ctx, nsteps: int):
    return _check("bhac_graph_capture", lib().bhac_graph_capture(ctx, nsteps))


def bhac_graph_launch(ctx):
    return _check("bhac_graph_launch", lib().bhac_graph_launch(ctx))


def bhac_cfl_dt_static(desc: GridDesc, blocks, prims_ptr: int, dt_ptr: int, stream_ptr: int):
    """Allocation-free CFL step: device primitives in, device dt out."""
    return _check("bhac_cfl_dt_static", lib().bhac_cfl_dt_static(
        C.byref(desc), blocks, len(blocks), C.c_void_p(prims_ptr), C.c_void_p(dt_ptr), C.c_void_p(stream_ptr)))


def bhac_destroy(ctx):
    lib().bhac_destroy(ctx)


def bhac_status_string(st: int) -> str:
    return status_string(st)


# ---- convenience wrapper ----

def desc_of(grid, precision: str = "fp64") -> GridDesc:
    d = GridDesc()
    d.ndim = grid.ndim
    for k in range(3):
        d.nx[k] = grid.nx[k]
        d.nroot[k] = grid.nroot[k]
        d.xmin[k] = grid.xmin[k]
        d.xmax[k] = grid.xmax[k]
        d.bc[k][0] = BCS[grid.bc[k][0]]
        d.bc[k][1] = BCS[grid.bc[k][1]]
    d.nghost = grid.ng
    d.nlevels = grid.nlevels
    d.coords = COORDS[grid.coords]
    d.spin = grid.spin
    d.mass = grid.mass
    d.recon = RECON[grid.recon]
    d.riemann = RIEMANN[grid.riemann]
    d.precision = PREC[precision]
    d.gamma_ad = grid.gamma_ad
    d.cfl = grid.cfl
    d.ch = grid.ch
    d.kappa = grid.kappa
    d.c2p_tol = grid.c2p_tol
    d.c2p_maxit = grid.c2p_maxit
    d.rho_floor = grid.rho_floor
    d.rho_floor_pow = grid.rho_floor_pow
    d.p_floor = grid.p_floor
    d.p_floor_pow = grid.p_floor_pow
    d.w_max = grid.w_max
    d.divb = 1 if getattr(grid, "divb", "glm") == "ct" else 0
    d.imex = 1 if getattr(grid, "imex", False) else 0
    d.c2p_solver = {"newton": 0, "nk": 1}[getattr(grid, "c2p", "newton")]
    return d


def blocks_of(grid):
    arr = (BlockDesc * grid.nb)()
    for n, (lev, ix, iy, iz) in enumerate(np.asarray(grid.blocks)):
        arr[n].level, arr[n].ix, arr[n].iy, arr[n].iz = int(lev), int(ix), int(iy), int(iz)
    return arr


class Solver:
    """A grid on the current CUDA device: arena from torch, stream from torch.
    The library launches on the device current at each call, so the arena,
    the stream and the calls all belong to that device (select it with
    torch.cuda.set_device first; one process per GPU)."""

    def __init__(self, grid, precision: str = "fp64", device=None, stream=None):
        import torch

        self.torch = torch
        self.grid = grid
        self.precision = precision
        cur = torch.device("cuda", torch.cuda.current_device())
        self.device = cur if device is None else torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if self.device != cur:
            raise ValueError(f"Solver device {self.device} is not the current CUDA device {cur}; "
                             "call torch.cuda.set_device first")
        if stream is not None and stream.device != self.device:
            raise ValueError(f"stream on {stream.device}, solver on {self.device}")
        self.desc = desc_of(grid, precision)
        self.blocks = blocks_of(grid)
        self.nbytes = bhac_query_sizes(self.desc, self.blocks)
        self.arena = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        self.base = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = bhac_init_grid(self.desc, self.blocks, self.base, self.nbytes, self.stream.cuda_stream)
        bhac_set_metric(self.ctx, self.desc.coords, grid.spin, grid.mass)
        self.shape = (grid.nb, NV, grid.nx[2], grid.nx[1], grid.nx[0])

    def close(self):
        if getattr(self, "ctx", None):
            # the arena returns to PyTorch's allocator with the tensor, so the
            # kernels and transfers still reading or writing it finish first
            bhac_host_fence(self.ctx)
            self.stream.synchronize()
            bhac_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_prims(self, prims):
        torch = self.torch
        if isinstance(prims, torch.Tensor) and prims.is_cuda:
            t = prims.to(torch.float64).contiguous()
            bhac_set_prims(self.ctx, t.data_ptr(), True)
            self.stream.synchronize()
        else:
            a = np.ascontiguousarray(prims, dtype=np.float64)
            assert a.size == int(np.prod(self.shape))
            bhac_set_prims(self.ctx, a.ctypes.data, False)

    def prims(self) -> np.ndarray:
        out = np.empty(self.shape)
        bhac_get_prims(self.ctx, out.ctypes.data, False)
        return out

    def _pinned(self, t):
        torch = self.torch
        if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.is_pinned()
                and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == self.shape):
            raise ValueError(f"expected a contiguous pinned CPU float64 tensor of shape {self.shape}")
        return t.data_ptr()

    def set_prims_host_async(self, host):
        """Enqueues a load of the primitives from a pinned CPU tensor; the copy
        overlaps kernels already enqueued (see bhac_set_prims_host_async)."""
        bhac_set_prims_host_async(self.ctx, self._pinned(host))

    def get_prims_host_async(self, host):
        """Enqueues a read-back of the primitives into a pinned CPU tensor; the
        copy overlaps kernels enqueued afterwards."""
        bhac_get_prims_host_async(self.ctx, self._pinned(host))

    def host_fence(self):
        """Orders the copy streams and the solver's stream both ways."""
        bhac_host_fence(self.ctx)

    def c2p_status(self) -> np.ndarray:
        """Per interior cell (blocks, nz, ny, nx): the last stage's inversion outcome."""
        g = self.grid
        out = np.zeros((g.nb, g.nx[2], g.nx[1], g.nx[0]), dtype=np.uint8)
        bhac_get_c2p_status(self.ctx, out.ctypes.data, False)
        return out

    def set_cons(self, cons):
        """Replaces the conserved state derived by set_prims (densitized, as cons() returns it)."""
        c = np.ascontiguousarray(cons, dtype=np.float64)
        bhac_set_cons(self.ctx, c.ctypes.data, False)

    def checkpoint(self) -> dict:
        """The state a bit-identical resume needs: primitives and conserved variables."""
        return {"prims": self.prims(), "cons": self.cons()}

    def restore(self, state: dict):
        """Resumes from checkpoint(): the next steps are bit-identical to an uninterrupted run."""
        self.set_prims(state["prims"])
        self.set_cons(state["cons"])

    def set_faces(self, faces):
        """Face fields Phi^d = sqrt(gamma) B^d (constrained transport), owned
        faces per block and direction (problems.ct layout); call after set_prims."""
        a = np.ascontiguousarray(faces, dtype=np.float64)
        bhac_set_faces(self.ctx, a.ctypes.data, False)

    def faces(self) -> np.ndarray:
        n = self.grid.nb * sum(int(np.prod([self.grid.nx[e] + (e == d) for e in range(3)]))
                               for d in range(self.grid.ndim))
        out = np.empty(n)
        bhac_get_faces(self.ctx, out.ctypes.data, False)
        return out

    def estimate(self, eps: float = 0.01) -> np.ndarray:
        """Loehner's estimator on the density, maximum per block (bhac_estimate)."""
        return bhac_estimate(self.ctx, eps, self.grid.nb)

    def regridded(self, new_blocks):
        """A new Solver on the leaf list new_blocks (same descriptor, device and
        stream) holding the conservative transfer of this one's state."""
        g = self.grid.with_(blocks=np.asarray(new_blocks, dtype=np.int32).reshape(-1, 4))
        fresh = Solver(g, self.precision, device=self.device, stream=self.stream)
        bhac_regrid_transfer(self.ctx, fresh.ctx)
        return fresh

    def prims_ghosted(self) -> np.ndarray:
        """FP64 primitives with ghost cells, (blocks, 9, Nz, Ny, Nx) (FP64 form)."""
        g = self.grid
        gd = [g.ng if d < g.ndim else 0 for d in range(3)]
        out = np.zeros((g.nb, NV, g.nx[2] + 2 * gd[2], g.nx[1] + 2 * gd[1], g.nx[0] + 2 * gd[0]))
        bhac_get_prims_ghosted(self.ctx, out.ctypes.data, False)
        return out

    def cons(self) -> np.ndarray:
        out = np.empty(self.shape)
        bhac_get_cons(self.ctx, out.ctypes.data, False)
        return out

    def prims_device(self, out=None):
        torch = self.torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        bhac_get_prims(self.ctx, out.data_ptr(), True)
        return out

    def fill_ghosts(self):
        bhac_fill_ghosts(self.ctx)

    def cfl_dt(self) -> float:
        return bhac_cfl_dt(self.ctx, True)

    def step(self, dt: float = 0.0):
        bhac_step(self.ctx, dt)

    def stage(self, stage: int, dt: float):
        bhac_stage(self.ctx, stage, dt)

    def diagnostics(self):
        return bhac_get_diagnostics(self.ctx)[0]

    def count_flops(self, dt: float, nsamples: int = 2000, seed: int = 1):
        return bhac_count_flops(self.ctx, dt, nsamples, seed)

    def launches_per_step(self) -> int:
        return bhac_launches_per_step(self.ctx)

    def capture(self, nsteps: int):
        bhac_graph_capture(self.ctx, nsteps)

    def replay(self):
        bhac_graph_launch(self.ctx)

    def set_launch(self, tx=0, ty=0, threads=0, persistent=0, min_ctas=0, producer_warps=0):
        bhac_set_launch(self.ctx, tx, ty, threads, persistent, min_ctas, producer_warps)

    def set_split(self, chunks: int):
        """Split form of the stage in `chunks` chunks (0: the fused kernel)."""
        bhac_set_split(self.ctx, chunks)

    def set_zsplit(self, parts: int):
        """Z parts per (block, tile) work item (0: the library's choice)."""
        bhac_set_zsplit(self.ctx, parts)

    def zsplit_in_force(self) -> int:
        return bhac_zsplit_in_force(self.ctx)


# Fail loudly at import if the library cannot be loaded.
lib()
