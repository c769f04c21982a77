"""Launch-shape autotuner for the stage kernel.

Candidates are CTA tiles (tx, ty) that divide the block, threads per CTA,
the register bound of the 3-D kernel (one or two resident CTAs per SM) and
the persistent work-queue schedule.  Each candidate is timed on the caller's
own grid and state with CUDA events over a few device-dt steps; the fastest
is applied and cached in a JSON file keyed by GPU name, block shape, level
count, dimensionality and precision, so later runs skip the search.  Every
candidate gives bit-identical results (the launch shape changes only the
order in which blocks are visited), so tuning never changes the answer.
"""
from __future__ import annotations

import json
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
SMEM_LIMIT = 226 * 1024
TWO_CTA_SMEM = 113 * 1024  # per CTA, two CTAs on one SM
# names the stage kernel's shared-memory design; cached shapes of another
# design are not reused
KERNEL_TAG = "edge-staged"


def smem_bytes(tx: int, ty: int, ndim: int, precision: str, producers: int = 0) -> int:
    """Dynamic shared memory of the stage kernel (the library's own sizing)."""
    t = 4 if precision == "mixed" else 8
    sfx, sfy, sfz = ty * (tx + 1), (ty + 1) * tx, tx * ty
    if ndim == 3 and producers:
        return 9 * (2 * sfx + 2 * sfy + 3 * sfz) * t
    n = sfx + sfy + 2 * (tx + 2) * ty + 2 * tx * (ty + 2)
    if ndim == 3:
        n += 3 * sfz
    return 9 * n * t


def candidates(grid, precision: str, include_ws: bool = False):
    """Launch shapes to time.  160 threads (one-CTA register bound) lets two
    CTAs of a ~190-register build share an SM with fewer idle threads in the
    last round of a phase than 128 or 256.  The warp-specialised form measured
    slower on every grid tried and is timed only on request."""
    nx, ny = grid.nx[0], grid.nx[1]
    tiles = [(tx, ty) for tx in (32, 16, 8) for ty in (16, 8, 4) if nx % tx == 0 and ny % ty == 0 and tx * ty >= 64]
    if not tiles:
        tiles = [(nx, ny)]
    out = []
    for tx, ty in tiles:
        if smem_bytes(tx, ty, grid.ndim, precision) > SMEM_LIMIT:
            continue
        for threads in (256, 160, 128):
            if threads > 2 * tx * ty:
                continue
            for minb in ((1, 2) if grid.ndim == 3 and threads != 160 else (1,)):
                out.append((tx, ty, threads, 0, minb, 0))
    # the warp-specialised form (3-D): producer warps feed consumer warps
    if grid.ndim == 3 and include_ws:
        for tx, ty in tiles:
            for prod in (2, 4):
                if smem_bytes(tx, ty, 3, precision, prod) > SMEM_LIMIT:
                    continue
                for minb in (1, 2):
                    out.append((tx, ty, 256, 0, minb, prod))
    return out


def key_of(grid, precision: str) -> str:
    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return (f"{name}|{KERNEL_TAG}|nx={grid.nx[0]}x{grid.nx[1]}x{grid.nx[2]}|ndim={grid.ndim}"
            f"|levels={grid.nlevels}|{precision}|{grid.recon}")


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_shape(solver, prims, shape, steps: int = 2) -> float:
    """ms per step of `shape` on the solver's grid (device dt)."""
    import torch
    solver.set_launch(*shape)
    solver.set_prims(prims)
    solver.cfl_dt()
    solver.step(0.0)  # warm-up (first use of a kernel variant configures it)
    torch.cuda.synchronize()
    st = solver.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(steps):
            solver.step(0.0)
        e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(solver, prims, cache_path: str = DEFAULT_CACHE, steps: int = 2, force: bool = False):
    """Picks and applies the fastest launch shape for `solver` (a Solver).
    Returns (shape, table) where table maps each tried shape to ms per step
    (empty when the cache already had the answer)."""
    grid, precision = solver.grid, solver.precision
    cache = load_cache(cache_path)
    key = key_of(grid, precision)
    if not force and key in cache:
        shape = tuple(cache[key]["shape"])
        solver.set_launch(*shape)
        return shape, {}
    table = {}
    for shape in candidates(grid, precision):
        table[shape] = time_shape(solver, prims, shape, steps)
    best = min(table, key=table.get)
    # the persistent work queue for the best tile, one and two CTAs per SM slot
    for k in (1, 2):
        shape = (best[0], best[1], best[2], k, best[4], best[5])
        table[shape] = time_shape(solver, prims, shape, steps)
    best = min(table, key=table.get)
    cache[key] = {"shape": list(best), "ms_per_step": table[best],
                  "tried": {",".join(map(str, s)): ms for s, ms in table.items()}}
    save_cache(cache, cache_path)
    solver.set_launch(*best)
    return best, table


def cached_or_default(solver, cache_path: str = DEFAULT_CACHE):
    """Applies the cached shape for this grid and form if there is one;
    otherwise keeps the library's default.  Returns the shape in force."""
    cache = load_cache(cache_path)
    key = key_of(solver.grid, solver.precision)
    if key in cache:
        shape = tuple(cache[key]["shape"])
        solver.set_launch(*shape)
        return shape
    # the library's own default (the rule of bhac_init_grid)
    nx, ny = solver.grid.nx[0], solver.grid.nx[1]
    two = solver.grid.ndim == 3 and solver.precision == "mixed"
    for tx, ty in ((32, 16), (16, 16), (16, 8), (8, 8)):
        if two and tx * ty > 256:
            continue
        limit = TWO_CTA_SMEM if two else SMEM_LIMIT
        if nx % tx == 0 and ny % ty == 0 and smem_bytes(tx, ty, solver.grid.ndim, solver.precision) <= limit:
            return (tx, ty, 256, 0, 2 if two else 1, 0)
    return (nx, ny, 256, 0, 1, 0)
