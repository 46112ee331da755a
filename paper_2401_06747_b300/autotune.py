"""Autotuner for the solver parameters that set speed but not the result.

The inpainting and tonal solves stop at the same relative residual whatever
the Robin weight of the ORAS interfaces, the local CG stop fractions, the
inner-solve tolerances or the kernels' tiling are, so these can be chosen per
GPU and problem class by timing: each candidate set runs the real solve
(through the C ABI) on a representative input, the fastest one that
converges wins. Two stages: first the tiling and layout choices (the ORAS
subdomain layout -- one warp or two per 32x32 subdomain --, the rows per warp
of the streaming strip kernels, and for tonal optimisation the RAS block
side, 32 or 64, the sweep size below which the ORAS sweep keeps two warps per
subdomain, and which level-0 kernels stage their rows in shared memory), then
the scalar parameters with the best tiling. Results are
kept in a JSON cache keyed by GPU name, size class, channel count,
mask-density bucket and solve kind, and applied by creating a Context with
them.

    best = tune(ctx_device, f, mask, kind="inpaint")      # dict of parameters
    ctx = Context(0, **best)
"""

from __future__ import annotations

import json
import math
import os

# candidate grids (every value is accepted by hdi_set_param)
INPAINT_GRID = {
    "oras_theta": (0.2, 0.3, 0.45),
    "oras_eta": (1e-2, 1e-3),
    "coarse_level_eta": (0.1, 0.3),
}
TONAL_GRID = {
    "tonal_oras_eta": (1e-2, 3e-2),
    "tonal_inner_ratio": (0.05, 0.1, 0.2),
    "tonal_fine_pre": (1, 2),
    "tonal_echo_rtol": (3e-3, 1e-2),
}
# tiling and layout (stage 1); strip_rows 0 = chosen by level size
INPAINT_SHAPES = {
    "oras_warp": (0, 1),
    "oras_warp_waves": (0, 2, 8),
    "stage_loads": (0, 3),
    "strip_rows": (0, 8, 16),
}
TONAL_SHAPES = {
    "oras_warp": (0, 1),
    "oras_warp_waves": (2, 8),
    "stage_loads": (0, 3),
    "strip_rows": (0, 16),
    "tonal_block": (32, 64),
}


def size_class(h: int, w: int) -> str:
    """Pixel count rounded to the nearest power of two (e.g. '2^23')."""
    return f"2^{int(round(math.log2(max(h * w, 1))))}"


def density_bucket(d: float) -> str:
    """Mask density rounded to the nearest power of two in percent."""
    return f"{2.0 ** round(math.log2(max(d, 1e-6) * 100)):g}%"


def cache_key(gpu: str, h: int, w: int, ch: int, density: float, kind: str) -> str:
    return "|".join([gpu, size_class(h, w), f"c{ch}", density_bucket(density), kind])


def candidates(grid: dict) -> list:
    """All combinations of a grid, in a fixed order."""
    out = [{}]
    for name in sorted(grid):
        out = [dict(c, **{name: v}) for c in out for v in grid[name]]
    return out


def load_cache(path: str) -> dict:
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def save_cache(path: str, cache: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(device: int, f, mask, kind: str = "inpaint", tol: float = 1e-6, reps: int = 2,
         cache_path: str | None = None, grid: dict | None = None, shapes: dict | None = None) -> dict:
    """Fastest converging parameter set for solves like (f, mask).

    f, mask: device tensors as for Context.inpaint / tonal_opt. Every
    candidate runs one untimed solve and then `reps` timed ones (CUDA events
    on the current stream); candidates that do not reach `tol` are dropped.
    Stage 1 times the tiling grid `shapes` (default INPAINT_SHAPES /
    TONAL_SHAPES; {} skips it), stage 2 the parameter grid `grid` with the
    best tiling. With `cache_path` the result is read from / stored in that
    JSON file."""
    import torch

    H, W = int(mask.shape[-2]), int(mask.shape[-1])
    ch = 1 if f.dim() == 2 else int(f.shape[0])
    density = float(mask.float().mean().item())
    key = cache_key(torch.cuda.get_device_name(device), H, W, ch, density, kind)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache:
        return dict(cache[key]["params"])
    if shapes is None:
        shapes = INPAINT_SHAPES if kind == "inpaint" else TONAL_SHAPES
    grid = grid or (INPAINT_GRID if kind == "inpaint" else TONAL_GRID)
    table = []
    base = {}
    if shapes:
        base, _, t1 = _search(device, f, mask, kind, tol, reps, candidates(shapes), {})
        table += [dict(row, stage="tiling") for row in t1]
    best, best_ms, t2 = _search(device, f, mask, kind, tol, reps, candidates(grid), base)
    table += [dict(row, stage="parameters") for row in t2]
    if cache_path:
        cache[key] = {"params": best, "ms": round(best_ms, 3), "table": table}
        save_cache(cache_path, cache)
    return dict(best)


def _search(device, f, mask, kind, tol, reps, cands, base):
    """Times every candidate (merged over `base`); returns the fastest
    converging set, its time and the table of all candidates."""
    import torch
    from . import Context
    stream = torch.cuda.current_stream(device)
    out = torch.empty_like(f)
    best, best_ms, table = None, math.inf, []
    for c in cands:
        cand = dict(base, **c)
        ctx = Context(device, stream=stream, **cand)
        run = (lambda: ctx.inpaint(f, mask, out, tol=tol, allow_not_converged=True)) if kind == "inpaint" else \
              (lambda: ctx.tonal_opt(f, mask, out, tol=tol, allow_not_converged=True))
        st = run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            st = run()
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1) / reps
        ok = st["rel_res"] <= tol
        table.append({"params": cand, "ms": round(ms, 3), "converged": ok})
        if ok and ms < best_ms:
            best, best_ms = cand, ms
        ctx.close()
    if best is None:
        raise RuntimeError("no candidate parameter set converged")
    return best, best_ms, table
