"""Autotuner for the launch shapes of the per-system batched GMRES (tpp_batch_gmres).

Each lane-group width (8, 16 or 32 lanes per system) runs as its own persistent
launch; its shape is a choice of warps per CTA, CTAs per SM and register budget
(the kernel variant compiled for one or two resident 256-thread CTAs per SM).
Every system's arithmetic is the same in every shape, so the choice changes the
time and never the result.  The tuner solves a sample batch once per candidate
shape, reads each width's device time from the report (one CUDA-event pair per
launch) and keeps the fastest shape per width.  Choices are cached in a JSON
file keyed by the GPU, the precision, the restart length and the (dim, n) groups
of the width, so a second run on the same GPU skips the timing.  This module only
sequences calls to the C ABI (through BatchGmres).
"""
from __future__ import annotations

import json
import os

import torch

# (warps per CTA, CTAs per SM (0: as many as fit), register budget)
CANDIDATES = [(8, 0, 1), (4, 0, 1), (8, 0, 2), (4, 0, 2), (2, 0, 2)]


def default_cache_path() -> str:
    return os.environ.get("TPP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache",
                                       "paper_1704_04549_gb300", "batch_gmres.json"))


def _width(n: int) -> int:
    return 0 if n <= 8 else (1 if n <= 16 else 2)


def _keys(contexts, mixed: bool, restart: int, device) -> list:
    name = torch.cuda.get_device_name(device)
    keys = []
    for k in range(3):
        groups = sorted({(c.dim, c.n) for c in contexts if _width(c.n) == k})
        keys.append(None if not groups else
                    f"{name}|{'mixed' if mixed else 'fp64'}|m{restart}|w{(8, 16, 32)[k]}|"
                    + ",".join(f"{d}d{n}" for d, n in groups))
    return keys


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_batch_gmres(contexts, bs, xs, *, mixed: bool = False, restart: int = 20,
                     rtol: float = 1e-8, max_iters: int = 300, inner_rtol: float = 1e-4,
                     max_outer: int = 8, candidates=CANDIDATES, cache_path: str | None = None,
                     use_cache: bool = True) -> dict:
    """Choose the launch shape of every width for these contexts (a representative
    sample of the batch to be solved: same (dim, n) groups, fewer elements).

    bs, xs: right-hand sides and solution buffers of the sample.  Returns
    dict(warps, ctas_per_sm, reg_budget (3-tuples for the 8-, 16-, 32-lane launches),
    table (per candidate: shape and the three launch times in ms), cached (bool))."""
    from .batch import BatchGmres
    device = contexts[0].device
    path = cache_path or default_cache_path()
    keys = _keys(contexts, mixed, restart, device)
    cache = _load(path) if use_cache else {}
    if use_cache and all(k is None or k in cache for k in keys):
        pick = [cache[k] if k else {"warps": 0, "ctas_per_sm": 0, "reg_budget": 0} for k in keys]
        return {"warps": tuple(p["warps"] for p in pick),
                "ctas_per_sm": tuple(p["ctas_per_sm"] for p in pick),
                "reg_budget": tuple(p["reg_budget"] for p in pick), "table": [],
                "cached": True}
    common = dict(restart=restart, rtol=rtol, max_iters=max_iters, mixed=mixed,
                  inner_rtol=inner_rtol, max_outer=max_outer)
    table = []
    for w, c, rb in candidates:
        solver = BatchGmres(contexts, warps=(w,) * 3, ctas_per_sm=(c,) * 3,
                            reg_budget=(rb,) * 3, **common)
        solver.solve(bs, xs)                      # warm-up (first launch of the variant)
        rep = solver.solve(bs, xs)
        table.append({"warps": w, "ctas_per_sm": c, "reg_budget": rb,
                      "launch_ms": rep["launch_ms"]})
        del solver
    best = []
    for k in range(3):
        if keys[k] is None:
            best.append({"warps": 0, "ctas_per_sm": 0, "reg_budget": 0})
            continue
        row = min(table, key=lambda r: r["launch_ms"][k])
        best.append({"warps": row["warps"], "ctas_per_sm": row["ctas_per_sm"],
                     "reg_budget": row["reg_budget"], "ms": row["launch_ms"][k]})
    if use_cache:
        cache = _load(path)
        for k in range(3):
            if keys[k] is not None:
                cache[keys[k]] = best[k]
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return {"warps": tuple(b["warps"] for b in best),
            "ctas_per_sm": tuple(b["ctas_per_sm"] for b in best),
            "reg_budget": tuple(b["reg_budget"] for b in best), "table": table,
            "cached": False}
