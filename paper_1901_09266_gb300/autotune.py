"""Autotuner for the fused kernel's launch shape.

Sweeps CTA size, CTAs per SM and the cap on resident CTAs (which sets how many
days each CTA drains from the work queue), times a short solve of the loaded
days for each with the library's own CUDA-event kernel timer, keeps the
fastest, and caches it in a JSON file keyed by the problem's signature.  The
solver state is saved before and restored after the sweep, and results do not
depend on the launch shape (each day is solved by one CTA and link-flow sums
are exact), so tuning changes only speed.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional

from .dode import DodeError

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dode_autotune.json")

# (block_threads, ctas_per_sm, max_ctas as a fraction of the SM count; 0 = all)
DEFAULT_CANDIDATES = [
    (1024, 1, 0), (768, 1, 0), (512, 1, 0), (512, 2, 0), (384, 2, 0), (256, 3, 0), (256, 4, 0),
    (1024, 1, 0.5), (512, 2, 0.5),
]


def signature(ctx) -> str:
    """Problem signature: sizes, precision, form and a power-of-two day bucket."""
    d = max(1, int(ctx.D))
    bucket = 1 << (d - 1).bit_length()
    return (f"N{ctx.N}-A{ctx.A}-O{ctx.O}-K{ctx.K}-P{ctx.P}-D{bucket}-"
            f"prec{int(ctx.opt.precision)}-form{int(ctx.opt.form)}")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(ctx, iters: int = 3, step: float = 5.0, n_sm: int = 152,
         candidates: Optional[Iterable] = None, cache_path: Optional[str] = DEFAULT_CACHE,
         force: bool = False) -> dict:
    """Pick and apply the fastest launch shape for ``ctx``'s loaded days.

    Returns {"block": b, "ctas_per_sm": c, "max_ctas": m, "ms": t, "cached": bool,
    "tried": [...]}.
    """
    key = signature(ctx)
    cache = _load(cache_path) if cache_path else {}
    if not force and key in cache:
        best = dict(cache[key])
        ctx.set_launch(best["block"], best["ctas_per_sm"], best["max_ctas"])
        best["cached"] = True
        return best
    q, G = ctx.get_state()
    tried = []
    for blk, cps, frac in (candidates or DEFAULT_CANDIDATES):
        maxc = int(round(frac * n_sm * cps)) if frac else 0
        try:
            ctx.set_launch(blk, cps, maxc)
            ctx.solve(1, step)                       # warm-up (and shared-memory attribute)
            ctx.set_state(q, G)
            ctx.solve(iters, step)
            ms = float(ctx.last_kernel_ms())
        except DodeError as e:                      # shape does not fit this problem
            tried.append({"block": blk, "ctas_per_sm": cps, "max_ctas": maxc, "error": str(e)})
            continue
        finally:
            ctx.set_state(q, G)
        tried.append({"block": blk, "ctas_per_sm": cps, "max_ctas": maxc, "ms": ms})
    ok = [t for t in tried if "ms" in t]
    if not ok:
        raise DodeError(-10, "no candidate launch shape fits this problem")
    best = min(ok, key=lambda t: t["ms"])
    ctx.set_launch(best["block"], best["ctas_per_sm"], best["max_ctas"])
    if cache_path:
        cache = _load(cache_path)
        cache[key] = {k: best[k] for k in ("block", "ctas_per_sm", "max_ctas", "ms")}
        _save(cache_path, cache)
    return {**best, "cached": False, "tried": tried}
