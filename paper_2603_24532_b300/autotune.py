"""Launch-shape autotuner for the batched VEGAS iteration.

Times one iteration of the caller's own batch for every compiled kernel shape
(threads per block x minimum resident blocks, i.e. a register cap) and every
candidate samples-per-thread, optionally refines samples-per-thread order by
order for a batch of several orders, restoring every integral's state (grid,
sums, iteration counter) after each trial so tuning leaves no trace in the
results, and leaves the fastest setting on the context.
"""
from __future__ import annotations

from typing import Dict, Iterable, Optional, Sequence

import numpy as np

from . import mbpt as M

DEFAULT_SPT = (8, 16, 32, 64, 128)


def _time_batch(ctx, diags, states, trials):
    M.mbpt_vegas_iterate(ctx, diags, 1)          # graph capture, first-touch
    ms = []
    for _ in range(trials):
        M.mbpt_vegas_iterate(ctx, diags, 1)
        it_ms, fin_ms = M.mbpt_ctx_last_timing(ctx)
        ms.append(it_ms + fin_ms)
    for g, st in zip(diags, states):
        M.mbpt_set_state(g, st)
    return float(np.median(ms))


def autotune(ctx, diags: Sequence, spts: Iterable[int] = DEFAULT_SPT, variants: Optional[Sequence] = None,
             trials: int = 2, orders: Iterable[int] = (2, 3, 4, 5, 6),
             per_order: Optional[Iterable[int]] = None) -> Dict:
    """Search the kernel shape and one samples-per-thread value for all orders; then, for each order
    in per_order (the orders present in a mixed batch), search that order's samples per thread alone
    with the others held at their best (per_order_table, per_order_spt in the result)."""
    if not diags:
        raise ValueError("autotune needs a non-empty batch")
    spts = tuple(spts)
    orders = tuple(orders)
    states = [M.mbpt_get_state(g) for g in diags]
    table, per_order_table, per_order_spt = [], [], {}
    try:
        for tpb, minb in (variants or M.mbpt_kernel_variants()):
            M.mbpt_ctx_set_kernel(ctx, tpb, minb)
            for spt in spts:
                for o in orders:
                    M.mbpt_ctx_set_launch(ctx, o, spt)
                table.append({"threads": tpb, "min_blocks": minb, "spt": spt,
                              "ms": _time_batch(ctx, diags, states, trials)})
        best = min(table, key=lambda r: r["ms"])
        M.mbpt_ctx_set_kernel(ctx, best["threads"], best["min_blocks"])
        for o in orders:
            M.mbpt_ctx_set_launch(ctx, o, best["spt"])
        for o in (per_order or ()):
            trial = []
            for spt in spts:
                M.mbpt_ctx_set_launch(ctx, o, spt)
                ms = _time_batch(ctx, diags, states, trials)
                trial.append((ms, spt))
                per_order_table.append({"order": o, "spt": spt, "ms": ms})
            per_order_spt[o] = min(trial)[1]
            M.mbpt_ctx_set_launch(ctx, o, per_order_spt[o])
    finally:
        for g, st in zip(diags, states):
            M.mbpt_set_state(g, st)
    return {"best": best, "table": table, "per_order_table": per_order_table, "per_order_spt": per_order_spt}
