"""Launch autotuner for the batched VEGAS iteration.

Times one iteration of the caller's own batch for every compiled kernel shape
(threads per block x minimum resident blocks, i.e. a register cap) and every
candidate samples-per-thread; then, on the best shape, the per-chunk histogram
layout (warp-private FP32 bins or one block-shared FP64 histogram), the
Goldstone-sum strategy of the mixed modes (product table or vertex-by-vertex
fold) and, for a batch of several orders, samples-per-thread order by order.  Every integral's
state (grid, sums, iteration counter) is restored after each trial, so tuning
leaves no trace in the results, and the fastest setting is left on the context.
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


def batch_orders(states) -> list:
    """The orders present in a batch, read from the integrals' state images (header word 4)."""
    return sorted({int(np.frombuffer(st, dtype=np.int32, count=1, offset=16)[0]) for st in states})


def autotune(ctx, diags: Sequence, spts: Iterable[int] = DEFAULT_SPT, variants: Optional[Sequence] = None,
             trials: int = 2, orders: Iterable[int] = (2, 3, 4, 5, 6), per_order="auto",
             layouts: Iterable[int] = (M.MBPT_HIST_WARP_F32, M.MBPT_HIST_BLOCK_F64),
             spin_sums: Iterable[int] = (M.MBPT_SPIN_TABLE, M.MBPT_SPIN_FOLD)) -> Dict:
    """Search the kernel shape and one samples-per-thread value for all orders; then the histogram
    layout on that shape (layout_table; the FP64 block layout is taken only if it is faster); then the
    Goldstone-sum strategy (spin_table; the fold is taken only if it is faster); then, for
    each order in per_order -- by default ("auto") the orders present when the batch has more than one --
    that order's samples per thread alone with the others held at their best (per_order_table,
    per_order_spt).  The result's "launch" summarises the chosen setting."""
    if not diags:
        raise ValueError("autotune needs a non-empty batch")
    spts = tuple(spts)
    orders = tuple(orders)
    states = [M.mbpt_get_state(g) for g in diags]
    present = batch_orders(states)
    if per_order == "auto":
        per_order = present if len(present) > 1 else ()
    table, per_order_table, per_order_spt, layout_table, spin_table = [], [], {}, [], []
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
        layout = M.MBPT_HIST_WARP_F32
        for lay in layouts:
            M.mbpt_ctx_set_hist_layout(ctx, lay)
            layout_table.append({"layout": lay, "ms": _time_batch(ctx, diags, states, trials)})
        if layout_table:
            layout = min(layout_table, key=lambda r: r["ms"])["layout"]
        M.mbpt_ctx_set_hist_layout(ctx, layout)
        spin = M.MBPT_SPIN_TABLE
        for sp in spin_sums:
            M.mbpt_ctx_set_spin_sum(ctx, sp)
            spin_table.append({"spin_sum": sp, "ms": _time_batch(ctx, diags, states, trials)})
        if spin_table:
            spin = min(spin_table, key=lambda r: r["ms"])["spin_sum"]
        M.mbpt_ctx_set_spin_sum(ctx, spin)
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
    launch = {"threads": best["threads"], "min_blocks": best["min_blocks"],
              "spt_by_order": {o: M.mbpt_ctx_get_launch(ctx, o)[2] for o in present},
              "hist_layout": "block_f64" if layout == M.MBPT_HIST_BLOCK_F64 else "warp_f32",
              "spin_sum": "fold" if spin == M.MBPT_SPIN_FOLD else "table"}
    return {"best": best, "table": table, "layout_table": layout_table, "spin_table": spin_table,
            "per_order_table": per_order_table, "per_order_spt": per_order_spt, "launch": launch}
