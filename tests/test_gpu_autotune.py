"""Autotuner and kernel shapes: every compiled shape gives the same iteration (to FP64
summation-order rounding), tuning restores the integrals' states bit for bit, and a
tuned context is deterministic."""
import numpy as np
import pytest

import oracle as O
from helpers import make_desc, matter_pair, random_grid
from paper_2603_24532_b300 import autotune as A
from paper_2603_24532_b300 import mbpt as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = M.mbpt_ctx_create(0, 1 << 30)
    yield c
    M.mbpt_ctx_destroy(c)


def _batch(ctx):
    po, pm = matter_pair("pnm")
    ps, pms = matter_pair("snm")
    gs = []
    for n, k, p in ((2, 1, pm), (3, 3, pm), (4, 3, pms), (5, 2, pm)):
        for D in O.enumerate_diagrams(n)[:k]:
            if O.is_anomalous(D):
                continue
            gs.append(M.mbpt_create_diagram(ctx, make_desc(D), p, M.vegas_cfg(
                samples=30011 + D.diagram_id, seed=9, stream_id=1000 * n + D.diagram_id, precision=M.MBPT_FP64)))
    return gs


def test_all_shapes_agree_and_tuning_restores_state(ctx):
    gs = _batch(ctx)
    rng = np.random.default_rng(3)
    try:
        for g in gs:
            img = M.mbpt_get_state(g)
            d = int(np.frombuffer(img, dtype=np.int32, count=3, offset=8)[0])
            M.mbpt_set_state(g, M.state_with_grid(img, random_grid(d, 50, rng, strength=0.5)))
        before = [M.mbpt_get_state(g) for g in gs]
        means = {}
        for tpb, minb in M.mbpt_kernel_variants():
            for spt in (8, 64):
                M.mbpt_ctx_set_kernel(ctx, tpb, minb)
                for o in (2, 3, 4, 5):
                    M.mbpt_ctx_set_launch(ctx, o, spt)
                M.mbpt_vegas_iterate(ctx, gs, 1)
                means[(tpb, minb, spt)] = np.array([r.last_mean for r in M.mbpt_estimate_batch(gs)])
                for g, st in zip(gs, before):
                    M.mbpt_set_state(g, st)
        ref = means[(256, 2, 8)]
        for k, v in means.items():
            assert np.allclose(v, ref, rtol=1e-12, atol=0.0), k
        res = A.autotune(ctx, gs, spts=(16, 32), trials=1, per_order=())
        assert [M.mbpt_get_state(g) for g in gs] == before
        b = res["best"]
        assert M.mbpt_ctx_get_launch(ctx, 3) == (b["threads"], b["min_blocks"], b["spt"])
        assert len(res["table"]) == 2 * len(M.mbpt_kernel_variants())
        # the histogram layout was searched on the best shape and the chosen one is on the context
        assert len(res["layout_table"]) == 2
        want = M.MBPT_HIST_BLOCK_F64 if res["launch"]["hist_layout"] == "block_f64" else M.MBPT_HIST_WARP_F32
        assert M.mbpt_ctx_get_hist_layout(ctx) == want
        # so was the Goldstone-sum strategy
        assert len(res["spin_table"]) == 2
        want = M.MBPT_SPIN_FOLD if res["launch"]["spin_sum"] == "fold" else M.MBPT_SPIN_TABLE
        assert M.mbpt_ctx_get_spin_sum(ctx) == want
        M.mbpt_ctx_set_spin_sum(ctx, M.MBPT_SPIN_TABLE)
        assert sorted(res["launch"]["spt_by_order"]) == [2, 3, 4, 5]
        M.mbpt_ctx_set_hist_layout(ctx, M.MBPT_HIST_WARP_F32)
        # per-order refinement of a mixed-order batch: one entry per (order, candidate), the chosen
        # values left on the context, the states untouched
        res = A.autotune(ctx, gs, spts=(16, 32), trials=1, variants=[(256, 2)], per_order=(3, 5),
                         layouts=(M.MBPT_HIST_WARP_F32,))
        assert [M.mbpt_get_state(g) for g in gs] == before
        assert len(res["per_order_table"]) == 4 and set(res["per_order_spt"]) == {3, 5}
        for o, spt in res["per_order_spt"].items():
            assert M.mbpt_ctx_get_launch(ctx, o) == (256, 2, spt)
        # by default a batch of several orders is refined order by order
        res = A.autotune(ctx, gs, spts=(16, 32), trials=1, variants=[(256, 2)], layouts=(M.MBPT_HIST_WARP_F32,))
        assert set(res["per_order_spt"]) == {2, 3, 4, 5} and len(res["per_order_table"]) == 8
        assert [M.mbpt_get_state(g) for g in gs] == before
        # deterministic under the tuned shape
        M.mbpt_vegas_iterate(ctx, gs, 2)
        r1 = [r.as_dict() for r in M.mbpt_estimate_batch(gs)]
        for g, st in zip(gs, before):
            M.mbpt_set_state(g, st)
        M.mbpt_vegas_iterate(ctx, gs, 2)
        r2 = [r.as_dict() for r in M.mbpt_estimate_batch(gs)]
        assert r1 == r2
    finally:
        for g in gs:
            M.mbpt_destroy_diagram(g)
    with pytest.raises(M.MbptError):
        M.mbpt_ctx_set_kernel(ctx, 96, 1)
    with pytest.raises(M.MbptError):
        M.mbpt_ctx_set_spin_sum(ctx, 2)
