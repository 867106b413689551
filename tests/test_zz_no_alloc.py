"""The allocation-free single-iteration entry point (mbpt_vegas_iteration_noalloc).

The paper has no counterpart to this call.  It exists for callers that must not
allocate device memory once they are running -- a process whose device memory
belongs to another allocator or a fixed budget, or a loop where cudaMalloc's
implicit synchronisation is not acceptable.  Its scratch is one fixed device
array shared by all calls, so the test makes different calls in a row (each
smaller than the one before, so stale slots of an earlier call would show) and
checks each against the arena-backed mbpt_vegas_iterate path on the same grid.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from helpers import make_desc, matter_pair, random_grid
from paper_2603_24532_b300 import mbpt as M

pytestmark = pytest.mark.gpu


def _arena_path(ctx, desc, pm, cfg, grid):
    g = M.mbpt_create_diagram(ctx, desc, pm, cfg)
    try:
        M.mbpt_set_state(g, M.state_with_grid(M.mbpt_get_state(g), grid))
        M.mbpt_vegas_iterate(ctx, [g], 1)
        r = M.mbpt_estimate(g)
        hist = M.state_last_hist(M.mbpt_get_state(g), grid.shape[0], grid.shape[1] - 1)
        return r.last_mean, r.last_sigma, hist
    finally:
        M.mbpt_destroy_diagram(g)


def test_noalloc_matches_iterate_on_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = M.mbpt_ctx_create(0, 1 << 30)
    rng = np.random.default_rng(2024)
    cases = [  # (order, diagram index, matter, precision, samples) -- each call smaller than the one before
        (6, 20000, "pnm", M.MBPT_MIXED, 90001),
        (4, 7, "snm", M.MBPT_MIXED, 70001),
        (3, 1, "pnm", M.MBPT_FP64, 40123),
    ]
    try:
        for order, idx, matter, prec, ns in cases:
            D = O.enumerate_diagrams(order)[idx]
            po, pm = matter_pair(matter)
            cfg = M.vegas_cfg(samples=ns, seed=77, stream_id=5 + idx, precision=prec)
            desc = make_desc(D)
            grid = random_grid(D.d, 50, rng, strength=0.5)
            mean_a, sigma_a, hist_a = _arena_path(ctx, desc, pm, cfg, grid)
            g_dev = torch.tensor(grid, dtype=torch.float64, device="cuda")
            out = torch.full((2 + D.d * 50,), float("nan"), dtype=torch.float64, device="cuda")
            M.mbpt_vegas_iteration_noalloc(0, desc, pm, cfg, 0, g_dev.data_ptr(), out.data_ptr(), 0)
            torch.cuda.synchronize()
            o = out.cpu().numpy()
            mean_b = o[0] / ns
            sigma_b = np.sqrt((o[1] / ns - mean_b ** 2) / (ns - 1))
            hist_b = o[2:].reshape(D.d, 50)
            assert mean_b == pytest.approx(mean_a, rel=1e-12, abs=0.0)
            assert sigma_b == pytest.approx(sigma_a, rel=1e-10, abs=0.0)
            assert np.allclose(hist_b, hist_a, rtol=1e-12, atol=0.0)
        # an invalid descriptor is rejected on the host and leaves the output untouched
        D = O.enumerate_diagrams(4)[7]
        po, pm = matter_pair("pnm")
        bad = make_desc(D)
        bad.chord_line[0] = 40
        out = torch.full((2 + D.d * 50,), 12345.0, dtype=torch.float64, device="cuda")
        g_dev = torch.tensor(O.uniform_grid(D.d, 50), dtype=torch.float64, device="cuda")
        with pytest.raises(M.MbptError) as e:
            M.mbpt_vegas_iteration_noalloc(0, bad, pm, M.vegas_cfg(samples=4096), 0, g_dev.data_ptr(),
                                           out.data_ptr(), 0)
        assert e.value.status == M.MBPT_EINVAL
        torch.cuda.synchronize()
        assert bool(torch.all(out == 12345.0))
        # a request beyond the fixed scratch is rejected with a clear error
        D = O.enumerate_diagrams(5)[3]
        po, pm = matter_pair("pnm")
        big = M.vegas_cfg(samples=(1 << 32) - 1)
        g_dev = torch.tensor(O.uniform_grid(D.d, 50), dtype=torch.float64, device="cuda")
        out = torch.zeros(2 + D.d * 50, dtype=torch.float64, device="cuda")
        with pytest.raises(M.MbptError) as e:
            M.mbpt_vegas_iteration_noalloc(0, make_desc(D), pm, big, 0, g_dev.data_ptr(), out.data_ptr(), 0)
        assert e.value.status == M.MBPT_EINVAL and "samples per call" in str(e.value)
    finally:
        M.mbpt_ctx_destroy(ctx)
