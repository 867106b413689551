"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point the header declares, and its CPU generator reproduces
Table I and the oracle's independent enumeration descriptor for descriptor."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from conftest import ROOT, golden_rows
from paper_2603_24532_b300 import mbpt as M


def header_symbols():
    src = open(os.path.join(ROOT, "include", "mbpt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mbpt_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    L = M.lib()
    syms = header_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(L, s), s


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_generator_counts(n):
    want = {int(r[0]): int(r[1]) for r in golden_rows("table1_counts.txt")}
    assert len(M.mbpt_generate(n)) == want[n]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_generator_matches_oracle_enumeration(n):
    ds = M.mbpt_generate(n)
    Os = O.enumerate_diagrams(n)
    idx = {D.A: k for k, D in enumerate(Os)}
    for d, D in zip(ds, Os):
        assert d.lines() == D.lines
        assert d.ports() == [tuple(p) for p in D.ports]
        assert d.chords() == D.chords
        assert np.array_equal(d.coef(), D.coef())
        assert d.anomalous == O.is_anomalous(D)
        assert d.mirror_id == idx[O.mirror_matrix(D.A)]
        assert bool(d.flags & M.FLAG_SELF_MIRROR) == (O.mirror_matrix(D.A) == D.A)
        assert M.mbpt_hole_chords(d) == O.hole_chords(D)
        assert d.repeated_denominator == O.has_repeated_denominator(D)


def test_generator_argument_errors():
    L = M.lib()
    n = ctypes.c_int(0)
    assert L.mbpt_generate(1, None, 0, ctypes.byref(n)) == M.MBPT_EINVAL
    assert L.mbpt_generate(7, None, 0, ctypes.byref(n)) == M.MBPT_EINVAL
    arr = (M.mbpt_diagram_desc * 2)()
    assert L.mbpt_generate(4, arr, 2, ctypes.byref(n)) == M.MBPT_ENOMEM
    assert n.value == 39


def test_diag_bytes_and_bad_sizes():
    d = M.mbpt_generate(5)[0]
    assert M.mbpt_diag_bytes(d, M.vegas_cfg()) > 18 * 51 * 8
    bad = M.vegas_cfg(n_bins=1000)
    with pytest.raises(M.MbptError):
        M.mbpt_diag_bytes(d, bad)


def test_no_device_fails_cleanly():
    """Without a GPU, creating a context returns an error status (no crash, no fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(M.MbptError):
        M.mbpt_ctx_create(0, 1 << 20)


@pytest.mark.parametrize("kfp", [0.0, 1.2])
def test_hf_self_energy_table_matches_oracle(kfp):
    """The product's Hartree-Fock table (its own quadrature, spline and per-interval cubics) against
    the oracle's spline of its own knot values, at knots, between knots and beyond the table."""
    kfn = 1.2 if kfp else 1.0
    po = O.Physics(kF_n=kfn, kF_p=kfp, K_max=kfn + 6.0, spectrum=1)
    pm = M.physics(kF_n=kfn, kF_p=kfp, K_max=kfn + 6.0, spectrum=1)
    ks = np.concatenate([np.linspace(0.0, 2 * po.K_max * 0.999, 257), [0.3 * po.K_max / 1023, 2 * po.K_max + 0.5]])
    got = M.mbpt_hf_self_energy(pm, ks)
    ref = np.array([O.sp_energy(po, k) - 0.5 * po.hbar2_over_m * k * k for k in ks])
    assert np.max(np.abs(got - ref)) < 1e-11
    assert got[-1] == 0.0


def test_hf_self_energy_rejects_two_fermi_momenta():
    with pytest.raises(M.MbptError):
        M.mbpt_hf_self_energy(M.physics(kF_n=1.2, kF_p=0.8, spectrum=1), [0.5])
