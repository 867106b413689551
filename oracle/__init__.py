"""Plain FP64 CPU oracle for the Monte Carlo evaluation of Hugenholtz diagrams.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` import this package.  It shares no
code with the product library (``paper_2603_24532_b300``) and imports nothing
from it.

Contents
--------
* ``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` (ctypes).
* ``enumerate_diagrams(n)`` -- brute-force list of the order-n Hugenholtz
  diagrams with two-body vertices (Table I of arXiv:2603.24532 counts them:
  1, 3, 39, 840, 27300 at n = 2..6) in the canonical line/port/chord convention below.
* ``Diagram`` -- one diagram with the oracle's own derived quantities.
* ``integrand`` / ``vegas_iteration`` / ``refine`` / ``combine`` /
  ``combine_pooled`` -- the per-sample integrand, one VEGAS iteration
  (multi-threaded over sample ranges with a fixed-order reduction), grid
  refinement, and the two iteration combinations: Lepage's inverse-variance
  mean, and the evaluation phase of PVegas (Sec. III.C: training iterations,
  then a frozen grid whose samples all carry the same weight).
* ``discrete_diagram`` and ``rspt_coefficients`` -- the finite-space check of
  the diagram rules against exact Rayleigh-Schroedinger perturbation theory.

Canonical convention for a diagram (the oracle's reading; a product generator
that follows the same written rules must produce the same lists):

1. Vertices 0..n-1 in time order.  The adjacency matrix A[i][j] counts lines
   from vertex i to vertex j (zero diagonal, row and column sums 2, connected).
   Diagrams are ordered lexicographically by the row-major entries of A.
2. Lines are listed by (src, dst) in row-major order of A, A[i][j] copies each.
   src < dst: particle; src > dst: hole.
3. Vertex v is <o1 o2|V|i1 i2> with (o1, o2) the lines leaving v and (i1, i2)
   the lines entering v, each pair in increasing line index.
4. Chords: scan particles (increasing index) then holes (increasing index),
   union-find over vertices; a line that joins two components is a tree line,
   otherwise a chord.  Chords are listed hole chords first, then particle
   chords, each in increasing line index.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(tests/test_oracle_pins.py, tests/test_oracle_rspt.py, tests/test_philox.py,
tests/test_census.py); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lib = None
_lock = threading.Lock()

MAXC = 7
MAXL = 12


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.POINTER
            L.oracle_info_ints.restype = ctypes.c_int
            L.oracle_derive.restype = ctypes.c_int
            L.oracle_derive.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]
            L.oracle_integrand.restype = ctypes.c_double
            L.oracle_integrand.argtypes = [P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
            L.oracle_integrand_momenta.restype = ctypes.c_double
            L.oracle_integrand_momenta.argtypes = [P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double),
                                                   P(ctypes.c_double)]
            L.oracle_line_ksq.restype = None
            L.oracle_line_ksq.argtypes = [P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
            L.oracle_first_order_integrand.restype = ctypes.c_double
            L.oracle_first_order_integrand.argtypes = [P(ctypes.c_double), P(ctypes.c_double)]
            L.oracle_philox4x32_10.restype = None
            L.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            L.oracle_vegas_samples.restype = None
            L.oracle_vegas_samples.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double), ctypes.c_int,
                                               ctypes.c_int, P(ctypes.c_double), ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                               P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                               P(ctypes.c_double)]
            L.oracle_vegas_samples_group.restype = None
            L.oracle_vegas_samples_group.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double),
                                                     P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                                     P(ctypes.c_double), ctypes.c_uint64, ctypes.c_uint32,
                                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                                     P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                                                     P(ctypes.c_double)]
            L.oracle_hf_self_energy.restype = ctypes.c_double
            L.oracle_hf_self_energy.argtypes = [P(ctypes.c_double), ctypes.c_double, ctypes.c_int, ctypes.c_int]
            L.oracle_spline_build.restype = None
            L.oracle_spline_build.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double)]
            L.oracle_spline_eval.restype = ctypes.c_double
            L.oracle_spline_eval.argtypes = [ctypes.c_int, ctypes.c_double, P(ctypes.c_double), P(ctypes.c_double),
                                             ctypes.c_double]
            L.oracle_gauss_legendre.restype = None
            L.oracle_gauss_legendre.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
            L.oracle_refine.restype = None
            L.oracle_refine.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                        P(ctypes.c_double)]
            L.oracle_discrete_diagram.restype = ctypes.c_double
            L.oracle_discrete_diagram.argtypes = [P(ctypes.c_int), ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                                                  P(ctypes.c_double)]
            _lib = L
    return _lib


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------
# Philox4x32-10
# ----------------------------------------------------------------------------
def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return list(o)


# ----------------------------------------------------------------------------
# Diagram enumeration (Table I counts; OEIS A064732)
# ----------------------------------------------------------------------------
def _row_choices(n: int, i: int):
    """All rows of length n with zero at i, entries >= 0, summing to 2."""
    out = []
    others = [j for j in range(n) if j != i]
    for a in others:
        for b in others:
            if b < a:
                continue
            row = [0] * n
            row[a] += 1
            row[b] += 1
            out.append(tuple(row))
    return sorted(set(out))


def _connected(A) -> bool:
    n = len(A)
    seen = {0}
    stack = [0]
    while stack:
        v = stack.pop()
        for u in range(n):
            if (A[v][u] or A[u][v]) and u not in seen:
                seen.add(u)
                stack.append(u)
    return len(seen) == n


def adjacency_matrices(n: int) -> List[tuple]:
    """All n x n matrices (zero diagonal, row/col sums 2, connected), sorted
    lexicographically by their row-major entries."""
    rows = [_row_choices(n, i) for i in range(n)]
    out = []
    for combo in itertools.product(*rows):
        ok = True
        for j in range(n):
            if sum(combo[i][j] for i in range(n)) != 2:
                ok = False
                break
        if ok and _connected(combo):
            out.append(tuple(tuple(r) for r in combo))
    out.sort(key=lambda A: tuple(x for r in A for x in r))
    return out


@dataclass
class Diagram:
    n: int
    A: tuple
    lines: List[tuple]          # (src, dst)
    ports: List[tuple]          # (o1, o2, i1, i2) per vertex
    chords: List[int]
    diagram_id: int = -1
    info: np.ndarray = field(default=None, repr=False)

    @property
    def nl(self) -> int:
        return 2 * self.n

    @property
    def d(self) -> int:
        return 3 * (self.n + 1)

    def hole(self, l: int) -> bool:
        s, t = self.lines[l]
        return s > t

    @property
    def h(self) -> int:
        """number of hole lines"""
        return int(self.info[_OI_H])

    @property
    def n_eq(self) -> int:
        """number of ordered vertex pairs joined by two equivalent lines"""
        return int(self.info[_OI_NEQ])

    @property
    def l0(self) -> int:
        """closed loops of the all-direct vertex pairing"""
        return int(self.info[_OI_L0])

    def coef(self) -> np.ndarray:
        nl, nc = self.nl, self.n + 1
        c = np.asarray(self.info[_OI_COEF:_OI_COEF + MAXL * MAXC]).reshape(MAXL, MAXC)
        return c[:nl, :nc].copy()

    def cut_lines(self, m: int) -> List[int]:
        return [l for l, (s, t) in enumerate(self.lines) if min(s, t) <= m < max(s, t)]

    def arrays(self):
        lines = np.asarray([x for st in self.lines for x in st], dtype=np.int32)
        ports = np.asarray([x for p in self.ports for x in p], dtype=np.int32)
        chords = np.asarray(self.chords, dtype=np.int32)
        return lines, ports, chords


_OI_H, _OI_NEQ, _OI_L0 = 3, 4, 5
_OI_COEF = 8 + MAXL + MAXL + 4 * 6 + MAXC


def diagram_from_matrix(A, diagram_id: int = -1) -> Diagram:
    n = len(A)
    lines = []
    for i in range(n):
        for j in range(n):
            for _ in range(A[i][j]):
                lines.append((i, j))
    ports = []
    for v in range(n):
        outs = [l for l, (s, t) in enumerate(lines) if s == v]
        ins = [l for l, (s, t) in enumerate(lines) if t == v]
        ports.append((outs[0], outs[1], ins[0], ins[1]))
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    order = [l for l, (s, t) in enumerate(lines) if s < t] + [l for l, (s, t) in enumerate(lines) if s > t]
    chords = []
    for l in order:
        s, t = lines[l]
        rs, rt = find(s), find(t)
        if rs == rt:
            chords.append(l)
        else:
            parent[rs] = rt
    # hole chords first, then particle chords, each in line order (any basis gives the same integral; with
    # this order diagrams with equally many hole chords share the chord ranges of the loop-momentum map)
    chords.sort(key=lambda l: (lines[l][0] < lines[l][1], l))
    D = Diagram(n=n, A=tuple(tuple(r) for r in A), lines=lines, ports=ports, chords=chords, diagram_id=diagram_id)
    derive(D)
    return D


def derive(D: Diagram) -> Diagram:
    L = lib()
    info = np.zeros(L.oracle_info_ints(), dtype=np.int32)
    lines, ports, chords = D.arrays()
    ok = L.oracle_derive(D.n, _ip(lines), _ip(ports), _ip(chords), _ip(info))
    if not ok:
        raise ValueError("oracle_derive rejected the diagram")
    D.info = info
    return D


_cache = {}


def enumerate_diagrams(n: int) -> List[Diagram]:
    if n not in _cache:
        _cache[n] = [diagram_from_matrix(A, k) for k, A in enumerate(adjacency_matrices(n))]
    return _cache[n]


def mirror_matrix(A) -> tuple:
    """Time reversal plus arrow reversal: A'[i][j] = A[n-1-j][n-1-i]."""
    n = len(A)
    return tuple(tuple(A[n - 1 - j][n - 1 - i] for j in range(n)) for i in range(n))


def is_anomalous(D: Diagram) -> bool:
    """A hole and a particle line forced to carry the same momentum (equal
    coefficient rows up to sign): n_k (1 - n_k) = 0 at T = 0, so the diagram
    vanishes identically."""
    C = D.coef()
    for a in range(D.nl):
        for b in range(D.nl):
            if D.hole(a) and not D.hole(b):
                if np.array_equal(C[a], C[b]) or np.array_equal(C[a], -C[b]):
                    return True
    return False


# ----------------------------------------------------------------------------
# Physics parameters
# ----------------------------------------------------------------------------
@dataclass
class Physics:
    kF_n: float = 1.0
    kF_p: float = 0.0
    hbar2_over_m: float = 41.47
    C_S: float = -50.0
    C_Y: float = -200.0
    m_pi: float = 0.7
    Lam: float = 2.0
    reg_power: int = 4
    K_max: float = 7.0
    map_kind: int = 0
    shift: float = 0.0      # denominator shift s (MeV): D_m -> D_m - s, the regulator of Sec. III.A
    spectrum: int = 0       # 0 free, 1 Hartree-Fock (Eq. (7), spline of the self-energy)

    def base_array(self) -> np.ndarray:
        return np.asarray([self.kF_n, self.kF_p, self.hbar2_over_m, self.C_S, self.C_Y, self.m_pi, self.Lam,
                           float(self.reg_power), self.K_max, float(self.map_kind), self.shift,
                           float(self.spectrum)], dtype=np.float64)

    def array(self) -> np.ndarray:
        a = self.base_array()
        if self.spectrum == 0:
            return a
        y, m, h = hf_table(self)
        return np.concatenate([a, [float(len(y)), h], y, m])

    def dim(self, D: "Diagram") -> int:
        """integration dimension of diagram D under this chord map"""
        return D.d - 3 * self.map_kind

    @property
    def density(self) -> float:
        return (self.kF_n ** 3 + self.kF_p ** 3) / (3.0 * math.pi ** 2)


# The method's fixed Hartree-Fock tabulation: Sigma at HF_KNOTS knots k_i = i h, h = 2 K_max/(HF_KNOTS - 1),
# each from an HF_QUAD x HF_QUAD Gauss-Legendre rule; cubic spline in k (zero slope at 0, zero curvature
# at the last knot), Sigma = 0 beyond.
HF_KNOTS = 1024
HF_QUAD = 64
_HF_CACHE = {}


def hf_self_energy(ph: "Physics", k: float, n_rad: int = HF_QUAD, n_ang: int = HF_QUAD) -> float:
    """Sigma(k) in MeV by direct quadrature (one Fermi momentum: neutron or symmetric matter)."""
    return lib().oracle_hf_self_energy(_dp(ph.base_array()), float(k), n_rad, n_ang)


def hf_table(ph: "Physics"):
    """(Sigma at the knots, spline second derivatives, knot spacing)."""
    if ph.kF_n > 0 and ph.kF_p > 0 and ph.kF_n != ph.kF_p:
        raise ValueError("the Hartree-Fock spectrum needs one Fermi momentum (neutron or symmetric matter)")
    key = tuple(ph.base_array()[[0, 1, 2, 3, 4, 5, 6, 7, 8]])
    if key not in _HF_CACHE:
        L = lib()
        h = 2.0 * ph.K_max / (HF_KNOTS - 1)
        base = ph.base_array()
        y = np.array([L.oracle_hf_self_energy(_dp(base), i * h, HF_QUAD, HF_QUAD) for i in range(HF_KNOTS)])
        m = np.zeros(HF_KNOTS)
        L.oracle_spline_build(HF_KNOTS, h, _dp(y), _dp(m))
        _HF_CACHE[key] = (y, m, h)
    return _HF_CACHE[key]


def sp_energy(ph: "Physics", k: float) -> float:
    """Single-particle energy (MeV) of momentum k in the physics point's spectrum."""
    kin = 0.5 * ph.hbar2_over_m * k * k
    if ph.spectrum == 0:
        return kin
    y, m, h = hf_table(ph)
    return kin + lib().oracle_spline_eval(len(y), h, _dp(y), _dp(m), float(k))


def integrand(D: Diagram, ph: Physics, x: np.ndarray, with_cond: bool = False):
    """f(x) for one point (x in [0,1]^d); optionally the denominator condition number."""
    L = lib()
    x = np.ascontiguousarray(x, dtype=np.float64)
    cond = ctypes.c_double(0.0)
    f = L.oracle_integrand(_ip(D.info), _dp(ph.array()), _dp(x), ctypes.byref(cond))
    return (f, cond.value) if with_cond else f


def integrand_momenta(D: Diagram, ph: Physics, chord_k: np.ndarray) -> float:
    """Integrand at given chord momenta ((n+1) x 3), without map Jacobian and measure."""
    ck = np.ascontiguousarray(chord_k, dtype=np.float64).ravel()
    return lib().oracle_integrand_momenta(_ip(D.info), _dp(ph.array()), _dp(ck), None)


def line_ksq(D: Diagram, ph: Physics, x: np.ndarray) -> np.ndarray:
    """|k_l|^2 of every line at the point x."""
    out = np.zeros(D.nl)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    lib().oracle_line_ksq(_ip(D.info), _dp(ph.array()), _dp(xx), _dp(out))
    return out


def diagram_from_lists(n, lines, ports, chords) -> Diagram:
    """A diagram given in the line/port/chord form (e.g. a descriptor produced elsewhere)."""
    D = Diagram(n=n, A=None, lines=[tuple(x) for x in lines], ports=[tuple(p) for p in ports],
                chords=list(chords))
    return derive(D)


def line_momenta(D: Diagram, chord_k: np.ndarray) -> np.ndarray:
    return D.coef() @ np.asarray(chord_k, dtype=np.float64).reshape(D.n + 1, 3)


def first_order_integrand(ph: Physics, x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().oracle_first_order_integrand(_dp(ph.array()), _dp(x))


# ----------------------------------------------------------------------------
# VEGAS
# ----------------------------------------------------------------------------
def uniform_grid(d: int, nb: int = 50) -> np.ndarray:
    return np.tile(np.linspace(0.0, 1.0, nb + 1), (d, 1))


@dataclass
class IterationResult:
    sum_w: float
    sum_w2: float
    hist: np.ndarray
    n: int

    @property
    def mean(self) -> float:
        return self.sum_w / self.n

    @property
    def var_of_mean(self) -> float:
        return (self.sum_w2 / self.n - self.mean ** 2) / (self.n - 1)


def has_repeated_denominator(D: Diagram) -> bool:
    """Two cuts whose energy denominators are the same function of the loop momenta (a squared
    denominator, e.g. a self-energy insertion).  D_m = sum_h |k_h|^2 - sum_p |k_p|^2 with
    k_l = sum_c C_lc l_c is the quadratic form sum_l s_l C_l C_l^T (s = +1 hole, -1 particle) in the
    loop momenta: compare the integer matrices."""
    C = D.coef().astype(np.int64)
    forms = []
    for m in range(D.n - 1):
        Q = np.zeros((C.shape[1], C.shape[1]), dtype=np.int64)
        for l, (a, b) in enumerate(D.lines):
            if min(a, b) <= m < max(a, b):
                Q += (1 if D.hole(l) else -1) * np.outer(C[l], C[l])
        forms.append(Q.tobytes())
    return len(set(forms)) < len(forms)


def hole_chords(D: Diagram) -> int:
    """Number of loop momenta that are hole momenta (integrated over the Fermi ball): the
    particle-hole composition of the integration domain.  Grouping key of Sec. III.A (reading): at
    orders 2-6 it takes 1, 2, 4, 5, 6 distinct values, the N_grp column of Table I."""
    return int(sum(D.hole(l) for l in D.chords))


@dataclass
class Group:
    """Sum of same-order diagrams integrated as one integrand (Sec. III.A): f(x) = sum_m scale_m f_m(x),
    every member through its own chord map at the same point x."""
    members: List[Diagram]
    scales: List[float]

    @property
    def n(self) -> int:
        return self.members[0].n

    @property
    def d(self) -> int:
        return self.members[0].d


def groups(n: int, skip_anomalous: bool = True) -> dict:
    """Diagrams of order n grouped by hole_chords (unit scales), key -> Group."""
    out = {}
    for D in enumerate_diagrams(n):
        if skip_anomalous and is_anomalous(D):
            continue
        out.setdefault(hole_chords(D), []).append(D)
    return {k: Group(v, [1.0] * len(v)) for k, v in sorted(out.items())}


def group_integrand(G: Group, ph: Physics, x: np.ndarray) -> float:
    return float(sum(c * integrand(D, ph, x) for D, c in zip(G.members, G.scales)))


def vegas_samples(kind: int, D, ph_arr: np.ndarray, d: int, grid: np.ndarray, seed: int,
                  sid: int, t: int, s_begin: int, s_end: int, dump: bool = False):
    L = lib()
    nb = grid.shape[1] - 1
    grid = np.ascontiguousarray(grid, dtype=np.float64)
    sums = np.zeros(2)
    hist = np.zeros(d * nb)
    cnt = s_end - s_begin
    dx = np.zeros(cnt * d) if dump else None
    dw = np.zeros(cnt) if dump else None
    if isinstance(D, Group):
        infos = np.ascontiguousarray(np.concatenate([m.info for m in D.members]), dtype=np.int32)
        sc = np.ascontiguousarray(D.scales, dtype=np.float64)
        L.oracle_vegas_samples_group(len(D.members), _ip(infos), _dp(sc), _dp(ph_arr), d, nb, _dp(grid), seed, sid,
                                     t, s_begin, s_end, _dp(sums), _dp(hist), _dp(dx), _dp(dw))
    else:
        info = D.info if D is not None else np.zeros(L.oracle_info_ints(), dtype=np.int32)
        L.oracle_vegas_samples(kind, _ip(info), _dp(ph_arr), d, nb, _dp(grid), seed, sid, t, s_begin, s_end,
                               _dp(sums), _dp(hist), _dp(dx), _dp(dw))
    if dump:
        return sums, hist.reshape(d, nb), dx.reshape(cnt, d), dw
    return sums, hist.reshape(d, nb)


def vegas_iteration(D: Optional[Diagram], ph, grid: np.ndarray, seed: int, sid: int, t: int, n_samples: int,
                    threads: Optional[int] = None, kind: int = 0, first: int = 0) -> IterationResult:
    """One VEGAS iteration over samples [first, first + n_samples): sample ranges
    run on `threads` Python threads (ctypes releases the GIL) and are reduced in
    range order."""
    if isinstance(ph, Physics):
        ph_arr = ph.array()
    else:
        ph_arr = np.asarray(ph, dtype=np.float64)
    d = grid.shape[0]
    nb = grid.shape[1] - 1
    threads = threads or (os.cpu_count() or 1)
    threads = max(1, min(threads, n_samples))
    bounds = [first + (n_samples * k) // threads for k in range(threads + 1)]
    results = [None] * threads

    def work(k):
        results[k] = vegas_samples(kind, D, ph_arr, d, grid, seed, sid, t, bounds[k], bounds[k + 1])

    ths = [threading.Thread(target=work, args=(k,)) for k in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    sw = sw2 = 0.0
    hist = np.zeros((d, nb))
    for s, h in results:
        sw += s[0]
        sw2 += s[1]
        hist += h
    return IterationResult(sw, sw2, hist, n_samples)


def refine(grid: np.ndarray, hist: np.ndarray, alpha: float = 1.5) -> np.ndarray:
    L = lib()
    d, nbp1 = grid.shape
    out = np.zeros_like(grid)
    for a in range(d):
        g = np.ascontiguousarray(grid[a])
        h = np.ascontiguousarray(hist[a])
        o = np.zeros(nbp1)
        L.oracle_refine(_dp(h), _dp(g), nbp1 - 1, alpha, _dp(o))
        out[a] = o
    return out


def combine(means: Sequence[float], variances: Sequence[float], skip: int = 0):
    """Inverse-variance weighted mean of the iteration estimates, its standard
    error and chi^2 per degree of freedom.  Iterations whose sample variance is
    exactly zero (an integrand that vanished on every sample) carry no weight;
    if every iteration has zero variance the last estimate is returned with
    zero error."""
    means = np.asarray(means, dtype=np.float64)[skip:]
    variances = np.asarray(variances, dtype=np.float64)[skip:]
    pos = variances > 0.0
    if not np.any(pos):
        return float(means[-1]), 0.0, 0.0
    m_, v_ = means[pos], variances[pos]
    wts = 1.0 / v_
    mean = float(np.sum(m_ * wts) / np.sum(wts))
    sigma = float(1.0 / math.sqrt(np.sum(wts)))
    dof = len(m_) - 1
    chi2 = float(np.sum((m_ - mean) ** 2 * wts) / dof) if dof > 0 else 0.0
    return mean, sigma, chi2


def combine_pooled(sums_w: Sequence[float], sums_w2: Sequence[float], counts: Sequence[int]):
    """PVegas' evaluation phase (Sec. III.C): the iterations ran on one frozen grid, so their samples are
    draws from one distribution and every sample carries the same weight.  With S1 = sum w, S2 = sum w^2
    and N samples over all of them: mean = S1/N, sigma^2 = (S2/N - mean^2)/(N - 1) -- the estimate and
    standard error of one run of N samples.  chi^2/dof compares the iterations' own estimates with that
    mean (each with its own variance)."""
    s1, s2, n = float(np.sum(sums_w)), float(np.sum(sums_w2)), float(np.sum(counts))
    mean = s1 / n
    var = (s2 / n - mean * mean) / (n - 1.0)
    sigma = math.sqrt(var) if var > 0.0 else 0.0
    chi2 = 0.0
    if len(counts) > 1:
        c2, used = 0.0, 0
        for a, b, m in zip(sums_w, sums_w2, counts):
            it = a / m
            v = (b / m - it * it) / (m - 1.0)
            if v > 0.0:
                c2 += (it - mean) ** 2 / v
                used += 1
        chi2 = c2 / (used - 1) if used > 1 else 0.0
    return mean, sigma, chi2


def vegas(D: Optional[Diagram], ph, n_iter: int, n_samples: int, seed: int = 1, sid: int = 0, nb: int = 50,
          alpha: float = 1.5, threads: Optional[int] = None, kind: int = 0, d: Optional[int] = None,
          train_iters: int = 0, pooled: bool = False):
    """Full VEGAS run.  Default: refine after every iteration and combine every iteration from train_iters
    on with inverse-variance weights (Lepage).  pooled: the first train_iters iterations train the grid
    (refined after each) and are not combined; the grid is then frozen and the remaining iterations are
    combined by combine_pooled."""
    if d is None:
        d = (ph.dim(D) if isinstance(ph, Physics) else D.d) if kind == 0 else 6
    grid = uniform_grid(d, nb)
    means, vars_, s1, s2, cnt = [], [], [], [], []
    for t in range(n_iter):
        r = vegas_iteration(D, ph, grid, seed, sid, t, n_samples, threads=threads, kind=kind)
        means.append(r.mean)
        vars_.append(r.var_of_mean)
        if t >= train_iters:
            s1.append(r.sum_w)
            s2.append(r.sum_w2)
            cnt.append(r.n)
        if not pooled or t < train_iters:
            grid = refine(grid, r.hist, alpha)
    if pooled:
        return combine_pooled(s1, s2, cnt) + (grid,)
    return combine(means, vars_, skip=train_iters) + (grid,)


# ----------------------------------------------------------------------------
# Finite-space Rayleigh-Schroedinger check of the diagram rules
# ----------------------------------------------------------------------------
def discrete_diagram(D: Diagram, nh: int, np_: int, wbar: np.ndarray, eps: np.ndarray) -> float:
    w = np.ascontiguousarray(wbar, dtype=np.float64).ravel()
    e = np.ascontiguousarray(eps, dtype=np.float64)
    return lib().oracle_discrete_diagram(_ip(D.info), nh, np_, _dp(w), _dp(e))


def random_antisymmetric_w(N: int, rng: np.random.Generator, scale: float = 0.3) -> np.ndarray:
    """Real wbar[p,q,r,s] = -wbar[q,p,r,s] = -wbar[p,q,s,r] = wbar[r,s,p,q]."""
    w = rng.normal(size=(N, N, N, N)) * scale
    w = w - w.transpose(1, 0, 2, 3)
    w = w - w.transpose(0, 1, 3, 2)
    w = 0.5 * (w + w.transpose(2, 3, 0, 1))
    return w


def _apply_annihilate(det: int, p: int):
    if not (det >> p) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1
    return det & ~(1 << p), sign


def _apply_create(det: int, p: int):
    if (det >> p) & 1:
        return None, 0
    sign = -1 if bin(det & ((1 << p) - 1)).count("1") % 2 else 1
    return det | (1 << p), sign


def rspt_coefficients(wbar: np.ndarray, eps: np.ndarray, nh: int, max_order: int = 5) -> List[float]:
    """Exact Rayleigh-Schroedinger energy coefficients E^(1..max_order) of
    H = H0 + W_N in the determinant space of N orbitals with nh holes, where
    H0 = sum_p eps_p a+_p a_p and W_N is the normal-ordered two-body part of
    (1/4) sum wbar_pqrs a+_p a+_q a_s a_r with respect to the reference that
    fills orbitals 0..nh-1."""
    N = len(eps)
    dets = [sum(1 << k for k in occ) for occ in itertools.combinations(range(N), nh)]
    index = {dd: k for k, dd in enumerate(dets)}
    M = len(dets)
    W = np.zeros((M, M))
    for col, det in enumerate(dets):
        for p in range(N):
            for q in range(N):
                for r in range(N):
                    for s in range(N):
                        val = wbar[p, q, r, s]
                        if val == 0.0:
                            continue
                        d1, s1 = _apply_annihilate(det, r)
                        if d1 is None:
                            continue
                        d2, s2 = _apply_annihilate(d1, s)
                        if d2 is None:
                            continue
                        d3, s3 = _apply_create(d2, q)
                        if d3 is None:
                            continue
                        d4, s4 = _apply_create(d3, p)
                        if d4 is None:
                            continue
                        W[index[d4], col] += 0.25 * val * s1 * s2 * s3 * s4
    F = np.zeros((M, M))
    f = np.zeros((N, N))
    for p in range(N):
        for q in range(N):
            f[p, q] = sum(wbar[p, i, q, i] for i in range(nh))
    for col, det in enumerate(dets):
        for p in range(N):
            for q in range(N):
                if f[p, q] == 0.0:
                    continue
                d1, s1 = _apply_annihilate(det, q)
                if d1 is None:
                    continue
                d2, s2 = _apply_create(d1, p)
                if d2 is None:
                    continue
                F[index[d2], col] += f[p, q] * s1 * s2
    const = sum(f[i, i] for i in range(nh)) - 0.5 * sum(wbar[i, j, i, j] for i in range(nh) for j in range(nh))
    WN = W - F + const * np.eye(M)
    H0 = np.array([sum(eps[k] for k in range(N) if (det >> k) & 1) for det in dets])
    ref = index[sum(1 << k for k in range(nh))]
    E0 = H0[ref]
    R = np.zeros(M)
    for k in range(M):
        if k != ref:
            R[k] = 1.0 / (E0 - H0[k])
    psi = [np.zeros(M)]
    psi[0][ref] = 1.0
    E = [E0]
    for k in range(1, max_order + 1):
        Ek = float((WN @ psi[k - 1])[ref])
        E.append(Ek)
        rhs = WN @ psi[k - 1]
        for j in range(1, k + 1):
            rhs = rhs - E[j] * psi[k - j]
        nxt = R * rhs
        nxt[ref] = 0.0
        psi.append(nxt)
    return E[1:], WN, ref
