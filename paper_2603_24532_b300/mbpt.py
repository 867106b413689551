"""Thin ctypes binding of libmbpt (include/mbpt.h): same names, argument
marshalling only.  Every computation runs in the CUDA library; if the library
cannot be loaded the calls raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

MBPT_OK = 0
MBPT_EINVAL = -1
MBPT_ENOMEM = -2
MBPT_ECUDA = -3
MBPT_EDEVICE = -4
MBPT_ETIMEOUT = -5
MBPT_ENUMERIC = -6
MBPT_EBUSY = -7
MBPT_FP64 = 0
MBPT_MIXED = 1
MBPT_MIXED_MAP64 = 2
MBPT_COMBINE_INVVAR = 0
MBPT_COMBINE_POOLED = 1
MBPT_HIST_WARP_F32 = 0
MBPT_HIST_BLOCK_F64 = 1
MBPT_SPIN_TABLE = 0
MBPT_SPIN_FOLD = 1
MAX_ORDER = 6
MAX_LINES = 12
MAX_CHORDS = 7
MAX_BINS = 64
FLAG_ANOMALOUS = 1
FLAG_SELF_MIRROR = 2
FLAG_REPEATED_DENOMINATOR = 4

_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EDEVICE", -5: "ETIMEOUT", -6: "ENUMERIC",
           -7: "EBUSY"}


class MbptError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class mbpt_diagram_desc(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32),
        ("n_lines", ctypes.c_int32),
        ("line_src", ctypes.c_int8 * MAX_LINES),
        ("line_dst", ctypes.c_int8 * MAX_LINES),
        ("vtx_out", (ctypes.c_int8 * 2) * MAX_ORDER),
        ("vtx_in", (ctypes.c_int8 * 2) * MAX_ORDER),
        ("n_chords", ctypes.c_int8),
        ("chord_line", ctypes.c_int8 * MAX_CHORDS),
        ("line_coef", (ctypes.c_int8 * MAX_CHORDS) * MAX_LINES),
        ("diagram_id", ctypes.c_int32),
        ("mirror_id", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]

    # convenience views
    def lines(self):
        return [(self.line_src[l], self.line_dst[l]) for l in range(self.n_lines)]

    def ports(self):
        return [(self.vtx_out[v][0], self.vtx_out[v][1], self.vtx_in[v][0], self.vtx_in[v][1])
                for v in range(self.order)]

    def chords(self):
        return [self.chord_line[c] for c in range(self.n_chords)]

    def coef(self):
        return np.array([[self.line_coef[l][c] for c in range(self.n_chords)] for l in range(self.n_lines)])

    @property
    def anomalous(self) -> bool:
        return bool(self.flags & FLAG_ANOMALOUS)

    @property
    def repeated_denominator(self) -> bool:
        return bool(self.flags & FLAG_REPEATED_DENOMINATOR)

    @classmethod
    def from_lists(cls, order, lines, ports, chords, coef, diagram_id=-1, mirror_id=-1, flags=0):
        d = cls()
        d.order = order
        d.n_lines = len(lines)
        for l, (s, t) in enumerate(lines):
            d.line_src[l] = s
            d.line_dst[l] = t
        for v, (o1, o2, i1, i2) in enumerate(ports):
            d.vtx_out[v][0], d.vtx_out[v][1] = o1, o2
            d.vtx_in[v][0], d.vtx_in[v][1] = i1, i2
        d.n_chords = len(chords)
        for c, l in enumerate(chords):
            d.chord_line[c] = l
        coef = np.asarray(coef)
        for l in range(coef.shape[0]):
            for c in range(coef.shape[1]):
                d.line_coef[l][c] = int(coef[l, c])
        d.diagram_id, d.mirror_id, d.flags = diagram_id, mirror_id, flags
        return d


class mbpt_physics(ctypes.Structure):
    _fields_ = [
        ("kF_n", ctypes.c_double), ("kF_p", ctypes.c_double),
        ("hbar2_over_m", ctypes.c_double),
        ("C_S", ctypes.c_double), ("C_Y", ctypes.c_double), ("m_pi", ctypes.c_double), ("Lambda", ctypes.c_double),
        ("reg_power", ctypes.c_int32), ("map_kind", ctypes.c_int32),
        ("K_max", ctypes.c_double),
        ("spectrum", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class mbpt_vegas_cfg(ctypes.Structure):
    _fields_ = [
        ("n_bins", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("stream_id", ctypes.c_uint32), ("freeze_after", ctypes.c_uint32),
        ("samples_per_iter", ctypes.c_uint64),
        ("target_rel", ctypes.c_double), ("target_abs", ctypes.c_double),
        ("train_iters", ctypes.c_uint32), ("n_shifts", ctypes.c_uint32),
        ("shift", ctypes.c_double * 3),
        ("combine", ctypes.c_uint32), ("near_band", ctypes.c_float),
    ]


class mbpt_result(ctypes.Structure):
    _fields_ = [
        ("mean", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
        ("last_mean", ctypes.c_double), ("last_sigma", ctypes.c_double),
        ("n_iter", ctypes.c_int64), ("n_evals", ctypes.c_int64),
        ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load the in-tree libmbpt.so (building it first if it is missing), or the library named by the
    MBPT_LIBRARY environment variable (another build of the same sources)."""
    global _lib
    if _lib is None:
        path = os.environ.get("MBPT_LIBRARY") or _build.LIB
        if path == _build.LIB and (not os.path.exists(path) or os.environ.get("MBPT_REBUILD")):
            _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        sig = {
            "mbpt_generate": [ctypes.c_int, P(mbpt_diagram_desc), ctypes.c_int, P(ctypes.c_int)],
            "mbpt_ctx_create": [P(vp), ctypes.c_int, vp, ctypes.c_size_t, vp],
            "mbpt_ctx_destroy": [vp],
            "mbpt_ctx_mem": [vp, P(ctypes.c_size_t), P(ctypes.c_size_t)],
            "mbpt_diag_bytes": [P(mbpt_diagram_desc), P(mbpt_vegas_cfg), P(ctypes.c_size_t)],
            "mbpt_kernel_variants": [P(ctypes.c_int), P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)],
            "mbpt_ctx_set_kernel": [vp, ctypes.c_int, ctypes.c_int],
            "mbpt_ctx_set_launch": [vp, ctypes.c_int, ctypes.c_int],
            "mbpt_ctx_get_launch": [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)],
            "mbpt_ctx_set_hist_layout": [vp, ctypes.c_int],
            "mbpt_ctx_get_hist_layout": [vp, P(ctypes.c_int)],
            "mbpt_ctx_set_spin_sum": [vp, ctypes.c_int],
            "mbpt_ctx_get_spin_sum": [vp, P(ctypes.c_int)],
            "mbpt_ctx_last_timing": [vp, P(ctypes.c_double), P(ctypes.c_double)],
            "mbpt_ctx_stream": [vp, P(vp)],
            "mbpt_create_diagram": [vp, P(mbpt_diagram_desc), P(mbpt_physics), P(mbpt_vegas_cfg), P(vp)],
            "mbpt_create_group": [vp, P(mbpt_diagram_desc), ctypes.c_int, P(ctypes.c_double), P(mbpt_physics),
                                  P(mbpt_vegas_cfg), P(vp)],
            "mbpt_hole_chords": [P(mbpt_diagram_desc), P(ctypes.c_int)],
            "mbpt_group_bytes": [P(mbpt_diagram_desc), ctypes.c_int, P(mbpt_vegas_cfg), P(ctypes.c_size_t)],
            "mbpt_hf_self_energy": [P(mbpt_physics), ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)],
            "mbpt_destroy_diagram": [vp],
            "mbpt_set_config": [vp, P(mbpt_vegas_cfg)],
            "mbpt_vegas_iterate": [vp, P(vp), ctypes.c_int, ctypes.c_int],
            "mbpt_estimate": [vp, P(mbpt_result)],
            "mbpt_estimate_batch": [P(vp), ctypes.c_int, P(mbpt_result)],
            "mbpt_estimate_shifts": [vp, P(ctypes.c_double), P(ctypes.c_double)],
            "mbpt_get_state": [vp, vp, ctypes.c_size_t, P(ctypes.c_size_t)],
            "mbpt_set_state": [vp, vp, ctypes.c_size_t],
            "mbpt_dump_samples": [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P(ctypes.c_double),
                                  P(ctypes.c_double)],
            "mbpt_philox_device": [vp, P(ctypes.c_uint32), P(ctypes.c_uint32), ctypes.c_int64, P(ctypes.c_uint32)],
            "mbpt_vegas_iteration_noalloc": [ctypes.c_int, P(mbpt_diagram_desc), P(mbpt_physics), P(mbpt_vegas_cfg),
                                             ctypes.c_uint32, vp, vp, vp],
            "mbpt_fp64_rate": [ctypes.c_int, vp, P(ctypes.c_double)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.mbpt_last_error.restype = ctypes.c_char_p
        L.mbpt_last_error.argtypes = []
        _lib = L
    return _lib


def check(status: int):
    if status != MBPT_OK:
        raise MbptError(status, lib().mbpt_last_error().decode(errors="replace"))
    return status


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# Functions, same names as the C ABI
# ---------------------------------------------------------------------------
def mbpt_generate(order: int) -> List[mbpt_diagram_desc]:
    n = ctypes.c_int(0)
    check(lib().mbpt_generate(order, None, 0, ctypes.byref(n)))
    arr = (mbpt_diagram_desc * n.value)()
    check(lib().mbpt_generate(order, arr, n.value, ctypes.byref(n)))
    return list(arr)


def mbpt_ctx_create(device: int = 0, arena_bytes: int = 1 << 30, arena_ptr: int = 0, stream: int = 0):
    c = ctypes.c_void_p()
    check(lib().mbpt_ctx_create(ctypes.byref(c), device, ctypes.c_void_p(arena_ptr or None), arena_bytes,
                                ctypes.c_void_p(stream or None)))
    return c


def mbpt_ctx_destroy(ctx):
    check(lib().mbpt_ctx_destroy(ctx))


def mbpt_ctx_mem(ctx):
    u, f = ctypes.c_size_t(), ctypes.c_size_t()
    check(lib().mbpt_ctx_mem(ctx, ctypes.byref(u), ctypes.byref(f)))
    return u.value, f.value


def mbpt_diag_bytes(desc: mbpt_diagram_desc, cfg: mbpt_vegas_cfg) -> int:
    b = ctypes.c_size_t()
    check(lib().mbpt_diag_bytes(ctypes.byref(desc), ctypes.byref(cfg), ctypes.byref(b)))
    return b.value


def mbpt_group_bytes(descs: Sequence[mbpt_diagram_desc], cfg: mbpt_vegas_cfg) -> int:
    arr = (mbpt_diagram_desc * max(1, len(descs)))(*descs)
    b = ctypes.c_size_t()
    check(lib().mbpt_group_bytes(arr, len(descs), ctypes.byref(cfg), ctypes.byref(b)))
    return b.value


def mbpt_hf_self_energy(phys: mbpt_physics, k) -> np.ndarray:
    """Hartree-Fock self-energy (MeV) of the physics point's spectrum table at momenta k (fm^-1)."""
    kk = np.ascontiguousarray(np.atleast_1d(k), dtype=np.float64)
    out = np.zeros_like(kk)
    check(lib().mbpt_hf_self_energy(ctypes.byref(phys), len(kk), _dp(kk), _dp(out)))
    return out


def mbpt_kernel_variants():
    n = ctypes.c_int()
    check(lib().mbpt_kernel_variants(None, None, 0, ctypes.byref(n)))
    t = (ctypes.c_int * n.value)()
    m = (ctypes.c_int * n.value)()
    check(lib().mbpt_kernel_variants(t, m, n.value, ctypes.byref(n)))
    return list(zip(list(t), list(m)))


def mbpt_ctx_set_kernel(ctx, threads_per_block: int, min_blocks_per_sm: int):
    check(lib().mbpt_ctx_set_kernel(ctx, threads_per_block, min_blocks_per_sm))


def mbpt_ctx_set_launch(ctx, order: int, samples_per_thread: int):
    check(lib().mbpt_ctx_set_launch(ctx, order, samples_per_thread))


def mbpt_ctx_get_launch(ctx, order: int):
    t, m, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().mbpt_ctx_get_launch(ctx, order, ctypes.byref(t), ctypes.byref(m), ctypes.byref(s)))
    return t.value, m.value, s.value


def mbpt_ctx_set_hist_layout(ctx, layout: int):
    check(lib().mbpt_ctx_set_hist_layout(ctx, layout))


def mbpt_ctx_get_hist_layout(ctx) -> int:
    v = ctypes.c_int()
    check(lib().mbpt_ctx_get_hist_layout(ctx, ctypes.byref(v)))
    return v.value


def mbpt_ctx_set_spin_sum(ctx, strategy: int):
    check(lib().mbpt_ctx_set_spin_sum(ctx, strategy))


def mbpt_ctx_get_spin_sum(ctx) -> int:
    v = ctypes.c_int()
    check(lib().mbpt_ctx_get_spin_sum(ctx, ctypes.byref(v)))
    return v.value


def mbpt_ctx_last_timing(ctx):
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib().mbpt_ctx_last_timing(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mbpt_ctx_stream(ctx) -> int:
    s = ctypes.c_void_p()
    check(lib().mbpt_ctx_stream(ctx, ctypes.byref(s)))
    return s.value or 0


def mbpt_create_diagram(ctx, desc: mbpt_diagram_desc, phys: mbpt_physics, cfg: mbpt_vegas_cfg):
    g = ctypes.c_void_p()
    check(lib().mbpt_create_diagram(ctx, ctypes.byref(desc), ctypes.byref(phys), ctypes.byref(cfg),
                                    ctypes.byref(g)))
    return g


def mbpt_create_group(ctx, descs: Sequence[mbpt_diagram_desc], phys: mbpt_physics, cfg: mbpt_vegas_cfg,
                      scales: Optional[Sequence[float]] = None):
    """One integral over the sum of same-order diagrams (member m scaled by scales[m])."""
    k = len(descs)
    arr = (mbpt_diagram_desc * max(1, k))(*descs)
    sc = None
    if scales is not None:
        if len(scales) != k:
            raise ValueError("one scale per member")
        sc = (ctypes.c_double * k)(*[float(v) for v in scales])
    g = ctypes.c_void_p()
    check(lib().mbpt_create_group(ctx, arr, k, sc, ctypes.byref(phys), ctypes.byref(cfg), ctypes.byref(g)))
    return g


def mbpt_hole_chords(desc: mbpt_diagram_desc) -> int:
    out = ctypes.c_int(0)
    check(lib().mbpt_hole_chords(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def mbpt_destroy_diagram(diag):
    check(lib().mbpt_destroy_diagram(diag))


def mbpt_set_config(diag, cfg: mbpt_vegas_cfg):
    check(lib().mbpt_set_config(diag, ctypes.byref(cfg)))


def mbpt_vegas_iterate(ctx, diags: Sequence, n_iters: int):
    arr = (ctypes.c_void_p * max(1, len(diags)))(*[d.value for d in diags])
    check(lib().mbpt_vegas_iterate(ctx, arr, len(diags), n_iters))


def mbpt_estimate(diag) -> mbpt_result:
    r = mbpt_result()
    check(lib().mbpt_estimate(diag, ctypes.byref(r)))
    return r


def mbpt_estimate_shifts(diag):
    """(mean[4], sigma[4]): the three shifted integrals and their extrapolation to zero shift."""
    mean = np.zeros(4)
    sigma = np.zeros(4)
    check(lib().mbpt_estimate_shifts(diag, _dp(mean), _dp(sigma)))
    return mean, sigma


def mbpt_estimate_batch(diags: Sequence) -> List[mbpt_result]:
    k = len(diags)
    if k == 0:
        return []
    arr = (ctypes.c_void_p * k)(*[d.value for d in diags])
    out = (mbpt_result * k)()
    check(lib().mbpt_estimate_batch(arr, k, out))
    return list(out)


def mbpt_get_state(diag) -> bytes:
    need = ctypes.c_size_t()
    check(lib().mbpt_get_state(diag, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    check(lib().mbpt_get_state(diag, buf, need.value, ctypes.byref(need)))
    return buf.raw


def mbpt_set_state(diag, image: bytes):
    buf = ctypes.create_string_buffer(image, len(image))
    check(lib().mbpt_set_state(diag, buf, len(image)))


def mbpt_dump_samples(diag, iter_: int, first: int, count: int, d: int, with_x: bool = True):
    w = np.zeros(count)
    x = np.zeros((count, d)) if with_x else None
    check(lib().mbpt_dump_samples(diag, iter_, first, count, _dp(x), _dp(w)))
    return x, w


def mbpt_philox_device(ctx, ctr: Sequence[int], key: Sequence[int], count: int) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = np.zeros(4 * count, dtype=np.uint32)
    check(lib().mbpt_philox_device(ctx, c, k, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return out.reshape(count, 4)


def mbpt_fp64_rate(device: int = 0, stream: int = 0) -> float:
    """FP64 thread operations per second that a dependency-free DFMA loop reaches on the device now
    (the roofline denominator of the FP64-bound kernels)."""
    v = ctypes.c_double()
    check(lib().mbpt_fp64_rate(device, ctypes.c_void_p(stream or None), ctypes.byref(v)))
    return v.value


def mbpt_vegas_iteration_noalloc(device: int, desc: mbpt_diagram_desc, phys: mbpt_physics, cfg: mbpt_vegas_cfg,
                                 iter_: int, grid_ptr: int, out_ptr: int, stream: int = 0):
    """One iteration without device allocation; grid_ptr / out_ptr are device addresses
    (d x (n_bins+1) edges in, 2 + d*n_bins doubles out)."""
    check(lib().mbpt_vegas_iteration_noalloc(device, ctypes.byref(desc), ctypes.byref(phys), ctypes.byref(cfg),
                                             iter_, ctypes.c_void_p(grid_ptr), ctypes.c_void_p(out_ptr),
                                             ctypes.c_void_p(stream or None)))


# ---------------------------------------------------------------------------
# State image layout helpers (header, DiagState, grid, last histogram)
# ---------------------------------------------------------------------------
# bytes moved per integral and batch by mbpt_vegas_iterate (work item, work header) and mbpt_estimate_batch
WORK_ITEM_BYTES = 112
WORK_HEADER_BYTES = 128
RESULT_BYTES = 80
STATE_HEADER_BYTES = 24
MAX_ITERS = 512
N_COMP = 4
DIAGSTATE_BYTES = 7 * 8 + 8 + 4 * 4 + 2 * MAX_ITERS * 8 + 4 * N_COMP * 8 + 4 * 8 + 2 * N_COMP * 8   # = 8496


def state_grid(image: bytes, d: int, nb: int) -> np.ndarray:
    off = STATE_HEADER_BYTES + DIAGSTATE_BYTES
    return np.frombuffer(image, dtype=np.float64, count=d * (nb + 1), offset=off).reshape(d, nb + 1).copy()


def state_last_hist(image: bytes, d: int, nb: int) -> np.ndarray:
    off = STATE_HEADER_BYTES + DIAGSTATE_BYTES + 8 * d * (nb + 1)
    return np.frombuffer(image, dtype=np.float64, count=d * nb, offset=off).reshape(d, nb).copy()


def state_with_iter(image: bytes, iteration: int) -> bytes:
    """Image with the iteration counter (the next iteration's Philox counter word 1) replaced."""
    off = STATE_HEADER_BYTES + 7 * 8 + 8
    b = bytearray(image)
    b[off:off + 4] = int(iteration).to_bytes(4, "little", signed=True)
    return bytes(b)


def state_with_grid(image: bytes, grid: np.ndarray) -> bytes:
    d, nbp1 = grid.shape
    off = STATE_HEADER_BYTES + DIAGSTATE_BYTES
    b = bytearray(image)
    b[off:off + 8 * d * nbp1] = np.ascontiguousarray(grid, dtype=np.float64).tobytes()
    return bytes(b)


def physics(kF_n=1.0, kF_p=0.0, hbar2_over_m=41.47, C_S=-50.0, C_Y=-200.0, m_pi=0.7, Lam=2.0, reg_power=4,
            K_max=None, map_kind=0, spectrum=0) -> mbpt_physics:
    """Physics point of the toy potential; K_max defaults to max kF + 3 Lambda."""
    p = mbpt_physics()
    p.kF_n, p.kF_p, p.hbar2_over_m = kF_n, kF_p, hbar2_over_m
    p.C_S, p.C_Y, p.m_pi, p.Lambda = C_S, C_Y, m_pi, Lam
    p.reg_power, p.map_kind, p.spectrum = reg_power, map_kind, spectrum
    p.K_max = K_max if K_max is not None else max(kF_n, kF_p) + 3.0 * Lam
    return p


def vegas_cfg(samples=1 << 18, seed=1, stream_id=0, precision=MBPT_FP64, n_bins=50, alpha=1.5, freeze_after=0,
              target_rel=0.0, target_abs=0.0, train_iters=0, shifts=None, combine=MBPT_COMBINE_INVVAR,
              near_band=0.0) -> mbpt_vegas_cfg:
    c = mbpt_vegas_cfg()
    c.n_bins, c.precision, c.alpha = n_bins, precision, alpha
    c.seed, c.stream_id, c.freeze_after = seed, stream_id, freeze_after
    c.samples_per_iter = samples
    c.target_rel, c.target_abs = target_rel, target_abs
    c.train_iters = train_iters
    c.combine, c.near_band = combine, near_band
    if shifts:
        if len(shifts) != 3:
            raise ValueError("the denominator regulator takes exactly three shifts")
        c.n_shifts = 3
        for k, v in enumerate(shifts):
            c.shift[k] = float(v)
    return c
