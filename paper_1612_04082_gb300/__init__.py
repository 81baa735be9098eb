"""Python binding of the kifmm_elastic C-ABI library (GB300, sm_103a).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  The functions keep the C names (``kfmm_create``, ``kfmm_build``, ``kfmm_eval``,
...).  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed to the
library as raw pointers (device or host; the library stages host arrays itself).

There is no fallback: importing this package loads ``_lib/libkifmm_elastic.so`` and raises
if it is missing (run ``python -m paper_1612_04082_gb300.build`` or
``__graft_entry__.build()`` first).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libkifmm_elastic.so")
HEADER_PATH = os.path.join(_HERE, "..", "include", "kifmm_elastic.h")

KFMM_OK = 0
KFMM_ERR_INVALID_ARG = -1
KFMM_ERR_OOM = -2
KFMM_ERR_CUDA = -3
KFMM_ERR_NOT_CONVERGED = -4
KFMM_ERR_DEVICE_TIMEOUT = -5
KFMM_ERR_NOT_BUILT = -6
KFMM_ERR_INTERNAL = -7
KFMM_DISP = 0
KFMM_STRESS = 1
KFMM_TD = 2
KFMM_FP32 = 0
KFMM_FP64 = 1


class kfmm_options(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("leaf_cap", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double), ("pinv_rtol", ctypes.c_double),
                ("m2l_rtol", ctypes.c_double), ("m2l_rank_max", ctypes.c_int), ("m2l_tensor_cores", ctypes.c_int),
                ("device", ctypes.c_int), ("graphs", ctypes.c_int), ("autotune", ctypes.c_int),
                ("streams", ctypes.c_int), ("eval_item_cost", ctypes.c_int)]


class kfmm_stats(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_trg", ctypes.c_int64), ("n_boxes", ctypes.c_int32),
                ("n_leaves", ctypes.c_int32), ("n_levels", ctypes.c_int32), ("m2l_rank", ctypes.c_int32),
                ("n_surf", ctypes.c_int32), ("n_u_pairs", ctypes.c_int64), ("n_v_pairs", ctypes.c_int64),
                ("n_w_pairs", ctypes.c_int64), ("n_x_pairs", ctypes.c_int64),
                ("p2p_interactions", ctypes.c_int64), ("s2m_interactions", ctypes.c_int64),
                ("l2p_interactions", ctypes.c_int64), ("p2l_interactions", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("up_rank", ctypes.c_int32), ("down_rank", ctypes.c_int32),
                ("n_xboxes", ctypes.c_int32), ("n_wboxes", ctypes.c_int32), ("m2l_chunk", ctypes.c_int32),
                ("eval_item_cost", ctypes.c_float), ("fp32_box_ratio", ctypes.c_float)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"kifmm_elastic library not built: {LIB_PATH} is missing "
                      "(run paper_1612_04082_gb300/build.py or __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_sig = {
    "kfmm_default_options": (None, [ctypes.POINTER(kfmm_options)]),
    "kfmm_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(kfmm_options)]),
    "kfmm_destroy": (ctypes.c_int, [_vp]),
    "kfmm_set_material": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
    "kfmm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "kfmm_set_periodic": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_double]),
    "kfmm_build": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp, _i64]),
    "kfmm_build_sets": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "kfmm_selftest_bounded_wait": (ctypes.c_int, [_vp, _i64]),
    "kfmm_eval": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
    "kfmm_direct": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _i64, _vp, _vp, _i64, _vp, _vp, ctypes.c_int, _vp]),
    "kfmm_direct_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _i64, _vp, _vp, _i64, _vp, _vp, ctypes.c_int,
                                           _vp]),
    "kfmm_direct_hi": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _i64, _vp, _vp, ctypes.c_double, _vp]),
    "kfmm_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(kfmm_stats)]),
    "kfmm_export_tree": (ctypes.c_int, [_vp] + [_vp] * 7),
    "kfmm_export_list": (ctypes.c_int, [_vp, ctypes.c_char, _vp, _vp, ctypes.POINTER(_i64)]),
    "kfmm_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "kfmm_get_phase_times": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "kfmm_measure_fp32_peak": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int32)]),
    "kfmm_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "kfmm_shard_plan": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp]),
    "kfmm_shard_let": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "kfmm_last_error": (ctypes.c_char_p, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class KfmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.kfmm_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _nrows(a):
    return int(a.shape[0])


def _check(ctx_handle, status):
    if status != KFMM_OK:
        msg = _lib.kfmm_last_error(ctx_handle).decode() if ctx_handle else ""
        raise KfmmError(status, msg)


def kfmm_default_options(**overrides) -> kfmm_options:
    o = kfmm_options()
    _lib.kfmm_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def kfmm_create(options: kfmm_options | None = None, **overrides):
    o = options if options is not None else kfmm_default_options()
    for k, v in overrides.items():
        setattr(o, k, v)
    h = _vp()
    _check(None, _lib.kfmm_create(ctypes.byref(h), ctypes.byref(o)))
    return h


def kfmm_destroy(ctx):
    _check(None, _lib.kfmm_destroy(ctx))


def kfmm_set_material(ctx, K: float, G: float):
    _check(ctx, _lib.kfmm_set_material(ctx, float(K), float(G)))


def kfmm_set_periodic(ctx, lo=None, side=1.0):
    """Periodic cubic cell [lo, lo + side]^3 for the next build (lo None: free space)."""
    if lo is None:
        _check(ctx, _lib.kfmm_set_periodic(ctx, 0, None, 1.0))
        return
    c = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
    _check(ctx, _lib.kfmm_set_periodic(ctx, 1, c.ctypes.data, float(side)))


ENT_BITS = 26


def list_entries(items):
    """Box index and image offset [n, 3] (whole cells, -1..1) of interaction-list entries: the
    box in the low 26 bits, the image of a periodic tree above them (kifmm_elastic.h)."""
    items = np.asarray(items, dtype=np.int64)
    code = ((items >> ENT_BITS) & 31) ^ 13
    shift = np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=-1)
    return items & ((1 << ENT_BITS) - 1), shift


def kfmm_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (default stream)."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(ctx, _lib.kfmm_set_stream(ctx, raw))


def kfmm_build(ctx, src_xyz, src_nrm, trg_xyz):
    _check(ctx, _lib.kfmm_build(ctx, _ptr(src_xyz), _ptr(src_nrm), _nrows(src_xyz), _ptr(trg_xyz), _nrows(trg_xyz)))


def kfmm_build_sets(ctx, src_off, src_xyz, src_nrm, trg_off, trg_xyz):
    """src_off, trg_off: n_sets + 1 offsets (host int64) of the sets in the concatenated points."""
    so = np.ascontiguousarray(src_off, dtype=np.int64)
    to = np.ascontiguousarray(trg_off, dtype=np.int64)
    if so.shape != to.shape or so.ndim != 1 or len(so) < 2:
        raise ValueError("src_off and trg_off need the same n_sets + 1 entries")
    _check(ctx, _lib.kfmm_build_sets(ctx, len(so) - 1, so.ctypes.data, _ptr(src_xyz), _ptr(src_nrm),
                                     to.ctypes.data, _ptr(trg_xyz)))


def kfmm_eval(ctx, sl_den, dl_den, out, kind=KFMM_DISP, ncol=1):
    _check(ctx, _lib.kfmm_eval(ctx, _ptr(sl_den), _ptr(dl_den), int(ncol), int(kind), _ptr(out)))
    return out


def kfmm_direct(ctx, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, kind=KFMM_DISP, precision=KFMM_FP32):
    _check(ctx, _lib.kfmm_direct(ctx, int(precision), _ptr(trg_xyz), _nrows(trg_xyz), _ptr(src_xyz), _ptr(src_nrm),
                                 _nrows(src_xyz), _ptr(sl_den), _ptr(dl_den), int(kind), _ptr(out)))
    return out


def kfmm_direct_noalloc(ctx, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, kind=KFMM_DISP,
                        precision=KFMM_FP32):
    """kfmm_direct for callers that cannot allocate device memory: device arrays only, partial
    sums in the library's fixed 16 MiB scratch array.  Enqueued on the context stream (no
    synchronisation); overlapping calls race on the shared scratch."""
    _check(ctx, _lib.kfmm_direct_noalloc(ctx, int(precision), _ptr(trg_xyz), _nrows(trg_xyz), _ptr(src_xyz),
                                         _ptr(src_nrm), _nrows(src_xyz), _ptr(sl_den), _ptr(dl_den), int(kind),
                                         _ptr(out)))
    return out


def kfmm_direct_hi(ctx, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, near_radius=0.0):
    """FP64-grade displacement sum at FP32 rate (FP64 arrays); pairs closer than near_radius
    are summed wholly in FP64."""
    _check(ctx, _lib.kfmm_direct_hi(ctx, _ptr(trg_xyz), _nrows(trg_xyz), _ptr(src_xyz), _ptr(src_nrm),
                                    _nrows(src_xyz), _ptr(sl_den), _ptr(dl_den), float(near_radius), _ptr(out)))
    return out


def kfmm_get_stats(ctx) -> dict:
    st = kfmm_stats()
    _check(ctx, _lib.kfmm_get_stats(ctx, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in kfmm_stats._fields_}


def kfmm_export_tree(ctx) -> dict:
    st = kfmm_get_stats(ctx)
    nb, ns, nt = st["n_boxes"], st["n_src"], st["n_trg"]
    out = {"level": np.zeros(nb, np.int32), "anchor": np.zeros((nb, 3), np.int32), "parent": np.zeros(nb, np.int32),
           "src": np.zeros((nb, 2), np.int32), "trg": np.zeros((nb, 2), np.int32),
           "src_perm": np.zeros(ns, np.int32), "trg_perm": np.zeros(nt, np.int32)}
    _check(ctx, _lib.kfmm_export_tree(ctx, *[_ptr(out[k]) for k in
                                             ("level", "anchor", "parent", "src", "trg", "src_perm", "trg_perm")]))
    return out


def kfmm_export_list(ctx, which: str):
    n = _i64(0)
    _check(ctx, _lib.kfmm_export_list(ctx, which.encode(), None, None, ctypes.byref(n)))
    nb = kfmm_get_stats(ctx)["n_boxes"]
    off = np.zeros(nb + 1, np.int32)
    items = np.zeros(max(1, n.value), np.int32)
    _check(ctx, _lib.kfmm_export_list(ctx, which.encode(), _ptr(off), _ptr(items), ctypes.byref(n)))
    return off, items[: n.value]


# ------------------------------------------------------------- partition over several GPUs
class kfmm_tree_view(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int32)] + [(f, ctypes.c_void_p) for f in (
        "level", "anchor", "parent", "box_src", "box_trg", "u_off", "u_idx", "v_off", "v_idx", "w_off", "w_idx",
        "x_off", "x_idx")]


class TreeView:
    """Host arrays of a tree (kfmm_export_tree / kfmm_export_list layout) and the C view of
    them.  tree: dict with level, anchor, parent, src, trg; lists: {"U": (off, idx), ...}."""

    def __init__(self, tree, lists):
        c = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
        self.arrays = {"level": c(tree["level"]), "anchor": c(tree["anchor"]), "parent": c(tree["parent"]),
                       "box_src": c(tree["src"]), "box_trg": c(tree["trg"])}
        for k in "UVWX":
            off, idx = lists[k]
            self.arrays[k.lower() + "_off"] = c(off)
            self.arrays[k.lower() + "_idx"] = c(idx) if len(idx) else np.zeros(1, np.int32)
        self.n_boxes = len(self.arrays["level"])
        self.view = kfmm_tree_view(self.n_boxes, *[self.arrays[f].ctypes.data for f, _ in kfmm_tree_view._fields_[1:]])

    @classmethod
    def from_context(cls, ctx):
        """The tree of a built context."""
        return cls(kfmm_export_tree(ctx), {k: kfmm_export_list(ctx, k) for k in "UVWX"})


def kfmm_shard_plan(tv: TreeView, n_ranks: int, box_cost=None):
    """(box_owner [n_boxes], leaf_order [n_leaves], rank_cost [n_ranks])."""
    owner = np.zeros(tv.n_boxes, np.int32)
    order = np.zeros(tv.n_boxes, np.int32)
    rc = np.zeros(n_ranks, np.float64)
    cost = None if box_cost is None else np.ascontiguousarray(box_cost, dtype=np.float64)
    _check(None, _lib.kfmm_shard_plan(ctypes.byref(tv.view), int(n_ranks), _ptr(cost), _ptr(owner), _ptr(order),
                                      _ptr(rc)))
    n_leaves = int(np.sum(~np.isin(np.arange(tv.n_boxes), tv.arrays["parent"])))
    return owner, order[:n_leaves], rc


def kfmm_shard_let(tv: TreeView, box_owner, rank: int):
    """Locally essential tree of `rank`: (source boxes, upward boxes, shared boxes)."""
    own = np.ascontiguousarray(box_owner, dtype=np.int32)
    ns, nu, nh = _i64(0), _i64(0), _i64(0)
    _check(None, _lib.kfmm_shard_let(ctypes.byref(tv.view), _ptr(own), int(rank), None, ctypes.byref(ns), None,
                                     ctypes.byref(nu), None, ctypes.byref(nh)))
    s, u, h = (np.zeros(max(1, n.value), np.int32) for n in (ns, nu, nh))
    _check(None, _lib.kfmm_shard_let(ctypes.byref(tv.view), _ptr(own), int(rank), _ptr(s), ctypes.byref(ns), _ptr(u),
                                     ctypes.byref(nu), _ptr(h), ctypes.byref(nh)))
    return s[:ns.value], u[:nu.value], h[:nh.value]


PHASES = ("tree", "pack", "s2m", "up_pinv", "m2m", "m2l", "p2l", "down", "eval", "m2l_basis", "tree_split",
          "tree_lists", "plans")


def kfmm_set_profiling(ctx, enable: bool):
    _check(ctx, _lib.kfmm_set_profiling(ctx, int(bool(enable))))


def kfmm_get_phase_times(ctx, reset: bool = False) -> dict:
    """{phase: (milliseconds, calls)} accumulated since the last reset."""
    ms = np.zeros(len(PHASES), np.float64)
    cnt = np.zeros(len(PHASES), np.int64)
    _check(ctx, _lib.kfmm_get_phase_times(ctx, _ptr(ms), _ptr(cnt), int(bool(reset))))
    return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}


def kfmm_measure_fp32_peak(ctx) -> dict:
    """Measured FP32 FMA throughput of the context's GPU: {"tflops", "ms", "n_sms"}."""
    tf, ms, sms = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int32(0)
    _check(ctx, _lib.kfmm_measure_fp32_peak(ctx, ctypes.byref(tf), ctypes.byref(ms), ctypes.byref(sms)))
    return {"tflops": tf.value, "ms": ms.value, "n_sms": sms.value}


def kfmm_status_str(status: int) -> str:
    return _lib.kfmm_status_str(status).decode()


class Kfmm:
    """Small owner of a context: ``with Kfmm(p=6) as f: f.build(...); f.eval(...)``."""

    def __init__(self, options: kfmm_options | None = None, **overrides):
        self.handle = kfmm_create(options, **overrides)

    def close(self):
        if self.handle:
            kfmm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, K, G):
        kfmm_set_material(self.handle, K, G)

    def set_stream(self, stream):
        kfmm_set_stream(self.handle, stream)

    def set_periodic(self, lo=None, side=1.0):
        """Sums over the cubic lattice of the cell [lo, lo + side]^3 from the next build on
        (lo None: free space again)."""
        kfmm_set_periodic(self.handle, lo, side)

    def build(self, src_xyz, src_nrm, trg_xyz):
        kfmm_build(self.handle, src_xyz, src_nrm, trg_xyz)

    def build_sets(self, src_off, src_xyz, src_nrm, trg_off, trg_xyz):
        kfmm_build_sets(self.handle, src_off, src_xyz, src_nrm, trg_off, trg_xyz)

    def selftest_bounded_wait(self, polls=4096):
        """Status of the bounded-wait check (KFMM_ERR_DEVICE_TIMEOUT as designed)."""
        return int(_lib.kfmm_selftest_bounded_wait(self.handle, int(polls)))

    def eval(self, sl_den, dl_den, out, kind=KFMM_DISP, ncol=1):
        return kfmm_eval(self.handle, sl_den, dl_den, out, kind, ncol)

    def direct(self, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, kind=KFMM_DISP, precision=KFMM_FP32):
        return kfmm_direct(self.handle, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, kind, precision)

    def direct_hi(self, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, near_radius=0.0):
        return kfmm_direct_hi(self.handle, trg_xyz, src_xyz, src_nrm, sl_den, dl_den, out, near_radius)

    def stats(self):
        return kfmm_get_stats(self.handle)

    def measure_fp32_peak(self):
        return kfmm_measure_fp32_peak(self.handle)

    def set_profiling(self, enable=True):
        kfmm_set_profiling(self.handle, enable)

    def phase_times(self, reset=False):
        return kfmm_get_phase_times(self.handle, reset)

    def export_tree(self):
        return kfmm_export_tree(self.handle)

    def export_list(self, which):
        return kfmm_export_list(self.handle, which)


# ------------------------------------------------------------------------------- BEM layer
BEM_FMM = 0
BEM_DIRECT_FP64 = 1
BEM_DIRECT_HI = 2


class bem_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("x0", ctypes.c_void_p), ("refine", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int)]


class bem_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("matvecs", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres", ctypes.c_double), ("seconds", ctypes.c_double), ("outer", ctypes.c_int),
                ("matvecs_hi", ctypes.c_int), ("x0_relres", ctypes.c_double)]


_bsig = {
    "bem_default_solve_opts": (None, [ctypes.POINTER(bem_solve_opts)]),
    "bem_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(kfmm_options), ctypes.c_int, _vp, _i64, _vp,
                                  _i64]),
    "bem_destroy": (ctypes.c_int, [_vp]),
    "bem_set_material": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
    "bem_set_stream": (ctypes.c_int, [_vp, _vp]),
    "bem_set_bc": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "bem_set_quadrature": (ctypes.c_int, [_vp, ctypes.c_int]),
    "bem_set_periodic": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_double]),
    "bem_set_macro_stress": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "bem_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bem_matvec": (ctypes.c_int, [_vp, _vp, _vp]),
    "bem_rhs": (ctypes.c_int, [_vp, _vp]),
    "bem_solve": (ctypes.c_int, [_vp, ctypes.POINTER(bem_solve_opts), _vp, _vp, ctypes.POINTER(bem_stats)]),
    "bem_set_solution": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "bem_interior": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "bem_topo_derivative": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "bem_last_error": (ctypes.c_char_p, [_vp]),
}
for _name, (_res, _args) in _bsig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _bcheck(h, status):
    if status != KFMM_OK:
        raise KfmmError(status, _lib.bem_last_error(h).decode() if h else "")


def bem_create(verts, tris, op=BEM_FMM, options: kfmm_options | None = None, **overrides):
    """verts [nv,3] float64, tris [nt,3] int32 (host or device).  Without options or a
    leaf_cap override the BEM picks its own leaf caps (leaf_cap = 0)."""
    o = options if options is not None else kfmm_default_options()
    if options is None:
        o.leaf_cap = 0
    for k, v in overrides.items():
        setattr(o, k, v)
    h = _vp()
    _bcheck(None, _lib.bem_create(ctypes.byref(h), ctypes.byref(o), int(op), _ptr(verts), _nrows(verts), _ptr(tris),
                                  _nrows(tris)))
    return h


def bem_destroy(h):
    _bcheck(None, _lib.bem_destroy(h))


def bem_set_material(h, K, G):
    _bcheck(h, _lib.bem_set_material(h, float(K), float(G)))


def bem_set_stream(h, stream):
    _bcheck(h, _lib.bem_set_stream(h, getattr(stream, "cuda_stream", stream)))


def _ncol3(a):
    """Columns of a [nt, 3*ncol] array."""
    if a.ndim != 2 or a.shape[1] % 3:
        raise ValueError("expected an array of shape [nt, 3*ncol]")
    return a.shape[1] // 3


def bem_set_bc(h, known_is_disp, values):
    """known_is_disp [nt,3] uint8; values [nt,3*ncol] float64 (ncol load cases)."""
    _bcheck(h, _lib.bem_set_bc(h, _ptr(known_is_disp), _ptr(values), _ncol3(values)))


def bem_apply(h, u, t, out):
    _bcheck(h, _lib.bem_apply(h, _ptr(u), _ptr(t), _ptr(out)))
    return out


def bem_matvec(h, x, y):
    _bcheck(h, _lib.bem_matvec(h, _ptr(x), _ptr(y)))
    return y


def bem_rhs(h, out):
    _bcheck(h, _lib.bem_rhs(h, _ptr(out)))
    return out


def bem_solve(h, u=None, t=None, tol=1e-6, restart=30, maxit=1000, x0=None, raise_on_fail=True, refine=False,
              inner_tol=1e-3, max_outer=30):
    """GMRES solve of Eq. num2; fills u, t [nt,3] float64 (host or device). With refine=True or 1
    (FMM contexts): mixed-precision iterative refinement, FP64-grade residuals by the
    compensated direct sum, FMM corrections; refine=2: the same with FP64 direct residuals.
    Returns stats dict."""
    o = bem_solve_opts()
    _lib.bem_default_solve_opts(ctypes.byref(o))
    o.tol, o.restart, o.maxit = float(tol), int(restart), int(maxit)
    o.refine, o.inner_tol, o.max_outer = int(refine), float(inner_tol), int(max_outer)
    o.x0 = _ptr(x0)
    st = bem_stats()
    status = _lib.bem_solve(h, ctypes.byref(o), _ptr(u), _ptr(t), ctypes.byref(st))
    if raise_on_fail or status not in (KFMM_OK, KFMM_ERR_NOT_CONVERGED):
        _bcheck(h, status)
    return {f: getattr(st, f) for f, _ in bem_stats._fields_}


def bem_set_solution(h, u, t):
    """u, t [nt, 3*ncol] float64."""
    _bcheck(h, _lib.bem_set_solution(h, _ptr(u), _ptr(t), _ncol3(u)))


def bem_interior(h, pts, disp=None, stress=None):
    _bcheck(h, _lib.bem_interior(h, _ptr(pts), _nrows(pts), _ptr(disp), _ptr(stress)))


def bem_topo_derivative(h, pts, td=None, energy=None, stress=None):
    _bcheck(h, _lib.bem_topo_derivative(h, _ptr(pts), _nrows(pts), _ptr(td), _ptr(energy), _ptr(stress)))


class Bem:
    """Owner of a BEM context: ``with Bem(verts, tris) as b: b.set_bc(...); b.solve(u, t)``."""

    def __init__(self, verts, tris, op=BEM_FMM, options: kfmm_options | None = None, **overrides):
        self.handle = bem_create(verts, tris, op, options, **overrides)

    def close(self):
        if self.handle:
            bem_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, K, G):
        bem_set_material(self.handle, K, G)

    def set_stream(self, stream):
        bem_set_stream(self.handle, stream)

    def set_bc(self, known_is_disp, values):
        bem_set_bc(self.handle, known_is_disp, values)

    def set_quadrature(self, near_levels):
        """Upsampled quadrature of the triangles sharing a vertex with a collocation triangle:
        the 4-node rule on 4^near_levels sub-triangles (1 = the 16-point rule everywhere)."""
        _bcheck(self.handle, _lib.bem_set_quadrature(self.handle, int(near_levels)))

    def set_periodic(self, lo=None, side=1.0):
        """The surface is one cell [lo, lo + side]^3 of a periodic surface: every sum runs over
        the lattice (lo None: free space again)."""
        if lo is None:
            _bcheck(self.handle, _lib.bem_set_periodic(self.handle, 0, None, 1.0))
            return
        c = np.ascontiguousarray(lo, dtype=np.float64).reshape(3)
        _bcheck(self.handle, _lib.bem_set_periodic(self.handle, 1, c.ctypes.data, float(side)))

    def set_macro_stress(self, stress6=None):
        """Uniform stress per load case [ncol, 6] (Voigt xx, yy, zz, yz, xz, xy) added before the
        TD (the homogeneous part of a periodic cell's total stress); None clears."""
        if stress6 is None:
            _bcheck(self.handle, _lib.bem_set_macro_stress(self.handle, None, 0))
            return
        m = np.ascontiguousarray(stress6, dtype=np.float64).reshape(-1, 6)
        _bcheck(self.handle, _lib.bem_set_macro_stress(self.handle, m.ctypes.data, m.shape[0]))

    def apply(self, u, t, out):
        return bem_apply(self.handle, u, t, out)

    def matvec(self, x, y):
        return bem_matvec(self.handle, x, y)

    def rhs(self, out):
        return bem_rhs(self.handle, out)

    def solve(self, u=None, t=None, **kw):
        return bem_solve(self.handle, u, t, **kw)

    def set_solution(self, u, t):
        bem_set_solution(self.handle, u, t)

    def interior(self, pts, disp=None, stress=None):
        bem_interior(self.handle, pts, disp, stress)

    def topo_derivative(self, pts, td=None, energy=None, stress=None):
        bem_topo_derivative(self.handle, pts, td, energy, stress)


def material_K(G: float, nu: float) -> float:
    """Bulk modulus from G and nu (the ABI takes K and G, Eq. elast)."""
    return 2.0 * G * (1.0 + nu) / (3.0 * (1.0 - 2.0 * nu))


# ------------------------------------------------------------------ optimisation driver (host)
_vsig = {
    "kfmm_voxel_surface": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _vp,
                                          _vp, ctypes.POINTER(_i64), _vp, ctypes.POINTER(_i64), _vp, _vp]),
    "kfmm_voxel_surface_periodic": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                   _vp, _vp, ctypes.POINTER(_i64), _vp, ctypes.POINTER(_i64), _vp,
                                                   _vp]),
    "kfmm_voxel_threshold": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                            ctypes.c_double, ctypes.POINTER(_i64)]),
    "kfmm_voxel_clean": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                        ctypes.POINTER(_i64)]),
}
for _name, (_res, _args) in _vsig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _mask_arg(mask):
    if not (isinstance(mask, np.ndarray) and mask.dtype == np.uint8 and mask.ndim == 3 and mask.flags["C_CONTIGUOUS"]):
        raise ValueError("mask must be a C-contiguous uint8 [nx, ny, nz] numpy array")
    return mask.shape


def voxel_surface(mask, h=1.0, origin=(0.0, 0.0, 0.0), periodic=False):
    """Boundary triangles of the material voxels: (verts [nv,3], tris [nt,3] int32,
    face_cell [nt] int64, face_dir [nt] int8).  periodic: the mask is one cell of a periodic
    pattern (neighbours wrap around, no faces on the cell's boundary)."""
    nx, ny, nz = _mask_arg(mask)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    nv, nt = _i64(0), _i64(0)
    fn = _lib.kfmm_voxel_surface_periodic if periodic else _lib.kfmm_voxel_surface
    _check(None, fn(_ptr(mask), nx, ny, nz, float(h), _ptr(o), None, ctypes.byref(nv), None,
                    ctypes.byref(nt), None, None))
    V = np.zeros((nv.value, 3))
    T = np.zeros((nt.value, 3), np.int32)
    cell = np.zeros(nt.value, np.int64)
    fdir = np.zeros(nt.value, np.int8)
    _check(None, fn(_ptr(mask), nx, ny, nz, float(h), _ptr(o), _ptr(V), ctypes.byref(nv),
                    _ptr(T), ctypes.byref(nt), _ptr(cell), _ptr(fdir)))
    return V, T, cell, fdir


def voxel_threshold(mask, td, C, frozen=None):
    """In place: material voxels below D_min + C (D_max - D_min) become void. Returns the count."""
    nx, ny, nz = _mask_arg(mask)
    td = np.ascontiguousarray(td, dtype=np.float32).reshape(-1)
    if td.size != mask.size:
        raise ValueError("td must have one value per voxel")
    fz = None if frozen is None else np.ascontiguousarray(frozen, dtype=np.uint8)
    n = _i64(0)
    _check(None, _lib.kfmm_voxel_threshold(_ptr(mask), nx, ny, nz, _ptr(td), _ptr(fz), float(C), ctypes.byref(n)))
    return n.value


def voxel_clean(mask, support=None, keep=None):
    """In place: isolated voxels and material not connected to `support` become void
    (support and keep voxels stay). Returns the count."""
    nx, ny, nz = _mask_arg(mask)
    sp = None if support is None else np.ascontiguousarray(support, dtype=np.uint8)
    kp = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    n = _i64(0)
    _check(None, _lib.kfmm_voxel_clean(_ptr(mask), nx, ny, nz, _ptr(sp), _ptr(kp), ctypes.byref(n)))
    return n.value


# ------------------------------------------------------------------ learned warm start (MLP)
class mlp_train_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double), ("seed", ctypes.c_uint64)]


class mlp_train_stats(ctypes.Structure):
    _fields_ = [("final_loss", ctypes.c_double), ("steps", ctypes.c_int64)]


_msig = {
    "mlp_default_train_opts": (None, [ctypes.POINTER(mlp_train_opts)]),
    "mlp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_uint64]),
    "mlp_destroy": (ctypes.c_int, [_vp]),
    "mlp_set_stream": (ctypes.c_int, [_vp, _vp]),
    "mlp_num_params": (ctypes.c_int64, [_vp]),
    "mlp_set_bf16": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mlp_get_params": (ctypes.c_int, [_vp, _vp]),
    "mlp_set_params": (ctypes.c_int, [_vp, _vp]),
    "mlp_get_normalizers": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "mlp_forward": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "mlp_train": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(mlp_train_opts),
                                 ctypes.POINTER(mlp_train_stats)]),
    "mlp_last_error": (ctypes.c_char_p, [_vp]),
}
for _name, (_res, _args) in _msig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _mcheck(h, status):
    if status != KFMM_OK:
        raise KfmmError(status, _lib.mlp_last_error(h).decode() if h else "")


def _f32(a):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float32)


class Mlp:
    """Warm-start network: n_in -> n_hidden (ReLU) x (n_layers - 1) -> n_out, trained on the GPU."""

    def __init__(self, n_in=11, n_hidden=256, n_layers=4, n_out=3, seed=1612):
        h = _vp()
        _mcheck(None, _lib.mlp_create(ctypes.byref(h), n_in, n_hidden, n_layers, n_out, seed))
        self.handle = h
        self.n_in, self.n_out = n_in, n_out

    def close(self):
        if self.handle:
            _lib.mlp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(_lib.mlp_num_params(self.handle))

    def set_bf16(self, on=True):
        _mcheck(self.handle, _lib.mlp_set_bf16(self.handle, int(bool(on))))

    def get_params(self):
        p = np.zeros(self.num_params, np.float32)
        _mcheck(self.handle, _lib.mlp_get_params(self.handle, _ptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError("wrong parameter count")
        _mcheck(self.handle, _lib.mlp_set_params(self.handle, _ptr(p)))

    def normalizers(self):
        xm, xs = np.zeros(self.n_in, np.float32), np.zeros(self.n_in, np.float32)
        ym, ys = np.zeros(self.n_out, np.float32), np.zeros(self.n_out, np.float32)
        _mcheck(self.handle, _lib.mlp_get_normalizers(self.handle, _ptr(xm), _ptr(xs), _ptr(ym), _ptr(ys)))
        return xm, xs, ym, ys

    def forward(self, X, out=None):
        X = _f32(X)
        if out is None:
            out = np.zeros((_nrows(X), self.n_out), np.float32)
        _mcheck(self.handle, _lib.mlp_forward(self.handle, _ptr(X), _nrows(X), _ptr(out)))
        return out

    def loss_grad(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        loss = ctypes.c_double(0.0)
        g = np.zeros(self.num_params, np.float32)
        _mcheck(self.handle, _lib.mlp_loss_grad(self.handle, _ptr(X), _ptr(Y), _nrows(X), ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, X, Y, epochs=200, batch=4096, lr=1e-3, seed=1612):
        X, Y = _f32(X), _f32(Y)
        o = mlp_train_opts(int(epochs), int(batch), float(lr), int(seed))
        st = mlp_train_stats()
        _mcheck(self.handle, _lib.mlp_train(self.handle, _ptr(X), _ptr(Y), _nrows(X), ctypes.byref(o), ctypes.byref(st)))
        return {"final_loss": st.final_loss, "steps": st.steps}
