"""ctypes binding of libejoin (the C ABI declared in include/ejoin.h).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  Names mirror the C entry points.  Device arrays are torch CUDA
tensors; host arrays are numpy arrays (or CPU tensors).  If the compiled
library is missing, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import weakref
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libejoin.so")

EJOIN_OK, EJOIN_EINVAL, EJOIN_ENOMEM, EJOIN_EOVERFLOW = 0, 1, 2, 3
EJOIN_ENONFINITE, EJOIN_ECUDA, EJOIN_ETIMEOUT, EJOIN_EUNSUPPORTED = 4, 5, 6, 7
EJOIN_F32, EJOIN_BF16, EJOIN_FP8_E4M3, EJOIN_TF32 = 0, 1, 2, 3
EJOIN_FLAG_COUNT_ONLY, EJOIN_FLAG_TIMING, EJOIN_FLAG_FUSED, EJOIN_FLAG_NO_SYMMETRY = 0x1, 0x2, 0x4, 0x8
EJOIN_FLAG_HOST_COPY, EJOIN_FLAG_GATHER_RESCORE, EJOIN_FLAG_SORT, EJOIN_FLAG_PANEL_RESCORE = 0x10, 0x20, 0x40, 0x80
OPS = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}
PRECS = {"f32": EJOIN_F32, "bf16": EJOIN_BF16, "fp8": EJOIN_FP8_E4M3, "tf32": EJOIN_TF32}


class ejoin_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("prec", ctypes.c_int32),
                ("band", ctypes.c_float), ("fp64_band", ctypes.c_float), ("capacity_hint", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("timeout_cycles", ctypes.c_uint64), ("group_m", ctypes.c_int32)]


class ejoin_rel(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("ld", ctypes.c_int64)]


class ejoin_sel(ctypes.Structure):
    _fields_ = [("attr", ctypes.c_void_p), ("op", ctypes.c_int32), ("c", ctypes.c_int32),
                ("bits", ctypes.c_void_p)]


class ejoin_pair(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("sim", ctypes.c_float)]


class ejoin_pairs(ctypes.Structure):
    _fields_ = [("d_pairs", ctypes.c_void_p), ("capacity", ctypes.c_uint64), ("d_count", ctypes.c_void_p),
                ("count", ctypes.c_uint64)]


class ejoin_stats(ctypes.Structure):
    _fields_ = [("n_sel_r", ctypes.c_uint64), ("n_sel_s", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("fp64_rescored", ctypes.c_uint64), ("pairs", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("band", ctypes.c_float), ("ms_select", ctypes.c_float), ("ms_normalize", ctypes.c_float),
                ("ms_contract", ctypes.c_float), ("ms_rescore", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_h2d", ctypes.c_float), ("ms_d2h", ctypes.c_float), ("contract_retries", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("h2d_bytes", ctypes.c_uint64), ("host_in_place", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ejoin_job(ctypes.Structure):
    _fields_ = [("R", ejoin_rel), ("S", ejoin_rel), ("eps", ctypes.c_float)]


class ejoin_job_sel(ctypes.Structure):
    _fields_ = [("R", ejoin_sel), ("S", ejoin_sel)]


class ejoin_batch_stats(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_int32), ("total_tiles", ctypes.c_int64), ("rows_r", ctypes.c_int64),
                ("rows_s", ctypes.c_int64), ("group_m", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("candidate_capacity", ctypes.c_uint64), ("pair_capacity", ctypes.c_uint64),
                ("band", ctypes.c_float), ("ms_normalize", ctypes.c_float), ("ms_contract", ctypes.c_float),
                ("ms_rescore", ctypes.c_float)]


EJOIN_BATCH_GRAPH, EJOIN_BATCH_AUTOTUNE = 0x1, 0x2


class ejoin_prune_stats(ctypes.Structure):
    _fields_ = [("tiles_total", ctypes.c_uint64), ("tiles_kept", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("pairs", ctypes.c_uint64), ("ms_prepare", ctypes.c_float), ("ms_bound", ctypes.c_float),
                ("ms_contract", ctypes.c_float), ("ms_rescore", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ball_radius_mean_a", ctypes.c_float), ("ball_radius_mean_b", ctypes.c_float),
                ("wide_ball_frac_a", ctypes.c_float), ("wide_ball_frac_b", ctypes.c_float),
                ("anchors_a", ctypes.c_uint64), ("max_group_rows_a", ctypes.c_uint64),
                ("ms_sketch_a", ctypes.c_float), ("ms_cover_a", ctypes.c_float), ("ms_assign_a", ctypes.c_float),
                ("recall_est", ctypes.c_float), ("recall_sample_rows", ctypes.c_uint64),
                ("recall_sample_matches", ctypes.c_uint64), ("ms_tile_stats", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class ejoin_sketch_train_cfg(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("label_margin", ctypes.c_float), ("w_join", ctypes.c_float),
                ("n_pairs", ctypes.c_int64), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("recall", ctypes.c_float), ("cal_margin", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("init", ctypes.c_int32)]


class ejoin_sketch_train_report(ctypes.Structure):
    _fields_ = [("label_join_pairs", ctypes.c_uint64), ("labelled_join", ctypes.c_uint64),
                ("labelled_random", ctypes.c_uint64), ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float),
                ("calibration_matches", ctypes.c_uint64), ("eps_sketch", ctypes.c_float),
                ("ms_label", ctypes.c_float), ("ms_train", ctypes.c_float), ("ms_calibrate", ctypes.c_float)]

_lib = None


def _open(path: str):
    if not os.path.exists(path):
        raise RuntimeError(f"libejoin.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    return ctypes.CDLL(path)


def load_library(path: str = LIB_PATH):
    """Load libejoin.so (built by paper_2312_01476_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    lib = _open(path)
    P = ctypes.POINTER
    lib.ejoin_create.restype = ctypes.c_int
    lib.ejoin_create.argtypes = [P(ctypes.c_void_p), P(ejoin_config)]
    lib.ejoin_destroy.restype = None
    lib.ejoin_destroy.argtypes = [ctypes.c_void_p]
    lib.ejoin_set_timeout.restype = ctypes.c_int
    lib.ejoin_set_timeout.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.ejoin_normalize.restype = ctypes.c_int
    lib.ejoin_normalize.argtypes = [ctypes.c_void_p, ejoin_rel, P(ejoin_sel), ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    lib.ejoin_padded_dim.restype = ctypes.c_int64
    lib.ejoin_padded_dim.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.ejoin_threshold.restype = ctypes.c_int
    lib.ejoin_threshold.argtypes = [ctypes.c_void_p, ejoin_rel, ejoin_rel, ctypes.c_float, P(ejoin_sel),
                                    P(ejoin_sel), P(ejoin_pairs)]
    lib.ejoin_threshold_host.restype = ctypes.c_int
    lib.ejoin_threshold_host.argtypes = [ctypes.c_void_p, ejoin_rel, ejoin_rel, ctypes.c_float, P(ejoin_sel),
                                         P(ejoin_sel), ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_uint64)]
    lib.ejoin_top1.restype = ctypes.c_int
    lib.ejoin_top1.argtypes = [ctypes.c_void_p, ejoin_rel, ejoin_rel, P(ejoin_sel), P(ejoin_sel), P(ejoin_pairs)]
    lib.ejoin_eselect.restype = ctypes.c_int
    lib.ejoin_eselect.argtypes = [ctypes.c_void_p, ejoin_rel, P(ejoin_sel), ejoin_rel, ctypes.c_float,
                                  P(ejoin_pairs)]
    lib.ejoin_topk.restype = ctypes.c_int
    lib.ejoin_topk.argtypes = [ctypes.c_void_p, ejoin_rel, ejoin_rel, ctypes.c_int32, P(ejoin_sel), P(ejoin_sel),
                               P(ejoin_pairs)]
    lib.ejoin_pairs_free.restype = ctypes.c_int
    lib.ejoin_pairs_free.argtypes = [ctypes.c_void_p, P(ejoin_pairs)]
    lib.ejoin_last_stats.restype = ctypes.c_int
    lib.ejoin_last_stats.argtypes = [ctypes.c_void_p, P(ejoin_stats)]
    lib.ejoin_strerror.restype = ctypes.c_char_p
    lib.ejoin_strerror.argtypes = [ctypes.c_int]
    lib.ejoin_version.restype = ctypes.c_char_p
    lib.ejoin_version.argtypes = []
    lib.ejoin_batch_create_sel.restype = ctypes.c_int
    lib.ejoin_batch_create_sel.argtypes = [ctypes.c_void_p, P(ejoin_job), P(ejoin_job_sel), ctypes.c_int32,
                                           ctypes.c_uint32, P(ctypes.c_void_p)]
    lib.ejoin_batch_create.restype = ctypes.c_int
    lib.ejoin_batch_create.argtypes = [ctypes.c_void_p, P(ejoin_job), ctypes.c_int32, ctypes.c_uint32,
                                       P(ctypes.c_void_p)]
    lib.ejoin_batch_run.restype = ctypes.c_int
    lib.ejoin_batch_run.argtypes = [ctypes.c_void_p]
    lib.ejoin_batch_wait.restype = ctypes.c_int
    lib.ejoin_batch_wait.argtypes = [ctypes.c_void_p, P(ctypes.c_uint64)]
    lib.ejoin_batch_result.restype = ctypes.c_int
    lib.ejoin_batch_result.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), P(ctypes.c_uint64)]
    lib.ejoin_batch_info.restype = ctypes.c_int
    lib.ejoin_batch_info.argtypes = [ctypes.c_void_p, P(ejoin_batch_stats)]
    lib.ejoin_batch_destroy.restype = None
    lib.ejoin_batch_destroy.argtypes = [ctypes.c_void_p]
    vp = ctypes.c_void_p
    lib.ejoin_sketch_create.restype = ctypes.c_int
    lib.ejoin_sketch_create.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(vp)]
    lib.ejoin_sketch_destroy.restype = None
    lib.ejoin_sketch_destroy.argtypes = [vp]
    lib.ejoin_sketch_num_params.restype = ctypes.c_int64
    lib.ejoin_sketch_num_params.argtypes = [vp]
    lib.ejoin_sketch_set_params.restype = ctypes.c_int
    lib.ejoin_sketch_set_params.argtypes = [vp, vp]
    lib.ejoin_sketch_get_params.restype = ctypes.c_int
    lib.ejoin_sketch_get_params.argtypes = [vp, vp]
    lib.ejoin_sketch_forward.restype = ctypes.c_int
    lib.ejoin_sketch_forward.argtypes = [vp, ejoin_rel, vp]
    lib.ejoin_sketch_grad.restype = ctypes.c_int
    lib.ejoin_sketch_grad.argtypes = [vp, ejoin_rel, vp, vp, vp, vp, vp, ctypes.c_int64, vp, P(ctypes.c_float)]
    lib.ejoin_sketch_train_step.restype = ctypes.c_int
    lib.ejoin_sketch_train_step.argtypes = [vp, ejoin_rel, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float,
                                            P(ctypes.c_float)]
    lib.ejoin_sketch_pair_sims.restype = ctypes.c_int
    lib.ejoin_sketch_pair_sims.argtypes = [vp, ejoin_rel, vp, vp, vp, ctypes.c_int64, vp]
    lib.ejoin_row_inv_norm.restype = ctypes.c_int
    lib.ejoin_row_inv_norm.argtypes = [vp, ejoin_rel, vp]
    lib.ejoin_score_pairs.restype = ctypes.c_int
    lib.ejoin_score_pairs.argtypes = [vp, ejoin_rel, ejoin_rel, vp, vp, ctypes.c_int64, vp]
    lib.ejoin_threshold_pruned.restype = ctypes.c_int
    lib.ejoin_threshold_pruned.argtypes = [vp, vp, ejoin_rel, ejoin_rel, ctypes.c_float, ctypes.c_float,
                                           P(ejoin_pairs), P(ejoin_prune_stats), P(ctypes.c_float)]
    lib.ejoin_sketch_forward_tc.restype = ctypes.c_int
    lib.ejoin_sketch_forward_tc.argtypes = [vp, ejoin_rel, vp]
    lib.ejoin_sketch_train.restype = ctypes.c_int
    lib.ejoin_sketch_train.argtypes = [vp, ejoin_rel, ejoin_rel, P(ejoin_sketch_train_cfg), P(ctypes.c_float),
                                       P(ejoin_sketch_train_report)]
    if path == LIB_PATH:
        _lib = lib
    return lib


# Live handles, closed in dependency order when the interpreter exits (sketches and batches
# before the contexts they were created on), so that no handle is released after the
# objects it refers to, whatever order the interpreter tears its objects down in.
_live_dependents = weakref.WeakSet()
_live_contexts = weakref.WeakSet()


@atexit.register
def _close_live_handles():
    for group in (_live_dependents, _live_contexts):
        for obj in list(group):
            try:
                obj.close()
            except Exception:
                pass


class EJoinError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {ejoin_strerror(status)} (status {status})")


def ejoin_strerror(status: int) -> str:
    return load_library().ejoin_strerror(int(status)).decode()


def ejoin_version() -> str:
    return load_library().ejoin_version().decode()


def ejoin_padded_dim(prec: int, d: int) -> int:
    return int(load_library().ejoin_padded_dim(int(prec), int(d)))


def _check(status: int, where: str):
    if status != EJOIN_OK:
        raise EJoinError(status, where)


@dataclass
class Sel:
    """Selection ``attr op c`` (and/or a bitmask) on one relation (Sec. III-C, Eq. Selection)."""
    attr: object = None  # int32 array (torch CUDA tensor for device calls, numpy for host calls)
    op: str = "<"
    c: int = 0
    bits: object = None  # uint32 words, bit r % 32 of word r // 32


class Ctx:
    """An ejoin context: device, stream, precision, bands, flags."""

    def __init__(self, device: int = 0, stream: Optional[int] = None, prec="bf16", band: float = -1.0,
                 fp64_band: float = -1.0, capacity_hint: int = 0, flags: int = 0, timeout_cycles: int = 0,
                 group_m: int = 0):
        lib = load_library()
        self.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
        cfg = ejoin_config(int(device), ctypes.c_void_p(stream or 0), self.prec, float(band), float(fp64_band),
                           int(capacity_hint), int(flags), int(timeout_cycles), int(group_m))
        h = ctypes.c_void_p()
        _check(lib.ejoin_create(ctypes.byref(h), ctypes.byref(cfg)), "ejoin_create")
        self.handle = h
        self.device = device
        self._out = None  # cached device result buffer (torch int32 [cap, 3])
        _live_contexts.add(self)

    def close(self):
        if getattr(self, "handle", None):
            load_library().ejoin_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ejoin_create(**kw) -> Ctx:
    return Ctx(**kw)


def ejoin_destroy(ctx: Ctx):
    ctx.close()


def ejoin_set_timeout(ctx: Ctx, timeout_cycles: int):
    """Bound (SM cycles, 0 = default) on the device-side waits of later calls on ctx."""
    _check(load_library().ejoin_set_timeout(ctx.handle, int(timeout_cycles)), "ejoin_set_timeout")


def _dev_rel(x) -> ejoin_rel:
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise TypeError("relation must be a 2-D float32 CUDA tensor")
    if x.shape[0] == 0 or x.shape[1] == 0:
        return ejoin_rel(ctypes.c_void_p(x.data_ptr() or 0), x.shape[0], x.shape[1], x.shape[1])
    if x.stride(1) != 1 and x.shape[1] > 1:
        raise TypeError("relation rows must be contiguous")
    ld = x.stride(0) if x.shape[0] > 1 else x.shape[1]
    return ejoin_rel(ctypes.c_void_p(x.data_ptr()), x.shape[0], x.shape[1], ld)


def _dev_sel(s: Optional[Sel]):
    if s is None:
        return None
    import torch
    for a, dt in ((s.attr, torch.int32), (s.bits, torch.int32)):
        if a is not None and (not isinstance(a, torch.Tensor) or not a.is_cuda or not a.is_contiguous()
                              or a.dtype not in (torch.int32, torch.uint32)):
            raise TypeError("selection arrays must be contiguous int32 CUDA tensors")
    return ejoin_sel(ctypes.c_void_p(s.attr.data_ptr() if s.attr is not None else 0), OPS[s.op], int(s.c),
                     ctypes.c_void_p(s.bits.data_ptr() if s.bits is not None else 0))


def _sel_ptr(s):
    return ctypes.byref(s) if s is not None else None


@dataclass
class Result:
    i: object    # uint32-valued int32 tensor (original R row ids)
    j: object    # original S row ids
    sim: object  # float32 similarities
    count: int


def ejoin_threshold(ctx: Ctx, R, S, eps: float, selR: Optional[Sel] = None, selS: Optional[Sel] = None,
                    capacity: Optional[int] = None) -> Result:
    """Device E-join (Sec. III-C, Eq. (E-theta-Join)) of CUDA tensors R, S; returns views of a
    cached device result buffer (valid until the next call on ctx)."""
    import torch
    lib = load_library()
    rR, rS = _dev_rel(R), _dev_rel(S)
    sR, sS = _dev_sel(selR), _dev_sel(selS)
    cap = capacity or (ctx._out.shape[0] if ctx._out is not None else 1 << 16)
    for _ in range(3):
        if ctx._out is None or ctx._out.shape[0] < cap:
            ctx._out = torch.empty((cap, 3), dtype=torch.int32, device=R.device)
        out = ejoin_pairs(ctypes.c_void_p(ctx._out.data_ptr()), ctx._out.shape[0], None, 0)
        st = lib.ejoin_threshold(ctx.handle, rR, rS, ctypes.c_float(eps), _sel_ptr(sR), _sel_ptr(sS),
                                 ctypes.byref(out))
        if st == EJOIN_EOVERFLOW:
            cap = int(out.count) + 1024
            continue
        _check(st, "ejoin_threshold")
        n = int(out.count)
        v = ctx._out[:n]
        return Result(v[:, 0], v[:, 1], v[:, 2].view(torch.float32), n)
    raise EJoinError(EJOIN_EOVERFLOW, "ejoin_threshold")


def ejoin_eselect(ctx: Ctx, R, Q, eps: float, selR: Optional[Sel] = None, capacity: Optional[int] = None) -> Result:
    """Device ℰ-selection (Sec. III-C, Eq. (ℰ-Selection)) of the rows of CUDA tensor R against the query
    rows of CUDA tensor Q: every (i, q) with selR(i) and cos(R_i, Q_q) >= eps, as (i, j = q, sim).
    Returns views of a cached device result buffer (valid until the next call on ctx)."""
    import torch
    lib = load_library()
    rR, rQ = _dev_rel(R), _dev_rel(Q)
    sR = _dev_sel(selR)
    cap = capacity or (ctx._out.shape[0] if ctx._out is not None else 1 << 16)
    for _ in range(3):
        if ctx._out is None or ctx._out.shape[0] < cap:
            ctx._out = torch.empty((cap, 3), dtype=torch.int32, device=R.device)
        out = ejoin_pairs(ctypes.c_void_p(ctx._out.data_ptr()), ctx._out.shape[0], None, 0)
        st = lib.ejoin_eselect(ctx.handle, rR, _sel_ptr(sR), rQ, ctypes.c_float(eps), ctypes.byref(out))
        if st == EJOIN_EOVERFLOW:
            cap = int(out.count) + 1024
            continue
        _check(st, "ejoin_eselect")
        n = int(out.count)
        v = ctx._out[:n]
        return Result(v[:, 0], v[:, 1], v[:, 2].view(torch.float32), n)
    raise EJoinError(EJOIN_EOVERFLOW, "ejoin_eselect")


def ejoin_topk(ctx: Ctx, R, S, k: int, selR: Optional[Sel] = None, selS: Optional[Sel] = None) -> Result:
    """Device top-k join condition (Sec. VI-E), 1 <= k <= 32, of CUDA tensors R, S: for every kept R
    row i, the min(k, kept S rows) kept S rows of largest cosine similarity in descending similarity
    (ties: the smaller j); rows in ascending i, each row's records consecutive.  Returns views of a
    cached device result buffer (valid until the next call on ctx)."""
    import torch
    lib = load_library()
    rR, rS = _dev_rel(R), _dev_rel(S)
    sR, sS = _dev_sel(selR), _dev_sel(selS)
    cap = max(int(R.shape[0]) * max(int(k), 1), 1)
    if ctx._out is None or ctx._out.shape[0] < cap:
        ctx._out = torch.empty((cap, 3), dtype=torch.int32, device=R.device)
    out = ejoin_pairs(ctypes.c_void_p(ctx._out.data_ptr()), ctx._out.shape[0], None, 0)
    _check(lib.ejoin_topk(ctx.handle, rR, rS, int(k), _sel_ptr(sR), _sel_ptr(sS), ctypes.byref(out)), "ejoin_topk")
    n = int(out.count)
    v = ctx._out[:n]
    return Result(v[:, 0], v[:, 1], v[:, 2].view(torch.float32), n)


def ejoin_top1(ctx: Ctx, R, S, selR: Optional[Sel] = None, selS: Optional[Sel] = None) -> Result:
    """ejoin_topk with k = 1: one record per kept R row."""
    return ejoin_topk(ctx, R, S, 1, selR, selS)


def _host_arr(a, dtype):
    if a is None:
        return None
    if hasattr(a, "numpy"):
        a = a.numpy()
    a = np.asarray(a)
    if a.dtype != dtype:
        raise TypeError(f"expected {dtype} host array, got {a.dtype}")
    return a


def ejoin_threshold_host(ctx: Ctx, R, S, eps: float, selR: Optional[Sel] = None, selS: Optional[Sel] = None,
                         out=None):
    """Host-memory E-join: pinned (device-accessible) inputs are read in place, only the predicate
    columns and the kept rows crossing the link; pageable inputs are copied whole.  The pairs are
    copied back.

    ``out``: optional numpy structured buffer (pinned memory recommended) of dtype PAIR_DTYPE.
    Returns (pairs numpy structured array view, count)."""
    lib = load_library()
    Rh = _host_arr(R, np.float32)
    Sh = _host_arr(S, np.float32)
    if Rh.ndim != 2 or Sh.ndim != 2 or Rh.strides[1] != 4 or Sh.strides[1] != 4:
        raise TypeError("host relations must be 2-D float32 with contiguous rows")
    rR = ejoin_rel(ctypes.c_void_p(Rh.ctypes.data), Rh.shape[0], Rh.shape[1], Rh.strides[0] // 4)
    rS = ejoin_rel(ctypes.c_void_p(Sh.ctypes.data), Sh.shape[0], Sh.shape[1], Sh.strides[0] // 4)
    keep = []

    def hsel(s):
        if s is None:
            return None
        a = _host_arr(s.attr, np.int32)
        b = None if s.bits is None else np.asarray(s.bits).view(np.uint32)
        keep.extend([a, b])
        return ejoin_sel(ctypes.c_void_p(a.ctypes.data if a is not None else 0), OPS[s.op], int(s.c),
                         ctypes.c_void_p(b.ctypes.data if b is not None else 0))

    sR, sS = hsel(selR), hsel(selS)
    if out is None:
        out = np.empty(1 << 16, dtype=PAIR_DTYPE)
    for _ in range(3):
        cnt = ctypes.c_uint64(0)
        st = lib.ejoin_threshold_host(ctx.handle, rR, rS, ctypes.c_float(eps), _sel_ptr(sR), _sel_ptr(sS),
                                      ctypes.c_void_p(out.ctypes.data), len(out), ctypes.byref(cnt))
        if st == EJOIN_EOVERFLOW:
            out = np.empty(int(cnt.value) + 1024, dtype=PAIR_DTYPE)
            continue
        _check(st, "ejoin_threshold_host")
        return out[: int(cnt.value)], int(cnt.value)
    raise EJoinError(EJOIN_EOVERFLOW, "ejoin_threshold_host")


PAIR_DTYPE = np.dtype([("i", np.uint32), ("j", np.uint32), ("sim", np.float32)])


def ejoin_normalize(ctx: Ctx, X, prec="bf16", sel: Optional[Sel] = None):
    """Selection + normalisation of one device relation.  Returns (rows, inv_norm, scale, ids, n_sel)
    where rows is the padded normalised matrix in the precision's storage type."""
    import torch
    lib = load_library()
    p = PRECS[prec] if isinstance(prec, str) else int(prec)
    r = _dev_rel(X)
    n, d = X.shape
    kp = ejoin_padded_dim(p, d)
    dt = {EJOIN_F32: torch.float32, EJOIN_TF32: torch.float32, EJOIN_BF16: torch.bfloat16,
          EJOIN_FP8_E4M3: torch.uint8}[p]
    out = torch.zeros((max(n, 1), kp), dtype=dt, device=X.device)
    inv = torch.zeros(max(n, 1), dtype=torch.float32, device=X.device)
    scale = torch.zeros(max(n, 1), dtype=torch.float32, device=X.device)
    ids = torch.zeros(max(n, 1), dtype=torch.int32, device=X.device)
    n_sel = torch.zeros(1, dtype=torch.int64, device=X.device)
    s = _dev_sel(sel)
    _check(lib.ejoin_normalize(ctx.handle, r, _sel_ptr(s), p, ctypes.c_void_p(out.data_ptr()), kp,
                               ctypes.c_void_p(inv.data_ptr()), ctypes.c_void_p(scale.data_ptr()),
                               ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(n_sel.data_ptr())),
           "ejoin_normalize")
    return out, inv, scale, ids, n_sel


def ejoin_last_stats(ctx: Ctx) -> dict:
    st = ejoin_stats()
    _check(load_library().ejoin_last_stats(ctx.handle, ctypes.byref(st)), "ejoin_last_stats")
    return {name: getattr(st, name) for name, _ in ejoin_stats._fields_}


class Batch:
    """A planned batch of independent E-joins (ejoin_batch_create); runs replay a CUDA graph
    when ``graph`` is set.  ``jobs``: list of (R, S, eps) with R, S float32 CUDA tensors."""

    def __init__(self, ctx: Ctx, jobs, graph: bool = True, autotune: bool = False, sels=None):
        """sels (optional): per job a pair (Sel or None for R, Sel or None for S)."""
        lib = load_library()
        self.ctx = ctx
        self._keep = [(R, S) for R, S, _ in jobs]
        arr = (ejoin_job * len(jobs))()
        for k, (R, S, eps) in enumerate(jobs):
            arr[k].R = _dev_rel(R)
            arr[k].S = _dev_rel(S)
            arr[k].eps = float(eps)
        flags = (EJOIN_BATCH_GRAPH if graph else 0) | (EJOIN_BATCH_AUTOTUNE if autotune else 0)
        h = ctypes.c_void_p()
        if sels is None:
            _check(lib.ejoin_batch_create(ctx.handle, arr, len(jobs), flags, ctypes.byref(h)), "ejoin_batch_create")
        else:
            if len(sels) != len(jobs):
                raise ValueError("one (selR, selS) pair per job")
            sarr = (ejoin_job_sel * len(jobs))()
            none = ejoin_sel(None, 0, 0, None)
            for k, (sR, sS) in enumerate(sels):
                sarr[k].R = _dev_sel(sR) or none
                sarr[k].S = _dev_sel(sS) or none
                self._keep.append((sR, sS))
            _check(lib.ejoin_batch_create_sel(ctx.handle, arr, sarr, len(jobs), flags, ctypes.byref(h)),
                   "ejoin_batch_create_sel")
        self.handle = h
        _live_dependents.add(self)

    def run(self):
        _check(load_library().ejoin_batch_run(self.handle), "ejoin_batch_run")

    def wait(self) -> int:
        cnt = ctypes.c_uint64(0)
        _check(load_library().ejoin_batch_wait(self.handle, ctypes.byref(cnt)), "ejoin_batch_wait")
        return int(cnt.value)

    def result(self, count: int):
        """(job, i, j, sim) as torch tensors viewing the plan's device buffer."""
        import torch
        p = ctypes.c_void_p()
        cap = ctypes.c_uint64(0)
        _check(load_library().ejoin_batch_result(self.handle, ctypes.byref(p), ctypes.byref(cap)),
               "ejoin_batch_result")
        n = min(int(count), int(cap.value))
        dev = f"cuda:{self.ctx.device}"
        if n == 0:
            z = torch.zeros(0, dtype=torch.int32, device=dev)
            return z, z, z, z.view(torch.float32)
        # wrap the device buffer without copying it: 4 x 32-bit words per record
        buf = _DevBuf(p.value, n * 16)
        t = torch.as_tensor(buf, device=dev).view(torch.int32).view(n, 4)
        return t[:, 0], t[:, 1], t[:, 2], t[:, 3].view(torch.float32)

    def info(self) -> dict:
        st = ejoin_batch_stats()
        _check(load_library().ejoin_batch_info(self.handle, ctypes.byref(st)), "ejoin_batch_info")
        return {name: getattr(st, name) for name, _ in ejoin_batch_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load_library().ejoin_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevBuf:
    """Minimal __cuda_array_interface__ over a device buffer owned by the library."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def ejoin_batch(ctx: Ctx, jobs, graph: bool = True, autotune: bool = False, sels=None):
    """One-shot batched join: plan, run, wait; returns (job, i, j, sim) host numpy arrays."""
    b = Batch(ctx, jobs, graph=graph, autotune=autotune, sels=sels)
    b.run()
    n = b.wait()
    job, i, j, sim = (x.cpu().numpy() for x in b.result(n))
    b.close()
    return job, i, j, sim


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def ejoin_row_inv_norm(ctx: Ctx, X):
    import torch
    inv = torch.empty(max(X.shape[0], 1), dtype=torch.float32, device=X.device)
    _check(load_library().ejoin_row_inv_norm(ctx.handle, _dev_rel(X), _ptr(inv)), "ejoin_row_inv_norm")
    return inv[: X.shape[0]]


def ejoin_score_pairs(ctx: Ctx, R, S, i, j):
    """Exact FP32 cosine of pairs (R[i[k]], S[j[k]]) (int32 CUDA index tensors)."""
    import torch
    out = torch.empty(max(len(i), 1), dtype=torch.float32, device=R.device)
    _check(load_library().ejoin_score_pairs(ctx.handle, _dev_rel(R), _dev_rel(S), _ptr(i), _ptr(j), len(i),
                                            _ptr(out)), "ejoin_score_pairs")
    return out[: len(i)]


class Sketch:
    """The learned sketch network (ejoin_sketch_*): d -> hidden -> 64, GELU, unit output."""

    def __init__(self, ctx: Ctx, d: int, hidden: int = 256, out: int = 64):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.ejoin_sketch_create(ctx.handle, d, hidden, out, ctypes.byref(h)), "ejoin_sketch_create")
        self.handle, self.ctx, self.d, self.hidden, self.out = h, ctx, d, hidden, out
        self.n_params = int(lib.ejoin_sketch_num_params(h))
        _live_dependents.add(self)

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {flat.size}")
        _check(load_library().ejoin_sketch_set_params(self.handle, flat.ctypes.data), "ejoin_sketch_set_params")

    def get_params(self) -> np.ndarray:
        flat = np.empty(self.n_params, dtype=np.float32)
        _check(load_library().ejoin_sketch_get_params(self.handle, flat.ctypes.data), "ejoin_sketch_get_params")
        return flat

    def unflatten(self, flat):
        d, h, o = self.d, self.hidden, self.out
        a = 0
        W1 = flat[a:a + h * d].reshape(h, d); a += h * d
        b1 = flat[a:a + h]; a += h
        W2 = flat[a:a + o * h].reshape(o, h); a += o * h
        b2 = flat[a:a + o]
        return {"W1": W1, "b1": b1, "W2": W2, "b2": b2}

    @staticmethod
    def flatten(p):
        return np.concatenate([p["W1"].ravel(), p["b1"].ravel(), p["W2"].ravel(), p["b2"].ravel()]).astype(np.float32)

    def forward(self, X):
        import torch
        S = torch.empty((max(X.shape[0], 1), self.out), dtype=torch.float32, device=X.device)
        _check(load_library().ejoin_sketch_forward(self.handle, _dev_rel(X), _ptr(S)), "ejoin_sketch_forward")
        return S[: X.shape[0]]

    def forward_tc(self, X):
        """Sketches on the tensor cores (TF32 layers), as the pruned join computes them."""
        import torch
        S = torch.empty((max(X.shape[0], 1), self.out), dtype=torch.float32, device=X.device)
        _check(load_library().ejoin_sketch_forward_tc(self.handle, _dev_rel(X), _ptr(S)), "ejoin_sketch_forward_tc")
        return S[: X.shape[0]]

    def grad(self, X, inv, p, q, t, w):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = ctypes.c_float(0)
        _check(load_library().ejoin_sketch_grad(self.handle, _dev_rel(X), _ptr(inv), _ptr(p), _ptr(q), _ptr(t),
                                                _ptr(w), len(p), _ptr(g), ctypes.byref(loss)), "ejoin_sketch_grad")
        return g, float(loss.value)

    def train_step(self, X, inv, p, q, t, w, lr: float, want_loss: bool = False):
        loss = ctypes.c_float(0)
        _check(load_library().ejoin_sketch_train_step(self.handle, _dev_rel(X), _ptr(inv), _ptr(p), _ptr(q), _ptr(t),
                                                      _ptr(w), len(p), ctypes.c_float(lr),
                                                      ctypes.byref(loss) if want_loss else None),
               "ejoin_sketch_train_step")
        return float(loss.value) if want_loss else None

    def pair_sims(self, X, inv, p, q):
        import torch
        out = torch.empty(max(len(p), 1), dtype=torch.float32, device=X.device)
        _check(load_library().ejoin_sketch_pair_sims(self.handle, _dev_rel(X), _ptr(inv), _ptr(p), _ptr(q), len(p),
                                                     _ptr(out)), "ejoin_sketch_pair_sims")
        return out[: len(p)]

    def close(self):
        if getattr(self, "handle", None):
            load_library().ejoin_sketch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ejoin_sketch_train(sk: Sketch, X_train, X_cal, eps: float, label_margin: float = 0.2, w_join: float = 8.0,
                       n_pairs: int = 10_000_000, epochs: int = 3, batch: int = 65536, lr: float = 2e-3,
                       recall: float = 0.999, cal_margin: float = 0.01, seed: int = 0, init: bool = True):
    """Train the sketch network in the library (labelled set from the exact join of X_train, seeded epochs,
    calibration on X_cal) and return (eps_sketch, report dict)."""
    cfg = ejoin_sketch_train_cfg(float(eps), float(label_margin), float(w_join), int(n_pairs), int(epochs),
                                 int(batch), float(lr), float(recall), float(cal_margin), int(seed), int(bool(init)))
    eps_sk = ctypes.c_float(0)
    rep = ejoin_sketch_train_report()
    _check(load_library().ejoin_sketch_train(sk.handle, _dev_rel(X_train), _dev_rel(X_cal), ctypes.byref(cfg),
                                             ctypes.byref(eps_sk), ctypes.byref(rep)), "ejoin_sketch_train")
    return float(eps_sk.value), {name: getattr(rep, name) for name, _ in ejoin_sketch_train_report._fields_}


def ejoin_threshold_pruned(ctx: Ctx, sk: Sketch, R, S, eps: float, eps_sketch: float, capacity=None,
                           recall_est: bool = False):
    """Pruned device join; returns (Result, stats dict).  recall_est: also estimate the recall against the
    plain join on sampled rows (stats["recall_est"])."""
    import torch
    lib = load_library()
    rR, rS = _dev_rel(R), _dev_rel(S)
    cap = capacity or (ctx._out.shape[0] if ctx._out is not None else 1 << 16)
    for _ in range(3):
        if ctx._out is None or ctx._out.shape[0] < cap:
            ctx._out = torch.empty((cap, 3), dtype=torch.int32, device=R.device)
        out = ejoin_pairs(ctypes.c_void_p(ctx._out.data_ptr()), ctx._out.shape[0], None, 0)
        st = ejoin_prune_stats()
        rec = ctypes.c_float(0)
        status = lib.ejoin_threshold_pruned(ctx.handle, sk.handle, rR, rS, ctypes.c_float(eps),
                                            ctypes.c_float(eps_sketch), ctypes.byref(out), ctypes.byref(st),
                                            ctypes.byref(rec) if recall_est else None)
        if status == EJOIN_EOVERFLOW:
            cap = int(out.count) + 1024
            continue
        _check(status, "ejoin_threshold_pruned")
        n = int(out.count)
        v = ctx._out[:n]
        stats = {name: getattr(st, name) for name, _ in ejoin_prune_stats._fields_}
        return Result(v[:, 0], v[:, 1], v[:, 2].view(torch.float32), n), stats
    raise EJoinError(EJOIN_EOVERFLOW, "ejoin_threshold_pruned")
