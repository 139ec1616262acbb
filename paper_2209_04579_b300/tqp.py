"""Python binding of the TQP C ABI (``include/tqp.h``).

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step of every operator runs in the library's CUDA
kernels.  Importing this module loads ``libtqp.so`` and raises if it is
missing -- there is no fallback implementation.

Each function has the name of the C entry point it calls.  Device counts
(result sizes) are returned as 1-element int64 CUDA tensors so that calls can
be chained without a host synchronisation; ``.item()`` reads them.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libtqp.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libtqp.so not built ({_LIB_PATH}); run python -m paper_2209_04579_b300.build")
_lib = ctypes.CDLL(_LIB_PATH)

# ------------------------------------------------------------------ constants
OK, ERR_INVALID, ERR_DTYPE, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_WORKSPACE, ERR_UNSUPPORTED, ERR_TOO_LARGE = range(9)
NOALLOC_MAX_ROWS = 1 << 28
I8, I16, I32, I64 = 1, 2, 3, 4
LT, LE, GT, GE, EQ, NE = range(6)
COUNT, SUM, MIN, MAX = range(4)

_DTYPE = {torch.int8: I8, torch.int16: I16, torch.int32: I32, torch.int64: I64}
_TORCH = {v: k for k, v in _DTYPE.items()}


class Col(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class Pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("op", ctypes.c_int32), ("lit", ctypes.c_int64)]


class Term(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("pad_", ctypes.c_int32), ("mul", ctypes.c_int64),
                ("add", ctypes.c_int64)]


class Expr(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int32), ("pad_", ctypes.c_int32), ("term", Term * 3)]


class Agg(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("expr", ctypes.c_int32)]


class Dim(ctypes.Structure):
    _fields_ = [("key", Col), ("n", ctypes.c_int64), ("group", Col), ("preds", ctypes.POINTER(Pred)),
                ("npred", ctypes.c_int), ("ncols", ctypes.c_int), ("cols", ctypes.POINTER(Col))]


class ValRef(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int32), ("col", ctypes.c_int32)]


H = 64  # TQP_CDF_HIDDEN


class CdfModel(ctypes.Structure):
    _fields_ = [("w", ctypes.c_float * H), ("b", ctypes.c_float * H), ("a", ctypes.c_float * H),
                ("c", ctypes.c_float), ("shift", ctypes.c_int32), ("inv", ctypes.c_float), ("pad_", ctypes.c_int32),
                ("umin", ctypes.c_uint64)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("pad_", ctypes.c_int32)]


class LearnedCfg(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_int32), ("buckets", ctypes.c_int32), ("train", ctypes.c_int32),
                ("heavy", ctypes.c_int32), ("train_cfg", TrainCfg), ("init", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class LearnedStats(ctypes.Structure):
    _fields_ = [("buckets", ctypes.c_int64), ("heavy_keys", ctypes.c_int64), ("light_rows", ctypes.c_int64),
                ("max_bucket", ctypes.c_int64), ("over_capacity", ctypes.c_int64), ("nonempty", ctypes.c_int64),
                ("over_capacity_rows", ctypes.c_int64), ("small_rows", ctypes.c_int64),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float)]


BATCH_MAX_COLS = 4


class BatchShape(ctypes.Structure):
    _fields_ = [("nfact_cols", ctypes.c_int32), ("fact_dtype", ctypes.c_int32 * BATCH_MAX_COLS),
                ("fk_col", ctypes.c_int32), ("key_dtype", ctypes.c_int32), ("group_dtype", ctypes.c_int32),
                ("npred", ctypes.c_int32), ("preds", Pred * 4), ("nexprs", ctypes.c_int32), ("exprs", Expr * 8),
                ("naggs", ctypes.c_int32), ("aggs", Agg * 8)]


class Problem(ctypes.Structure):
    _fields_ = [("n_fact", ctypes.c_int64), ("fact_cols", ctypes.c_void_p * BATCH_MAX_COLS),
                ("n_dim", ctypes.c_int64), ("dim_key", ctypes.c_void_p), ("dim_group", ctypes.c_void_p),
                ("out_keys", ctypes.c_void_p), ("out_aggs", ctypes.c_void_p), ("cap", ctypes.c_int64),
                ("d_out_groups", ctypes.c_void_p)]


class BatchCfg(ctypes.Structure):
    _fields_ = [("probe_items", ctypes.c_int32), ("pad_", ctypes.c_int32)]


_vp, _i64, _sz, _int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
_P = ctypes.POINTER

_lib.tqp_filter.argtypes = [_P(Col), _int, _P(Pred), _int, _i64, _vp, _vp, _i64, _vp, _vp, _P(_sz), _vp]
_lib.tqp_gather.argtypes = [Col, _vp, _i64, _vp, _vp, _vp]
_lib.tqp_like_prefix.argtypes = [_vp, _i64, ctypes.c_int32, ctypes.c_char_p, ctypes.c_int32, _vp, _vp]
_lib.tqp_date_parse_iso.argtypes = [_vp, _i64, ctypes.c_int32, _vp, _vp]
_lib.tqp_date_from_days.argtypes = [_vp, _i64, _vp, _vp]
_lib.tqp_date_parts.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp]
_lib.tqp_string_codes.argtypes = [_vp, _i64, ctypes.c_int32, _vp, _vp, _vp, _vp, _P(_sz), _vp]
_lib.tqp_sort_pairs.argtypes = [ctypes.c_int32, _vp, _vp, _vp, _vp, _i64, _vp, _int, _int, _vp, _P(_sz), _vp]
_lib.tqp_join_eq.argtypes = [Col, _i64, _vp, Col, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _P(_sz), _vp]
_lib.tqp_groupby_agg.argtypes = [_P(Col), _int, _P(Col), _int, _P(Expr), _int, _P(Agg), _int, _vp, _i64, _vp,
                                 _P(_vp), _vp, _i64, _vp, _vp, _P(_sz), _vp]
_lib.tqp_star_agg.argtypes = [_P(Col), _int, _i64, _P(Pred), _int, _P(_int), _P(Dim), _int, _P(ValRef), _int,
                              _P(Expr), _int, _P(Agg), _int, _P(_vp), _vp, _i64, _vp, _vp, _P(_sz), _vp]
_lib.tqp_star_agg_learned.argtypes = _lib.tqp_star_agg.argtypes[:-3] + [_P(LearnedCfg), _vp, _P(_sz), _vp]
_lib.tqp_cdf_forward.argtypes = [_vp, _vp, _i64, _vp, _vp, _int, _vp]
_lib.tqp_cdf_backward.argtypes = [_vp, _vp, _vp, _i64, _vp, _vp, _P(_sz), _vp]
_lib.tqp_cdf_train.argtypes = [_vp, _vp, _i64, _vp, _P(TrainCfg), _vp, _vp, _P(_sz), _vp]
_lib.tqp_groupby_agg_learned.argtypes = [_P(Col), _int, _P(Col), _int, _P(Expr), _int, _P(Agg), _int, _vp, _i64,
                                         _vp, _P(_vp), _vp, _i64, _vp, _P(LearnedCfg), _vp, _vp, _vp, _P(_sz), _vp]
_lib.tqp_partition_learned.argtypes = [_P(Col), _int, _vp, _i64, _vp, _P(LearnedCfg), _vp, _vp, _vp, _vp, _vp, _vp,
                                       _vp, _vp, _P(_sz), _vp]
_lib.tqp_star_agg_batched.argtypes = [_P(BatchShape), _P(Problem), _int, _P(BatchCfg), _vp, _P(_sz), _vp]
_lib.tqp_filter_noalloc.argtypes = [_P(Col), _int, _P(Pred), _int, _i64, _vp, _vp, _i64, _vp, _vp]
_lib.tqp_filter_noalloc.restype = ctypes.c_int
_lib.tqp_status_poll.argtypes = [_vp]
_lib.tqp_sort_tiles.argtypes = [_int, _int]
_lib.tqp_sort_tiles.restype = ctypes.c_int
_lib.tqp_debug_set_spin_limit.argtypes = [_i64]
_lib.tqp_debug_inject_unpublished_tile.argtypes = [_i64]
_lib.tqp_status_string.restype = ctypes.c_char_p
_lib.tqp_debug_launch_count.restype = ctypes.c_int64
_lib.tqp_debug_launch_count.argtypes = []
_lib.tqp_profile_events.argtypes = [_int, _vp, _vp]
for _f in ("tqp_filter", "tqp_gather", "tqp_like_prefix", "tqp_string_codes", "tqp_date_parse_iso",
           "tqp_date_from_days", "tqp_date_parts", "tqp_sort_pairs", "tqp_join_eq", "tqp_groupby_agg", "tqp_star_agg",
           "tqp_star_agg_learned",
           "tqp_status_poll", "tqp_profile_events", "tqp_cdf_forward", "tqp_cdf_backward", "tqp_cdf_train",
           "tqp_groupby_agg_learned", "tqp_partition_learned", "tqp_star_agg_batched", "tqp_debug_set_spin_limit", "tqp_debug_inject_unpublished_tile"):
    getattr(_lib, _f).restype = ctypes.c_int


class TQPError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_lib.tqp_status_string(status).decode()} (status {status})")
        self.status = status


def _check(st: int, where: str):
    if st != OK:
        raise TQPError(st, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _col(t):
    if t.dtype not in _DTYPE:
        raise TypeError(f"unsupported column dtype {t.dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("columns must be contiguous CUDA tensors")
    return Col(t.data_ptr(), _DTYPE[t.dtype], 0)


def _cols(ts):
    arr = (Col * max(1, len(ts)))()
    for i, t in enumerate(ts):
        arr[i] = _col(t)
    return arr


def _preds(preds):
    arr = (Pred * max(1, len(preds)))()
    for i, (c, op, lit) in enumerate(preds):
        arr[i] = Pred(c, op, lit)
    return arr


def _exprs(exprs):
    arr = (Expr * max(1, len(exprs)))()
    for i, e in enumerate(exprs):
        arr[i].nterms = len(e)
        for t, (c, m, a) in enumerate(e):
            arr[i].term[t] = Term(c, 0, m, a)
    return arr


def _aggs(aggs):
    arr = (Agg * max(1, len(aggs)))()
    for i, (op, e) in enumerate(aggs):
        arr[i] = Agg(op, e)
    return arr


class Workspace:
    """Grow-only device scratch buffer for one (device, stream) pair."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        return self.buf


_WS: dict = {}


def _workspace(nbytes: int, device, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    key = (str(device), s.cuda_stream)
    ws = _WS.setdefault(key, Workspace())
    return ws.get(nbytes, device)


def _two_phase(fn, name, args_before_ws, device, stream):
    need = ctypes.c_size_t(0)
    _check(fn(*args_before_ws, None, ctypes.byref(need), _stream(stream)), name + " (size query)")
    ws = _workspace(need.value, device, stream)
    have = ctypes.c_size_t(ws.numel())
    _check(fn(*args_before_ws, _ptr(ws), ctypes.byref(have), _stream(stream)), name)


# ------------------------------------------------------------------ operators

def tqp_filter(cols, preds, n=None, d_n=None, out=None, cap=None, stream=None):
    """Ascending int32 row ids where every predicate (col, op, literal) holds,
    and their count as a device int64[1]."""
    dev = cols[0].device
    n = cols[0].numel() if n is None else n
    cap = n if cap is None else cap
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if out is None else out
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    c, p = _cols(cols), _preds(preds)
    _two_phase(_lib.tqp_filter, "tqp_filter",
               [c, len(cols), p, len(preds), n, _ptr(d_n), _ptr(out), cap, _ptr(cnt)], dev, stream)
    return out, cnt


def tqp_filter_noalloc(cols, preds, n=None, d_n=None, out=None, cap=None, stream=None):
    """tqp_filter for callers that cannot provide a workspace: the library's
    fixed scratch array is used instead (n <= NOALLOC_MAX_ROWS; calls must
    not overlap on the GPU).  The caller passes the outputs (allocated here
    when not given)."""
    dev = cols[0].device
    n = cols[0].numel() if n is None else n
    cap = n if cap is None else cap
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev) if out is None else out
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    _check(_lib.tqp_filter_noalloc(_cols(cols), len(cols), _preds(preds), len(preds), n, _ptr(d_n), _ptr(out), cap,
                                   _ptr(cnt), _stream(stream)), "tqp_filter_noalloc")
    return out, cnt


def tqp_gather(col, idx, n=None, d_n=None, out=None, stream=None):
    n = idx.numel() if n is None else n
    out = torch.empty(max(n, 1), dtype=col.dtype, device=col.device) if out is None else out
    _check(_lib.tqp_gather(_col(col), _ptr(idx), n, _ptr(d_n), _ptr(out), _stream(stream)), "tqp_gather")
    return out


def tqp_like_prefix(strings, prefix: bytes, out=None, stream=None):
    """strings: (n, width) uint8 device tensor of zero-padded UTF-8 rows;
    returns int8 [n], 1 where the value starts with prefix (LIKE 'prefix%')."""
    n, width = strings.shape
    if strings.dtype != torch.uint8 or not strings.is_contiguous():
        raise ValueError("tqp_like_prefix: a contiguous (n, width) uint8 tensor")
    out = torch.empty(max(n, 1), dtype=torch.int8, device=strings.device) if out is None else out
    _check(_lib.tqp_like_prefix(_ptr(strings), n, width, bytes(prefix), len(prefix), _ptr(out), _stream(stream)),
           "tqp_like_prefix")
    return out[:n]


def tqp_date_parse_iso(strings, stream=None):
    """(n, width) uint8 zero-padded 'YYYY-MM-DD' rows -> int64 epoch ns [n]
    (INT64_MIN, and TQP_ERR_INVALID in the device status, for a bad row)."""
    n, width = strings.shape
    if strings.dtype != torch.uint8 or not strings.is_contiguous():
        raise ValueError("tqp_date_parse_iso: a contiguous (n, width) uint8 tensor")
    out = torch.empty(max(n, 1), dtype=torch.int64, device=strings.device)
    _check(_lib.tqp_date_parse_iso(_ptr(strings), n, width, _ptr(out), _stream(stream)), "tqp_date_parse_iso")
    return out[:n]


def tqp_date_from_days(days, stream=None):
    """int32 days since 1970-01-01 -> int64 epoch ns."""
    n = days.numel()
    out = torch.empty(max(n, 1), dtype=torch.int64, device=days.device)
    _check(_lib.tqp_date_from_days(_ptr(days), n, _ptr(out), _stream(stream)), "tqp_date_from_days")
    return out[:n]


def tqp_date_parts(ns, stream=None):
    """int64 epoch ns -> (day number, year, month, day of month), int32 each."""
    n = ns.numel()
    out = [torch.empty(max(n, 1), dtype=torch.int32, device=ns.device) for _ in range(4)]
    _check(_lib.tqp_date_parts(_ptr(ns), n, *[_ptr(o) for o in out], _stream(stream)), "tqp_date_parts")
    return tuple(o[:n] for o in out)


def tqp_string_codes(strings, stream=None):
    """Dictionary codes of a (n, width) uint8 string tensor: (codes int32 [n],
    representative row per code int32 [n], device int64 number of codes)."""
    n, width = strings.shape
    if strings.dtype != torch.uint8 or not strings.is_contiguous():
        raise ValueError("tqp_string_codes: a contiguous (n, width) uint8 tensor")
    dev = strings.device
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    rep = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    _two_phase(_lib.tqp_string_codes, "tqp_string_codes", [_ptr(strings), n, width, _ptr(codes), _ptr(rep), _ptr(k)],
               dev, stream)
    return codes[:n], rep[:n], k


def tqp_sort_pairs(keys, vals=None, begin_bit=0, end_bit=None, n=None, d_n=None, stream=None):
    """Stable sort of (key, value); value None -> payload = input row index."""
    dev = keys.device
    n = keys.numel() if n is None else n
    end_bit = keys.element_size() * 8 if end_bit is None else end_bit
    ko = torch.empty(max(n, 1), dtype=keys.dtype, device=dev)
    vo = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    _two_phase(_lib.tqp_sort_pairs, "tqp_sort_pairs",
               [_DTYPE[keys.dtype], _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, _ptr(d_n), begin_bit, end_bit],
               dev, stream)
    return ko[:n], vo[:n]


def tqp_join_eq(probe, build, cap, n_probe=None, d_n_probe=None, n_build=None, d_n_build=None, stream=None):
    """Pairs (probe_row, build_row) with equal keys, by (probe_row, build_row);
    returns (out_probe, out_build, device count)."""
    dev = probe.device
    n_probe = probe.numel() if n_probe is None else n_probe
    n_build = build.numel() if n_build is None else n_build
    op = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    ob = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    _two_phase(_lib.tqp_join_eq, "tqp_join_eq",
               [_col(probe), n_probe, _ptr(d_n_probe), _col(build), n_build, _ptr(d_n_build), _ptr(op), _ptr(ob),
                cap, _ptr(cnt)], dev, stream)
    return op, ob, cnt


def tqp_groupby_agg(keys, vals, exprs, aggs, cap, sel=None, n=None, d_n=None, stream=None):
    """Group-by aggregate.  exprs: lists of (val_col, mul, add) terms;
    aggs: (op, expr).  Returns (key columns, aggs int64 [cap, naggs], device G)."""
    dev = keys[0].device
    if n is None:
        n = sel.numel() if sel is not None else keys[0].numel()
    out_keys = [torch.empty(max(cap, 1), dtype=k.dtype, device=dev) for k in keys]
    out_aggs = torch.empty((max(cap, 1), len(aggs)), dtype=torch.int64, device=dev)
    G = torch.empty(1, dtype=torch.int64, device=dev)
    kp = (ctypes.c_void_p * len(keys))(*[k.data_ptr() for k in out_keys])
    _two_phase(_lib.tqp_groupby_agg, "tqp_groupby_agg",
               [_cols(keys), len(keys), _cols(vals), len(vals), _exprs(exprs), len(exprs), _aggs(aggs), len(aggs),
                _ptr(sel), n, _ptr(d_n), kp, _ptr(out_aggs), cap, _ptr(G)], dev, stream)
    return out_keys, out_aggs, G


class DimSpec:
    """One dimension of tqp_star_agg: key column, optional group column,
    predicates over `cols`, and the columns values may reference."""

    def __init__(self, key, cols=(), preds=(), group=None):
        self.key, self.cols, self.preds, self.group = key, list(cols), list(preds), group


def tqp_star_agg(fact_cols, fact_preds, fk_cols, dims, vals, exprs, aggs, cap, stream=None, learned=None):
    """Fused star join + filter + group-by.  vals: (src, col) with src 0 =
    fact column, 1 + d = column of dimension d.  learned: a learned_cfg to
    sort large dimensions' keys through the learned range partitioner
    (tqp_star_agg_learned).  Returns (key columns, aggs, device G)."""
    dev = fact_cols[0].device
    keep = []
    darr = (Dim * len(dims))()
    nkeys = 0
    for d, D in enumerate(dims):
        cols = _cols(D.cols)
        preds = _preds(D.preds)
        keep += [cols, preds]
        darr[d].key = _col(D.key)
        darr[d].n = D.key.numel()
        darr[d].group = _col(D.group) if D.group is not None else Col(None, 0, 0)
        darr[d].preds = ctypes.cast(preds, _P(Pred))
        darr[d].npred = len(D.preds)
        darr[d].ncols = len(D.cols)
        darr[d].cols = ctypes.cast(cols, _P(Col))
        nkeys += D.group is not None
    out_keys = [torch.empty(max(cap, 1), dtype=D.group.dtype, device=dev) for D in dims if D.group is not None]
    out_aggs = torch.empty((max(cap, 1), len(aggs)), dtype=torch.int64, device=dev)
    G = torch.empty(1, dtype=torch.int64, device=dev)
    kp = (ctypes.c_void_p * max(1, nkeys))(*[k.data_ptr() for k in out_keys])
    fk = (ctypes.c_int * len(fk_cols))(*fk_cols)
    vr = (ValRef * max(1, len(vals)))(*[ValRef(s, c) for s, c in vals])
    args = [_cols(fact_cols), len(fact_cols), fact_cols[0].numel(), _preds(fact_preds), len(fact_preds), fk, darr,
            len(dims), vr, len(vals), _exprs(exprs), len(exprs), _aggs(aggs), len(aggs), kp, _ptr(out_aggs), cap,
            _ptr(G)]
    if learned is None:
        _two_phase(_lib.tqp_star_agg, "tqp_star_agg", args, dev, stream)
    else:
        keep.append(learned)
        _two_phase(_lib.tqp_star_agg_learned, "tqp_star_agg_learned", args + [learned], dev, stream)
    return out_keys, out_aggs, G


# ------------------------------------------------------------------ learned partitioner

def model_to_device(w, b, a, c, shift=0, inv=1.0, umin=0, device="cuda"):
    m = CdfModel()
    for i in range(H):
        m.w[i], m.b[i], m.a[i] = float(w[i]), float(b[i]), float(a[i])
    m.c, m.shift, m.inv, m.umin = float(c), int(shift), float(inv), int(umin)
    return torch.frombuffer(bytearray(bytes(m)), dtype=torch.uint8).to(device)


def model_from_device(t):
    m = CdfModel.from_buffer_copy(t.cpu().numpy().tobytes())
    return {"w": list(m.w), "b": list(m.b), "a": list(m.a), "c": m.c, "shift": m.shift, "inv": m.inv, "umin": m.umin}


def empty_model(device="cuda"):
    return torch.zeros(ctypes.sizeof(CdfModel), dtype=torch.uint8, device=device)


def tqp_cdf_forward(model, x, B=0, want_F=True, stream=None):
    """(F, buckets of B or None); want_F=False (with B) writes the buckets alone and returns F None."""
    n = x.numel()
    F = torch.empty(max(n, 1), dtype=torch.float32, device=x.device) if want_F or not B else None
    bk = torch.empty(max(n, 1), dtype=torch.int32, device=x.device) if B else None
    _check(_lib.tqp_cdf_forward(_ptr(model), _ptr(x), n, _ptr(F), _ptr(bk), B, _stream(stream)), "tqp_cdf_forward")
    return (F[:n] if F is not None else None), (bk[:n] if B else None)


def tqp_cdf_backward(model, x, y, stream=None):
    """[dL/dw (H), dL/db (H), dL/da (H), dL/dc, L] as a float32 device tensor."""
    g = torch.empty(3 * H + 2, dtype=torch.float32, device=x.device)
    _two_phase(_lib.tqp_cdf_backward, "tqp_cdf_backward", [_ptr(model), _ptr(x), _ptr(y), x.numel(), _ptr(g)],
               x.device, stream)
    return g


def train_cfg(epochs=200, lr=5e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    return TrainCfg(epochs, lr, beta1, beta2, eps, 0)


def tqp_cdf_train(x, y, model, cfg=None, stream=None):
    """Trains `model` (device bytes) in place; returns the per-step loss."""
    cfg = cfg or train_cfg()
    loss = torch.empty(max(cfg.epochs, 1), dtype=torch.float32, device=x.device)
    _two_phase(_lib.tqp_cdf_train, "tqp_cdf_train",
               [_ptr(x), _ptr(y), x.numel(), _ptr(model), ctypes.byref(cfg), _ptr(loss)], x.device, stream)
    return loss[:cfg.epochs]


def learned_cfg(sample=65536, buckets=0, train=True, heavy=True, tcfg=None, init=None):
    """init: 0 = identity CDF, 1 = sample-quantile knots (default: 1 when training).
    The default training refines the knots with small Adam steps (100 epochs,
    lr 1e-4): larger steps disturb a fit that starts close."""
    init = (1 if train else 0) if init is None else init
    if tcfg is None:
        tcfg = train_cfg(epochs=100, lr=1e-4) if init == 1 else train_cfg()
    return LearnedCfg(sample, buckets, int(train), int(heavy), tcfg, int(init), 0)


def tqp_groupby_agg_learned(keys, vals, exprs, aggs, cap, cfg=None, sel=None, n=None, d_n=None, stream=None):
    """The group-by of tqp_groupby_agg through the learned range partitioner.
    Returns (key columns, aggs [cap, naggs], device G, trained model bytes, stats bytes)."""
    dev = keys[0].device
    cfg = cfg or learned_cfg()
    if n is None:
        n = sel.numel() if sel is not None else keys[0].numel()
    out_keys = [torch.empty(max(cap, 1), dtype=k.dtype, device=dev) for k in keys]
    out_aggs = torch.empty((max(cap, 1), len(aggs)), dtype=torch.int64, device=dev)
    G = torch.empty(1, dtype=torch.int64, device=dev)
    model = empty_model(dev)
    stats = torch.zeros(ctypes.sizeof(LearnedStats), dtype=torch.uint8, device=dev)
    kp = (ctypes.c_void_p * len(keys))(*[k.data_ptr() for k in out_keys])
    _two_phase(_lib.tqp_groupby_agg_learned, "tqp_groupby_agg_learned",
               [_cols(keys), len(keys), _cols(vals), len(vals), _exprs(exprs), len(exprs), _aggs(aggs), len(aggs),
                _ptr(sel), n, _ptr(d_n), kp, _ptr(out_aggs), cap, _ptr(G), ctypes.byref(cfg), _ptr(model),
                _ptr(stats)], dev, stream)
    return out_keys, out_aggs, G, model, stats


MAX_HEAVY = 1024  # TQP_MAX_HEAVY


def tqp_partition_learned(keys, cfg=None, sel=None, n=None, d_n=None, stream=None):
    """The learned range partition alone.  Returns a dict: bucket (int32 [n],
    light buckets 0..B-1, heavy key h -> B + h), rows (int32 [n], grouped by
    bucket id, input order within a bucket), offsets (int64 [B + MAX_HEAVY +
    1]), train_x / train_y (float32 [sample]), model (device bytes), stats
    (device bytes)."""
    dev = keys[0].device
    cfg = cfg or learned_cfg()
    if n is None:
        n = sel.numel() if sel is not None else keys[0].numel()
    B = cfg.buckets
    if B == 0:
        B = 256
        while B < (1 << 17) and B * 512 < n:
            B <<= 1
    out = {"bucket": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
           "rows": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
           "offsets": torch.empty(B + MAX_HEAVY + 1, dtype=torch.int64, device=dev),
           "train_x": torch.empty(cfg.sample, dtype=torch.float32, device=dev),
           "train_y": torch.empty(cfg.sample, dtype=torch.float32, device=dev),
           "model": empty_model(dev),
           "stats": torch.zeros(ctypes.sizeof(LearnedStats), dtype=torch.uint8, device=dev), "B": B}
    _two_phase(_lib.tqp_partition_learned, "tqp_partition_learned",
               [_cols(keys), len(keys), _ptr(sel), n, _ptr(d_n), ctypes.byref(cfg), _ptr(out["bucket"]),
                _ptr(out["rows"]), _ptr(out["offsets"]), _ptr(out["train_x"]), _ptr(out["train_y"]),
                _ptr(out["model"]), _ptr(out["stats"])], dev, stream)
    return out


def tqp_sort_tiles(items32=0, items64=0):
    """Rows per thread of the radix sort's tiles (0: unchanged)."""
    _check(_lib.tqp_sort_tiles(items32, items64), "tqp_sort_tiles")


def stats_from_device(t):
    st = LearnedStats.from_buffer_copy(t.cpu().numpy().tobytes())
    return {f: getattr(st, f) for f, _ in LearnedStats._fields_}


# ------------------------------------------------------------------ batched instances

def batch_shape(fact_dtypes, fk_col, group_dtype, preds, exprs, aggs, key_dtype=torch.int32):
    sh = BatchShape()
    sh.nfact_cols = len(fact_dtypes)
    for i, d in enumerate(fact_dtypes):
        sh.fact_dtype[i] = _DTYPE[d]
    sh.fk_col, sh.key_dtype, sh.group_dtype = fk_col, _DTYPE[key_dtype], _DTYPE[group_dtype]
    sh.npred = len(preds)
    for i, (c, op, lit) in enumerate(preds):
        sh.preds[i] = Pred(c, op, lit)
    sh.nexprs = len(exprs)
    for i, e in enumerate(exprs):
        sh.exprs[i].nterms = len(e)
        for t, (c, m, a) in enumerate(e):
            sh.exprs[i].term[t] = Term(c, 0, m, a)
    sh.naggs = len(aggs)
    for i, (op, e) in enumerate(aggs):
        sh.aggs[i] = Agg(op, e)
    return sh


def tqp_star_agg_batched(shape, problems, cap=64, probe_items=8, stream=None):
    """problems: list of (fact_cols list, dim_key, dim_group).  Returns one
    (group keys, aggs [cap, naggs], device G) per problem."""
    dev = problems[0][1].device
    arr = (Problem * len(problems))()
    outs = []
    for i, (fact, key, grp) in enumerate(problems):
        ok = torch.empty(max(cap, 1), dtype=grp.dtype, device=dev)
        oa = torch.empty((max(cap, 1), shape.naggs), dtype=torch.int64, device=dev)
        G = torch.empty(1, dtype=torch.int64, device=dev)
        outs.append((ok, oa, G))
        arr[i].n_fact = fact[0].numel()
        for c, t in enumerate(fact):
            arr[i].fact_cols[c] = t.data_ptr() if t.numel() else None
        arr[i].n_dim = key.numel()
        arr[i].dim_key = key.data_ptr() if key.numel() else None
        arr[i].dim_group = grp.data_ptr() if grp.numel() else None
        arr[i].out_keys, arr[i].out_aggs, arr[i].cap, arr[i].d_out_groups = ok.data_ptr(), oa.data_ptr(), cap, \
            G.data_ptr()
    cfg = BatchCfg(probe_items, 0)
    _two_phase(_lib.tqp_star_agg_batched, "tqp_star_agg_batched",
               [ctypes.byref(shape), arr, len(problems), ctypes.byref(cfg)], dev, stream)
    return outs


def tqp_status_poll(stream=None) -> int:
    return _lib.tqp_status_poll(_stream(stream))


def tqp_debug_set_spin_limit(rounds: int):
    _check(_lib.tqp_debug_set_spin_limit(rounds), "tqp_debug_set_spin_limit")


def tqp_debug_inject_unpublished_tile(tile: int):
    _check(_lib.tqp_debug_inject_unpublished_tile(tile), "tqp_debug_inject_unpublished_tile")


PROF_STAR_PROBE, PROF_SORT_PASSES, PROF_FILTER, PROF_GROUPBY_REDUCE, PROF_JOIN_PROBE = 1, 2, 3, 4, 5
PROF_BATCH_PROBE, PROF_BUCKET_SORT, PROF_PARTITION_SCATTER = 6, 7, 8


def tqp_debug_launch_count() -> int:
    return int(_lib.tqp_debug_launch_count())


def tqp_profile_events(kernel_class: int, start=None, stop=None):
    """Record torch.cuda.Event `start` / `stop` around kernels of one class
    (each event must have been recorded once, which creates it)."""
    for e in (start, stop):
        if e is not None and not e.cuda_event:
            raise ValueError("record the event once before handing it to the library")
    sp = ctypes.c_void_p(start.cuda_event if start is not None else 0)
    ep = ctypes.c_void_p(stop.cuda_event if stop is not None else 0)
    _check(_lib.tqp_profile_events(kernel_class, sp, ep), "tqp_profile_events")


def lib_path() -> str:
    return _LIB_PATH
