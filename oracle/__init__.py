"""Plain CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it.  The arithmetic lives in
``tqp_oracle.cpp`` (single-threaded C++, standard library containers); this
module loads it with ctypes and composes the per-workload query pipelines from
its operators.

Every function is pinned by CPU tests against something other than itself
(brute force on tiny tables, textbook library routines, invariants, closed
forms, finite differences); there is no "parity unpinned" function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tqp_oracle.cpp")
_LIB = os.path.join(_HERE, "libtqp_oracle.so")

LT, LE, GT, GE, EQ, NE = range(6)
COUNT, SUM, MIN, MAX = range(4)
_DT = {np.dtype(np.int8): 1, np.dtype(np.int16): 2, np.dtype(np.int32): 3, np.dtype(np.int64): 4}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library in place (g++, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.orc_filter.restype = ctypes.c_int64
        _lib.orc_join_eq.restype = ctypes.c_int64
        _lib.orc_groupby_agg.restype = ctypes.c_int64
        _lib.orc_cdf_grad_f64.restype = ctypes.c_double
        _lib.orc_string_codes.restype = ctypes.c_int64
        _lib.orc_light_cdf_targets.restype = ctypes.c_int64
        _lib.orc_date_parse_iso.restype = ctypes.c_int64
        _lib.orc_date_from_days.restype = ctypes.c_int64
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _ptrs(arrs):
    return (ctypes.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])


def _ints(xs):
    return (ctypes.c_int * max(1, len(xs)))(*xs)


def _i64s(xs):
    return (ctypes.c_int64 * max(1, len(xs)))(*xs)


def filter(cols, preds):
    """cols: list of int arrays (same length); preds: [(col, op, literal)].
    Returns the ascending int32 indices of rows where every predicate holds."""
    cols = [np.ascontiguousarray(c) for c in cols]
    n = len(cols[0]) if cols else 0
    out = np.empty(max(n, 1), dtype=np.int32)
    k = lib().orc_filter(_ptrs(cols), _ints([_DT[c.dtype] for c in cols]), ctypes.c_int64(n),
                         len(preds), _ints([p[0] for p in preds]), _ints([p[1] for p in preds]),
                         _i64s([p[2] for p in preds]), _p(out))
    return out[:k].copy()


def sort_pairs(keys, vals=None, begin_bit=0, end_bit=None):
    """Stable ascending sort of (key, val) by bits [begin_bit, end_bit) of the
    sign-flipped key.  vals None -> the payload is the input row index."""
    keys = np.ascontiguousarray(keys)
    n = len(keys)
    if end_bit is None:
        end_bit = keys.dtype.itemsize * 8
    ko = np.empty_like(keys)
    vo = np.empty(n, dtype=np.int32)
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.int32)
    lib().orc_sort_pairs(_p(keys), _DT[keys.dtype], _p(v), ctypes.c_int64(n), begin_bit, end_bit,
                         _p(ko), _p(vo))
    return ko, vo


def join_eq(probe, build):
    """Inner equi-join pairs (probe_row, build_row), ordered by (probe_row, build_row)."""
    probe = np.ascontiguousarray(probe)
    build = np.ascontiguousarray(build)
    lb = lib()
    cnt = lb.orc_join_eq(_p(probe), _DT[probe.dtype], ctypes.c_int64(len(probe)), _p(build),
                         _DT[build.dtype], ctypes.c_int64(len(build)), ctypes.c_void_p(0),
                         ctypes.c_void_p(0), ctypes.c_int64(0))
    op = np.empty(max(cnt, 1), dtype=np.int32)
    ob = np.empty(max(cnt, 1), dtype=np.int32)
    lb.orc_join_eq(_p(probe), _DT[probe.dtype], ctypes.c_int64(len(probe)), _p(build),
                   _DT[build.dtype], ctypes.c_int64(len(build)), _p(op), _p(ob), ctypes.c_int64(cnt))
    return op[:cnt].copy(), ob[:cnt].copy()


def gather(col, idx):
    col = np.ascontiguousarray(col)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(len(idx), dtype=col.dtype)
    lib().orc_gather(_p(col), _DT[col.dtype], _p(idx), ctypes.c_int64(len(idx)), _p(out))
    return out


def groupby_agg(keys, vals, exprs, aggs, sel=None, n=None):
    """keys: list of key columns; vals: list of value columns; exprs: list of
    expressions, each a list of up to 3 terms (col, mul, add) multiplied
    together; aggs: list of (op, expr) with op in COUNT/SUM/MIN/MAX.
    Returns (group_keys int64 [nkeys][G], aggs int64 [G][naggs], overflow)."""
    keys = [np.ascontiguousarray(k) for k in keys]
    vals = [np.ascontiguousarray(v) for v in vals]
    if n is None:
        n = len(sel) if sel is not None else len(keys[0])
    selp = None if sel is None else np.ascontiguousarray(sel, dtype=np.int32)
    nt, tc, tm, ta = [], [], [], []
    for e in exprs:
        assert 1 <= len(e) <= 3
        nt.append(len(e))
        for t in range(3):
            c, m, a = e[t] if t < len(e) else (0, 0, 1)
            tc.append(c); tm.append(m); ta.append(a)
    of = ctypes.c_int(0)
    lb = lib()
    args = [_ptrs(keys), _ints([_DT[k.dtype] for k in keys]), len(keys), _ptrs(vals),
            _ints([_DT[v.dtype] for v in vals]), _ints(nt), _ints(tc), _i64s(tm), _i64s(ta),
            len(exprs), _ints([a[0] for a in aggs]), _ints([a[1] for a in aggs]), len(aggs),
            _p(selp), ctypes.c_int64(n)]
    g = lb.orc_groupby_agg(*args, ctypes.c_void_p(0), ctypes.c_void_p(0), ctypes.c_int64(0),
                           ctypes.byref(of))
    ok = np.empty((len(keys), max(g, 1)), dtype=np.int64)
    oa = np.empty((max(g, 1), len(aggs)), dtype=np.int64)
    lb.orc_groupby_agg(*args, _p(ok), _p(oa), ctypes.c_int64(max(g, 1)), ctypes.byref(of))
    return ok[:, :g].copy(), oa[:g].copy(), bool(of.value)


# ---------------------------------------------------------------- CDF model

def cdf_normalize(keys, umin, shift, inv):
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    x = np.empty(len(keys), dtype=np.float32)
    lib().orc_cdf_normalize(_p(keys), ctypes.c_int64(len(keys)), ctypes.c_uint64(umin), shift,
                            ctypes.c_float(inv), _p(x))
    return x


def cdf_forward_f32(w, b, a, c, x):
    w, b, a = (np.ascontiguousarray(t, dtype=np.float32) for t in (w, b, a))
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(len(x), dtype=np.float32)
    lib().orc_cdf_forward_f32(_p(w), _p(b), _p(a), ctypes.c_float(c), len(w), _p(x),
                              ctypes.c_int64(len(x)), _p(out))
    return out


def cdf_bucket(F, B):
    F = np.ascontiguousarray(F, dtype=np.float32)
    out = np.empty(len(F), dtype=np.int32)
    lib().orc_cdf_bucket(_p(F), ctypes.c_int64(len(F)), B, _p(out))
    return out


def cdf_forward_f64(w, b, a, c, x):
    w, b, a, x = (np.ascontiguousarray(t, dtype=np.float64) for t in (w, b, a, x))
    out = np.empty(len(x), dtype=np.float64)
    lib().orc_cdf_forward_f64(_p(w), _p(b), _p(a), ctypes.c_double(c), len(w), _p(x),
                              ctypes.c_int64(len(x)), _p(out))
    return out


def cdf_grad_f64(w, b, a, c, x, y):
    """Returns (loss, gw, gb, ga, gc) of the MSE loss in float64."""
    w, b, a, x, y = (np.ascontiguousarray(t, dtype=np.float64) for t in (w, b, a, x, y))
    H = len(w)
    gw, gb, ga = np.empty(H), np.empty(H), np.empty(H)
    gc = ctypes.c_double(0)
    loss = lib().orc_cdf_grad_f64(_p(w), _p(b), _p(a), ctypes.c_double(c), H, _p(x), _p(y),
                                  ctypes.c_int64(len(x)), _p(gw), _p(gb), _p(ga), ctypes.byref(gc))
    return loss, gw, gb, ga, gc.value


def adam_step_f64(p, g, m, v, nonneg, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step plus projection of the flagged entries onto >= 0."""
    nn = np.ascontiguousarray(nonneg, dtype=np.int32)
    lib().orc_adam_step_f64(_p(p), _p(np.ascontiguousarray(g, dtype=np.float64)), _p(m), _p(v),
                            _p(nn), len(p), t, ctypes.c_double(lr), ctypes.c_double(beta1),
                            ctypes.c_double(beta2), ctypes.c_double(eps))


def cdf_targets(sorted_keys):
    s = np.ascontiguousarray(sorted_keys, dtype=np.int64)
    y = np.empty(len(s), dtype=np.float64)
    lib().orc_cdf_targets(_p(s), ctypes.c_int64(len(s)), _p(y))
    return y


def partition(bucket, B):
    bucket = np.ascontiguousarray(bucket, dtype=np.int32)
    rows = np.empty(len(bucket), dtype=np.int32)
    off = np.empty(B + 1, dtype=np.int64)
    lib().orc_partition(_p(bucket), ctypes.c_int64(len(bucket)), B, _p(rows), _p(off))
    return rows, off


def like_prefix(strings, prefix: bytes):
    """strings: (n, m) uint8, zero-padded rows; 1 where the value starts with prefix."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    n, m = s.shape
    p = np.frombuffer(prefix, dtype=np.uint8) if prefix else np.zeros(1, np.uint8)
    out = np.empty(n, dtype=np.int8)
    lib().orc_like_prefix(_p(s), ctypes.c_int64(n), m, _p(np.ascontiguousarray(p)), len(prefix), _p(out))
    return out


def string_codes(strings):
    """(codes int32 [n], number of distinct values): each row's rank among
    the distinct zero-padded rows in ascending byte order."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    n, m = s.shape
    code = np.empty(n, dtype=np.int32)
    k = lib().orc_string_codes(_p(s), ctypes.c_int64(n), m, _p(code))
    return code, int(k)


def light_cdf_targets(sorted_keys, mult, s_train, min_count, max_heavy):
    """Training targets over the CDF of the light sample keys (heavy runs:
    count >= the cut, aggregated directly).  sorted_keys: uint64 ascending.
    Returns (y float32 [s_train], heavy keys uint64 ascending)."""
    s = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    y = np.empty(max(s_train, 1), dtype=np.float32)
    heavy = np.empty(max(max_heavy, 1), dtype=np.uint64)
    k = lib().orc_light_cdf_targets(_p(s), ctypes.c_int64(len(s)), ctypes.c_int64(mult), ctypes.c_int64(s_train),
                                    ctypes.c_int64(min_count), ctypes.c_int64(max_heavy), _p(heavy), _p(y))
    return y[:s_train].copy(), heavy[:k].copy()


def date_parse_iso(strings):
    """(n, m) uint8 zero-padded 'YYYY-MM-DD' rows -> (epoch ns int64, ok int8)."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    n, m = s.shape
    ns = np.empty(n, dtype=np.int64)
    ok = np.empty(n, dtype=np.int8)
    lib().orc_date_parse_iso(_p(s), ctypes.c_int64(n), m, _p(ns), _p(ok))
    return ns, ok


def date_from_days(days):
    d = np.ascontiguousarray(days, dtype=np.int32)
    ns = np.empty(len(d), dtype=np.int64)
    lib().orc_date_from_days(_p(d), ctypes.c_int64(len(d)), _p(ns))
    return ns


def date_parts(ns):
    """Epoch ns -> (day number, year, month, day of month), all int32."""
    t = np.ascontiguousarray(ns, dtype=np.int64)
    out = [np.empty(len(t), dtype=np.int32) for _ in range(4)]
    lib().orc_date_parts(_p(t), ctypes.c_int64(len(t)), *[_p(o) for o in out])
    return tuple(out)
