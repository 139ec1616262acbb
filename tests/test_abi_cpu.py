"""The C-ABI libraries load and export every function their headers declare;
host-side argument checks and workspace size queries work without a GPU
(no compute call is made here)."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2209_04579_b300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2209_04579_b300 import build
    build.build()


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tqp[a-z_0-9]*)\s*\(", text, flags=re.M)))


@pytest.mark.parametrize("header,lib", [("tqp.h", "libtqp.so"), ("tqp_datagen.h", "libtqpgen.so")])
def test_every_declared_symbol_is_exported(header, lib):
    names = declared(header)
    assert names, header
    so = ctypes.CDLL(os.path.join(PKG, lib))
    for n in names:
        assert hasattr(so, n), n


def test_declared_list_is_complete():
    names = declared("tqp.h")
    for must in ("tqp_filter", "tqp_sort_pairs", "tqp_join_eq", "tqp_groupby_agg", "tqp_star_agg",
                 "tqp_gather", "tqp_status_poll"):
        assert must in names


def test_host_argument_checks_and_size_queries():
    from paper_2209_04579_b300 import tqp
    lib = tqp._lib
    sz = ctypes.c_size_t(0)
    # negative n -> invalid, before any device work
    st = lib.tqp_filter(None, 0, None, 0, -1, None, None, 0, None, None, ctypes.byref(sz), None)
    assert st == tqp.ERR_INVALID
    # size query of a sort: no device work, a positive size
    st = lib.tqp_sort_pairs(tqp.I32, None, None, None, None, 1000, None, 0, 32, None, ctypes.byref(sz), None)
    assert st == tqp.OK and sz.value > 1000 * 4
    # bad bit range and bad dtype
    assert lib.tqp_sort_pairs(tqp.I32, None, None, None, None, 10, None, 5, 40, None, ctypes.byref(sz), None) \
        == tqp.ERR_INVALID
    assert lib.tqp_sort_pairs(9, None, None, None, None, 10, None, 0, 8, None, ctypes.byref(sz), None) \
        == tqp.ERR_DTYPE
    # group-by: size query, and too many keys
    keys = (tqp.Col * 5)(*[tqp.Col(None, tqp.I32, 0) for _ in range(5)])
    aggs = (tqp.Agg * 1)(tqp.Agg(tqp.COUNT, 0))
    st = lib.tqp_groupby_agg(keys, 1, None, 0, None, 0, aggs, 1, None, 100, None, None, None, 0, None, None,
                             ctypes.byref(sz), None)
    assert st == tqp.OK and sz.value > 0
    st = lib.tqp_groupby_agg(keys, 5, None, 0, None, 0, aggs, 1, None, 100, None, None, None, 0, None, None,
                             ctypes.byref(sz), None)
    assert st == tqp.ERR_INVALID
    # join with mismatched dtypes
    st = lib.tqp_join_eq(tqp.Col(None, tqp.I32, 0), 10, None, tqp.Col(None, tqp.I64, 0), 10, None, None, None, 0,
                         None, None, ctypes.byref(sz), None)
    assert st == tqp.ERR_DTYPE
    # workspace too small is reported before launching
    st = lib.tqp_sort_pairs(tqp.I32, None, None, None, None, 1000, None, 0, 32, ctypes.c_void_p(256),
                            ctypes.byref(ctypes.c_size_t(16)), None)
    assert st == tqp.ERR_WORKSPACE
    assert lib.tqp_status_string(tqp.ERR_TIMEOUT) == b"bounded wait ran out"


def test_empty_inputs_accept_null_data():
    """Empty columns have no storage (NULL data); n = 0 must not be an argument error."""
    from paper_2209_04579_b300 import tqp
    lib = tqp._lib
    sz = ctypes.c_size_t(0)
    cols = (tqp.Col * 1)(tqp.Col(None, tqp.I32, 0))
    preds = (tqp.Pred * 1)(tqp.Pred(0, tqp.LT, 5))
    assert lib.tqp_filter(cols, 1, preds, 1, 0, None, None, 0, None, None, ctypes.byref(sz), None) == tqp.OK
    if not torch.cuda.is_available():
        # no device here: the call gets past the argument checks and its first
        # CUDA call (a memset of the count) reports ERR_CUDA; placeholder
        # pointers are never handed to a real device
        ws = ctypes.c_void_p(256)
        st = lib.tqp_filter(cols, 1, preds, 1, 0, None, None, 0, ctypes.c_void_p(512), ws, ctypes.byref(sz), None)
        assert st == tqp.ERR_CUDA
    vals = (tqp.Col * 1)(tqp.Col(None, tqp.I64, 0))
    ex = (tqp.Expr * 1)()
    ex[0].nterms = 1
    ex[0].term[0] = tqp.Term(0, 0, 1, 0)
    aggs = (tqp.Agg * 1)(tqp.Agg(tqp.SUM, 0))
    st = lib.tqp_groupby_agg(cols, 1, vals, 1, ex, 1, aggs, 1, None, 0, None, None, None, 0, None, None,
                             ctypes.byref(sz), None)
    assert st == tqp.OK


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror of a header struct has the C size and field offsets."""
    import subprocess
    from paper_2209_04579_b300 import tqp
    mirrors = {"tqp_col": tqp.Col, "tqp_pred": tqp.Pred, "tqp_term": tqp.Term, "tqp_expr": tqp.Expr,
               "tqp_agg": tqp.Agg, "tqp_dim": tqp.Dim, "tqp_valref": tqp.ValRef, "tqp_cdf_model": tqp.CdfModel,
               "tqp_train_cfg": tqp.TrainCfg, "tqp_learned_cfg": tqp.LearnedCfg,
               "tqp_learned_stats": tqp.LearnedStats, "tqp_batch_shape": tqp.BatchShape,
               "tqp_problem": tqp.Problem, "tqp_batch_cfg": tqp.BatchCfg}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tqp.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    want = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            want[(a, b)] = int(v)
    for cname, cls in mirrors.items():
        assert want[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert want[(cname, f)] == getattr(cls, f).offset, (cname, f)


def _header_text():
    text = open(os.path.join(ROOT, "include", "tqp.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _enum_values(text, name):
    """Values of the members of `typedef enum { ... } name;` (explicit or
    counted from the previous member)."""
    body = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text, flags=re.S).group(1)
    out, nxt = {}, 0
    for item in body.split(","):
        item = item.strip()
        if not item:
            continue
        m = re.match(r"([A-Z_0-9]+)\s*(?:=\s*(-?\d+))?$", item)
        assert m, item
        nxt = int(m.group(2)) if m.group(2) is not None else nxt
        out[m.group(1)] = nxt
        nxt += 1
    return out


def test_binding_constants_match_header():
    """The Python binding restates the header's status codes, enums and
    limits; they must stay in step with include/tqp.h."""
    from paper_2209_04579_b300 import tqp
    text = _header_text()
    status = _enum_values(text, "tqp_status")
    assert status == {"TQP_OK": tqp.OK, "TQP_ERR_INVALID": tqp.ERR_INVALID, "TQP_ERR_DTYPE": tqp.ERR_DTYPE,
                      "TQP_ERR_CAPACITY": tqp.ERR_CAPACITY, "TQP_ERR_CUDA": tqp.ERR_CUDA,
                      "TQP_ERR_TIMEOUT": tqp.ERR_TIMEOUT, "TQP_ERR_WORKSPACE": tqp.ERR_WORKSPACE,
                      "TQP_ERR_UNSUPPORTED": tqp.ERR_UNSUPPORTED, "TQP_ERR_TOO_LARGE": tqp.ERR_TOO_LARGE}
    assert _enum_values(text, "tqp_dtype") == {"TQP_I8": tqp.I8, "TQP_I16": tqp.I16, "TQP_I32": tqp.I32,
                                               "TQP_I64": tqp.I64}
    assert _enum_values(text, "tqp_cmp") == {"TQP_LT": tqp.LT, "TQP_LE": tqp.LE, "TQP_GT": tqp.GT,
                                             "TQP_GE": tqp.GE, "TQP_EQ": tqp.EQ, "TQP_NE": tqp.NE}
    assert _enum_values(text, "tqp_aggop") == {"TQP_COUNT": tqp.COUNT, "TQP_SUM": tqp.SUM, "TQP_MIN": tqp.MIN,
                                               "TQP_MAX": tqp.MAX}
    m = re.search(r"#define\s+TQP_NOALLOC_MAX_ROWS\s+\(1LL\s*<<\s*(\d+)\)", text)
    assert m and (1 << int(m.group(1))) == tqp.NOALLOC_MAX_ROWS
    m = re.search(r"#define\s+TQP_CDF_HIDDEN\s+(\d+)", text)
    assert m and int(m.group(1)) == tqp.H


def test_sort_tiles_setting_checks():
    """The sort tile setting accepts only its compiled choices (no device work)."""
    from paper_2209_04579_b300 import tqp
    lib = tqp._lib
    assert lib.tqp_sort_tiles(7, 0) == tqp.ERR_INVALID
    assert lib.tqp_sort_tiles(0, 16) == tqp.ERR_INVALID
    assert lib.tqp_sort_tiles(0, 0) == tqp.OK
    assert lib.tqp_sort_tiles(16, 12) == tqp.OK      # the defaults
