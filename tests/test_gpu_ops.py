"""GPU parity of every C-ABI operator against the CPU oracle, element by
element, on seeded inputs: sizes from empty through several tiles with ragged
tails, every dtype, degenerate inputs.  All integer results: bit-exact."""
import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu

DT = [np.int8, np.int16, np.int32, np.int64]
TD = {np.int8: torch.int8, np.int16: torch.int16, np.int32: torch.int32, np.int64: torch.int64}


@pytest.fixture(scope="module")
def T():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import tqp
    return tqp


def rng(seed):
    return np.random.default_rng(seed)


def col(r, n, dt, lo=None, hi=None):
    info = np.iinfo(dt)
    lo = info.min if lo is None else lo
    hi = info.max if hi is None else hi
    return r.integers(lo, hi, size=n, endpoint=True, dtype=np.int64).astype(dt)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


SIZES = [0, 1, 2, 31, 4095, 4096, 4097, 3 * 4096 + 17, 100_003]


@pytest.mark.parametrize("n", SIZES)
def test_filter(T, n):
    r = rng(n + 1)
    cols = [col(r, n, DT[i % 4], -50, 50) for i in range(4)]
    for preds in ([], [(0, orc.LT, 10)], [(1, orc.GE, -3), (2, orc.NE, 0)],
                  [(0, orc.LE, 40), (1, orc.GT, -40), (2, orc.EQ, 7), (3, orc.NE, 1)],
                  [(3, orc.LT, -1000)], [(2, orc.GE, -1000)]):
        want = orc.filter(cols, preds)
        out, cnt = T.tqp_filter([dev(c) for c in cols], preds, n=n)
        k = int(cnt.item())
        assert k == len(want)
        assert np.array_equal(host(out, k), want)
    assert T.tqp_status_poll() == T.OK


def test_filter_large_ragged_and_device_count(T):
    n = 5_000_011
    r = rng(5)
    c = col(r, n, np.int32, 0, 2556)
    want = orc.filter([c], [(0, orc.LE, 2400)])
    out, cnt = T.tqp_filter([dev(c)], [(0, T.LE, 2400)])
    assert int(cnt.item()) == len(want) and np.array_equal(host(out, len(want)), want)
    # the row count read from the device
    dn = torch.tensor([1_234_567], dtype=torch.int64, device="cuda")
    out, cnt = T.tqp_filter([dev(c)], [(0, T.LE, 2400)], d_n=dn)
    want = orc.filter([c[:1_234_567]], [(0, orc.LE, 2400)])
    assert int(cnt.item()) == len(want) and np.array_equal(host(out, len(want)), want)


def test_filter_capacity_status(T):
    c = np.arange(10000, dtype=np.int32)
    out, cnt = T.tqp_filter([dev(c)], [(0, T.LT, 5000)], cap=100)
    assert int(cnt.item()) == 5000                      # the required size is still reported
    assert np.array_equal(host(out, 100), np.arange(100))
    assert T.tqp_status_poll() == T.ERR_CAPACITY
    assert T.tqp_status_poll() == T.OK                  # polling clears it


@pytest.mark.parametrize("dt", DT)
@pytest.mark.parametrize("n", [0, 1, 2, 3071, 3072, 4097, 5 * 4096 + 3, 200_001])
def test_sort_pairs(T, dt, n):
    r = rng(n * 7 + np.dtype(dt).itemsize)
    keys = col(r, n, dt)
    vals = r.integers(-2**31, 2**31 - 1, n).astype(np.int32)
    wk, wv = orc.sort_pairs(keys, vals)
    ko, vo = T.tqp_sort_pairs(dev(keys), dev(vals))
    assert np.array_equal(host(ko, n), wk) and np.array_equal(host(vo, n), wv)
    wk, wv = orc.sort_pairs(keys)                       # payload = row index
    ko, vo = T.tqp_sort_pairs(dev(keys))
    assert np.array_equal(host(ko, n), wk) and np.array_equal(host(vo, n), wv)


@pytest.mark.parametrize("dt", [np.int32, np.int64])
def test_sort_degenerate_and_bit_ranges(T, dt):
    w = np.dtype(dt).itemsize * 8
    r = rng(3)
    n = 70_001
    cases = {
        "equal": np.full(n, -5, dtype=dt),
        "sorted": np.sort(col(r, n, dt)),
        "reversed": np.sort(col(r, n, dt))[::-1].copy(),
        "few": col(r, n, dt, -2, 2),
        "extremes": r.choice(np.array([np.iinfo(dt).min, np.iinfo(dt).max, 0, -1], dtype=dt), n),
    }
    for name, keys in cases.items():
        wk, wv = orc.sort_pairs(keys)
        ko, vo = T.tqp_sort_pairs(dev(keys))
        assert np.array_equal(host(ko, n), wk), name
        assert np.array_equal(host(vo, n), wv), name
    keys = col(r, n, dt)
    for lo, hi in [(0, 8), (3, 17), (w - 9, w), (5, w - 3)]:
        wk, wv = orc.sort_pairs(keys, None, lo, hi)
        ko, vo = T.tqp_sort_pairs(dev(keys), None, lo, hi)
        assert np.array_equal(host(vo, n), wv), (lo, hi)
        assert np.array_equal(host(ko, n), wk), (lo, hi)


@pytest.mark.parametrize("dt", [np.int8, np.int32, np.int64])
@pytest.mark.parametrize("np_,nb", [(0, 10), (10, 0), (1, 1), (1000, 37), (50_001, 20_000), (300_007, 4093)])
def test_join_eq(T, dt, np_, nb):
    r = rng(np_ + nb)
    hi = 40 if dt == np.int8 else max(1, nb * 2)
    probe = col(r, np_, dt, -hi if dt == np.int8 else 0, hi)
    build = col(r, nb, dt, -hi if dt == np.int8 else 0, hi)
    wp, wb = orc.join_eq(probe, build)
    cap = max(1, len(wp))
    op, ob, cnt = T.tqp_join_eq(dev(probe), dev(build), cap)
    k = int(cnt.item())
    assert k == len(wp)
    assert np.array_equal(host(op, k), wp) and np.array_equal(host(ob, k), wb)


def test_join_unique_keys_and_capacity(T):
    r = rng(9)
    build = r.permutation(200_000).astype(np.int64) * 3 - 1000
    probe = r.integers(-2000, 700_000, 400_000).astype(np.int64)
    wp, wb = orc.join_eq(probe, build)
    op, ob, cnt = T.tqp_join_eq(dev(probe), dev(build), len(wp))
    k = int(cnt.item())
    assert k == len(wp) and np.array_equal(host(op, k), wp) and np.array_equal(host(ob, k), wb)
    op, ob, cnt = T.tqp_join_eq(dev(probe), dev(build), 10)
    assert int(cnt.item()) == len(wp)
    assert np.array_equal(host(op, 10), wp[:10])
    assert T.tqp_status_poll() == T.ERR_CAPACITY


GB_EXPRS = [[(0, 1, 0)], [(1, -1, 100), (2, 3, -7)], [(0, 1, 0), (1, 1, 5), (2, -2, 9)]]
GB_AGGS = [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 1), (orc.MAX, 1), (orc.SUM, 2), (orc.MIN, 2), (orc.MAX, 0),
           (orc.SUM, 1)]


def check_groupby(T, keys, vals, exprs, aggs, sel=None, n=None):
    wk, wa, _ = orc.groupby_agg(keys, vals, exprs, aggs, sel=sel, n=n)
    G = wa.shape[0]
    cap = max(G, 1)
    ok, oa, g = T.tqp_groupby_agg([dev(k) for k in keys], [dev(v) for v in vals], exprs, aggs, cap,
                                  sel=None if sel is None else dev(sel), n=n)
    assert int(g.item()) == G
    for i, k in enumerate(keys):
        assert np.array_equal(host(ok[i], G).astype(np.int64), wk[i])
    assert np.array_equal(host(oa)[:G], wa)
    assert T.tqp_status_poll() == T.OK


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2048, 2049, 3 * 2048 + 5, 150_001])
def test_groupby_shapes(T, n):
    r = rng(n + 11)
    vals = [col(r, n, np.int64, -10**9, 10**9), col(r, n, np.int32), col(r, n, np.int16)]
    # one int8 key (32-bit path), two keys, and a 64-bit composite key
    check_groupby(T, [col(r, n, np.int8, -3, 3)], vals, GB_EXPRS, GB_AGGS)
    check_groupby(T, [col(r, n, np.int16, -100, 100), col(r, n, np.int8)], vals, GB_EXPRS, GB_AGGS[:5])
    check_groupby(T, [col(r, n, np.int32, -5000, 5000), col(r, n, np.int64, -2, 2**40)], vals, GB_EXPRS,
                  GB_AGGS)


@pytest.mark.parametrize("n", [1, 4097, 300_001])
def test_groupby_small_key_domains(T, n):
    """A packed key of at most 10 bits folds straight into slots (no sort);
    11 bits take the sort.  Both sides of the boundary, two keys packed into
    one slot index, every aggregate, and a selection."""
    r = rng(n + 5)
    vals = [col(r, n, np.int64, -10**9, 10**9), col(r, n, np.int32), col(r, n, np.int16)]

    def with_ends(k, lo, hi):
        k[:2] = [lo, hi][:len(k[:2])]
        return k

    check_groupby(T, [with_ends(col(r, n, np.int16, -512, 511), -512, 511)], vals, GB_EXPRS, GB_AGGS)
    check_groupby(T, [with_ends(col(r, n, np.int16, -512, 512), -512, 512)], vals, GB_EXPRS, GB_AGGS)
    check_groupby(T, [col(r, n, np.int8, 0, 31), col(r, n, np.int64, -16, 15)], vals, GB_EXPRS, GB_AGGS)
    sel = np.sort(r.choice(n, max(1, n // 3), replace=False)).astype(np.int32)
    check_groupby(T, [col(r, n, np.int8, -2, 5)], vals, GB_EXPRS, GB_AGGS, sel=sel)


def test_groupby_small_domain_capacity(T):
    """More groups than the capacity: the count is still the group count,
    the first groups are written, and the status reports the overflow."""
    r = rng(8)
    n = 10_000
    k = col(r, n, np.int8, 0, 7)
    v = col(r, n, np.int64, -1000, 1000)
    wk, wa, _ = orc.groupby_agg([k], [v], [[(0, 1, 0)]], [(orc.SUM, 0), (orc.COUNT, 0)])
    ok, oa, g = T.tqp_groupby_agg([dev(k)], [dev(v)], [[(0, 1, 0)]], [(orc.SUM, 0), (orc.COUNT, 0)], 3)
    assert int(g.item()) == wa.shape[0] == 8
    assert np.array_equal(host(oa)[:3], wa[:3]) and np.array_equal(host(ok[0])[:3].astype(np.int64), wk[0][:3])
    assert T.tqp_status_poll() == T.ERR_CAPACITY


def test_groupby_degenerate(T):
    r = rng(2)
    n = 100_000
    v = [col(r, n, np.int64)]
    e = [[(0, 1, 0)]]
    a = [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 0), (orc.MAX, 0)]
    check_groupby(T, [np.full(n, 7, np.int32)], v, e, a)                      # one group
    check_groupby(T, [np.arange(n, dtype=np.int64)[::-1].copy()], v, e, a)     # all distinct
    ext = r.choice(np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).max, 0], np.int64), n)
    check_groupby(T, [ext], v, e, a)                                           # full 64-bit range
    check_groupby(T, [col(r, n, np.int64)], v, e, a)                           # 64 random bits
    sel = np.sort(r.choice(n, 33_333, replace=False)).astype(np.int32)
    check_groupby(T, [col(r, n, np.int16, -9, 9)], v, e, a, sel=sel)          # with a selection


def test_groupby_too_wide_key_reports_unsupported(T):
    r = rng(4)
    n = 1000
    k = [col(r, n, np.int64), col(r, n, np.int64)]
    ok, oa, g = T.tqp_groupby_agg([dev(x) for x in k], [dev(k[0])], [[(0, 1, 0)]], [(orc.COUNT, 0)], 2000)
    assert int(g.item()) == 0
    assert T.tqp_status_poll() == T.ERR_UNSUPPORTED


@pytest.mark.parametrize("dt", DT)
def test_gather(T, dt):
    r = rng(1)
    c = col(r, 10_000, dt)
    idx = r.integers(0, 10_000, 123_457).astype(np.int32)
    assert np.array_equal(host(T.tqp_gather(dev(c), dev(idx))), orc.gather(c, idx))


def test_bounded_wait_timeout_keeps_context_usable(T):
    """A scan tile that never publishes: its successors' bounded waits run
    out, the kernel records TIMEOUT and returns; the context stays usable."""
    c = np.arange(4096 * 12, dtype=np.int32)
    T.tqp_debug_set_spin_limit(2000)
    T.tqp_debug_inject_unpublished_tile(3)
    try:
        out, cnt = T.tqp_filter([dev(c)], [(0, T.GE, 0)])
        assert T.tqp_status_poll() == T.ERR_TIMEOUT
    finally:
        T.tqp_debug_inject_unpublished_tile(-1)
        T.tqp_debug_set_spin_limit(1 << 20)
    out, cnt = T.tqp_filter([dev(c)], [(0, T.GE, 0)])
    assert int(cnt.item()) == len(c) and np.array_equal(host(out), c)
    assert T.tqp_status_poll() == T.OK


# ---------------------------------------------------------------- strings
def string_tensor(r, n, width, alphabet=b"ABC"):
    """n zero-padded rows of random lengths 0..width over a small alphabet."""
    s = np.zeros((n, width), np.uint8)
    lens = r.integers(0, width + 1, n)
    letters = np.frombuffer(alphabet, np.uint8)[r.integers(0, len(alphabet), (n, width))]
    mask = np.arange(width)[None, :] < lens[:, None]
    s[mask] = letters[mask]
    return s


@pytest.mark.parametrize("width", [1, 7, 25, 256])
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 100_003])
def test_like_prefix(T, width, n):
    r = rng(width * 1000 + n)
    s = string_tensor(r, n, width)
    d = dev(s)
    # prefixes: empty, short, the full width, longer than the width (up to
    # the 64-byte limit of the call)
    for p in [b"", b"A", b"AB", b"ABCA"[: max(1, min(4, width))], b"C" * min(width, 64), b"B" * min(width + 1, 64)]:
        got = T.tqp_like_prefix(d, p)
        assert np.array_equal(host(got), orc.like_prefix(s, p)), p


def test_like_prefix_unaligned_rows_and_utf8(T):
    """A column that starts off a 16-byte boundary (byte loads), and
    multi-byte UTF-8 values with byte prefixes inside a character."""
    r = rng(5)
    vals = ["été", "étage", "ete", "é", "", "abé"] * 5000
    m = 9
    s = np.zeros((len(vals), m), np.uint8)
    for i, v in enumerate(vals):
        b = v.encode("utf-8")
        s[i, :len(b)] = np.frombuffer(b, np.uint8)
    flat = torch.zeros(s.size + 16, dtype=torch.uint8, device="cuda")
    off = flat[3:3 + s.size].view(len(vals), m)
    off.copy_(dev(s))
    assert off.data_ptr() % 16 == 3
    for p in ["é".encode(), "é".encode()[:1], "ét".encode(), b"a", b"e"]:
        assert np.array_equal(host(T.tqp_like_prefix(off, p)), orc.like_prefix(s, p)), p
    del r


def test_like_prefix_rejects_zero_byte_and_long_prefix(T):
    d = dev(np.zeros((4, 8), np.uint8))
    with pytest.raises(Exception):
        T.tqp_like_prefix(d, b"A\x00B")
    with pytest.raises(Exception):
        T.tqp_like_prefix(d, b"A" * 65)


@pytest.mark.parametrize("n,width", [(1, 1), (5000, 3), (100_003, 9), (300_000, 25)])
def test_string_codes(T, n, width):
    """Codes are the ranks among distinct values in byte order (unique, so
    compared exactly); each representative row holds its code's value."""
    r = rng(n + width)
    s = string_tensor(r, n, width, alphabet=b"ab\xc3\xa9")
    codes, rep, k = T.tqp_string_codes(dev(s))
    want, nk = orc.string_codes(s)
    assert int(k.item()) == nk
    assert np.array_equal(host(codes), want)
    rep = host(rep)[:nk]
    assert np.array_equal(want[rep], np.arange(nk))


def test_group_by_string_column(T):
    """GROUP BY the synthetic type strings of the promotion-revenue dimension:
    groups in string order with their aggregates."""
    from paper_2209_04579_b300 import datagen as dg
    from paper_2209_04579_b300 import queries as Q
    m = 400_000
    rec = dg.q14_promo_tables(m)
    table, _ = dg.type_strings()
    types = dg.type_column(m, rec["type_seed"], table)
    key = dg.make_table(rec["dim"], m)["key"].astype(np.int32)
    code, nk = orc.string_codes(types)
    wk, wa, _ = orc.groupby_agg([code], [key], [[(0, 1, 0)]], [(orc.COUNT, 0), (orc.MIN, 0), (orc.MAX, 0)])
    gk, ga, g, rep = Q.group_by_string(dev(types), [dev(key)], [[(0, 1, 0)]],
                                       [(T.COUNT, 0), (T.MIN, 0), (T.MAX, 0)], 256)
    G = wa.shape[0]
    assert int(g.item()) == G == nk == len(table)
    assert np.array_equal(host(gk)[:G].astype(np.int64), wk[0]) and np.array_equal(host(ga)[:G], wa)
    vals = [bytes(types[i]) for i in host(rep)[host(gk)[:G]]]
    assert vals == sorted(vals) and len(set(vals)) == G
    assert T.tqp_status_poll() == T.OK


@pytest.mark.parametrize("items32,items64", [(8, 6), (12, 8), (16, 12)])
def test_sort_every_tile_choice(T, items32, items64):
    """Every tile size the autotuner may pick sorts exactly as the oracle:
    stable, several tiles and a ragged tail, 32- and 64-bit keys, full and
    partial bit ranges."""
    r = rng(items32 * 7 + items64)
    try:
        T.tqp_sort_tiles(items32, items64)
        for dt, n in ((np.int32, 250_003), (np.int64, 180_001), (np.int16, 70_001)):
            k = col(r, n, dt)
            k[::5] = k[3]                        # ties: the payload shows stability
            v = r.integers(-2**31, 2**31, n).astype(np.int32)
            want = orc.sort_pairs(k, v)
            ko, vo = T.tqp_sort_pairs(dev(k), dev(v))
            assert np.array_equal(host(ko), want[0]) and np.array_equal(host(vo), want[1])
            bits = np.dtype(dt).itemsize * 8
            want = orc.sort_pairs(k, v, 3, bits - 5)
            ko, vo = T.tqp_sort_pairs(dev(k), dev(v), 3, bits - 5)
            assert np.array_equal(host(vo), want[1])
    finally:
        T.tqp_sort_tiles(16, 12)
    assert T.tqp_status_poll() == T.OK


def test_misaligned_workspace_is_rejected(T):
    """A workspace off the 256-byte boundary the header asks for is refused
    before any launch; the same call on the aligned buffer sorts."""
    import ctypes
    keys = torch.arange(1000, 0, -1, dtype=torch.int64, device="cuda")
    ko = torch.empty_like(keys)
    vo = torch.empty(1000, dtype=torch.int32, device="cuda")
    args = [T._DTYPE[keys.dtype], T._ptr(keys), None, T._ptr(ko), T._ptr(vo), 1000, None, 0, 64]
    need = ctypes.c_size_t(0)
    assert T._lib.tqp_sort_pairs(*args, None, ctypes.byref(need), None) == T.OK
    ws = torch.empty(need.value + 512, dtype=torch.uint8, device="cuda")
    have = ctypes.c_size_t(need.value)
    base = ws.data_ptr()
    aligned = (base + 255) & ~255
    assert T._lib.tqp_sort_pairs(*args, ctypes.c_void_p(aligned + 32), ctypes.byref(have), None) == T.ERR_INVALID
    assert T._lib.tqp_sort_pairs(*args, ctypes.c_void_p(aligned), ctypes.byref(have), None) == T.OK
    torch.cuda.synchronize()
    assert torch.equal(ko, torch.arange(1, 1001, dtype=torch.int64, device="cuda"))
