"""Pins of the CPU oracle against things other than itself: brute-force loops
on tiny tables, Python's and numpy's stable sorts, collection counters,
invariants, closed forms and a hand-worked example.  CPU only."""
import collections
import itertools

import numpy as np
import pytest

import oracle as orc
from oracle import pipelines as pl
from paper_2209_04579_b300 import datagen as dg

RNG = np.random.default_rng(7)
DTS = [np.int8, np.int16, np.int32, np.int64]
OPS = {orc.LT: lambda v, l: v < l, orc.LE: lambda v, l: v <= l, orc.GT: lambda v, l: v > l,
       orc.GE: lambda v, l: v >= l, orc.EQ: lambda v, l: v == l, orc.NE: lambda v, l: v != l}


def rand_col(n, dt, lo=None, hi=None):
    info = np.iinfo(dt)
    lo = info.min if lo is None else lo
    hi = info.max if hi is None else hi
    return RNG.integers(lo, hi, size=n, endpoint=True, dtype=np.int64).astype(dt)


# ------------------------------------------------------------------ filter

@pytest.mark.parametrize("n", [0, 1, 2, 17, 300])
def test_filter_brute_force(n):
    for trial in range(20):
        cols = [rand_col(n, DTS[(trial + c) % 4], -5, 5) for c in range(3)]
        npred = trial % 5
        preds = [(int(RNG.integers(0, 3)), int(RNG.integers(0, 6)), int(RNG.integers(-6, 7)))
                 for _ in range(npred)]
        got = orc.filter(cols, preds)
        want = [i for i in range(n) if all(OPS[op](int(cols[c][i]), lit) for c, op, lit in preds)]
        assert got.tolist() == want


def test_filter_extreme_literals():
    c = np.array([np.iinfo(np.int64).min, -1, 0, 1, np.iinfo(np.int64).max], dtype=np.int64)
    assert orc.filter([c], [(0, orc.LT, np.iinfo(np.int64).min)]).tolist() == []
    assert orc.filter([c], [(0, orc.LE, np.iinfo(np.int64).max)]).tolist() == [0, 1, 2, 3, 4]
    c8 = np.array([-128, 127, 0], dtype=np.int8)
    # literal outside the int8 range compares as a 64-bit signed value
    assert orc.filter([c8], [(0, orc.LT, 1000)]).tolist() == [0, 1, 2]
    assert orc.filter([c8], [(0, orc.GT, -1000)]).tolist() == [0, 1, 2]


def test_filter_selectivity_closed_form():
    t = dg.make_table(dg.q6_lineitem(), 1_000_000)
    k = len(orc.filter([t["ship_day"]], [(0, orc.LE, 2400)]))
    p = 2401 / 2557
    sd = (1_000_000 * p * (1 - p)) ** 0.5
    assert abs(k - 1_000_000 * p) < 6 * sd


# ------------------------------------------------------------------ sort

@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("n", [0, 1, 2, 33, 500])
def test_sort_pairs_stable_python_sorted(dt, n):
    keys = rand_col(n, dt, -20, 20) if n < 100 else rand_col(n, dt)
    vals = RNG.integers(-1000, 1000, size=n).astype(np.int32)
    ko, vo = orc.sort_pairs(keys, vals)
    order = sorted(range(n), key=lambda i: int(keys[i]))   # Python's sort is stable
    assert ko.tolist() == [int(keys[i]) for i in order]
    assert vo.tolist() == [int(vals[i]) for i in order]


@pytest.mark.parametrize("dt", DTS)
def test_sort_pairs_bit_range_numpy(dt):
    n = 5000
    keys = rand_col(n, dt)
    w = np.dtype(dt).itemsize * 8
    ub = keys.astype(np.int64).view(np.uint64) & np.uint64((1 << w) - 1 if w < 64 else 2**64 - 1)
    ub = ub ^ np.uint64(1 << (w - 1))
    for lo, hi in [(0, w), (0, 3), (2, 7), (w - 5, w), (1, w - 1)]:
        ko, vo = orc.sort_pairs(keys, None, lo, hi)
        field = (ub >> np.uint64(lo)) & np.uint64((1 << (hi - lo)) - 1)
        perm = np.argsort(field, kind="stable")
        assert np.array_equal(vo, perm.astype(np.int32))
        assert np.array_equal(ko, keys[perm])


def test_sort_extremes_and_invariants():
    k = np.array([0, np.iinfo(np.int64).max, np.iinfo(np.int64).min, -1, 1, -1, 0], dtype=np.int64)
    ko, vo = orc.sort_pairs(k)
    assert ko.tolist() == sorted(k.tolist())
    assert vo.tolist() == [2, 3, 5, 0, 6, 4, 1]
    big = rand_col(20000, np.int32, -50, 50)
    ko, vo = orc.sort_pairs(big)
    assert np.all(ko[1:] >= ko[:-1])                       # non-decreasing
    assert np.array_equal(np.sort(vo), np.arange(20000))   # permutation
    same = ko[1:] == ko[:-1]
    assert np.all(vo[1:][same] > vo[:-1][same])            # stable: ties in input order
    assert np.array_equal(big[vo], ko)


# ------------------------------------------------------------------ join

@pytest.mark.parametrize("np_,nb", [(0, 0), (0, 5), (5, 0), (1, 1), (40, 30), (200, 7)])
def test_join_nested_loops(np_, nb):
    for dt_p, dt_b in [(np.int32, np.int32), (np.int64, np.int64), (np.int8, np.int16)]:
        p = rand_col(np_, dt_p, -4, 4)
        b = rand_col(nb, dt_b, -4, 4)
        got = orc.join_eq(p, b)
        want = [(i, j) for i in range(np_) for j in range(nb) if int(p[i]) == int(b[j])]
        assert list(zip(got[0].tolist(), got[1].tolist())) == want


def test_join_cardinality_invariant():
    p = rand_col(100_000, np.int32, 0, 3000)
    b = rand_col(5000, np.int32, 0, 3000)
    pr, br = orc.join_eq(p, b)
    cp, cb = collections.Counter(p.tolist()), collections.Counter(b.tolist())
    assert len(pr) == sum(cp[k] * cb[k] for k in cp)
    assert np.array_equal(p[pr], b[br])
    order = np.lexsort((br, pr))
    assert np.array_equal(order, np.arange(len(pr)))


def test_join_no_match_all_match():
    p = np.arange(100, dtype=np.int32)
    assert len(orc.join_eq(p, p + 1000)[0]) == 0
    pr, br = orc.join_eq(np.zeros(50, np.int32), np.zeros(3, np.int32))
    assert len(pr) == 150 and pr.tolist() == [i for i in range(50) for _ in range(3)]


# ------------------------------------------------------------------ group-by

def brute_groupby(keys, vals, exprs, aggs, rows):
    """O(n * G) search over a list of groups; 64-bit wrap by masking."""
    groups = []
    M = 1 << 64

    def wrap(x):
        x %= M
        return x - M if x >= 1 << 63 else x

    for r in rows:
        kt = tuple(int(k[r]) for k in keys)
        ev = []
        for e in exprs:
            v = 1
            for c, m, a in e:
                v = wrap(v * wrap(m * int(vals[c][r]) + a))
            ev.append(v)
        for g in groups:
            if g[0] == kt:
                break
        else:
            g = [kt, []]
            groups.append(g)
        g[1].append(ev)
    groups.sort(key=lambda g: g[0])
    out_k, out_a = [], []
    for kt, evs in groups:
        out_k.append(kt)
        row = []
        for op, e in aggs:
            xs = [ev[e] for ev in evs]
            row.append(len(xs) if op == orc.COUNT else wrap(sum(xs)) if op == orc.SUM
                       else min(xs) if op == orc.MIN else max(xs))
        out_a.append(row)
    return out_k, out_a


@pytest.mark.parametrize("n", [0, 1, 5, 64, 400])
def test_groupby_brute_force(n):
    for trial in range(6):
        nk = 1 + trial % 3
        keys = [rand_col(n, DTS[(trial + i) % 4], -3, 3) for i in range(nk)]
        vals = [rand_col(n, DTS[(trial + i + 1) % 4]) for i in range(3)]
        exprs = [[(0, 1, 0)], [(1, -1, 100), (2, 3, -7)], [(0, 1, 0), (1, 1, 5), (2, -2, 9)]]
        aggs = [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 1), (orc.MAX, 1), (orc.SUM, 2), (orc.MIN, 2)]
        sel = None
        rows = list(range(n))
        if trial % 2 and n:
            sel = np.sort(RNG.choice(n, size=n // 2, replace=False)).astype(np.int32)
            rows = sel.tolist()
        gk, ga, _ = orc.groupby_agg(keys, vals, exprs, aggs, sel=sel)
        wk, wa = brute_groupby(keys, vals, exprs, aggs, rows)
        assert [tuple(c) for c in gk.T.tolist()] == wk
        assert ga.tolist() == wa


def test_groupby_invariants_and_overflow():
    t = dg.make_table(dg.q6_lineitem(), 200_000)
    gk, ga, of = pl.q6(t)
    assert not of
    sel = orc.filter([t["ship_day"]], [(0, orc.LE, 2400)])
    assert ga[:, 4].sum() == len(sel)                            # sum of COUNT = |selection|
    assert int(ga[:, 1].sum()) == int(t["price"][sel].sum())     # sum of SUM = column SUM
    kk = [tuple(c) for c in gk.T.tolist()]
    assert kk == sorted(set(kk)) and len(kk) == 6                # strictly increasing, 3 x 2 groups
    # wrapping and the overflow flag
    big = np.array([2**62, 2**62, 2**62], dtype=np.int64)
    _, ga, of = orc.groupby_agg([np.zeros(3, np.int8)], [big], [[(0, 1, 0)]], [(orc.SUM, 0)])
    assert of and int(ga[0, 0]) == (3 * 2**62) - 2**64
    _, _, of = orc.groupby_agg([np.zeros(1, np.int8)], [big[:1]], [[(0, 4, 0)]], [(orc.SUM, 0)])
    assert of


def test_q6_hand_worked_example():
    """Eight rows worked by hand.  Rows with ship_day <= 2400: 0, 1, 2, 4, 5, 7.
    Groups (flag_a, flag_b): (0,0) <- rows 0, 4; (0,1) <- row 5; (2,1) <- rows 1, 2, 7.
    (0,0): qty 100+300=400; price 1000+3000=4000; price*(100-disc): 1000*95 + 3000*100
           = 395000; *(100+tax): 1000*95*108 + 3000*100*100 = 10260000 + 30000000 = 40260000.
    (0,1): qty 500; price 5000; 5000*90 = 450000; 450000*101 = 45450000.
    (2,1): qty 200+100+700=1000; price 2000+7000+9000=18000;
           2000*100 + 7000*99 + 9000*98 = 200000 + 693000 + 882000 = 1775000;
           200000*100 + 693000*102 + 882000*100 = 20000000 + 70686000 + 88200000 = 178886000."""
    t = {
        "ship_day": np.array([10, 2400, 0, 2401, 5, 77, 2556, 1500], np.int32),
        "flag_a": np.array([0, 2, 2, 0, 0, 0, 1, 2], np.int8),
        "flag_b": np.array([0, 1, 1, 0, 0, 1, 0, 1], np.int8),
        "qty": np.array([100, 200, 100, 900, 300, 500, 400, 700], np.int64),
        "price": np.array([1000, 2000, 7000, 8000, 3000, 5000, 6000, 9000], np.int64),
        "disc": np.array([5, 0, 1, 3, 0, 10, 2, 2], np.int64),
        "tax": np.array([8, 0, 2, 1, 0, 1, 4, 0], np.int64),
    }
    gk, ga, of = pl.q6(t)
    assert gk.T.tolist() == [[0, 0], [0, 1], [2, 1]]
    assert ga.tolist() == [[400, 4000, 395000, 40260000, 2],
                           [500, 5000, 450000, 45450000, 1],
                           [1000, 18000, 1775000, 178886000, 3]]


def test_q14_pipeline_vs_brute_force():
    fact = {"fk": rand_col(300, np.int32, 0, 40)}
    dim = {"key": np.arange(0, 60, 2, dtype=np.int32)[RNG.permutation(30)],
           "region": rand_col(30, np.int8, 0, 24), "price": rand_col(30, np.int64, 100, 10**6)}
    gk, ga, _ = pl.q14(fact, dim)
    acc = collections.defaultdict(lambda: [0, 0])
    for i in range(300):
        for j in range(30):
            if fact["fk"][i] == dim["key"][j] and dim["region"][j] < 5:
                acc[int(dim["region"][j])][0] += int(dim["price"][j])
                acc[int(dim["region"][j])][1] += 1
    ks = sorted(acc)
    assert gk[0].tolist() == ks
    assert ga.tolist() == [acc[k] for k in ks]


def test_star_and_batched_pipelines_vs_brute_force():
    fact = {"fk1": rand_col(200, np.int32, 0, 9), "fk2": rand_col(200, np.int64, 0, 12),
            "m1": rand_col(200, np.int64, 0, 10**7), "m2": rand_col(200, np.int64, 0, 10**7),
            "m3": rand_col(200, np.int64, 0, 10**7), "date": rand_col(200, np.int32, 0, 2556)}
    d1 = {"key": np.arange(8, dtype=np.int32), "cat": rand_col(8, np.int16, 0, 3)}
    d2 = {"key": np.arange(10, dtype=np.int64) * 1, "cat": rand_col(10, np.int8, 0, 2)}
    gk, ga, _ = pl.star(fact, d1, d2)
    acc = collections.defaultdict(lambda: [0, 0, 0, 0])
    for i in range(200):
        if fact["date"][i] >= 767:
            continue
        for j1 in range(8):
            for j2 in range(10):
                if fact["fk1"][i] == d1["key"][j1] and fact["fk2"][i] == d2["key"][j2]:
                    a = acc[(int(d1["cat"][j1]), int(d2["cat"][j2]))]
                    a[0] += int(fact["m1"][i]); a[1] += int(fact["m2"][i])
                    a[2] += int(fact["m3"][i]); a[3] += 1
    ks = sorted(acc)
    assert [tuple(c) for c in gk.T.tolist()] == ks
    assert ga.tolist() == [acc[k] for k in ks]
    fact = {"fk": rand_col(300, np.int32, 0, 20), "day": rand_col(300, np.int32, 0, 2556),
            "v": rand_col(300, np.int64, 0, 10**7)}
    dim = {"key": np.arange(15, dtype=np.int32), "grp": rand_col(15, np.int8, 0, 4)}
    gk, ga, _ = pl.batched_one(fact, dim)
    acc = collections.defaultdict(lambda: [0, 0])
    for i in range(300):
        for j in range(15):
            if fact["fk"][i] == dim["key"][j] and fact["day"][i] < 1278:
                acc[int(dim["grp"][j])][0] += int(fact["v"][i]); acc[int(dim["grp"][j])][1] += 1
    ks = sorted(acc)
    assert gk[0].tolist() == ks and ga.tolist() == [acc[k] for k in ks]


# ------------------------------------------------------------------ gather / partition

def test_gather_and_partition():
    col = rand_col(1000, np.int16)
    idx = RNG.integers(0, 1000, 3000).astype(np.int32)
    assert np.array_equal(orc.gather(col, idx), col[idx])
    b = RNG.integers(0, 17, 5000).astype(np.int32)
    rows, off = orc.partition(b, 17)
    assert np.array_equal(rows, np.argsort(b, kind="stable").astype(np.int32))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(b, minlength=17))]))


# ------------------------------------------------------------------ CDF model

def rand_model(H, rng):
    w = rng.uniform(0.5, 8, H)
    b = rng.uniform(-4, 1, H)
    a = rng.uniform(0, 2.0 / H, H)
    return w, b, a, float(rng.uniform(-0.1, 0.1))


def test_cdf_identity_unit_closed_form():
    x = np.linspace(0, 1, 1001, dtype=np.float32)
    F = orc.cdf_forward_f32([1.0], [0.0], [1.0], 0.0, x)
    assert np.array_equal(F, x)                               # F(x) = x on [0, 1]
    F = orc.cdf_forward_f32([2.0, 2.0], [0.0, -1.0], [0.5, 0.5], 0.0, x)
    assert np.array_equal(F, x)                               # two half-ramps also give x
    b = orc.cdf_bucket(F, 8)
    assert np.array_equal(b, np.minimum(7, (x * 8).astype(np.int32)))


def test_cdf_forward_f32_vs_f64_and_monotone():
    rng = np.random.default_rng(3)
    w, b, a, c = rand_model(64, rng)
    x = np.sort(rng.uniform(0, 1, 20000)).astype(np.float32)
    F32 = orc.cdf_forward_f32(w, b, a, c, x)
    F64 = orc.cdf_forward_f64(w.astype(np.float32), b.astype(np.float32),
                              a.astype(np.float32), float(np.float32(c)), x.astype(np.float64))
    # 64 rounded fma steps on values of magnitude <= ~2: error well under 1e-5
    assert np.max(np.abs(F32 - F64)) < 1e-5
    assert np.all(np.diff(F32) >= 0)                          # non-decreasing in x
    bk = orc.cdf_bucket(F32, 4096)
    assert np.all(np.diff(bk) >= 0) and bk.min() >= 0 and bk.max() <= 4095


def test_cdf_normalize_monotone_exact():
    keys = np.sort(rand_col(50000, np.int64))
    u = keys.view(np.uint64) ^ np.uint64(1 << 63)
    umin, umax = int(u.min()), int(u.max())
    span = umax - umin
    shift = max(0, span.bit_length() - 24)
    inv = np.float32(1.0) / np.float32(span >> shift)
    x = orc.cdf_normalize(keys, umin, shift, float(inv))
    assert np.all(np.diff(x) >= 0) and x[0] == 0
    q = ((u - np.uint64(umin)) >> np.uint64(shift)).astype(np.float32)   # exact below 2^24
    assert np.array_equal(x, q * inv)


def test_cdf_grad_finite_differences():
    rng = np.random.default_rng(11)
    H = 16
    w, b, a, c = rand_model(H, rng)
    x = rng.uniform(0, 1, 400)
    y = np.sort(rng.uniform(0, 1, 400))
    loss, gw, gb, ga, gc = orc.cdf_grad_f64(w, b, a, c, x, y)
    z = np.outer(x, w) + b
    kink = np.min(np.minimum(np.abs(z), np.abs(z - 1)))
    h = 1e-7
    assert kink > 10 * h * 10        # no sample sits within the finite-difference step of a kink

    def L(w_, b_, a_, c_):
        return orc.cdf_grad_f64(w_, b_, a_, c_, x, y)[0]

    for name, vec, g in (("w", w, gw), ("b", b, gb), ("a", a, ga)):
        for j in range(H):
            p, m = vec.copy(), vec.copy()
            p[j] += h; m[j] -= h
            args_p = {"w": (p, b, a), "b": (w, p, a), "a": (w, b, p)}[name]
            args_m = {"w": (m, b, a), "b": (w, m, a), "a": (w, b, m)}[name]
            fd = (L(*args_p, c) - L(*args_m, c)) / (2 * h)
            assert abs(fd - g[j]) <= 1e-6 * max(1e-3, abs(g[j])) + 1e-9, (name, j, fd, g[j])
    fd = (L(w, b, a, c + h) - L(w, b, a, c - h)) / (2 * h)
    assert abs(fd - gc) <= 1e-6 * abs(gc) + 1e-9
    # the loss itself against its definition through the float64 forward
    F = orc.cdf_forward_f64(w, b, a, c, x)
    assert abs(loss - np.mean((F - y) ** 2)) < 1e-12


def test_adam_first_step_closed_form():
    # at t = 1 the bias-corrected moments are g and g^2: step = lr * g / (|g| + eps)
    p = np.array([0.5, 0.5, 0.01, 2.0])
    g = np.array([0.3, -2.0, 1.0, 1e-9])
    m, v = np.zeros(4), np.zeros(4)
    orc.adam_step_f64(p, g, m, v, [0, 0, 1, 0], 1, lr=0.1)
    want = np.array([0.5 - 0.1 * 0.3 / (0.3 + 1e-8), 0.5 + 0.1 * 2.0 / (2.0 + 1e-8), 0.0,
                     2.0 - 0.1 * 1e-9 / (1e-9 + 1e-8)])
    assert np.allclose(p, want, rtol=1e-12, atol=1e-15)      # entry 2 projected onto >= 0


def test_cdf_targets_closed_form():
    y = orc.cdf_targets(np.array([1, 1, 2, 3, 3, 3], dtype=np.int64))
    assert y.tolist() == [1 / 6, 1 / 6, 2.5 / 6, 4.5 / 6, 4.5 / 6, 4.5 / 6]
    assert orc.cdf_targets(np.array([5], np.int64)).tolist() == [0.5]


# ------------------------------------------------------------------ generator

def test_generator_slices_and_bijections():
    rec = dg.q6_lineitem()["price"]
    full = dg.generate(rec, 1000)
    assert np.array_equal(dg.generate(rec, 300, start=700), full[700:])
    p = dg.perm(np.arange(1000, dtype=np.uint64), 1000, 12345)
    assert np.array_equal(np.sort(p), np.arange(1000))
    x = np.arange(1 << 16, dtype=np.uint32)
    assert len(np.unique(dg.fmix32(x))) == 1 << 16
    assert len(np.unique(dg.mix64(x.astype(np.uint64)))) == 1 << 16
    # SplitMix64 from state 0: first outputs of the published generator
    assert int(dg.draw(0, np.array([0], np.uint64))[0]) == 0xE220A8397B1DCDAF
    assert int(dg.draw(0, np.array([1], np.uint64))[0]) == 0x6E789E6AA1B965F4


def test_zipf_top_rank_frequency():
    z = dg.zipf_table(1.0, 1000)
    u = dg.draw(99, np.arange(400_000, dtype=np.uint64))
    r = dg.zipf_rank(u, z)
    H = np.sum(1.0 / np.arange(1, 1001))
    p0 = 1 / H
    sd = (400_000 * p0 * (1 - p0)) ** 0.5
    assert abs(np.sum(r == 0) - 400_000 * p0) < 6 * sd
    assert r.max() <= 999


# ---------------------------------------------------------------- strings
def _pad(values, m):
    """Section 2.1's string tensor: each UTF-8 value right-padded with zeros to m bytes."""
    out = np.zeros((len(values), m), np.uint8)
    for i, v in enumerate(values):
        b = v.encode("utf-8")
        out[i, :len(b)] = np.frombuffer(b, np.uint8)
    return out


def test_like_prefix_worked_example():
    vals = ["", "a", "ab", "abc", "abd", "b", "abcabc", "abé", "été"]
    s = _pad(vals, 7)
    assert orc.like_prefix(s, b"ab").tolist() == [0, 0, 1, 1, 1, 0, 1, 1, 0]
    assert orc.like_prefix(s, b"").tolist() == [1] * len(vals)            # LIKE '%'
    assert orc.like_prefix(s, b"abcabc").tolist() == [0, 0, 0, 0, 0, 0, 1, 0, 0]
    assert orc.like_prefix(s, b"abcabcx").tolist() == [0] * len(vals)     # longer than every value
    assert orc.like_prefix(s, b"abcabcxy").tolist() == [0] * len(vals)    # longer than the width
    e = "é".encode("utf-8")                                         # two bytes
    assert orc.like_prefix(s, e).tolist() == [0, 0, 0, 0, 0, 0, 0, 0, 1]
    assert orc.like_prefix(s, e[:1]).tolist() == [0, 0, 0, 0, 0, 0, 0, 0, 1]  # a byte prefix


@pytest.mark.parametrize("m", [1, 3, 25])
def test_like_prefix_brute_force(m):
    r = np.random.default_rng(m)
    alphabet = "ABCé"
    vals = []
    for _ in range(3000):
        v = "".join(alphabet[j] for j in r.integers(0, len(alphabet), r.integers(0, m + 1)))
        while len(v.encode("utf-8")) > m:
            v = v[:-1]
        vals.append(v)
    s = _pad(vals, m)
    for k in range(0, m + 2):
        for _ in range(3):
            p = "".join(alphabet[j] for j in r.integers(0, 3, k)).encode("utf-8")[:k]
            want = [1 if v.encode("utf-8").startswith(p) and len(p) <= m else 0 for v in vals]
            assert orc.like_prefix(s, p).tolist() == want, (m, p)


@pytest.mark.parametrize("m", [1, 9, 25])
def test_string_codes_brute_force(m):
    r = np.random.default_rng(40 + m)
    vals = ["", "a", "ab", "b", "é", "aé", "ba"] + ["".join("ab"[j] for j in r.integers(0, 2, r.integers(0, 4)))
                                                  for _ in range(500)]
    vals = [v for v in vals if len(v.encode("utf-8")) <= m]
    s = _pad(vals, m)
    code, k = orc.string_codes(s)
    distinct = sorted(set(v.encode("utf-8") for v in vals))   # bytes order: a prefix sorts first
    assert k == len(distinct)
    assert code.tolist() == [distinct.index(v.encode("utf-8")) for v in vals]


def test_string_codes_worked_example():
    s = _pad(["b", "a", "ab", "a", "", "b"], 3)
    code, k = orc.string_codes(s)
    assert k == 4 and code.tolist() == [3, 1, 2, 1, 0, 3]


def test_cdf_normalize_hand_worked_example():
    """Key normalisation worked by hand (the reading: a 24-bit shifted
    integer times a float reciprocal).  Keys -2^63, -2^63 + 2^40, 0, 2^63 - 1
    have order-preserving images 0, 2^40, 2^63, 2^64 - 1; with umin = 0 and
    shift 40 their q are 0, 1, 2^23, 2^24 - 1.
    - With inv = 2^-24 (a power of two) every product is exact: 0, 2^-24,
      1/2 and 1 - 2^-24.
    - With inv = float(1/3) = 0x3EAAAAAB (= 1/3 + 2^-25/3), q = 3 gives
      3 * inv = 1 + 2^-25, which rounds to 1.0 (the nearest floats are 1 and
      1 + 2^-23); q = 1 gives inv itself."""
    keys = np.array([-2**63, -2**63 + 2**40, 0, 2**63 - 1], np.int64)
    x = orc.cdf_normalize(keys, 0, 40, 2.0**-24)
    assert x.tolist() == [0.0, 2.0**-24, 0.5, 1.0 - 2.0**-24]
    third = np.frombuffer(np.array([0x3EAAAAAB], np.uint32).tobytes(), np.float32)[0]
    keys = np.array([-2**63, -2**63 + 2**40, -2**63 + 3 * 2**40], np.int64)
    x = orc.cdf_normalize(keys, 0, 40, float(third))
    assert x[0] == 0.0 and x[1] == third and x[2] == np.float32(1.0)


def test_light_cdf_targets_worked_example():
    """Sample 1, 2, 2, 2, 2, 3, 4, 4 with runs of 1, 4, 1, 2 keys; counts
    from 2 on may be heavy, at most 4 heavy keys: keys 2 and 4 are heavy, the
    light keys are 1 and 3 (total 2).  Key 1 sits at (0 + 1/2) / 2, each
    heavy key 2 at 1 / 2 (one light key before it, zero width), key 3 at
    (1 + 1/2) / 2, heavy key 4 at 2 / 2.  With at most one heavy key only
    the run of 4 qualifies; with none, the plain midpoints (first rank +
    count / 2) / 8."""
    s = np.array([1, 2, 2, 2, 2, 3, 4, 4], np.uint64)
    y, h = orc.light_cdf_targets(s, 1, 8, 2, 4)
    assert y.tolist() == [0.25, 0.5, 0.5, 0.5, 0.5, 0.75, 1.0, 1.0] and h.tolist() == [2, 4]
    y, h = orc.light_cdf_targets(s, 1, 8, 2, 1)
    assert h.tolist() == [2]
    assert y.tolist() == [0.125, 0.25, 0.25, 0.25, 0.25, 0.375, 0.75, 0.75]
    y, h = orc.light_cdf_targets(s, 2, 4, 2, 0)
    assert h.tolist() == [] and y.tolist() == [1 / 16, 3 / 8, 3 / 8, 14 / 16]


@pytest.mark.parametrize("seed", range(6))
def test_light_cdf_targets_brute_force(seed):
    """Random samples against a direct statement: heavy keys by counting
    (the largest counts first, while at most max_heavy keys have reached
    them), y = (light keys strictly below k + half the light copies of k) /
    the light total; and without heavy keys the plain targets."""
    r = np.random.default_rng(seed)
    SH = int(r.integers(1, 3000))
    s = np.sort(r.integers(0, int(r.integers(1, 400)), SH).astype(np.uint64))
    mult = int(r.integers(1, 4))
    S_train = (SH - 1) // mult + 1
    min_count, max_heavy = int(r.integers(1, 20)), int(r.integers(0, 12))
    y, h = orc.light_cdf_targets(s, mult, S_train, min_count, max_heavy)
    cnt = collections.Counter(s.tolist())
    cut = None
    for c in sorted(set(cnt.values()), reverse=True):
        if c < min_count or max_heavy == 0 or sum(1 for v in cnt.values() if v >= c) > max_heavy:
            break
        cut = c
    heavy = sorted(k for k, v in cnt.items() if cut is not None and v >= cut)
    assert h.tolist() == heavy
    light = {k: (0 if k in heavy else v) for k, v in cnt.items()}
    total = sum(light.values()) or 1
    for t in range(S_train):
        k = int(s[t * mult])
        below = sum(v for kk, v in light.items() if kk < k)
        assert y[t] == np.float32((below + 0.5 * light[k]) / total)
    y0, h0 = orc.light_cdf_targets(s, 1, SH, min_count, 0)
    assert h0.size == 0 and np.array_equal(y0, orc.cdf_targets(s.astype(np.int64)).astype(np.float32))


def _iso(dates, m=12):
    out = np.zeros((len(dates), m), np.uint8)
    for i, t in enumerate(dates):
        b = t.encode()
        out[i, :len(b)] = np.frombuffer(b, np.uint8)
    return out


def test_date_conversions_against_datetime():
    """ISO strings and day numbers to epoch nanoseconds, and back to the
    calendar, against Python's datetime (the proleptic Gregorian calendar),
    over every day of 1600..2300 that an int64 nanosecond count reaches and
    random instants (negative ones included, not on day boundaries)."""
    import datetime as dt
    epoch = dt.date(1970, 1, 1)
    first, last = dt.date(1677, 9, 22), dt.date(2262, 4, 11)
    ns_day = 86400 * 10**9
    assert (first - epoch).days * ns_day >= -2**63 and ((first - epoch).days - 1) * ns_day < -2**63
    assert (last - epoch).days * ns_day < 2**63 and ((last - epoch).days + 1) * ns_day >= 2**63
    d = dt.date(1600, 1, 1)
    dates, want = [], []
    while d <= dt.date(2300, 12, 31):
        dates.append(d.isoformat())
        want.append((d - epoch).days * ns_day if first <= d <= last else -2**63)
        d += dt.timedelta(days=1)
    ns, ok = orc.date_parse_iso(_iso(dates))
    assert ns.tolist() == want and ok.tolist() == [int(w != -2**63) for w in want]
    days = np.array([(dt.date.fromisoformat(t) - epoch).days for t in dates], np.int64)
    inr = (days >= -106751) & (days <= 106751)
    assert orc.date_from_days(days.astype(np.int32)).tolist() == np.where(inr, days * ns_day, -2**63).tolist()
    r = np.random.default_rng(3)
    t = np.concatenate([r.integers(-2**63, 2**63 - 1, 20000, dtype=np.int64), [0, -1, 1, ns_day, -ns_day,
                        -ns_day - 1, -2**63, 2**63 - 1]]).astype(np.int64)
    dn, y, mo, md = orc.date_parts(t)
    for i in range(len(t)):
        q = int(t[i]) // ns_day          # Python floors
        c = epoch + dt.timedelta(days=q)
        assert (dn[i], y[i], mo[i], md[i]) == (q, c.year, c.month, c.day)


def test_date_parse_rejects_malformed():
    bad = ["1900-02-29", "2023-13-01", "2023-00-10", "2023-04-31", "2023-04-00", "1970/01/01", "1970-1-01",
           "19700101", "", "1677-09-21", "2262-04-12", "abcd-ef-gh"]
    ns, ok = orc.date_parse_iso(_iso(bad))
    assert ok.tolist() == [0] * len(bad) and ns.tolist() == [-2**63] * len(bad)
    trailing = _iso(["1970-01-02"])
    trailing[0, 10] = ord("T")                # a byte after the date that is not padding
    assert orc.date_parse_iso(trailing)[1].tolist() == [0]
    assert orc.date_parse_iso(_iso(["2000-02-29"], 10))[0].tolist() == [11016 * 86400 * 10**9]
