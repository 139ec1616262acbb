"""Exact parity of the kernel variants that only large inputs reach, against
the oracle, group by group:

- the star probe whose first dimension is too large for its cell bitmap to
  live in shared memory (more than 4M passing rows), in the int32-key form
  (every dimension key int32) and the mixed int32/int64 form, with one and
  with two dimensions, wide cells (sparse keys) and unit cells (dense keys),
  through the radix and the learned dimension sorts;
- the group-by whose value columns are gathered into sorted order before
  the reduce (from 2^22 rows on), through the plain radix path and the
  learned partitioner (light rows above 2^22 too).

The full-size benchmark workloads run exactly these variants; here they run
at sizes the oracle finishes in seconds."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import pipelines as pl
from paper_2209_04579_b300 import datagen as dg

pytestmark = pytest.mark.gpu

PREGATHER_ROWS = 1 << 22
SMEM_BITMAP_DIM_ROWS = 4_000_000


@pytest.fixture(scope="module")
def G():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import datagen_device, queries, tqp
    return tqp, queries, datagen_device


def cu(t):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in t.items()}


def host(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def compare(got, want):
    ok, oa, g = got
    wk, wa, of = want
    assert not of
    Gn = wa.shape[0]
    assert int(g.item()) == Gn
    for i in range(len(ok)):
        assert np.array_equal(host(ok[i], Gn).astype(np.int64), wk[i])
    assert np.array_equal(host(oa)[:Gn], wa)


def unique_keys(m, dtype, seed):
    """m distinct keys spread over the dtype's range: an odd multiplier is a
    bijection modulo 2^bits, so distinct indices give distinct keys."""
    bits = np.dtype(dtype).itemsize * 8
    i = np.arange(m, dtype=np.uint64)
    mult = np.uint64(0x9E3779B1) if bits == 32 else np.uint64(0x9E3779B97F4A7C15)
    u = i * mult + np.uint64(seed)
    if bits == 32:
        return (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    return u.view(np.int64)


def star_case(n1, n2, n, dt2, seed):
    r = np.random.default_rng(seed)
    k1 = unique_keys(n1, np.int32, seed)[r.permutation(n1)]
    k2 = unique_keys(n2, dt2, seed + 1)[r.permutation(n2)]
    dim1 = {"key": k1, "cat": r.integers(0, 1000, n1).astype(np.int16)}
    dim2 = {"key": k2, "cat": r.integers(0, 50, n2).astype(np.int8)}
    # foreign keys drawn from the dimension keys, plus a few that miss
    fk1 = k1[r.integers(0, n1, n)]
    fk1[::997] = fk1[::997] + 1
    fk2 = k2[r.integers(0, n2, n)]
    fk2[::1009] = fk2[::1009] ^ 1
    fact = {"fk1": fk1, "fk2": fk2.astype(dt2), "date": r.integers(0, 2557, n).astype(np.int32)}
    for c in ("m1", "m2", "m3"):
        fact[c] = r.integers(0, 10**7, n).astype(np.int64)
    return fact, dim1, dim2


@pytest.mark.parametrize("dt2", [np.int64, np.int32])
@pytest.mark.parametrize("learned", [False, True])
def test_star_first_dimension_beyond_shared_bitmap(G, dt2, learned):
    """Two dimensions, the first with 4.2M keys: the probe variant whose
    first cell bitmap stays in global memory (the full star join's probe).
    int64 second keys give the mixed form, int32 the all-int32 form."""
    tqp, Q, _ = G
    n1, n2, n = 4_200_000, 1_500_000, 3_000_000
    assert n1 > SMEM_BITMAP_DIM_ROWS
    fact, dim1, dim2 = star_case(n1, n2, n, dt2, 31 + (dt2 == np.int32))
    want = pl.star(fact, dim1, dim2)
    cfg = tqp.learned_cfg(sample=16384, tcfg=tqp.train_cfg(epochs=5, lr=1e-4)) if learned else None
    compare(Q.star(cu(fact), cu(dim1), cu(dim2), learned=cfg), want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_star_full_size_dimensions_scaled_fact(G):
    """The full star join's dimensions (20M and 150M rows, the benchmark's
    generator) with 4M fact rows: every dimension variant of the benchmark
    (wide cells over 20M int32 and 150M int64 keys, the learned dimension
    sort) compared group by group."""
    tqp, Q, gd = G
    n1, n2, n = 20_000_000, 150_000_000, 4_000_000
    rec = dg.star_tables(n1, n2)
    fact_h = dg.make_table(rec["fact"], n)
    d1h = dg.make_table(rec["dim1"], n1)
    d2h = dg.make_table(rec["dim2"], n2)
    want = pl.star(fact_h, d1h, d2h)
    del d1h, d2h
    fact = gd.make_table(rec["fact"], n)
    d1, d2 = gd.make_table(rec["dim1"], n1), gd.make_table(rec["dim2"], n2)
    compare(Q.star(fact, d1, d2), want)
    compare(Q.star(fact, d1, d2, learned=tqp.learned_cfg(sample=65536, tcfg=tqp.train_cfg(epochs=10, lr=1e-4))),
            want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("kind", ["sparse32", "dense32", "sparse64"])
def test_one_dimension_beyond_shared_bitmap(G, kind):
    """One filtered dimension of 4.5M rows (the Q14 shape): int32 keys
    spread over their range (wide cells), int32 keys dense in their range
    (unit cells filled without the sort), and int64 keys."""
    tqp, Q, _ = G
    m, n = 4_500_000, 3_000_000
    r = np.random.default_rng(5 + len(kind))
    if kind == "dense32":
        key = (-1_000_000 + r.permutation(m)).astype(np.int32)
    else:
        key = unique_keys(m, np.int32 if kind == "sparse32" else np.int64, 77)[r.permutation(m)]
    dim = {"key": key, "region": r.integers(0, 25, m).astype(np.int8),
           "price": r.integers(100, 10**6, m).astype(np.int64)}
    fk = key[r.integers(0, m, n)]
    fk[::501] = fk[::501] + 3
    fact = {"fk": fk}
    want = pl.q14(fact, dim)
    compare(Q.q14(cu(fact), cu(dim)), want)
    compare(Q.q14(cu(fact), cu(dim), learned=tqp.learned_cfg(sample=16384, tcfg=tqp.train_cfg(epochs=5, lr=1e-4))),
            want)
    assert tqp.tqp_status_poll() == tqp.OK


EXPRS = [[(0, 1, 0)], [(1, 1, 0)], [(0, 1, 0), (1, -1, 100)]]
AGGS = [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 1), (orc.MAX, 0), (orc.SUM, 2)]


def test_groupby_pregather_branch(G):
    """4.3M rows (above 2^22), a packed key of about 17 bits (the sort path,
    not the small-domain slots), two value columns and a product: the values
    are gathered into sorted order before the reduce."""
    tqp, _, _ = G
    r = np.random.default_rng(22)
    n = 4_300_003
    assert n >= PREGATHER_ROWS
    k1 = r.integers(-40_000, 40_000, n).astype(np.int32)
    k2 = r.integers(0, 2, n).astype(np.int8)
    v0 = r.integers(-10**9, 10**9, n).astype(np.int64)
    v1 = r.integers(0, 100, n).astype(np.int16)
    want = orc.groupby_agg([k1, k2], [v0, v1], EXPRS, AGGS)
    c = lambda a: torch.from_numpy(a).cuda()
    got = tqp.tqp_groupby_agg([c(k1), c(k2)], [c(v0), c(v1)], EXPRS, AGGS, want[1].shape[0])
    compare(got, want)
    # a selection of about 4.25M of 4.4M rows
    sel = np.flatnonzero(r.random(n) < 0.99).astype(np.int32)
    want = orc.groupby_agg([k1, k2], [v0, v1], EXPRS, AGGS, sel=sel)
    got = tqp.tqp_groupby_agg([c(k1), c(k2)], [c(v0), c(v1)], EXPRS, AGGS, want[1].shape[0], sel=c(sel))
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("heavy,n", [(True, 6_500_000), (False, 4_500_000)])
def test_learned_groupby_pregather_branch(G, heavy, n):
    """The skewed keys (more than 2^22 light rows: at 6.5M rows about a
    quarter of the rows belong to the directly aggregated heavy keys) with
    two value columns and a product, through the learned partitioner: its
    light rows' values are gathered into sorted order before the reduce that
    merges the heavy keys.  The largest skewed case the oracle checks row by
    row (its std::map takes about a minute per 10M rows)."""
    tqp, _, gd = G
    z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
    rec = dg.skew_groupby()
    t = dg.make_table(rec, n, zipf=z)
    r = np.random.default_rng(9)
    v1 = r.integers(0, 100, n).astype(np.int16)
    want = orc.groupby_agg([t["key"]], [t["value"], v1], EXPRS, AGGS)
    dev = gd.make_table(rec, n, zipf=torch.from_numpy(z).cuda())
    cfg = tqp.learned_cfg(sample=65536, heavy=heavy, tcfg=tqp.train_cfg(epochs=20, lr=1e-4))
    got = tqp.tqp_groupby_agg_learned([dev["key"]], [dev["value"], torch.from_numpy(v1).cuda()], EXPRS, AGGS,
                                      want[1].shape[0], cfg=cfg)
    compare(got[:3], want)
    st = tqp.stats_from_device(got[4])
    assert st["light_rows"] >= PREGATHER_ROWS
    assert (st["heavy_keys"] > 0) == heavy
    assert tqp.tqp_status_poll() == tqp.OK
