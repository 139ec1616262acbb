"""GPU parity of the workload queries against the oracle's pipelines, and of
the device input generator against the host generator.

Inputs: the GPU side generates its tables on the device, the oracle side on
the host, from the same seeded recipes (the generator test below shows the
two are identical).  Full-size cases run in the same launch configuration as
the benchmark."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import pipelines as pl
from paper_2209_04579_b300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import datagen_device, queries, tqp
    return tqp, queries, datagen_device


def host(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def all_recipes():
    out = list(dg.q6_lineitem().items())
    for sparse in (False, True):
        t = dg.q14_tables(1_500_000, sparse)
        out += [(f"q14{sparse}.{k}", r) for tab in t.values() for k, r in tab.items()]
    out += list(dg.skew_groupby().items())
    ns, ms, gs = dg.batched_sizes()
    t = dg.batched_problem(7, int(ns[7]), int(ms[7]), int(gs[7]))
    out += [(f"b.{k}", r) for tab in t.values() for k, r in tab.items()]
    t = dg.star_tables()
    out += [(f"s.{k}", r) for tab in t.values() for k, r in tab.items()]
    return out


def test_device_generator_matches_host(G):
    _, _, gd = G
    z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
    zd = torch.from_numpy(z).cuda()
    for name, rec in all_recipes():
        far = 123_456_789 if rec.kind != dg.PERM_KEY else rec.m - 5_003   # a permutation is defined on [0, m)
        for start, n in ((0, 100_000), (far, 5_003)):
            want = dg.generate(rec, n, start, zipf=z)
            got = host(gd.generate(rec, n, start, zipf=zd))
            assert np.array_equal(got, want), (name, start)


def compare(got, want):
    ok, oa, g = got
    wk, wa, of = want
    assert not of
    Gn = wa.shape[0]
    assert int(g.item()) == Gn
    for i in range(len(ok)):
        assert np.array_equal(host(ok[i], Gn).astype(np.int64), wk[i])
    assert np.array_equal(host(oa)[:Gn], wa)


@pytest.mark.parametrize("n", [1, 4097, 1_000_000])
def test_q6(G, n):
    tqp, Q, gd = G
    rec = dg.q6_lineitem()
    want = pl.q6(dg.make_table(rec, n))
    compare(Q.q6(gd.make_table(rec, n)), want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("sparse", [False, True])
@pytest.mark.parametrize("n,m", [(1, 1), (100_000, 2_000), (2_000_003, 50_000)])
def test_q14_fused_and_unfused(G, sparse, n, m):
    tqp, Q, gd = G
    rec = dg.q14_tables(m, sparse)
    want = pl.q14(dg.make_table(rec["fact"], n), dg.make_table(rec["dim"], m))
    fact, dim = gd.make_table(rec["fact"], n), gd.make_table(rec["dim"], m)
    compare(Q.q14(fact, dim), want)
    compare(Q.q14_unfused(fact, dim), want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_q14_full_size(G):
    """Fact 60M x dim 1.5M, the benchmark's workload and launch configuration."""
    tqp, Q, gd = G
    rec = dg.q14_tables(1_500_000)
    want = pl.q14(dg.make_table(rec["fact"], 60_000_000), dg.make_table(rec["dim"], 1_500_000))
    got = Q.q14(gd.make_table(rec["fact"], 60_000_000), gd.make_table(rec["dim"], 1_500_000))
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("n", [10_000, 2_000_000])
def test_skew_groupby(G, n):
    tqp, Q, gd = G
    z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
    rec = dg.skew_groupby()
    want = pl.skew(dg.make_table(rec, n, zipf=z))
    got = Q.skew(gd.make_table(rec, n, zipf=torch.from_numpy(z).cuda()), cap=n)
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_batched_instances_small(G):
    tqp, Q, gd = G
    ns, ms, gs = dg.batched_sizes()
    for p in range(0, 512, 37):
        n, m, g = int(ns[p]), int(ms[p]), int(gs[p])
        rec = dg.batched_problem(p, n, m, g)
        want = pl.batched_one(dg.make_table(rec["fact"], n), dg.make_table(rec["dim"], m))
        compare(Q.batched_one(gd.make_table(rec["fact"], n), gd.make_table(rec["dim"], m)), want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_star_scaled(G):
    """Star join at 1/100 of the fact rows, dimension sizes scaled alike."""
    tqp, Q, gd = G
    rec = dg.star_tables(200_000, 1_500_000)
    n = 6_000_000
    want = pl.star(dg.make_table(rec["fact"], n), dg.make_table(rec["dim1"], 200_000),
                   dg.make_table(rec["dim2"], 1_500_000))
    got = Q.star(gd.make_table(rec["fact"], n), gd.make_table(rec["dim1"], 200_000),
                 gd.make_table(rec["dim2"], 1_500_000))
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_star_scaled_learned_dimension_sort(G):
    """The scaled star join with the dimensions' keys sorted through the
    learned range partitioner (tqp_star_agg_learned): dim2 (1.5M keys) takes
    the learned sort, dim1 (200K) the radix sort; the same groups."""
    tqp, Q, gd = G
    rec = dg.star_tables(200_000, 1_500_000)
    n = 6_000_000
    want = pl.star(dg.make_table(rec["fact"], n), dg.make_table(rec["dim1"], 200_000),
                   dg.make_table(rec["dim2"], 1_500_000))
    got = Q.star(gd.make_table(rec["fact"], n), gd.make_table(rec["dim1"], 200_000),
                 gd.make_table(rec["dim2"], 1_500_000), learned=tqp.learned_cfg(sample=16384, tcfg=tqp.train_cfg(epochs=10, lr=1e-4)))
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_star_learned_both_dimensions(G):
    """Both dimensions above the learned sort's threshold (1.2M and 2M keys,
    untrained identity network and a fixed bucket count included)."""
    tqp, Q, gd = G
    rec = dg.star_tables(1_200_000, 2_000_000)
    n = 3_000_000
    want = pl.star(dg.make_table(rec["fact"], n), dg.make_table(rec["dim1"], 1_200_000),
                   dg.make_table(rec["dim2"], 2_000_000))
    for cfg in (tqp.learned_cfg(sample=8192, tcfg=tqp.train_cfg(epochs=5, lr=1e-4)),
                tqp.learned_cfg(sample=4096, buckets=1024, train=False)):
        got = Q.star(gd.make_table(rec["fact"], n), gd.make_table(rec["dim1"], 1_200_000),
                     gd.make_table(rec["dim2"], 2_000_000), learned=cfg)
        compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_q14_learned_filtered_dimension(G):
    """The Q14 shape at 3M fact rows with a 1.5M-row dimension whose passing
    rows (region < 5) are sorted through the learned partitioner, their row
    ids carried as the payload."""
    tqp, Q, gd = G
    rec = dg.q14_tables(1_500_000)
    n = 3_000_000
    want = pl.q14(dg.make_table(rec["fact"], n), dg.make_table(rec["dim"], 1_500_000))
    got = Q.q14(gd.make_table(rec["fact"], n), gd.make_table(rec["dim"], 1_500_000),
                learned=tqp.learned_cfg(sample=16384, tcfg=tqp.train_cfg(epochs=5, lr=1e-4)))
    compare(got, want)
    assert tqp.tqp_status_poll() == tqp.OK


def test_star_crowded_directory_cells(G):
    """Dimension keys clustered in a tiny part of their range (plus far
    outliers), so one directory cell holds hundreds of keys: the in-cell
    bound search must find every one."""
    tqp, Q, gd = G
    r = np.random.default_rng(12)
    key = np.concatenate([np.arange(-500, 500), [2**30, -2**30, 2**31 - 1]]).astype(np.int32)
    key = key[r.permutation(len(key))]
    m = len(key)
    dim = {"key": key, "region": r.integers(0, 25, m).astype(np.int8),
           "price": r.integers(100, 10**6, m).astype(np.int64)}
    fk = r.choice(np.concatenate([key, np.arange(600, 700, dtype=np.int32)]), 500_000).astype(np.int32)
    fact = {"fk": fk}
    want = pl.q14(fact, dim)
    cu = lambda t: {k: torch.from_numpy(v).cuda() for k, v in t.items()}
    compare(Q.q14(cu(fact), cu(dim)), want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("stride", [1, 3, 1000])
def test_q14_dense_and_spread_dimension_keys(G, stride):
    """Dimension keys key0 + stride * permutation, five in six passing the
    region predicate: with stride 1 and 3 the passing keys are dense (span
    within 8x their count), so the directory cells are filled straight from
    the rows without a key sort; stride 1000 takes the sorted form.  Foreign
    keys also fall between and beyond the dimension keys."""
    tqp, Q, gd = G
    r = np.random.default_rng(40 + stride)
    m = 300_000
    key = (-123_456 + stride * r.permutation(m)).astype(np.int32)
    dim = {"key": key, "region": r.integers(0, 6, m).astype(np.int8),
           "price": r.integers(100, 10**6, m).astype(np.int64)}
    fk = np.concatenate([r.choice(key, 900_000), r.integers(-200_000, 200_000 + stride * m, 100_000)]).astype(np.int32)
    fact = {"fk": fk[r.permutation(len(fk))]}
    want = pl.q14(fact, dim)
    cu = lambda t: {k: torch.from_numpy(v).cuda() for k, v in t.items()}
    compare(Q.q14(cu(fact), cu(dim)), want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("passing", [0, 1, 2])
def test_q14_few_passing_dimension_rows(G, passing):
    """No, one or two dimension rows pass the region predicate (an empty
    directory, a single cell, two far-apart cells)."""
    tqp, Q, gd = G
    r = np.random.default_rng(90 + passing)
    m = 20_000
    key = (5 + r.permutation(m)).astype(np.int32)
    region = np.full(m, 9, np.int8)
    region[:passing] = [1, 3][:passing]
    if passing == 2:
        key[:2] = [-(2**31), 2**31 - 1]
    dim = {"key": key, "region": region, "price": r.integers(100, 10**6, m).astype(np.int64)}
    fk = np.concatenate([r.choice(key, 200_000), key[:passing].repeat(7)]).astype(np.int32)
    fact = {"fk": fk}
    want = pl.q14(fact, dim)
    cu = lambda t: {k: torch.from_numpy(v).cuda() for k, v in t.items()}
    compare(Q.q14(cu(fact), cu(dim)), want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("stride", [1, 1000])
def test_q14_repeated_dimension_key_is_unsupported(G, stride):
    """A repeated key among the passing dimension rows is reported as
    unsupported, in the dense (direct) and the sorted form alike."""
    tqp, Q, gd = G
    r = np.random.default_rng(7)
    m = 50_000
    key = (stride * r.permutation(m)).astype(np.int32)
    key[17] = key[4242]
    dim = {"key": key, "region": np.zeros(m, np.int8), "price": np.ones(m, np.int64)}
    fact = {"fk": r.choice(key, 100_000).astype(np.int32)}
    cu = lambda t: {k: torch.from_numpy(v).cuda() for k, v in t.items()}
    Q.q14(cu(fact), cu(dim))
    assert tqp.tqp_status_poll() == tqp.ERR_UNSUPPORTED


@pytest.mark.parametrize("n,m", [(1, 10), (100_000, 5_000), (6_000_000, 1_500_000)])
def test_q14_promo(G, n, m):
    """The promotion-revenue shape of Q14: LIKE over the dimension's
    zero-padded string tensor, its 0/1 column as the CASE factor of one
    aggregate, and a one-month range on the epoch-nanosecond ship column."""
    tqp, Q, gd = G
    rec = dg.q14_promo_tables(m)
    table, words = dg.type_strings()
    d0 = (dg.EPOCH_DAY0 + 1300) * dg.SECONDS_PER_DAY * 10**9
    d1 = d0 + 30 * dg.SECONDS_PER_DAY * 10**9
    fact_h = dg.make_table(rec["fact"], n)
    dim_h = dg.make_table(rec["dim"], m)
    dim_h["type"] = dg.type_column(m, rec["type_seed"], table)
    fact = gd.make_table(rec["fact"], n)
    dim = gd.make_table(rec["dim"], m)
    dim["type"] = torch.from_numpy(dim_h["type"]).cuda()
    for prefix, lo, hi in [(words[0][0], d0, d1), (words[0][2][:2], d0, d1), (b"", d0, d1 + 400 * 86_400 * 10**9),
                           (b"Q" * 26, d0, d1)]:
        want = pl.q14_promo(fact_h, dim_h, prefix, lo, hi)
        keys, aggs, g = Q.q14_promo(fact, dim, prefix, lo, hi)
        G_ = want[1].shape[0]
        assert int(g.item()) == G_
        assert np.array_equal(host(aggs)[:G_], want[1])
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("n", [1, 100_003, 10_000_000])
def test_predict_query(G, n):
    """The prediction query: the network's output over a float column,
    thresholded at one half, counted per rating among the filtered rows."""
    tqp, Q, gd = G
    rec = dg.reviews_table()
    host_t = dg.make_table(rec, n)
    host_t["score"] = (host_t["score_q"].astype(np.float64) / 2**dg.SCORE_BITS).astype(np.float32)
    t = gd.make_table(rec, n)
    t["score"] = t["score_q"].to(torch.float32) / 2**dg.SCORE_BITS
    assert np.array_equal(host(t["score"]), host_t["score"])
    w, b, a, c = dg.predict_model()
    model = tqp.model_to_device(w, b, a, c)
    for votes in (0, 5, 51):
        compare(Q.predict(t, model, votes), pl.predict(host_t, (w, b, a, c), votes))
    assert tqp.tqp_status_poll() == tqp.OK


# group columns of the two dimensions: dtype and the span of their values.
# Spans below 2^24 rank through the value-domain bitmap, wider ones through
# the sort of the packed group keys; both paths meet at the 2^24 boundary.
GROUP_DOMAINS = [
    ((np.int16, -300, 300), (np.int8, -128, 127)),
    ((np.int8, 7, 7), (np.int16, -32768, 32767)),
    ((np.int32, 5, 5 + 2**24 - 1), (np.int32, -(2**24), -1)),
    ((np.int32, -(2**31), 2**31 - 1), (np.int64, -(2**40), 2**40)),
    ((np.int64, 2**62, 2**62 + 2**23), (np.int32, 0, 2**24)),
]


@pytest.mark.parametrize("case", range(len(GROUP_DOMAINS)))
def test_star_group_value_domains(G, case):
    """Star join whose group columns take 40 (or fewer) distinct values
    spread over spans from one value to the full 64-bit range, including
    both ends of each span."""
    tqp, Q, gd = G
    g1, g2 = GROUP_DOMAINS[case]
    r = np.random.default_rng(700 + case)

    def column(spec, m):
        dt, lo, hi = spec
        vals = np.unique(np.concatenate([[lo, hi], r.integers(lo, hi, 38, endpoint=True)])).astype(dt)
        col = vals[r.integers(0, len(vals), m)]
        col[:len(vals)] = vals  # every value present
        return col[r.permutation(m)]

    n1, n2, n = 2_000, 3_000, 400_000
    k1 = r.permutation(np.arange(-10**6, 10**6, dtype=np.int32))[:n1]
    k2 = r.permutation(np.arange(0, 5 * 10**6, dtype=np.int64))[:n2] * 1_000_003 - 2**40
    dim1 = {"key": k1, "cat": column(g1, n1)}
    dim2 = {"key": k2, "cat": column(g2, n2)}
    fk1 = r.choice(np.concatenate([k1, np.arange(2 * 10**6, 2 * 10**6 + 100, dtype=np.int32)]), n).astype(np.int32)
    fk2 = r.choice(np.concatenate([k2, k2[:50] + 1]), n).astype(np.int64)
    fact = {"fk1": fk1, "fk2": fk2, "date": r.integers(0, 2557, n).astype(np.int32)}
    for c in ("m1", "m2", "m3"):
        fact[c] = r.integers(0, 10**7, n).astype(np.int64)
    want = pl.star(fact, dim1, dim2)
    cu = lambda t: {k: torch.from_numpy(v).cuda() for k, v in t.items()}
    compare(Q.star(cu(fact), cu(dim1), cu(dim2)), want)
    assert tqp.tqp_status_poll() == tqp.OK


@pytest.mark.parametrize("learned", [False, True])
def test_star_full_size_invariants(G, learned):
    """The full star join (fact 600M rows, dims 20M and 150M) in the
    benchmark's configuration, with the radix or the learned dimension sort.  At this size the oracle checks properties
    that hold at any size: every fact row matches exactly one row of each
    dimension (foreign keys drawn from the dimension keys), so the group
    counts sum to the number of rows with date < 767 and each measure's sums
    add up to that measure's total over those rows; group keys are unique and
    ascending and within the category domains.  The scaled test above checks
    every group exactly."""
    tqp, Q, gd = G
    n, n1, n2 = 600_000_000, 20_000_000, 150_000_000
    rec = dg.star_tables(n1, n2)
    fact = gd.make_table(rec["fact"], n)
    d1, d2 = gd.make_table(rec["dim1"], n1), gd.make_table(rec["dim2"], n2)
    cfg = tqp.learned_cfg(sample=65536, tcfg=tqp.train_cfg(epochs=10, lr=1e-4)) if learned else None
    ok, oa, g = Q.star(fact, d1, d2, learned=cfg)
    assert tqp.tqp_status_poll() == tqp.OK
    del fact, d1, d2
    torch.cuda.empty_cache()
    G_ = int(g.item())
    aggs = host(oa)[:G_]
    k1, k2 = host(ok[0], G_).astype(np.int64), host(ok[1], G_).astype(np.int64)
    assert np.all((k1 >= 0) & (k1 <= 999) & (k2 >= 0) & (k2 <= 49))
    key = k1 * 100 + k2
    assert np.all(np.diff(key) > 0)
    cnt, s1, s2, s3 = 0, 0, 0, 0
    chunk = 50_000_000
    for start in range(0, n, chunk):
        m = min(chunk, n - start)
        date = dg.generate(rec["fact"]["date"], m, start)
        sel = orc.filter([date], [(0, orc.LT, 767)])
        cnt += len(sel)
        for name in ("m1", "m2", "m3"):
            col = orc.gather(dg.generate(rec["fact"][name], m, start), sel)
            total = int(col.sum())
            if name == "m1":
                s1 += total
            elif name == "m2":
                s2 += total
            else:
                s3 += total
    assert int(aggs[:, 3].sum()) == cnt
    assert [int(aggs[:, 0].sum()), int(aggs[:, 1].sum()), int(aggs[:, 2].sum())] == [s1, s2, s3]
