"""The synthetic workloads' queries, composed from the C-ABI operators.

Each function states its SQL.  Results are returned on the device; counts
are device tensors (no host synchronisation inside), so a whole query can be
captured in a CUDA graph.  The query shapes follow the paper's Section 2.3:
a filter plus an aggregation (Q6) and a join plus an aggregation (Q14).
"""
from __future__ import annotations

from . import tqp

Q6_DAY_MAX = 2400
Q14_REGION_LT = 5
BATCH_DAY_LT = 1278
STAR_DATE_LT = 767

Q6_EXPRS = [
    [(0, 1, 0)],                              # qty
    [(1, 1, 0)],                              # price
    [(1, 1, 0), (2, -1, 100)],                # price * (100 - disc)
    [(1, 1, 0), (2, -1, 100), (3, 1, 100)],   # price * (100 - disc) * (100 + tax)
]
Q6_AGGS = [(tqp.SUM, 0), (tqp.SUM, 1), (tqp.SUM, 2), (tqp.SUM, 3), (tqp.COUNT, 0)]


def q6(t, cap: int = 64):
    """SELECT flag_a, flag_b, SUM(qty), SUM(price), SUM(price*(100-disc)),
    SUM(price*(100-disc)*(100+tax)), COUNT(*) FROM lineitem
    WHERE ship_day <= 2400 GROUP BY flag_a, flag_b."""
    sel, cnt = tqp.tqp_filter([t["ship_day"]], [(0, tqp.LE, Q6_DAY_MAX)])
    return tqp.tqp_groupby_agg([t["flag_a"], t["flag_b"]], [t["qty"], t["price"], t["disc"], t["tax"]],
                               Q6_EXPRS, Q6_AGGS, cap, sel=sel, n=t["ship_day"].numel(), d_n=cnt)


def q14(fact, dim, cap: int = 64, learned=None):
    """SELECT region, SUM(price), COUNT(*) FROM fact JOIN dim ON fk = key
    WHERE region < 5 GROUP BY region -- fused star aggregate.  learned: a
    learned_cfg (the dimension's keys sorted through the learned range
    partitioner)."""
    D = tqp.DimSpec(dim["key"], cols=[dim["region"], dim["price"]], preds=[(0, tqp.LT, Q14_REGION_LT)],
                    group=dim["region"])
    return tqp.tqp_star_agg([fact["fk"]], [], [0], [D], [(1, 1)], [[(0, 1, 0)]],
                            [(tqp.SUM, 0), (tqp.COUNT, 0)], cap, learned=learned)


def q14_promo(fact, dim, prefix: bytes, d0: int, d1: int):
    """SELECT SUM(CASE WHEN type LIKE 'prefix%' THEN price*(100-disc) ELSE 0
    END), SUM(price*(100-disc)) FROM fact JOIN dim ON fk = key WHERE ship_ns
    >= d0 AND ship_ns < d1 -- the promotion-revenue shape of Q14 (its ratio is
    100 * first / second).  The LIKE runs once over the dimension's string
    tensor; its 0/1 column is the CASE's factor in the fused aggregate, and
    the date range is two predicates on the int64 epoch-nanosecond column."""
    promo = tqp.tqp_like_prefix(dim["type"], prefix)
    D = tqp.DimSpec(dim["key"], cols=[promo])
    cols = [fact["fk"], fact["ship_ns"], fact["price"], fact["disc"]]
    return tqp.tqp_star_agg(cols, [(1, tqp.GE, d0), (1, tqp.LT, d1)], [0], [D], [(0, 2), (0, 3), (1, 0)],
                            [[(0, 1, 0), (1, -1, 100), (2, 1, 0)], [(0, 1, 0), (1, -1, 100)]],
                            [(tqp.SUM, 0), (tqp.SUM, 1)], 1)


def q14_unfused(fact, dim, cap: int = 64, pair_cap: int | None = None):
    """The same query as a chain of separate operators: join (bound search +
    expand into pairs), gathers, filter on the joined rows, group-by."""
    n = fact["fk"].numel()
    pair_cap = n if pair_cap is None else pair_cap
    pr, br, npairs = tqp.tqp_join_eq(fact["fk"], dim["key"], pair_cap)
    region = tqp.tqp_gather(dim["region"], br, n=pair_cap, d_n=npairs)
    price = tqp.tqp_gather(dim["price"], br, n=pair_cap, d_n=npairs)
    keep, nkeep = tqp.tqp_filter([region], [(0, tqp.LT, Q14_REGION_LT)], n=pair_cap, d_n=npairs)
    return tqp.tqp_groupby_agg([region], [price], [[(0, 1, 0)]], [(tqp.SUM, 0), (tqp.COUNT, 0)], cap,
                               sel=keep, n=pair_cap, d_n=nkeep)


def skew(t, cap: int):
    """SELECT key, COUNT(*), SUM(value), MIN(value), MAX(value) FROM t GROUP BY key."""
    return tqp.tqp_groupby_agg([t["key"]], [t["value"]], [[(0, 1, 0)]],
                               [(tqp.COUNT, 0), (tqp.SUM, 0), (tqp.MIN, 0), (tqp.MAX, 0)], cap)


def skew_learned(t, cap: int, cfg=None):
    """The skewed group-by through the learned range partitioner (same
    results as skew())."""
    return tqp.tqp_groupby_agg_learned([t["key"]], [t["value"]], [[(0, 1, 0)]],
                                       [(tqp.COUNT, 0), (tqp.SUM, 0), (tqp.MIN, 0), (tqp.MAX, 0)], cap, cfg=cfg)


def batched_one(fact, dim, cap: int = 64):
    """SELECT grp, SUM(v), COUNT(*) FROM fact JOIN dim ON fk = key
    WHERE day < 1278 GROUP BY grp."""
    D = tqp.DimSpec(dim["key"], cols=[dim["grp"]], group=dim["grp"])
    return tqp.tqp_star_agg([fact["fk"], fact["day"], fact["v"]], [(1, tqp.LT, BATCH_DAY_LT)], [0], [D],
                            [(0, 2)], [[(0, 1, 0)]], [(tqp.SUM, 0), (tqp.COUNT, 0)], cap)


def batched_shape():
    """Query shape of every batched instance: fact (fk int32, day int32,
    v int64) JOIN dim (key int32, grp int8) WHERE day < 1278 GROUP BY grp:
    SUM(v), COUNT(*)."""
    import torch
    return tqp.batch_shape([torch.int32, torch.int32, torch.int64], 0, torch.int8,
                           [(1, tqp.LT, BATCH_DAY_LT)], [[(2, 1, 0)]], [(tqp.SUM, 0), (tqp.COUNT, 0)])


def batched(problems, cap: int = 64, probe_items: int = 8, shape=None):
    """All instances in one batched call; problems: list of (fact, dim) tables."""
    shape = shape or batched_shape()
    return tqp.tqp_star_agg_batched(shape, [([f["fk"], f["day"], f["v"]], d["key"], d["grp"]) for f, d in problems],
                                    cap=cap, probe_items=probe_items)


def star(fact, dim1, dim2, cap: int = 50_000, learned=None):
    """SELECT dim1.cat, dim2.cat, SUM(m1), SUM(m2), SUM(m3), COUNT(*)
    FROM fact JOIN dim1 ON fk1 = dim1.key JOIN dim2 ON fk2 = dim2.key
    WHERE date < 767 GROUP BY dim1.cat, dim2.cat.  learned: a learned_cfg
    (the dimensions' keys sorted through the learned range partitioner)."""
    D1 = tqp.DimSpec(dim1["key"], cols=[dim1["cat"]], group=dim1["cat"])
    D2 = tqp.DimSpec(dim2["key"], cols=[dim2["cat"]], group=dim2["cat"])
    cols = [fact["fk1"], fact["fk2"], fact["m1"], fact["m2"], fact["m3"], fact["date"]]
    return tqp.tqp_star_agg(cols, [(5, tqp.LT, STAR_DATE_LT)], [0, 1], [D1, D2], [(0, 2), (0, 3), (0, 4)],
                            [[(0, 1, 0)], [(1, 1, 0)], [(2, 1, 0)]],
                            [(tqp.SUM, 0), (tqp.SUM, 1), (tqp.SUM, 2), (tqp.COUNT, 0)], cap, learned=learned)


def predict(t, model, min_votes: int, cap: int = 16):
    """SELECT rating, SUM(CASE WHEN PREDICT(model, score) >= 0.5 THEN 1 ELSE
    0 END), COUNT(*) FROM reviews WHERE votes >= min_votes GROUP BY rating --
    a prediction query (Section 3.3): the network's output over the score
    column, as its bucket of two (0/1: output below or at least one half),
    is the CASE factor of a filtered group-by.  Every step runs in the
    library's kernels on one stream, so the whole query captures into one
    CUDA graph."""
    _, positive = tqp.tqp_cdf_forward(model, t["score"], B=2, want_F=False)
    sel, cnt = tqp.tqp_filter([t["votes"]], [(0, tqp.GE, min_votes)])
    return tqp.tqp_groupby_agg([t["rating"]], [positive], [[(0, 1, 0)]], [(tqp.SUM, 0), (tqp.COUNT, 0)], cap,
                               sel=sel, n=t["votes"].numel(), d_n=cnt)


def group_by_string(strings, vals, exprs, aggs, cap: int):
    """GROUP BY a string column: its dictionary codes (the values' ranks in
    ascending byte order) are the group key.  Returns (the groups' codes,
    aggs, device G, a representative row of each code)."""
    codes, rep, _ = tqp.tqp_string_codes(strings)
    ok, oa, g = tqp.tqp_groupby_agg([codes], vals, exprs, aggs, cap)
    return ok[0], oa, g, rep
