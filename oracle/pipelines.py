"""Query pipelines of the synthetic workloads, composed from the oracle's
operators in the literal order of each query (test infrastructure only).

Section 2.3 of the paper benchmarks a filter-plus-aggregation query (TPC-H
Q6: "four filters ... and aggregation") and a join-plus-aggregation query
(Q14: "a join, as well as aggregation over a CASE expression").  The
workloads below keep those shapes on synthetic tables.  Each function states
its SQL; the plan is the textbook one (join, then WHERE on the joined rows,
then GROUP BY), with no pushed-down or fused step.
"""
from __future__ import annotations

import numpy as np

import oracle as orc

Q6_DAY_MAX = 2400
Q14_REGION_LT = 5
BATCH_DAY_LT = 1278
STAR_DATE_LT = 767


def q6(t):
    """SELECT flag_a, flag_b, SUM(qty), SUM(price), SUM(price*(100-disc)),
    SUM(price*(100-disc)*(100+tax)), COUNT(*) FROM lineitem
    WHERE ship_day <= 2400 GROUP BY flag_a, flag_b ORDER BY flag_a, flag_b."""
    sel = orc.filter([t["ship_day"]], [(0, orc.LE, Q6_DAY_MAX)])
    vals = [t["qty"], t["price"], t["disc"], t["tax"]]
    exprs = [
        [(0, 1, 0)],
        [(1, 1, 0)],
        [(1, 1, 0), (2, -1, 100)],
        [(1, 1, 0), (2, -1, 100), (3, 1, 100)],
    ]
    aggs = [(orc.SUM, 0), (orc.SUM, 1), (orc.SUM, 2), (orc.SUM, 3), (orc.COUNT, 0)]
    return orc.groupby_agg([t["flag_a"], t["flag_b"]], vals, exprs, aggs, sel=sel)


def q14(fact, dim):
    """SELECT region, SUM(price), COUNT(*) FROM fact JOIN dim ON fk = key
    WHERE region < 5 GROUP BY region ORDER BY region."""
    pr, br = orc.join_eq(fact["fk"], dim["key"])
    region = orc.gather(dim["region"], br)
    price = orc.gather(dim["price"], br)
    keep = orc.filter([region], [(0, orc.LT, Q14_REGION_LT)])
    return orc.groupby_agg([region], [price], [[(0, 1, 0)]], [(orc.SUM, 0), (orc.COUNT, 0)], sel=keep)


def q14_promo(fact, dim, prefix: bytes, d0: int, d1: int):
    """SELECT SUM(CASE WHEN type LIKE 'prefix%' THEN price*(100-disc) ELSE 0 END),
    SUM(price*(100-disc)) FROM fact JOIN dim ON fk = key
    WHERE ship_ns >= d0 AND ship_ns < d1 (one group: a constant key)."""
    pr, br = orc.join_eq(fact["fk"], dim["key"])
    ship = orc.gather(fact["ship_ns"], pr)
    keep = orc.filter([ship], [(0, orc.GE, d0), (0, orc.LT, d1)])
    promo = orc.gather(orc.like_prefix(dim["type"], prefix), br)
    price = orc.gather(fact["price"], pr)
    disc = orc.gather(fact["disc"], pr)
    one = np.zeros(len(pr), np.int8)
    return orc.groupby_agg([one], [price, disc, promo], [[(0, 1, 0), (1, -1, 100), (2, 1, 0)],
                                                        [(0, 1, 0), (1, -1, 100)]],
                           [(orc.SUM, 0), (orc.SUM, 1)], sel=keep)


def predict(t, model, min_votes: int):
    """SELECT rating, SUM(CASE WHEN PREDICT(model, score) >= 0.5 THEN 1 ELSE
    0 END), COUNT(*) FROM reviews WHERE votes >= min_votes GROUP BY rating
    ORDER BY rating.  model: (w, b, a, c); the prediction is the float32
    network output's bucket of two."""
    w, b, a, c = model
    positive = orc.cdf_bucket(orc.cdf_forward_f32(w, b, a, c, t["score"]), 2)
    keep = orc.filter([t["votes"]], [(0, orc.GE, min_votes)])
    return orc.groupby_agg([t["rating"]], [positive], [[(0, 1, 0)]], [(orc.SUM, 0), (orc.COUNT, 0)], sel=keep)


def skew(t):
    """SELECT key, COUNT(*), SUM(value), MIN(value), MAX(value) FROM t
    GROUP BY key ORDER BY key."""
    return orc.groupby_agg([t["key"]], [t["value"]], [[(0, 1, 0)]],
                           [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 0), (orc.MAX, 0)])


def batched_one(fact, dim):
    """One batched instance: SELECT grp, SUM(v), COUNT(*) FROM fact JOIN dim
    ON fk = key WHERE day < 1278 GROUP BY grp ORDER BY grp."""
    pr, br = orc.join_eq(fact["fk"], dim["key"])
    day = orc.gather(fact["day"], pr)
    keep = orc.filter([day], [(0, orc.LT, BATCH_DAY_LT)])
    grp = orc.gather(dim["grp"], br)
    v = orc.gather(fact["v"], pr)
    return orc.groupby_agg([grp], [v], [[(0, 1, 0)]], [(orc.SUM, 0), (orc.COUNT, 0)], sel=keep)


def star(fact, dim1, dim2):
    """SELECT dim1.cat, dim2.cat, SUM(m1), SUM(m2), SUM(m3), COUNT(*)
    FROM fact JOIN dim1 ON fk1 = dim1.key JOIN dim2 ON fk2 = dim2.key
    WHERE date < 767 GROUP BY dim1.cat, dim2.cat ORDER BY dim1.cat, dim2.cat."""
    p1, b1 = orc.join_eq(fact["fk1"], dim1["key"])
    fk2 = orc.gather(fact["fk2"], p1)
    p2, b2 = orc.join_eq(fk2, dim2["key"])
    rows = orc.gather(p1, p2)            # fact row of each joined triple
    cat1 = orc.gather(orc.gather(dim1["cat"], b1), p2)
    cat2 = orc.gather(dim2["cat"], b2)
    date = orc.gather(fact["date"], rows)
    keep = orc.filter([date], [(0, orc.LT, STAR_DATE_LT)])
    vals = [orc.gather(fact[c], rows) for c in ("m1", "m2", "m3")]
    exprs = [[(0, 1, 0)], [(1, 1, 0)], [(2, 1, 0)]]
    aggs = [(orc.SUM, 0), (orc.SUM, 1), (orc.SUM, 2), (orc.COUNT, 0)]
    return orc.groupby_agg([cat1, cat2], vals, exprs, aggs, sel=keep)
