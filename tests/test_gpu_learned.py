"""GPU parity of the learned range partitioner: the network's forward pass
(bit-exact against the oracle's float32 evaluation in the same order), its
gradients (against the oracle's float64 analytic gradients), the Adam step,
and the learned group-by (bit-identical to the oracle and to the plain radix
path for every configuration, including the global-memory fallback)."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import pipelines as pl
from paper_2209_04579_b300 import datagen as dg

pytestmark = pytest.mark.gpu
H = 64


@pytest.fixture(scope="module")
def T():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import tqp
    return tqp


def rand_model(rng, H=H):
    w = rng.uniform(0.5, 80, H).astype(np.float32)
    b = rng.uniform(-60, 1, H).astype(np.float32)
    a = rng.uniform(0, 2.0 / H, H).astype(np.float32)
    c = np.float32(rng.uniform(-0.05, 0.05))
    return w, b, a, c


def test_forward_bit_exact_and_buckets(T):
    rng = np.random.default_rng(1)
    w, b, a, c = rand_model(rng)
    x = rng.uniform(-0.1, 1.1, 300_001).astype(np.float32)
    m = T.model_to_device(w, b, a, c)
    F, bk = T.tqp_cdf_forward(m, torch.from_numpy(x).cuda(), B=4096)
    want = orc.cdf_forward_f32(w, b, a, float(c), x)
    assert np.array_equal(F.cpu().numpy().view(np.uint32), want.view(np.uint32))
    assert np.array_equal(bk.cpu().numpy(), orc.cdf_bucket(want, 4096))
    F2, bk2 = T.tqp_cdf_forward(m, torch.from_numpy(x).cuda(), B=2, want_F=False)  # buckets alone
    assert F2 is None and np.array_equal(bk2.cpu().numpy(), orc.cdf_bucket(want, 2))


def test_backward_vs_float64(T):
    rng = np.random.default_rng(2)
    for n in (1000, 65536, 200_003):
        w, b, a, c = rand_model(rng)
        x = rng.uniform(0, 1, n).astype(np.float32)
        y = np.sort(rng.uniform(0, 1, n)).astype(np.float32)
        g = T.tqp_cdf_backward(T.model_to_device(w, b, a, c), torch.from_numpy(x).cuda(),
                               torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
        loss, gw, gb, ga, gc = orc.cdf_grad_f64(w.astype(np.float64), b.astype(np.float64), a.astype(np.float64),
                                                float(c), x.astype(np.float64), y.astype(np.float64))
        want = np.concatenate([gw, gb, ga, [gc]])
        scale = np.max(np.abs(want))
        # float32 sums over n samples: relative error well under 1e-4 of the largest component
        assert np.all(np.abs(g[:3 * H + 1] - want) <= 1e-4 * scale + 1e-4 * np.abs(want)), n
        assert abs(g[3 * H + 1] - loss) <= 1e-4 * loss


def test_adam_step_vs_float64(T):
    rng = np.random.default_rng(3)
    w, b, a, c = rand_model(rng)
    x = rng.uniform(0, 1, 8192).astype(np.float32)
    y = np.sort(rng.uniform(0, 1, 8192)).astype(np.float32)
    m = T.model_to_device(w, b, a, c)
    loss = T.tqp_cdf_train(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), m, T.train_cfg(epochs=1, lr=1e-2))
    got = T.model_from_device(m)
    p = np.concatenate([w, b, a, [c]]).astype(np.float64)
    l0, gw, gb, ga, gc = orc.cdf_grad_f64(w.astype(np.float64), b.astype(np.float64), a.astype(np.float64), float(c),
                                          x.astype(np.float64), y.astype(np.float64))
    nonneg = np.r_[np.ones(H), np.zeros(H), np.ones(H), [0]].astype(np.int32)
    orc.adam_step_f64(p, np.concatenate([gw, gb, ga, [gc]]), np.zeros(3 * H + 1), np.zeros(3 * H + 1), nonneg, 1,
                      lr=1e-2)
    gp = np.concatenate([got["w"], got["b"], got["a"], [got["c"]]])
    # first Adam step moves each parameter by about lr * sign(g); float32 vs float64 agree to ~1e-6
    assert np.max(np.abs(gp - p)) < 2e-5 * max(1.0, np.max(np.abs(p)))
    assert abs(loss.cpu().numpy()[0] - l0) <= 1e-4 * l0
    assert min(got["w"]) >= 0 and min(got["a"]) >= 0


def test_training_reduces_loss_and_stays_monotone(T):
    z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
    keys = np.sort(dg.make_table(dg.skew_groupby(), 65536, zipf=z)["key"])
    u = keys.view(np.uint64) ^ np.uint64(1 << 63)
    umin, span = int(u[0]), int(u[-1] - u[0])
    shift = max(0, span.bit_length() - 24)
    inv = float(np.float32(1.0) / np.float32(span >> shift))
    x = orc.cdf_normalize(keys, umin, shift, inv)
    y = orc.cdf_targets(keys).astype(np.float32)
    j = np.arange(H)
    m = T.model_to_device(np.full(H, float(H)), -j.astype(np.float64), np.full(H, 1.0 / H), 0.0)
    loss = T.tqp_cdf_train(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), m, T.train_cfg(epochs=200))
    loss = loss.cpu().numpy()
    assert loss[-1] < 0.2 * loss[0]
    F, _ = T.tqp_cdf_forward(m, torch.from_numpy(np.linspace(0, 1, 100_001, dtype=np.float32)).cuda())
    assert np.all(np.diff(F.cpu().numpy()) >= 0)


def skew_case(n, master=20220904):
    z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
    rec = dg.skew_groupby(master=master)
    return dg.make_table(rec, n, zipf=z), rec, z


def compare(got, want):
    ok, oa, g = got[:3]
    wk, wa, _ = want
    G = wa.shape[0]
    assert int(g.item()) == G
    for i in range(len(ok)):
        assert np.array_equal(ok[i].cpu().numpy()[:G].astype(np.int64), wk[i])
    assert np.array_equal(oa.cpu().numpy()[:G], wa)


@pytest.mark.parametrize("n", [1, 1000, 70_001, 3_000_000])
@pytest.mark.parametrize("train,heavy,buckets", [(1, 1, 0), (0, 1, 0), (1, 0, 0), (1, 1, 2), (0, 0, 16), (1, 1, 1 << 15),
                                                (1, 1, 1 << 17),
                                                # no heavy keys, repeated keys: buckets of thousands of rows
                                                # (the MSD kernel, which flags parts holding several keys),
                                                # and more buckets than one block counts (coarse counts,
                                                # fine counts after split 1)
                                                (1, 0, 1 << 10), (0, 0, 1 << 15)])
def test_learned_groupby_parity(T, n, train, heavy, buckets):
    from paper_2209_04579_b300 import datagen_device as gd
    from paper_2209_04579_b300 import queries as Q
    host, rec, z = skew_case(n)
    want = pl.skew(host)
    dev = gd.make_table(rec, n, zipf=torch.from_numpy(z).cuda())
    cfg = T.learned_cfg(sample=4096 if n < 100_000 else 65536, buckets=buckets, train=bool(train),
                        heavy=bool(heavy), tcfg=T.train_cfg(epochs=50))
    got = Q.skew_learned(dev, cap=max(n, 1), cfg=cfg)
    compare(got, want)
    assert T.tqp_status_poll() == T.OK
    compare(Q.skew(dev, cap=max(n, 1)), want)     # the plain radix path agrees


def test_learned_groupby_general_keys(T):
    """Two key columns of mixed widths, a selection, several aggregates."""
    rng = np.random.default_rng(5)
    n = 500_000
    k1 = rng.integers(-30_000, 30_000, n).astype(np.int16)
    k2 = (rng.zipf(1.3, n) % 1000).astype(np.int32) - 500
    v = rng.integers(-10**9, 10**9, n).astype(np.int64)
    sel = np.sort(rng.choice(n, n // 3, replace=False)).astype(np.int32)
    ex = [[(0, 1, 0)], [(0, 3, -7), (0, 1, 1)]]
    ag = [(orc.COUNT, 0), (orc.SUM, 0), (orc.MIN, 1), (orc.MAX, 0), (orc.SUM, 1)]
    want = orc.groupby_agg([k1, k2], [v], ex, ag, sel=sel)
    cu = lambda a: torch.from_numpy(a).cuda()
    got = T.tqp_groupby_agg_learned([cu(k1), cu(k2)], [cu(v)], ex, ag, n, cfg=T.learned_cfg(sample=16384),
                                    sel=cu(sel))
    compare(got, want)
    assert T.tqp_status_poll() == T.OK


@pytest.mark.parametrize("kind", ["lognormal", "skew"])
def test_trained_network_gains(T, kind):
    """What the network gains, three ways on the same keys: the identity CDF
    (the method without a network), the network initialised at the sample's
    quantile knots (no training: the serving form), and those knots trained
    on the GPU.  Every form gives the exact group-by.  On log-normal keys
    (far from uniform in key space) both fitted forms route far fewer rows
    to the global-memory fallback than the identity CDF; on the skewed
    workload's keys the fitted forms are no worse.  Training keeps the best
    parameters it evaluates and strictly lowers its training loss."""
    rng = np.random.default_rng(7)
    if kind == "lognormal":
        n = 4_000_000
        keys = np.exp(rng.normal(12, 1.5, n)).astype(np.int64)
    else:
        n = 3_000_000
        keys = skew_case(n)[0]["key"]
    vals = rng.integers(0, 2**31, n).astype(np.int64)
    want = orc.groupby_agg([keys], [vals], [[(0, 1, 0)]], [(orc.COUNT, 0), (orc.SUM, 0)])
    cu = lambda a: torch.from_numpy(a).cuda()
    forms = {"identity": T.learned_cfg(sample=65536, buckets=4096, train=False, init=0),
             "knots": T.learned_cfg(sample=65536, buckets=4096, train=False, init=1),
             "trained": T.learned_cfg(sample=65536, buckets=4096, train=True, init=1,
                                      tcfg=T.train_cfg(epochs=100, lr=1e-5))}
    res = {}
    for name, cfg in forms.items():
        got = T.tqp_groupby_agg_learned([cu(keys)], [cu(vals)], [[(0, 1, 0)]], [(orc.COUNT, 0), (orc.SUM, 0)], n,
                                        cfg=cfg)
        compare(got, want)
        res[name] = T.stats_from_device(got[4])
    tr, kn, ide = res["trained"], res["knots"], res["identity"]
    assert tr["loss_last"] < tr["loss_first"]
    if kind == "lognormal":
        for fit in (tr, kn):
            assert fit["max_bucket"] * 4 < ide["max_bucket"]
            assert fit["over_capacity_rows"] * 4 < ide["over_capacity_rows"]
    else:
        for fit in (tr, kn):
            assert fit["over_capacity_rows"] <= ide["over_capacity_rows"]
    assert T.tqp_status_poll() == T.OK


def _partition_case(case):
    r = np.random.default_rng(len(case) * 7 + 3)
    sel = None
    if case == "skew_heavy" or case == "skew_light":
        z = dg.zipf_table(dg.ZIPF_S, dg.ZIPF_N)
        keys = dg.make_table(dg.skew_groupby(), 600_000, zipf=z)["key"]
    elif case == "lognormal_sel":
        keys = np.exp(r.normal(12, 1.5, 800_000)).astype(np.int64) - 2**40
        sel = np.sort(r.choice(len(keys), 500_000, replace=False)).astype(np.int32)
    else:  # int32 keys over the full range with repeats
        keys = r.integers(-2**31, 2**31, 400_000, dtype=np.int64).astype(np.int32)
        keys[::3] = keys[5]
    return keys, sel


@pytest.mark.parametrize("case", ["skew_heavy", "skew_light", "lognormal_sel", "int32"])
def test_partition_learned_against_oracle(T, case):
    """The standalone learned partition, bit for bit: its training pairs
    against the oracle's light-CDF targets (heavy keys set apart) and key
    normalisation on the same sorted sample; every row's bucket against the
    oracle's float32 evaluation of the returned network (the GPU finds the
    bucket from the network's step positions, never by evaluating it per
    row); heavy rows' ids against the oracle's heavy keys; the grouped rows
    and offsets against the oracle's stable partition by bucket id."""
    keys, sel = _partition_case(case)
    heavy = case != "skew_light"
    S = 16384
    cfg = T.learned_cfg(sample=S, heavy=heavy, tcfg=T.train_cfg(epochs=20, lr=1e-4))
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = T.tqp_partition_learned([cu(keys)], cfg=cfg, sel=None if sel is None else cu(sel))
    B = out["B"]
    rows = np.arange(len(keys), dtype=np.int64) if sel is None else sel.astype(np.int64)
    n = len(rows)
    kr = keys[rows].astype(np.int64)
    kmin = int(kr.min())
    packed = (kr - kmin).astype(np.uint64)          # key - min: exact in 64-bit two's complement
    SH = min(4 * S, 1 << 20)
    mult = SH // S
    samp = (np.arange(SH, dtype=np.int64) * n) // SH
    order = np.argsort(packed[samp], kind="stable")
    sorted_packed = packed[samp][order]
    sorted_keys = kr[samp][order]
    minc = max(2, min(4095, int(SH * 8192 / (2.0 * n)) + 1))
    y_want, heavy_keys = orc.light_cdf_targets(sorted_packed, mult, S, minc, 1024 if heavy else 0)
    m = T.model_from_device(out["model"])
    umin = (kmin ^ (1 << 63)) if kmin >= 0 else (kmin + 2**64) ^ (1 << 63)
    x_want = orc.cdf_normalize(sorted_keys[::mult][:S], umin, m["shift"], m["inv"])
    assert np.array_equal(out["train_y"].cpu().numpy(), y_want)
    assert np.array_equal(out["train_x"].cpu().numpy(), x_want)
    st = T.stats_from_device(out["stats"])
    assert st["heavy_keys"] == len(heavy_keys)
    assert (len(heavy_keys) > 0) == (case in ("skew_heavy", "int32"))
    # bucket ids: the network evaluated per row by the oracle, heavy keys apart
    x = orc.cdf_normalize(kr, umin, m["shift"], m["inv"])
    F = orc.cdf_forward_f32(np.array(m["w"], np.float32), np.array(m["b"], np.float32),
                            np.array(m["a"], np.float32), m["c"], x)
    want = orc.cdf_bucket(F, B)
    hidx = np.searchsorted(heavy_keys, packed)
    is_heavy = (hidx < len(heavy_keys)) & (heavy_keys[np.minimum(hidx, max(len(heavy_keys) - 1, 0))] == packed) \
        if len(heavy_keys) else np.zeros(n, bool)
    want = np.where(is_heavy, B + hidx, want).astype(np.int32)
    got = out["bucket"].cpu().numpy()[:n]
    assert np.array_equal(got, want)
    light = ~is_heavy
    assert np.all(np.diff(want[light][np.argsort(kr[light], kind="stable")]) >= 0)   # monotone in the key
    prow, poff = orc.partition(want, B + T.MAX_HEAVY)
    assert np.array_equal(out["offsets"].cpu().numpy(), poff)
    assert np.array_equal(out["rows"].cpu().numpy()[:n], rows[prow].astype(np.int32))
    assert st["light_rows"] == int(light.sum()) and st["buckets"] == B
    assert T.tqp_status_poll() == T.OK
