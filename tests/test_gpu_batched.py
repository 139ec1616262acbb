"""GPU parity of the batched instances: every problem of one batched call
equals the oracle's pipeline on that problem alone, and the unbatched GPU
call; every probe tile size (the autotuner's choices) gives identical
bytes; empty problems and duplicate dimension keys are handled."""
import numpy as np
import pytest
import torch

import oracle as orc
from oracle import pipelines as pl
from paper_2209_04579_b300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import datagen_device, queries, tqp
    return tqp, queries, datagen_device


def problems(scale, count=512, stride=1):
    ns, ms, gs = dg.batched_sizes()
    out = []
    for p in range(0, count, stride):
        n = max(1, int(ns[p]) // scale)
        m = max(1, n // 40)
        out.append((p, n, m, int(gs[p])))
    return out


def check(got, want):
    ok, oa, G = got
    wk, wa, _ = want
    g = wa.shape[0]
    assert int(G.item()) == g
    assert np.array_equal(ok.cpu().numpy()[:g].astype(np.int64), wk[0])
    assert np.array_equal(oa.cpu().numpy()[:g], wa)


def make(M, spec):
    tqp, Q, gd = M
    host, dev = [], []
    for p, n, m, g in spec:
        rec = dg.batched_problem(p, n, m, g)
        host.append((dg.make_table(rec["fact"], n), dg.make_table(rec["dim"], m)))
        dev.append((gd.make_table(rec["fact"], n), gd.make_table(rec["dim"], m)))
    return host, dev


@pytest.mark.parametrize("items", [4, 8, 16])
def test_batched_equals_oracle_and_unbatched(M, items):
    tqp, Q, gd = M
    host, dev = make(M, problems(scale=100))
    res = Q.batched(dev, probe_items=items)
    assert tqp.tqp_status_poll() == tqp.OK
    for (fh, dh), (fd, dd), got in zip(host, dev, res):
        check(got, pl.batched_one(fh, dh))
    for (fd, dd), got in list(zip(dev, res))[::37]:
        one = Q.batched_one(fd, dd)
        check(got, (one[0][0].cpu().numpy()[:int(one[2].item())].astype(np.int64)[None, :],
                    one[1].cpu().numpy()[:int(one[2].item())], False))


def test_batched_edge_problems(M):
    tqp, Q, gd = M
    z32, z8, z64 = (torch.empty(0, dtype=d, device="cuda") for d in (torch.int32, torch.int8, torch.int64))
    r = np.random.default_rng(4)
    fk = torch.from_numpy(r.integers(0, 50, 5000).astype(np.int32)).cuda()
    day = torch.from_numpy(r.integers(0, 2557, 5000).astype(np.int32)).cuda()
    v = torch.from_numpy(r.integers(0, 10**7, 5000).astype(np.int64)).cuda()
    key = torch.arange(40, dtype=torch.int32, device="cuda")
    grp = torch.from_numpy(r.integers(-3, 3, 40).astype(np.int8)).cuda()
    probs = [
        ({"fk": z32, "day": z32, "v": z64}, {"key": key, "grp": grp}),      # no fact rows
        ({"fk": fk, "day": day, "v": v}, {"key": z32, "grp": z8}),          # empty dimension
        ({"fk": fk, "day": day, "v": v}, {"key": key, "grp": grp}),
    ]
    res = Q.batched(probs)
    assert tqp.tqp_status_poll() == tqp.OK
    assert int(res[0][2].item()) == 0 and int(res[1][2].item()) == 0
    h = lambda t: t.cpu().numpy()
    check(res[2], pl.batched_one({"fk": h(fk), "day": h(day), "v": h(v)}, {"key": h(key), "grp": h(grp)}))
    dup = torch.cat([key, key[:1]])
    Q.batched([({"fk": fk, "day": day, "v": v}, {"key": dup, "grp": torch.cat([grp, grp[:1]])})])
    assert tqp.tqp_status_poll() == tqp.ERR_UNSUPPORTED


def test_batched_full_size_sampled(M):
    """All 512 problems at full size (fact rows sum to ~247M); 16 problems,
    spread over the size range, checked against the oracle."""
    tqp, Q, gd = M
    spec = problems(scale=1)
    _, dev = [], []
    dev = []
    for p, n, m, g in spec:
        rec = dg.batched_problem(p, n, m, g)
        dev.append((gd.make_table(rec["fact"], n), gd.make_table(rec["dim"], m)))
    res = Q.batched(dev)
    assert tqp.tqp_status_poll() == tqp.OK
    order = np.argsort([s[1] for s in spec])
    for i in order[::len(order) // 16]:
        p, n, m, g = spec[i]
        rec = dg.batched_problem(p, n, m, g)
        check(res[i], pl.batched_one(dg.make_table(rec["fact"], n), dg.make_table(rec["dim"], m)))
