"""Date columns on the GPU against the oracle, element by element: ISO date
strings and day numbers to epoch nanoseconds (Section 2.1's date tensor),
and epoch nanoseconds back to the calendar.  Integer results: bit-exact."""
import datetime as dt

import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import tqp
    return tqp


def iso_rows(dates, width):
    out = np.zeros((len(dates), width), np.uint8)
    for i, t in enumerate(dates):
        b = t.encode()[:width]
        out[i, :len(b)] = np.frombuffer(b, np.uint8)
    return out


def every_day(first, last):
    d, out = first, []
    while d <= last:
        out.append(d.isoformat())
        d += dt.timedelta(days=1)
    return out


@pytest.mark.parametrize("width", [10, 12, 16, 33])
def test_date_parse_iso(T, width):
    """Every day of 1600..2300 (including the first and last representable
    days and the days beyond them), malformed rows mixed in, over several
    tiles with a ragged tail; 16-byte-aligned and unaligned row widths."""
    dates = every_day(dt.date(1600, 1, 1), dt.date(2300, 12, 31))
    bad = ["1900-02-29", "2023-13-01", "2023-00-10", "2023-04-31", "1970/01/01", "19700101", "", "abcd-ef-gh",
           "2262-04-12", "1677-09-21"]
    r = np.random.default_rng(width)
    rows = np.array(dates + bad * 50, dtype=object)[r.permutation(len(dates) + 50 * len(bad))]
    s = iso_rows(list(rows), width)
    if width > 10:
        s[7, 10] = ord("Z")      # a byte after the date that is not padding: malformed
    want, ok = orc.date_parse_iso(s)
    got = T.tqp_date_parse_iso(torch.from_numpy(s).cuda())
    assert np.array_equal(got.cpu().numpy(), want)
    assert T.tqp_status_poll() == (T.OK if ok.all() else T.ERR_INVALID)
    good = s[ok.astype(bool)]
    got = T.tqp_date_parse_iso(torch.from_numpy(np.ascontiguousarray(good)).cuda())
    assert np.array_equal(got.cpu().numpy(), want[ok.astype(bool)])
    assert T.tqp_status_poll() == T.OK


def test_date_from_days_and_parts(T):
    r = np.random.default_rng(5)
    days = np.concatenate([np.arange(-106760, -106740), np.arange(106740, 106760), np.arange(-800, 800),
                           r.integers(-106751, 106752, 300_000)]).astype(np.int32)
    want = orc.date_from_days(days)
    got = T.tqp_date_from_days(torch.from_numpy(days).cuda())
    assert np.array_equal(got.cpu().numpy(), want)
    assert T.tqp_status_poll() == T.ERR_INVALID      # the out-of-range days
    ns = np.concatenate([r.integers(-2**63, 2**63 - 1, 500_000, dtype=np.int64),
                         want[want != -2**63], want[want != -2**63] - 1,
                         np.array([0, -1, 1, -2**63, 2**63 - 1], np.int64)])
    got = T.tqp_date_parts(torch.from_numpy(ns).cuda())
    for g, w in zip(got, orc.date_parts(ns)):
        assert np.array_equal(g.cpu().numpy(), w)
    assert T.tqp_status_poll() == T.OK


def test_date_empty_and_arguments(T):
    e = torch.zeros((0, 10), dtype=torch.uint8, device="cuda")
    assert T.tqp_date_parse_iso(e).numel() == 0
    with pytest.raises(T.TQPError):
        T.tqp_date_parse_iso(torch.zeros((4, 9), dtype=torch.uint8, device="cuda"))   # narrower than a date
    assert T.tqp_status_poll() == T.OK
