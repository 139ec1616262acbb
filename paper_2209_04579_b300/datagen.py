"""Seeded synthetic column generators (host side, numpy).

These produce the synthetic decision-support tables that stand in for the
TPC-H SF1 lineitem/part-style inputs of the paper's evaluation (Section 2.3:
Q6 is four filters plus an aggregation, Q14 a join plus an aggregation).  The
TPC-H data, generator and query text are not used.

Every column is a pure function of (recipe, row index): row ``i`` of a column
is computed from a counter-based generator, so any slice can be generated
independently and the device generator (``csrc/datagen.cu``) produces the same
bits for the same recipe.  The module holds no arithmetic of the query
operators themselves; it only makes inputs.

Primitives (each written from its published definition):

* ``mix64``  -- the SplitMix64 output finaliser (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014; constants of
  Vigna's public-domain splitmix64.c).  It is a bijection on 64-bit words.
* ``draw(seed, i)`` -- the i-th SplitMix64 output from state ``seed``:
  ``mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)`` (mod 2^64).
* ``fmix32`` -- the MurmurHash3 32-bit finaliser (Appleby), a bijection on
  32-bit words.
* ``uniform`` -- Lemire's multiply-shift range reduction of the top 32 bits
  (Lemire, "Fast random integer generation in an interval", TOMACS 2019),
  without the rejection step, so it is a fixed function of the draw.
* ``perm`` -- a 4-round balanced Feistel network over 2^(2h) >= N with cycle
  walking (Black & Rogaway, "Ciphers with arbitrary finite domains", 2002):
  a seeded bijection of [0, N).
* ``zipf`` -- inverse-CDF sampling from a Zipf(s, N) table of float64
  cumulative probabilities built here on the host and shared with the device.
"""
from __future__ import annotations

import dataclasses
import math

import itertools

import numpy as np

MASTER_SEED = 20220904

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U64 = np.uint64

# recipe kinds (same codes as the device generator's header)
UNIFORM = 1        # mul * U[lo, hi]
PERM_KEY = 2       # perm_N(i) + lo
FMIX32_KEY = 3     # fmix32(i ^ seed32) as int32
MIX64_KEY = 4      # mix64(i ^ key_seed) as int64
FK_FMIX32 = 5      # fmix32(U[0, m-1] ^ seed32) as int32
FK_MIX64 = 6       # mix64(U[0, m-1] ^ key_seed) as int64
ZIPF_NOISE_KEY = 7 # Zipf rank keys mixed with uniform 64-bit noise
RAW64 = 8          # the raw 64-bit draw as int64

DTYPES = {1: np.int8, 2: np.int16, 3: np.int32, 4: np.int64}
DTYPE_CODE = {np.dtype(np.int8): 1, np.dtype(np.int16): 2,
              np.dtype(np.int32): 3, np.dtype(np.int64): 4}


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
    return z ^ (z >> _U64(31))


def stream_seed(master: int, stream: int) -> int:
    """Seed of one column stream: mix64(master ^ mix64(stream))."""
    s = mix64(np.array([stream], dtype=np.uint64))[0]
    return int(mix64(np.array([np.uint64(master) ^ s], dtype=np.uint64))[0])


def draw(seed: int, i):
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_U64(seed) + (i + _U64(1)) * _GAMMA)


def fmix32(h):
    h = np.asarray(h, dtype=np.uint32)
    with np.errstate(over="ignore"):
        h = h ^ (h >> np.uint32(16))
        h = h * np.uint32(0x85EBCA6B)
        h = h ^ (h >> np.uint32(13))
        h = h * np.uint32(0xC2B2AE35)
        h = h ^ (h >> np.uint32(16))
    return h


def uniform_from(u, lo: int, hi: int):
    """lo + floor(hi32(u) * (hi - lo + 1) / 2^32), for hi - lo + 1 <= 2^32."""
    rng = hi - lo + 1
    assert 1 <= rng <= (1 << 32)
    with np.errstate(over="ignore"):
        t = ((u >> _U64(32)) * _U64(rng)) >> _U64(32)
    return t.astype(np.int64) + np.int64(lo)


def _feistel_params(n: int):
    k = max(2, (max(n - 1, 1)).bit_length())
    half = (k + 1) // 2
    return half, (1 << half) - 1


def _feistel(x, seed: int, half: int, mask: int):
    x = np.asarray(x, dtype=np.uint64)
    left = x >> _U64(half)
    right = x & _U64(mask)
    for r in range(4):
        with np.errstate(over="ignore"):
            f = mix64(_U64(seed) + _U64(r) * _GAMMA + right) & _U64(mask)
        left, right = right, left ^ f
    return (left << _U64(half)) | right


def perm(i, n: int, seed: int):
    """Seeded bijection of [0, n): Feistel network plus cycle walking."""
    i = np.asarray(i, dtype=np.uint64)
    if i.size and int(i.max()) >= n:
        raise ValueError("perm is defined on [0, n) only")
    half, mask = _feistel_params(n)
    y = _feistel(i, seed, half, mask)
    todo = y >= _U64(n)
    while np.any(todo):
        y[todo] = _feistel(y[todo], seed, half, mask)
        todo = y >= _U64(n)
    return y


def zipf_table(s: float, n: int) -> np.ndarray:
    """cdf[k] = sum_{j<=k} (j+1)^-s / H_{n,s}, float64, k = 0..n-1."""
    w = 1.0 / np.power(np.arange(1, n + 1, dtype=np.float64), s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_rank(u, table: np.ndarray):
    """Rank r in [0, n): first index with table[r] > x, x = (u >> 11) * 2^-53."""
    x = (u >> _U64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.searchsorted(table, x, side="right")
    return np.minimum(r, len(table) - 1).astype(np.uint64)


@dataclasses.dataclass(frozen=True)
class Recipe:
    """How row i of one column is made.  ``dtype`` is 1..4 (int8..int64)."""
    kind: int
    dtype: int
    seed: int = 0          # draw stream
    key_seed: int = 0      # seed of the key bijection (keys / foreign keys)
    lo: int = 0
    hi: int = 0
    mul: int = 1
    m: int = 0             # dimension size for foreign keys / permutations
    noise_p32: int = 0     # noise iff hi32(draw) < noise_p32
    seed2: int = 0         # second stream (noise key / zipf draw)


def generate(rec: Recipe, n: int, start: int = 0, zipf: np.ndarray | None = None) -> np.ndarray:
    """Rows [start, start + n) of the column described by ``rec``."""
    i = np.arange(start, start + n, dtype=np.uint64)
    k = rec.kind
    if k == UNIFORM:
        v = uniform_from(draw(rec.seed, i), rec.lo, rec.hi) * np.int64(rec.mul)
    elif k == PERM_KEY:
        v = perm(i, rec.m, rec.key_seed).astype(np.int64) + np.int64(rec.lo)
    elif k == FMIX32_KEY:
        v = fmix32((i & _U64(0xFFFFFFFF)).astype(np.uint32) ^ np.uint32(rec.key_seed & 0xFFFFFFFF)).view(np.int32).astype(np.int64)
    elif k == MIX64_KEY:
        v = mix64(i ^ _U64(rec.key_seed)).view(np.int64)
    elif k == FK_FMIX32:
        j = uniform_from(draw(rec.seed, i), 0, rec.m - 1).astype(np.uint32)
        v = fmix32(j ^ np.uint32(rec.key_seed & 0xFFFFFFFF)).view(np.int32).astype(np.int64)
    elif k == FK_MIX64:
        j = uniform_from(draw(rec.seed, i), 0, rec.m - 1).astype(np.uint64)
        v = mix64(j ^ _U64(rec.key_seed)).view(np.int64)
    elif k == ZIPF_NOISE_KEY:
        assert zipf is not None
        sel = draw(rec.seed, i)
        noise = (sel >> _U64(32)) < _U64(rec.noise_p32)
        nz = draw(rec.seed2, i).view(np.int64)
        r = zipf_rank(draw(rec.seed2 ^ 0x5A5A5A5A5A5A5A5A, i), zipf)
        zk = mix64(r ^ _U64(rec.key_seed)).view(np.int64)
        v = np.where(noise, nz, zk)
    elif k == RAW64:
        v = draw(rec.seed, i).view(np.int64)
    else:
        raise ValueError(f"unknown recipe kind {k}")
    return v.astype(DTYPES[rec.dtype])


# --------------------------------------------------------------------------
# Workloads.  Each returns {table: {column: Recipe}} plus sizes.  Seeds come
# from MASTER_SEED and a fixed stream id per column.
# --------------------------------------------------------------------------

def _s(stream: int, master: int = MASTER_SEED) -> int:
    return stream_seed(master, stream)


def q6_lineitem(master: int = MASTER_SEED):
    """Filter + group-by table shaped like lineitem for a Q6-style query.

    ship_day int32 U[0,2556]; flag_a int8 U{0,1,2}; flag_b int8 U{0,1};
    qty int64 100*U{1..50}; price int64 U[90000, 10500000] (cents);
    disc int64 U[0,10]; tax int64 U[0,8].
    """
    return {
        "ship_day": Recipe(UNIFORM, 3, _s(101, master), lo=0, hi=2556),
        "flag_a": Recipe(UNIFORM, 1, _s(102, master), lo=0, hi=2),
        "flag_b": Recipe(UNIFORM, 1, _s(103, master), lo=0, hi=1),
        "qty": Recipe(UNIFORM, 4, _s(104, master), lo=1, hi=50, mul=100),
        "price": Recipe(UNIFORM, 4, _s(105, master), lo=90000, hi=10500000),
        "disc": Recipe(UNIFORM, 4, _s(106, master), lo=0, hi=10),
        "tax": Recipe(UNIFORM, 4, _s(107, master), lo=0, hi=8),
    }


def q14_tables(m: int, sparse_keys: bool = False, master: int = MASTER_SEED):
    """Join + group-by: fact(fk int32) into dim(key int32 unique, region int8
    U[0,24], price int64 U[100, 1e6]).

    Dense keys: key = perm_m(i) + 1, a seeded permutation of {1..m}, and
    fk = U[1, m].  Sparse keys: key = fmix32(i ^ s) (a bijection, so unique)
    and fk = fmix32(U[0, m-1] ^ s).
    """
    ks = _s(201, master)
    if sparse_keys:
        key = Recipe(FMIX32_KEY, 3, key_seed=ks & 0xFFFFFFFF)
        fk = Recipe(FK_FMIX32, 3, _s(202, master), key_seed=ks & 0xFFFFFFFF, m=m)
    else:
        key = Recipe(PERM_KEY, 3, key_seed=ks, m=m, lo=1)
        fk = Recipe(UNIFORM, 3, _s(202, master), lo=1, hi=m)
    dim = {
        "key": key,
        "region": Recipe(UNIFORM, 1, _s(203, master), lo=0, hi=24),
        "price": Recipe(UNIFORM, 4, _s(204, master), lo=100, hi=1000000),
    }
    return {"fact": {"fk": fk}, "dim": dim}


ZIPF_S = 1.0
ZIPF_N = 10_000_000
NOISE_P32 = 429496730   # ceil(0.1 * 2^32): a row is noise with probability 0.1


def skew_groupby(master: int = MASTER_SEED, zipf_n: int = ZIPF_N):
    """Skewed group-by: key int64 = 90% Zipf(1.0) ranks over zipf_n values
    (bijectively mixed) + 10% uniform 64-bit noise; value int64 U[0, 2^31]."""
    return {
        "key": Recipe(ZIPF_NOISE_KEY, 4, _s(301, master), key_seed=_s(302, master),
                      noise_p32=NOISE_P32, seed2=_s(303, master), m=zipf_n),
        "value": Recipe(UNIFORM, 4, _s(304, master), lo=0, hi=1 << 31),
    }


def batched_sizes(nprob: int = 512, lo: float = 1e3, hi: float = 4e6, master: int = MASTER_SEED):
    """Per-problem fact sizes n_i = floor(exp(U(ln lo, ln hi))), dim sizes
    m_i = max(1, n_i // 40), group counts g_i = U[1,64].  Host-only (float64)."""
    i = np.arange(nprob, dtype=np.uint64)
    u = (draw(_s(401, master), i) >> _U64(11)).astype(np.float64) * (2.0 ** -53)
    n = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    m = np.maximum(1, n // 40)
    g = uniform_from(draw(_s(402, master), i), 1, 64)
    return n, m, g


def batched_problem(p: int, n: int, m: int, g: int, master: int = MASTER_SEED):
    """Problem p of the batched workload: fact(fk, day int32 U[0,2556],
    v int64 U[0,1e7]) joined to dim(key unique int32, grp int8 U[0, g-1])."""
    base = 1000 + 10 * p
    ks = _s(base, master) & 0xFFFFFFFF
    fact = {
        "fk": Recipe(FK_FMIX32, 3, _s(base + 1, master), key_seed=ks, m=m),
        "day": Recipe(UNIFORM, 3, _s(base + 2, master), lo=0, hi=2556),
        "v": Recipe(UNIFORM, 4, _s(base + 3, master), lo=0, hi=10_000_000),
    }
    dim = {
        "key": Recipe(FMIX32_KEY, 3, key_seed=ks),
        "grp": Recipe(UNIFORM, 1, _s(base + 4, master), lo=0, hi=g - 1),
    }
    return {"fact": fact, "dim": dim}


def star_tables(n1: int = 20_000_000, n2: int = 150_000_000, master: int = MASTER_SEED):
    """Star join: fact(fk1 int32, fk2 int64, m1..m3 int64 U[0,1e7], date int32
    U[0,2556]); dim1(key int32 unique, cat int16 U[0,999]); dim2(key int64
    unique, cat int8 U[0,49])."""
    k1 = _s(501, master) & 0xFFFFFFFF
    k2 = _s(502, master)
    fact = {
        "fk1": Recipe(FK_FMIX32, 3, _s(503, master), key_seed=k1, m=n1),
        "fk2": Recipe(FK_MIX64, 4, _s(504, master), key_seed=k2, m=n2),
        "m1": Recipe(UNIFORM, 4, _s(505, master), lo=0, hi=10_000_000),
        "m2": Recipe(UNIFORM, 4, _s(506, master), lo=0, hi=10_000_000),
        "m3": Recipe(UNIFORM, 4, _s(507, master), lo=0, hi=10_000_000),
        "date": Recipe(UNIFORM, 3, _s(508, master), lo=0, hi=2556),
    }
    dim1 = {"key": Recipe(FMIX32_KEY, 3, key_seed=k1),
            "cat": Recipe(UNIFORM, 2, _s(509, master), lo=0, hi=999)}
    dim2 = {"key": Recipe(MIX64_KEY, 4, key_seed=k2),
            "cat": Recipe(UNIFORM, 1, _s(510, master), lo=0, hi=49)}
    return {"fact": fact, "dim1": dim1, "dim2": dim2}


# ---- string columns (Section 2.1: an (n x m) byte tensor, each UTF-8 value
# right-padded with zeros to m bytes)
EPOCH_DAY0 = 8035          # first day of the synthetic date range, in days since the UNIX epoch
SECONDS_PER_DAY = 86_400


def type_strings(width: int = 25, master: int = MASTER_SEED, slots=(6, 8, 5)):
    """Synthetic type names: one word per slot (4 to 7 uppercase letters,
    seeded), joined by single spaces; every combination of the slots' words,
    zero-padded to width bytes.  Returns (table [combinations, width] uint8,
    the words of each slot)."""
    words = []
    for si, count in enumerate(slots):
        u = draw(_s(600 + si, master), np.arange(count * 8, dtype=np.uint64)).reshape(count, 8)
        slot = []
        for w in range(count):
            length = 4 + int(u[w, 0] % np.uint64(4))
            slot.append(bytes(65 + int(u[w, 1 + j] % np.uint64(26)) for j in range(length)))
        words.append(slot)
    rows = [b" ".join(c) for c in itertools.product(*words)]
    assert max(len(r) for r in rows) <= width
    table = np.zeros((len(rows), width), np.uint8)
    for i, r in enumerate(rows):
        table[i, :len(r)] = np.frombuffer(r, np.uint8)
    return table, words


def type_column(n: int, seed: int, table: np.ndarray, start: int = 0) -> np.ndarray:
    """Rows [start, start + n): each row's type drawn uniformly from the table."""
    i = np.arange(start, start + n, dtype=np.uint64)
    return table[uniform_from(draw(seed, i), 0, len(table) - 1)]


def q14_promo_tables(m: int, master: int = MASTER_SEED):
    """The promotion-revenue shape of Q14: fact(fk int32 U[1, m], ship_ns
    int64 epoch nanoseconds at whole seconds over 2557 days, price int64
    U[90000, 10500000], disc int64 U[0, 10]) into dim(key int32 = seeded
    permutation of 1..m, type: 25-byte zero-padded strings).  The type column
    is drawn on the host (type_seed) from type_strings()."""
    s0 = EPOCH_DAY0 * SECONDS_PER_DAY
    fact = {
        "fk": Recipe(UNIFORM, 3, _s(611, master), lo=1, hi=m),
        "ship_ns": Recipe(UNIFORM, 4, _s(612, master), lo=s0, hi=s0 + 2557 * SECONDS_PER_DAY - 1, mul=10**9),
        "price": Recipe(UNIFORM, 4, _s(613, master), lo=90000, hi=10500000),
        "disc": Recipe(UNIFORM, 4, _s(614, master), lo=0, hi=10),
    }
    dim = {"key": Recipe(PERM_KEY, 3, key_seed=_s(615, master), m=m, lo=1)}
    return {"fact": fact, "dim": dim, "type_seed": _s(616, master)}


# ---- prediction query: reviews and a synthetic network
SCORE_BITS = 24  # score = score_q / 2^24, exact in float32


def reviews_table(master: int = MASTER_SEED):
    """reviews(score_q int32 U[0, 2^24 - 1] (the model input is score_q / 2^24),
    rating int8 U[1, 5], votes int32 U[0, 50])."""
    return {"score_q": Recipe(UNIFORM, 3, _s(621, master), lo=0, hi=(1 << SCORE_BITS) - 1),
            "rating": Recipe(UNIFORM, 1, _s(622, master), lo=1, hi=5),
            "votes": Recipe(UNIFORM, 3, _s(623, master), lo=0, hi=50)}


def predict_model(H: int = 64, master: int = MASTER_SEED):
    """Synthetic weights of the 1 -> H -> 1 monotone network (no trained
    model is used): unit j ramps over [k_j, k_j + 1/s_j] with a random knot
    k_j in [0, 1) and slope s_j in [2, 18); output weights a_j sum to about
    one.  Returns float32 (w, b, a, c)."""
    u = draw(_s(624, master), np.arange(3 * H, dtype=np.uint64)).reshape(3, H)
    f = (u >> np.uint64(40)).astype(np.float64) / float(1 << 24)
    w = (2.0 + 16.0 * f[0]).astype(np.float32)
    b = (-w.astype(np.float64) * f[1]).astype(np.float32)
    a = (2.0 * f[2] / H).astype(np.float32)
    return w, b, a, np.float32(0.0)


def make_table(recipes: dict, n: int, start: int = 0, zipf: np.ndarray | None = None) -> dict:
    return {name: generate(r, n, start, zipf) for name, r in recipes.items()}
