// Plain CPU oracle for the tensor query processor's relational core.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
// load this file or the library built from it; only the tests, the smoke
// check and the benchmark's CPU-baseline leg do.  It shares no code with the
// CUDA library: it is the slow, obviously correct statement of what every
// operator computes, against which the GPU results are compared bit for bit.
//
// The paper (Section 2.1) stores every column as an (n x 1) tensor of
// integers; Section 2.2 compiles relational operators (filter, join,
// aggregation) over such columns; Section 2.3 exercises filters plus an
// aggregation (TPC-H Q6) and a join plus an aggregation (Q14).  The paper
// gives no formal definitions, so each function below states the standard
// relational meaning it implements.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (no fast-math:
// the float model functions rely on IEEE round-to-nearest and on fmaf).
//
// Parity status: every function is pinned by the CPU tests (brute force on
// tiny tables, textbook library routines, invariants, closed forms,
// finite differences); none is unpinned.

#include <algorithm>
#include <climits>
#include <functional>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

namespace {

enum Dtype { I8 = 1, I16 = 2, I32 = 3, I64 = 4 };
enum Cmp { LT = 0, LE = 1, GT = 2, GE = 3, EQ = 4, NE = 5 };
enum AggOp { COUNT = 0, SUM = 1, MIN = 2, MAX = 3 };

int64_t load(const void* p, int dt, int64_t i) {
  switch (dt) {
    case I8: return static_cast<const int8_t*>(p)[i];
    case I16: return static_cast<const int16_t*>(p)[i];
    case I32: return static_cast<const int32_t*>(p)[i];
    default: return static_cast<const int64_t*>(p)[i];
  }
}

void store(void* p, int dt, int64_t i, int64_t v) {
  switch (dt) {
    case I8: static_cast<int8_t*>(p)[i] = static_cast<int8_t>(v); break;
    case I16: static_cast<int16_t*>(p)[i] = static_cast<int16_t>(v); break;
    case I32: static_cast<int32_t*>(p)[i] = static_cast<int32_t>(v); break;
    default: static_cast<int64_t*>(p)[i] = v; break;
  }
}

int width_bits(int dt) { return dt == I8 ? 8 : dt == I16 ? 16 : dt == I32 ? 32 : 64; }

bool compare(int64_t v, int op, int64_t lit) {
  switch (op) {
    case LT: return v < lit;
    case LE: return v <= lit;
    case GT: return v > lit;
    case GE: return v >= lit;
    case EQ: return v == lit;
    default: return v != lit;
  }
}

// Order-preserving unsigned image of a signed w-bit integer: flip the sign bit.
uint64_t order_bits(int64_t v, int dt) {
  int w = width_bits(dt);
  uint64_t mask = (w == 64) ? ~0ull : ((1ull << w) - 1);
  return (static_cast<uint64_t>(v) & mask) ^ (1ull << (w - 1));
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Filter (Section 2.2 relational filter; Section 2.3 "four filters" of Q6).
// Selected rows are those where every predicate holds (conjunction); each
// predicate compares the column's signed value with a 64-bit literal.  The
// result lists the selected row indices in ascending order.  Returns the count.
// ---------------------------------------------------------------------------
int64_t orc_filter(const void* const* cols, const int* dtypes, int64_t n, int npred,
                   const int* pred_col, const int* pred_op, const int64_t* pred_lit,
                   int32_t* out_idx) {
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    bool keep = true;
    for (int p = 0; p < npred; ++p) {
      int c = pred_col[p];
      if (!compare(load(cols[c], dtypes[c], i), pred_op[p], pred_lit[p])) keep = false;
    }
    if (keep) out_idx[k++] = static_cast<int32_t>(i);
  }
  return k;
}

// ---------------------------------------------------------------------------
// Stable sort of (key, value) pairs by bits [begin_bit, end_bit) of the
// order-preserving image of the signed key (the whole key when the range is
// the full width): ascending, ties keep input order.  std::stable_sort on an
// index permutation is the definition.
// ---------------------------------------------------------------------------
void orc_sort_pairs(const void* keys, int dt, const int32_t* vals, int64_t n, int begin_bit,
                    int end_bit, void* keys_out, int32_t* vals_out) {
  std::vector<int64_t> perm(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  int w = end_bit - begin_bit;
  uint64_t mask = (w >= 64) ? ~0ull : ((1ull << w) - 1);
  auto field = [&](int64_t i) { return (order_bits(load(keys, dt, i), dt) >> begin_bit) & mask; };
  std::stable_sort(perm.begin(), perm.end(),
                   [&](int64_t a, int64_t b) { return field(a) < field(b); });
  for (int64_t j = 0; j < n; ++j) {
    store(keys_out, dt, j, load(keys, dt, perm[j]));
    if (vals_out) vals_out[j] = vals ? vals[perm[j]] : static_cast<int32_t>(perm[j]);
  }
}

// ---------------------------------------------------------------------------
// Inner equi-join (Section 2.2 join; Section 2.3 Q14): every pair (i, j) with
// probe[i] == build[j], listed by ascending i and, for equal i, ascending j.
// A hash map from key to the ascending list of build rows, then one pass over
// the probe side in row order.  Returns the number of pairs (which may exceed
// cap; only the first cap pairs are written).
// ---------------------------------------------------------------------------
int64_t orc_join_eq(const void* probe, int pdt, int64_t np, const void* build, int bdt,
                    int64_t nb, int32_t* out_probe, int32_t* out_build, int64_t cap) {
  std::unordered_map<int64_t, std::vector<int32_t>> rows_of;
  rows_of.reserve(static_cast<size_t>(nb) * 2 + 1);
  for (int64_t j = 0; j < nb; ++j) rows_of[load(build, bdt, j)].push_back(static_cast<int32_t>(j));
  int64_t k = 0;
  for (int64_t i = 0; i < np; ++i) {
    auto it = rows_of.find(load(probe, pdt, i));
    if (it == rows_of.end()) continue;
    for (int32_t j : it->second) {
      if (k < cap) {
        out_probe[k] = static_cast<int32_t>(i);
        out_build[k] = j;
      }
      ++k;
    }
  }
  return k;
}

// ---------------------------------------------------------------------------
// Group-by aggregation (Section 2.2 aggregation; Section 2.3 Q6/Q14
// aggregates; Fig. 4's aggregation over an expression).
//
// Rows: sel[0..nsel) when sel is given, else 0..n-1.  Groups: the distinct
// tuples of key values over those rows, in ascending lexicographic signed
// order (std::map order); empty groups do not exist.  Value expressions:
// expr e is the product over its terms t of (mul[t] * col[t][row] + add[t]),
// evaluated per row in 64-bit two's complement.  Aggregates per group:
// COUNT (rows), SUM(expr) (wrapping mod 2^64), MIN(expr), MAX(expr).
//
// Outputs: out_keys[k * cap + g] (int64) for key column k, out_aggs[g * naggs
// + a].  Returns the group count G (only min(G, cap) groups are written).
// *overflow is set to 1 if any expression value or any SUM left the int64
// range, checked with a 128-bit shadow computation.
// ---------------------------------------------------------------------------
int64_t orc_groupby_agg(const void* const* key_cols, const int* key_dt, int nkeys,
                        const void* const* val_cols, const int* val_dt,
                        const int* expr_nterms, const int* term_col, const int64_t* term_mul,
                        const int64_t* term_add, int nexprs,  // terms: 3 slots per expr
                        const int* agg_op, const int* agg_expr, int naggs,
                        const int32_t* sel, int64_t n_rows, int64_t* out_keys, int64_t* out_aggs,
                        int64_t cap, int* overflow) {
  struct Acc {
    int64_t count = 0;
    std::vector<uint64_t> sum;
    std::vector<__int128> shadow;
    std::vector<int64_t> mn, mx;
  };
  std::map<std::vector<int64_t>, Acc> groups;
  *overflow = 0;
  std::vector<int64_t> key(static_cast<size_t>(nkeys));
  std::vector<int64_t> ev(static_cast<size_t>(nexprs));
  const __int128 lo64 = INT64_MIN, hi64 = INT64_MAX;
  for (int64_t r = 0; r < n_rows; ++r) {
    int64_t row = sel ? sel[r] : r;
    for (int k = 0; k < nkeys; ++k) key[k] = load(key_cols[k], key_dt[k], row);
    for (int e = 0; e < nexprs; ++e) {
      uint64_t v = 1;
      __int128 v128 = 1;
      for (int t = 0; t < expr_nterms[e]; ++t) {
        int c = term_col[e * 3 + t];
        int64_t x = load(val_cols[c], val_dt[c], row);
        uint64_t f = static_cast<uint64_t>(term_mul[e * 3 + t]) * static_cast<uint64_t>(x) +
                     static_cast<uint64_t>(term_add[e * 3 + t]);
        v *= f;
        v128 *= static_cast<__int128>(term_mul[e * 3 + t]) * x + term_add[e * 3 + t];
        if (v128 < lo64 || v128 > hi64) *overflow = 1;
      }
      ev[e] = static_cast<int64_t>(v);
    }
    Acc& acc = groups[key];
    if (acc.sum.empty()) {
      acc.sum.assign(naggs, 0);
      acc.shadow.assign(naggs, 0);
      acc.mn.assign(naggs, INT64_MAX);
      acc.mx.assign(naggs, INT64_MIN);
    }
    acc.count += 1;
    for (int a = 0; a < naggs; ++a) {
      if (agg_op[a] == COUNT) continue;
      int64_t x = ev[agg_expr[a]];
      acc.sum[a] += static_cast<uint64_t>(x);
      acc.shadow[a] += x;
      if (acc.shadow[a] < lo64 || acc.shadow[a] > hi64) *overflow = 1;
      acc.mn[a] = std::min(acc.mn[a], x);
      acc.mx[a] = std::max(acc.mx[a], x);
    }
  }
  int64_t g = 0;
  for (auto& kv : groups) {
    if (g < cap) {
      for (int k = 0; k < nkeys; ++k) out_keys[k * cap + g] = kv.first[k];
      for (int a = 0; a < naggs; ++a) {
        int64_t v;
        switch (agg_op[a]) {
          case COUNT: v = kv.second.count; break;
          case SUM: v = static_cast<int64_t>(kv.second.sum[a]); break;
          case MIN: v = kv.second.mn[a]; break;
          default: v = kv.second.mx[a]; break;
        }
        out_aggs[g * naggs + a] = v;
      }
    }
    ++g;
  }
  return g;
}

// ---------------------------------------------------------------------------
// Column gather: out[j] = col[idx[j]].
// ---------------------------------------------------------------------------
void orc_gather(const void* col, int dt, const int32_t* idx, int64_t n, void* out) {
  for (int64_t j = 0; j < n; ++j) store(out, dt, j, load(col, dt, idx[j]));
}

// ---------------------------------------------------------------------------
// Learned CDF model (the range partitioner).  The paper's third scenario
// (Section 3.3) runs neural-network inference inside the same tensor program
// as the relational operators; here a small network is trained on the key
// distribution and used to route rows to ordered buckets.
//
// Key normalisation: u = order-preserving image of the int64 key; q = (u -
// umin) >> shift (an integer below 2^24, so the conversion is exact);
// x = (float)q * inv, one IEEE single multiplication.  Non-decreasing in key.
//
// Model (H hidden units): z_j = fmaf(w_j, x, b_j); h_j = min(max(z_j, 0), 1);
// F = c, then F = fmaf(a_j, h_j, F) for j = 0..H-1 in that order.  With
// w_j >= 0 and a_j >= 0 every step is non-decreasing, so F is non-decreasing
// in x.  Bucket of a row: t = min(max(F, 0), 1) * B (single multiply),
// bucket = min(B - 1, (int)t).
// ---------------------------------------------------------------------------
void orc_cdf_normalize(const int64_t* keys, int64_t n, uint64_t umin, int shift, float inv,
                       float* x) {
  for (int64_t i = 0; i < n; ++i) {
    uint64_t u = static_cast<uint64_t>(keys[i]) ^ (1ull << 63);
    uint64_t q = (u - umin) >> shift;
    x[i] = static_cast<float>(q) * inv;
  }
}

void orc_cdf_forward_f32(const float* w, const float* b, const float* a, float c, int H,
                         const float* x, int64_t n, float* out) {
  for (int64_t i = 0; i < n; ++i) {
    float f = c;
    for (int j = 0; j < H; ++j) {
      float z = std::fmaf(w[j], x[i], b[j]);
      float h = std::fmin(std::fmax(z, 0.0f), 1.0f);
      f = std::fmaf(a[j], h, f);
    }
    out[i] = f;
  }
}

void orc_cdf_bucket(const float* F, int64_t n, int B, int32_t* bucket) {
  for (int64_t i = 0; i < n; ++i) {
    float t = std::fmin(std::fmax(F[i], 0.0f), 1.0f) * static_cast<float>(B);
    int b = static_cast<int>(t);
    bucket[i] = b < B - 1 ? b : B - 1;
  }
}

// The same network in float64 (no output clamp), for gradient checks.
void orc_cdf_forward_f64(const double* w, const double* b, const double* a, double c, int H,
                         const double* x, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    double f = c;
    for (int j = 0; j < H; ++j) {
      double z = w[j] * x[i] + b[j];
      double h = z < 0 ? 0 : (z > 1 ? 1 : z);
      f += a[j] * h;
    }
    out[i] = f;
  }
}

// Mean-squared-error loss L = (1/n) sum_i (F(x_i) - y_i)^2 and its gradient
// in float64.  dF/dc = 1; dF/da_j = h_j; where 0 < z_j < 1 (strictly),
// dF/db_j = a_j and dF/dw_j = a_j * x, else both 0 (the clamp is flat there;
// at the two kinks the one-sided derivative 0 is taken).  Returns L.
double orc_cdf_grad_f64(const double* w, const double* b, const double* a, double c, int H,
                        const double* x, const double* y, int64_t n, double* gw, double* gb,
                        double* ga, double* gc) {
  for (int j = 0; j < H; ++j) gw[j] = gb[j] = ga[j] = 0;
  *gc = 0;
  double loss = 0;
  std::vector<double> z(static_cast<size_t>(H)), h(static_cast<size_t>(H));
  for (int64_t i = 0; i < n; ++i) {
    double f = c;
    for (int j = 0; j < H; ++j) {
      z[j] = w[j] * x[i] + b[j];
      h[j] = z[j] < 0 ? 0 : (z[j] > 1 ? 1 : z[j]);
      f += a[j] * h[j];
    }
    double r = f - y[i];
    loss += r * r;
    double d = 2.0 * r / static_cast<double>(n);
    *gc += d;
    for (int j = 0; j < H; ++j) {
      ga[j] += d * h[j];
      if (z[j] > 0 && z[j] < 1) {
        gb[j] += d * a[j];
        gw[j] += d * a[j] * x[i];
      }
    }
  }
  return loss / static_cast<double>(n);
}

// One Adam step (Kingma & Ba 2015) on parameter vector p with gradient g,
// moments m and v, step number t >= 1, followed by the projection onto the
// constraint set: entries flagged in nonneg are clamped to >= 0.
void orc_adam_step_f64(double* p, const double* g, double* m, double* v, const int* nonneg,
                       int np, int t, double lr, double beta1, double beta2, double eps) {
  double c1 = 1.0 - std::pow(beta1, t), c2 = 1.0 - std::pow(beta2, t);
  for (int k = 0; k < np; ++k) {
    m[k] = beta1 * m[k] + (1 - beta1) * g[k];
    v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k];
    double mh = m[k] / c1, vh = v[k] / c2;
    p[k] -= lr * mh / (std::sqrt(vh) + eps);
    if (nonneg[k] && p[k] < 0) p[k] = 0;
  }
}

// Training targets from a sorted sample of S keys: each distinct key whose
// first occurrence is at rank r0 and which occurs c times gets the empirical
// CDF midpoint y = (r0 + c / 2) / S; every sample of that key carries it.
void orc_cdf_targets(const int64_t* sorted, int64_t S, double* y) {
  int64_t i = 0;
  while (i < S) {
    int64_t j = i;
    while (j < S && sorted[j] == sorted[i]) ++j;
    double t = (static_cast<double>(i) + 0.5 * static_cast<double>(j - i)) / static_cast<double>(S);
    for (int64_t k = i; k < j; ++k) y[k] = t;
    i = j;
  }
}

// Stable partition of rows by bucket id (a counting sort): rows of bucket 0
// first, then bucket 1, ..., each bucket in input order.  out_rows holds the
// row indices, offsets[b] the first position of bucket b (offsets[B] = n).
void orc_partition(const int32_t* bucket, int64_t n, int B, int32_t* out_rows, int64_t* offsets) {
  std::vector<int64_t> cnt(static_cast<size_t>(B) + 1, 0);
  for (int64_t i = 0; i < n; ++i) cnt[bucket[i] + 1]++;
  for (int b = 0; b < B; ++b) cnt[b + 1] += cnt[b];
  for (int b = 0; b <= B; ++b) offsets[b] = cnt[b];
  for (int64_t i = 0; i < n; ++i) out_rows[cnt[bucket[i]]++] = static_cast<int32_t>(i);
}

// String columns (Section 2.1): an (n x m) byte tensor, row i holding the
// UTF-8 bytes of value i right-padded with zeros to m bytes.  SQL
// `value LIKE 'p%'` for a prefix p of k bytes (no zero byte in p) holds when
// the value's first k bytes are p.  A value shorter than k bytes has a zero
// among them (its padding), which p lacks, so the byte comparison over the
// row is exact; k > m never matches, and the empty prefix matches every row.
void orc_like_prefix(const uint8_t* str, int64_t n, int m, const uint8_t* prefix, int k, int8_t* out) {
  for (int64_t i = 0; i < n; ++i) {
    bool match = k <= m;
    for (int j = 0; match && j < k; ++j) match = str[i * m + j] == prefix[j];
    out[i] = match ? 1 : 0;
  }
}

// Dictionary codes of a string column: code[i] = the rank of row i's value
// among the column's distinct values in ascending byte order (the zero
// padding sorts a value before every longer value it prefixes), and the
// number of distinct values.  Grouping by the code groups by the string.
int64_t orc_string_codes(const uint8_t* str, int64_t n, int m, int32_t* code) {
  std::map<std::vector<uint8_t>, int32_t> dict;
  for (int64_t i = 0; i < n; ++i) dict.emplace(std::vector<uint8_t>(str + i * m, str + (i + 1) * m), 0);
  int32_t next = 0;
  for (auto& kv : dict) kv.second = next++;
  for (int64_t i = 0; i < n; ++i) code[i] = dict[std::vector<uint8_t>(str + i * m, str + (i + 1) * m)];
  return (int64_t)dict.size();
}

// Training targets of the learned range partitioner when the sample's
// frequent ("heavy") keys are aggregated directly instead of routed through
// the buckets, so that the network is fit to the CDF of the rows the buckets
// receive (the light rows).  sorted: the sample's SH packed keys ascending.
//  - A run of c equal keys is heavy when c >= cut, where cut is the smallest
//    count >= min_count that at most max_heavy runs reach (no heavy key when
//    max_heavy == 0 or no such count exists).
//  - light(i) = the number of non-heavy sample keys before position i.
//  - Training pair t (t < S_train) takes sample position j = t * mult, whose
//    key k has its run [lo, hi): y[t] = (light(lo) + light count of the run
//    / 2) / (total light count), computed in double and rounded once to
//    float.  A heavy run has light count 0: it sits on the light CDF with
//    zero width.  Without heavy keys this is the plain empirical-CDF
//    midpoint (first rank + count / 2) / SH of orc_cdf_targets.
// heavy_out receives the heavy keys ascending; returns their number.
int64_t orc_light_cdf_targets(const uint64_t* sorted, int64_t SH, int64_t mult, int64_t S_train, int64_t min_count,
                              int64_t max_heavy, uint64_t* heavy_out, float* y) {
  // runs of equal keys
  std::vector<int64_t> run_lo, run_hi;
  for (int64_t i = 0; i < SH;) {
    int64_t j = i;
    while (j < SH && sorted[j] == sorted[i]) ++j;
    run_lo.push_back(i);
    run_hi.push_back(j);
    i = j;
  }
  // the count cut: walk the distinct counts from the largest down
  std::map<int64_t, int64_t, std::greater<int64_t>> by_count;
  for (size_t r = 0; r < run_lo.size(); ++r) by_count[run_hi[r] - run_lo[r]] += 1;
  int64_t cut = INT64_MAX, reached = 0;
  if (max_heavy > 0) {
    for (const auto& kv : by_count) {
      if (kv.first < min_count) break;
      if (reached + kv.second > max_heavy) break;
      reached += kv.second;
      cut = kv.first;
    }
  }
  std::vector<int64_t> light_before(static_cast<size_t>(SH) + 1, 0);
  int64_t nheavy = 0;
  for (size_t r = 0; r < run_lo.size(); ++r) {
    const int64_t c = run_hi[r] - run_lo[r];
    const bool heavy = c >= cut;
    if (heavy) heavy_out[nheavy++] = sorted[run_lo[r]];
    for (int64_t i = run_lo[r]; i < run_hi[r]; ++i)
      light_before[i + 1] = light_before[i] + (heavy ? 0 : 1);
  }
  const int64_t light_total = light_before[SH];
  const double tot = light_total > 0 ? static_cast<double>(light_total) : 1.0;
  for (int64_t t = 0; t < S_train; ++t) {
    const int64_t j = t * mult;
    // the run holding j: the last run starting at or before j
    const size_t r = static_cast<size_t>(std::upper_bound(run_lo.begin(), run_lo.end(), j) - run_lo.begin()) - 1;
    const int64_t lo = run_lo[r], hi = run_hi[r];
    const int64_t light = light_before[hi] - light_before[lo];
    y[t] = static_cast<float>((static_cast<double>(light_before[lo]) + 0.5 * static_cast<double>(light)) / tot);
  }
  return nheavy;
}

// Date columns (Section 2.1): a date is stored as its UNIX epoch time in
// nanoseconds, an int64 (n x 1) tensor.  Dates here are days of the
// proleptic Gregorian calendar; an int64 nanosecond count reaches from
// 1677-09-22 to 2262-04-11, so only days in [-106751, 106751] relative to
// 1970-01-01 convert.  The oracle counts days by walking years and months
// one by one with the leap-year rule (divisible by 4, except centuries not
// divisible by 400).
}  // extern "C"
namespace {
bool leap_year(int64_t y) { return (y % 4 == 0 && y % 100 != 0) || y % 400 == 0; }
int days_in_month(int64_t y, int m) {
  static const int d[12] = {31, 28, 31, 30, 31, 30, 31, 31, 30, 31, 30, 31};
  return m == 2 && leap_year(y) ? 29 : d[m - 1];
}
constexpr int64_t kNsPerDay = 86400LL * 1000000000LL;
constexpr int64_t kMinDay = -106751, kMaxDay = 106751;  // whole days whose nanoseconds fit in int64

// Days from 1970-01-01 to y-m-d (1 <= m <= 12, 1 <= d <= days in month).
int64_t days_of(int64_t y, int m, int d) {
  int64_t days = 0;
  if (y >= 1970) {
    for (int64_t k = 1970; k < y; ++k) days += leap_year(k) ? 366 : 365;
  } else {
    for (int64_t k = y; k < 1970; ++k) days -= leap_year(k) ? 366 : 365;
  }
  for (int k = 1; k < m; ++k) days += days_in_month(y, k);
  return days + (d - 1);
}
}  // namespace
extern "C" {

// Parses row i of an (n x m) zero-padded string tensor as an ISO date
// "YYYY-MM-DD" (exactly 10 bytes, then only zero padding): ns[i] = the
// date's epoch nanoseconds and ok[i] = 1; a malformed or out-of-range row
// gives ns[i] = INT64_MIN and ok[i] = 0.  Returns the number of bad rows.
int64_t orc_date_parse_iso(const uint8_t* str, int64_t n, int m, int64_t* ns, int8_t* ok) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    const uint8_t* r = str + i * m;
    bool good = m >= 10 && r[4] == '-' && r[7] == '-';
    int v[8] = {0};
    const int at[8] = {0, 1, 2, 3, 5, 6, 8, 9};
    for (int k = 0; good && k < 8; ++k) {
      const uint8_t c = r[at[k]];
      good = c >= '0' && c <= '9';
      v[k] = c - '0';
    }
    for (int k = 10; good && k < m; ++k) good = r[k] == 0;
    int64_t y = 0;
    int mo = 0, d = 0;
    if (good) {
      y = v[0] * 1000 + v[1] * 100 + v[2] * 10 + v[3];
      mo = v[4] * 10 + v[5];
      d = v[6] * 10 + v[7];
      good = mo >= 1 && mo <= 12 && d >= 1 && d <= days_in_month(y, mo);
    }
    int64_t days = good ? days_of(y, mo, d) : 0;
    good = good && days >= kMinDay && days <= kMaxDay;
    ns[i] = good ? days * kNsPerDay : INT64_MIN;
    ok[i] = good ? 1 : 0;
    bad += good ? 0 : 1;
  }
  return bad;
}

// Day numbers (days since 1970-01-01, int32) to epoch nanoseconds; a day
// outside [-106751, 106751] gives INT64_MIN and counts as bad.
int64_t orc_date_from_days(const int32_t* days, int64_t n, int64_t* ns) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    const bool good = days[i] >= kMinDay && days[i] <= kMaxDay;
    ns[i] = good ? static_cast<int64_t>(days[i]) * kNsPerDay : INT64_MIN;
    bad += good ? 0 : 1;
  }
  return bad;
}

// Epoch nanoseconds to the calendar: the day number (floor of ns / one
// day, so an instant before 1970 belongs to the earlier day), and that
// day's year, month and day of month, found by walking from 1970.
void orc_date_parts(const int64_t* ns, int64_t n, int32_t* days, int32_t* year, int32_t* month, int32_t* mday) {
  for (int64_t i = 0; i < n; ++i) {
    int64_t q = ns[i] / kNsPerDay;
    if (ns[i] % kNsPerDay != 0 && ns[i] < 0) q -= 1;
    int64_t y = 1970, rest = q;
    while (rest < 0) {
      y -= 1;
      rest += leap_year(y) ? 366 : 365;
    }
    while (rest >= (leap_year(y) ? 366 : 365)) {
      rest -= leap_year(y) ? 366 : 365;
      y += 1;
    }
    int m = 1;
    while (rest >= days_in_month(y, m)) {
      rest -= days_in_month(y, m);
      ++m;
    }
    days[i] = static_cast<int32_t>(q);
    year[i] = static_cast<int32_t>(y);
    month[i] = m;
    mday[i] = static_cast<int32_t>(rest + 1);
  }
}

}  // extern "C"
