// Sort-based group-by aggregation.
//
// 1. key range: per key column min and max over the rows (one read);
// 2. plan: each column is trimmed to its range and the columns are packed
//    lexicographically (first key column in the high bits) into one
//    order-preserving unsigned word;
// 3. encode: packed key + row id per row;
// 4. stable radix sort of (packed key, row id) -- the passes over constant
//    high digits are skipped by the sort itself;
// 5. reduce-by-key: segment heads are the adjacent differences of the sorted
//    keys; a single-pass segmented scan with decoupled look-back carries the
//    open segment's partial aggregates across tiles, so every group is
//    written exactly once, by the thread holding its last row, with plain
//    stores.  Aggregates are exact 64-bit integers (SUM/COUNT wrap mod 2^64).
#pragma once

#include "common.cuh"
#include "sort.cuh"

namespace tqp {

struct KeySet {
  int nkeys;
  const void* col[TQP_MAX_KEYS];
  int dt[TQP_MAX_KEYS];
  void* out[TQP_MAX_KEYS];
};

struct GroupPlan {
  long long kmin[TQP_MAX_KEYS];
  long long kmax[TQP_MAX_KEYS];
  int shift[TQP_MAX_KEYS];
  int bits[TQP_MAX_KEYS];
  int total_bits;
  int unsupported;
};

struct AggProgram {
  int naggs;
  int op[TQP_MAX_AGGS];
  int expr[TQP_MAX_AGGS];
  int nexprs;
  int nterms[TQP_MAX_EXPRS];
  int tcol[TQP_MAX_EXPRS][3];
  long long tmul[TQP_MAX_EXPRS][3];
  long long tadd[TQP_MAX_EXPRS][3];
  int nvals;
  const void* val[TQP_MAX_VALS];
  int vdt[TQP_MAX_VALS];
  int simple;  // every aggregate is COUNT or one column read as is
};

// ---------------------------------------------------------------- aggregates
template <int N>
struct PartialT {
  long long v[N];
  int c;  // segment heads inside the span
};
using Partial = PartialT<TQP_MAX_AGGS>;  // storage layout of the per-tile carries

__device__ __forceinline__ long long agg_identity(int op) {
  return op == TQP_MIN ? LLONG_MAX : (op == TQP_MAX ? LLONG_MIN : 0ll);
}

__device__ __forceinline__ long long agg_fold(int op, long long acc, long long x) {
  switch (op) {
    case TQP_MIN: return x < acc ? x : acc;
    case TQP_MAX: return x > acc ? x : acc;
    default: return (long long)((unsigned long long)acc + (unsigned long long)x);
  }
}

template <int N>
__device__ __forceinline__ void partial_identity(PartialT<N>& p, const AggProgram& P) {
#pragma unroll
  for (int a = 0; a < N; ++a) p.v[a] = (a < P.naggs) ? agg_identity(P.op[a]) : 0;
  p.c = 0;
}

// Expression e at row: product of (mul * val + add) over its terms, mod 2^64.
__device__ __forceinline__ long long eval_expr(const AggProgram& P, int e, int64_t row) {
  unsigned long long v = 1;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t < P.nterms[e]) {
      int c = P.tcol[e][t];
      long long x = load_as_i64(P.val[c], P.vdt[c], row);
      v *= (unsigned long long)P.tmul[e][t] * (unsigned long long)x + (unsigned long long)P.tadd[e][t];
    }
  }
  return (long long)v;
}

template <int N>
__device__ __forceinline__ void fold_row(PartialT<N>& p, const AggProgram& P, int64_t row) {
  // each aggregate evaluates its own expression (a value shared by several
  // aggregates is re-read from L1)
#pragma unroll
  for (int a = 0; a < N; ++a) {
    if (a < P.naggs) {
      long long x = P.op[a] == TQP_COUNT ? 1 : eval_expr(P, P.expr[a], row);
      p.v[a] = agg_fold(P.op[a], p.v[a], x);
    }
  }
}

// ---------------------------------------------------------------- key plan
__global__ void gb_init_kernel(GroupPlan* plan) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < TQP_MAX_KEYS; ++k) {
      plan->kmin[k] = LLONG_MAX;
      plan->kmax[k] = LLONG_MIN;
      plan->shift[k] = plan->bits[k] = 0;
    }
    plan->total_bits = 0;
    plan->unsupported = 0;
  }
}

// Minimum and maximum of one column of T over rows i = first + j * stride,
// eight rows a thread in flight (independent loads issued together).
template <typename T>
__device__ __forceinline__ void column_range(const T* col, int64_t n, int64_t first, int64_t stride, long long* mn,
                                             long long* mx) {
  constexpr int U = 8;
  for (int64_t base = first; base < n; base += stride * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * stride;
      v[u] = i < n ? __ldg(col + i) : __ldg(col + base);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long x = (long long)v[u];
      *mn = x < *mn ? x : *mn;
      *mx = x > *mx ? x : *mx;
    }
  }
}

// The same for a 1- or 2-byte column at a 16-byte aligned address: 16-byte
// words, four in flight per thread (a byte load per row would leave too few
// bytes in flight to stream the column), then the scalar tail.
template <typename T>
__device__ __forceinline__ void column_range_narrow(const T* col, int64_t n, int64_t first, int64_t stride,
                                                    long long* mn, long long* mx) {
  constexpr int PER = 16 / sizeof(T);
  constexpr int U = 4;
  const int64_t nw = n / PER;
  const int4* w = reinterpret_cast<const int4*>(col);
  int lo = INT_MAX, hi = INT_MIN;
  for (int64_t base = first; base < nw; base += stride * U) {
    int4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * stride;
      v[u] = __ldg(w + (i < nw ? i : base));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T* e = reinterpret_cast<const T*>(&v[u]);
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int x = (int)e[j];
        lo = x < lo ? x : lo;
        hi = x > hi ? x : hi;
      }
    }
  }
  for (int64_t i = nw * PER + first; i < n; i += stride) {
    const int x = (int)__ldg(col + i);
    lo = x < lo ? x : lo;
    hi = x > hi ? x : hi;
  }
  if (lo != INT_MAX) {
    *mn = (long long)lo < *mn ? (long long)lo : *mn;
    *mx = (long long)hi > *mx ? (long long)hi : *mx;
  }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) gb_keyrange_kernel(KeySet ks, const int32_t* sel, int64_t n_max,
                                                              const int64_t* d_n, GroupPlan* plan) {
  __shared__ long long s_min[THREADS / 32][TQP_MAX_KEYS], s_max[THREADS / 32][TQP_MAX_KEYS];
  const int64_t n = clamp_n(n_max, d_n);
  long long mn[TQP_MAX_KEYS], mx[TQP_MAX_KEYS];
#pragma unroll
  for (int k = 0; k < TQP_MAX_KEYS; ++k) { mn[k] = LLONG_MAX; mx[k] = LLONG_MIN; }
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  const int64_t first = (int64_t)blockIdx.x * THREADS + threadIdx.x;
  if (ks.nkeys == 1 && sel == nullptr) {
    // one column over every row: typed loads, several in flight
    switch (ks.dt[0]) {
      case TQP_I8:
        if (((uintptr_t)ks.col[0] & 15) == 0)
          column_range_narrow(static_cast<const signed char*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]);
        else
          column_range(static_cast<const signed char*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]);
        break;
      case TQP_I16:
        if (((uintptr_t)ks.col[0] & 15) == 0)
          column_range_narrow(static_cast<const short*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]);
        else
          column_range(static_cast<const short*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]);
        break;
      case TQP_I32: column_range(static_cast<const int*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]); break;
      default: column_range(static_cast<const long long*>(ks.col[0]), n, first, stride, &mn[0], &mx[0]); break;
    }
  }
  for (int64_t i = first; i < n && !(ks.nkeys == 1 && sel == nullptr); i += stride) {
    int64_t row = sel ? sel[i] : i;
#pragma unroll
    for (int k = 0; k < TQP_MAX_KEYS; ++k) {
      if (k < ks.nkeys) {
        long long v = load_as_i64(ks.col[k], ks.dt[k], row);
        mn[k] = v < mn[k] ? v : mn[k];
        mx[k] = v > mx[k] ? v : mx[k];
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < TQP_MAX_KEYS; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long a = __shfl_xor_sync(0xffffffffu, mn[k], o), b = __shfl_xor_sync(0xffffffffu, mx[k], o);
      mn[k] = a < mn[k] ? a : mn[k];
      mx[k] = b > mx[k] ? b : mx[k];
    }
    if (lane == 0) { s_min[warp][k] = mn[k]; s_max[warp][k] = mx[k]; }
  }
  __syncthreads();
  if (threadIdx.x < ks.nkeys) {
    int k = threadIdx.x;
    long long a = LLONG_MAX, b = LLONG_MIN;
    for (int w = 0; w < THREADS / 32; ++w) {
      a = s_min[w][k] < a ? s_min[w][k] : a;
      b = s_max[w][k] > b ? s_max[w][k] : b;
    }
    if (a != LLONG_MAX) atomicMin(&plan->kmin[k], a);
    if (b != LLONG_MIN) atomicMax(&plan->kmax[k], b);
  }
}

__global__ void gb_plan_kernel(GroupPlan* plan, int nkeys, int word_bits) {
  if (threadIdx.x != 0) return;
  int shift = 0;
  for (int k = nkeys - 1; k >= 0; --k) {
    int b = 0;
    if (plan->kmax[k] > plan->kmin[k]) {
      unsigned long long span = (unsigned long long)plan->kmax[k] - (unsigned long long)plan->kmin[k];
      b = 64 - __clzll((long long)span);
    }
    plan->bits[k] = b;
    plan->shift[k] = shift;
    shift += b;
  }
  plan->total_bits = shift;
  if (shift > word_bits) {
    plan->unsupported = 1;
    raise_status(TQP_ERR_UNSUPPORTED);
  }
}

template <typename K>
__global__ void gb_encode_kernel(KeySet ks, const int32_t* sel, int64_t n_max, const int64_t* d_n,
                                 const GroupPlan* plan, K* packed, int32_t* rows) {
  const int64_t n = clamp_n(n_max, d_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  long long kmin[TQP_MAX_KEYS];
  int shift[TQP_MAX_KEYS];
#pragma unroll
  for (int k = 0; k < TQP_MAX_KEYS; ++k) {
    kmin[k] = plan->kmin[k];
    shift[k] = plan->shift[k];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t row = sel ? sel[i] : i;
    unsigned long long u = 0;
#pragma unroll
    for (int k = 0; k < TQP_MAX_KEYS; ++k)
      if (k < ks.nkeys)
        u |= ((unsigned long long)load_as_i64(ks.col[k], ks.dt[k], row) - (unsigned long long)kmin[k]) << shift[k];
    packed[i] = (K)u;
    rows[i] = (int32_t)row;
  }
}

// ---------------------------------------------------------------- reduce-by-key
struct ReduceArgs {
  const void* keys;        // sorted packed keys (K words)
  const int32_t* rows;     // sorted row ids
  int64_t n_max;
  const int64_t* d_n;
  const GroupPlan* plan;
  KeySet ks;
  long long* out_aggs;
  int64_t cap;
  int64_t* d_out_groups;
  uint32_t* tile_heads;    // [num_tiles] segment heads per tile, then the heads before each tile
  Partial* carry;          // [num_tiles] partial of the rows before each tile's first head (c = 1: present)
  uint32_t num_tiles;
  // keys aggregated outside the sorted rows (learned path), merged in key
  // order: sorted packed keys, their count (device) and aggregates [nh][naggs]
  const unsigned long long* heavy;
  const int* d_nheavy;
  const long long* heavy_acc;
};

// Writes the key columns of group g, decoded from the packed word.
__device__ __forceinline__ void write_group_keys(const KeySet& ks, const GroupPlan* plan, long long g,
                                                 unsigned long long u) {
  for (int j = 0; j < ks.nkeys; ++j) {
    int b = plan->bits[j];
    unsigned long long m = b >= 64 ? ~0ull : ((1ull << b) - 1);
    long long kv = (long long)(((u >> plan->shift[j]) & m) + (unsigned long long)plan->kmin[j]);
    store_from_i64(ks.out[j], ks.dt[j], g, kv);
  }
}

// Writes group g: key columns and aggregates (from memory).
__device__ __forceinline__ void write_group(const ReduceArgs& a, const KeySet& ks, int naggs, long long g,
                                            unsigned long long u, const long long* v) {
  if (g < 0 || g >= a.cap) return;
  write_group_keys(ks, a.plan, g, u);
  for (int q = 0; q < naggs; ++q) a.out_aggs[g * naggs + q] = v[q];
}

// Writes group g: key columns and aggregates (from registers).
template <int N>
__device__ __forceinline__ void write_group_regs(const ReduceArgs& a, const KeySet& ks, int naggs, long long g,
                                                 unsigned long long u, const PartialT<N>& r) {
  if (g < 0 || g >= a.cap) return;
  write_group_keys(ks, a.plan, g, u);
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q < naggs) a.out_aggs[g * naggs + q] = r.v[q];
}

// Heavy groups when no row went through the sort: group i at position i
// (the reduce kernel then writes the group count, nh).
__global__ void gb_heavy_only_kernel(ReduceArgs a, int naggs) {
  if (a.plan->unsupported || clamp_n(a.n_max, a.d_n) > 0) return;
  const int nh = a.d_nheavy ? *a.d_nheavy : 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += gridDim.x * blockDim.x)
    write_group(a, a.ks, naggs, i, a.heavy[i], a.heavy_acc + (size_t)i * naggs);
}

// ---------------------------------------------------------------- reduce by key
// Reduce-by-key over the sorted packed keys in four launches, none of which
// waits on another block:
//   gb_heads_kernel      segment heads per tile of TILE rows;
//   gb_tile_scan_kernel  exclusive scan of the tiles' head counts (the light
//                        index of each tile's first group) and the total;
//   gb_reduce_kernel     per tile: every thread folds its ITEMS consecutive
//                        rows and stores each group whose head it holds; the
//                        rows before its first head (its lead) belong to an
//                        earlier group: after a block barrier they are
//                        combined atomically into that group's output when
//                        it started in this tile, else into the tile's carry;
//   gb_carry_kernel      each tile's carry combined atomically into the group
//                        that reaches into the tile from before.
// SUM wraps mod 2^64 and MIN / MAX / COUNT commute, so the atomic
// combinations give exactly the sequential result.  Keys aggregated outside
// the rows (heavy keys of the learned path) interleave in key order: a light
// group of light index g and key k goes to g + (heavy keys below k), heavy
// key i between the light groups g-1 and g to g + i.
constexpr int kReduceHeavyMax = 1024;  // heavy keys merged by the reduce

template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) gb_heads_kernel(ReduceArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_red[THREADS / 32];
  const int64_t n = a.plan->unsupported ? 0 : clamp_n(a.n_max, a.d_n);
  const K* keys = static_cast<const K*>(a.keys);
  for (int64_t t = blockIdx.x; t < (int64_t)a.num_tiles; t += gridDim.x) {
    int h = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t p = t * TILE + (int64_t)k * THREADS + threadIdx.x;
      if (p < n) h += (p == 0 || keys[p] != keys[p - 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < THREADS / 32; ++w) tot += s_red[w];
      a.tile_heads[t] = (uint32_t)tot;
    }
    __syncthreads();
  }
}

// One block of 1024 threads: flags[t] becomes the heads before tile t; the
// group count (light groups + heavy keys) goes to d_out_groups.
__global__ void __launch_bounds__(1024) gb_tile_scan_kernel(ReduceArgs a) {
  __shared__ int s_scan[33];
  const int64_t T = a.num_tiles;
  const int64_t per = (T + 1023) / 1024;
  const int64_t t0 = threadIdx.x * per;
  long long sum = 0;
  for (int64_t t = t0; t < t0 + per && t < T; ++t) sum += a.tile_heads[t];
  int total;
  long long run = block_exclusive_sum<1024>((int)sum, s_scan, &total);
  for (int64_t t = t0; t < t0 + per && t < T; ++t) {
    const uint32_t c = a.tile_heads[t];
    a.tile_heads[t] = (uint32_t)run;
    run += c;
  }
  if (threadIdx.x == 0) {
    const int nh = (a.heavy && a.d_nheavy) ? *a.d_nheavy : 0;
    const long long g = (long long)total + nh;
    *a.d_out_groups = g;
    if (g > a.cap) raise_status(TQP_ERR_CAPACITY);
  }
}

// Heavy keys below x (s_heavy ascending, nh entries).
template <typename K>
__device__ __forceinline__ int heavy_below(const unsigned long long* h, int nh, K x) {
  int lo = 0, len = nh;
  while (len > 0) {
    const int half = len >> 1;
    if (h[lo + half] < (unsigned long long)x) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

// Combines the partial p into the output of group g with atomics.
template <int N>
__device__ __forceinline__ void combine_group_atomic(const ReduceArgs& a, const AggProgram& P, long long g,
                                                     const PartialT<N>& p) {
  if (g < 0 || g >= a.cap) return;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    if (q >= P.naggs) break;
    long long* d = a.out_aggs + g * P.naggs + q;
    switch (P.op[q]) {
      case TQP_MIN: atomicMin(d, p.v[q]); break;
      case TQP_MAX: atomicMax(d, p.v[q]); break;
      default: atomicAdd(reinterpret_cast<unsigned long long*>(d), (unsigned long long)p.v[q]); break;
    }
  }
}

template <typename K, int THREADS, int ITEMS, int NAGG>
__global__ void __launch_bounds__(THREADS) gb_reduce_kernel(ReduceArgs a, AggProgram Pg) {
  constexpr int TILE = THREADS * ITEMS;
  using PT = PartialT<NAGG>;
  __shared__ AggProgram P;  // the program and the key set in shared memory: indexed by runtime values below
  __shared__ KeySet s_ks;
  __shared__ int s_scan[33];
  __shared__ long long s_carry[NAGG];
  __shared__ int s_carry_used;
  __shared__ unsigned long long s_heavy[kReduceHeavyMax];
  __shared__ long long s_val[ITEMS][THREADS];  // gathered values, [item][thread]
  if (threadIdx.x == 0) {
    P = Pg;
    s_ks = a.ks;
  }
  const int nh = (a.heavy && a.d_nheavy) ? *a.d_nheavy : 0;
  for (int i = threadIdx.x; i < nh; i += THREADS) s_heavy[i] = a.heavy[i];
  __syncthreads();
  const int64_t n = a.plan->unsupported ? 0 : clamp_n(a.n_max, a.d_n);
  const K* keys = static_cast<const K*>(a.keys);
  const int32_t* rows = a.rows;  // null: the value columns are already in sorted order
  // a simple program in registers: each aggregate's op and column
  const bool simple = P.simple != 0;
  int qop[NAGG], qdt[NAGG];
  const void* qcol[NAGG];
#pragma unroll
  for (int q = 0; q < NAGG; ++q) {
    qop[q] = q < P.naggs ? P.op[q] : TQP_COUNT;
    const int c = (q < P.naggs && qop[q] != TQP_COUNT) ? P.tcol[P.expr[q]][0] : 0;
    qcol[q] = P.nvals ? P.val[c] : nullptr;
    qdt[q] = P.nvals ? P.vdt[c] : TQP_I64;
  }
  // one value column read through the row ids: the thread's values are
  // gathered into shared memory first, their reads in flight together
  const bool gather = simple && rows != nullptr && P.nvals == 1;
  auto fold = [&](PT& acc, int64_t r, int k) {
    if (gather) {
      const long long v = s_val[k][threadIdx.x];
#pragma unroll
      for (int q = 0; q < NAGG; ++q)
        if (q < P.naggs) acc.v[q] = agg_fold(qop[q], acc.v[q], qop[q] == TQP_COUNT ? 1 : v);
    } else if (simple) {
#pragma unroll
      for (int q = 0; q < NAGG; ++q)
        if (q < P.naggs) acc.v[q] = agg_fold(qop[q], acc.v[q], qop[q] == TQP_COUNT ? 1 : load_as_i64(qcol[q], qdt[q], r));
    } else {
      fold_row(acc, P, r);
    }
  };

  for (int64_t t = blockIdx.x; t < (int64_t)a.num_tiles; t += gridDim.x) {
    if (threadIdx.x == 0) s_carry_used = 0;
    if (threadIdx.x < NAGG) s_carry[threadIdx.x] = threadIdx.x < P.naggs ? agg_identity(P.op[threadIdx.x]) : 0;
    const int64_t base = t * TILE + (int64_t)threadIdx.x * ITEMS;
    // ---- segment heads of the thread's rows
    uint32_t head = 0;
    const K prev = (base > 0 && base < n) ? keys[base - 1] : (K)0;
    {
      K pk = prev;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int64_t p = base + k;
        const K kk = p < n ? keys[p] : (K)0;
        if (p < n && (p == 0 || kk != pk)) head |= 1u << k;
        pk = kk;
      }
    }
    const K key0 = base < n ? keys[base] : (K)0;
    if (gather) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        s_val[k][threadIdx.x] = base + k < n ? load_as_i64(P.val[0], P.vdt[0], rows[base + k]) : 0;
    }
    int tile_heads;
    const int before = block_exclusive_sum<THREADS>(__popc(head), s_scan, &tile_heads);
    const long long g0 = (long long)a.tile_heads[t] + before;  // light index of the thread's first head
    // ---- fold, storing every group whose head this thread holds
    PT acc, lead;
    partial_identity(acc, P);
    partial_identity(lead, P);
    bool lead_open = true;  // rows so far belong to a group from before this thread
    long long g = g0 - 1;
    int hl = (nh && base < n) ? heavy_below(s_heavy, nh, base > 0 ? prev : key0) : 0;  // heavy keys below the current key
    K gkey = 0;
#pragma unroll 1
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t p = base + k;
      if (p < n) {
        if (head & (1u << k)) {
          const K kk = keys[p];
          if (lead_open) {
            lead = acc;
            lead_open = false;
          } else {
            write_group_regs(a, s_ks, P.naggs, g + hl, (unsigned long long)gkey, acc);
          }
          ++g;
          gkey = kk;
          partial_identity(acc, P);
          if (nh) {
            // heavy keys between the previous row's key and this one go just before this group
            const int hl_new = heavy_below(s_heavy, nh, kk);
            for (int i = (p == 0 ? 0 : hl); i < hl_new; ++i)
              write_group(a, s_ks, P.naggs, g + i, s_heavy[i], a.heavy_acc + (size_t)i * P.naggs);
            hl = hl_new;
          }
        }
        fold(acc, rows ? rows[p] : p, k);
        if (nh && p == n - 1) {
          // heavy keys above the last light key
          for (int i = hl; i < nh; ++i)
            write_group(a, s_ks, P.naggs, g + 1 + i, s_heavy[i], a.heavy_acc + (size_t)i * P.naggs);
        }
      }
    }
    const bool has_rows = base < n;
    if (has_rows && !lead_open) write_group_regs(a, s_ks, P.naggs, g + hl, (unsigned long long)gkey, acc);
    if (lead_open) lead = acc;
    const bool has_lead = has_rows && !(head & 1u);
    __syncthreads();  // every group stored by its head's thread
    if (has_lead) {
      if (before > 0) {
        // the group started earlier in this tile
        const int hl0 = nh ? heavy_below(s_heavy, nh, key0) : 0;
        combine_group_atomic(a, P, g0 - 1 + hl0, lead);
      } else {
        // the group reaches into this tile from before: the tile's carry
#pragma unroll
        for (int q = 0; q < NAGG; ++q) {
          if (q >= P.naggs) break;
          long long* d = &s_carry[q];
          switch (P.op[q]) {
            case TQP_MIN: atomicMin(d, lead.v[q]); break;
            case TQP_MAX: atomicMax(d, lead.v[q]); break;
            default: shared_add_u64(reinterpret_cast<unsigned long long*>(d), (unsigned long long)lead.v[q]); break;
          }
        }
        s_carry_used = 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Partial c;
      for (int q = 0; q < TQP_MAX_AGGS; ++q) c.v[q] = q < NAGG ? s_carry[q < NAGG ? q : 0] : 0;
      c.c = s_carry_used;
      a.carry[t] = c;
    }
    __syncthreads();  // the carry is read before the next tile resets it
  }
}

// Each tile's carry into the group that reaches into it from before (the
// light group just before the tile's first head).
template <typename K, int THREADS, int ITEMS>
__global__ void gb_carry_kernel(ReduceArgs a, AggProgram P) {
  constexpr int TILE = THREADS * ITEMS;
  const int nh = (a.heavy && a.d_nheavy) ? *a.d_nheavy : 0;
  const K* keys = static_cast<const K*>(a.keys);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)a.num_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Partial& c = a.carry[t];
    if (!c.c) continue;
    const K k0 = keys[t * TILE];
    const long long g = (long long)a.tile_heads[t] - 1 + (nh ? heavy_below(a.heavy, nh, k0) : 0);
    if (g < 0 || g >= a.cap) continue;
    for (int q = 0; q < P.naggs; ++q) {
      long long* d = a.out_aggs + g * P.naggs + q;
      switch (P.op[q]) {
        case TQP_MIN: atomicMin(d, c.v[q]); break;
        case TQP_MAX: atomicMax(d, c.v[q]); break;
        default: atomicAdd(reinterpret_cast<unsigned long long*>(d), (unsigned long long)c.v[q]); break;
      }
    }
  }
}

// ---------------------------------------------------------------- small key domains
// When the packed group key spans at most 2^kDirectBits values (a handful
// of flags, a rating, a region), the packed key is itself the group's slot
// in key order: the rows fold straight into per-warp slot accumulators in
// shared memory, with no sort.  The decision is the device's (the packed
// width is known only after the key range pass); the sort path then runs
// on no rows.
constexpr int kDirectBits = 10;
constexpr int kDirectSlots = 1 << kDirectBits;
constexpr int kDirectMaxSmemBytes = kDirectSlots * (TQP_MAX_AGGS + 1) * 8;  // one copy of the widest program

// One thread: direct[0] = 1 when the packed key fits the slots; sort_n:
// the rows the sort path then takes (0 when direct).
__global__ void gb_direct_plan_kernel(const GroupPlan* plan, int64_t n_max, const int64_t* d_n, int* direct,
                                      int64_t* sort_n) {
  if (threadIdx.x != 0) return;
  const int64_t n = clamp_n(n_max, d_n);
  const int on = n > 0 && !plan->unsupported && plan->total_bits <= kDirectBits;
  *direct = on;
  *sort_n = on ? 0 : n;
}

// Identity of every accumulator (naggs aggregates + the row count) of every slot.
__global__ void gb_direct_init_kernel(const int* direct, AggProgram P, long long* acc) {
  if (!*direct) return;
  const int nacc = P.naggs + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kDirectSlots * nacc; i += gridDim.x * blockDim.x) {
    const int q = i % nacc;
    acc[i] = q < P.naggs ? agg_identity(P.op[q]) : 0;
  }
}

__device__ __forceinline__ void direct_fold(long long* slot, int op, long long x, bool shared) {
  switch (op) {
    case TQP_MIN: atomicMin(slot, x); break;
    case TQP_MAX: atomicMax(slot, x); break;
    default:
      if (shared) shared_add_u64(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)x);
      else atomicAdd(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)x);
      break;
  }
}

// Rows fold into one accumulator copy per warp (as many copies as fit in
// smem_bytes, which holds at least one copy of all 2^kDirectBits slots),
// merged into the global slots at the end.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) gb_direct_kernel(KeySet ks, const int32_t* sel, int64_t n_max,
                                                            const int64_t* d_n, const GroupPlan* plan,
                                                            AggProgram Pg, const int* direct, long long* acc,
                                                            int smem_bytes) {
  extern __shared__ long long s_dacc[];
  __shared__ long long s_kmin[TQP_MAX_KEYS];
  __shared__ int s_shift[TQP_MAX_KEYS];
  __shared__ AggProgram P;  // indexed by runtime values: kept in shared memory
  __shared__ const void* s_col[TQP_MAX_KEYS];
  __shared__ int s_dt[TQP_MAX_KEYS];
  if (!*direct) return;
  if (threadIdx.x == 0) P = Pg;
  if (threadIdx.x < TQP_MAX_KEYS) {
    s_col[threadIdx.x] = ks.col[threadIdx.x];
    s_dt[threadIdx.x] = ks.dt[threadIdx.x];
    s_kmin[threadIdx.x] = plan->kmin[threadIdx.x];
    s_shift[threadIdx.x] = plan->shift[threadIdx.x];
  }
  __syncthreads();  // the program and the key plan, before any thread reads them
  constexpr int WARPS = THREADS / 32;
  const int nacc = P.naggs + 1;
  const int slots = 1 << plan->total_bits;
  const int per = slots * nacc;
  int copies = (smem_bytes / 8) / per;
  copies = copies < 1 ? 1 : (copies > WARPS ? WARPS : copies);
  for (int i = threadIdx.x; i < per * copies; i += THREADS) {
    const int q = (i % per) % nacc;
    s_dacc[i] = q < P.naggs ? agg_identity(P.op[q]) : 0;
  }
  __syncthreads();
  long long* my = s_dacc + ((threadIdx.x >> 5) % copies) * per;
  const int64_t n = clamp_n(n_max, d_n);
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n; i += stride) {
    const int64_t row = sel ? sel[i] : i;
    unsigned long long u = 0;
    for (int k = 0; k < ks.nkeys; ++k)
      u |= ((unsigned long long)load_as_i64(s_col[k], s_dt[k], row) - (unsigned long long)s_kmin[k]) << s_shift[k];
    long long* dst = my + (int)u * nacc;
    for (int q = 0; q < P.naggs; ++q)
      direct_fold(dst + q, P.op[q], P.op[q] == TQP_COUNT ? 1 : eval_expr(P, P.expr[q], row), true);
    shared_add_u64(reinterpret_cast<unsigned long long*>(dst + P.naggs), 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < per; i += THREADS) {
    const int q = i % nacc;
    long long v = s_dacc[i];
    for (int w = 1; w < copies; ++w) {
      const long long x = s_dacc[w * per + i];
      v = q < P.naggs ? agg_fold(P.op[q], v, x) : v + x;
    }
    if (v == (q < P.naggs ? agg_identity(P.op[q]) : 0)) continue;
    direct_fold(&acc[i], q < P.naggs ? P.op[q] : TQP_SUM, v, false);
  }
}

// One block: the non-empty slots in key order become the groups.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) gb_direct_out_kernel(KeySet ks, const GroupPlan* plan, AggProgram P,
                                                                const int* direct, const long long* acc,
                                                                long long* out_aggs, int64_t cap,
                                                                int64_t* d_out_groups) {
  __shared__ int s_scan[33];
  if (!*direct) return;
  const int nacc = P.naggs + 1;
  const int slots = 1 << plan->total_bits;
  constexpr int PER = kDirectSlots / THREADS;
  int live[PER];
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int sl = threadIdx.x * PER + j;
    live[j] = sl < slots && acc[(long long)sl * nacc + P.naggs] > 0;
    cnt += live[j];
  }
  int total;
  long long g = block_exclusive_sum<THREADS>(cnt, s_scan, &total);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    if (!live[j]) continue;
    const int sl = threadIdx.x * PER + j;
    if (g < cap) {
      write_group_keys(ks, plan, g, (unsigned long long)sl);
      for (int q = 0; q < P.naggs; ++q) out_aggs[g * P.naggs + q] = acc[(long long)sl * nacc + q];
    }
    ++g;
  }
  if (threadIdx.x == 0) {
    *d_out_groups = total;
    if (total > cap) raise_status(TQP_ERR_CAPACITY);
  }
}

}  // namespace tqp
