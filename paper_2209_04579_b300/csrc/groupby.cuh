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
};

// ---------------------------------------------------------------- aggregates
template <int N>
struct PartialT {
  long long v[N];
  int c;  // segment heads inside the span
};
using Partial = PartialT<TQP_MAX_AGGS>;  // storage layout of the look-back payloads

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

// left (+) right of the segmented reduction: a head inside `right` cuts off `left`.
template <int N>
__device__ __forceinline__ PartialT<N> partial_combine(const PartialT<N>& l, const PartialT<N>& r,
                                                      const AggProgram& P) {
  PartialT<N> o;
#pragma unroll
  for (int a = 0; a < N; ++a)
    o.v[a] = (r.c > 0 || a >= P.naggs) ? r.v[a] : agg_fold(P.op[a], l.v[a], r.v[a]);
  o.c = l.c + r.c;
  return o;
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

template <int N>
__device__ __forceinline__ PartialT<N> shfl_down_partial(const PartialT<N>& p, int d) {
  PartialT<N> o;
#pragma unroll
  for (int a = 0; a < N; ++a) o.v[a] = __shfl_down_sync(0xffffffffu, p.v[a], d);
  o.c = __shfl_down_sync(0xffffffffu, p.c, d);
  return o;
}

template <int N>
__device__ __forceinline__ PartialT<N> shfl_up_partial(const PartialT<N>& p, int d) {
  PartialT<N> o;
#pragma unroll
  for (int a = 0; a < N; ++a) o.v[a] = __shfl_up_sync(0xffffffffu, p.v[a], d);
  o.c = __shfl_up_sync(0xffffffffu, p.c, d);
  return o;
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

template <int THREADS>
__global__ void __launch_bounds__(THREADS) gb_keyrange_kernel(KeySet ks, const int32_t* sel, int64_t n_max,
                                                              const int64_t* d_n, GroupPlan* plan) {
  __shared__ long long s_min[THREADS / 32][TQP_MAX_KEYS], s_max[THREADS / 32][TQP_MAX_KEYS];
  const int64_t n = clamp_n(n_max, d_n);
  long long mn[TQP_MAX_KEYS], mx[TQP_MAX_KEYS];
#pragma unroll
  for (int k = 0; k < TQP_MAX_KEYS; ++k) { mn[k] = LLONG_MAX; mx[k] = LLONG_MIN; }
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n; i += stride) {
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
  uint32_t* flags;         // [num_tiles] look-back flags
  Partial* agg_payload;    // [num_tiles]
  Partial* pre_payload;    // [num_tiles]
  uint32_t* tile_counter;
  uint32_t num_tiles;
  // keys aggregated outside the sorted rows (learned path), merged in key
  // order: sorted packed keys, their count (device) and aggregates [nh][naggs]
  const unsigned long long* heavy;
  const int* d_nheavy;
  const long long* heavy_acc;
};

__device__ __forceinline__ int64_t heavy_lower(const unsigned long long* h, int nh, unsigned long long x) {
  int lo = 0, len = nh;
  while (len > 0) {
    int half = len >> 1;
    if (h[lo + half] < x) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

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

template <int N>
__device__ __forceinline__ void store_partial_relaxed(Partial* dst, const PartialT<N>& p, int naggs) {
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst->v);
#pragma unroll
  for (int a = 0; a < N; ++a)
    if (a < naggs) st_volatile_u64(d + a, (unsigned long long)p.v[a]);
  st_volatile_u32(reinterpret_cast<uint32_t*>(&dst->c), (uint32_t)p.c);
}

template <int N>
__device__ __forceinline__ PartialT<N> load_partial_relaxed(const Partial* src, const AggProgram& P) {
  PartialT<N> p;
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src->v);
#pragma unroll
  for (int a = 0; a < N; ++a) p.v[a] = (a < P.naggs) ? (long long)ld_volatile_u64(s + a) : 0;
  p.c = (int)ld_volatile_u32(reinterpret_cast<const uint32_t*>(&src->c));
  return p;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename K, int THREADS, int ITEMS, int NAGG>
__global__ void __launch_bounds__(THREADS) gb_reduce_kernel(ReduceArgs a, AggProgram Pg) {
  constexpr int TILE = THREADS * ITEMS;
  constexpr int WARPS = THREADS / 32;
  using PT = PartialT<NAGG>;
  __shared__ PT s_warp[WARPS];
  __shared__ PT s_tile_excl;
  __shared__ AggProgram P;  // the program and the key set in shared memory: indexed by runtime values below
  __shared__ KeySet s_ks;
  if (threadIdx.x == 0) {
    P = Pg;
    s_ks = a.ks;
  }
  __syncthreads();
  __shared__ uint32_t s_tile;
  __shared__ int s_failed;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  const K* keys = static_cast<const K*>(a.keys);
  const int32_t* rows = a.rows;  // null: the value columns are already in sorted order
  const bool unsupported = a.plan->unsupported != 0;
  const long long limit = g_spin_limit;
  const int nh = (a.heavy && a.d_nheavy) ? *a.d_nheavy : 0;

  while (true) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(a.tile_counter, 1u);
      s_failed = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) break;
    const int64_t base = (int64_t)tile * TILE + (int64_t)threadIdx.x * ITEMS;
    const int64_t nn = unsupported ? 0 : n;

    // ---- pass 1: heads, and the partial of the thread's trailing run
    K key[ITEMS];
    uint32_t head = 0;
    K prev = 0;
    if (base > 0 && base < nn) prev = keys[base - 1];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      int64_t p = base + k;
      key[k] = (p < nn) ? keys[p] : (K)0;
      if (p < nn && (p == 0 || key[k] != (k ? key[k - 1] : prev))) head |= 1u << k;
    }
    PT mine;
    partial_identity(mine, P);
    mine.c = __popc(head);
    {
      int last_head = head ? (31 - __clz(head)) : 0;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        if (k >= last_head && base + k < nn) fold_row(mine, P, rows ? rows[base + k] : base + k);
    }

    // ---- block exclusive segmented scan of the thread partials
    PT incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      PT up = shfl_up_partial(incl, d);
      if (lane >= d) incl = partial_combine(up, incl, P);
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    PT wexcl;
    partial_identity(wexcl, P);
    for (int w = 0; w < warp; ++w) wexcl = partial_combine(wexcl, s_warp[w], P);
    PT texcl = shfl_up_partial(incl, 1);
    if (lane == 0) partial_identity(texcl, P);
    PT thread_excl = partial_combine(wexcl, texcl, P);

    // ---- tile look-back (warp 0: 32 predecessors per step, folded in order)
    if (warp == 0) {
      PT tile_agg;
      partial_identity(tile_agg, P);
      for (int w = 0; w < WARPS; ++w) tile_agg = partial_combine(tile_agg, s_warp[w], P);
      const bool inject = ((long long)tile == g_unpublished_tile);
      PT acc;
      partial_identity(acc, P);
      bool failed = false;
      if (tile == 0) {
        if (lane == 0 && !inject) {
          store_partial_relaxed(&a.pre_payload[0], tile_agg, P.naggs);
          st_release_u32(&a.flags[0], 2u);
        }
      } else {
        if (lane == 0 && !inject) {
          store_partial_relaxed(&a.agg_payload[tile], tile_agg, P.naggs);
          st_release_u32(&a.flags[tile], 1u);
        }
        long long window_end = tile;
        while (true) {
          const long long t = window_end - 1 - lane;
          uint32_t f = 2u;  // before tile 0: an empty inclusive prefix
          PT v;
          partial_identity(v, P);
          if (t >= 0) {
            long long rounds = 0;
            unsigned sleep_ns = 32;
            while (true) {
              f = ld_acquire_u32(&a.flags[t]);
              if (f) break;
              if (++rounds > limit) { f = 3u; break; }
              __nanosleep(sleep_ns);
              if (sleep_ns < 1024) sleep_ns <<= 1;
            }
            if (f == 1u || f == 2u) v = load_partial_relaxed<NAGG>(f == 2u ? &a.pre_payload[t] : &a.agg_payload[t], P);
          }
          if (__ballot_sync(0xffffffffu, f == 3u)) { failed = true; break; }
          const unsigned pm = __ballot_sync(0xffffffffu, f == 2u);
          const int first = pm ? __ffs(pm) - 1 : 31;
          if (lane > first) partial_identity(v, P);
          // fold lanes first .. 0 (higher lanes are further left)
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            PT other = shfl_down_partial(v, o);
            if (lane + o < 32) v = partial_combine(other, v, P);
          }
          acc = partial_combine(v, acc, P);  // lane 0 holds the window's fold
          if (pm) break;
          window_end -= 32;
        }
        if (lane == 0 && !inject) {
          if (failed) {
            st_release_u32(&a.flags[tile], 3u);
          } else {
            store_partial_relaxed(&a.pre_payload[tile], partial_combine(acc, tile_agg, P), P.naggs);
            st_release_u32(&a.flags[tile], 2u);
          }
        }
      }
      if (lane == 0) {
        if (failed) {
          raise_status(TQP_ERR_TIMEOUT);
          s_failed = 1;
        }
        s_tile_excl = acc;
        if (!failed && tile == a.num_tiles - 1) {
          long long g = (long long)acc.c + tile_agg.c + nh;
          *a.d_out_groups = g;
          if (g > a.cap) raise_status(TQP_ERR_CAPACITY);
        }
      }
    }
    __syncthreads();
    const int tile_failed = s_failed;
    PT in = partial_combine(s_tile_excl, thread_excl, P);
    __syncthreads();
    if (tile_failed) continue;

    // ---- pass 2: finish every segment whose last row this thread holds
    PT run = in;
    long long seg = (long long)in.c - 1;
    K next_after = 0;
    if (base + ITEMS < nn) next_after = keys[base + ITEMS];
#pragma unroll 1
    for (int k = 0; k < ITEMS; ++k) {
      int64_t p = base + k;
      if (p < nn) {
        if (head & (1u << k)) {
          ++seg;
#pragma unroll
          for (int q = 0; q < NAGG; ++q) run.v[q] = (q < P.naggs) ? agg_identity(P.op[q]) : 0;
          if (nh) {
            // heavy keys between the previous group's key and this one go just before it
            int64_t hi_i = heavy_lower(a.heavy, nh, (unsigned long long)key[k]);
            int64_t lo_i = p == 0 ? 0 : heavy_lower(a.heavy, nh, (unsigned long long)(k ? key[k - 1] : prev));
            for (int64_t i = lo_i; i < hi_i; ++i)
              write_group(a, s_ks, P.naggs, seg + i, a.heavy[i], a.heavy_acc + (size_t)i * P.naggs);
          }
        }
        fold_row(run, P, rows ? rows[p] : p);
        K nk = (k + 1 < ITEMS) ? key[k + 1] : next_after;
        bool last = (p == nn - 1) || (nk != key[k]);
        if (last && seg >= 0) {
          long long hr = nh ? heavy_lower(a.heavy, nh, (unsigned long long)key[k]) : 0;
          write_group_regs(a, s_ks, P.naggs, seg + hr, (unsigned long long)key[k], run);
          if (nh && p == nn - 1) {
            // heavy keys above the last group's key
            for (int64_t i = hr; i < nh; ++i)
              write_group(a, s_ks, P.naggs, seg + 1 + i, a.heavy[i], a.heavy_acc + (size_t)i * P.naggs);
          }
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace tqp
