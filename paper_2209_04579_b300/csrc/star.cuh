// Fused star join + filter + group-by aggregate over one or two dimension
// tables (the join-plus-aggregation shape of the paper's Q14 experiment,
// Section 2.3).
//
// Per dimension d (all on the device, no host round trip):
//   filter the dimension rows (stream compaction) and gather their keys;
//   give each passing row the dense rank of its group value (a presence
//   bitmap over a small value domain, else sort + adjacent difference +
//   look-back scan); sort (key, rank or row), gather the rank and any
//   aggregated dimension column into key order, and build the directory:
//   cell bitmap, and a 32-byte record per wide cell with its first keys
//   inline.  Keys dense in their range skip the sort: one cell per key
//   value, filled straight from the rows.
// Then one pass over the fact table: fact predicates, one directory probe
// per dimension, and the row's expression values folded into the
// accumulator slot of its group combination (ranks are in ascending value
// order, so slot order is the lexicographic group order).  Few slots live in
// shared memory per block; many go straight to global 64-bit atomics.
// A final single-pass scan compacts the non-empty slots into the output.
#pragma once

#include "common.cuh"
#include "filter.cuh"
#include "groupby.cuh"
#include "join.cuh"

namespace tqp {

constexpr int kMaxDims = 2;
constexpr int kSmemAccWords = 4096;  // slots * (naggs + 1) that fit the shared accumulators

struct StarPlan {
  long long G[kMaxDims];       // distinct group values per dimension (1 without a group column)
  long long stride[kMaxDims];  // slot = sum code_d * stride_d
  long long S;                 // number of slots
  int use_smem;
  int unsupported;
};

__device__ __forceinline__ unsigned long long key_image(const void* p, int dt, int64_t i) {
  return dt == TQP_I32 ? (unsigned long long)((uint32_t) static_cast<const int32_t*>(p)[i] ^ 0x80000000u)
                       : ((unsigned long long) static_cast<const long long*>(p)[i] ^ 0x8000000000000000ull);
}

// Sorted passing keys side by side with their group ranks, so that the
// probe's key comparison and the rank share one memory access.
struct KeyRank32 {
  uint32_t image;  // order-preserving image of the key
  int32_t rank;
};
struct KeyRank64 {
  unsigned long long image;
  long long rank;
};

// ---- group ranks of one dimension: heads of the sorted packed group keys,
// scanned into dense ranks; rank scattered to the row, key value kept.
template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) rank_kernel(const K* sorted, const int32_t* rows, int64_t n_max,
                                                       const int64_t* d_n, const GroupPlan* gp,
                                                       int32_t* rank_of_row, long long* gkey,
                                                       long long* d_G, unsigned long long* status,
                                                       uint32_t* counter, uint32_t num_tiles) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ long long s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = clamp_n(n_max, d_n);
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const int64_t base = (int64_t)tile * TILE + (int64_t)threadIdx.x * ITEMS;
    uint32_t head = 0;
    K prev = (base > 0 && base < n) ? sorted[base - 1] : (K)0;
    K key[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      int64_t p = base + k;
      key[k] = p < n ? sorted[p] : (K)0;
      if (p < n && (p == 0 || key[k] != (k ? key[k - 1] : prev))) head |= 1u << k;
    }
    int total;
    int off = block_exclusive_sum<THREADS>(__popc(head), s_scan, &total);
    if (warp == 0) {
      long long e = lookback_exclusive(status, tile, total);
      if (lane == 0) s_excl = e;
    }
    __syncthreads();
    long long excl = s_excl;
    if (excl >= 0) {
      long long r = excl + off - 1;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        int64_t p = base + k;
        if (p < n) {
          if (head & (1u << k)) {
            ++r;
            unsigned long long m = gp->bits[0] >= 64 ? ~0ull : ((1ull << gp->bits[0]) - 1);
            gkey[r] = (long long)(((unsigned long long)key[k] & m) + (unsigned long long)gp->kmin[0]);
          }
          rank_of_row[rows[p]] = (int32_t)r;
        }
      }
      if (tile == num_tiles - 1 && threadIdx.x == 0) *d_G = excl + total;
    }
    __syncthreads();
  }
}

// ---- group ranks of one dimension over a small value domain: the group
// column's passing values span at most 2^kDomBits (kmax - kmin < 2^24, the
// case of every int8 and int16 column).  A bitmap marks the values present;
// the dense rank of v is the number of marked values below it, read from a
// per-word prefix count and one popcount.  No sort and no scatter by row.
constexpr int kDomBits = 24;
constexpr int kDomSmemWords = 2048;  // domains up to 2^16 values are marked in shared memory first


__global__ void dom_plan_kernel(const GroupPlan* gp, int64_t n_max, const int64_t* d_n, DomPlan* dp,
                                int64_t* sort_n) {
  if (threadIdx.x != 0) return;
  const int64_t n = clamp_n(n_max, d_n);
  DomPlan r;
  r.on = n > 0 && !gp->unsupported && gp->bits[0] <= kDomBits;
  r.kmin = gp->kmin[0];
  r.words = r.on ? (int)(((unsigned long long)gp->kmax[0] - (unsigned long long)gp->kmin[0]) >> 5) + 1 : 0;
  *dp = r;
  *sort_n = r.on ? 0 : n;
}

constexpr int kDomItems = 8;  // rows per thread per round of the value-domain passes

__global__ void __launch_bounds__(256) dom_mark_kernel(const void* gcol, int gdt, const int32_t* sel, int64_t n_max,
                                                       const int64_t* d_n, const DomPlan* dp, uint32_t* bits) {
  __shared__ uint32_t s_bits[kDomSmemWords];
  const DomPlan p = *dp;
  if (!p.on) return;
  const int64_t n = clamp_n(n_max, d_n);
  const bool shared = p.words <= kDomSmemWords;
  if (shared) {
    for (int i = threadIdx.x; i < p.words; i += blockDim.x) s_bits[i] = 0;
    __syncthreads();
  }
  auto mark = [&](long long x) {
    const unsigned long long v = (unsigned long long)x - (unsigned long long)p.kmin;
    const uint32_t w = (uint32_t)(v >> 5), b = 1u << (v & 31);
    if (shared) {
      if (!(s_bits[w] & b)) atomicOr(&s_bits[w], b);
    } else if (!(__ldcg(&bits[w]) & b)) {
      atomicOr(&bits[w], b);
    }
  };
  const int esz = gdt == TQP_I8 ? 1 : gdt == TQP_I16 ? 2 : 0;
  if (sel == nullptr && esz && ((uintptr_t)gcol & 15) == 0) {
    // a 1- or 2-byte column read as 16-byte words, four in flight per
    // thread, then the scalar tail
    const int per = 16 / esz;
    const int64_t nw = n / per;
    const int4* wp = static_cast<const int4*>(gcol);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < nw; base += stride * 4) {
      int4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(wp + (base + u * stride < nw ? base + u * stride : base));
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (base + u * stride >= nw) continue;
        if (esz == 1) {
          const signed char* e = reinterpret_cast<const signed char*>(&v[u]);
#pragma unroll
          for (int j = 0; j < 16; ++j) mark(e[j]);
        } else {
          const short* e = reinterpret_cast<const short*>(&v[u]);
#pragma unroll
          for (int j = 0; j < 8; ++j) mark(e[j]);
        }
      }
    }
    for (int64_t i = nw * per + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
      mark(load_as_i64(gcol, gdt, i));
  } else {
    // kDomItems rows per thread at a time, their loads issued together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kDomItems;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kDomItems + threadIdx.x; base < n; base += stride) {
      int64_t row[kDomItems];
      bool ok[kDomItems];
      long long val[kDomItems];
#pragma unroll
      for (int k = 0; k < kDomItems; ++k) {
        const int64_t i = base + (int64_t)k * blockDim.x;
        ok[k] = i < n;
        row[k] = ok[k] ? (sel ? sel[i] : i) : 0;
      }
      load_many_as_i64(gcol, gdt, row, ok, val);
#pragma unroll
      for (int k = 0; k < kDomItems; ++k)
        if (ok[k]) mark(val[k]);
    }
  }
  if (shared) {
    __syncthreads();
    for (int i = threadIdx.x; i < p.words; i += blockDim.x)
      if (s_bits[i]) atomicOr(&bits[i], s_bits[i]);
  }
}

// One block: exclusive prefix counts per bitmap word, the group key value of
// every rank, and the number of groups.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) dom_scan_kernel(const DomPlan* dp, const uint32_t* bits, int* pre,
                                                           long long* gkey, long long* d_G) {
  __shared__ int s_scan[33];
  const DomPlan p = *dp;
  if (!p.on) return;
  const int per = (p.words + THREADS - 1) / THREADS;
  const int w0 = threadIdx.x * per, w1 = min(p.words, w0 + per);
  int cnt = 0;
  for (int w = w0; w < w1; ++w) cnt += __popc(bits[w]);
  int total;
  int r = block_exclusive_sum<THREADS>(cnt, s_scan, &total);
  for (int w = w0; w < w1; ++w) {
    pre[w] = r;
    uint32_t m = bits[w];
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      gkey[r++] = p.kmin + (long long)w * 32 + b;
    }
  }
  if (threadIdx.x == 0) *d_G = total;
}


// Sort payload of the passing rows: the group rank when the bitmap ranks and
// the caller allows it (rank_payload), else the row.
__global__ void dom_payload_kernel(const void* gcol, int gdt, const int32_t* sel, int64_t n_max, const int64_t* d_n,
                                   const DomPlan* dp, const uint32_t* bits, const int* pre, int rank_payload,
                                   int32_t* out) {
  __shared__ uint32_t s_bits[kDomSmemWords];
  __shared__ int s_pre[kDomSmemWords];
  const DomPlan p = *dp;
  const bool rk = rank_payload && p.on;
  const int64_t n = clamp_n(n_max, d_n);
  const int esz = gdt == TQP_I8 ? 1 : gdt == TQP_I16 ? 2 : 0;
  if (rk && sel == nullptr && esz && p.words <= kDomSmemWords && ((uintptr_t)gcol & 15) == 0 &&
      ((uintptr_t)out & 15) == 0) {
    // a 1- or 2-byte group column read as 16-byte words, its bitmap and
    // prefix counts in shared memory, the ranks written as 16-byte words;
    // then the scalar tail
    for (int i = threadIdx.x; i < p.words; i += blockDim.x) {
      s_bits[i] = bits[i];
      s_pre[i] = pre[i];
    }
    __syncthreads();
    auto rank_of = [&](int v) -> int {
      const unsigned x = (unsigned)((long long)v - p.kmin);
      return s_pre[x >> 5] + __popc(s_bits[x >> 5] & ((1u << (x & 31)) - 1u));
    };
    const int per = 16 / esz;
    const int64_t nw = n / per;
    const int4* wp = static_cast<const int4*>(gcol);
    int4* op = reinterpret_cast<int4*>(out);
    const int64_t tstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += tstride) {
      const int4 v = __ldg(wp + w);
      int r[16];
      if (esz == 1) {
        const signed char* e = reinterpret_cast<const signed char*>(&v);
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = rank_of(e[j]);
      } else {
        const short* e = reinterpret_cast<const short*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = rank_of(e[j]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q * 4 < per) op[w * (per / 4) + q] = make_int4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
    for (int64_t i = nw * per + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += tstride)
      out[i] = rank_of((int)load_as_i64(gcol, gdt, i));
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kDomItems;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kDomItems + threadIdx.x; base < n; base += stride) {
    int64_t row[kDomItems];
    bool ok[kDomItems];
    long long val[kDomItems];
#pragma unroll
    for (int k = 0; k < kDomItems; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x;
      ok[k] = i < n;
      row[k] = ok[k] ? (sel ? sel[i] : i) : 0;
    }
    if (rk) {
      load_many_as_i64(gcol, gdt, row, ok, val);
#pragma unroll
      for (int k = 0; k < kDomItems; ++k)
        if (ok[k]) out[base + (int64_t)k * blockDim.x] = dom_rank(p, bits, pre, val[k]);
    } else {
#pragma unroll
      for (int k = 0; k < kDomItems; ++k)
        if (ok[k]) out[base + (int64_t)k * blockDim.x] = (int32_t)row[k];
    }
  }
}

// ---- key directory of one dimension: the range of its sorted passing keys
// is cut into at most 2^log2_cells cells of 2^bshift key values; dir[c] is
// the first sorted position whose key falls in cell c or later, and a bitmap
// marks the non-empty cells.  A probe tests the cell's bit (an L1-resident
// word) and then compares the few keys of dir[c] .. dir[c+1]: a bound search
// whose first levels are the directory.  Exact for any key distribution.
struct DimDir {
  unsigned long long umin, umax;  // order-preserving images of the first and last key
  int bshift;
  int use_bits;                   // probes test the cell bitmap first (unit cells, or a filtered dimension)
  long long ncells;               // 0: no passing rows (every probe misses)
  int direct;                     // dense keys: unit cells filled straight from the rows, no key sort
  int fused;                      // the whole directory comes from one pass over the sorted packed keys
};

// ---- gather ranks and aggregated dimension columns into key order; check
// that keys are unique among the passing rows.
struct PregatherArgs {
  const void* skeys;
  int key_dt;
  const int32_t* srows;
  int64_t n_max;
  const int64_t* d_n;
  const int32_t* rank_of_row;  // null: no group column
  // the domain path (dom->on): rank of the row's group value in the bitmap
  const DomPlan* dom;
  const void* gcol;
  int gdt;
  const uint32_t* dbits;
  const int* dpre;
  int rank_payload;            // with dom->on: srows holds each sorted key's group rank
  const DimDir* dd;            // nothing to do when the fused pass built the directory
  int32_t* rank_sorted;
  void* kr;                    // KeyRank32 (int32 keys) or KeyRank64 per sorted position
  int nv;
  const void* vcol[TQP_MAX_VALS];
  int vdt[TQP_MAX_VALS];
  long long* vout[TQP_MAX_VALS];
  StarPlan* plan;
};

__global__ void star_pregather_kernel(PregatherArgs a) {
  if (a.dd && a.dd->fused) return;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  DomPlan dom;
  dom.on = 0;
  if (a.dom) dom = *a.dom;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    int32_t row = a.srows[p];
    const int32_t rk = !a.rank_of_row              ? 0
                       : dom.on && a.rank_payload ? row
                       : dom.on                   ? dom_rank(dom, a.dbits, a.dpre, load_as_i64(a.gcol, a.gdt, row))
                                                  : a.rank_of_row[row];
    a.rank_sorted[p] = rk;
    if (a.key_dt == TQP_I32)
      static_cast<KeyRank32*>(a.kr)[p] = KeyRank32{(uint32_t)key_image(a.skeys, a.key_dt, p), rk};
    else
      static_cast<KeyRank64*>(a.kr)[p] = KeyRank64{key_image(a.skeys, a.key_dt, p), (long long)rk};
    for (int v = 0; v < a.nv; ++v) a.vout[v][p] = load_as_i64(a.vcol[v], a.vdt[v], row);
    if (p > 0 && load_as_i64(a.skeys, a.key_dt, p) == load_as_i64(a.skeys, a.key_dt, p - 1)) {
      if (atomicExch(&a.plan->unsupported, 1) == 0) raise_status(TQP_ERR_UNSUPPORTED);
    }
  }
}

__global__ void star_slots_kernel(StarPlan* plan, int ndims, const long long* d_G0, const long long* d_G1,
                                  long long slots_cap, int nacc) {
  if (threadIdx.x != 0) return;
  long long G[kMaxDims] = {d_G0 ? *d_G0 : 1, d_G1 ? *d_G1 : 1};
  long long S = 1;
  for (int d = ndims - 1; d >= 0; --d) {
    plan->G[d] = G[d];
    plan->stride[d] = S;
    S *= G[d] > 0 ? G[d] : 1;
  }
  plan->S = S;
  if (S > slots_cap) {
    plan->unsupported = 1;
    raise_status(TQP_ERR_UNSUPPORTED);
  }
  // 2: one accumulator copy per warp of the probe block (no cross-warp
  // contention on few groups); 1: one copy per block; 0: global atomics
  plan->use_smem = (S * nacc * 8 <= kSmemAccWords) ? 2 : (S * nacc <= kSmemAccWords) ? 1 : 0;
}

struct StarAcc {
  int naggs;
  int cnt;               // accumulator that counts rows: a COUNT aggregate, else naggs
  int op[TQP_MAX_AGGS];  // aggregate ops; accumulator naggs holds the row count
  int expr[TQP_MAX_AGGS];
  int nexprs;
  int nterms[TQP_MAX_EXPRS];
  int tval[TQP_MAX_EXPRS][3];
  long long tmul[TQP_MAX_EXPRS][3];
  long long tadd[TQP_MAX_EXPRS][3];
};

__device__ __forceinline__ long long acc_identity(const StarAcc& A, int q) {
  return q < A.naggs ? agg_identity(A.op[q]) : 0;
}

__global__ void star_init_acc_kernel(const StarPlan* plan, const StarAcc A, long long* acc) {
  const long long S = plan->S;
  const int nacc = A.naggs + 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (plan->unsupported) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S * nacc; i += stride)
    acc[i] = acc_identity(A, (int)(i % nacc));
}


// ---- dense keys without the sort.  When the passing keys are unique and
// dense in their range (span < 8 x their count, within the cell budget),
// the directory has one cell per key value: sorting the keys would only
// place each at key - min, which the cell index already does.  The key
// range is taken first; dense dimensions then skip the key sort and fill
// their cells straight from the rows.
__global__ void dim_range_kernel(const void* keys, int key_dt, int64_t n_max, const int64_t* d_n,
                                 unsigned long long* range) {
  const int64_t n = clamp_n(n_max, d_n);
  unsigned long long lo = ~0ull, hi = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long u = key_image(keys, key_dt, i);
    lo = u < lo ? u : lo;
    hi = u > hi ? u : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = l2 < lo ? l2 : lo;
    hi = h2 > hi ? h2 : hi;
  }
  if ((threadIdx.x & 31) == 0 && lo <= hi) {
    atomicMin(&range[0], lo);
    atomicMax(&range[1], hi);
  }
}

// One thread: the directory plan of a dense dimension (unit cells, direct),
// or direct = 0; sort_n: the rows the key sort then takes (0 when direct).
__global__ void dim_direct_plan_kernel(const unsigned long long* range, int64_t n_max, const int64_t* d_n,
                                       int log2_cells_max, DimDir* dd, int64_t* sort_n) {
  if (threadIdx.x != 0) return;
  const int64_t nd = clamp_n(n_max, d_n);
  DimDir r;
  r.umin = range[0];
  r.umax = range[1];
  r.bshift = 0;
  r.use_bits = 1;
  r.direct = 0;
  r.fused = 0;
  r.ncells = 0;
  if (nd > 0 && r.umin <= r.umax) {
    const unsigned long long span = r.umax - r.umin;
    const int bits = span ? 64 - __clzll((long long)span) : 0;
    r.direct = span < 8ull * (unsigned long long)nd && bits <= log2_cells_max;
    r.ncells = (long long)span + 1;
  }
  if (!r.direct) r.ncells = 0;
  *dd = r;
  *sort_n = r.direct ? 0 : nd;
}

// Cells of a direct dimension: the bit, the group rank and the aggregated
// values of each passing row at cell key - min.  A bit already set is a
// repeated key (unsupported, as in the sorted form).
struct DirectArgs {
  const void* keys;  // passing keys (compacted when the dimension is filtered)
  int key_dt;
  const int32_t* sel;  // row of each passing key (null: the position)
  int64_t n_max;
  const int64_t* d_n;
  const DimDir* dd;
  uint32_t* bitmap;
  int32_t* rank_cell;
  // group rank: the domain bitmap (dom->on), else rank_of_row; none without a group column
  const int32_t* rank_of_row;
  const DomPlan* dom;
  const void* gcol;
  int gdt;
  const uint32_t* dbits;
  const int* dpre;
  int nv;
  const void* vcol[TQP_MAX_VALS];
  int vdt[TQP_MAX_VALS];
  long long* dval_cell[TQP_MAX_VALS];
  StarPlan* plan;
};

__global__ void dir_direct_kernel(DirectArgs a) {
  const DimDir r = *a.dd;
  if (!r.direct) return;
  DomPlan dom;
  dom.on = 0;
  if (a.dom) dom = *a.dom;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t row = a.sel ? a.sel[i] : (int32_t)i;
    const unsigned long long c = key_image(a.keys, a.key_dt, i) - r.umin;
    const uint32_t bit = 1u << (c & 31);
    if (atomicOr(&a.bitmap[c >> 5], bit) & bit) {
      if (atomicExch(&a.plan->unsupported, 1) == 0) raise_status(TQP_ERR_UNSUPPORTED);
      continue;
    }
    a.rank_cell[c] = !a.rank_of_row ? 0
                     : dom.on      ? dom_rank(dom, a.dbits, a.dpre, load_as_i64(a.gcol, a.gdt, row))
                                   : a.rank_of_row[row];
    for (int v = 0; v < a.nv; ++v) a.dval_cell[v][c] = load_as_i64(a.vcol[v], a.vdt[v], row);
  }
}



// Wide cells (bshift > 0) get a table of one 32-byte record per cell, so
// that a probe reads one record instead of the directory entry and then the
// keys it points to.  The record holds the cell's first keys inline with
// their group ranks, its first sorted position lo and its key count cnt:
//   int32 keys: a = {img0, img1, img2, rank0}, b = {rank1, rank2, lo, cnt}
//   int64 keys: a = {img0 (2 words), img1 (2 words)}, b = {rank0, rank1, lo, cnt}
// A cell with more keys than fit inline keeps the rest in the sorted
// key/rank pairs, after position lo + inline count.
struct __align__(16) DirCell {
  int4 a, b;
};
__host__ __device__ constexpr int cell_inline(bool k32) { return k32 ? 3 : 2; }
// Wide cells wanted for nd keys: one per key for 32-bit keys (three inline
// in a record), two per key for 64-bit keys (two inline), so that few cells
// hold more keys than their record.
__host__ __device__ inline long long wide_cells_wanted(int64_t nd, int key_dt) {
  return key_dt == TQP_I32 ? (long long)nd : 2ll * nd;
}

// The cell plan of nd sorted passing keys whose images run from umin to
// umax.  n_all: the dimension's rows before its predicates.  Wide cells of a
// dimension that no predicate filtered skip the bitmap: foreign keys find
// their row, and a miss is still found by the directory and the key.
__device__ DimDir plan_cells(unsigned long long umin, unsigned long long umax, int64_t nd, int64_t n_all,
                             int log2_cells_max, const long long* d_G, int key_dt) {
  DimDir r;
  r.direct = 0;
  r.fused = 0;
  r.use_bits = 1;
  if (nd == 0) {
    r.umin = 1;
    r.umax = 0;
    r.bshift = 0;
    r.ncells = 0;
    return r;
  }
  r.umin = umin;
  r.umax = umax;
  unsigned long long span = r.umax - r.umin;
  int tb = 1;
  while (tb < log2_cells_max && (1ll << tb) < wide_cells_wanted(nd, key_dt)) ++tb;
  int bits = span ? 64 - __clzll((long long)span) : 0;
  // keys dense in their range (span within 8x their count): one cell per key
  // value, so the bit alone decides membership
  if (span < 8ull * (unsigned long long)nd && bits <= log2_cells_max) tb = bits > tb ? bits : tb;
  r.bshift = bits > tb ? bits - tb : 0;
  r.ncells = (long long)(span >> r.bshift) + 1;
  r.use_bits = (r.bshift == 0 || nd < n_all) ? 1 : 0;
  return r;
}

__global__ void dir_plan_kernel(const void* skeys, int key_dt, int64_t n_max, const int64_t* d_n, int64_t n_all,
                                int log2_cells_max, const long long* d_G, DimDir* dd) {
  if (threadIdx.x != 0) return;
  if (dd->direct || dd->fused) return;  // planned from the key range, or by the fused pass
  const int64_t nd = clamp_n(n_max, d_n);
  *dd = plan_cells(nd ? key_image(skeys, key_dt, 0) : 1, nd ? key_image(skeys, key_dt, nd - 1) : 0, nd, n_all,
                   log2_cells_max, d_G, key_dt);
}

// ---- the directory in one pass, for a dimension sorted by the learned
// partitioner: its keys sorted as packed words (key - kmin), and each
// sorted key's group rank as the sort's payload (or no group column).
// The plan is taken from the first and last packed keys; when the cells
// are wide and no dimension value is aggregated (eligible), dir_emit_kernel
// writes every structure the probe reads -- the bitmap, the 32-byte
// records, and the key/rank pairs of keys past a record's inline ones -- and
// the decode, gather and directory passes of the sorted form skip their
// work (fused = 1).  The cell starts (dir) are not written: the records
// carry each cell's first position and count.
__device__ __forceinline__ unsigned long long packed_image(unsigned long long packed, long long kmin, int key_dt) {
  const unsigned long long key = packed + (unsigned long long)kmin;  // the key, 64-bit two's complement
  return key_dt == TQP_I32 ? (unsigned long long)((uint32_t)key ^ 0x80000000u) : key ^ 0x8000000000000000ull;
}

__global__ void dir_plan_packed_kernel(const unsigned long long* packed, const GroupPlan* gp, int key_dt,
                                       int64_t n_max, const int64_t* d_n, int64_t n_all, int log2_cells_max,
                                       const long long* d_G, const DomPlan* dom, int eligible, DimDir* dd) {
  if (threadIdx.x != 0) return;
  if (dd->direct) return;
  const int64_t nd = clamp_n(n_max, d_n);
  const long long kmin = gp->kmin[0];
  DimDir r = plan_cells(nd ? packed_image(packed[0], kmin, key_dt) : 1,
                        nd ? packed_image(packed[nd - 1], kmin, key_dt) : 0, nd, n_all, log2_cells_max, d_G, key_dt);
  // the payload is each key's group rank (a bitmap-ranked group column) or
  // there is no group column
  const bool ranks_in_payload = dom == nullptr || dom->on;
  r.fused = eligible && ranks_in_payload && nd > 0 && r.bshift > 0;
  *dd = r;
}

struct EmitArgs {
  const unsigned long long* packed;  // sorted packed keys
  const int32_t* payload;            // their group ranks (when the dimension has a group column)
  int has_group;
  const GroupPlan* gp;               // kmin of the key column
  int key_dt;
  int64_t n_max;
  const int64_t* d_n;
  const DimDir* dd;
  void* kr;                          // KeyRank32 / KeyRank64 per sorted position (overflow keys only)
  uint32_t* bitmap;
  DirCell* table;
  StarPlan* plan;
};

// A warp takes 32 consecutive sorted positions at a time: one coalesced load
// of the keys and ranks, cell heads found by ballot, a head's count from the
// next head in the chunk (or, for the chunk's last cell, in the next chunk,
// which is already loaded), its inline keys and ranks from the following
// lanes.  Each head writes its record and the (zero) records of the empty
// cells before it.
constexpr int kEmitThreads = 256;

// One 32-byte record in a single 256-bit store (records are 32-byte aligned:
// the table starts on a 256-byte boundary).
__device__ __forceinline__ void store_cell(DirCell* dst, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(w[0]), "r"(w[1]),
               "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

__global__ void __launch_bounds__(kEmitThreads) dir_emit_kernel(EmitArgs a) {
  const DimDir r = *a.dd;
  if (!r.fused) return;
  const int64_t nd = clamp_n(a.n_max, a.d_n);
  const long long kmin = a.gp->kmin[0];
  const bool k32 = a.key_dt == TQP_I32;
  const int cap = cell_inline(k32);
  const int lane = threadIdx.x & 31;
  auto image_at = [&](int64_t q) -> unsigned long long { return packed_image(__ldg(&a.packed[q]), kmin, a.key_dt); };
  auto cell_of = [&](unsigned long long u) -> long long { return (long long)((u - r.umin) >> r.bshift); };
  auto rank_at = [&](int64_t q) -> int32_t { return a.has_group ? __ldg(&a.payload[q]) : 0; };
  // each warp takes a contiguous run of 32-position chunks; the next chunk's
  // keys and ranks are loaded while the current chunk is processed, and give
  // the last cell of a chunk its count and its inline keys past the chunk
  auto fetch = [&](int64_t q, unsigned long long& pk, int32_t& rk) {
    pk = 0;
    rk = 0;
    if (q < nd) {
      pk = __ldg(&a.packed[q]);
      rk = rank_at(q);
    }
  };
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nchunks = (nd + 31) / 32;
  const int64_t per = (nchunks + nwarps - 1) / nwarps;
  const int64_t cbeg = wid * per;
  const int64_t cend = cbeg + per < nchunks ? cbeg + per : nchunks;
  if (cbeg >= cend) return;
  int64_t base = cbeg * 32;
  unsigned long long pk_n;
  int32_t rk_n;
  fetch(base + lane, pk_n, rk_n);
  unsigned long long before = base > 0 ? __ldg(&a.packed[base - 1]) : 0ull;  // the key before the run
  for (int64_t ch = cbeg; ch < cend; ++ch, base += 32) {
    const int64_t p = base + lane;
    const bool valid = p < nd;
    const unsigned long long pk = pk_n;
    const int32_t rk = rk_n;
    fetch(base + 32 + lane, pk_n, rk_n);
    const unsigned long long u = valid ? packed_image(pk, kmin, a.key_dt) : 0ull;
    const long long c = valid ? cell_of(u) : -2;
    unsigned long long prev_pk = __shfl_up_sync(0xffffffffu, pk, 1);
    long long prev_c = __shfl_up_sync(0xffffffffu, c, 1);
    if (lane == 0) {
      prev_pk = p > 0 ? before : ~pk;
      prev_c = p > 0 ? cell_of(packed_image(prev_pk, kmin, a.key_dt)) : -1;
    }
    before = __shfl_sync(0xffffffffu, pk, 31);  // the next chunk's predecessor
    if (valid && p > 0 && prev_pk == pk) {
      if (atomicExch(&a.plan->unsupported, 1) == 0) raise_status(TQP_ERR_UNSUPPORTED);
    }
    const bool head = valid && c != prev_c;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    // the following lanes' keys and ranks (inline keys of a head), in this
    // chunk or, past lane 31, in the next
    const bool valid_n = base + 32 + lane < nd;
    const unsigned long long u_n = valid_n ? packed_image(pk_n, kmin, a.key_dt) : 0ull;
    unsigned long long un[3], wn[3];
    int32_t rn[3], wr[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      un[j] = __shfl_down_sync(0xffffffffu, u, j);
      rn[j] = __shfl_down_sync(0xffffffffu, rk, j);
      wn[j] = __shfl_sync(0xffffffffu, u_n, (lane + j) & 31);
      wr[j] = __shfl_sync(0xffffffffu, rk_n, (lane + j) & 31);
    }
    // where the chunk's last cell ends in the next chunk
    const int last = nd - base < 32 ? (int)(nd - base) - 1 : 31;
    const long long c_last = __shfl_sync(0xffffffffu, c, last);
    const unsigned ends = __ballot_sync(0xffffffffu, valid_n && cell_of(u_n) != c_last);
    if (head) {
      // the first key of cell c writes the cell's bit, its record, the
      // records of the empty cells before it, and the key/rank pairs of the
      // keys beyond the record's inline ones (the only pairs a probe reads)
      if (r.use_bits) atomicOr(&a.bitmap[c >> 5], 1u << (c & 31));
      const uint32_t zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (long long h = prev_c + 1; h < c; ++h) store_cell(&a.table[h], zero);
      const unsigned later = lane < 31 ? heads & (0xfffffffeu << lane) : 0u;
      int64_t e;
      if (later) {
        e = base + (__ffs(later) - 1);
      } else if (ends) {  // the chunk's last cell ends in the next chunk
        e = base + 32 + (__ffs(ends) - 1);
      } else {  // it covers the next chunk's keys (or the keys end)
        e = base + 64;
        while (e < nd && cell_of(image_at(e)) == c) ++e;
        if (e > nd) e = nd;
      }
      const int cnt = (int)(e - p);
      uint32_t w[8] = {0, 0, 0, 0, 0, 0, (uint32_t)p, (uint32_t)cnt};
      const int ninl = cnt < cap ? cnt : cap;
      for (int j = 0; j < ninl; ++j) {
        const bool in_warp = lane + j < 32;
        const unsigned long long uj = in_warp ? (j == 0 ? un[0] : j == 1 ? un[1] : un[2]) : (j == 1 ? wn[1] : wn[2]);
        const int32_t rj = in_warp ? (j == 0 ? rn[0] : j == 1 ? rn[1] : rn[2]) : (j == 1 ? wr[1] : wr[2]);
        if (k32) {
          w[j] = (uint32_t)uj;
          w[3 + j] = (uint32_t)rj;
        } else {
          w[2 * j] = (uint32_t)uj;
          w[2 * j + 1] = (uint32_t)(uj >> 32);
          w[4 + j] = (uint32_t)rj;
        }
      }
      for (int j = cap; j < cnt; ++j) {
        const unsigned long long uj = image_at(p + j);
        const int32_t rj = rank_at(p + j);
        if (k32)
          static_cast<KeyRank32*>(a.kr)[p + j] = KeyRank32{(uint32_t)uj, rj};
        else
          static_cast<KeyRank64*>(a.kr)[p + j] = KeyRank64{uj, (long long)rj};
      }
      store_cell(&a.table[c], w);
    }
  }
}


__global__ void dir_fill_kernel(const void* skeys, int key_dt, int64_t n_max, const int64_t* d_n, const DimDir* dd,
                                int* dir, uint32_t* bitmap) {
  const int64_t nd = clamp_n(n_max, d_n);
  const DimDir r = *dd;
  if (r.fused) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd; p += stride) {
    long long c = (long long)((key_image(skeys, key_dt, p) - r.umin) >> r.bshift);
    long long prev = p ? (long long)((key_image(skeys, key_dt, p - 1) - r.umin) >> r.bshift) : -1;
    if (c != prev) {
      for (long long h = prev + 1; h <= c; ++h) dir[h] = (int)p;
      atomicOr(&bitmap[c >> 5], 1u << (c & 31));
    }
    if (p == nd - 1) dir[c + 1] = (int)nd;
  }
}

// Unit-width cells (bshift == 0) also get per-cell copies of the group rank
// and of the aggregated dimension values, so that a probe hit reads them
// directly by cell instead of through the position table.
struct CellArgs {
  const void* skeys;
  int key_dt;
  int64_t n_max;
  const int64_t* d_n;
  const DimDir* dd;
  const int32_t* rank_sorted;
  int32_t* rank_cell;
  int nv;
  const long long* dval[TQP_MAX_VALS];
  long long* dval_cell[TQP_MAX_VALS];
};

__global__ void dir_cells_kernel(CellArgs a) {
  const DimDir r = *a.dd;
  if (r.bshift != 0 || r.ncells == 0) return;
  const int64_t nd = clamp_n(a.n_max, a.d_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nd; p += stride) {
    const long long c = (long long)(key_image(a.skeys, a.key_dt, p) - r.umin);
    a.rank_cell[c] = a.rank_sorted[p];
    for (int v = 0; v < a.nv; ++v) a.dval_cell[v][c] = a.dval[v][p];
  }
}

__global__ void dir_table_kernel(const void* kr, int key_dt, const DimDir* dd, const int* dir, DirCell* table) {
  const DimDir r = *dd;
  if (r.bshift == 0 || r.ncells == 0 || r.fused) return;
  const bool k32 = key_dt == TQP_I32;
  const int cap = cell_inline(k32);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < r.ncells; c += stride) {
    const int lo = dir[c], cnt = dir[c + 1] - lo;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, (uint32_t)lo, (uint32_t)cnt};
    for (int j = 0; j < cap && j < cnt; ++j) {
      if (k32) {
        const KeyRank32 e = static_cast<const KeyRank32*>(kr)[lo + j];
        w[j] = e.image;
        w[3 + j] = (uint32_t)e.rank;
      } else {
        const KeyRank64 e = static_cast<const KeyRank64*>(kr)[lo + j];
        w[2 * j] = (uint32_t)e.image;
        w[2 * j + 1] = (uint32_t)(e.image >> 32);
        w[4 + j] = (uint32_t)e.rank;
      }
    }
    table[c].a = make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]);
    table[c].b = make_int4((int)w[4], (int)w[5], (int)w[6], (int)w[7]);
  }
}

struct ProbeDim {
  const void* kr;      // sorted passing keys' images with their group ranks (KeyRank32 / KeyRank64)
  int key_dt;
  const int32_t* rank_cell;
  const void* fk;      // fact foreign-key column (same dtype as the key)
  const DimDir* dir_plan;
  const DirCell* table;
  const uint32_t* bitmap;
};

struct ProbeArgs {
  unsigned* wcounter;  // warp tiles taken (predicate path)
  int ndims;
  int vec0;  // the first dimension's fact keys are int32 at a 16-byte aligned address
  ProbeDim dim[kMaxDims];
  int npred;
  const void* pcol[TQP_MAX_PREDS];
  int pdt[TQP_MAX_PREDS];
  int pop[TQP_MAX_PREDS];
  long long plit[TQP_MAX_PREDS];
  int nvals;
  int vsrc[TQP_MAX_VALS];     // 0 = fact column, 1 + d = pre-gathered dimension column
  const void* vptr[TQP_MAX_VALS];
  const void* vptr_cell[TQP_MAX_VALS];  // the same dimension column by cell (unit-width cells)
  int vdt[TQP_MAX_VALS];
  int64_t n_fact;
  const StarPlan* plan;
  long long* acc;
};

// ---- warp-level compaction queues of the probe
// A ring of 64 entries of F ints per warp in shared memory (field-major),
// with its head and fill count in registers (warp-uniform).
template <int F>
struct WarpRing {
  int* base;  // this warp's ring: F x 64 ints
  int head;
  int n;
};

// Appends the entries of the lanes whose flag is set.  Each time 32 entries
// are pending, drain(e, 32) runs with lane i holding entry i (in e[]), and
// those 32 leave the ring.  Every lane of the warp must call it.
template <int F, typename Drain>
__device__ __forceinline__ void ring_push(WarpRing<F>& q, bool flag, const int (&val)[F], Drain&& drain) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (m == 0) return;
  if (flag) {
    const int idx = (q.head + q.n + __popc(m & ((1u << lane) - 1u))) & 63;
#pragma unroll
    for (int f = 0; f < F; ++f) q.base[f * 64 + idx] = val[f];
  }
  q.n += __popc(m);
  if (q.n < 32) return;
  __syncwarp();
  int e[F];
#pragma unroll
  for (int f = 0; f < F; ++f) e[f] = q.base[f * 64 + ((q.head + lane) & 63)];
  __syncwarp();
  q.head = (q.head + 32) & 63;
  q.n -= 32;
  drain(e, 32);
}

// Drains what is pending (fewer than 32 entries).
template <int F, typename Drain>
__device__ __forceinline__ void ring_flush(WarpRing<F>& q, Drain&& drain) {
  if (q.n == 0) return;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  int e[F];
#pragma unroll
  for (int f = 0; f < F; ++f) e[f] = lane < q.n ? q.base[f * 64 + ((q.head + lane) & 63)] : 0;
  __syncwarp();
  const int cnt = q.n;
  q.head = (q.head + cnt) & 63;
  q.n = 0;
  drain(e, cnt);
}

// Fused probe + aggregate as a warp pipeline with dense stages.
//  1. Each thread takes ITEMS fact rows of the tile.  Without fact predicates
//     they go straight to the dimension probe.  With predicates, the passing
//     rows are compacted into a warp queue that feeds the probe 32 at a time.
//  2. Dimension probe per row: key image, range, cell bit; a unit-width cell
//     proves the key, otherwise the cell's record (and, past its inline
//     keys, the cell's sorted keys) gives its sorted position and rank.
//  3. Rows that find every dimension are compacted (row, partial group
//     slot, positions) into a second queue; the fold runs on 32 of them at
//     a time with all lanes active: unit cells' ranks, values and
//     expressions, accumulator updates.
// Compacting before the expensive stages keeps a warp's instructions on
// live rows (a fifth of the rows reach the fold in the Q14 shape).
// SMEM_BM: the first dimension's cell bitmap is copied into dynamic shared
// memory (when it fits in smem_bm_words) so that a miss costs one shared
// read; used for small first dimensions, one large block per SM.
// K32: every dimension key is int32, so the key image, its range test and
// the cell index are 32-bit arithmetic.
template <int THREADS, int ITEMS, bool SMEM_BM, bool K32, int ND>
__global__ void __launch_bounds__(THREADS, SMEM_BM ? 1 : 3) star_probe_kernel(ProbeArgs a, StarAcc Ag, int smem_bm_words) {
  using UK = typename std::conditional<K32, uint32_t, unsigned long long>::type;
  constexpr int WARPS = THREADS / 32;
  // the shared bitmap variant keeps a smaller accumulator array
  constexpr int ACC_WORDS = SMEM_BM ? kSmemAccWords / 4 : kSmemAccWords;
  __shared__ long long s_acc[ACC_WORDS];
  __shared__ int s_fring[WARPS][(2 + ND) * 64];  // probe survivors: row, slot, positions
  __shared__ int s_pring[WARPS][64];                   // rows that pass the fact predicates
  // the aggregate program and value references in shared memory: they are
  // indexed by runtime values below (kernel parameters indexed that way are
  // copied to local memory)
  __shared__ StarAcc A;
  __shared__ int s_vsrc[TQP_MAX_VALS], s_vdt[TQP_MAX_VALS];
  __shared__ const void* s_vptr[TQP_MAX_VALS];
  __shared__ const void* s_vptr_cell[TQP_MAX_VALS];
  if (threadIdx.x == 0) {
    A = Ag;
    for (int v = 0; v < TQP_MAX_VALS; ++v) {
      s_vsrc[v] = a.vsrc[v];
      s_vdt[v] = a.vdt[v];
      s_vptr[v] = a.vptr[v];
      s_vptr_cell[v] = a.vptr_cell[v];
    }
  }
  __syncthreads();
  const StarPlan* plan = a.plan;
  if (plan->unsupported) return;
  const long long S = plan->S;
  const int nacc = A.naggs + 1;
  const bool use_smem = plan->use_smem != 0 && S * nacc <= ACC_WORDS;
  const int lane = threadIdx.x & 31;
  // accumulator copies: as many as fit (up to one per warp); warp w uses copy w % copies
  int copies = 1;
  if (use_smem) {
    long long fit = ACC_WORDS / (S * nacc);
    copies = (int)(fit < WARPS ? fit : WARPS);
    if (copies < 1) copies = 1;
  }
  long long* my_acc = s_acc + ((threadIdx.x >> 5) % copies) * S * nacc;
  if (use_smem) {
    for (int i = threadIdx.x; i < S * nacc * copies; i += THREADS) s_acc[i] = acc_identity(A, (i % (S * nacc)) % nacc);
  }
  DimDir dd[ND];
  long long stride[ND];
  bool unit[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    dd[d] = *a.dim[d].dir_plan;
    stride[d] = plan->stride[d];
    unit[d] = dd[d].bshift == 0;
  }
  extern __shared__ uint32_t s_bm[];
  bool sbm = false;
  if (SMEM_BM) {
    const long long words = (dd[0].ncells + 31) / 32;
    sbm = words <= smem_bm_words;
    if (sbm)
      for (long long i = threadIdx.x; i < words; i += THREADS) s_bm[i] = __ldg(&a.dim[0].bitmap[i]);
  }
  // The simple program: every aggregate a COUNT or one term mul * v + add of
  // an int64 value (a fact column at the row, or a dimension column at the
  // row's position or cell).  Its fold reads each aggregate's value straight
  // through one pointer and index kind.
  __shared__ int s_simple;
  __shared__ const long long* s_ap[TQP_MAX_AGGS];
  __shared__ int s_ai[TQP_MAX_AGGS];  // value index: 0 the row, 1 the first dimension's position, 2 the last's
  __shared__ long long s_am[TQP_MAX_AGGS], s_aa[TQP_MAX_AGGS];
  if (threadIdx.x == 0) {
    int simple = 1;
    for (int q = 0; q < A.naggs; ++q) {
      s_ap[q] = nullptr;
      s_ai[q] = 0;
      s_am[q] = 1;
      s_aa[q] = 0;
      if (A.op[q] == TQP_COUNT) continue;
      const int e = A.expr[q];
      if (A.nterms[e] != 1) {
        simple = 0;
        continue;
      }
      const int vi = A.tval[e][0], src = s_vsrc[vi];
      if (src == 0 && s_vdt[vi] != TQP_I64) {
        simple = 0;
        continue;
      }
      const bool cell = src == 1 ? unit[0] : (src > 1 && unit[ND - 1]);
      s_ap[q] = static_cast<const long long*>(cell ? s_vptr_cell[vi] : s_vptr[vi]);
      s_ai[q] = src == 0 ? 0 : src == 1 ? 1 : 2;
      s_am[q] = A.tmul[e][0];
      s_aa[q] = A.tadd[e][0];
    }
    s_simple = simple;
  }
  __syncthreads();
  const bool simple = s_simple;

  // 2. probe of one fact row through every dimension.  The dimensions'
  // foreign keys load together, then their wide cells' records (after the
  // cell bit where a bitmap is tested), so a row waits on two dependent reads
  // whatever the number of dimensions.  pos: the sorted position (the cell of
  // a unit-width dimension); slot: the sum of rank * stride over the wide
  // dimensions (a unit cell's rank is read by the fold, on compacted rows).
  // pre: the first dimension's key image u0 is already loaded.
  auto fk_image = [&](int d, int64_t row) -> UK {
    const ProbeDim& D = a.dim[d];
    if (K32 || D.key_dt == TQP_I32) return (UK)((uint32_t)__ldg(static_cast<const int32_t*>(D.fk) + row) ^ 0x80000000u);
    return (UK)((unsigned long long)__ldg(static_cast<const long long*>(D.fk) + row) ^ 0x8000000000000000ull);
  };
  // The keys of a wide cell beyond its inline ones: the first key >= x in
  // kr[l, h), narrowed while the interval is long, then scanned.
  auto overflow = [&](int d, UK x, int l, const int hi, int& rk) -> int {
    const bool k32d = K32 || a.dim[d].key_dt == TQP_I32;
    auto img = [&](int i) -> UK {
      return k32d ? (UK)__ldg(&static_cast<const KeyRank32*>(a.dim[d].kr)[i].image)
                  : (UK)__ldg(&static_cast<const KeyRank64*>(a.dim[d].kr)[i].image);
    };
    int h = hi;
    while (h - l > 4) {
      const int mid = (l + h) >> 1;
      if (img(mid) < x) l = mid + 1; else h = mid;
    }
    for (int i = l; i < hi; ++i) {
      const UK ki = img(i);
      if (ki >= x) {
        if (ki != x) return -1;
        rk = k32d ? __ldg(&static_cast<const KeyRank32*>(a.dim[d].kr)[i].rank)
                  : (int)__ldg(&static_cast<const KeyRank64*>(a.dim[d].kr)[i].rank);
        return i;
      }
    }
    return -1;
  };
  auto probe = [&](bool live, int64_t row, int (&pos)[ND], int& slot, bool pre, UK u0) -> bool {
    UK u[ND], c[ND];
    bool lv[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      u[d] = 0;
      if (live) u[d] = (d == 0 && pre) ? u0 : fk_image(d, row);
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      lv[d] = live && u[d] >= (UK)dd[d].umin && u[d] <= (UK)dd[d].umax;
      c[d] = lv[d] ? (u[d] - (UK)dd[d].umin) >> dd[d].bshift : (UK)0;
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      if (lv[d] && dd[d].use_bits) {
        const uint32_t w = (SMEM_BM && d == 0 && sbm) ? s_bm[c[d] >> 5] : __ldg(&a.dim[d].bitmap[c[d] >> 5]);
        lv[d] = (w >> (c[d] & 31)) & 1u;
      }
    }
    int4 ra[ND], rb[ND];
    int rk[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      ra[d] = rb[d] = make_int4(0, 0, 0, 0);
      rk[d] = 0;
      if (lv[d] && !unit[d]) {
        ra[d] = __ldg(&a.dim[d].table[c[d]].a);
        rb[d] = __ldg(&a.dim[d].table[c[d]].b);
      }
    }
    bool all = live;
    int sl = 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      pos[d] = (int)c[d];
      if (!unit[d]) {
        // match the inline keys; a key above the last inline one of a fuller
        // cell is searched among the cell's remaining sorted keys
        const int lo = rb[d].z, cnt = rb[d].w;
        int found = -1;
        if (K32 || a.dim[d].key_dt == TQP_I32) {
          const uint32_t x = (uint32_t)u[d];
          if (cnt > 0 && (uint32_t)ra[d].x == x) { found = lo; rk[d] = ra[d].w; }
          else if (cnt > 1 && (uint32_t)ra[d].y == x) { found = lo + 1; rk[d] = rb[d].x; }
          else if (cnt > 2 && (uint32_t)ra[d].z == x) { found = lo + 2; rk[d] = rb[d].y; }
          else if (cnt > 3 && x > (uint32_t)ra[d].z) found = overflow(d, u[d], lo + 3, lo + cnt, rk[d]);
        } else {
          const unsigned long long x = (unsigned long long)u[d];
          const unsigned long long i0 = (unsigned long long)(uint32_t)ra[d].x | ((unsigned long long)(uint32_t)ra[d].y << 32);
          const unsigned long long i1 = (unsigned long long)(uint32_t)ra[d].z | ((unsigned long long)(uint32_t)ra[d].w << 32);
          if (cnt > 0 && i0 == x) { found = lo; rk[d] = rb[d].x; }
          else if (cnt > 1 && i1 == x) { found = lo + 1; rk[d] = rb[d].y; }
          else if (cnt > 2 && x > i1) found = overflow(d, u[d], lo + 2, lo + cnt, rk[d]);
        }
        lv[d] = lv[d] && found >= 0;
        pos[d] = found;
      }
      all = all && lv[d];
      sl += rk[d] * (int)stride[d];
    }
    slot = sl;
    return all;
  };

  // 3. fold of one surviving row: aggregate expressions, accumulator updates
  // in its group's slot
  auto term_value = [&](int vi, int row, const int (&pos)[ND]) -> long long {
    const int src = s_vsrc[vi];
    if (src == 0) return load_as_i64(s_vptr[vi], s_vdt[vi], row);
    const bool cell = src == 1 ? unit[0] : unit[ND - 1];
    return static_cast<const long long*>(cell ? s_vptr_cell[vi] : s_vptr[vi])[src == 1 ? pos[0] : pos[ND - 1]];
  };
  auto fold = [&](bool v, int row, int slot, const int (&pos)[ND]) {
    if (!v) return;
    int urk[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) urk[d] = unit[d] ? __ldg(&a.dim[d].rank_cell[pos[d]]) : 0;
#pragma unroll
    for (int d = 0; d < ND; ++d) slot += urk[d] * (int)stride[d];
    long long* dst = use_smem ? my_acc + (long long)slot * nacc : a.acc + (long long)slot * nacc;
    for (int q = 0; q < A.naggs; ++q) {
      long long x = 1;
      const int op = A.op[q];
      if (op != TQP_COUNT && simple) {
        const int ai = s_ai[q];
        const int idx = ai == 0 ? row : ai == 1 ? pos[0] : pos[ND - 1];
        x = (long long)((unsigned long long)s_am[q] * (unsigned long long)__ldg(s_ap[q] + idx) +
                        (unsigned long long)s_aa[q]);
      } else if (op != TQP_COUNT) {
        const int e = A.expr[q];
        unsigned long long ev = 1;
        for (int t = 0; t < A.nterms[e]; ++t)
          ev *= (unsigned long long)A.tmul[e][t] * (unsigned long long)term_value(A.tval[e][t], row, pos) +
                (unsigned long long)A.tadd[e][t];
        x = (long long)ev;
      }
      unsigned long long* d64 = reinterpret_cast<unsigned long long*>(dst + q);
      switch (op) {
        case TQP_MIN: atomicMin(dst + q, x); break;
        case TQP_MAX: atomicMax(dst + q, x); break;
        default:
          if (use_smem) shared_add_u64(d64, (unsigned long long)x);
          else atomicAdd(d64, (unsigned long long)x);
          break;
      }
    }
    if (A.cnt == A.naggs) {  // no COUNT aggregate: the extra accumulator counts the rows
      unsigned long long* d64 = reinterpret_cast<unsigned long long*>(dst + A.naggs);
      if (use_smem) shared_add_u64(d64, 1ull);
      else atomicAdd(d64, 1ull);
    }
  };

  WarpRing<2 + ND> fq;  // rows that found every dimension: row, slot, positions
  fq.base = s_fring[threadIdx.x >> 5];
  fq.head = fq.n = 0;
  WarpRing<1> pq;  // rows that pass the fact predicates
  pq.base = s_pring[threadIdx.x >> 5];
  pq.head = pq.n = 0;
  auto drain_fold = [&](const int (&e)[2 + ND], int cnt) {
    int pos[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) pos[d] = e[2 + d];
    fold(lane < cnt, e[0], e[1], pos);
  };
  auto push_survivor = [&](bool alive, int row, int slot, const int (&pos)[ND]) {
    int val[2 + ND];
    val[0] = row;
    val[1] = slot;
#pragma unroll
    for (int d = 0; d < ND; ++d) val[2 + d] = pos[d];
    ring_push(fq, alive, val, drain_fold);
  };
  auto drain_probe = [&](const int (&e)[1], int cnt) {
    int pos[ND], slot;
    const bool alive = probe(lane < cnt, e[0], pos, slot, false, (UK)0);
    push_survivor(alive, e[0], slot, pos);
  };
  // Pushes a tile's ITEMS probed rows (row0 + k * rstep) in a rolled loop:
  // the fold behind the queue then exists once in the loop's code (the
  // instruction cache holds the whole loop).  Each step takes item 0 and
  // shifts the rest down, so the arrays stay in registers.
  auto push_items = [&](bool (&alive)[ITEMS], int (&slot)[ITEMS], int (&pos)[ITEMS][ND], int row0, int rstep) {
#pragma unroll 1
    for (int k = 0; k < ITEMS; ++k) {
      push_survivor(alive[0], row0 + k * rstep, slot[0], pos[0]);
#pragma unroll
      for (int j = 0; j + 1 < ITEMS; ++j) {
        alive[j] = alive[j + 1];
        slot[j] = slot[j + 1];
#pragma unroll
        for (int d = 0; d < ND; ++d) pos[j][d] = pos[j + 1][d];
      }
    }
  };

  // 1. every warp walks its own tiles of 32 x ITEMS rows (no block barrier
  // in the loop)
  constexpr int WT = 32 * ITEMS;
  const int64_t nwt = (a.n_fact + WT - 1) / WT;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS;
  int64_t wt = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (a.npred == 0 && a.vec0 && ITEMS % 4 == 0) {
    // every row goes to the probe.  Lane l takes rows l*ITEMS .. l*ITEMS +
    // ITEMS - 1 of the tile, whose int32 first-dimension keys arrive in
    // ITEMS/4 16-byte loads; the next tile's keys load while this one is
    // probed.
    const int32_t* fk0 = static_cast<const int32_t*>(a.dim[0].fk);
    const bool bit_only = SMEM_BM && K32 && ND == 1 && unit[0] && sbm && dd[0].use_bits && dd[0].ncells > 0;
    const uint32_t umin0 = (uint32_t)dd[0].umin, span0 = (uint32_t)(dd[0].umax - dd[0].umin);
    auto load4 = [&](int64_t w, int j, UK (&dst)[ITEMS]) {
      const int64_t r = w * WT + (int64_t)lane * ITEMS + 4 * j;
      if (w < nwt && r + 3 < a.n_fact) {
        const int4 q = __ldg(reinterpret_cast<const int4*>(fk0 + r));
        dst[4 * j] = (UK)((uint32_t)q.x ^ 0x80000000u);
        dst[4 * j + 1] = (UK)((uint32_t)q.y ^ 0x80000000u);
        dst[4 * j + 2] = (UK)((uint32_t)q.z ^ 0x80000000u);
        dst[4 * j + 3] = (UK)((uint32_t)q.w ^ 0x80000000u);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          dst[4 * j + e] = (w < nwt && r + e < a.n_fact) ? (UK)((uint32_t)__ldg(fk0 + r + e) ^ 0x80000000u) : (UK)0;
      }
    };
    UK nxt[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS / 4; ++j) load4(wt, j, nxt);
    for (; wt < nwt; wt += nwarps) {
      UK cur[ITEMS];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) cur[k] = nxt[k];
#pragma unroll
      for (int j = 0; j < ITEMS / 4; ++j) load4(wt + nwarps, j, nxt);
      const int64_t r0 = wt * WT + (int64_t)lane * ITEMS;
      int pos[ITEMS][ND], slot[ITEMS];
      bool alive[ITEMS];
      if (bit_only) {
        // one dimension of unit cells with its bitmap in shared memory: the
        // cell bit is the whole probe
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
          const uint32_t c = (uint32_t)cur[k] - umin0;
          alive[k] = r0 + k < a.n_fact && c <= span0 && ((s_bm[c >> 5] >> (c & 31)) & 1u);
          pos[k][0] = (int)c;
          slot[k] = 0;
        }
      } else {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) alive[k] = probe(r0 + k < a.n_fact, r0 + k, pos[k], slot[k], true, cur[k]);
      }
      push_items(alive, slot, pos, (int)r0, 1);
    }
  } else if (a.npred == 0) {
    // every row goes to the probe; the next tile's first-dimension keys are
    // loaded while this tile is probed
    UK nxt[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t r = wt * WT + k * 32 + lane;
      nxt[k] = (wt < nwt && r < a.n_fact) ? fk_image(0, r) : (UK)0;
    }
    for (; wt < nwt; wt += nwarps) {
      UK cur[ITEMS];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) cur[k] = nxt[k];
      const int64_t wn = wt + nwarps;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int64_t r = wn * WT + k * 32 + lane;
        nxt[k] = (wn < nwt && r < a.n_fact) ? fk_image(0, r) : (UK)0;
      }
      int pos[ITEMS][ND], slot[ITEMS];
      bool alive[ITEMS];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int64_t r = wt * WT + k * 32 + lane;
        alive[k] = probe(r < a.n_fact, r, pos[k], slot[k], true, cur[k]);
      }
      push_items(alive, slot, pos, (int)(wt * WT + lane), 32);
    }
  } else {
    // fact predicates, then the passing rows into the probe queue.  Warp
    // tiles are taken from a counter: a tile's cost varies with the
    // dependent reads of its surviving rows.
    while (true) {
      {
        unsigned tk = 0;
        if (lane == 0) tk = atomicAdd(a.wcounter, 1u);
        wt = __shfl_sync(0xffffffffu, tk, 0);
      }
      if (wt >= nwt) break;
      unsigned pass = 0;  // bit k: row k * 32 + lane of the tile
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) pass |= (unsigned)(wt * WT + k * 32 + lane < a.n_fact) << k;
      for (int p = 0; p < a.npred; ++p) {
#pragma unroll
        for (int k = 0; k < ITEMS; ++k)
          if ((pass >> k) & 1u)
            if (!compare(load_as_i64(a.pcol[p], a.pdt[p], wt * WT + k * 32 + lane), a.pop[p], a.plit[p]))
              pass &= ~(1u << k);
      }
      // one rolled loop, so that the probe and the fold behind the queue
      // exist once in the loop's code
#pragma unroll 1
      for (int k = 0; k < ITEMS; ++k) {
        const int val[1] = {(int)(wt * WT + k * 32 + lane)};
        ring_push(pq, (pass >> k) & 1u, val, drain_probe);
      }
    }
  }
  // the partly filled queues: probe what is pending, then fold the rest
  ring_flush(pq, drain_probe);
  ring_flush(fq, drain_fold);
  if (use_smem) {
    __syncthreads();
    for (int i = threadIdx.x; i < S * nacc; i += THREADS) {
      int q = i % nacc;
      long long v = s_acc[i];
      for (int w = 1; w < copies; ++w) {  // merge the warps' copies
        long long x = s_acc[(long long)w * S * nacc + i];
        v = (q < A.naggs) ? agg_fold(A.op[q], v, x) : v + x;
      }
      if (v == acc_identity(A, q)) continue;
      if (q < A.naggs && A.op[q] == TQP_MIN) atomicMin(&a.acc[i], v);
      else if (q < A.naggs && A.op[q] == TQP_MAX) atomicMax(&a.acc[i], v);
      else atomicAdd(reinterpret_cast<unsigned long long*>(&a.acc[i]), (unsigned long long)v);
    }
  }
}

// ---- compaction of non-empty slots into the output (single-pass scan)
struct CompactArgs {
  const StarPlan* plan;
  const long long* acc;
  int naggs;
  int cnt;  // accumulator that counts rows (non-zero: the slot is a group)
  int ndims;
  const long long* gkey[kMaxDims];  // per dimension group key values by rank (null: no group column)
  int out_key_index[kMaxDims];      // which output key column (or -1)
  void* out_keys[kMaxDims];
  int out_dt[kMaxDims];
  long long* out_aggs;
  int64_t cap;
  int64_t* d_out_groups;
  unsigned long long* status;
  uint32_t* counter;
  uint32_t num_tiles;
};

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) star_compact_kernel(CompactArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ long long s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long S = a.plan->unsupported ? 0 : a.plan->S;
  const int nacc = a.naggs + 1;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) break;
    const int64_t base = (int64_t)tile * TILE + (int64_t)threadIdx.x * ITEMS;
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
      if (base + k < S && a.acc[(base + k) * nacc + a.cnt] > 0) live |= 1u << k;
    int total;
    int off = block_exclusive_sum<THREADS>(__popc(live), s_scan, &total);
    if (warp == 0) {
      long long e = lookback_exclusive(a.status, tile, total);
      if (lane == 0) s_excl = e;
    }
    __syncthreads();
    long long excl = s_excl;
    if (excl >= 0) {
      long long g = excl + off;
      for (int k = 0; k < ITEMS; ++k) {
        if (!(live & (1u << k))) continue;
        long long slot = base + k;
        if (g < a.cap) {
          for (int q = 0; q < a.naggs; ++q) a.out_aggs[g * a.naggs + q] = a.acc[slot * nacc + q];
          for (int d = 0; d < a.ndims; ++d) {
            if (a.out_key_index[d] < 0) continue;
            long long r = (slot / a.plan->stride[d]) % a.plan->G[d];
            store_from_i64(a.out_keys[a.out_key_index[d]], a.out_dt[d], g, a.gkey[d][r]);
          }
        }
        ++g;
      }
      if (tile == a.num_tiles - 1 && threadIdx.x == 0) {
        *a.d_out_groups = excl + total;
        if (excl + total > a.cap) raise_status(TQP_ERR_CAPACITY);
      }
    }
    __syncthreads();
  }
}

}  // namespace tqp
