// Batched instances of the join + filter + group-by query: all problems'
// dimension tables are encoded as (problem, key) and (problem, group) words
// and sorted together; one persistent probe kernel pulls fact tiles of every
// problem from one atomic work queue; one block per problem writes its
// groups.  The per-problem descriptors reach the device through kernel
// parameters (an upload kernel), so the whole sequence can be captured in a
// CUDA graph and replayed.
#pragma once

#include "common.cuh"
#include "join.cuh"
#include "sort.cuh"

namespace tqp {

constexpr int kBatchSmemWords = 5760;  // shared accumulator words per probe block (static smem < 48 KB)
constexpr int kUploadChunk = 96;

struct BatchProb {
  long long n_fact;
  const void* fact[TQP_BATCH_MAX_COLS];
  long long n_dim;
  const void* key;
  const void* group;
  void* out_keys;
  long long* out_aggs;
  long long cap;
  long long* d_out_groups;
  long long dim_off;   // first row in the concatenated dimension arrays
  long long tile_off;  // first global probe tile
  long long slot_off;  // first accumulator slot
  long long cell_off;  // first directory entry of this problem
  long long word_off;  // first bitmap word of this problem
  int log2cells;       // directory size bound (2^log2cells cells)
  int pad_;
};

// Per-problem key directory (as for a star dimension): cells of 2^bshift key
// values over [umin, umax]; dir[c] = first position of the problem's sorted
// keys in cell c or later; bit c marks a non-empty cell.
struct ProbDir {
  unsigned umin, umax;
  int bshift;
  int ncells;  // 0: no dimension rows
};

__global__ void batch_dir_plan_kernel(const BatchProb* probs, int nprob, const int32_t* key32, ProbDir* pd) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const BatchProb& P = probs[p];
  ProbDir r;
  if (P.n_dim == 0) {
    r.umin = 1;
    r.umax = 0;
    r.bshift = 0;
    r.ncells = 0;
  } else {
    r.umin = (unsigned)key32[P.dim_off] ^ 0x80000000u;
    r.umax = (unsigned)key32[P.dim_off + P.n_dim - 1] ^ 0x80000000u;
    unsigned span = r.umax - r.umin;
    int bits = span ? 32 - __clz((int)span) : 0;
    r.bshift = bits > P.log2cells ? bits - P.log2cells : 0;
    r.ncells = (int)(span >> r.bshift) + 1;
  }
  pd[p] = r;
}

__global__ void batch_dir_fill_kernel(const BatchProb* probs, const long long* dim_off, int nprob, long long total,
                                      const unsigned long long* skey, const int32_t* key32, const ProbDir* pd,
                                      int* dir, uint32_t* bitmap) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x; pos < total; pos += stride) {
    const int p = (int)(skey[pos] >> 32);
    const BatchProb& P = probs[p];
    const ProbDir r = pd[p];
    const long long j = pos - P.dim_off;
    int* d = dir + P.cell_off;
    uint32_t* bm = bitmap + P.word_off;
    int c = (int)((((unsigned)key32[pos] ^ 0x80000000u) - r.umin) >> r.bshift);
    int prev = j ? (int)((((unsigned)key32[pos - 1] ^ 0x80000000u) - r.umin) >> r.bshift) : -1;
    if (c != prev) {
      for (int h = prev + 1; h <= c; ++h) d[h] = (int)j;
      atomicOr(&bm[c >> 5], 1u << (c & 31));
    }
    if (j == P.n_dim - 1) d[c + 1] = (int)P.n_dim;
  }
}

struct UploadChunk {
  int first, count;
  BatchProb p[kUploadChunk];
};

__global__ void batch_upload_kernel(UploadChunk c, BatchProb* dst) {
  int i = threadIdx.x;
  if (i < c.count) dst[c.first + i] = c.p[i];
}

__global__ void batch_offsets_kernel(UploadChunk c, long long* dim_off, long long* tile_off) {
  int i = threadIdx.x;
  if (i < c.count) {
    dim_off[c.first + i] = c.p[i].dim_off;
    tile_off[c.first + i] = c.p[i].tile_off;
  }
}

struct BatchShape {
  int nfact_cols;
  int fact_dt[TQP_BATCH_MAX_COLS];
  int fk_col;
  int group_dt;
  int npred;
  int pcol[TQP_MAX_PREDS];
  int pop[TQP_MAX_PREDS];
  long long plit[TQP_MAX_PREDS];
  int nexprs;
  int nterms[TQP_MAX_EXPRS];
  int tcol[TQP_MAX_EXPRS][3];
  long long tmul[TQP_MAX_EXPRS][3];
  long long tadd[TQP_MAX_EXPRS][3];
  int naggs;
  int op[TQP_MAX_AGGS];
  int expr[TQP_MAX_AGGS];
};

__device__ __forceinline__ int find_problem(const long long* off, int nprob, long long x) {
  // last problem whose offset is <= x
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ unsigned group_bits(int dt, long long v) {
  switch (dt) {
    case TQP_I8: return (unsigned)(uint8_t)v ^ 0x80u;
    case TQP_I16: return (unsigned)(uint16_t)v ^ 0x8000u;
    default: return (unsigned)v ^ 0x80000000u;
  }
}

__device__ __forceinline__ long long group_value(int dt, unsigned b) {
  switch (dt) {
    case TQP_I8: return (int8_t)(uint8_t)(b ^ 0x80u);
    case TQP_I16: return (int16_t)(uint16_t)(b ^ 0x8000u);
    default: return (int32_t)(b ^ 0x80000000u);
  }
}

// Concatenated dimension rows -> (problem << 32 | key bits) and
// (problem << 32 | group bits), payload = row within the problem.
__global__ void batch_dim_encode_kernel(const BatchProb* probs, const long long* dim_off, int nprob, long long total,
                                        int group_dt, unsigned long long* ckey, int32_t* crow,
                                        unsigned long long* cgrp, int32_t* grow) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
    int p = find_problem(dim_off, nprob, r);
    long long j = r - dim_off[p];
    const BatchProb& P = probs[p];
    unsigned kb = (unsigned)static_cast<const int32_t*>(P.key)[j] ^ 0x80000000u;
    unsigned gb = group_bits(group_dt, load_as_i64(P.group, group_dt, j));
    ckey[r] = ((unsigned long long)p << 32) | kb;
    cgrp[r] = ((unsigned long long)p << 32) | gb;
    crow[r] = (int32_t)j;
    grow[r] = (int32_t)j;
  }
}

// Segment id of every position of the sorted (problem, group) words, and
// the group value at each segment head (single-pass look-back scan).
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) batch_seg_kernel(const unsigned long long* sorted, long long n,
                                                            int group_dt, int32_t* seg, long long* gval,
                                                            unsigned long long* status, uint32_t* counter,
                                                            uint32_t num_tiles) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ long long s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const long long base = (long long)tile * TILE + (long long)threadIdx.x * ITEMS;
    uint32_t head = 0;
    unsigned long long prev = (base > 0 && base < n) ? sorted[base - 1] : 0ull;
    unsigned long long key[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      long long p = base + k;
      key[k] = p < n ? sorted[p] : 0ull;
      if (p < n && (p == 0 || key[k] != (k ? key[k - 1] : prev))) head |= 1u << k;
    }
    int total;
    int off = block_exclusive_sum<THREADS>(__popc(head), s_scan, &total);
    if (warp == 0) {
      long long e = lookback_exclusive(status, tile, total);
      if (lane == 0) s_excl = e;
    }
    __syncthreads();
    const long long excl = s_excl;
    if (excl >= 0) {
      long long r = excl + off - 1;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        long long p = base + k;
        if (p < n) {
          if (head & (1u << k)) {
            ++r;
            gval[r] = group_value(group_dt, (unsigned)key[k]);
          }
          seg[p] = (int32_t)r;
        }
      }
    }
    __syncthreads();
  }
}

// Rank of each dimension row's group within its problem; group count per problem.
__global__ void batch_rank_kernel(const BatchProb* probs, const long long* dim_off, int nprob, long long total,
                                  const unsigned long long* sgrp, const int32_t* sgrow, const int32_t* seg,
                                  int32_t* rank_of_row, long long* G, long long* first_seg) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x; pos < total; pos += stride) {
    int p = (int)(sgrp[pos] >> 32);
    long long d0 = dim_off[p];
    int s0 = seg[d0];
    rank_of_row[d0 + sgrow[pos]] = seg[pos] - s0;
    if (pos == d0 + probs[p].n_dim - 1) {
      G[p] = (long long)(seg[pos] - s0) + 1;
      first_seg[p] = s0;
    }
  }
}

__global__ void batch_empty_groups_kernel(const BatchProb* probs, int nprob, long long* G) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob && probs[p].n_dim == 0) G[p] = 0;
}

// Key-sorted positions: local key (int32) and group rank; uniqueness check.
__global__ void batch_pregather_kernel(const unsigned long long* skey, const int32_t* srow, const long long* dim_off,
                                       long long total, const int32_t* rank_of_row, int32_t* key32,
                                       int32_t* rank_sorted, int* flag) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x; pos < total; pos += stride) {
    unsigned long long k = skey[pos];
    int p = (int)(k >> 32);
    key32[pos] = (int32_t)((unsigned)k ^ 0x80000000u);
    rank_sorted[pos] = rank_of_row[dim_off[p] + srow[pos]];
    if (pos > 0 && skey[pos - 1] == k) {
      if (atomicExch(flag, 1) == 0) raise_status(TQP_ERR_UNSUPPORTED);
    }
  }
}

__global__ void batch_init_acc_kernel(const BatchShape S, long long* acc, long long nslots) {
  const int nacc = S.naggs + 1;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nslots * nacc; i += stride) {
    int q = (int)(i % nacc);
    acc[i] = q < S.naggs ? agg_identity(S.op[q]) : 0;
  }
}

struct BatchProbeArgs {
  const ProbDir* pdir;
  const int* dir;
  const uint32_t* bitmap;
  const BatchProb* probs;
  const long long* tile_off;
  int nprob;
  long long num_tiles;
  const int32_t* key32;
  const int32_t* rank_sorted;
  const long long* G;
  const int* flag;
  long long* acc;
  uint32_t* queue;
};

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) batch_probe_kernel(BatchProbeArgs a, BatchShape Sg) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ long long s_acc[kBatchSmemWords];
  __shared__ uint32_t s_tile;
  __shared__ BatchShape S;  // indexed by runtime values: kept in shared memory
  // the simple program: every aggregate a COUNT or one term mul * col + add
  // of an int64 fact column
  __shared__ int s_simple;
  __shared__ int s_acol[TQP_MAX_AGGS];
  __shared__ long long s_am[TQP_MAX_AGGS], s_aa[TQP_MAX_AGGS];
  if (threadIdx.x == 0) {
    S = Sg;
    int simple = 1;
    for (int q = 0; q < Sg.naggs; ++q) {
      s_acol[q] = 0;
      s_am[q] = 1;
      s_aa[q] = 0;
      if (Sg.op[q] == TQP_COUNT) continue;
      const int e = Sg.expr[q];
      if (Sg.nterms[e] != 1 || Sg.fact_dt[Sg.tcol[e][0]] != TQP_I64) {
        simple = 0;
        continue;
      }
      s_acol[q] = Sg.tcol[e][0];
      s_am[q] = Sg.tmul[e][0];
      s_aa[q] = Sg.tadd[e][0];
    }
    s_simple = simple;
  }
  __syncthreads();
  const bool simple = s_simple;
  if (*a.flag) return;
  const int nacc = S.naggs + 1;
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1u);
    __syncthreads();
    const long long t = s_tile;
    __syncthreads();
    if (t >= a.num_tiles) break;
    const int p = find_problem(a.tile_off, a.nprob, t);
    const BatchProb& P = a.probs[p];
    const long long r0 = (t - a.tile_off[p]) * TILE;
    const long long Gp = a.G[p];
    const bool shared = Gp * nacc <= kBatchSmemWords;
    // one accumulator copy per warp when they fit (no cross-warp contention)
    const int copies = (Gp * nacc * (THREADS / 32) <= kBatchSmemWords) ? THREADS / 32 : 1;
    long long* my_acc = s_acc + (copies > 1 ? (threadIdx.x >> 5) * Gp * nacc : 0);
    long long* gacc = a.acc + P.slot_off * nacc;
    if (shared) {
      for (int i = threadIdx.x; i < Gp * nacc * copies; i += THREADS) {
        int q = (int)((i % (Gp * nacc)) % nacc);
        s_acc[i] = q < S.naggs ? agg_identity(S.op[q]) : 0;
      }
      __syncthreads();
    }
    const int32_t* keys = a.key32 + P.dim_off;
    const int32_t* ranks = a.rank_sorted + P.dim_off;
    const ProbDir pd = a.pdir[p];
    const int* dir = a.dir + P.cell_off;
    const uint32_t* bm = a.bitmap + P.word_off;
    // Rows in groups of four per thread, stage by stage (predicates, foreign
    // keys, cell bits, directory bounds, keys, ranks): each stage issues the
    // four rows' reads together, so a thread waits on one round trip per
    // stage instead of one per read of every row.  The fold then takes the
    // surviving rows one at a time in a rolled loop (one copy in the code).
    constexpr int Q = 4;
    static_assert(ITEMS % Q == 0, "rows per thread: a multiple of 4");
#pragma unroll 1
    for (int k0 = 0; k0 < ITEMS; k0 += Q) {
      long long row[Q];
      bool live[Q];
      int32_t x[Q];
      int c[Q], l[Q], hi[Q];
      long long g[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        row[j] = r0 + (long long)(k0 + j) * THREADS + threadIdx.x;
        live[j] = row[j] < P.n_fact;
      }
      for (int q = 0; q < S.npred; ++q) {
#pragma unroll
        for (int j = 0; j < Q; ++j)
          if (live[j]) live[j] = compare(load_as_i64(P.fact[S.pcol[q]], S.fact_dt[S.pcol[q]], row[j]), S.pop[q], S.plit[q]);
      }
      const int32_t* fk = static_cast<const int32_t*>(P.fact[S.fk_col]);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        x[j] = live[j] ? __ldg(fk + row[j]) : 0;
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const unsigned u = (unsigned)x[j] ^ 0x80000000u;
        live[j] = live[j] && u >= pd.umin && u <= pd.umax;
        c[j] = live[j] ? (int)((u - pd.umin) >> pd.bshift) : 0;
      }
#pragma unroll
      for (int j = 0; j < Q; ++j)
        if (live[j]) live[j] = (__ldg(&bm[c[j] >> 5]) >> (c[j] & 31)) & 1u;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        l[j] = hi[j] = 0;
        if (live[j]) {
          l[j] = __ldg(&dir[c[j]]);
          hi[j] = __ldg(&dir[c[j] + 1]);
        }
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        if (!live[j]) continue;
        int lo = l[j], h = hi[j];
        while (h - lo > 4) {  // first key >= x lies in [lo, h]
          const int mid = (lo + h) >> 1;
          if (keys[mid] < x[j]) lo = mid + 1; else h = mid;
        }
        while (lo < hi[j] && keys[lo] < x[j]) ++lo;
        live[j] = lo < hi[j] && keys[lo] == x[j];
        l[j] = lo;
      }
#pragma unroll
      for (int j = 0; j < Q; ++j) g[j] = live[j] ? (long long)__ldg(&ranks[l[j]]) : 0;
#pragma unroll 1
      for (int j = 0; j < Q; ++j) {
        if (live[0]) {
          const long long rw = row[0];
          long long* dst = shared ? my_acc + g[0] * nacc : gacc + g[0] * nacc;
          for (int q = 0; q < S.naggs; ++q) {
            long long xq = 1;
            const int op = S.op[q];
            if (op != TQP_COUNT && simple) {
              xq = (long long)((unsigned long long)s_am[q] *
                                   (unsigned long long)__ldg(static_cast<const long long*>(P.fact[s_acol[q]]) + rw) +
                               (unsigned long long)s_aa[q]);
            } else if (op != TQP_COUNT) {
              const int e = S.expr[q];
              unsigned long long v = 1;
              for (int tt = 0; tt < S.nterms[e]; ++tt) {
                const int cc = S.tcol[e][tt];
                const long long xv = load_as_i64(P.fact[cc], S.fact_dt[cc], rw);
                v *= (unsigned long long)S.tmul[e][tt] * (unsigned long long)xv + (unsigned long long)S.tadd[e][tt];
              }
              xq = (long long)v;
            }
            unsigned long long* d64 = reinterpret_cast<unsigned long long*>(dst + q);
            switch (op) {
              case TQP_MIN: atomicMin(dst + q, xq); break;
              case TQP_MAX: atomicMax(dst + q, xq); break;
              default:
                if (shared) shared_add_u64(d64, (unsigned long long)xq);
                else atomicAdd(d64, (unsigned long long)xq);
                break;
            }
          }
          unsigned long long* c64 = reinterpret_cast<unsigned long long*>(dst + S.naggs);
          if (shared) shared_add_u64(c64, 1ull);
          else atomicAdd(c64, 1ull);
        }
#pragma unroll
        for (int m = 0; m + 1 < Q; ++m) {  // next row into place 0 (registers, no indexing)
          live[m] = live[m + 1];
          row[m] = row[m + 1];
          g[m] = g[m + 1];
        }
      }
    }
    if (shared) {
      __syncthreads();
      for (int i = threadIdx.x; i < Gp * nacc; i += THREADS) {
        int q = i % nacc;
        long long v = s_acc[i];
        for (int w = 1; w < copies; ++w) {  // merge the warps' copies
          long long x = s_acc[(long long)w * Gp * nacc + i];
          v = (q < S.naggs) ? agg_fold(S.op[q], v, x) : v + x;
        }
        long long id = q < S.naggs ? agg_identity(S.op[q]) : 0;
        if (v == id) continue;
        if (q < S.naggs && S.op[q] == TQP_MIN) atomicMin(&gacc[i], v);
        else if (q < S.naggs && S.op[q] == TQP_MAX) atomicMax(&gacc[i], v);
        else atomicAdd(reinterpret_cast<unsigned long long*>(&gacc[i]), (unsigned long long)v);
      }
    }
    __syncthreads();
  }
}

// One block per problem: non-empty groups in rank (= group value) order.
__global__ void __launch_bounds__(256) batch_compact_kernel(const BatchProb* probs, const long long* G,
                                                            const long long* first_seg, const long long* gval,
                                                            const long long* acc, int naggs, int group_dt,
                                                            const int* flag) {
  __shared__ int s_scan[33];
  __shared__ long long s_base;
  const int p = blockIdx.x;
  const BatchProb& P = probs[p];
  const long long Gp = *flag ? 0 : G[p];
  const int nacc = naggs + 1;
  const long long* pacc = acc + P.slot_off * nacc;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (long long g0 = 0; g0 < Gp; g0 += 256) {
    long long g = g0 + threadIdx.x;
    int live = (g < Gp && pacc[g * nacc + naggs] > 0) ? 1 : 0;
    int total;
    int off = block_exclusive_sum<256>(live, s_scan, &total);
    long long pos = s_base + off;
    if (live && pos < P.cap) {
      store_from_i64(P.out_keys, group_dt, pos, gval[first_seg[p] + g]);
      for (int q = 0; q < naggs; ++q) P.out_aggs[pos * naggs + q] = pacc[g * nacc + q];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *P.d_out_groups = s_base;
    if (s_base > P.cap) raise_status(TQP_ERR_CAPACITY);
  }
}

}  // namespace tqp
