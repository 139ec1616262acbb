// Learned range partitioner: a monotone 1 -> H -> 1 network (clamp units,
// non-negative weights) trained on the GPU on the empirical CDF of a sorted
// key sample, then used to route the rows of a group-by into ordered
// key-range buckets that are sorted on-chip.
//
// Forward, gradient and Adam kernels are hand-written and deterministic
// (fixed reduction orders, no floating-point atomics).  The partition uses
// the network's bucket function exactly: because the bucket is a
// non-decreasing step function of the 24-bit normalised key q, it is fully
// described by its B-1 step positions t_b = min{q : bucket(q) >= b}, found
// by binary search with the same forward evaluation; a row's bucket is then
// the number of steps at or below its q.  Keys that are frequent in the
// sample are not scattered at all: their aggregates are folded in shared
// memory during the partition pass and merged into the output in key order.
#pragma once

#include "common.cuh"
#include "groupby.cuh"
#include "sort.cuh"

namespace tqp {

constexpr int kH = TQP_CDF_HIDDEN;
constexpr int kNP = 3 * kH + 1;   // parameters: w, b, a, c
constexpr int kGradLen = kNP + 1; // + loss
constexpr int kGradChunk = 1024;  // samples per gradient block
constexpr int kMaxHeavy = TQP_MAX_HEAVY;
constexpr int kDirBits = 12;      // directory over the top bits of q
constexpr int kLocalCap = 8192;   // rows a block sorts on-chip
constexpr int kWarpCap = 1024;    // rows one warp sorts on-chip
#ifndef TQP_LOCAL_THREADS
#define TQP_LOCAL_THREADS 512
#endif
constexpr int kLocalThreads = TQP_LOCAL_THREADS;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kLocalItems = kLocalCap / kLocalThreads;  // 16
// Bucket cursors of the scatter sit this many words apart (32: one per
// 128-byte L2 line), so that the per-row atomics on different cursors do
// not queue behind each other at one L2 line.
#ifndef TQP_CURSOR_STRIDE
#define TQP_CURSOR_STRIDE 32
#endif
constexpr int kCursorStride = TQP_CURSOR_STRIDE;

__device__ __forceinline__ float cdf_eval(const tqp_cdf_model& m, float x) {
  float f = m.c;
#pragma unroll 16
  for (int j = 0; j < kH; ++j) {
    float z = fmaf(m.w[j], x, m.b[j]);
    float h = fminf(fmaxf(z, 0.0f), 1.0f);
    f = fmaf(m.a[j], h, f);
  }
  return f;
}

__device__ __forceinline__ int cdf_bucket_of(float F, int B) {
  float t = fminf(fmaxf(F, 0.0f), 1.0f) * (float)B;
  int b = (int)t;
  return b < B - 1 ? b : B - 1;
}

__device__ __forceinline__ void load_model_shared(tqp_cdf_model& dst, const tqp_cdf_model* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(tqp_cdf_model) / 4); i += blockDim.x) d[i] = s[i];
}

// ---------------------------------------------------------------- forward
__global__ void cdf_forward_kernel(const tqp_cdf_model* gm, const float* x, int64_t n, float* F, int32_t* bucket,
                                   int B) {
  __shared__ tqp_cdf_model m;
  load_model_shared(m, gm);
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float f = cdf_eval(m, x[i]);
    if (F) F[i] = f;
    if (bucket) bucket[i] = cdf_bucket_of(f, B);
  }
}

struct AdamState {
  float m[kNP];
  float v[kNP];
  unsigned done;  // blocks of the current gradient launch that have written their partials
  int has_best;   // best[] holds the parameters of the lowest loss evaluated so far
  float best_loss;
  float best[kNP];
};

// Training modes of one gradient launch: a plain Adam step; an Adam step
// that first records the parameters it evaluated when their loss is the
// lowest so far; and the closing evaluation, which records likewise, takes
// no step, and restores the best parameters (so training never returns a
// network worse on its training pairs than the one it started from).
constexpr int kTrainStep = 0, kTrainStepKeepBest = 1, kTrainRestoreBest = 2;

__device__ __forceinline__ float* param_ptr(tqp_cdf_model* md, int k) {
  return k < kH ? &md->w[k] : k < 2 * kH ? &md->b[k - kH] : k < 3 * kH ? &md->a[k - 2 * kH] : &md->c;
}

// One Adam step (parameter k < kNP) from the summed gradient g, then the
// projection w, a >= 0.
__device__ __forceinline__ void adam_update(tqp_cdf_model* md, AdamState* st, const tqp_train_cfg& cfg, int step,
                                            int k, float g) {
  const float t = (float)(step + 1);
  float mk = cfg.beta1 * st->m[k] + (1.0f - cfg.beta1) * g;
  float vk = cfg.beta2 * st->v[k] + (1.0f - cfg.beta2) * g * g;
  st->m[k] = mk;
  st->v[k] = vk;
  float mh = mk / (1.0f - powf(cfg.beta1, t));
  float vh = vk / (1.0f - powf(cfg.beta2, t));
  float* p = param_ptr(md, k);
  float np = *p - cfg.lr * mh / (sqrtf(vh) + cfg.eps);
  bool nonneg = (k < kH) || (k >= 2 * kH && k < 3 * kH);
  if (nonneg && np < 0.0f) np = 0.0f;
  *p = np;
}

// ---------------------------------------------------------------- gradient
// One block per chunk of kGradChunk samples writes its partial sums
// [gw(H), gb(H), ga(H), gc, sum of squared residuals] to partial[block].
// With an Adam state, the block that finishes last sums the partials in block order (the same
// result whatever the finishing order), takes one Adam step, records the
// epoch's loss and re-arms the counter for the next launch.
__global__ void __launch_bounds__(256) cdf_grad_kernel(tqp_cdf_model* gm, const float* x, const float* y,
                                                       const int64_t* d_n, int64_t n_max, float* partial,
                                                       AdamState* st, tqp_train_cfg cfg, int step, float* loss_out,
                                                       int mode = kTrainStep) {
  __shared__ tqp_cdf_model m;
  __shared__ float sx[kGradChunk], sd[kGradChunk];
  __shared__ float red[4][3 * kH];
  __shared__ float s_loss[8], s_gc[8];
  load_model_shared(m, gm);
  __syncthreads();
  const int64_t n = clamp_n(n_max, d_n);
  const float scale = n > 0 ? 2.0f / (float)n : 0.0f;
  const int64_t base = (int64_t)blockIdx.x * kGradChunk;
  float loss = 0.0f, gc = 0.0f;
  for (int k = threadIdx.x; k < kGradChunk; k += 256) {
    int64_t i = base + k;
    float xi = 0.0f, d = 0.0f;
    if (i < n) {
      xi = x[i];
      float r = cdf_eval(m, xi) - y[i];
      loss = fmaf(r, r, loss);
      d = r * scale;
      gc += d;
    }
    sx[k] = xi;
    sd[k] = d;
  }
  // block sums of loss and gc in a fixed order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    loss += __shfl_xor_sync(0xffffffffu, loss, o);
    gc += __shfl_xor_sync(0xffffffffu, gc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_loss[threadIdx.x >> 5] = loss;
    s_gc[threadIdx.x >> 5] = gc;
  }
  __syncthreads();
  const int j = threadIdx.x & (kH - 1), q = threadIdx.x / kH;  // 4 quarters of the chunk
  const float wj = m.w[j], bj = m.b[j], aj = m.a[j];
  float gw = 0.0f, gb = 0.0f, ga = 0.0f;
  for (int k = q * (kGradChunk / 4); k < (q + 1) * (kGradChunk / 4); ++k) {
    float z = fmaf(wj, sx[k], bj);
    float h = fminf(fmaxf(z, 0.0f), 1.0f);
    float d = sd[k];
    ga = fmaf(d, h, ga);
    if (z > 0.0f && z < 1.0f) {
      float da = d * aj;
      gb += da;
      gw = fmaf(da, sx[k], gw);
    }
  }
  red[q][j] = gw;
  red[q][kH + j] = gb;
  red[q][2 * kH + j] = ga;
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * kGradLen;
  if (threadIdx.x < 3 * kH) {
    int t = threadIdx.x;
    out[t] = ((red[0][t] + red[1][t]) + red[2][t]) + red[3][t];
  } else if (threadIdx.x == 3 * kH) {
    float s = 0.0f;
    for (int w = 0; w < 8; ++w) s += s_gc[w];
    out[kNP - 1] = s;
  } else if (threadIdx.x == 3 * kH + 1) {
    float s = 0.0f;
    for (int w = 0; w < 8; ++w) s += s_loss[w];
    out[kNP] = s;
  }
  // ---- the last block to finish: the Adam step (st null: gradient only)
  if (st == nullptr) return;
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ float s_L;
  const int k = threadIdx.x;
  float g = 0.0f;
  if (k < kGradLen)
    for (unsigned b = 0; b < gridDim.x; ++b) g += __ldcg(&partial[(size_t)b * kGradLen + k]);
  if (k == kNP) {
    s_L = n > 0 ? g / (float)n : 0.0f;
    if (loss_out && mode != kTrainRestoreBest) loss_out[step] = s_L;
  }
  __syncthreads();
  if (mode != kTrainStep) {
    // the parameters this launch evaluated, if their loss is the lowest yet
    const bool better = !st->has_best || s_L < st->best_loss;
    if (better && k < kNP) st->best[k] = *param_ptr(gm, k);
    __syncthreads();
    if (better && k == 0) {
      st->best_loss = s_L;
      st->has_best = 1;
    }
  }
  if (mode != kTrainRestoreBest) {
    if (k < kNP) adam_update(gm, st, cfg, step, k, g);
  } else {
    if (k < kNP) *param_ptr(gm, k) = st->best[k];
    __syncthreads();
    if (k == 0 && loss_out) loss_out[step] = st->best_loss;  // the returned parameters' loss
  }
  if (k == 0) st->done = 0;
}

// Sums the block partials in block order: grad[k] (k < kNP), grad[kNP] = loss.
__global__ void cdf_grad_finish_kernel(const float* partial, int nblocks, const int64_t* d_n, int64_t n_max,
                                       float* grad) {
  int k = threadIdx.x;
  if (k >= kGradLen) return;
  float s = 0.0f;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * kGradLen + k];
  const int64_t n = clamp_n(n_max, d_n);
  grad[k] = (k == kNP) ? (n > 0 ? s / (float)n : 0.0f) : s;
}

// ---------------------------------------------------------------- learned group-by plan
struct LearnedPlan {
  int shift;            // q = p >> shift
  float inv;            // x = q * inv
  unsigned long long qmax;
  int dshift;           // directory index = q >> dshift
  int B;
  int nheavy;
  int min_count;
  int slight;           // sample keys that are not heavy
  int heavy_cut;        // sample count from which a key is heavy
};

// Identity CDF F(x) = x on [0, 1]: unit j ramps over [j/H, (j+1)/H].
__device__ __forceinline__ void model_identity(tqp_cdf_model* md) {
  for (int j = 0; j < kH; ++j) {
    md->w[j] = (float)kH;
    md->b[j] = -(float)j;
    md->a[j] = 1.0f / (float)kH;
  }
  md->c = 0.0f;
}

// Normalisation of the packed keys from the group plan: p <= pmax, where
// pmax packs every key column's (max - min).
__global__ void lp_init_kernel(const GroupPlan* gp, int nkeys, tqp_cdf_model* md, LearnedPlan* lp, AdamState* st,
                               int B, int min_count) {
  if (threadIdx.x != 0) return;
  unsigned long long pmax = 0;
  for (int k = 0; k < nkeys; ++k)
    if (gp->kmax[k] >= gp->kmin[k])
      pmax |= ((unsigned long long)gp->kmax[k] - (unsigned long long)gp->kmin[k]) << gp->shift[k];
  int bits = pmax ? 64 - __clzll((long long)pmax) : 0;
  int shift = bits > 24 ? bits - 24 : 0;
  unsigned long long qmax = pmax >> shift;
  model_identity(md);
  md->shift = shift;
  md->umin = 0;
  md->inv = qmax ? 1.0f / (float)qmax : 0.0f;
  lp->shift = shift;
  lp->inv = md->inv;
  lp->qmax = qmax;
  int qbits = qmax ? 64 - __clzll((long long)qmax) : 0;
  lp->dshift = qbits > kDirBits ? qbits - kDirBits : 0;
  lp->B = B;
  lp->nheavy = 0;
  lp->min_count = min_count;
  for (int k = 0; k < kNP; ++k) st->m[k] = st->v[k] = 0.0f;
  st->done = 0;
  st->has_best = 0;
}

__device__ __forceinline__ unsigned long long pack_row(const KeySet& ks, const GroupPlan* gp, int64_t row) {
  unsigned long long u = 0;
  for (int k = 0; k < ks.nkeys; ++k)
    u |= ((unsigned long long)load_as_i64(ks.col[k], ks.dt[k], row) - (unsigned long long)gp->kmin[k]) << gp->shift[k];
  return u;
}

// Strided sample: sample[j] = packed key of selected row floor(j * n / S).
__global__ void lp_sample_kernel(KeySet ks, const int32_t* sel, int64_t n_max, const int64_t* d_n,
                                 const GroupPlan* gp, int S, unsigned long long* sample) {
  const int64_t n = clamp_n(n_max, d_n);
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S) return;
  int64_t i = n > 0 ? (int64_t)j * n / S : 0;
  int64_t row = sel ? sel[i] : i;
  sample[j] = n > 0 ? pack_row(ks, gp, row) : 0ull;
}

// First index after the run of equal keys that holds i (sorted ascending),
// by galloping forward from i: a run of length r costs O(log r) loads.
__device__ __forceinline__ int run_end(const unsigned long long* a, int n, int i) {
  const unsigned long long k = a[i];
  int lo = i, step = 1;  // a[lo] == k
  while (lo + step < n && a[lo + step] == k) {
    lo += step;
    step <<= 1;
  }
  int hi = lo + step < n ? lo + step : n;  // a[hi] != k or hi == n
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] == k) lo = mid; else hi = mid;
  }
  return hi;
}

// First index of the run that holds i, by galloping backward.
__device__ __forceinline__ int run_begin(const unsigned long long* a, int i) {
  const unsigned long long k = a[i];
  int hi = i, step = 1;  // a[hi] == k
  while (hi - step >= 0 && a[hi - step] == k) {
    hi -= step;
    step <<= 1;
  }
  int lo = hi - step >= 0 ? hi - step : -1;  // a[lo] != k or lo == -1
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] == k) hi = mid; else lo = mid;
  }
  return hi;
}

// Heavy keys of the sorted sample and the light prefix, over chunks of
// kHeavyChunk consecutive samples (one thread each), in five launches:
//  - lp_runhist_kernel: counts of the runs of equal keys that start in each
//    chunk, as a histogram (counts >= min_count);
//  - lp_cut_kernel: the count cut: the smallest count >= min_count such
//    that at most kMaxHeavy keys reach it (none when want_heavy is 0);
//  - lp_chunk_kernel: per chunk, the heavy runs that start in it and its
//    light samples;
//  - lp_chunk_scan_kernel: exclusive scans of both, the totals (nheavy,
//    slight);
//  - lp_heavy_write_kernel: heavy keys in ascending order, and lpre[i] =
//    sample keys before i that are not heavy.
constexpr int kHeavyChunk = 16;
constexpr int kCutBins = 4096;

__global__ void lp_runhist_kernel(const unsigned long long* sorted, int S, const LearnedPlan* lp, int* hist) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = t * kHeavyChunk, i1 = i0 + kHeavyChunk < S ? i0 + kHeavyChunk : S;
  const int minc = lp->min_count;
  for (int i = i0; i < i1;) {
    const int e = run_end(sorted, S, i);
    if (i == 0 || sorted[i - 1] != sorted[i]) {
      const int c = e - i;
      if (c >= minc) atomicAdd(&hist[c < kCutBins - 1 ? c : kCutBins - 1], 1);
    }
    i = e;
  }
}

__global__ void lp_cut_kernel(const int* hist, int want_heavy, LearnedPlan* lp) {
  if (threadIdx.x != 0) return;
  const int minc = lp->min_count;
  int acc = 0, cut = 1 << 30;
  if (want_heavy)
    for (int c = kCutBins - 1; c >= minc && c >= 1; --c) {
      if (acc + hist[c] > kMaxHeavy) break;
      acc += hist[c];
      cut = c;
    }
  lp->heavy_cut = cut;
}

__global__ void lp_chunk_kernel(const unsigned long long* sorted, int S, const LearnedPlan* lp, int* ch, int* cl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = t * kHeavyChunk;
  if (i0 >= S) return;
  const int i1 = i0 + kHeavyChunk < S ? i0 + kHeavyChunk : S;
  const int cut = lp->heavy_cut;
  int nh = 0, nl = 0;
  for (int i = i0; i < i1;) {
    const int b = run_begin(sorted, i), e = run_end(sorted, S, i);
    const int ce = e < i1 ? e : i1;
    if (e - b >= cut) nh += (b == i);
    else nl += ce - i;
    i = ce;
  }
  ch[t] = nh;
  cl[t] = nl;
}

// One block of 1024 threads over the chunk counts.
__global__ void __launch_bounds__(1024) lp_chunk_scan_kernel(int nchunks, int* ch, int* cl, LearnedPlan* lp) {
  __shared__ int s_scan[33];
  const int per = (nchunks + 1023) / 1024;
  const int c0 = threadIdx.x * per, c1 = c0 + per < nchunks ? c0 + per : nchunks;
  int sh = 0, sl = 0;
  for (int c = c0; c < c1; ++c) {
    sh += ch[c];
    sl += cl[c];
  }
  int htot, ltot;
  int hrun = block_exclusive_sum<1024>(sh, s_scan, &htot);
  int lrun = block_exclusive_sum<1024>(sl, s_scan, &ltot);
  for (int c = c0; c < c1; ++c) {
    const int h = ch[c], l = cl[c];
    ch[c] = hrun;
    cl[c] = lrun;
    hrun += h;
    lrun += l;
  }
  if (threadIdx.x == 0) {
    lp->nheavy = htot;
    lp->slight = ltot;
  }
}

__global__ void lp_heavy_write_kernel(const unsigned long long* sorted, int S, const LearnedPlan* lp, const int* ch,
                                      const int* cl, unsigned long long* heavy, int32_t* lpre) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = t * kHeavyChunk;
  if (i0 >= S) return;
  const int i1 = i0 + kHeavyChunk < S ? i0 + kHeavyChunk : S;
  const int cut = lp->heavy_cut;
  int hbase = ch[t], lrun = cl[t];
  for (int i = i0; i < i1;) {
    const int b = run_begin(sorted, i), e = run_end(sorted, S, i);
    const int ce = e < i1 ? e : i1;
    const bool hv = e - b >= cut;
    if (hv && b == i) heavy[hbase++] = sorted[i];
    for (int j = i; j < ce; ++j) lpre[j] = hv ? lrun : lrun + (j - i);
    if (!hv) lrun += ce - i;
    i = ce;
  }
}

// Training pairs from every mult-th key of the sorted sample (S keys):
// x = normalised key, y = the CDF of the light rows (the rows the buckets
// receive) over the whole sample at the key's midpoint:
// (light keys before the key + its light count / 2) / light total.  A heavy
// key has no light count: its pair sits on the light CDF with zero width.
// Without heavy keys this is (first rank + count / 2) / S.
__global__ void lp_targets_kernel(const unsigned long long* sorted, int S, int mult, int S_train,
                                  const LearnedPlan* lp, const int32_t* lpre, float* x, float* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S_train) return;
  const int j = (int)((int64_t)i * mult);
  const unsigned long long k = sorted[j];
  const int lo = run_begin(sorted, j), hi = run_end(sorted, S, j);
  const int light = (hi < S ? lpre[hi] : lp->slight) - lpre[lo];
  const double tot = lp->slight > 0 ? (double)lp->slight : 1.0;
  y[i] = (float)(((double)lpre[lo] + 0.5 * (double)light) / tot);
  x[i] = (float)(k >> lp->shift) * lp->inv;
}

// Knots at the quantiles of the training targets: unit j ramps from the
// first x whose target reaches j/H to the first whose target reaches
// (j+1)/H, with weight 1/H, so F starts as the piecewise-linear empirical CDF
// of the light rows (a ramp at least one q step wide stands for a step).
__device__ __forceinline__ int first_at_least(const float* ys, int S, float t) {
  int lo = 0, len = S;
  while (len > 0) {
    int h = len >> 1;
    if (ys[lo + h] < t) { lo += h + 1; len -= h + 1; } else { len = h; }
  }
  return lo < S ? lo : S - 1;
}

__global__ void lp_quantile_init_kernel(const float* xs, const float* ys, int S, const LearnedPlan* lp,
                                        tqp_cdf_model* md) {
  const int j = threadIdx.x;
  if (j >= kH) return;
  int i0 = first_at_least(ys, S, (float)j / (float)kH);
  int i1 = first_at_least(ys, S, (float)(j + 1) / (float)kH);
  float x0 = xs[i0], x1 = xs[i1];
  float step = lp->inv > 0.0f ? lp->inv : 1.0f;
  float width = x1 - x0 > step ? x1 - x0 : step;
  float w = 1.0f / width;
  md->w[j] = w;
  md->b[j] = -x0 * w;
  md->a[j] = 1.0f / (float)kH;
  if (j == 0) md->c = 0.0f;
}


// Step positions of the bucket function: thr[b-1] = min{q : bucket(q) >= b}
// (qmax + 1 if none), b = 1..B-1.
__global__ void lp_thresholds_kernel(const tqp_cdf_model* gm, const LearnedPlan* lp, unsigned* thr) {
  __shared__ tqp_cdf_model m;
  load_model_shared(m, gm);
  __syncthreads();
  const int B = lp->B;
  int b = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (b >= B) return;
  const unsigned long long qmax = lp->qmax;
  unsigned long long lo = 0, hi = qmax + 1;
  while (lo < hi) {
    unsigned long long mid = (lo + hi) >> 1;
    float x = (float)mid * m.inv;
    if (cdf_bucket_of(cdf_eval(m, x), B) >= b) hi = mid; else lo = mid + 1;
  }
  thr[b - 1] = (unsigned)lo;
}

// dir[h] = number of steps below h << dshift, h = 0..2^kDirBits.
__global__ void lp_directory_kernel(const LearnedPlan* lp, const unsigned* thr, int* dir) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h > (1 << kDirBits)) return;
  const int nt = lp->B - 1;
  unsigned long long v = (unsigned long long)h << lp->dshift;
  int lo = 0, len = nt;
  while (len > 0) {
    int half = len >> 1;
    if ((unsigned long long)thr[lo + half] < v) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  dir[h] = lo;
}

// Bucket of packed key p: the directory narrows the steps to those of q's
// top bits, a binary search finds the first step above q.  thr is in shared
// memory (THR_SMEM) or global memory.
template <bool THR_SMEM>
__device__ __forceinline__ int lp_bucket(unsigned long long p, const LearnedPlan& lp, const int* s_dir,
                                         const unsigned* thr) {
  unsigned long long q = p >> lp.shift;
  int h = (int)(q >> lp.dshift);
  int lo = s_dir[h], hi = s_dir[h + 1];
  while (lo < hi) {  // first step above q
    int mid = (lo + hi) >> 1;
    const unsigned t = THR_SMEM ? thr[mid] : __ldg(&thr[mid]);
    if ((unsigned long long)t <= q) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct PartArgs {
  KeySet ks;
  const int32_t* sel;       // keys at sel[i] (null: at i)
  const int32_t* payload;   // row id written for key i (null: the key's row)
  int64_t n_max;
  const int64_t* d_n;
  const GroupPlan* gp;
  const LearnedPlan* lp;
  const unsigned* thr;
  const int* dir;
  const unsigned long long* heavy;
  unsigned* count;          // [B]
  unsigned* cursor;         // [B * kCursorStride]: bucket b's cursor at b * kCursorStride
  unsigned* bcount;         // kBlockHist: [blocks][B] counts
  unsigned long long* out_p;
  int32_t* out_row;
  long long* heavy_acc;     // [nheavy][naggs]
  unsigned short* ids;      // the counting pass's bucket of every row (no heavy keys, B <= 65536), or null
  int coarse_F;             // > 0: the counting pass counts coarse buckets b >> coarse_F only (into
                            // count[c << coarse_F]); the fine counts come after split 1
};

// ---- partition kernels: shared-memory layout and setup
constexpr int kHeavyBits = 11;
constexpr int kHeavySlots = 1 << kHeavyBits;  // open addressing, load <= 1/2
constexpr int kPartThreads = 1024;
constexpr int kPartItems = 4;
constexpr int kHistItems = 8;  // rows per thread per round of the counting pass (loads in flight)

// Partition modes: the bucket function's steps in global memory, in shared
// memory, or (counting only) in shared memory with per-block bucket counts:
// each block counts one contiguous chunk of rows in shared memory.
constexpr int kThrGlobal = 0, kThrShared = 1, kBlockHist = 2;
constexpr int kPartCoarseBins = 512;  // coarse buckets a counting pass may count in shared memory
constexpr int kBlockHistMaxB = 1 << 14;

// Dynamic shared memory: directory, heavy-key table (key, index; index -1 =
// empty), the heavy accumulators (scatter), the steps (kThrShared and up)
// and the block's bucket counts (kBlockHist).
struct PartSmem {
  int* dir;
  unsigned long long* hk;
  int* hv;
  long long* acc;
  unsigned* thr;
  unsigned* bh;
};

inline __host__ __device__ size_t part_smem_bytes(int B, int naggs, int mode) {
  size_t o = ((((size_t)1 << kDirBits) + 1) * 4 + 15) & ~(size_t)15;
  o += (size_t)kHeavySlots * 8 + (size_t)kHeavySlots * 4;
  o += (size_t)kMaxHeavy * naggs * 8;
  if (mode >= kThrShared) o += (size_t)(B > 1 ? B - 1 : 1) * 4;
  if (mode == kBlockHist) o += (size_t)B * 4;
  return o;
}

__device__ __forceinline__ PartSmem part_carve(unsigned char* base, int naggs, int B) {
  PartSmem S;
  size_t o = ((((size_t)1 << kDirBits) + 1) * 4 + 15) & ~(size_t)15;
  S.dir = reinterpret_cast<int*>(base);
  S.hk = reinterpret_cast<unsigned long long*>(base + o);
  o += (size_t)kHeavySlots * 8;
  S.hv = reinterpret_cast<int*>(base + o);
  o += (size_t)kHeavySlots * 4;
  S.acc = reinterpret_cast<long long*>(base + o);
  o += (size_t)kMaxHeavy * naggs * 8;
  S.thr = reinterpret_cast<unsigned*>(base + o);
  o += (size_t)(B > 1 ? B - 1 : 1) * 4;
  S.bh = reinterpret_cast<unsigned*>(base + o);
  return S;
}

__device__ __forceinline__ int heavy_slot(unsigned long long p) {
  return (int)((p * 0x9E3779B97F4A7C15ull) >> (64 - kHeavyBits));
}

// Index of p among the heavy keys, or -1.  The table is at most half full,
// so a probe sequence ends at an empty slot.
__device__ __forceinline__ int heavy_lookup(const PartSmem& S, unsigned long long p) {
  int slot = heavy_slot(p);
  for (int t = 0; t < kHeavySlots; ++t) {
    const int v = S.hv[slot];
    if (v < 0) return -1;
    if (S.hk[slot] == p) return v;
    slot = (slot + 1) & (kHeavySlots - 1);
  }
  return -1;
}

// The key columns and their packing, staged in shared memory.
struct PackPlan {
  int nkeys;
  const void* col[TQP_MAX_KEYS];
  int dt[TQP_MAX_KEYS];
  long long kmin[TQP_MAX_KEYS];
  int shift[TQP_MAX_KEYS];
};

__device__ __forceinline__ unsigned long long pack_row_plan(const PackPlan& K, int64_t row) {
  unsigned long long u = 0;
  for (int k = 0; k < K.nkeys; ++k)
    u |= ((unsigned long long)load_as_i64(K.col[k], K.dt[k], row) - (unsigned long long)K.kmin[k]) << K.shift[k];
  return u;
}

// The packed keys of N rows (rows[k], where valid[k]; 0 elsewhere).  With
// one key column the N loads are issued together under one switch on its
// dtype, instead of one round trip per row through pack_row_plan.
template <int N>
__device__ __forceinline__ void pack_rows(const PackPlan& K, const int64_t (&rows)[N], const bool (&valid)[N],
                                          unsigned long long (&out)[N]) {
  if (K.nkeys == 1) {
    const unsigned long long kmin = (unsigned long long)K.kmin[0];
    const int sh = K.shift[0];
    long long v[N];
    switch (K.dt[0]) {
      case TQP_I8: {
        const int8_t* c = static_cast<const int8_t*>(K.col[0]);
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = valid[k] ? c[rows[k]] : 0;
        break;
      }
      case TQP_I16: {
        const int16_t* c = static_cast<const int16_t*>(K.col[0]);
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = valid[k] ? c[rows[k]] : 0;
        break;
      }
      case TQP_I32: {
        const int32_t* c = static_cast<const int32_t*>(K.col[0]);
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = valid[k] ? c[rows[k]] : 0;
        break;
      }
      default: {
        const long long* c = static_cast<const long long*>(K.col[0]);
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = valid[k] ? c[rows[k]] : 0;
        break;
      }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = valid[k] ? ((unsigned long long)v[k] - kmin) << sh : 0ull;
    return;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) out[k] = valid[k] ? pack_row_plan(K, rows[k]) : 0ull;
}

// Directory, heavy table, steps (kThrShared and up) and key plan into shared memory.
template <int MODE>
__device__ __forceinline__ void part_setup(const PartArgs& a, const LearnedPlan& lp, const PartSmem& S, PackPlan& K) {
  for (int i = threadIdx.x; i <= (1 << kDirBits); i += blockDim.x) S.dir[i] = a.dir[i];
  for (int i = threadIdx.x; i < kHeavySlots; i += blockDim.x) S.hv[i] = -1;
  if (MODE >= kThrShared)
    for (int i = threadIdx.x; i < lp.B - 1; i += blockDim.x) S.thr[i] = a.thr[i];
  if (threadIdx.x == 0) {
    K.nkeys = a.ks.nkeys;
    for (int k = 0; k < TQP_MAX_KEYS; ++k) {
      K.col[k] = a.ks.col[k];
      K.dt[k] = a.ks.dt[k];
      K.kmin[k] = a.gp->kmin[k];
      K.shift[k] = a.gp->shift[k];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < lp.nheavy; i += blockDim.x) {
    const unsigned long long p = a.heavy[i];
    int slot = heavy_slot(p);
    while (atomicCAS(&S.hv[slot], -1, i) != -1) slot = (slot + 1) & (kHeavySlots - 1);
    S.hk[slot] = p;
  }
  __syncthreads();
}

// Rows a block partitions in kBlockHist mode: one contiguous chunk.
__device__ __forceinline__ void block_chunk(int64_t n, int64_t* c0, int64_t* c1) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  *c0 = (int64_t)blockIdx.x * chunk;
  *c1 = *c0 + chunk < n ? *c0 + chunk : n;
}

// Light rows per bucket (kBlockHist: per block, into bcount).  Each thread
// carries kHistItems rows at a time.
template <int MODE>
__global__ void __launch_bounds__(kPartThreads, 1) lp_hist_kernel(PartArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PackPlan K;
  __shared__ unsigned s_coarse[kPartCoarseBins];  // coarse_F > 0: the block's coarse counts
  const LearnedPlan lp = *a.lp;
  const PartSmem S = part_carve(smem, 0, lp.B);
  const int cF = MODE == kBlockHist ? 0 : a.coarse_F;
  if (MODE == kBlockHist)
    for (int b = threadIdx.x; b < lp.B; b += kPartThreads) S.bh[b] = 0;
  if (cF)
    for (int c = threadIdx.x; c < kPartCoarseBins; c += kPartThreads) s_coarse[c] = 0;
  part_setup<MODE>(a, lp, S, K);
  const unsigned* thr = MODE >= kThrShared ? S.thr : a.thr;
  const int nh = lp.nheavy;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  constexpr int TILE = kPartThreads * kHistItems;
  int64_t c0 = (int64_t)blockIdx.x * TILE, c1 = n, step = (int64_t)gridDim.x * TILE;
  if (MODE == kBlockHist) {
    block_chunk(n, &c0, &c1);
    step = TILE;
  }
  for (int64_t base = c0; base < c1; base += step) {
    unsigned long long p[kHistItems];
    bool v[kHistItems];
    int64_t rw[kHistItems];
#pragma unroll
    for (int k = 0; k < kHistItems; ++k) {
      const int64_t i = base + k * kPartThreads + threadIdx.x;
      v[k] = i < c1;
      rw[k] = v[k] ? (a.sel ? (int64_t)a.sel[i] : i) : 0;
    }
    pack_rows(K, rw, v, p);
#pragma unroll
    for (int k = 0; k < kHistItems; ++k) {
      if (!v[k] || (nh && heavy_lookup(S, p[k]) >= 0)) continue;
      const int b = lp_bucket<MODE >= kThrShared>(p[k], lp, S.dir, thr);
      if (MODE == kBlockHist) atomicAdd(&S.bh[b], 1u);
      else if (cF) atomicAdd(&s_coarse[b >> cF], 1u);
      else atomicAdd(&a.count[b], 1u);
      if (a.ids) a.ids[base + k * kPartThreads + threadIdx.x] = (unsigned short)b;
    }
  }
  if (MODE == kBlockHist) {
    __syncthreads();
    for (int b = threadIdx.x; b < lp.B; b += kPartThreads) a.bcount[(size_t)blockIdx.x * lp.B + b] = S.bh[b];
  }
  if (cF) {
    __syncthreads();
    for (int c = threadIdx.x; c < (lp.B >> cF); c += kPartThreads)
      if (s_coarse[c]) atomicAdd(&a.count[c << cF], s_coarse[c]);
  }
}

// Bucket id of every (selected) row for the standalone partition: a light
// row its learned bucket 0..B-1, a row of heavy key h (ascending heavy keys)
// the id B + h.
template <int MODE>  // kThrGlobal or kThrShared
__global__ void __launch_bounds__(kPartThreads, 1) lp_bucket_ids_kernel(PartArgs a, int32_t* ids) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PackPlan K;
  const LearnedPlan lp = *a.lp;
  const PartSmem S = part_carve(smem, 0, lp.B);
  part_setup<MODE>(a, lp, S, K);
  const unsigned* thr = MODE >= kThrShared ? S.thr : a.thr;
  const int nh = lp.nheavy;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  const int64_t stride = (int64_t)gridDim.x * kPartThreads;
  for (int64_t i = (int64_t)blockIdx.x * kPartThreads + threadIdx.x; i < n; i += stride) {
    const unsigned long long p = pack_row_plan(K, a.sel ? (int64_t)a.sel[i] : i);
    const int h = nh ? heavy_lookup(S, p) : -1;
    ids[i] = h >= 0 ? lp.B + h : lp_bucket<MODE >= kThrShared>(p, lp, S.dir, thr);
  }
}

// off[b] = the first position of bucket id b among the n sorted ids
// (n where no id >= b follows), b = 0..nb.
__global__ void lp_offsets_sorted_kernel(const uint32_t* sorted, int64_t n_max, const int64_t* d_n, int nb,
                                         long long* off) {
  const int64_t n = clamp_n(n_max, d_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n == 0) {
    for (int64_t b = t0; b <= nb; b += stride) off[b] = 0;
    return;
  }
  for (int64_t p = t0; p < n; p += stride) {
    const long long cur = sorted[p];
    const long long prev = p ? (long long)sorted[p - 1] : -1;
    for (long long b = prev + 1; b <= cur; ++b) off[b] = p;
    if (p == n - 1)
      for (long long b = cur + 1; b <= nb; ++b) off[b] = n;
  }
}

// Statistics of a standalone partition from its offsets (one block).
__global__ void __launch_bounds__(1024) lp_partition_stats_kernel(const LearnedPlan* lp, const long long* off,
                                                                  const float* loss, int epochs,
                                                                  tqp_learned_stats* st) {
  __shared__ long long s_mx[32], s_ov[32], s_ne[32], s_or[32], s_sm[32];
  const int B = lp->B;
  long long mx = 0, ov = 0, ne = 0, orows = 0, small = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const long long c = off[b + 1] - off[b];
    mx = c > mx ? c : mx;
    ov += c > kLocalCap;
    orows += c > kLocalCap ? c : 0;
    ne += c > 0;
    small += (c > 1 && c <= kWarpCap) ? c : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
    ov += __shfl_xor_sync(0xffffffffu, ov, o);
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    orows += __shfl_xor_sync(0xffffffffu, orows, o);
    small += __shfl_xor_sync(0xffffffffu, small, o);
  }
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    s_mx[w] = mx; s_ov[w] = ov; s_ne[w] = ne; s_or[w] = orows; s_sm[w] = small;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  tqp_learned_stats r;
  r.buckets = B;
  r.heavy_keys = lp->nheavy;
  r.light_rows = off[B];
  r.max_bucket = r.over_capacity = r.nonempty = r.over_capacity_rows = r.small_rows = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    r.max_bucket = s_mx[w] > r.max_bucket ? s_mx[w] : r.max_bucket;
    r.over_capacity += s_ov[w];
    r.nonempty += s_ne[w];
    r.over_capacity_rows += s_or[w];
    r.small_rows += s_sm[w];
  }
  r.loss_first = (loss && epochs > 0) ? loss[0] : 0.0f;
  r.loss_last = (loss && epochs > 0) ? loss[epochs] : 0.0f;
  *st = r;
}

// kBlockHist: bucket totals over the blocks' counts.
__global__ void lp_bcols_kernel(const unsigned* bcount, int nblk, const LearnedPlan* lp, unsigned* count) {
  const int B = lp->B;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  unsigned t = 0;
  for (int k = 0; k < nblk; ++k) t += bcount[(size_t)k * B + b];
  count[b] = t;
}

// Exclusive scan of the bucket counts into offsets (and cursors), the
// light-row total, and statistics.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) lp_offsets_kernel(const LearnedPlan* lp, const unsigned* count, unsigned* off,
                                                          unsigned* cursor, tqp_learned_stats* stats,
                                                          const float* loss, int epochs, int64_t* light_n) {
  __shared__ int s_scan[33];
  __shared__ unsigned s_max[32];
  __shared__ int s_over[32], s_ne[32];
  __shared__ unsigned long long s_orows[32], s_srows[32];
  const int B = lp->B;
  const int per = (B + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  unsigned sum = 0, mx = 0;
  int over = 0, ne = 0;
  unsigned long long over_rows = 0, small_rows = 0;
#pragma unroll 8
  for (int b = b0; b < b0 + per && b < B; ++b) {
    unsigned c = count[b];
    sum += c;
    small_rows += (c > 1 && c <= (unsigned)kWarpCap) ? c : 0;
    mx = c > mx ? c : mx;
    over += c > (unsigned)kLocalCap;
    over_rows += c > (unsigned)kLocalCap ? c : 0;
    ne += c > 0;
  }
  int total;
  int excl = block_exclusive_sum<1024>((int)sum, s_scan, &total);
  unsigned run = (unsigned)excl;
#pragma unroll 8
  for (int b = b0; b < b0 + per && b < B; ++b) {
    off[b] = run;
    cursor[(size_t)b * kCursorStride] = run;
    run += count[b];
  }
  if (threadIdx.x == 1023) {
    off[B] = (unsigned)total;
    *light_n = total;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
    over += __shfl_xor_sync(0xffffffffu, over, o);
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
    over_rows += __shfl_xor_sync(0xffffffffu, over_rows, o);
    small_rows += __shfl_xor_sync(0xffffffffu, small_rows, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_max[threadIdx.x >> 5] = mx;
    s_over[threadIdx.x >> 5] = over;
    s_ne[threadIdx.x >> 5] = ne;
    s_orows[threadIdx.x >> 5] = over_rows;
    s_srows[threadIdx.x >> 5] = small_rows;
  }
  __syncthreads();
  if (threadIdx.x == 0 && stats) {
    unsigned m3 = 0;
    long long o3 = 0, n3 = 0, r3 = 0, q3 = 0;
    for (int w = 0; w < 32; ++w) {
      q3 += (long long)s_srows[w];
      m3 = s_max[w] > m3 ? s_max[w] : m3;
      o3 += s_over[w];
      n3 += s_ne[w];
      r3 += (long long)s_orows[w];
    }
    stats->over_capacity_rows = r3;
    stats->small_rows = q3;
    stats->buckets = B;
    stats->heavy_keys = lp->nheavy;
    stats->light_rows = total;
    stats->max_bucket = m3;
    stats->over_capacity = o3;
    stats->nonempty = n3;
    stats->loss_first = (loss && epochs > 0) ? loss[0] : 0.0f;
    stats->loss_last = (loss && epochs > 0) ? loss[epochs] : 0.0f;  // the returned (best) network's
  }
}

__global__ void lp_heavy_init_kernel(const LearnedPlan* lp, AggProgram P, long long* acc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < lp->nheavy * P.naggs) acc[i] = agg_identity(P.op[i % P.naggs]);
}

__device__ __forceinline__ void fold_atomic(long long* slot, int op, long long x) {
  switch (op) {
    case TQP_MIN: atomicMin(slot, x); break;
    case TQP_MAX: atomicMax(slot, x); break;
    default: atomicAdd(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)x); break;
  }
}

// The same fold into an accumulator in shared memory (SUM and COUNT through
// the split 32-bit adds).
// MIN / MAX read the current value first and take the atomic only when x
// would change it: a hot key's extreme settles early, so most rows skip the
// compare-and-swap loop (the atomic alone decides; the read only filters).
__device__ __forceinline__ void fold_shared(long long* slot, int op, long long x) {
  switch (op) {
    case TQP_MIN:
      if (x < *reinterpret_cast<volatile long long*>(slot)) atomicMin(slot, x);
      break;
    case TQP_MAX:
      if (x > *reinterpret_cast<volatile long long*>(slot)) atomicMax(slot, x);
      break;
    default: shared_add_u64(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)x); break;
  }
}

// Scatter of the light rows into their buckets; heavy rows folded into
// per-block shared accumulators, flushed with atomics at the end.
template <int MODE>  // kThrGlobal or kThrShared
__global__ void __launch_bounds__(kPartThreads, 1) lp_scatter_kernel(PartArgs a, AggProgram P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PackPlan K;
  const LearnedPlan lp = *a.lp;
  const PartSmem S = part_carve(smem, P.naggs, lp.B);
  const int nh = lp.nheavy;
  for (int i = threadIdx.x; i < nh * P.naggs; i += blockDim.x) S.acc[i] = agg_identity(P.op[i % P.naggs]);
  part_setup<MODE>(a, lp, S, K);
  const unsigned* thr = MODE >= kThrShared ? S.thr : a.thr;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  constexpr int TILE = kPartThreads * kPartItems;
  const int64_t c1 = n;
  for (int64_t base = (int64_t)blockIdx.x * TILE; base < n; base += (int64_t)gridDim.x * TILE) {
    unsigned long long p[kPartItems];
    int64_t row[kPartItems];
    bool v[kPartItems];
    int h[kPartItems];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
      const int64_t i = base + k * kPartThreads + threadIdx.x;
      v[k] = i < c1;
      row[k] = v[k] ? (a.sel ? (int64_t)a.sel[i] : i) : 0;
    }
    pack_rows(K, row, v, p);
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) h[k] = v[k] ? (nh ? heavy_lookup(S, p[k]) : -1) : -2;  // -2: past the end
    // light rows: bucket, cursor, store
    unsigned pos[kPartItems];
#pragma unroll
    for (int k = 0; k < kPartItems; ++k) {
      if (h[k] != -1) continue;
      const int b = lp_bucket<MODE >= kThrShared>(p[k], lp, S.dir, thr);
      pos[k] = atomicAdd(&a.cursor[(size_t)b * kCursorStride], 1u);
    }
#pragma unroll
    for (int k = 0; k < kPartItems; ++k)
      if (h[k] == -1) {
        a.out_p[pos[k]] = p[k];
        a.out_row[pos[k]] = a.payload ? a.payload[base + k * kPartThreads + threadIdx.x] : (int32_t)row[k];
      }
    // heavy rows: folded into the block's accumulators
    if (nh) {
#pragma unroll
      for (int k = 0; k < kPartItems; ++k) {
        if (h[k] < 0) continue;
        long long* acc = &S.acc[h[k] * P.naggs];
        for (int q = 0; q < P.naggs; ++q) {
          const int op = P.op[q];
          fold_shared(&acc[q], op, op == TQP_COUNT ? 1 : eval_expr(P, P.expr[q], row[k]));
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nh * P.naggs; i += blockDim.x) {
    long long v = S.acc[i];
    int op = P.op[i % P.naggs];
    if (v != agg_identity(op)) fold_atomic(&a.heavy_acc[i], op, v);
  }
}

// ---- two-level scatter (no heavy keys): the rows reach their buckets in
// two splits, each a block-level multisplit of tiles of kSplitTile rows.
// Split 1 bins a tile by the coarse bucket (the bucket's top bits: at most
// 256 coarse buckets), split 2 bins a tile of one coarse bucket by the
// bucket itself.  A tile's rows are ranked per bin in shared memory, each
// non-empty bin reserves its run with one global atomic, and the tile is
// written out bin by bin from shared memory, so the rows leave in runs.
// One atomic per (tile, bin) replaces the returning per-row atomic of
// lp_scatter_kernel, whose latency bounded it.
constexpr int kSplitThreads = 512, kSplitItems = 8, kSplitTile = kSplitThreads * kSplitItems;
#ifndef TQP_SPLIT_COARSE_BITS
#define TQP_SPLIT_COARSE_BITS 8
#endif
constexpr int kSplitCoarseBits = TQP_SPLIT_COARSE_BITS;  // at most 256 coarse buckets (split 1's bins)
// bins of one split: the coarse buckets, or the buckets of one coarse bucket
// (B <= 2^17)
constexpr int kSplitMaxBins = (1 << kSplitCoarseBits) > (1 << (17 - kSplitCoarseBits)) ? (1 << kSplitCoarseBits)
                                                                                       : (1 << (17 - kSplitCoarseBits));
static_assert(kSplitCoarseBits <= 8, "split tiles are planned by one block of 256 threads");
// The bucket function's steps in shared memory when they fit (one block per
// SM), else read from global memory (several blocks per SM).
#ifndef TQP_SPLIT_THR_SHARED
#define TQP_SPLIT_THR_SHARED 1
#endif
constexpr bool kSplitThrShared = TQP_SPLIT_THR_SHARED != 0;

__host__ __device__ inline int split_fine_bits(int B) {  // log2(fine buckets per coarse bucket)
  int lb = 0;
  while ((1 << lb) < B) ++lb;
  return lb > kSplitCoarseBits ? lb - kSplitCoarseBits : 0;
}

// Split 1: directory, steps (thr_smem), staged keys, rows, bins and fine
// ids.  Split 2 needs only the staging (dir_thr = false).
inline __host__ __device__ size_t split_smem_bytes(int B, bool thr_smem, bool dir_thr = true) {
  size_t o = dir_thr ? ((((size_t)1 << kDirBits) + 1) * 4 + 15) & ~(size_t)15 : 0;
  if (dir_thr && thr_smem) o += (((size_t)(B > 1 ? B - 1 : 1) * 4) + 15) & ~(size_t)15;
  return o + (size_t)kSplitTile * (8 + 4 + 2 + 2);
}

struct SplitSmem {
  int* dir;
  unsigned* thr;
  unsigned long long* key;
  int32_t* row;
  unsigned short* bin;
  unsigned short* fine;  // split 1: each row's bucket within its coarse bucket
};

__device__ __forceinline__ SplitSmem split_carve(unsigned char* base, int B, bool thr_smem, bool dir_thr = true) {
  SplitSmem S;
  size_t o = dir_thr ? ((((size_t)1 << kDirBits) + 1) * 4 + 15) & ~(size_t)15 : 0;
  S.dir = reinterpret_cast<int*>(base);
  S.thr = reinterpret_cast<unsigned*>(base + o);
  if (dir_thr && thr_smem) o += (((size_t)(B > 1 ? B - 1 : 1) * 4) + 15) & ~(size_t)15;
  S.key = reinterpret_cast<unsigned long long*>(base + o);
  o += (size_t)kSplitTile * 8;
  S.row = reinterpret_cast<int32_t*>(base + o);
  o += (size_t)kSplitTile * 4;
  S.bin = reinterpret_cast<unsigned short*>(base + o);
  o += (size_t)kSplitTile * 2;
  S.fine = reinterpret_cast<unsigned short*>(base + o);
  return S;
}

template <bool THR_SMEM>
__device__ __forceinline__ void split_setup(const PartArgs& a, const LearnedPlan& lp, const SplitSmem& S) {
  for (int i = threadIdx.x; i <= (1 << kDirBits); i += blockDim.x) S.dir[i] = a.dir[i];
  if (THR_SMEM)
    for (int i = threadIdx.x; i < lp.B - 1; i += blockDim.x) S.thr[i] = a.thr[i];
}

struct SplitBins {
  unsigned hist[kSplitMaxBins];   // counts, ranked into by atomics
  unsigned start[kSplitMaxBins];  // the tile's bin starts
  unsigned base[kSplitMaxBins];   // the bins' global run starts
  int scan[33];
};

// The tile's rows (per thread: packed key, payload, bin or -1, rank in its
// bin) are counted in B.hist: reserve each bin's run at cur[(first + bin) *
// kCursorStride], stage the rows in bin order, write them out.
__device__ __forceinline__ void split_place(const unsigned long long (&p)[kSplitItems], const int32_t (&r)[kSplitItems],
                                            const int (&bin)[kSplitItems], const unsigned (&rk)[kSplitItems],
                                            int nbins, int first, unsigned* cur, SplitBins& B, const SplitSmem& S,
                                            unsigned long long* out_p, int32_t* out_row,
                                            const int* fine = nullptr, unsigned short* out_fine = nullptr) {
  __syncthreads();
  const unsigned cnt = threadIdx.x < nbins ? B.hist[threadIdx.x] : 0u;
  int total;
  const int st = block_exclusive_sum<kSplitThreads>((int)cnt, B.scan, &total);
  if (threadIdx.x < nbins) {
    B.start[threadIdx.x] = (unsigned)st;
    if (cnt) B.base[threadIdx.x] = atomicAdd(&cur[(size_t)(first + threadIdx.x) * kCursorStride], cnt);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSplitItems; ++k)
    if (bin[k] >= 0) {
      const unsigned slot = B.start[bin[k]] + rk[k];
      S.key[slot] = p[k];
      S.row[slot] = r[k];
      S.bin[slot] = (unsigned short)bin[k];
      if (out_fine) S.fine[slot] = (unsigned short)fine[k];
    }
  __syncthreads();
  for (int j = threadIdx.x; j < total; j += kSplitThreads) {
    const int b = S.bin[j];
    const unsigned dst = B.base[b] + ((unsigned)j - B.start[b]);
    out_p[dst] = S.key[j];
    out_row[dst] = S.row[j];
    if (out_fine) out_fine[dst] = S.fine[j];
  }
  __syncthreads();
}

// Split 1: the (selected) rows by coarse bucket (bucket >> F) into
// (out_p, out_row), coarse cursors in cur.
// IDS: the bucket comes from the counting pass (a.ids), so no bucket
// function is evaluated and shared memory holds only the staging.
template <bool THR_SMEM, bool IDS>
__global__ void __launch_bounds__(kSplitThreads, IDS ? 2 : 1) lp_split1_kernel(PartArgs a, int F, unsigned* cur,
                                                                     unsigned long long* out_p, int32_t* out_row,
                                                                     unsigned short* out_fine) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ PackPlan K;
  __shared__ SplitBins SB;
  const LearnedPlan lp = *a.lp;
  const SplitSmem S = split_carve(smem, lp.B, THR_SMEM, !IDS);
  if (!IDS) split_setup<THR_SMEM>(a, lp, S);
  if (threadIdx.x == 0) {
    K.nkeys = a.ks.nkeys;
    for (int k = 0; k < TQP_MAX_KEYS; ++k) {
      K.col[k] = a.ks.col[k];
      K.dt[k] = a.ks.dt[k];
      K.kmin[k] = a.gp->kmin[k];
      K.shift[k] = a.gp->shift[k];
    }
  }
  __syncthreads();
  const unsigned* thr = THR_SMEM ? S.thr : a.thr;
  const int nbins = lp.B >> F;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  for (int64_t base = (int64_t)blockIdx.x * kSplitTile; base < n; base += (int64_t)gridDim.x * kSplitTile) {
    for (int i = threadIdx.x; i < nbins; i += kSplitThreads) SB.hist[i] = 0;
    __syncthreads();
    unsigned long long p[kSplitItems];
    int32_t r[kSplitItems];
    int bin[kSplitItems], fine[kSplitItems];
    unsigned rk[kSplitItems];
    int64_t rw[kSplitItems];
    bool v[kSplitItems];
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
      const int64_t i = base + k * kSplitThreads + threadIdx.x;
      bin[k] = -1;
      fine[k] = 0;
      rk[k] = 0;
      v[k] = i < n;
      rw[k] = v[k] ? (a.sel ? (int64_t)a.sel[i] : i) : 0;
      r[k] = v[k] ? (a.payload ? a.payload[i] : (int32_t)rw[k]) : 0;
    }
    pack_rows(K, rw, v, p);
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k)
      if (base + k * kSplitThreads + threadIdx.x < n) {
        const int b = IDS ? (int)a.ids[base + k * kSplitThreads + threadIdx.x] : lp_bucket<THR_SMEM>(p[k], lp, S.dir, thr);
        bin[k] = b >> F;
        fine[k] = b & ((1 << F) - 1);
        rk[k] = atomicAdd(&SB.hist[bin[k]], 1u);
      }
    split_place(p, r, bin, rk, nbins, 0, cur, SB, S, out_p, out_row, fine, out_fine);
  }
}

// Tile starts of split 2 (one block of 256 threads): coarse bucket c has
// ceil(rows / kSplitTile) tiles, starting at tstart[c]; tstart[C] = all.
// Also the coarse cursors of split 1, at the coarse buckets' first rows.
__global__ void __launch_bounds__(256) lp_split_tiles_kernel(const unsigned* off, const LearnedPlan* lp, int F,
                                                             unsigned* tstart, unsigned* cur1) {
  __shared__ int s_scan[33];
  const int C = lp->B >> F;
  const int c = threadIdx.x;
  unsigned nt = 0;
  if (c < C) {
    nt = (off[(c + 1) << F] - off[c << F] + kSplitTile - 1) / kSplitTile;
    cur1[(size_t)c * kCursorStride] = off[c << F];
  }
  int total;
  const int ex = block_exclusive_sum<256>((int)nt, s_scan, &total);
  if (c < C) tstart[c] = (unsigned)ex;
  if (c == 0) tstart[C] = (unsigned)total;
}

// Split 2: each tile holds rows of one coarse bucket c; they go to their
// buckets (c << F) + fine id (the id split 1 computed), through the
// buckets' cursors.  No bucket function here: shared memory holds only the
// staging, so several blocks share an SM.
__global__ void __launch_bounds__(kSplitThreads, 2) lp_split2_kernel(const LearnedPlan* lpp, int F, const unsigned* off,
                                                                     const unsigned* tstart,
                                                                     const unsigned long long* in_p,
                                                                     const int32_t* in_row,
                                                                     const unsigned short* in_fine, unsigned* cursor,
                                                                     unsigned long long* out_p, int32_t* out_row) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SplitBins SB;
  __shared__ unsigned s_tstart[(1 << kSplitCoarseBits) + 1];
  const int Bk = lpp->B;
  const SplitSmem S = split_carve(smem, Bk, false, false);
  const int C = Bk >> F;
  for (int i = threadIdx.x; i <= C; i += kSplitThreads) s_tstart[i] = tstart[i];
  __syncthreads();
  const int nbins = 1 << F;
  const unsigned ntiles = s_tstart[C];
  for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // the coarse bucket of tile t: the last c with tstart[c] <= t
    int lo = 0, hi = C;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_tstart[mid] <= t) lo = mid; else hi = mid;
    }
    const int c = lo;
    const int64_t row0 = (int64_t)off[c << F] + (int64_t)(t - s_tstart[c]) * kSplitTile;
    const int64_t row1 = off[(c + 1) << F];
    for (int i = threadIdx.x; i < nbins; i += kSplitThreads) SB.hist[i] = 0;
    __syncthreads();
    unsigned long long p[kSplitItems];
    int32_t r[kSplitItems];
    int bin[kSplitItems];
    unsigned rk[kSplitItems];
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
      const int64_t i = row0 + k * kSplitThreads + threadIdx.x;
      bin[k] = -1;
      p[k] = 0;
      r[k] = 0;
      rk[k] = 0;
      if (i < row1) {
        p[k] = in_p[i];
        r[k] = in_row[i];
        bin[k] = in_fine[i];
      }
    }
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k)
      if (bin[k] >= 0) rk[k] = atomicAdd(&SB.hist[bin[k]], 1u);
    split_place(p, r, bin, rk, nbins, c << F, cursor, SB, S, out_p, out_row);
  }
}

// Fine counts after split 1: each tile of split 2's tiling (rows of one
// coarse bucket c) counts its rows' fine ids in shared memory and adds them
// into count[(c << F) + fine], one atomic per (tile, fine bucket).
__global__ void __launch_bounds__(kSplitThreads) lp_fine_count_kernel(const LearnedPlan* lpp, int F, const unsigned* off,
                                                                     const unsigned* tstart,
                                                                     const unsigned short* in_fine, unsigned* count) {
  __shared__ unsigned s_cnt[kSplitMaxBins];
  __shared__ unsigned s_tstart[(1 << kSplitCoarseBits) + 1];
  const int C = lpp->B >> F;
  for (int i = threadIdx.x; i <= C; i += kSplitThreads) s_tstart[i] = tstart[i];
  __syncthreads();
  const int nbins = 1 << F;
  const unsigned ntiles = s_tstart[C];
  for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int lo = 0, hi = C;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_tstart[mid] <= t) lo = mid; else hi = mid;
    }
    const int c = lo;
    const int64_t row0 = (int64_t)off[c << F] + (int64_t)(t - s_tstart[c]) * kSplitTile;
    const int64_t row1 = off[(c + 1) << F];
    for (int i = threadIdx.x; i < nbins; i += kSplitThreads) s_cnt[i] = 0;
    __syncthreads();
    unsigned short f[kSplitItems];
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k) {
      const int64_t i = row0 + k * kSplitThreads + threadIdx.x;
      f[k] = i < row1 ? in_fine[i] : (unsigned short)0xffff;
    }
#pragma unroll
    for (int k = 0; k < kSplitItems; ++k)
      if (f[k] != 0xffff) atomicAdd(&s_cnt[f[k]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += kSplitThreads)
      if (s_cnt[i]) atomicAdd(&count[(c << F) + i], s_cnt[i]);
    __syncthreads();
  }
}

// Sorted packed keys back to the key column's dtype (one key column,
// packed as key - kmin).  skip: a device flag that, when set, says the
// decoded keys are not needed.
__global__ void lp_decode_kernel(const unsigned long long* p, const GroupPlan* gp, int dt, int64_t n_max,
                                 const int64_t* d_n, void* out, const int* skip = nullptr) {
  if (skip && *skip) return;
  const int64_t n = clamp_n(n_max, d_n);
  const unsigned long long kmin = (unsigned long long)gp->kmin[0];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    store_from_i64(out, dt, i, (long long)(p[i] + kmin));
}

// ---------------------------------------------------------------- bucket sort
// Stable rank within a block whose warp w owns items [w * per, (w + 1) * per)
// in rounds of 32: returns in pos[] the block-local destination of each item
// for digit values dig[] (kRadix = invalid).  Only the first `rounds` rounds
// hold items (the same count in every warp).  s_cnt: [WARPS][kRadix + 1],
// s_start: [kRadix] (exclusive digit starts), s_scan: 33 ints.
template <int WARPS, int ITEMS>
__device__ __forceinline__ void block_rank(const unsigned (&dig)[ITEMS], int (&pos)[ITEMS], int rounds,
                                           unsigned* s_cnt, unsigned* s_start, int* s_scan, int* total_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < WARPS * (kRadix + 1); i += WARPS * 32) s_cnt[i] = 0;
  __syncthreads();
  unsigned rank[ITEMS];
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    if (it >= rounds) break;
    unsigned peers = match_digit9(dig[it]);
    int leader = 31 - __clz(peers);
    unsigned before = __popc(peers & ((1u << lane) - 1));
    unsigned* c = s_cnt + warp * (kRadix + 1) + dig[it];
    unsigned base = *c;
    __syncwarp();
    if (lane == leader) *c = base + __popc(peers);
    __syncwarp();
    rank[it] = base + before;
  }
  __syncthreads();
  int tc = 0;
  if (threadIdx.x < kRadix) {
    unsigned run = 0;
    for (int w = 0; w < WARPS; ++w) {
      unsigned c = s_cnt[w * (kRadix + 1) + threadIdx.x];
      s_cnt[w * (kRadix + 1) + threadIdx.x] = run;
      run += c;
    }
    tc = (int)run;
  }
  int total;
  int st = block_exclusive_sum<WARPS * 32>(tc, s_scan, &total);
  if (threadIdx.x < kRadix) s_start[threadIdx.x] = (unsigned)st;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ITEMS; ++it)
    pos[it] = (it < rounds && dig[it] < kRadix)
                  ? (int)(s_start[dig[it]] + s_cnt[warp * (kRadix + 1) + dig[it]] + rank[it])
                  : -1;
  *total_out = total;
  __syncthreads();
}

struct BucketSortArgs {
  const LearnedPlan* lp;
  const unsigned* off;          // [B + 1]
  unsigned long long* p;        // light rows, bucketed (sorted in place)
  int32_t* row;
  unsigned long long* alt_p;    // scratch of the same size (global fallback)
  int32_t* alt_row;
  uint32_t* queue;
  const uint32_t* big_flags;  // null, or: small buckets handled by the warp kernel unless flagged (bit 0)
  int only_flagged;           // the MSD kernel ran first: sort only the buckets it flagged (bit 1),
  uint32_t* flagged;          // listed here by the MSD kernel
  uint32_t* nflagged;         // (their count)
};

__device__ __forceinline__ bool warp_bucket_size(long long m) { return m > 1 && m <= 1024; }

__device__ __forceinline__ unsigned long long block_minmax_span(unsigned long long lo_in, unsigned long long hi_in,
                                                                unsigned long long* s_red, unsigned long long* mn) {
  unsigned long long lo = lo_in, hi = hi_in;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_red[2 * w] = lo;
    s_red[2 * w + 1] = hi;
  }
  __syncthreads();
  lo = ~0ull;
  hi = 0;
  for (int i = 0; i < kLocalWarps; ++i) {
    lo = s_red[2 * i] < lo ? s_red[2 * i] : lo;
    hi = s_red[2 * i + 1] > hi ? s_red[2 * i + 1] : hi;
  }
  __syncthreads();
  *mn = lo;
  return hi >= lo ? hi - lo : 0;
}

// Shared memory of the block bucket sort.
struct LocalSmem {
  unsigned long long* kA;
  unsigned long long* kB;
  int32_t* rA;
  int32_t* rB;
  unsigned* cnt;    // [kLocalWarps][kRadix + 1] (the on-chip sort's cursors: [kMsdBins])
  unsigned* start;  // [kRadix]
  int* scan;        // 33
  unsigned long long* red;  // [2 * kLocalWarps]
  unsigned* part;   // [kMsdBins + 1] on-chip sort's part starts
  int* nbig;        // the on-chip sort found a part beyond kSmallPart rows
};

// LSD sort, by one block, of the m <= kLocalCap keys and rows at (kX, rX) in
// shared memory over the bits of their span, (kY, rY) as scratch; the
// result in (kX, rX).
__device__ void lsd_shared(unsigned long long* kX, int32_t* rX, unsigned long long* kY, int32_t* rY, int m,
                           const LocalSmem& L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long lo = ~0ull, hi = 0;
  for (int i = threadIdx.x; i < m; i += kLocalThreads) {
    const unsigned long long k = kX[i];
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  unsigned long long pmin;
  const unsigned long long span = block_minmax_span(lo, hi, L.red, &pmin);
  if (span == 0) return;
  const int bits = 64 - __clzll((long long)span);
  const int per = (m + kLocalWarps - 1) / kLocalWarps;
  const int wbeg = warp * per;
  unsigned long long* kA = kX;
  unsigned long long* kB = kY;
  int32_t* rA = rX;
  int32_t* rB = rY;
  for (int sh = 0; sh < bits; sh += kRadixBits) {
    unsigned dig[kLocalItems];
    int pos[kLocalItems];
#pragma unroll
    for (int it = 0; it < kLocalItems; ++it) {
      int i = wbeg + it * 32 + lane;
      bool v = (it * 32 + lane < per) && i < m;
      dig[it] = v ? (unsigned)(((kA[i] - pmin) >> sh) & (kRadix - 1)) : kRadix;
    }
    int total;
    block_rank<kLocalWarps, kLocalItems>(dig, pos, (per + 31) >> 5, L.cnt, L.start, L.scan, &total);
#pragma unroll
    for (int it = 0; it < kLocalItems; ++it) {
      if (pos[it] >= 0) {
        int i = wbeg + it * 32 + lane;
        kB[pos[it]] = kA[i];
        rB[pos[it]] = rA[i];
      }
    }
    __syncthreads();
    unsigned long long* tk = kA; kA = kB; kB = tk;
    int32_t* tr = rA; rA = rB; rB = tr;
  }
  if (kA != kX) {  // odd number of passes
    for (int i = threadIdx.x; i < m; i += kLocalThreads) {
      kX[i] = kA[i];
      rX[i] = rA[i];
    }
    __syncthreads();
  }
}

// m <= kLocalCap rows from (sp, sr) sorted by key into (dp, dr) (which may
// be the same arrays), by one block: loaded into shared memory and counted
// by the top kMsdBits bits of the rows' key span.  When no part holds more
// than kSmallPart rows (keys spread over their range), one counting pass
// places the rows by those bits (block-wide counters: equal keys need no
// order) and every part is insertion-sorted by one thread; otherwise
// (repeated or clustered keys) the block's LSD sorts the whole bucket.
#ifndef TQP_MSD_BITS
#define TQP_MSD_BITS 12
#endif
constexpr int kMsdBits = TQP_MSD_BITS;
constexpr int kMsdBins = 1 << kMsdBits;
constexpr int kSmallPart = 32;

__device__ void onchip_sort(const unsigned long long* sp, const int32_t* sr, unsigned long long* dp, int32_t* dr,
                            int m, const LocalSmem& L) {
  if (m <= 0) return;
  unsigned long long* kA = L.kA;
  unsigned long long* kB = L.kB;
  int32_t* rA = L.rA;
  int32_t* rB = L.rB;
  // every row's loads are issued before any is used: the bucket comes in
  // one memory round trip, and stays in registers until it is placed
  unsigned long long kr[kLocalItems];
  int32_t rr[kLocalItems];
#pragma unroll
  for (int q = 0; q < kLocalItems; ++q) {
    const int i = q * kLocalThreads + threadIdx.x;
    kr[q] = 0;
    rr[q] = 0;
    if (i < m) {
      kr[q] = sp[i];
      rr[q] = sr[i];
    }
  }
  unsigned long long lo = ~0ull, hi = 0;
#pragma unroll
  for (int q = 0; q < kLocalItems; ++q)
    if (q * kLocalThreads + threadIdx.x < m) {
      lo = kr[q] < lo ? kr[q] : lo;
      hi = kr[q] > hi ? kr[q] : hi;
    }
  unsigned long long pmin;
  const unsigned long long span = block_minmax_span(lo, hi, L.red, &pmin);
  if (span == 0) {  // one key: already in order
    if (sp != dp) {
#pragma unroll
      for (int q = 0; q < kLocalItems; ++q) {
        const int i = q * kLocalThreads + threadIdx.x;
        if (i < m) {
          dp[i] = kr[q];
          dr[i] = rr[q];
        }
      }
    }
    __syncthreads();
    return;
  }
  const int bits = 64 - __clzll((long long)span);
  const int sh = bits > kMsdBits ? bits - kMsdBits : 0;
  unsigned* part = L.part;  // [kMsdBins + 1] part starts
  unsigned* cur = L.cnt;    // [kMsdBins] counts, then cursors
  for (int d = threadIdx.x; d < kMsdBins; d += kLocalThreads) cur[d] = 0;
  if (threadIdx.x == 0) *L.nbig = 0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kLocalItems; ++q)
    if (q * kLocalThreads + threadIdx.x < m) atomicAdd(&cur[(kr[q] - pmin) >> sh], 1u);
  __syncthreads();
  {
    constexpr int PER = kMsdBins / kLocalThreads;
    unsigned c[PER], sum = 0;
    bool big = false;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      c[q] = cur[threadIdx.x * PER + q];
      sum += c[q];
      big |= c[q] > (unsigned)kSmallPart;
    }
    if (big) *L.nbig = 1;
    int tot;
    unsigned run = (unsigned)block_exclusive_sum<kLocalThreads>((int)sum, L.scan, &tot);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      part[threadIdx.x * PER + q] = run;
      cur[threadIdx.x * PER + q] = run;
      run += c[q];
    }
    if (threadIdx.x == 0) part[kMsdBins] = (unsigned)m;
  }
  __syncthreads();
  if (*L.nbig) {
    // some part is large: the block's LSD over the whole bucket (rows in
    // their input order, which keeps it stable)
#pragma unroll
    for (int q = 0; q < kLocalItems; ++q) {
      const int i = q * kLocalThreads + threadIdx.x;
      if (i < m) {
        kA[i] = kr[q];
        rA[i] = rr[q];
      }
    }
    __syncthreads();
    lsd_shared(kA, rA, kB, rB, m, L);
    for (int i = threadIdx.x; i < m; i += kLocalThreads) {
      dp[i] = kA[i];
      dr[i] = rA[i];
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int q = 0; q < kLocalItems; ++q)
    if (q * kLocalThreads + threadIdx.x < m) {
      const unsigned pos = atomicAdd(&cur[(kr[q] - pmin) >> sh], 1u);
      kB[pos] = kr[q];
      rB[pos] = rr[q];
    }
  __syncthreads();
  for (int d = threadIdx.x; d < kMsdBins; d += kLocalThreads) {
    const int p0 = (int)part[d], p1 = (int)part[d + 1];
    for (int a = p0 + 1; a < p1; ++a) {
      const unsigned long long k = kB[a];
      const int32_t r = rB[a];
      int b = a - 1;
      while (b >= p0 && kB[b] > k) {
        kB[b + 1] = kB[b];
        rB[b + 1] = rB[b];
        --b;
      }
      kB[b + 1] = k;
      rB[b + 1] = r;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += kLocalThreads) {
    dp[i] = kB[i];
    dr[i] = rB[i];
  }
  __syncthreads();
}

// m rows at (p, row) sorted in place by one block, LSD in global memory
// tile by tile (tiles in order keep it stable), (alt_p, alt_row) scratch.
__device__ void global_lsd(unsigned long long* p, int32_t* row, unsigned long long* alt_p, int32_t* alt_row,
                           int64_t m, const LocalSmem& L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long lo = ~0ull, hi = 0;
  for (int64_t i = threadIdx.x; i < m; i += kLocalThreads) {
    unsigned long long k = p[i];
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  unsigned long long pmin;
  const unsigned long long span = block_minmax_span(lo, hi, L.red, &pmin);
  if (span == 0) return;
  const int bits = 64 - __clzll((long long)span);
  unsigned long long* src_p = p;
  int32_t* src_r = row;
  unsigned long long* dst_p = alt_p;
  int32_t* dst_r = alt_row;
  unsigned* s_base = reinterpret_cast<unsigned*>(L.kA);  // running digit offsets
  for (int sh = 0; sh < bits; sh += kRadixBits) {
    unsigned* s_hist = L.start;
    for (int d = threadIdx.x; d < kRadix; d += kLocalThreads) s_hist[d] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += kLocalThreads)
      atomicAdd(&s_hist[((src_p[i] - pmin) >> sh) & (kRadix - 1)], 1u);
    __syncthreads();
    int c = threadIdx.x < kRadix ? (int)s_hist[threadIdx.x] : 0;
    int tot;
    int ex = block_exclusive_sum<kLocalThreads>(c, L.scan, &tot);
    if (threadIdx.x < kRadix) s_base[threadIdx.x] = (unsigned)ex;
    __syncthreads();
    for (int64_t t0 = 0; t0 < m; t0 += kLocalCap) {
      const int tm = (int)(m - t0 < kLocalCap ? m - t0 : kLocalCap);
      const int per = (tm + kLocalWarps - 1) / kLocalWarps;
      const int wbeg = warp * per;
      unsigned dig[kLocalItems];
      int pos[kLocalItems];
      unsigned long long kk[kLocalItems];
#pragma unroll
      for (int it = 0; it < kLocalItems; ++it) {
        int i = wbeg + it * 32 + lane;
        bool v = (it * 32 + lane < per) && i < tm;
        kk[it] = v ? src_p[t0 + i] : 0ull;
        dig[it] = v ? (unsigned)(((kk[it] - pmin) >> sh) & (kRadix - 1)) : kRadix;
      }
      int total;
      block_rank<kLocalWarps, kLocalItems>(dig, pos, (per + 31) >> 5, L.cnt, L.start, L.scan, &total);
#pragma unroll
      for (int it = 0; it < kLocalItems; ++it) {
        if (pos[it] >= 0) {
          int i = wbeg + it * 32 + lane;
          unsigned d = dig[it];
          int64_t g = (int64_t)s_base[d] + (pos[it] - (int)L.start[d]);
          dst_p[g] = kk[it];
          dst_r[g] = src_r[t0 + i];
        }
      }
      __syncthreads();
      if (threadIdx.x < kRadix) {  // advance by this tile's digit counts
        unsigned d = threadIdx.x;
        unsigned next = (d + 1 < kRadix) ? L.start[d + 1] : (unsigned)total;
        s_base[d] += next - L.start[d];
      }
      __syncthreads();
    }
    unsigned long long* tp = src_p; src_p = dst_p; dst_p = tp;
    int32_t* tr = src_r; src_r = dst_r; dst_r = tr;
  }
  if (src_p != p) {  // odd number of passes: copy back
    for (int64_t i = threadIdx.x; i < m; i += kLocalThreads) {
      p[i] = src_p[i];
      row[i] = src_r[i];
    }
  }
  __syncthreads();
}

// Every bucket beyond one warp's share sorted by one block: on-chip up to
// kLocalCap rows.  A larger bucket is split by one pass on the top 8 bits of
// its key span into the scratch arrays (a counting scatter: equal keys need
// no order), then runs of consecutive parts of up to kLocalCap rows are
// sorted on-chip back into place; a part beyond that is one key (already in
// order) or is sorted in global memory.  After lp_bucket_msd_kernel
// (only_flagged), the block takes just the buckets that kernel listed.
__global__ void __launch_bounds__(kLocalThreads) lp_bucket_sort_kernel(BucketSortArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_scan[33];
  __shared__ unsigned long long s_red[2 * kLocalWarps];
  __shared__ unsigned s_part[kRadix + 1];
  __shared__ unsigned s_msd[kMsdBins + 1];
  __shared__ int s_nbig;
  __shared__ uint32_t s_b;
  LocalSmem L;
  L.part = s_msd;
  L.nbig = &s_nbig;
  L.kA = reinterpret_cast<unsigned long long*>(smem);
  L.kB = L.kA + kLocalCap;
  L.rA = reinterpret_cast<int32_t*>(L.kB + kLocalCap);
  L.rB = L.rA + kLocalCap;
  L.cnt = reinterpret_cast<unsigned*>(L.rB + kLocalCap);
  L.start = L.cnt + kLocalWarps * (kRadix + 1);
  L.scan = s_scan;
  L.red = s_red;
  const int B = a.lp->B;
  const uint32_t nlist = a.only_flagged ? *a.nflagged : 0u;
  while (true) {
    if (threadIdx.x == 0) s_b = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t i = s_b;
    __syncthreads();
    if (a.only_flagged ? i >= nlist : i >= (uint32_t)B) break;
    const uint32_t b = a.only_flagged ? a.flagged[i] : i;
    const int64_t o0 = a.off[b], o1 = a.off[b + 1];
    const int64_t m = o1 - o0;
    if (m <= 1) continue;
    if (a.only_flagged) {
      if (!(a.big_flags[b] & 2u)) continue;  // sorted by the warp or the MSD kernel
    } else if (a.big_flags && m <= kLocalCap && warp_bucket_size(m) && !(a.big_flags[b] & 1u)) {
      continue;  // sorted by a warp
    }
    if (m <= kLocalCap) {
      onchip_sort(a.p + o0, a.row + o0, a.p + o0, a.row + o0, (int)m, L);
      continue;
    }
    // ---- split by the top 8 bits of the key span
    unsigned long long lo = ~0ull, hi = 0;
    for (int64_t i = threadIdx.x; i < m; i += kLocalThreads) {
      unsigned long long k = a.p[o0 + i];
      lo = k < lo ? k : lo;
      hi = k > hi ? k : hi;
    }
    unsigned long long pmin;
    const unsigned long long span = block_minmax_span(lo, hi, s_red, &pmin);
    if (span == 0) continue;  // one key
    const int bits = 64 - __clzll((long long)span);
    const int sh = bits > kRadixBits ? bits - kRadixBits : 0;
    unsigned* s_hist = L.start;
    for (int d = threadIdx.x; d < kRadix; d += kLocalThreads) s_hist[d] = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += kLocalThreads) atomicAdd(&s_hist[(a.p[o0 + i] - pmin) >> sh], 1u);
    __syncthreads();
    {
      const int c = threadIdx.x < kRadix ? (int)s_hist[threadIdx.x] : 0;
      int tot;
      const int ex = block_exclusive_sum<kLocalThreads>(c, s_scan, &tot);
      if (threadIdx.x < kRadix) {
        s_part[threadIdx.x] = (unsigned)ex;
        s_hist[threadIdx.x] = (unsigned)ex;  // becomes the scatter cursor
      }
      if (threadIdx.x == 0) s_part[kRadix] = (unsigned)m;
      __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < m; i += kLocalThreads) {
      const unsigned long long k = a.p[o0 + i];
      const unsigned pos = atomicAdd(&s_hist[(k - pmin) >> sh], 1u);
      a.alt_p[o0 + pos] = k;
      a.alt_row[o0 + pos] = a.row[o0 + i];
    }
    __syncthreads();
    // ---- consecutive parts packed into on-chip runs, back into place
    int d = 0;
    while (d < kRadix) {
      const unsigned p0 = s_part[d];
      if (s_part[d + 1] - p0 > (unsigned)kLocalCap) {
        const int64_t pm = s_part[d + 1] - p0;
        for (int64_t i = threadIdx.x; i < pm; i += kLocalThreads) {
          a.p[o0 + p0 + i] = a.alt_p[o0 + p0 + i];
          a.row[o0 + p0 + i] = a.alt_row[o0 + p0 + i];
        }
        __syncthreads();
        global_lsd(a.p + o0 + p0, a.row + o0 + p0, a.alt_p + o0 + p0, a.alt_row + o0 + p0, pm, L);
        ++d;
        continue;
      }
      int e = d + 1;
      while (e < kRadix && s_part[e + 1] - p0 <= (unsigned)kLocalCap) ++e;
      onchip_sort(a.alt_p + o0 + p0, a.alt_row + o0 + p0, a.p + o0 + p0, a.row + o0 + p0, (int)(s_part[e] - p0), L);
      d = e;
    }
  }
}


// Buckets of up to kLocalCap rows whose keys spread over their range, two
// blocks per SM: the rows stay in registers from their load to their place,
// shared memory holds only the placed rows and the kMsdBins part cursors.
// The rows are counted by the top kMsdBits bits of the bucket's key span,
// placed by part, and each part (at most kSmallPart rows) is insertion-
// sorted by one thread; a bucket with a larger part, or beyond kLocalCap
// rows, is flagged (bit 1) and listed for lp_bucket_sort_kernel.  Buckets of the warp
// kernel's size are skipped unless it flagged them (bit 0).
constexpr size_t kMsdSortSmem = (size_t)kLocalCap * (8 + 4) + (size_t)kMsdBins * 4;

__global__ void __launch_bounds__(kLocalThreads, 2) lp_bucket_msd_kernel(BucketSortArgs a, uint32_t* queue,
                                                                        uint32_t* flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_scan[33];
  __shared__ unsigned long long s_red[2 * kLocalWarps];
  __shared__ int s_nbig;
  __shared__ uint32_t s_b;
  unsigned long long* kB = reinterpret_cast<unsigned long long*>(smem);
  int32_t* rB = reinterpret_cast<int32_t*>(kB + kLocalCap);
  unsigned* cur = reinterpret_cast<unsigned*>(rB + kLocalCap);  // [kMsdBins] counts, then part cursors
  const int B = a.lp->B;
  while (true) {
    if (threadIdx.x == 0) s_b = atomicAdd(queue, 1u);
    __syncthreads();
    const uint32_t b = s_b;
    __syncthreads();
    if (b >= (uint32_t)B) break;
    const int64_t o0 = a.off[b];
    const int m = (int)((int64_t)a.off[b + 1] - o0);
    if (m <= 1) continue;
    const uint32_t fl = flags[b];
    if (warp_bucket_size(m) && !(fl & 1u)) continue;  // sorted by a warp
    if (m > kLocalCap) {
      if (threadIdx.x == 0) {
        flags[b] = fl | 2u;
        a.flagged[atomicAdd(a.nflagged, 1u)] = b;
      }
      continue;
    }
    unsigned long long kr[kLocalItems];
    int32_t rr[kLocalItems];
#pragma unroll
    for (int q = 0; q < kLocalItems; ++q) {
      const int i = q * kLocalThreads + threadIdx.x;
      kr[q] = 0;
      rr[q] = 0;
      if (i < m) {
        kr[q] = a.p[o0 + i];
        rr[q] = a.row[o0 + i];
      }
    }
    unsigned long long lo = ~0ull, hi = 0;
#pragma unroll
    for (int q = 0; q < kLocalItems; ++q)
      if (q * kLocalThreads + threadIdx.x < m) {
        lo = kr[q] < lo ? kr[q] : lo;
        hi = kr[q] > hi ? kr[q] : hi;
      }
    unsigned long long pmin;
    const unsigned long long span = block_minmax_span(lo, hi, s_red, &pmin);
    if (span == 0) continue;  // one key: already in order
    const int bits = 64 - __clzll((long long)span);
    const int sh = bits > kMsdBits ? bits - kMsdBits : 0;
    for (int d = threadIdx.x; d < kMsdBins; d += kLocalThreads) cur[d] = 0;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kLocalItems; ++q)
      if (q * kLocalThreads + threadIdx.x < m) atomicAdd(&cur[(kr[q] - pmin) >> sh], 1u);
    __syncthreads();
    {
      constexpr int PER = kMsdBins / kLocalThreads;
      unsigned c[PER], sum = 0;
      bool big = false;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        c[q] = cur[threadIdx.x * PER + q];
        sum += c[q];
        big |= c[q] > (unsigned)kSmallPart;
      }
      if (big) s_nbig = 1;
      int tot;
      unsigned run = (unsigned)block_exclusive_sum<kLocalThreads>((int)sum, s_scan, &tot);
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        cur[threadIdx.x * PER + q] = run;
        run += c[q];
      }
    }
    __syncthreads();
    if (s_nbig) {  // a large part: the LSD of lp_bucket_sort_kernel
      if (threadIdx.x == 0) {
        flags[b] = fl | 2u;
        a.flagged[atomicAdd(a.nflagged, 1u)] = b;
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < kLocalItems; ++q)
      if (q * kLocalThreads + threadIdx.x < m) {
        const unsigned pos = atomicAdd(&cur[(kr[q] - pmin) >> sh], 1u);
        kB[pos] = kr[q];
        rB[pos] = rr[q];
      }
    __syncthreads();
    // part d now ends at cur[d] and starts where part d - 1 ends
    for (int d = threadIdx.x; d < kMsdBins; d += kLocalThreads) {
      const int p0 = d ? (int)cur[d - 1] : 0, p1 = (int)cur[d];
      for (int x = p0 + 1; x < p1; ++x) {
        const unsigned long long k = kB[x];
        const int32_t r = rB[x];
        int y = x - 1;
        while (y >= p0 && kB[y] > k) {
          kB[y + 1] = kB[y];
          rB[y + 1] = rB[y];
          --y;
        }
        kB[y + 1] = k;
        rB[y + 1] = r;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kLocalThreads) {
      a.p[o0 + i] = kB[i];
      a.row[o0 + i] = rB[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- warp bucket sort
// Small buckets (at most kWarpCap rows, key span below 2^48) are sorted by
// one warp each: item i becomes the word ((key - bucket min) << 16 | i), the
// words are LSD-sorted on their key bits in the warp's shared memory (the low
// 16 bits only carry the original index back), and the rows are permuted by
// the recovered indices.  No block barrier is involved.
constexpr int kWarpItems = kWarpCap / 32;
constexpr int kWarpSortWarps = 4;


__global__ void __launch_bounds__(kWarpSortWarps * 32) lp_bucket_sort_warp_kernel(BucketSortArgs a, uint32_t* queue,
                                                                                 uint32_t* big_flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* wA = reinterpret_cast<unsigned long long*>(smem) + (size_t)warp * 2 * kWarpCap;
  unsigned long long* wB = wA + kWarpCap;
  unsigned* cnt = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned long long*>(smem) +
                                              (size_t)kWarpSortWarps * 2 * kWarpCap) + warp * (kRadix + 1);
  const int B = a.lp->B;
  while (true) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(queue, 1u);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= (uint32_t)B) break;
    const long long o0 = a.off[b], m = (long long)a.off[b + 1] - o0;
    if (m <= 1 || m > kWarpCap) continue;
    unsigned long long lo = ~0ull, hi = 0;
    for (int i = lane; i < m; i += 32) {
      unsigned long long k = a.p[o0 + i];
      lo = k < lo ? k : lo;
      hi = k > hi ? k : hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long x = __shfl_xor_sync(0xffffffffu, lo, o), y = __shfl_xor_sync(0xffffffffu, hi, o);
      lo = x < lo ? x : lo;
      hi = y > hi ? y : hi;
    }
    const unsigned long long span = hi - lo;
    if (span == 0) continue;
    if (span >> 48) {  // too wide for the packed words: leave it to the block kernel
      if (lane == 0) big_flags[b] = 1;
      continue;
    }
    for (int i = lane; i < m; i += 32) wA[i] = ((a.p[o0 + i] - lo) << 16) | (unsigned long long)i;
    __syncwarp();
    const int bits = 64 - __clzll((long long)span);
    for (int sh = 16; sh < 16 + bits; sh += kRadixBits) {
      for (int d = lane; d <= kRadix; d += 32) cnt[d] = 0;
      __syncwarp();
      unsigned dig[kWarpItems], rank[kWarpItems];
#pragma unroll
      for (int it = 0; it < kWarpItems; ++it) {
        int i = it * 32 + lane;
        dig[it] = i < m ? (unsigned)((wA[i] >> sh) & (kRadix - 1)) : kRadix;
        unsigned peers = match_digit9(dig[it]);
        int leader = 31 - __clz(peers);
        unsigned before = __popc(peers & ((1u << lane) - 1));
        unsigned base = cnt[dig[it]];
        __syncwarp();
        if (lane == leader) cnt[dig[it]] = base + __popc(peers);
        __syncwarp();
        rank[it] = base + before;
      }
      // exclusive scan of the 256 digit counts: 8 consecutive digits per lane
      unsigned c8[8], run = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c8[q] = cnt[lane * 8 + q];
        run += c8[q];
      }
      unsigned incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      unsigned start = incl - run;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        cnt[lane * 8 + q] = start;
        start += c8[q];
      }
      __syncwarp();
#pragma unroll
      for (int it = 0; it < kWarpItems; ++it) {
        int i = it * 32 + lane;
        if (i < m) wB[cnt[dig[it]] + rank[it]] = wA[i];
      }
      __syncwarp();
      unsigned long long* t = wA; wA = wB; wB = t;
    }
    // permute: sorted key = lo + (word >> 16), row = rows[word & 0xffff];
    // the buffer not holding the sorted words is free for the rows
    int32_t* rtmp = reinterpret_cast<int32_t*>(wB);
    for (int i = lane; i < m; i += 32) rtmp[i] = a.row[o0 + (int)(wA[i] & 0xffffull)];
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
      a.p[o0 + i] = lo + (wA[i] >> 16);
      a.row[o0 + i] = rtmp[i];
    }
    __syncwarp();
    // restore this warp's buffer roles for the next bucket
    wA = reinterpret_cast<unsigned long long*>(smem) + (size_t)warp * 2 * kWarpCap;
    wB = wA + kWarpCap;
  }
}

}  // namespace tqp
