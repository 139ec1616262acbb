// Stable LSD radix sort of (key, int32 value) pairs, onesweep style
// (Adinets & Merrill, "Onesweep: A Faster Least Significant Digit Radix Sort
// for GPUs", 2022): one read of the keys builds the histograms of every
// digit, then each digit is one scatter pass in which every tile ranks its
// keys with warp match/ballot, learns its global digit offsets by decoupled
// look-back, stages the tile in shared memory and writes it out.
//
// Digits whose histogram holds all n keys in one bin are skipped on the
// device (a constant digit does not change a stable order), so the number of
// passes adapts to the data without a host round trip.
#pragma once

#include "common.cuh"

namespace tqp {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;

// Internal key codes on top of tqp_dtype: keys that are already
// order-preserving unsigned words (packed group keys).
constexpr int kKeyU32 = 5;
constexpr int kKeyU64 = 6;

// Order-preserving image of a key of dtype dt as an unsigned word.
__device__ __forceinline__ unsigned long long encode_key(const void* p, int dt, int64_t i) {
  switch (dt) {
    case TQP_I8: return (unsigned long long)(uint8_t)(static_cast<const int8_t*>(p)[i]) ^ 0x80ull;
    case TQP_I16: return (unsigned long long)(uint16_t)(static_cast<const int16_t*>(p)[i]) ^ 0x8000ull;
    case TQP_I32: return (unsigned long long)(uint32_t)(static_cast<const int32_t*>(p)[i]) ^ 0x80000000ull;
    case TQP_I64: return (unsigned long long)(static_cast<const int64_t*>(p)[i]) ^ 0x8000000000000000ull;
    case kKeyU32: return static_cast<const uint32_t*>(p)[i];
    default: return static_cast<const unsigned long long*>(p)[i];
  }
}

__device__ __forceinline__ void store_decoded(void* p, int dt, int64_t i, unsigned long long u) {
  switch (dt) {
    case TQP_I8: static_cast<int8_t*>(p)[i] = (int8_t)(uint8_t)(u ^ 0x80ull); break;
    case TQP_I16: static_cast<int16_t*>(p)[i] = (int16_t)(uint16_t)(u ^ 0x8000ull); break;
    case TQP_I32: static_cast<int32_t*>(p)[i] = (int32_t)(uint32_t)(u ^ 0x80000000ull); break;
    case TQP_I64: static_cast<int64_t*>(p)[i] = (int64_t)(u ^ 0x8000000000000000ull); break;
    case kKeyU32: static_cast<uint32_t*>(p)[i] = (uint32_t)u; break;
    default: static_cast<unsigned long long*>(p)[i] = u; break;
  }
}

__host__ __device__ __forceinline__ int key_bits(int dt) {
  return dt == TQP_I8 ? 8 : dt == TQP_I16 ? 16 : (dt == TQP_I32 || dt == kKeyU32) ? 32 : 64;
}

struct PassDesc {
  int active;
  int first;  // reads the caller's input (raw dtype) rather than an intermediate
  int last;   // writes the caller's output (decoded dtype)
  int src;    // 0 = input, 1 = alt A, 2 = alt B
  int dst;    // 0 = output, 1 = alt A, 2 = alt B
};

struct SortPlan {
  PassDesc pass[kMaxPasses];
  int num_active;
};

struct SortArgs {
  const void* keys_in;
  const int32_t* vals_in;  // may be null: payload = row index
  void* keys_out;
  int32_t* vals_out;
  void* alt_keys[2];       // K-word intermediates
  int32_t* alt_vals[2];
  int key_dt;
  int begin_bit;
  int nbits;               // end_bit - begin_bit
  int npasses;             // ceil(nbits / 8)
  int64_t n_max;
  const int64_t* d_n;
  uint32_t* hist;          // [npasses][256] counts, then exclusive offsets
  SortPlan* plan;
  uint32_t* tile_counters; // [npasses]
  uint32_t* status;        // [num_tiles][256] look-back words (zeroed per pass)
};

__device__ __forceinline__ unsigned digit_of(unsigned long long u, int begin_bit, int nbits, int pass) {
  unsigned long long field = u >> begin_bit;
  int lo = pass * kRadixBits;
  int w = nbits - lo;
  if (w > kRadixBits) w = kRadixBits;
  return (unsigned)((field >> lo) & ((1ull << w) - 1));
}

// ---------------------------------------------------------------- histograms
template <int THREADS>
__global__ void __launch_bounds__(THREADS) sort_hist_kernel(SortArgs a) {
  __shared__ uint32_t s_hist[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += THREADS) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = clamp_n(a.n_max, a.d_n);
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < n; i += stride) {
    unsigned long long u = encode_key(a.keys_in, a.key_dt, i);
    for (int p = 0; p < a.npasses; ++p) atomicAdd(&s_hist[p][digit_of(u, a.begin_bit, a.nbits, p)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.npasses * kRadix; i += THREADS) {
    uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(&a.hist[i], c);
  }
}

// One block of 256 threads: scans every digit histogram into offsets and
// decides which passes run and where each reads and writes.
__global__ void __launch_bounds__(kRadix) sort_plan_kernel(SortArgs a) {
  __shared__ int s_scan[33];
  __shared__ int s_trivial[kMaxPasses];
  const int64_t n = clamp_n(a.n_max, a.d_n);
  for (int p = 0; p < a.npasses; ++p) {
    uint32_t c = a.hist[p * kRadix + threadIdx.x];
    if (threadIdx.x == 0) s_trivial[p] = 1;
    __syncthreads();
    if ((int64_t)c != n && c != 0) s_trivial[p] = 0;
    int total;
    int excl = block_exclusive_sum<kRadix>((int)c, s_scan, &total);
    a.hist[p * kRadix + threadIdx.x] = (uint32_t)excl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int active[kMaxPasses];
    int k = 0;
    for (int p = 0; p < a.npasses; ++p) {
      active[p] = (n > 0) && !s_trivial[p];
      k += active[p];
    }
    if (k == 0 && n > 0) {  // every digit constant: one pass still copies in -> out
      active[a.npasses - 1] = 1;
      k = 1;
    }
    int j = 0;
    for (int p = 0; p < kMaxPasses; ++p) {
      PassDesc d = {0, 0, 0, 0, 0};
      if (p < a.npasses && active[p]) {
        ++j;
        d.active = 1;
        d.first = (j == 1);
        d.last = (j == k);
        d.src = d.first ? 0 : (((j - 1) & 1) ? 1 : 2);
        d.dst = d.last ? 0 : ((j & 1) ? 1 : 2);
      }
      a.plan->pass[p] = d;
    }
    a.plan->num_active = k;
  }
}

// ---------------------------------------------------------------- one pass
// Per-digit decoupled look-back on 32-bit words: bits 30..31 flag, 0..29 count.
constexpr uint32_t kSFlagAgg = 1u << 30, kSFlagPrefix = 2u << 30, kSFlagFailed = 3u << 30;
constexpr uint32_t kSFlagMask = 3u << 30, kSValMask = ~kSFlagMask;

// The ranks of a warp's keys by digit (stable: ordered by item, then lane).
// match_digit9 separates the padding rows of a partial tile (digit kRadix);
// a full tile needs only the 8 digit bits.
__device__ __forceinline__ unsigned match_digit8(unsigned v) {
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (v >> b) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// Order-preserving image of a word of K's own width: keys of a signed dtype
// of that width flip their sign bit, unsigned words stay as they are.
template <typename K>
__device__ __forceinline__ K sign_flip_of(int dt) {
  if (sizeof(K) == 4) return dt == TQP_I32 ? (K)0x80000000u : (K)0;
  return dt == TQP_I64 ? (K)0x8000000000000000ull : (K)0;
}

template <typename K>
__host__ __device__ __forceinline__ bool word_dtype(int dt) {
  return sizeof(K) == 4 ? (dt == TQP_I32 || dt == kKeyU32) : (dt == TQP_I64 || dt == kKeyU64);
}

template <typename K, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 3) sort_pass_kernel(SortArgs a, int pass, uint32_t num_tiles) {
  static_assert(THREADS == kRadix, "one thread per digit");
  constexpr int TILE = THREADS * ITEMS;
  constexpr int WARPS = THREADS / 32;
  const PassDesc pd = a.plan->pass[pass];
  if (!pd.active) return;

  __shared__ uint32_t s_wcnt[WARPS][kRadix + 1];  // per-warp digit counters (+1 bin for padding rows)
  __shared__ uint32_t s_tile_start[kRadix];
  __shared__ long long s_gofs[kRadix];  // global position of the digit's first staged slot, minus that slot
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ int s_failed;
  __shared__ uint8_t s_dig[TILE];  // digit of every staged slot
  extern __shared__ __align__(16) unsigned char s_raw[];  // TILE keys, then TILE values
  K* s_keys = reinterpret_cast<K*>(s_raw);
  int32_t* s_vals = reinterpret_cast<int32_t*>(s_raw + (size_t)TILE * sizeof(K));

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  // (no runtime index into the parameter arrays: that would copy them to local memory)
  const void* kin = pd.src == 0 ? a.keys_in : (pd.src == 1 ? a.alt_keys[0] : a.alt_keys[1]);
  const int32_t* vin = pd.src == 0 ? a.vals_in : (pd.src == 1 ? a.alt_vals[0] : a.alt_vals[1]);
  const int kin_dt = pd.first ? a.key_dt : (sizeof(K) == 4 ? kKeyU32 : kKeyU64);
  void* kout = pd.dst == 0 ? a.keys_out : (pd.dst == 1 ? a.alt_keys[0] : a.alt_keys[1]);
  int32_t* vout = pd.dst == 0 ? a.vals_out : (pd.dst == 1 ? a.alt_vals[0] : a.alt_vals[1]);
  const int kout_dt = pd.last ? a.key_dt : (sizeof(K) == 4 ? kKeyU32 : kKeyU64);
  // words of K's width load and store as K (an image that is a sign flip);
  // narrower dtypes (first or last pass only) go through encode/decode
  const bool word_in = word_dtype<K>(kin_dt), word_out = word_dtype<K>(kout_dt);
  const K flip_in = sign_flip_of<K>(kin_dt), flip_out = sign_flip_of<K>(kout_dt);
  const bool row_vals = pd.first && vin == nullptr;
  const int shift = a.begin_bit + pass * kRadixBits;
  const unsigned dmask = (a.nbits - pass * kRadixBits >= kRadixBits) ? (kRadix - 1u)
                                                                      : ((1u << (a.nbits - pass * kRadixBits)) - 1u);
  const uint32_t* digit_off = a.hist + pass * kRadix;
  const long long limit = g_spin_limit;

  while (true) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(&a.tile_counters[pass], 1u);
      s_failed = 0;
    }
    for (int i = threadIdx.x; i < WARPS * (kRadix + 1); i += THREADS) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= num_tiles) break;
    const int64_t tile_base = (int64_t)tile * TILE;
    const bool full = tile_base + TILE <= n;

    // ---- load (warp-striped) and rank within the warp
    K key[ITEMS];
    int32_t val[ITEMS];
    uint32_t dr[ITEMS];  // (rank within the warp's digit << 9) | digit (kRadix = padding row)
    const int64_t r0 = tile_base + (int64_t)warp * (32 * ITEMS) + lane;
    if (full && word_in) {
      const K* kp = static_cast<const K*>(kin) + r0;
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) key[it] = kp[it * 32] ^ flip_in;
      if (row_vals) {
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) val[it] = (int32_t)(r0 + it * 32);
      } else {
        const int32_t* vp = vin + r0;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) val[it] = vp[it * 32];
      }
    } else {
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int64_t row = r0 + it * 32;
        key[it] = 0;
        val[it] = 0;
        if (row < n) {
          key[it] = (K)encode_key(kin, kin_dt, row);
          val[it] = row_vals ? (int32_t)row : vin[row];
        }
      }
    }
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) dr[it] = (unsigned)(key[it] >> shift) & dmask;
    if (!full) {
#pragma unroll
      for (int it = 0; it < ITEMS; ++it)
        if (r0 + it * 32 >= n) dr[it] = kRadix;
    }
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const unsigned dg = dr[it];
      const unsigned peers = full ? match_digit8(dg) : match_digit9(dg);
      const int leader = 31 - __clz(peers);
      const uint32_t before = __popc(peers & ((1u << lane) - 1));
      const uint32_t base = s_wcnt[warp][dg];
      __syncwarp();
      if (lane == leader) s_wcnt[warp][dg] = base + __popc(peers);
      __syncwarp();
      dr[it] = ((base + before) << 9) | dg;
    }
    __syncthreads();

    // ---- per digit (thread d): warp prefix and tile count, published at
    // once; the tile is staged before the look-back waits on predecessors
    const int d = threadIdx.x;
    uint32_t tile_count = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      uint32_t c = s_wcnt[w][d];
      s_wcnt[w][d] = tile_count;  // becomes the warp's exclusive prefix for digit d
      tile_count += c;
    }
    uint32_t* st = a.status + (size_t)tile * kRadix + d;
    const bool inject = ((long long)tile == g_unpublished_tile);
    if (!inject) st_volatile_u32(st, (tile == 0 ? kSFlagPrefix : kSFlagAgg) | tile_count);
    int total;
    const int start = block_exclusive_sum<THREADS>((int)tile_count, s_scan, &total);  // (ends on a barrier)
    s_tile_start[d] = (uint32_t)start;
    __syncthreads();

    // ---- stage keys and values in tile order (with each slot's digit)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const unsigned dg = dr[it] & 511u;
      if (dg < kRadix) {
        const unsigned slot = s_tile_start[dg] + s_wcnt[warp][dg] + (dr[it] >> 9);
        s_keys[slot] = key[it];
        s_vals[slot] = val[it];
        s_dig[slot] = (uint8_t)dg;
      }
    }

    // ---- look-back (thread d): the count of digit d in all earlier tiles
    long long excl = 0;
    bool failed = false;
    if (tile > 0) {
      // walk back kLookWin predecessors at a time: their words are loaded
      // together, then consumed in order (waiting only on a word not yet set)
      constexpr int kLookWin = 8;
      bool done = false;
      for (long long t = (long long)tile - 1; t >= 0 && !done && !failed; t -= kLookWin) {
        const int cnt = t >= kLookWin - 1 ? kLookWin : (int)t + 1;
        uint32_t wv[kLookWin];
#pragma unroll
        for (int q = 0; q < kLookWin; ++q)
          wv[q] = q < cnt ? ld_volatile_u32(a.status + (size_t)(t - q) * kRadix + d) : 0u;
#pragma unroll
        for (int q = 0; q < kLookWin; ++q) {
          if (q >= cnt || done || failed) break;
          uint32_t sv = wv[q];
          long long rounds = 0;
          unsigned sleep_ns = 32;
          while (!(sv & kSFlagMask)) {
            if (++rounds > limit) { sv = kSFlagFailed; break; }
            __nanosleep(sleep_ns);
            if (sleep_ns < 1024) sleep_ns <<= 1;
            sv = ld_volatile_u32(a.status + (size_t)(t - q) * kRadix + d);
          }
          const uint32_t f = sv & kSFlagMask;
          if (f == kSFlagFailed) { failed = true; break; }
          excl += (sv & kSValMask);
          if (f == kSFlagPrefix) done = true;
        }
      }
      if (!inject) st_volatile_u32(st, failed ? kSFlagFailed : (kSFlagPrefix | (uint32_t)(excl + tile_count)));
    }
    if (failed) {
      raise_status(TQP_ERR_TIMEOUT);
      s_failed = 1;
    }
    s_gofs[d] = (long long)digit_off[d] + excl - start;
    __syncthreads();
    if (s_failed) {  // give up on this tile without writing
      __syncthreads();
      continue;
    }

    // ---- write each staged slot to its digit's run in the output
    if (word_out) {
      K* ko = static_cast<K*>(kout);
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int j = it * THREADS + threadIdx.x;
        if (j < total) {
          const long long g = s_gofs[s_dig[j]] + j;
          ko[g] = s_keys[j] ^ flip_out;
          vout[g] = s_vals[j];
        }
      }
    } else {
#pragma unroll
      for (int it = 0; it < ITEMS; ++it) {
        const int j = it * THREADS + threadIdx.x;
        if (j < total) {
          const long long g = s_gofs[s_dig[j]] + j;
          store_decoded(kout, kout_dt, g, (unsigned long long)s_keys[j]);
          vout[g] = s_vals[j];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace tqp
