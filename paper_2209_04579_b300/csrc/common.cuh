// Shared device helpers of the TQP CUDA library: dtype access, the
// per-device status word, bounded waits, and the decoupled look-back tile
// status used by every single-pass scan in the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/tqp.h"

namespace tqp {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- status
// First device-side error wins; tqp_status_poll reads and clears it.
__device__ int g_status;
// Bound on every inter-block wait (polling rounds) and the fault-injection
// hook of the tests (a tile id that never publishes, or -1).
__device__ long long g_spin_limit = 1ll << 20;
__device__ long long g_unpublished_tile = -1;

__device__ __forceinline__ void raise_status(int code) { atomicCAS(&g_status, 0, code); }

__device__ __forceinline__ int64_t clamp_n(int64_t n, const int64_t* d_n) {
  if (d_n == nullptr) return n;
  int64_t v = *d_n;
  return v < 0 ? 0 : (v < n ? v : n);
}

// ---------------------------------------------------------------- dtypes
__device__ __forceinline__ int64_t load_as_i64(const void* p, int dt, int64_t i) {
  switch (dt) {
    case TQP_I8: return static_cast<const int8_t*>(p)[i];
    case TQP_I16: return static_cast<const int16_t*>(p)[i];
    case TQP_I32: return static_cast<const int32_t*>(p)[i];
    default: return static_cast<const int64_t*>(p)[i];
  }
}

// N elements of a column (idx[k] where ok[k]; 0 elsewhere) widened to
// int64: one switch on the dtype, then the N loads issued together.
template <int N>
__device__ __forceinline__ void load_many_as_i64(const void* p, int dt, const int64_t (&idx)[N], const bool (&ok)[N],
                                                 long long (&out)[N]) {
  switch (dt) {
    case TQP_I8:
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = ok[k] ? static_cast<const int8_t*>(p)[idx[k]] : 0;
      break;
    case TQP_I16:
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = ok[k] ? static_cast<const int16_t*>(p)[idx[k]] : 0;
      break;
    case TQP_I32:
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = ok[k] ? static_cast<const int32_t*>(p)[idx[k]] : 0;
      break;
    default:
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = ok[k] ? static_cast<const long long*>(p)[idx[k]] : 0;
      break;
  }
}

// Group ranks over a small value domain (see the star join's dimension
// group columns): a bitmap marks the values present, and the dense rank of
// v is the number of marked values below it, from a per-word prefix count
// and one popcount.
struct DomPlan {
  int on;       // 1: the domain path gives the ranks (the sort path then runs on no rows)
  int words;    // bitmap words over [kmin, kmax]
  long long kmin;
};

__device__ __forceinline__ int32_t dom_rank(const DomPlan& p, const uint32_t* bits, const int* pre, long long v) {
  const unsigned long long x = (unsigned long long)v - (unsigned long long)p.kmin;
  const uint32_t w = (uint32_t)(x >> 5);
  return pre[w] + __popc(bits[w] & ((1u << (x & 31)) - 1u));
}

__device__ __forceinline__ void store_from_i64(void* p, int dt, int64_t i, int64_t v) {
  switch (dt) {
    case TQP_I8: static_cast<int8_t*>(p)[i] = static_cast<int8_t>(v); break;
    case TQP_I16: static_cast<int16_t*>(p)[i] = static_cast<int16_t>(v); break;
    case TQP_I32: static_cast<int32_t*>(p)[i] = static_cast<int32_t>(v); break;
    default: static_cast<int64_t*>(p)[i] = v; break;
  }
}

__host__ __device__ __forceinline__ int dtype_bytes(int dt) {
  return dt == TQP_I8 ? 1 : dt == TQP_I16 ? 2 : dt == TQP_I32 ? 4 : 8;
}

__device__ __forceinline__ bool compare(int64_t v, int op, int64_t lit) {
  switch (op) {
    case TQP_LT: return v < lit;
    case TQP_LE: return v <= lit;
    case TQP_GT: return v > lit;
    case TQP_GE: return v >= lit;
    case TQP_EQ: return v == lit;
    default: return v != lit;
  }
}

// ---------------------------------------------------------------- memory ops
// Lanes of the warp whose 9-bit value v (a radix digit, or 256 for an
// empty slot) equals this lane's: one ballot per bit, each kept as is where
// this lane's bit is set and complemented where it is clear.  Every lane of
// the warp must call it.
__device__ __forceinline__ unsigned match_digit9(unsigned v) {
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (v >> b) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// Exact 64-bit add into a word in shared memory through native 32-bit
// atomics.  The atomic on the low half returns the value it replaced, so each
// wrap of the low half is seen by exactly one adder, which carries it into
// the high half.  After a barrier the 8-byte word (little-endian halves)
// equals the sum of all addends mod 2^64, whatever the order of the adds.
// Shared-memory 64-bit adds have no single native instruction; this keeps a
// contended SUM or COUNT to one 32-bit atomic (two when the addend's high
// half is non-zero or the low half wraps).
__device__ __forceinline__ void shared_add_u64(unsigned long long* p, unsigned long long x) {
  unsigned* w = reinterpret_cast<unsigned*>(p);
  const unsigned lo = (unsigned)x;
  const unsigned old = atomicAdd(w, lo);
  const unsigned hi = (unsigned)(x >> 32) + (unsigned)(old + lo < old);
  if (hi) atomicAdd(w + 1, hi);
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------- look-back
// Tile status word for a single-pass scan of non-negative counts
// (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016): bits 62..63 hold the flag, bits 0..61 the value.
constexpr unsigned long long kFlagAgg = 1ull << 62;      // value = tile aggregate
constexpr unsigned long long kFlagPrefix = 2ull << 62;   // value = inclusive prefix
constexpr unsigned long long kFlagFailed = 3ull << 62;   // tile gave up (error path)
constexpr unsigned long long kFlagMask = 3ull << 62;
constexpr unsigned long long kValMask = ~kFlagMask;

// Publishes `aggregate` for `tile`, walks back over predecessors with one
// warp (32 status words per step), publishes the inclusive prefix and
// returns the exclusive prefix.  Called by all 32 lanes of one warp.
// On a wait that runs out, or a failed predecessor, publishes kFlagFailed,
// records TQP_ERR_TIMEOUT and returns -1: the caller must not write results.
__device__ __forceinline__ long long lookback_exclusive(unsigned long long* status, long long tile,
                                                        long long aggregate) {
  const int lane = threadIdx.x & 31;
  const bool inject = (tile == g_unpublished_tile);
  if (tile == 0) {
    if (lane == 0 && !inject) st_volatile_u64(&status[0], kFlagPrefix | (unsigned long long)aggregate);
    return 0;
  }
  if (lane == 0 && !inject) st_volatile_u64(&status[tile], kFlagAgg | (unsigned long long)aggregate);
  long long excl = 0;
  long long window_end = tile;  // examine tiles [window_end - 32, window_end)
  const long long limit = g_spin_limit;
  bool failed = false;
  while (true) {
    long long t = window_end - 1 - lane;
    unsigned long long s = kFlagPrefix;  // lanes before tile 0 read as prefix 0
    if (t >= 0) {
      long long rounds = 0;
      unsigned sleep_ns = 32;
      while (true) {
        s = ld_volatile_u64(&status[t]);
        if ((s & kFlagMask) != 0) break;
        if (++rounds > limit) { s = kFlagFailed; break; }
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns <<= 1;
      }
    }
    unsigned failed_mask = __ballot_sync(0xffffffffu, (s & kFlagMask) == kFlagFailed);
    if (failed_mask) { failed = true; break; }
    unsigned prefix_mask = __ballot_sync(0xffffffffu, (s & kFlagMask) == kFlagPrefix);
    // lanes up to and including the first prefix lane contribute
    int first = prefix_mask ? (__ffs(prefix_mask) - 1) : 31;
    long long v = (lane <= first) ? (long long)(s & kValMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (prefix_mask) break;
    window_end -= 32;
  }
  if (failed) {
    if (lane == 0) {
      raise_status(TQP_ERR_TIMEOUT);
      if (!inject) st_volatile_u64(&status[tile], kFlagFailed);
    }
    return -1;
  }
  if (lane == 0 && !inject)
    st_volatile_u64(&status[tile], kFlagPrefix | (unsigned long long)(excl + aggregate));
  return excl;
}

// Block-wide exclusive sum of one int per thread (any block size that is a
// multiple of 32, up to 1024).  scratch: >= 33 ints of shared memory.
template <int THREADS>
__device__ __forceinline__ int block_exclusive_sum(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < THREADS / 32) ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < THREADS / 32) scratch[lane] = w;  // inclusive warp totals
    if (lane == 31) scratch[32] = w;
  }
  __syncthreads();
  int warp_excl = warp ? scratch[warp - 1] : 0;
  *total = scratch[32];
  int r = warp_excl + x - v;
  __syncthreads();
  return r;
}

}  // namespace tqp
