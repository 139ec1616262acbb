// Sort-based inner equi-join: the build side is sorted by key (stable, so
// equal keys keep ascending build-row order); each probe row finds the range
// [lo, hi) of equal keys by two bound searches, the per-probe match counts
// are scanned in a single pass with decoupled look-back, and every tile then
// expands its pairs at its global offset, in probe-row order.
#pragma once

#include "common.cuh"

namespace tqp {

template <typename T>
__device__ __forceinline__ int64_t lower_bound_dev(const T* a, int64_t n, T x) {
  int64_t lo = 0, len = n;
  while (len > 0) {
    int64_t half = len >> 1;
    if (a[lo + half] < x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ int64_t upper_bound_dev(const T* a, int64_t lo, int64_t n, T x) {
  int64_t len = n - lo;
  while (len > 0) {
    int64_t half = len >> 1;
    if (!(x < a[lo + half])) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

template <typename T>
struct JoinArgs {
  const T* probe;
  int64_t np_max;
  const int64_t* d_np;
  const T* sorted_keys;
  const int32_t* sorted_rows;
  int64_t nb_max;
  const int64_t* d_nb;
  int32_t* out_probe;
  int32_t* out_build;
  int64_t cap;
  int64_t* d_out_n;
  unsigned long long* status;
  uint32_t* tile_counter;
  uint32_t num_tiles;
};

template <typename T, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) join_probe_kernel(JoinArgs<T> a) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ long long s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t np = clamp_n(a.np_max, a.d_np);
  const int64_t nb = clamp_n(a.nb_max, a.d_nb);
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) break;
    const int64_t base = (int64_t)tile * TILE + (int64_t)threadIdx.x * ITEMS;
    int64_t lo[ITEMS];
    int cnt[ITEMS];
    long long mine = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      lo[k] = 0;
      cnt[k] = 0;
      if (base + k < np) {
        T x = a.probe[base + k];
        int64_t l = lower_bound_dev(a.sorted_keys, nb, x);
        int64_t h = (l < nb && a.sorted_keys[l] == x) ? upper_bound_dev(a.sorted_keys, l, nb, x) : l;
        lo[k] = l;
        cnt[k] = (int)(h - l);
        mine += h - l;
      }
    }
    // counts per thread can exceed int range only for pathological joins;
    // the block scan is in 32-bit, so clamp the tile to int and flag overflow
    int mine32 = mine > 0x3fffffff ? 0x3fffffff : (int)mine;
    if (mine > 0x3fffffff) raise_status(TQP_ERR_UNSUPPORTED);
    int total;
    const int off = block_exclusive_sum<THREADS>(mine32, s_scan, &total);
    if (warp == 0) {
      long long e = lookback_exclusive(a.status, tile, total);
      if (lane == 0) s_excl = e;
    }
    __syncthreads();
    const long long excl = s_excl;
    if (excl >= 0) {
      long long pos = excl + off;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        for (int j = 0; j < cnt[k]; ++j, ++pos) {
          if (pos < a.cap) {
            a.out_probe[pos] = (int32_t)(base + k);
            a.out_build[pos] = a.sorted_rows[lo[k] + j];
          }
        }
      }
      if (tile == a.num_tiles - 1 && threadIdx.x == 0) {
        *a.d_out_n = excl + total;
        if (excl + total > a.cap) raise_status(TQP_ERR_CAPACITY);
      }
    }
    __syncthreads();
  }
}

}  // namespace tqp
