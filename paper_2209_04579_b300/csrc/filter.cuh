// Filter by single-pass stream compaction, and column gather.
//
// The paper expresses a filter as generic tensor calls (a comparison, then
// nonzero / masked_select / index_select over the mask, Fig. 3's listing
// keywords), which materialises the mask and re-reads it.  Here one kernel
// reads each predicate column once, evaluates the conjunction into a
// per-thread bit mask, ranks the survivors with a block scan, obtains the
// tile's output offset by decoupled look-back, stages the selected row ids
// in shared memory and writes them out contiguously, in ascending row order.
#pragma once

#include "common.cuh"

namespace tqp {

struct FilterArgs {
  const void* col[TQP_MAX_PREDS];
  int dt[TQP_MAX_PREDS];
  int op[TQP_MAX_PREDS];
  long long lit[TQP_MAX_PREDS];
  int npred;
  int64_t n_max;
  const int64_t* d_n;
  int32_t* out;
  int64_t cap;
  int64_t* d_out_n;
  unsigned long long* status;
  uint32_t* tile_counter;
  uint32_t num_tiles;
};

// Loads ITEMS consecutive values of column p starting at `base` as int64.
// Uses 16-byte vector loads when the whole run is in range and aligned.
template <int ITEMS>
__device__ __forceinline__ void load_run(const void* col, int dt, int64_t base, int64_t n,
                                         long long (&v)[ITEMS]) {
  const int eb = dtype_bytes(dt);
  const bool full = base + ITEMS <= n;
  const char* p = static_cast<const char*>(col) + base * eb;
  if (full && ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && (ITEMS * eb) % 16 == 0) {
    constexpr int kMaxVec = ITEMS * 8 / 16;
    uint4 buf[kMaxVec];
    const int nvec = ITEMS * eb / 16;
#pragma unroll
    for (int q = 0; q < kMaxVec; ++q)
      if (q < nvec) buf[q] = __ldg(reinterpret_cast<const uint4*>(p) + q);
    const char* b = reinterpret_cast<const char*>(buf);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      switch (dt) {
        case TQP_I8: v[k] = reinterpret_cast<const int8_t*>(b)[k]; break;
        case TQP_I16: v[k] = reinterpret_cast<const int16_t*>(b)[k]; break;
        case TQP_I32: v[k] = reinterpret_cast<const int32_t*>(b)[k]; break;
        default: v[k] = reinterpret_cast<const long long*>(b)[k]; break;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] = (base + k < n) ? load_as_i64(col, dt, base + k) : 0;
  }
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) filter_kernel(FilterArgs a) {
  constexpr int TILE = THREADS * ITEMS;
  __shared__ int s_scan[33];
  __shared__ uint32_t s_tile;
  __shared__ long long s_excl;
  __shared__ int32_t s_out[TILE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = clamp_n(a.n_max, a.d_n);
  while (true) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) break;
    const int64_t base = (int64_t)tile * TILE + (int64_t)threadIdx.x * ITEMS;
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
      if (base + k < n) mask |= 1u << k;
    for (int p = 0; p < a.npred; ++p) {
      long long v[ITEMS];
      load_run<ITEMS>(a.col[p], a.dt[p], base, n, v);
      const int op = a.op[p];
      const long long lit = a.lit[p];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        if (!compare(v[k], op, lit)) mask &= ~(1u << k);
    }
    int total;
    const int off = block_exclusive_sum<THREADS>(__popc(mask), s_scan, &total);
    if (warp == 0) {
      long long e = lookback_exclusive(a.status, tile, total);
      if (lane == 0) s_excl = e;
    }
    int k = off;
    for (uint32_t m = mask; m; m &= m - 1) s_out[k++] = (int32_t)(base + __ffs(m) - 1);
    __syncthreads();
    const long long excl = s_excl;
    if (excl >= 0) {
      for (int j = threadIdx.x; j < total; j += THREADS) {
        long long pos = excl + j;
        if (pos < a.cap) a.out[pos] = s_out[j];
      }
      if (tile == a.num_tiles - 1 && threadIdx.x == 0) {
        *a.d_out_n = excl + total;
        if (excl + total > a.cap) raise_status(TQP_ERR_CAPACITY);
      }
    }
    __syncthreads();
  }
}

// out[j] = col[idx[j]]; eight rows per thread with their reads in flight together
template <typename T>
__global__ void gather_kernel(const T* __restrict__ col, const int32_t* __restrict__ idx, int64_t n_max,
                              const int64_t* d_n, T* __restrict__ out) {
  constexpr int ITEMS = 8;
  const int64_t n = clamp_n(n_max, d_n);
  const int64_t tile = (int64_t)blockDim.x * ITEMS;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
    int32_t ix[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
      ix[k] = j < n ? __ldg(idx + j) : -1;
    }
    T v[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] = ix[k] >= 0 ? __ldg(col + ix[k]) : (T)0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t j = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (j < n) out[j] = v[k];
    }
  }
}

}  // namespace tqp
