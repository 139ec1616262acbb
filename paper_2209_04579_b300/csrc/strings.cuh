// String columns (Section 2.1): an (n x m) byte tensor whose row i holds the
// UTF-8 bytes of value i right-padded with zeros to m bytes.
//
// Prefix LIKE ('p%'): a row matches when its first k bytes equal p.  The
// prefix has no zero byte, so a value shorter than k bytes (zero padding
// among its first k) never matches, and k > m never matches.
#pragma once

#include "common.cuh"

namespace tqp {

constexpr int kLikeMaxPrefix = 64;
constexpr int kLikeMaxWidth = 256;
constexpr int kLikeRows = 512;  // rows per tile: a multiple of 16, so tile starts keep 16-byte alignment

struct LikePrefix {
  unsigned char b[kLikeMaxPrefix];
  int k;
};

// One tile of kLikeRows rows per block iteration: the tile's bytes (one
// contiguous run of rows x width) are staged in shared memory with 16-byte
// loads when the column is 16-byte aligned, then each thread compares rows
// against the prefix (kernel parameter, read as a broadcast) and writes one
// byte per row.  Shared memory: kLikeRows x width bytes (width <= kLikeMaxWidth).
__global__ void __launch_bounds__(256) like_prefix_kernel(const unsigned char* str, int64_t n, int width,
                                                          LikePrefix p, int8_t* out) {
  extern __shared__ __align__(16) unsigned char s_tile[];
  const bool vec = (reinterpret_cast<uintptr_t>(str) & 15) == 0;
  const int64_t ntiles = (n + kLikeRows - 1) / kLikeRows;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * kLikeRows;
    const int rows = (int)(n - r0 < kLikeRows ? n - r0 : kLikeRows);
    const int64_t base = r0 * width;
    const int bytes = rows * width;
    const int nvec = vec ? bytes / 16 : 0;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
      reinterpret_cast<int4*>(s_tile)[i] = __ldg(reinterpret_cast<const int4*>(str + base) + i);
    for (int i = nvec * 16 + threadIdx.x; i < bytes; i += blockDim.x) s_tile[i] = __ldg(str + base + i);
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      bool match = p.k <= width;
      for (int j = 0; match && j < p.k; ++j) match = s_tile[r * width + j] == p.b[j];
      out[r0 + r] = match ? 1 : 0;
    }
    __syncthreads();
  }
}

// ---- dictionary codes of a string column (grouping by a string).  The rows
// are sorted by their value as a multi-word key: 8-byte big-endian words,
// least significant word first, each round a stable radix sort of (word,
// row) carried in the order of the round before.  Then adjacent sorted rows
// that differ start a new code; a two-level scan numbers them, and each
// row gets its code and each code one of its rows.
constexpr int kCodeThreads = 1024, kCodeItems = 4, kCodeTile = kCodeThreads * kCodeItems;

// Word w of row r: bytes [8w, 8w + 8) big-endian, zero past the width.
__device__ __forceinline__ unsigned long long str_word(const unsigned char* str, int width, int64_t r, int w) {
  const unsigned char* p = str + r * width + 8 * w;
  const int k = width - 8 * w < 8 ? width - 8 * w : 8;
  unsigned long long x = 0;
  for (int j = 0; j < 8; ++j) x = (x << 8) | (j < k ? (unsigned long long)p[j] : 0ull);
  return x;
}

__global__ void str_word_kernel(const unsigned char* str, int width, const int32_t* perm, int64_t n, int w,
                                unsigned long long* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = str_word(str, width, perm ? perm[i] : i, w);
}

// flag[i] = 1 when sorted row i starts a new value.
__global__ void str_heads_kernel(const unsigned char* str, int width, const int32_t* perm, int64_t n,
                                 int32_t* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int f = i == 0;
    if (!f) {
      const unsigned char* a = str + (int64_t)perm[i] * width;
      const unsigned char* b = str + (int64_t)perm[i - 1] * width;
      for (int j = 0; j < width && !f; ++j) f = a[j] != b[j];
    }
    flag[i] = f;
  }
}

// One block per tile of kCodeTile positions: the tile's number of heads.
__global__ void __launch_bounds__(kCodeThreads) str_tile_sums_kernel(const int32_t* flag, int64_t n,
                                                                     int32_t* tsum) {
  __shared__ int s_scan[33];
  const int64_t base = (int64_t)blockIdx.x * kCodeTile + (int64_t)threadIdx.x * kCodeItems;
  int c = 0;
  for (int k = 0; k < kCodeItems; ++k)
    if (base + k < n) c += flag[base + k];
  int total;
  block_exclusive_sum<kCodeThreads>(c, s_scan, &total);
  if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

// One block: the tiles' counts become their exclusive offsets; the total
// is the number of codes.
__global__ void __launch_bounds__(kCodeThreads) str_tile_scan_kernel(int32_t* tsum, int64_t ntiles,
                                                                     int64_t* d_ncodes) {
  __shared__ int s_scan[33];
  int carry = 0;
  for (int64_t b0 = 0; b0 < ntiles; b0 += kCodeThreads) {
    const int64_t t = b0 + threadIdx.x;
    const int v = t < ntiles ? tsum[t] : 0;
    int total;
    const int ex = block_exclusive_sum<kCodeThreads>(v, s_scan, &total);
    if (t < ntiles) tsum[t] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *d_ncodes = carry;
}

// Codes of the sorted positions, scattered to their rows; each code's first
// sorted row as its representative.
__global__ void __launch_bounds__(kCodeThreads) str_codes_kernel(const int32_t* flag, const int32_t* perm,
                                                                 const int32_t* toff, int64_t n, int32_t* code,
                                                                 int32_t* rep) {
  __shared__ int s_scan[33];
  const int64_t base = (int64_t)blockIdx.x * kCodeTile + (int64_t)threadIdx.x * kCodeItems;
  int f[kCodeItems];
  int c = 0;
  for (int k = 0; k < kCodeItems; ++k) {
    f[k] = base + k < n ? flag[base + k] : 0;
    c += f[k];
  }
  int total;
  int run = toff[blockIdx.x] + block_exclusive_sum<kCodeThreads>(c, s_scan, &total);
  for (int k = 0; k < kCodeItems; ++k) {
    if (base + k >= n) break;
    run += f[k];
    const int32_t r = perm[base + k];
    code[r] = run - 1;
    if (f[k]) rep[run - 1] = r;
  }
}

}  // namespace tqp
