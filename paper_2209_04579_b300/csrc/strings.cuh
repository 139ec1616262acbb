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

}  // namespace tqp
