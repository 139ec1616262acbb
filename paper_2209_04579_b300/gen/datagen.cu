// Device generator of the seeded synthetic input columns (see
// include/tqp_datagen.h).  Each primitive follows its published definition
// and matches paper_2209_04579_b300/datagen.py bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tqp_datagen.h"

namespace {

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long draw(unsigned long long seed, unsigned long long i) {
  return mix64(seed + (i + 1) * kGamma);
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ long long uniform_from(unsigned long long u, long long lo, long long hi) {
  unsigned long long rng = (unsigned long long)(hi - lo) + 1ull;
  return (long long)(((u >> 32) * rng) >> 32) + lo;
}

__device__ __forceinline__ unsigned long long feistel(unsigned long long x, unsigned long long seed, int half,
                                                      unsigned long long mask) {
  unsigned long long left = x >> half, right = x & mask;
  for (int r = 0; r < 4; ++r) {
    unsigned long long f = mix64(seed + (unsigned long long)r * kGamma + right) & mask;
    unsigned long long nl = right;
    right = left ^ f;
    left = nl;
  }
  return (left << half) | right;
}

__device__ __forceinline__ unsigned long long perm(unsigned long long i, long long n, unsigned long long seed) {
  long long t = n - 1 > 1 ? n - 1 : 1;
  int k = 64 - __clzll(t);
  if (k < 2) k = 2;
  int half = (k + 1) / 2;
  unsigned long long mask = (1ull << half) - 1;
  unsigned long long y = feistel(i, seed, half, mask);
  // cycle walking: at most a few rounds in expectation (domain <= 4n)
  for (int guard = 0; y >= (unsigned long long)n && guard < 100000; ++guard) y = feistel(y, seed, half, mask);
  return y;
}

__device__ __forceinline__ long long zipf_rank(unsigned long long u, const double* table, long long n) {
  double x = (double)(u >> 11) * 0x1p-53;
  long long lo = 0, len = n;  // first index with table[idx] > x
  while (len > 0) {
    long long half = len >> 1;
    if (table[lo + half] <= x) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo < n - 1 ? lo : n - 1;
}

__global__ void gen_kernel(tqpgen_recipe r, long long start, long long n, void* out, const double* zipf,
                           long long zipf_n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    unsigned long long i = (unsigned long long)(start + j);
    long long v = 0;
    switch (r.kind) {
      case TQPGEN_UNIFORM: v = uniform_from(draw(r.seed, i), r.lo, r.hi) * r.mul; break;
      case TQPGEN_PERM_KEY: v = (long long)perm(i, r.m, r.key_seed) + r.lo; break;
      case TQPGEN_FMIX32_KEY: v = (int32_t)fmix32((uint32_t)i ^ (uint32_t)r.key_seed); break;
      case TQPGEN_MIX64_KEY: v = (long long)mix64(i ^ r.key_seed); break;
      case TQPGEN_FK_FMIX32: {
        uint32_t jj = (uint32_t)uniform_from(draw(r.seed, i), 0, r.m - 1);
        v = (int32_t)fmix32(jj ^ (uint32_t)r.key_seed);
        break;
      }
      case TQPGEN_FK_MIX64: {
        unsigned long long jj = (unsigned long long)uniform_from(draw(r.seed, i), 0, r.m - 1);
        v = (long long)mix64(jj ^ r.key_seed);
        break;
      }
      case TQPGEN_ZIPF_NOISE_KEY: {
        unsigned long long sel = draw(r.seed, i);
        if ((sel >> 32) < r.noise_p32) {
          v = (long long)draw(r.seed2, i);
        } else {
          long long rank = zipf_rank(draw(r.seed2 ^ 0x5A5A5A5A5A5A5A5Aull, i), zipf, zipf_n);
          v = (long long)mix64((unsigned long long)rank ^ r.key_seed);
        }
        break;
      }
      default: v = (long long)draw(r.seed, i); break;
    }
    switch (r.dtype) {
      case 1: static_cast<int8_t*>(out)[j] = (int8_t)v; break;
      case 2: static_cast<int16_t*>(out)[j] = (int16_t)v; break;
      case 3: static_cast<int32_t*>(out)[j] = (int32_t)v; break;
      default: static_cast<long long*>(out)[j] = v; break;
    }
  }
}

}  // namespace

extern "C" int tqpgen_column(const tqpgen_recipe* r, int64_t start, int64_t n, void* d_out, const double* d_zipf,
                             int64_t zipf_n, void* stream) {
  if (!r || n < 0 || start < 0 || r->dtype < 1 || r->dtype > 4 || r->kind < 1 || r->kind > 8) return 1;
  if (n == 0) return 0;
  if (!d_out) return 1;
  if (r->kind == TQPGEN_ZIPF_NOISE_KEY && (!d_zipf || zipf_n < 1)) return 1;
  if ((r->kind == TQPGEN_FK_FMIX32 || r->kind == TQPGEN_FK_MIX64 || r->kind == TQPGEN_PERM_KEY) && r->m < 1) return 1;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 255) / 256;
  if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
  gen_kernel<<<(int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(*r, start, n, d_out, d_zipf, zipf_n);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
