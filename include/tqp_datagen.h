/*
 * tqp_datagen.h -- device generator of the seeded synthetic input columns.
 *
 * Not part of the query operators: it produces the synthetic tables that
 * stand in for the TPC-H SF1 data of the paper's evaluation (Section 2.3).
 * Row i of a column is a pure function of (recipe, i), computed with the same
 * counter-based primitives as the host generator (SplitMix64 finaliser and
 * counter draws, MurmurHash3 fmix32, Lemire multiply-shift ranges, a Feistel
 * permutation with cycle walking, Zipf inverse-CDF sampling from a float64
 * table built on the host), so both produce identical bits.
 *
 * tqpgen_column writes rows [start, start + n) of the recipe's column to
 * d_out (device memory, recipe dtype, n elements).  d_zipf (device float64,
 * zipf_n entries) is required only for TQPGEN_ZIPF_NOISE_KEY.  Returns 0 on
 * success, 1 on a bad argument, 4 on a CUDA launch error.  Asynchronous on
 * `stream`; allocates nothing.
 */
#ifndef TQP_DATAGEN_H_
#define TQP_DATAGEN_H_
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum {
  TQPGEN_UNIFORM = 1,        /* mul * U[lo, hi] */
  TQPGEN_PERM_KEY = 2,       /* perm_m(i) + lo, a seeded bijection of [0, m) */
  TQPGEN_FMIX32_KEY = 3,     /* fmix32(i ^ key_seed) as int32 */
  TQPGEN_MIX64_KEY = 4,      /* mix64(i ^ key_seed) as int64 */
  TQPGEN_FK_FMIX32 = 5,      /* fmix32(U[0, m-1] ^ key_seed) */
  TQPGEN_FK_MIX64 = 6,       /* mix64(U[0, m-1] ^ key_seed) */
  TQPGEN_ZIPF_NOISE_KEY = 7, /* Zipf rank keys mixed with uniform 64-bit noise */
  TQPGEN_RAW64 = 8           /* the raw 64-bit draw */
};

typedef struct {
  int32_t kind;
  int32_t dtype; /* 1..4 = int8..int64 */
  uint64_t seed;
  uint64_t key_seed;
  int64_t lo, hi, mul, m;
  uint64_t noise_p32;
  uint64_t seed2;
} tqpgen_recipe;

int tqpgen_column(const tqpgen_recipe* r, int64_t start, int64_t n, void* d_out, const double* d_zipf,
                  int64_t zipf_n, void* stream);

#ifdef __cplusplus
}
#endif
#endif
