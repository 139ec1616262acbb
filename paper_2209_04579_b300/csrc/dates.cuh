// Date columns (Section 2.1): a date is held as its UNIX epoch time in
// nanoseconds, an int64 (n x 1) tensor, and converting a source format into
// that tensor is one of the two conversions the paper names (strings being
// the other).  Three conversions run here:
//   - ISO date strings "YYYY-MM-DD" (an (n x width) zero-padded byte tensor,
//     the string layout of Section 2.1) to epoch nanoseconds;
//   - day numbers (days since 1970-01-01, the common int32 date encoding of
//     columnar formats) to epoch nanoseconds;
//   - epoch nanoseconds back to the calendar (day number, year, month, day
//     of month), e.g. for grouping by year.
// Calendar arithmetic follows the era method of H. Hinnant's public
// "chrono-compatible low-level date algorithms": with years counted from
// March (so the leap day ends a year) the calendar repeats every 400 years
// of 146097 days, and a month's first day of year is a linear function of
// its index.  The int64 nanosecond range holds whole days -106751..106751
// (1677-09-22 to 2262-04-11); dates outside it are reported, not wrapped.
#pragma once

#include "common.cuh"

namespace tqp {

constexpr long long kNsPerDay = 86400LL * 1000000000LL;
constexpr long long kDateMinDay = -106751, kDateMaxDay = 106751;
constexpr long long kDaysToEpoch = 719468;  // days from 0000-03-01 to 1970-01-01
constexpr int kDateRows = 512;              // rows per staged tile (a multiple of 16)

// Days since 1970-01-01 of y-m-d (1 <= m <= 12, 1 <= d <= 31; the caller
// checks the day against the month).
__device__ __forceinline__ long long civil_to_days(long long y, int m, int d) {
  y -= (m <= 2) ? 1 : 0;                                    // January and February close the previous year
  const long long era = (y >= 0 ? y : y - 399) / 400;       // floor division by 400
  const int yoe = (int)(y - era * 400);                     // year of era, 0..399
  const int mar = m > 2 ? m - 3 : m + 9;                    // month counted from March, 0..11
  const int doy = (153 * mar + 2) / 5 + d - 1;              // day of the March-based year, 0..365
  const int doe = yoe * 365 + yoe / 4 - yoe / 100 + doy;    // day of era, 0..146096
  return era * 146097 + doe - kDaysToEpoch;
}

// Inverse: the civil date of day number z.
__device__ __forceinline__ void days_to_civil(long long z, int* y, int* m, int* d) {
  z += kDaysToEpoch;
  const long long era = (z >= 0 ? z : z - 146096) / 146097;
  const int doe = (int)(z - era * 146097);                                  // 0..146096
  const int yoe = (doe - doe / 1460 + doe / 36524 - doe / 146096) / 365;    // 0..399
  const int doy = doe - (365 * yoe + yoe / 4 - yoe / 100);                  // 0..365
  const int mar = (5 * doy + 2) / 153;                                      // 0..11
  *d = doy - (153 * mar + 2) / 5 + 1;
  *m = mar < 10 ? mar + 3 : mar - 9;
  *y = (int)(yoe + era * 400 + (*m <= 2 ? 1 : 0));
}

__device__ __forceinline__ int month_days(int y, int m) {
  const bool leap = (y % 4 == 0 && y % 100 != 0) || y % 400 == 0;
  return m == 2 ? (leap ? 29 : 28) : (m == 4 || m == 6 || m == 9 || m == 11) ? 30 : 31;
}

// Parses one staged row; INT64_MIN when malformed or out of range.
__device__ __forceinline__ long long parse_iso_row(const unsigned char* r, int width) {
  if (width < 10 || r[4] != '-' || r[7] != '-') return LLONG_MIN;
  int v[8];
  const int at[8] = {0, 1, 2, 3, 5, 6, 8, 9};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = (int)r[at[k]] - '0';
    if (c < 0 || c > 9) return LLONG_MIN;
    v[k] = c;
  }
  for (int k = 10; k < width; ++k)
    if (r[k] != 0) return LLONG_MIN;
  const int y = v[0] * 1000 + v[1] * 100 + v[2] * 10 + v[3];
  const int m = v[4] * 10 + v[5], d = v[6] * 10 + v[7];
  if (m < 1 || m > 12 || d < 1 || d > month_days(y, m)) return LLONG_MIN;
  const long long z = civil_to_days(y, m, d);
  if (z < kDateMinDay || z > kDateMaxDay) return LLONG_MIN;
  return z * kNsPerDay;
}

// ISO strings to epoch nanoseconds.  Tiles of kDateRows rows are staged in
// shared memory (16-byte loads when the column is 16-byte aligned), then
// each thread parses whole rows.  A bad row records TQP_ERR_INVALID in the
// device status word and writes INT64_MIN.
__global__ void __launch_bounds__(256) date_parse_kernel(const unsigned char* str, int64_t n, int width,
                                                         long long* out) {
  extern __shared__ __align__(16) unsigned char s_tile[];
  const bool vec = (reinterpret_cast<uintptr_t>(str) & 15) == 0;
  const int64_t ntiles = (n + kDateRows - 1) / kDateRows;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * kDateRows;
    const int rows = (int)(n - r0 < kDateRows ? n - r0 : kDateRows);
    const int64_t base = r0 * width;
    const int bytes = rows * width;
    const int nvec = vec ? bytes / 16 : 0;
    for (int i = threadIdx.x; i < nvec; i += blockDim.x)
      reinterpret_cast<int4*>(s_tile)[i] = __ldg(reinterpret_cast<const int4*>(str + base) + i);
    for (int i = nvec * 16 + threadIdx.x; i < bytes; i += blockDim.x) s_tile[i] = __ldg(str + base + i);
    __syncthreads();
    bool bad = false;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const long long v = parse_iso_row(s_tile + r * width, width);
      bad = bad || v == LLONG_MIN;
      out[r0 + r] = v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(TQP_ERR_INVALID);
    __syncthreads();
  }
}

// Day numbers to epoch nanoseconds (INT64_MIN and TQP_ERR_INVALID outside
// the representable days).
__global__ void date_from_days_kernel(const int32_t* days, int64_t n, long long* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long z = days[i];
    const bool ok = z >= kDateMinDay && z <= kDateMaxDay;
    bad = bad || !ok;
    out[i] = ok ? z * kNsPerDay : LLONG_MIN;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(TQP_ERR_INVALID);
}

// Epoch nanoseconds to the calendar; every output is optional.  The day is
// the floor of ns / one day (an instant before 1970 belongs to the earlier
// day).
__global__ void date_parts_kernel(const long long* ns, int64_t n, int32_t* days, int32_t* year, int32_t* month,
                                  int32_t* mday) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long t = ns[i];
    long long z = t / kNsPerDay;
    if (t % kNsPerDay < 0) z -= 1;
    if (days) days[i] = (int32_t)z;
    if (year || month || mday) {
      int y, m, d;
      days_to_civil(z, &y, &m, &d);
      if (year) year[i] = y;
      if (month) month[i] = m;
      if (mday) mday[i] = d;
    }
  }
}

}  // namespace tqp
