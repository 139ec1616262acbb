// C-ABI entry points of the TQP CUDA library (declared in include/tqp.h):
// argument checks on the host, workspace carving, and kernel launches on the
// caller's stream.  One translation unit holds every kernel so that the
// per-device status word is a single object.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "dates.cuh"
#include "filter.cuh"
#include "groupby.cuh"
#include "join.cuh"
#include "learned.cuh"
#include "batched.cuh"
#include "sort.cuh"
#include "strings.cuh"
#include "star.cuh"

namespace tqp {
namespace {

// ---------------------------------------------------------------- host helpers
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* ws) : base(static_cast<char*>(ws)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int num_sms() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 148;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  cache[dev] = n;
  return n;
}

// Persistent grid: enough resident blocks to fill every SM, never more than the tiles.
template <typename Kernel>
int persistent_grid(Kernel k, int threads, size_t smem, int64_t tiles) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  int per_sm = 1;
  {
    std::lock_guard<std::mutex> g(mu);
    const auto key = std::make_tuple(reinterpret_cast<const void*>(k), threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
      if (per_sm < 1) per_sm = 1;
      cache[key] = per_sm;
    }
  }
  int64_t g = (int64_t)per_sm * num_sms();
  if (tiles < g) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

int stride_grid(int64_t n, int threads, int per_sm = 8) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Makes a kernel accept `bytes` of dynamic shared memory on the current
// device.  The attribute belongs to one device and is a ceiling, so it is
// only ever raised: per (device, kernel) the largest value set so far is
// kept, under a lock shared by every host thread.  (Lowering it for a
// smaller launch would make a later, larger launch fail.)
cudaError_t smem_optin(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> ceiling;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(dev, fn);
  auto it = ceiling.find(key);
  if (it != ceiling.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) ceiling[key] = bytes;
  return e;
}

template <typename Kernel>
cudaError_t smem_optin(Kernel* k, int bytes) {
  return smem_optin(reinterpret_cast<const void*>(k), bytes);
}

// Static shared memory of a kernel (the same on every device), cached.
cudaError_t static_smem(const void* fn, int* bytes) {
  static std::mutex mu;
  static std::map<const void*, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) {
    *bytes = it->second;
    return cudaSuccess;
  }
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  cache[fn] = *bytes = (int)fa.sharedSizeBytes;
  return cudaSuccess;
}

// ---------------------------------------------------------------- launch accounting
std::atomic<long long> g_launches{0};
cudaEvent_t g_prof_start[16] = {};
cudaEvent_t g_prof_stop[16] = {};

inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Records the profiling event of kernel class `kid` (if one is set) on stream s.
// External records so that they also become event nodes under stream capture.
inline void prof_mark(int kid, bool start, cudaStream_t s) {
  cudaEvent_t e = start ? g_prof_start[kid] : g_prof_stop[kid];
  if (!e) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cudaError_t err = (cs == cudaStreamCaptureStatusActive) ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                                          : cudaEventRecord(e, s);
  if (err != cudaSuccess) cudaGetLastError();  // a profiling mark never fails the call
}

bool valid_dtype(int dt) { return dt >= TQP_I8 && dt <= TQP_I64; }

tqp_status last_launch() { return cudaGetLastError() == cudaSuccess ? TQP_OK : TQP_ERR_CUDA; }

#define TQP_CUDA(call)                               \
  do {                                               \
    if ((call) != cudaSuccess) return TQP_ERR_CUDA;  \
  } while (0)

// After a launch whose later kernels depend on it (and which can fail to
// launch, e.g. for its shared memory): stop before enqueueing them.
#define TQP_LAUNCHED()                                                  \
  do {                                                                  \
    if (cudaPeekAtLastError() != cudaSuccess) return last_launch();     \
  } while (0)

// ---------------------------------------------------------------- sort
constexpr int kSortThreads = 256;
// Rows per thread of a sort tile, per key width: a process-wide setting
// (tqp_sort_tiles, the autotuner's knob) among the compiled choices.
std::atomic<int> g_items32{16};
std::atomic<int> g_items64{12};
bool valid_items32(int v) { return v == 8 || v == 12 || v == 16; }
bool valid_items64(int v) { return v == 6 || v == 8 || v == 12; }

struct SortWs {
  uint32_t* ctrl;  // hist [P*256] + counters [P]
  SortPlan* plan;
  uint32_t* status;
  void* alt_keys[2];
  int32_t* alt_vals[2];
  size_t ctrl_words;
  uint32_t tiles;
  int items;  // rows per thread of a tile, fixed when the workspace is carved
};

SortWs carve_sort(Carver& c, int64_t n, int word_bytes, int npasses) {
  SortWs w;
  w.ctrl_words = (size_t)npasses * kRadix + npasses;
  w.ctrl = c.take<uint32_t>(w.ctrl_words);
  w.plan = c.take<SortPlan>(1);
  w.items = word_bytes == 4 ? g_items32.load() : g_items64.load();
  const int64_t tile = (int64_t)kSortThreads * w.items;
  int64_t t = (n + tile - 1) / tile;
  w.tiles = (uint32_t)t;
  w.status = c.take<uint32_t>((size_t)(t > 0 ? t : 1) * kRadix);
  for (int i = 0; i < 2; ++i) {
    w.alt_keys[i] = c.take<char>((size_t)(n > 0 ? n : 1) * word_bytes);
    w.alt_vals[i] = c.take<int32_t>((size_t)(n > 0 ? n : 1));
  }
  return w;
}

// Enqueues the full sort.  key_dt may be a tqp_dtype or kKeyU32 / kKeyU64.
tqp_status run_sort(const SortWs& w, int key_dt, const void* keys_in, const int32_t* vals_in, void* keys_out,
                    int32_t* vals_out, int64_t n, const int64_t* d_n, int begin_bit, int end_bit,
                    cudaStream_t s) {
  if (n == 0) return TQP_OK;
  const int word_bytes = key_bits(key_dt) <= 32 ? 4 : 8;
  SortArgs a;
  a.keys_in = keys_in;
  a.vals_in = vals_in;
  a.keys_out = keys_out;
  a.vals_out = vals_out;
  a.alt_keys[0] = w.alt_keys[0];
  a.alt_keys[1] = w.alt_keys[1];
  a.alt_vals[0] = w.alt_vals[0];
  a.alt_vals[1] = w.alt_vals[1];
  a.key_dt = key_dt;
  a.begin_bit = begin_bit;
  a.nbits = end_bit - begin_bit;
  a.npasses = (a.nbits + kRadixBits - 1) / kRadixBits;
  a.n_max = n;
  a.d_n = d_n;
  a.hist = w.ctrl;
  a.tile_counters = w.ctrl + (size_t)a.npasses * kRadix;
  a.plan = w.plan;
  a.status = w.status;
  TQP_CUDA(cudaMemsetAsync(w.ctrl, 0, w.ctrl_words * sizeof(uint32_t), s));
  sort_hist_kernel<256><<<stride_grid(n, 256), 256, 0, s>>>(a); note_launch();
  sort_plan_kernel<<<1, kRadix, 0, s>>>(a); note_launch();
  prof_mark(2, true, s);
  for (int p = 0; p < a.npasses; ++p) {
    TQP_CUDA(cudaMemsetAsync(w.status, 0, (size_t)w.tiles * kRadix * sizeof(uint32_t), s));
    if (word_bytes == 4) {
      auto k = w.items == 8    ? sort_pass_kernel<uint32_t, kSortThreads, 8>
               : w.items == 12 ? sort_pass_kernel<uint32_t, kSortThreads, 12>
                               : sort_pass_kernel<uint32_t, kSortThreads, 16>;
      size_t smem = (size_t)kSortThreads * w.items * (4 + 4);  // staged keys and values
      TQP_CUDA(smem_optin(k, (int)smem));
      k<<<persistent_grid(k, kSortThreads, smem, w.tiles), kSortThreads, smem, s>>>(a, p, w.tiles); note_launch();
    } else {
      auto k = w.items == 6   ? sort_pass_kernel<unsigned long long, kSortThreads, 6>
               : w.items == 8 ? sort_pass_kernel<unsigned long long, kSortThreads, 8>
                              : sort_pass_kernel<unsigned long long, kSortThreads, 12>;
      size_t smem = (size_t)kSortThreads * w.items * (8 + 4);  // staged keys and values
      TQP_CUDA(smem_optin(k, (int)smem));
      k<<<persistent_grid(k, kSortThreads, smem, w.tiles), kSortThreads, smem, s>>>(a, p, w.tiles); note_launch();
    }
  }
  prof_mark(2, false, s);
  return last_launch();
}

// ---------------------------------------------------------------- group-by (device part)
constexpr int kReduceThreads = 256;
constexpr int kReduceItems = 16;

struct GroupWs {
  void* gathered[TQP_MAX_VALS];  // value columns in sorted order (large inputs)
  GroupPlan* plan;
  void* packed;
  int32_t* rows;
  void* sorted;
  int32_t* sorted_rows;
  SortWs sort;
  uint32_t* ctrl;  // reduce counter + flags
  Partial* carry;
  uint32_t tiles;
  int* direct;       // small key domain: slots instead of the sort
  int64_t* sort_n;   // rows the sort path takes (0 when direct)
  long long* dacc;   // the slots' accumulators
};

// From this many rows on, the value columns are gathered into sorted order
// (one streaming gather kernel with many loads in flight) before the reduce,
// which then reads them sequentially instead of chasing row ids.
constexpr int64_t kPregatherRows = 1 << 22;

GroupWs carve_group(Carver& c, int64_t n, int word_bytes, const AggProgram* P = nullptr) {
  GroupWs w;
  std::memset(w.gathered, 0, sizeof(w.gathered));
  w.plan = c.take<GroupPlan>(1);
  size_t nn = (size_t)(n > 0 ? n : 1);
  if (P && n >= kPregatherRows)
    for (int v = 0; v < P->nvals; ++v) w.gathered[v] = c.take<char>(nn * dtype_bytes(P->vdt[v]));
  w.packed = c.take<char>(nn * word_bytes);
  w.rows = c.take<int32_t>(nn);
  w.sorted = c.take<char>(nn * word_bytes);
  w.sorted_rows = c.take<int32_t>(nn);
  w.sort = carve_sort(c, n, word_bytes, word_bytes == 4 ? 4 : 8);
  int64_t t = (n + kReduceThreads * kReduceItems - 1) / (kReduceThreads * kReduceItems);
  w.tiles = (uint32_t)t;
  w.ctrl = c.take<uint32_t>((size_t)(t > 0 ? t : 1));
  w.carry = c.take<Partial>((size_t)(t > 0 ? t : 1));
  w.direct = c.take<int>(1);
  w.sort_n = c.take<int64_t>(1);
  w.dacc = c.take<long long>((size_t)kDirectSlots * (TQP_MAX_AGGS + 1));
  return w;
}

// Reduce-by-key launch, specialised on the number of aggregates carried.
template <typename K, int NAGG>
void launch_reduce_n(const ReduceArgs& r, const AggProgram& P, uint32_t tiles, cudaStream_t s) {
  auto k = gb_reduce_kernel<K, kReduceThreads, kReduceItems, NAGG>;
  k<<<persistent_grid(k, kReduceThreads, 0, tiles), kReduceThreads, 0, s>>>(r, P);
  note_launch();
}

// Heads per tile, their scan (and the group count), the tiles' groups, the
// carries between tiles.
template <typename K>
void launch_reduce(const ReduceArgs& r, const AggProgram& P, uint32_t tiles, cudaStream_t s) {
  if (tiles > 0) {
    auto hk = gb_heads_kernel<K, kReduceThreads, kReduceItems>;
    hk<<<persistent_grid(hk, kReduceThreads, 0, tiles), kReduceThreads, 0, s>>>(r); note_launch();
  }
  gb_tile_scan_kernel<<<1, 1024, 0, s>>>(r); note_launch();
  if (tiles == 0) return;
  prof_mark(4, true, s);
  if (P.naggs <= 2) launch_reduce_n<K, 2>(r, P, tiles, s);
  else if (P.naggs <= 4) launch_reduce_n<K, 4>(r, P, tiles, s);
  else launch_reduce_n<K, TQP_MAX_AGGS>(r, P, tiles, s);
  prof_mark(4, false, s);
  gb_carry_kernel<K, kReduceThreads, kReduceItems><<<(tiles + 255) / 256, 256, 0, s>>>(r, P); note_launch();
}

// Gathers every value column into the order of `rows` (n or *d_n rows);
// returns the program reading the gathered columns.
AggProgram pregather_values(const AggProgram& P, void* const* dst, const int32_t* rows, int64_t n,
                            const int64_t* d_n, cudaStream_t s) {
  AggProgram Q = P;
  const int g = stride_grid(n, 256);
  for (int v = 0; v < P.nvals; ++v) {
    switch (P.vdt[v]) {
      case TQP_I8:
        gather_kernel<int8_t><<<g, 256, 0, s>>>((const int8_t*)P.val[v], rows, n, d_n, (int8_t*)dst[v]);
        break;
      case TQP_I16:
        gather_kernel<int16_t><<<g, 256, 0, s>>>((const int16_t*)P.val[v], rows, n, d_n, (int16_t*)dst[v]);
        break;
      case TQP_I32:
        gather_kernel<int32_t><<<g, 256, 0, s>>>((const int32_t*)P.val[v], rows, n, d_n, (int32_t*)dst[v]);
        break;
      default:
        gather_kernel<long long><<<g, 256, 0, s>>>((const long long*)P.val[v], rows, n, d_n, (long long*)dst[v]);
        break;
    }
    note_launch();
    Q.val[v] = dst[v];
  }
  return Q;
}

tqp_status build_agg_program(const tqp_col* vals, int nvals, const tqp_expr* exprs, int nexprs,
                             const tqp_agg* aggs, int naggs, AggProgram* P, bool have_rows) {
  if (nvals < 0 || nvals > TQP_MAX_VALS || nexprs < 0 || nexprs > TQP_MAX_EXPRS || naggs < 1 ||
      naggs > TQP_MAX_AGGS)
    return TQP_ERR_INVALID;
  if ((nvals && !vals) || (nexprs && !exprs) || !aggs) return TQP_ERR_INVALID;
  std::memset(P, 0, sizeof(*P));
  P->nvals = nvals;
  for (int v = 0; v < nvals; ++v) {
    if (!valid_dtype(vals[v].dtype)) return TQP_ERR_DTYPE;
    if (have_rows && !vals[v].data) return TQP_ERR_INVALID;
    P->val[v] = vals[v].data;
    P->vdt[v] = vals[v].dtype;
  }
  P->nexprs = nexprs;
  for (int e = 0; e < nexprs; ++e) {
    if (exprs[e].nterms < 1 || exprs[e].nterms > 3) return TQP_ERR_INVALID;
    P->nterms[e] = exprs[e].nterms;
    for (int t = 0; t < exprs[e].nterms; ++t) {
      if (exprs[e].term[t].col < 0 || exprs[e].term[t].col >= nvals) return TQP_ERR_INVALID;
      P->tcol[e][t] = exprs[e].term[t].col;
      P->tmul[e][t] = exprs[e].term[t].mul;
      P->tadd[e][t] = exprs[e].term[t].add;
    }
  }
  P->naggs = naggs;
  for (int a = 0; a < naggs; ++a) {
    if (aggs[a].op < TQP_COUNT || aggs[a].op > TQP_MAX) return TQP_ERR_INVALID;
    if (aggs[a].op != TQP_COUNT && (aggs[a].expr < 0 || aggs[a].expr >= nexprs)) return TQP_ERR_INVALID;
    P->op[a] = aggs[a].op;
    P->expr[a] = aggs[a].op == TQP_COUNT ? -1 : aggs[a].expr;
  }
  // every aggregate a plain column (one term, x * 1 + 0) or COUNT
  P->simple = 1;
  for (int a = 0; a < naggs; ++a) {
    if (aggs[a].op == TQP_COUNT) continue;
    const tqp_expr& e = exprs[aggs[a].expr];
    if (e.nterms != 1 || e.term[0].mul != 1 || e.term[0].add != 0) P->simple = 0;
  }
  return TQP_OK;
}

tqp_status run_groupby(const GroupWs& w, const KeySet& ks, const AggProgram& P, const int32_t* sel, int64_t n,
                       const int64_t* d_n, int word_bytes, long long* out_aggs, int64_t cap,
                       int64_t* d_out_groups, cudaStream_t s) {
  if (n == 0) {
    TQP_CUDA(cudaMemsetAsync(d_out_groups, 0, sizeof(int64_t), s));
    return TQP_OK;
  }
  gb_init_kernel<<<1, 32, 0, s>>>(w.plan); note_launch();
  gb_keyrange_kernel<256><<<stride_grid(n, 256, 4), 256, 0, s>>>(ks, sel, n, d_n, w.plan); note_launch();
  gb_plan_kernel<<<1, 32, 0, s>>>(w.plan, ks.nkeys, word_bytes * 8); note_launch();
  // a packed key of at most kDirectBits bits folds straight into slots (after
  // the sort path, which then takes no rows and counts no groups)
  gb_direct_plan_kernel<<<1, 32, 0, s>>>(w.plan, n, d_n, w.direct, w.sort_n); note_launch();
  const int64_t* sn = w.sort_n;
  if (word_bytes == 4) {
    gb_encode_kernel<uint32_t><<<stride_grid(n, 256), 256, 0, s>>>(ks, sel, n, sn, w.plan,
                                                                     static_cast<uint32_t*>(w.packed), w.rows); note_launch();
  } else {
    gb_encode_kernel<unsigned long long><<<stride_grid(n, 256), 256, 0, s>>>(
        ks, sel, n, sn, w.plan, static_cast<unsigned long long*>(w.packed), w.rows); note_launch();
  }
  tqp_status st = run_sort(w.sort, word_bytes == 4 ? kKeyU32 : kKeyU64, w.packed, w.rows, w.sorted,
                           w.sorted_rows, n, sn, 0, word_bytes * 8, s);
  if (st != TQP_OK) return st;
  ReduceArgs r;
  r.keys = w.sorted;
  r.rows = w.sorted_rows;
  r.n_max = n;
  r.d_n = sn;
  r.plan = w.plan;
  r.ks = ks;
  r.out_aggs = out_aggs;
  r.cap = cap;
  r.d_out_groups = d_out_groups;
  r.tile_heads = w.ctrl;
  r.carry = w.carry;
  r.num_tiles = w.tiles;
  r.heavy = nullptr;
  r.d_nheavy = nullptr;
  r.heavy_acc = nullptr;
  AggProgram Pr = P;
  const bool self_gather = P.simple && P.nvals == 1;  // the reduce reads the values through the row ids
  if ((w.gathered[0] && !self_gather) || P.nvals == 0) {
    if (P.nvals) Pr = pregather_values(P, w.gathered, w.sorted_rows, n, sn, s);
    r.rows = nullptr;
  }
  if (word_bytes == 4) {
    launch_reduce<uint32_t>(r, Pr, w.tiles, s);
  } else {
    launch_reduce<unsigned long long>(r, Pr, w.tiles, s);
  }
  TQP_CUDA(smem_optin(gb_direct_kernel<256>, kDirectMaxSmemBytes));
  // shared memory for one copy of every slot of this program: a narrow
  // program leaves room for several blocks per SM (the fold waits on reads)
  const int dsm = kDirectSlots * (P.naggs + 1) * 8;
  gb_direct_init_kernel<<<8, 256, 0, s>>>(w.direct, P, w.dacc); note_launch();
  prof_mark(4, true, s);
  gb_direct_kernel<256><<<stride_grid(n, 256, 8), 256, dsm, s>>>(ks, sel, n, d_n, w.plan, P, w.direct, w.dacc, dsm);
  note_launch();
  prof_mark(4, false, s);
  gb_direct_out_kernel<1024><<<1, 1024, 0, s>>>(ks, w.plan, P, w.direct, w.dacc, out_aggs, cap, d_out_groups);
  note_launch();
  return last_launch();
}


// ---------------------------------------------------------------- star aggregate

constexpr int kFilterT = 256, kFilterI = 16;
constexpr int kRankT = 256, kRankI = 8;
constexpr int kProbeT = 256, kProbeI = 8;
constexpr int kSmemBitmapBytes = 184 * 1024;       // shared bitmap of the first dimension (at most)
constexpr int kMaxSmemOptin = 227 * 1024;          // dynamic shared memory one block may opt in to
constexpr int kHeavyMult = 4;                      // heavy-key sample / training set
constexpr int64_t kLearnedSortMinRows = 1 << 20;   // star dimensions sorted by the learned partitioner from here
constexpr int kLearnedSortRowsPerBucket = 8192;  // spread distinct keys: 4096 to 8192 per bucket on average
constexpr int64_t kSmemBitmapDimRows = 4'000'000;  // first dimensions up to this size try it
constexpr int kCompactT = 256, kCompactI = 8;

}  // namespace
}  // namespace tqp

using namespace tqp;

// ============================================================================
extern "C" {

const char* tqp_status_string(tqp_status s) {
  switch (s) {
    case TQP_OK: return "ok";
    case TQP_ERR_INVALID: return "invalid argument";
    case TQP_ERR_DTYPE: return "unsupported or mismatched dtype";
    case TQP_ERR_CAPACITY: return "result exceeds capacity";
    case TQP_ERR_CUDA: return "CUDA error";
    case TQP_ERR_TIMEOUT: return "bounded wait ran out";
    case TQP_ERR_WORKSPACE: return "workspace too small";
    case TQP_ERR_UNSUPPORTED: return "unsupported input";
    case TQP_ERR_TOO_LARGE: return "input larger than the entry point's fixed scratch allows";
  }
  return "unknown status";
}

tqp_status tqp_status_poll(tqp_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TQP_ERR_CUDA;
  if (cudaMemcpyFromSymbol(&v, g_status, sizeof(int)) != cudaSuccess) return TQP_ERR_CUDA;
  int zero = 0;
  if (cudaMemcpyToSymbol(g_status, &zero, sizeof(int)) != cudaSuccess) return TQP_ERR_CUDA;
  return static_cast<tqp_status>(v);
}

int64_t tqp_debug_launch_count(void) { return g_launches.load(); }

tqp_status tqp_profile_events(int kernel_class, void* start_event, void* stop_event) {
  if (kernel_class < 1 || kernel_class > 15) return TQP_ERR_INVALID;
  g_prof_start[kernel_class] = static_cast<cudaEvent_t>(start_event);
  g_prof_stop[kernel_class] = static_cast<cudaEvent_t>(stop_event);
  return TQP_OK;
}

tqp_status tqp_sort_tiles(int items32, int items64) {
  if ((items32 && !valid_items32(items32)) || (items64 && !valid_items64(items64))) return TQP_ERR_INVALID;
  if (items32) g_items32.store(items32);
  if (items64) g_items64.store(items64);
  return TQP_OK;
}

tqp_status tqp_debug_set_spin_limit(int64_t rounds) {
  if (rounds < 1) return TQP_ERR_INVALID;
  long long v = rounds;
  return cudaMemcpyToSymbol(g_spin_limit, &v, sizeof(v)) == cudaSuccess ? TQP_OK : TQP_ERR_CUDA;
}

tqp_status tqp_debug_inject_unpublished_tile(int64_t tile) {
  long long v = tile;
  return cudaMemcpyToSymbol(g_unpublished_tile, &v, sizeof(v)) == cudaSuccess ? TQP_OK : TQP_ERR_CUDA;
}

// ---------------------------------------------------------------------------
tqp_status tqp_filter(const tqp_col* cols, int ncols, const tqp_pred* preds, int npred, int64_t n,
                      const int64_t* d_n, int32_t* d_out_idx, int64_t cap, int64_t* d_out_n, void* ws,
                      size_t* ws_bytes, tqp_stream_t stream) {
  constexpr int T = 256, I = 16;
  if (!ws_bytes || n < 0 || n > INT_MAX || npred < 0 || npred > TQP_MAX_PREDS || ncols < 0) return TQP_ERR_INVALID;
  if (npred && (!preds || !cols)) return TQP_ERR_INVALID;
  const int64_t tiles = (n + T * I - 1) / (T * I);
  Carver c(ws);
  unsigned long long* status = c.take<unsigned long long>((size_t)(tiles > 0 ? tiles : 1));
  uint32_t* counter = c.take<uint32_t>(1);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_out_n || (cap > 0 && !d_out_idx) || cap < 0) return TQP_ERR_INVALID;
  FilterArgs a;
  std::memset(&a, 0, sizeof(a));
  a.npred = npred;
  for (int p = 0; p < npred; ++p) {
    int col = preds[p].col;
    if (col < 0 || col >= ncols || (n > 0 && !cols[col].data)) return TQP_ERR_INVALID;
    if (!valid_dtype(cols[col].dtype)) return TQP_ERR_DTYPE;
    if (preds[p].op < TQP_LT || preds[p].op > TQP_NE) return TQP_ERR_INVALID;
    a.col[p] = cols[col].data;
    a.dt[p] = cols[col].dtype;
    a.op[p] = preds[p].op;
    a.lit[p] = preds[p].lit;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    TQP_CUDA(cudaMemsetAsync(d_out_n, 0, sizeof(int64_t), s));
    return TQP_OK;
  }
  a.n_max = n;
  a.d_n = d_n;
  a.out = d_out_idx;
  a.cap = cap;
  a.d_out_n = d_out_n;
  a.status = status;
  a.tile_counter = counter;
  a.num_tiles = (uint32_t)tiles;
  TQP_CUDA(cudaMemsetAsync(ws, 0, c.off, s));
  auto k = filter_kernel<T, I>;
  prof_mark(3, true, s);
  k<<<persistent_grid(k, T, 0, tiles), T, 0, s>>>(a); note_launch();
  prof_mark(3, false, s);
  return last_launch();
}

tqp_status tqp_gather(tqp_col col, const int32_t* d_idx, int64_t n, const int64_t* d_n, void* d_out,
                      tqp_stream_t stream) {
  if (n < 0 || n > INT_MAX) return TQP_ERR_INVALID;
  if (!valid_dtype(col.dtype)) return TQP_ERR_DTYPE;
  if (n == 0) return TQP_OK;
  if (!col.data || !d_idx || !d_out) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int g = stride_grid(n, 256);
  switch (col.dtype) {
    case TQP_I8: gather_kernel<int8_t><<<g, 256, 0, s>>>((const int8_t*)col.data, d_idx, n, d_n, (int8_t*)d_out); note_launch(); break;
    case TQP_I16: gather_kernel<int16_t><<<g, 256, 0, s>>>((const int16_t*)col.data, d_idx, n, d_n, (int16_t*)d_out); note_launch(); break;
    case TQP_I32: gather_kernel<int32_t><<<g, 256, 0, s>>>((const int32_t*)col.data, d_idx, n, d_n, (int32_t*)d_out); note_launch(); break;
    default: gather_kernel<long long><<<g, 256, 0, s>>>((const long long*)col.data, d_idx, n, d_n, (long long*)d_out); note_launch(); break;
  }
  return last_launch();
}

tqp_status tqp_like_prefix(const uint8_t* d_str, int64_t n, int32_t width, const uint8_t* prefix, int32_t plen,
                           int8_t* d_out, tqp_stream_t stream) {
  if (n < 0 || width < 1 || width > kLikeMaxWidth || plen < 0 || plen > kLikeMaxPrefix || (plen && !prefix))
    return TQP_ERR_INVALID;
  LikePrefix p;
  std::memset(&p, 0, sizeof(p));
  p.k = plen;
  for (int j = 0; j < plen; ++j) {
    if (prefix[j] == 0) return TQP_ERR_INVALID;  // zero bytes are padding
    p.b[j] = prefix[j];
  }
  if (n == 0) return TQP_OK;
  if (!d_str || !d_out) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int smem = kLikeRows * width;
  TQP_CUDA(smem_optin(like_prefix_kernel, kLikeRows * kLikeMaxWidth));
  const int64_t ntiles = (n + kLikeRows - 1) / kLikeRows;
  like_prefix_kernel<<<persistent_grid(like_prefix_kernel, 256, smem, ntiles), 256, smem, s>>>(d_str, n, width, p, d_out);
  note_launch();
  return last_launch();
}

tqp_status tqp_string_codes(const uint8_t* d_str, int64_t n, int32_t width, int32_t* d_codes, int32_t* d_rep_rows,
                            int64_t* d_ncodes, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || n < 0 || n >= (1ll << 30) || width < 1 || width > kLikeMaxWidth) return TQP_ERR_INVALID;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int64_t ntiles = (n + kCodeTile - 1) / kCodeTile;
  Carver c(ws);
  unsigned long long* keys_a = c.take<unsigned long long>(nn);
  unsigned long long* keys_b = c.take<unsigned long long>(nn);
  int32_t* perm_buf[2] = {c.take<int32_t>(nn), c.take<int32_t>(nn)};
  int32_t* flag = c.take<int32_t>(nn);
  int32_t* tsum = c.take<int32_t>((size_t)(ntiles > 0 ? ntiles : 1));
  SortWs sw = carve_sort(c, n, 8, 8);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_ncodes) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    TQP_CUDA(cudaMemsetAsync(d_ncodes, 0, sizeof(int64_t), s));
    return TQP_OK;
  }
  if (!d_str || !d_codes || !d_rep_rows) return TQP_ERR_INVALID;
  // least significant word first; each round sorts the previous round's order
  prof_mark(11, true, s);
  const int W = (width + 7) / 8;
  const int32_t* perm = nullptr;  // identity before the first round
  for (int w = W - 1, which = 0; w >= 0; --w, which ^= 1) {
    str_word_kernel<<<stride_grid(n, 256), 256, 0, s>>>(d_str, width, perm, n, w, keys_a); note_launch();
    const tqp_status st = run_sort(sw, kKeyU64, keys_a, perm, keys_b, perm_buf[which], n, nullptr, 0, 64, s);
    if (st != TQP_OK) return st;
    perm = perm_buf[which];
  }
  str_heads_kernel<<<stride_grid(n, 256), 256, 0, s>>>(d_str, width, perm, n, flag); note_launch();
  str_tile_sums_kernel<<<(unsigned)ntiles, kCodeThreads, 0, s>>>(flag, n, tsum); note_launch();
  str_tile_scan_kernel<<<1, kCodeThreads, 0, s>>>(tsum, ntiles, d_ncodes); note_launch();
  str_codes_kernel<<<(unsigned)ntiles, kCodeThreads, 0, s>>>(flag, perm, tsum, n, d_codes, d_rep_rows); note_launch();
  prof_mark(11, false, s);
  return last_launch();
}

tqp_status tqp_date_parse_iso(const uint8_t* d_str, int64_t n, int32_t width, int64_t* d_ns, tqp_stream_t stream) {
  if (n < 0 || n > INT_MAX || width < 10 || width > kLikeMaxWidth) return TQP_ERR_INVALID;
  if (n == 0) return TQP_OK;
  if (!d_str || !d_ns) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TQP_CUDA(smem_optin(date_parse_kernel, kDateRows * kLikeMaxWidth));
  const int smem = kDateRows * width;
  const int64_t ntiles = (n + kDateRows - 1) / kDateRows;
  date_parse_kernel<<<persistent_grid(date_parse_kernel, 256, smem, ntiles), 256, smem, s>>>(
      d_str, n, width, reinterpret_cast<long long*>(d_ns));
  note_launch();
  return last_launch();
}

tqp_status tqp_date_from_days(const int32_t* d_days, int64_t n, int64_t* d_ns, tqp_stream_t stream) {
  if (n < 0 || n > INT_MAX) return TQP_ERR_INVALID;
  if (n == 0) return TQP_OK;
  if (!d_days || !d_ns) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  date_from_days_kernel<<<stride_grid(n, 256), 256, 0, s>>>(d_days, n, reinterpret_cast<long long*>(d_ns));
  note_launch();
  return last_launch();
}

tqp_status tqp_date_parts(const int64_t* d_ns, int64_t n, int32_t* d_days, int32_t* d_year, int32_t* d_month,
                          int32_t* d_mday, tqp_stream_t stream) {
  if (n < 0 || n > INT_MAX) return TQP_ERR_INVALID;
  if (n == 0) return TQP_OK;
  if (!d_ns) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  date_parts_kernel<<<stride_grid(n, 256), 256, 0, s>>>(reinterpret_cast<const long long*>(d_ns), n, d_days, d_year,
                                                        d_month, d_mday);
  note_launch();
  return last_launch();
}

tqp_status tqp_sort_pairs(int32_t key_dtype, const void* d_keys_in, const int32_t* d_vals_in, void* d_keys_out,
                          int32_t* d_vals_out, int64_t n, const int64_t* d_n, int begin_bit, int end_bit,
                          void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || n < 0 || n >= (1ll << 30)) return TQP_ERR_INVALID;
  if (!valid_dtype(key_dtype)) return TQP_ERR_DTYPE;
  const int w = key_bits(key_dtype);
  if (begin_bit < 0 || end_bit > w || begin_bit >= end_bit) return TQP_ERR_INVALID;
  const int word_bytes = w <= 32 ? 4 : 8;
  const int npasses = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  Carver c(ws);
  SortWs sw = carve_sort(c, n, word_bytes, npasses);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (n > 0 && (!d_keys_in || !d_keys_out || !d_vals_out)) return TQP_ERR_INVALID;
  return run_sort(sw, key_dtype, d_keys_in, d_vals_in, d_keys_out, d_vals_out, n, d_n, begin_bit, end_bit,
                  reinterpret_cast<cudaStream_t>(stream));
}

tqp_status tqp_join_eq(tqp_col probe, int64_t n_probe, const int64_t* d_n_probe, tqp_col build, int64_t n_build,
                       const int64_t* d_n_build, int32_t* d_out_probe, int32_t* d_out_build, int64_t cap,
                       int64_t* d_out_n, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  constexpr int T = 256, I = 4;
  if (!ws_bytes || n_probe < 0 || n_probe > INT_MAX || n_build < 0 || n_build >= (1ll << 30)) return TQP_ERR_INVALID;
  if (!valid_dtype(probe.dtype) || probe.dtype != build.dtype) return TQP_ERR_DTYPE;
  const int eb = dtype_bytes(build.dtype);
  const int word_bytes = eb <= 4 ? 4 : 8;
  const int64_t tiles = (n_probe + T * I - 1) / (T * I);
  Carver c(ws);
  void* skeys = c.take<char>((size_t)(n_build > 0 ? n_build : 1) * eb);
  int32_t* srows = c.take<int32_t>((size_t)(n_build > 0 ? n_build : 1));
  SortWs sw = carve_sort(c, n_build, word_bytes, eb);  // eb bytes = eb digits of 8 bits
  unsigned long long* status = c.take<unsigned long long>((size_t)(tiles > 0 ? tiles : 1));
  uint32_t* counter = c.take<uint32_t>(1);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_out_n || cap < 0 || (cap > 0 && (!d_out_probe || !d_out_build))) return TQP_ERR_INVALID;
  if ((n_probe > 0 && !probe.data) || (n_build > 0 && !build.data)) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_probe == 0) {
    TQP_CUDA(cudaMemsetAsync(d_out_n, 0, sizeof(int64_t), s));
    return TQP_OK;
  }
  tqp_status st = run_sort(sw, build.dtype, build.data, nullptr, skeys, srows, n_build, d_n_build, 0, eb * 8, s);
  if (st != TQP_OK) return st;
  TQP_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * 8, s));
  TQP_CUDA(cudaMemsetAsync(counter, 0, 4, s));
#define TQP_JOIN_LAUNCH(TYPE)                                                                      \
  {                                                                                                \
    JoinArgs<TYPE> a;                                                                              \
    a.probe = static_cast<const TYPE*>(probe.data);                                                \
    a.np_max = n_probe;                                                                            \
    a.d_np = d_n_probe;                                                                            \
    a.sorted_keys = static_cast<const TYPE*>(skeys);                                               \
    a.sorted_rows = srows;                                                                         \
    a.nb_max = n_build;                                                                            \
    a.d_nb = d_n_build;                                                                            \
    a.out_probe = d_out_probe;                                                                     \
    a.out_build = d_out_build;                                                                     \
    a.cap = cap;                                                                                   \
    a.d_out_n = d_out_n;                                                                           \
    a.status = status;                                                                             \
    a.tile_counter = counter;                                                                      \
    a.num_tiles = (uint32_t)tiles;                                                                 \
    auto k = join_probe_kernel<TYPE, T, I>;                                                        \
    prof_mark(5, true, s); k<<<persistent_grid(k, T, 0, tiles), T, 0, s>>>(a); note_launch(); prof_mark(5, false, s); \
  }
  switch (build.dtype) {
    case TQP_I8: TQP_JOIN_LAUNCH(int8_t); break;
    case TQP_I16: TQP_JOIN_LAUNCH(int16_t); break;
    case TQP_I32: TQP_JOIN_LAUNCH(int32_t); break;
    default: TQP_JOIN_LAUNCH(long long); break;
  }
#undef TQP_JOIN_LAUNCH
  return last_launch();
}

tqp_status tqp_groupby_agg(const tqp_col* keys, int nkeys, const tqp_col* vals, int nvals, const tqp_expr* exprs,
                           int nexprs, const tqp_agg* aggs, int naggs, const int32_t* d_sel, int64_t n,
                           const int64_t* d_n, void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap,
                           int64_t* d_out_groups, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || n < 0 || n >= (1ll << 30) || nkeys < 1 || nkeys > TQP_MAX_KEYS || !keys) return TQP_ERR_INVALID;
  int declared_bits = 0;
  for (int k = 0; k < nkeys; ++k) {
    if (!valid_dtype(keys[k].dtype)) return TQP_ERR_DTYPE;
    declared_bits += dtype_bytes(keys[k].dtype) * 8;
  }
  AggProgram P;
  tqp_status st = build_agg_program(vals, nvals, exprs, nexprs, aggs, naggs, &P, n > 0);
  if (st != TQP_OK) return st;
  const int word_bytes = declared_bits <= 32 ? 4 : 8;
  Carver c(ws);
  GroupWs gw = carve_group(c, n, word_bytes, &P);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_out_groups || cap < 0 || (cap > 0 && (!d_out_aggs || !d_out_keys))) return TQP_ERR_INVALID;
  KeySet ks;
  std::memset(&ks, 0, sizeof(ks));
  ks.nkeys = nkeys;
  for (int k = 0; k < nkeys; ++k) {
    if (n > 0 && !keys[k].data) return TQP_ERR_INVALID;
    if (cap > 0 && !d_out_keys[k]) return TQP_ERR_INVALID;
    ks.col[k] = keys[k].data;
    ks.dt[k] = keys[k].dtype;
    ks.out[k] = cap > 0 ? d_out_keys[k] : nullptr;
  }
  return run_groupby(gw, ks, P, d_sel, n, d_n, word_bytes, reinterpret_cast<long long*>(d_out_aggs), cap,
                     d_out_groups, reinterpret_cast<cudaStream_t>(stream));
}



// ---------------------------------------------------------------------------
// Learned CDF model and the learned group-by.
tqp_status tqp_cdf_forward(const tqp_cdf_model* d_model, const float* d_x, int64_t n, float* d_F, int32_t* d_bucket,
                           int B, tqp_stream_t stream) {
  if (n < 0 || n > INT_MAX || (d_bucket && (B < 1 || B > (1 << 24)))) return TQP_ERR_INVALID;
  if (n == 0) return TQP_OK;
  if (!d_model || !d_x || (!d_F && !d_bucket)) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  prof_mark(10, true, s);
  cdf_forward_kernel<<<stride_grid(n, 256), 256, 0, s>>>(d_model, d_x, n, d_F, d_bucket, B); note_launch();
  prof_mark(10, false, s);
  return last_launch();
}

tqp_status tqp_cdf_backward(const tqp_cdf_model* d_model, const float* d_x, const float* d_y, int64_t n,
                            float* d_grad, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || n < 0 || n > (1 << 20)) return TQP_ERR_INVALID;
  const int nb = (int)((n + kGradChunk - 1) / kGradChunk);
  Carver c(ws);
  float* partial = c.take<float>((size_t)(nb > 0 ? nb : 1) * kGradLen);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_model || !d_grad || (n > 0 && (!d_x || !d_y))) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (nb > 0) {
    // gradient only: without an Adam state the model is not written
    cdf_grad_kernel<<<nb, 256, 0, s>>>(const_cast<tqp_cdf_model*>(d_model), d_x, d_y, nullptr, n, partial, nullptr,
                                       tqp_train_cfg{}, 0, nullptr); note_launch();
  }
  cdf_grad_finish_kernel<<<1, 256, 0, s>>>(partial, nb, nullptr, n, d_grad); note_launch();
  return last_launch();
}

namespace {
bool valid_train_cfg(const tqp_train_cfg* cfg) {
  return cfg && cfg->epochs >= 0 && cfg->epochs <= 100000 && cfg->lr > 0 && cfg->beta1 >= 0 && cfg->beta1 < 1 &&
         cfg->beta2 >= 0 && cfg->beta2 < 1 && cfg->eps > 0;
}

// cfg.epochs Adam steps.  keep_best: each step first records the parameters
// it evaluated when their loss is the lowest so far, and a closing
// evaluation restores the best (loss[epochs] then holds its loss).
void launch_training(tqp_cdf_model* model, const float* x, const float* y, int64_t n, const int64_t* d_n,
                     const tqp_train_cfg& cfg, float* partial, AdamState* st, float* loss, cudaStream_t s,
                     bool keep_best = false) {
  const int nb = (int)((n + kGradChunk - 1) / kGradChunk);
  for (int e = 0; e < cfg.epochs; ++e) {
    cdf_grad_kernel<<<nb, 256, 0, s>>>(model, x, y, d_n, n, partial, st, cfg, e, loss,
                                       keep_best ? kTrainStepKeepBest : kTrainStep); note_launch();
  }
  if (keep_best && cfg.epochs > 0) {
    cdf_grad_kernel<<<nb, 256, 0, s>>>(model, x, y, d_n, n, partial, st, cfg, cfg.epochs, loss, kTrainRestoreBest);
    note_launch();
  }
}
}  // namespace

tqp_status tqp_cdf_train(const float* d_x, const float* d_y, int64_t n, tqp_cdf_model* d_model,
                         const tqp_train_cfg* cfg, float* d_loss, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || n < 1 || n > (1 << 20) || !valid_train_cfg(cfg)) return TQP_ERR_INVALID;
  const int nb = (int)((n + kGradChunk - 1) / kGradChunk);
  Carver c(ws);
  float* partial = c.take<float>((size_t)nb * kGradLen);
  AdamState* st = c.take<AdamState>(1);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_x || !d_y || !d_model) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TQP_CUDA(cudaMemsetAsync(st, 0, sizeof(AdamState), s));
  launch_training(d_model, d_x, d_y, n, nullptr, *cfg, partial, st, d_loss, s);
  return last_launch();
}

namespace {
// Workspace of the learned range partitioner (the partition and the bucket
// sorts; the reduce arrays only for the group-by).
struct LearnedWs {
  int S, SH, mult, B, nblk, epochs;
  int64_t rtiles;
  GroupPlan* gp;
  unsigned long long* sample;
  unsigned long long* ssorted;
  int32_t* srows;
  int* cut_hist;
  int* chunk_h;
  int* chunk_l;
  SortWs ssort;
  float* tx;
  float* ty;
  tqp_cdf_model* model;
  LearnedPlan* lp;
  AdamState* adam;
  float* partial;
  float* loss;
  unsigned long long* heavy;
  long long* heavy_acc;
  unsigned* thr;
  int* dir;
  unsigned* count;
  unsigned* cursor;
  unsigned* bcount;
  unsigned* off;
  int64_t* light_n;
  unsigned long long* lpk;
  int32_t* lrow;
  unsigned long long* apk;
  int32_t* arow;
  uint32_t* queue;
  uint32_t* big_flags;
  uint32_t* flagged;  // buckets the MSD kernel left to the block kernel
  unsigned* tstart;  // two-level scatter: split 2's tile starts per coarse bucket
  unsigned* cur1;    // two-level scatter: coarse cursors
  unsigned short* fine;  // two-level scatter: each row's bucket within its coarse bucket
  unsigned short* ids;   // two-level scatter: each row's bucket from the counting pass (B <= 65536)
  uint32_t* rheads;
  Partial* rcarry;
  void* lgath[TQP_MAX_VALS];
};

// B: the bucket count (0 = from n, about rows_per_bucket rows each).
LearnedWs carve_learned(Carver& c, int64_t n, const tqp_learned_cfg* cfg, int rows_per_bucket, int naggs,
                        const AggProgram* P, int32_t* rows_out, bool scatter = true) {
  LearnedWs w;
  std::memset(&w, 0, sizeof(w));
  w.S = cfg->sample;
  w.B = cfg->buckets;
  if (w.B == 0) {
    w.B = 256;
    while (w.B < (1 << 17) && (int64_t)w.B * rows_per_bucket < n) w.B <<= 1;
  }
  w.epochs = cfg->train ? cfg->train_cfg.epochs : 0;
  // heavy keys are found in a sample kHeavyMult times larger than the
  // training set (a key far beyond a bucket's capacity must not escape by
  // sampling noise); the network trains on every kHeavyMult-th sorted key
  w.SH = w.S * kHeavyMult <= (1 << 20) ? w.S * kHeavyMult : (1 << 20);
  w.mult = w.SH / w.S;
  w.nblk = num_sms();
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int nb = w.S / kGradChunk;
  const int B = w.B;
  w.gp = c.take<GroupPlan>(1);
  w.sample = c.take<unsigned long long>(w.SH);
  w.ssorted = c.take<unsigned long long>(w.SH);
  w.srows = c.take<int32_t>(w.SH);
  w.cut_hist = c.take<int>(kCutBins);
  w.chunk_h = c.take<int>((w.SH + kHeavyChunk - 1) / kHeavyChunk);
  w.chunk_l = c.take<int>((w.SH + kHeavyChunk - 1) / kHeavyChunk);
  w.ssort = carve_sort(c, w.SH, 8, 8);
  w.tx = c.take<float>(w.S);
  w.ty = c.take<float>(w.S);
  w.model = c.take<tqp_cdf_model>(1);
  w.lp = c.take<LearnedPlan>(1);
  w.adam = c.take<AdamState>(1);
  w.partial = c.take<float>((size_t)nb * kGradLen);
  w.loss = c.take<float>((size_t)w.epochs + 1);  // per epoch, then the returned network's
  w.heavy = c.take<unsigned long long>(kMaxHeavy);
  w.heavy_acc = c.take<long long>((size_t)kMaxHeavy * (naggs > 0 ? naggs : 1));
  w.thr = c.take<unsigned>((size_t)B);
  w.dir = c.take<int>((1 << kDirBits) + 1);
  w.count = c.take<unsigned>((size_t)B);
  w.cursor = c.take<unsigned>((size_t)B * kCursorStride);
  w.bcount = c.take<unsigned>(B <= kBlockHistMaxB ? (size_t)w.nblk * B : 1);
  w.off = c.take<unsigned>((size_t)B + 1);
  w.light_n = c.take<int64_t>(1);
  if (scatter) {
    w.lpk = c.take<unsigned long long>(nn);
    w.lrow = rows_out ? rows_out : c.take<int32_t>(nn);
    w.apk = c.take<unsigned long long>(nn);
    w.arow = c.take<int32_t>(nn);
  }
  w.queue = c.take<uint32_t>(4);  // block, warp and MSD kernel queues; the flagged buckets' count
  w.big_flags = c.take<uint32_t>((size_t)B);
  w.flagged = c.take<uint32_t>((size_t)B);
  w.tstart = c.take<unsigned>((1 << kSplitCoarseBits) + 1);
  if (scatter) w.fine = c.take<unsigned short>(nn);
  if (scatter && B <= 65536) w.ids = c.take<unsigned short>(nn);
  w.cur1 = c.take<unsigned>((size_t)(1 << kSplitCoarseBits) * kCursorStride);
  if (P) {  // the group-by's reduce
    w.rtiles = (n + kReduceThreads * kReduceItems - 1) / (kReduceThreads * kReduceItems);
    w.rheads = c.take<uint32_t>((size_t)(w.rtiles > 0 ? w.rtiles : 1));
    w.rcarry = c.take<Partial>((size_t)(w.rtiles > 0 ? w.rtiles : 1));
    if (n >= kPregatherRows)
      for (int v = 0; v < P->nvals; ++v) w.lgath[v] = c.take<char>(nn * dtype_bytes(P->vdt[v]));
  }
  return w;
}

// Heavy-key threshold: a key whose sample count reaches it would fill half a
// bucket's on-chip capacity on its own.
long long heavy_min_count(int SH, int64_t n) {
  long long minc = (long long)((double)SH * kLocalCap / (2.0 * (double)(n > 0 ? n : 1))) + 1;
  if (minc < 2) minc = 2;
  if (minc > 4095) minc = 4095;
  return minc;
}

// Steps 1-4 of the learned range partition: key range and packing, the
// sorted sample, heavy keys (want_heavy) and the light-CDF training pairs,
// the network (knots, training), its step positions and their directory.
tqp_status run_learned_fit(const LearnedWs& w, const KeySet& ks, const int32_t* d_sel, int64_t n, const int64_t* d_n,
                           const tqp_learned_cfg* cfg, bool want_heavy, cudaStream_t s) {
  const int S = w.S, SH = w.SH, B = w.B;
  const long long minc = heavy_min_count(SH, n);
  // 1. key range and packing (always a 64-bit packed word on this path)
  gb_init_kernel<<<1, 32, 0, s>>>(w.gp); note_launch();
  gb_keyrange_kernel<256><<<stride_grid(n, 256, 4), 256, 0, s>>>(ks, d_sel, n, d_n, w.gp); note_launch();
  gb_plan_kernel<<<1, 32, 0, s>>>(w.gp, ks.nkeys, 64); note_launch();
  lp_init_kernel<<<1, 32, 0, s>>>(w.gp, ks.nkeys, w.model, w.lp, w.adam, B, (int)minc); note_launch();
  // 2. sample, sorted by the radix sort
  lp_sample_kernel<<<(SH + 255) / 256, 256, 0, s>>>(ks, d_sel, n, d_n, w.gp, SH, w.sample); note_launch();
  tqp_status st = run_sort(w.ssort, kKeyU64, w.sample, nullptr, w.ssorted, w.srows, SH, nullptr, 0, 64, s);
  if (st != TQP_OK) return st;
  // 3. heavy keys; training pairs on the CDF of the light rows (the sort's
  // row ids are no longer needed: srows holds the light prefix)
  {
    const int nch = (SH + kHeavyChunk - 1) / kHeavyChunk, g = (nch + 255) / 256;
    TQP_CUDA(cudaMemsetAsync(w.cut_hist, 0, kCutBins * sizeof(int), s));
    if (want_heavy) {
      lp_runhist_kernel<<<g, 256, 0, s>>>(w.ssorted, SH, w.lp, w.cut_hist); note_launch();
    }
    lp_cut_kernel<<<1, 32, 0, s>>>(w.cut_hist, want_heavy ? 1 : 0, w.lp); note_launch();
    lp_chunk_kernel<<<g, 256, 0, s>>>(w.ssorted, SH, w.lp, w.chunk_h, w.chunk_l); note_launch();
    lp_chunk_scan_kernel<<<1, 1024, 0, s>>>(nch, w.chunk_h, w.chunk_l, w.lp); note_launch();
    lp_heavy_write_kernel<<<g, 256, 0, s>>>(w.ssorted, SH, w.lp, w.chunk_h, w.chunk_l, w.heavy, w.srows); note_launch();
  }
  lp_targets_kernel<<<(S + 255) / 256, 256, 0, s>>>(w.ssorted, SH, w.mult, S, w.lp, w.srows, w.tx, w.ty); note_launch();
  if (cfg->init == 1) {
    lp_quantile_init_kernel<<<1, kH, 0, s>>>(w.tx, w.ty, S, w.lp, w.model); note_launch();
  }
  // 4. training, then the step positions of the bucket function and their directory
  if (w.epochs > 0)
    launch_training(w.model, w.tx, w.ty, S, nullptr, cfg->train_cfg, w.partial, w.adam, w.loss, s, true);
  if (B > 1) {
    lp_thresholds_kernel<<<(B - 1 + 255) / 256, 256, 0, s>>>(w.model, w.lp, w.thr); note_launch();
  }
  lp_directory_kernel<<<((1 << kDirBits) + 1 + 255) / 256, 256, 0, s>>>(w.lp, w.thr, w.dir); note_launch();
  return TQP_OK;
}

// The learned range partition of n packed keys and the sort of every
// bucket (see run_learned_fit for steps 1-4), then bucket counts, offsets
// and the scatter (heavy rows folded into heavy_acc by P), and every bucket
// sorted.  Leaves the light rows' packed keys and row ids sorted in
// (lpk, lrow), their count in light_n.
tqp_status run_learned_partition(const LearnedWs& w, const KeySet& ks, const int32_t* d_sel, const int32_t* payload,
                                 int64_t n, const int64_t* d_n, const tqp_learned_cfg* cfg, bool want_heavy,
                                 const AggProgram& P, tqp_learned_stats* d_stats, cudaStream_t s) {
  const int B = w.B, naggs = P.naggs;
  tqp_status st = run_learned_fit(w, ks, d_sel, n, d_n, cfg, want_heavy, s);
  if (st != TQP_OK) return st;
  // 5. partition: bucket counts, offsets, scatter (heavy rows folded on the fly)
  PartArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.ks = ks;
  pa.sel = d_sel;
  pa.payload = payload;
  pa.n_max = n;
  pa.d_n = d_n;
  pa.gp = w.gp;
  pa.lp = w.lp;
  pa.thr = w.thr;
  pa.dir = w.dir;
  pa.heavy = w.heavy;
  pa.count = w.count;
  pa.cursor = w.cursor;
  pa.out_p = w.lpk;
  pa.out_row = w.lrow;
  pa.heavy_acc = w.heavy_acc;
  pa.bcount = w.bcount;
  pa.ids = want_heavy ? nullptr : w.ids;  // the two-level scatter reads the counting pass's buckets
  TQP_CUDA(cudaMemsetAsync(w.count, 0, (size_t)B * sizeof(unsigned), s));
  {
    // the steps live in shared memory when the scatter's layout still fits.
    // Counting: up to kBlockHistMaxB buckets each block counts one chunk of
    // rows in shared memory (then the column sums); placing: one global
    // cursor per bucket, so each bucket fills as one stream
    const int smode = part_smem_bytes(B, naggs, kThrShared) <= (size_t)kMaxSmemOptin ? kThrShared : kThrGlobal;
    const int hmode = (B <= kBlockHistMaxB && part_smem_bytes(B, 0, kBlockHist) <= (size_t)kMaxSmemOptin) ? kBlockHist
                                                                                                       : smode;
    const size_t hsm = part_smem_bytes(B, 0, hmode), ssm = part_smem_bytes(B, naggs, smode);
    auto hk = hmode == kBlockHist ? lp_hist_kernel<kBlockHist>
                                  : (hmode == kThrShared ? lp_hist_kernel<kThrShared> : lp_hist_kernel<kThrGlobal>);
    auto sk = smode == kThrShared ? lp_scatter_kernel<kThrShared> : lp_scatter_kernel<kThrGlobal>;
    TQP_CUDA(smem_optin(hk, (int)hsm));
    TQP_CUDA(smem_optin(sk, (int)ssm));
    const int64_t ptiles = (n + kPartThreads * kPartItems - 1) / (kPartThreads * kPartItems);
    const int gh = hmode == kBlockHist ? w.nblk : persistent_grid(hk, kPartThreads, hsm, ptiles);
    // two-level scatter with the counting pass's ids and global counters:
    // the pass counts coarse buckets in shared memory, and the fine counts
    // are taken after split 1 from its fine ids (one atomic per tile and
    // fine bucket instead of one per row)
    const int Fsplit = split_fine_bits(B);
    const bool late_fine = !want_heavy && pa.ids != nullptr && Fsplit > 0 && hmode != kBlockHist;
    pa.coarse_F = late_fine ? Fsplit : 0;
    hk<<<gh, kPartThreads, hsm, s>>>(pa); note_launch();
    TQP_LAUNCHED();
    if (hmode == kBlockHist) {
      lp_bcols_kernel<<<(B + 255) / 256, 256, 0, s>>>(w.bcount, w.nblk, w.lp, w.count); note_launch();
    }
    lp_offsets_kernel<<<1, 1024, 0, s>>>(w.lp, w.count, w.off, w.cursor, d_stats, w.loss, w.epochs, w.light_n);
    note_launch();
    if (naggs > 0) {
      lp_heavy_init_kernel<<<(kMaxHeavy * naggs + 255) / 256, 256, 0, s>>>(w.lp, P, w.heavy_acc); note_launch();
    }
    prof_mark(8, true, s);
    if (want_heavy) {
      sk<<<persistent_grid(sk, kPartThreads, ssm, ptiles), kPartThreads, ssm, s>>>(pa, P); note_launch();
      TQP_LAUNCHED();
    } else {
      // no heavy keys: the two-level scatter (block-level multisplits)
      const int F = split_fine_bits(B);
      const bool ids = pa.ids != nullptr;
      const bool tsm = !ids && kSplitThrShared && split_smem_bytes(B, true) + 8192 <= (size_t)kMaxSmemOptin;
      const size_t xsm = split_smem_bytes(B, tsm, !ids);
      const size_t xsm2 = split_smem_bytes(B, false, false);
      auto k1 = ids ? lp_split1_kernel<false, true>
                    : (tsm ? lp_split1_kernel<true, false> : lp_split1_kernel<false, false>);
      auto k2 = lp_split2_kernel;
      TQP_CUDA(smem_optin(k1, (int)xsm));
      TQP_CUDA(smem_optin(k2, (int)xsm2));
      lp_split_tiles_kernel<<<1, 256, 0, s>>>(w.off, w.lp, F, w.tstart, w.cur1); note_launch();
      const int64_t tiles1 = (n + kSplitTile - 1) / kSplitTile;
      if (F == 0) {  // at most 256 buckets: one split, straight into the buckets
        k1<<<persistent_grid(k1, kSplitThreads, xsm, tiles1), kSplitThreads, xsm, s>>>(pa, 0, w.cursor, w.lpk, w.lrow,
                                                                                       nullptr);
        note_launch();
        TQP_LAUNCHED();
      } else {
        k1<<<persistent_grid(k1, kSplitThreads, xsm, tiles1), kSplitThreads, xsm, s>>>(pa, F, w.cur1, w.apk, w.arow,
                                                                                       w.fine);
        note_launch();
        TQP_LAUNCHED();
        const int64_t tiles2 = tiles1 + (B >> F) + 1;
        if (late_fine) {
          TQP_CUDA(cudaMemsetAsync(w.count, 0, (size_t)B * sizeof(unsigned), s));
          lp_fine_count_kernel<<<persistent_grid(lp_fine_count_kernel, kSplitThreads, 0, tiles2), kSplitThreads, 0, s>>>(
              w.lp, F, w.off, w.tstart, w.fine, w.count);
          note_launch();
          lp_offsets_kernel<<<1, 1024, 0, s>>>(w.lp, w.count, w.off, w.cursor, d_stats, w.loss, w.epochs, w.light_n);
          note_launch();
        }
        k2<<<persistent_grid(k2, kSplitThreads, xsm2, tiles2), kSplitThreads, xsm2, s>>>(w.lp, F, w.off, w.tstart, w.apk,
                                                                                            w.arow, w.fine, w.cursor, w.lpk,
                                                                                            w.lrow);
        note_launch();
        TQP_LAUNCHED();
      }
    }
    prof_mark(8, false, s);
  }
  // 6. every bucket sorted: on-chip up to the capacity, else by one block in global memory
  {
    BucketSortArgs ba;
    ba.lp = w.lp;
    ba.off = w.off;
    ba.p = w.lpk;
    ba.row = w.lrow;
    ba.alt_p = w.apk;
    ba.alt_row = w.arow;
    ba.queue = w.queue;
    ba.big_flags = w.big_flags;
    ba.only_flagged = 0;
    ba.flagged = w.flagged;
    ba.nflagged = w.queue + 3;
    size_t smem = (size_t)kLocalCap * (8 + 8 + 4 + 4) + (size_t)kLocalWarps * (kRadix + 1) * 4 + kRadix * 4;
    size_t wsmem = (size_t)kWarpSortWarps * (2 * kWarpCap * 8 + (kRadix + 1) * 4);
    TQP_CUDA(smem_optin(lp_bucket_sort_kernel, (int)smem));
    TQP_CUDA(smem_optin(lp_bucket_sort_warp_kernel, (int)wsmem));
    TQP_CUDA(cudaMemsetAsync(w.queue, 0, 4 * sizeof(uint32_t), s));
    TQP_CUDA(cudaMemsetAsync(w.big_flags, 0, (size_t)B * sizeof(uint32_t), s));
    {
      int gw = persistent_grid(lp_bucket_sort_warp_kernel, kWarpSortWarps * 32, wsmem,
                               (B + kWarpSortWarps - 1) / kWarpSortWarps);
      prof_mark(9, true, s);
      lp_bucket_sort_warp_kernel<<<gw, kWarpSortWarps * 32, wsmem, s>>>(ba, w.queue + 1, w.big_flags); note_launch();
      TQP_LAUNCHED();
      prof_mark(9, false, s);
    }
    int g = w.nblk;
    if (g > B) g = B;
    prof_mark(7, true, s);
    if (!want_heavy) {
      // distinct, spread keys (no heavy keys): the MSD kernel at two blocks
      // per SM takes the buckets it can; the block kernel the rest
      TQP_CUDA(smem_optin(lp_bucket_msd_kernel, (int)kMsdSortSmem));
      const int gm = persistent_grid(lp_bucket_msd_kernel, kLocalThreads, kMsdSortSmem, B);
      lp_bucket_msd_kernel<<<gm, kLocalThreads, kMsdSortSmem, s>>>(ba, w.queue + 2, w.big_flags); note_launch();
      TQP_LAUNCHED();
      ba.only_flagged = 1;
    }
    lp_bucket_sort_kernel<<<g, kLocalThreads, smem, s>>>(ba); note_launch();
    TQP_LAUNCHED();
    prof_mark(7, false, s);
  }
  return TQP_OK;
}

bool valid_learned_cfg(const tqp_learned_cfg* cfg) {
  if (!cfg) return false;
  const int S = cfg->sample;
  if (S < 1024 || S > (1 << 20) || (S & (S - 1))) return false;
  if (cfg->buckets < 0 || cfg->buckets == 1 || cfg->buckets > (1 << 17) || (cfg->buckets & (cfg->buckets - 1)))
    return false;
  if (cfg->train && !valid_train_cfg(&cfg->train_cfg)) return false;
  return cfg->init == 0 || cfg->init == 1;
}

// Sort of n keys (one int32 / int64 column, distinct keys) with their row
// ids (vals_in, null: the index) through the learned range partitioner
// without heavy keys: keys_out in the key's dtype, rows in w.lrow.  Rows of
// equal keys would come out in no particular order.
tqp_status run_sort_learned(const LearnedWs& w, int key_dt, const void* keys_in, const int32_t* vals_in,
                            void* keys_out, int64_t n, const int64_t* d_n, const tqp_learned_cfg* cfg,
                            cudaStream_t s) {
  if (n == 0) return TQP_OK;
  KeySet ks;
  std::memset(&ks, 0, sizeof(ks));
  ks.nkeys = 1;
  ks.col[0] = keys_in;
  ks.dt[0] = key_dt;
  AggProgram none;
  std::memset(&none, 0, sizeof(none));
  tqp_status st = run_learned_partition(w, ks, nullptr, vals_in, n, d_n, cfg, false, none, nullptr, s);
  if (st != TQP_OK) return st;
  if (keys_out) {
    lp_decode_kernel<<<stride_grid(n, 256), 256, 0, s>>>(w.lpk, w.gp, key_dt, n, w.light_n, keys_out); note_launch();
  }
  return TQP_OK;
}
}  // namespace

tqp_status tqp_groupby_agg_learned(const tqp_col* keys, int nkeys, const tqp_col* vals, int nvals,
                                   const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                                   const int32_t* d_sel, int64_t n, const int64_t* d_n, void* const* d_out_keys,
                                   int64_t* d_out_aggs, int64_t cap, int64_t* d_out_groups,
                                   const tqp_learned_cfg* cfg, tqp_cdf_model* d_model_out,
                                   tqp_learned_stats* d_stats, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || !cfg || n < 0 || n >= (1ll << 30) || nkeys < 1 || nkeys > TQP_MAX_KEYS || !keys)
    return TQP_ERR_INVALID;
  if (!valid_learned_cfg(cfg)) return TQP_ERR_INVALID;
  for (int k = 0; k < nkeys; ++k)
    if (!valid_dtype(keys[k].dtype)) return TQP_ERR_DTYPE;
  AggProgram P;
  tqp_status st = build_agg_program(vals, nvals, exprs, nexprs, aggs, naggs, &P, n > 0);
  if (st != TQP_OK) return st;
  Carver c(ws);
  // about 512 rows per bucket by default: most buckets fit one warp's sort
  const LearnedWs w = carve_learned(c, n, cfg, 512, naggs, &P, nullptr);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_out_groups || cap < 0 || (cap > 0 && (!d_out_aggs || !d_out_keys))) return TQP_ERR_INVALID;
  KeySet ks;
  std::memset(&ks, 0, sizeof(ks));
  ks.nkeys = nkeys;
  for (int k = 0; k < nkeys; ++k) {
    if (n > 0 && !keys[k].data) return TQP_ERR_INVALID;
    if (cap > 0 && !d_out_keys[k]) return TQP_ERR_INVALID;
    ks.col[k] = keys[k].data;
    ks.dt[k] = keys[k].dtype;
    ks.out[k] = cap > 0 ? d_out_keys[k] : nullptr;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    TQP_CUDA(cudaMemsetAsync(d_out_groups, 0, sizeof(int64_t), s));
    if (d_stats) TQP_CUDA(cudaMemsetAsync(d_stats, 0, sizeof(tqp_learned_stats), s));
    return TQP_OK;
  }
  st = run_learned_partition(w, ks, d_sel, nullptr, n, d_n, cfg, cfg->heavy != 0, P, d_stats, s);
  if (st != TQP_OK) return st;
  // 7. reduce-by-key over the sorted light rows, merging the heavy keys
  ReduceArgs r;
  r.keys = w.lpk;
  r.rows = w.lrow;
  r.n_max = n;
  r.d_n = w.light_n;
  r.plan = w.gp;
  r.ks = ks;
  r.out_aggs = reinterpret_cast<long long*>(d_out_aggs);
  r.cap = cap;
  r.d_out_groups = d_out_groups;
  r.tile_heads = w.rheads;
  r.carry = w.rcarry;
  r.num_tiles = (uint32_t)w.rtiles;
  r.heavy = w.heavy;
  r.d_nheavy = &w.lp->nheavy;
  r.heavy_acc = w.heavy_acc;
  AggProgram Pr = P;
  const bool self_gather = P.simple && P.nvals == 1;  // the reduce reads the values through the row ids
  if ((w.lgath[0] && !self_gather) || P.nvals == 0) {
    if (P.nvals) Pr = pregather_values(P, const_cast<void* const*>(w.lgath), w.lrow, n, w.light_n, s);
    r.rows = nullptr;
  }
  launch_reduce<unsigned long long>(r, Pr, (uint32_t)w.rtiles, s);
  gb_heavy_only_kernel<<<(kMaxHeavy + 255) / 256, 256, 0, s>>>(r, naggs); note_launch();
  if (d_model_out) TQP_CUDA(cudaMemcpyAsync(d_model_out, w.model, sizeof(tqp_cdf_model), cudaMemcpyDeviceToDevice, s));
  return last_launch();
}

tqp_status tqp_partition_learned(const tqp_col* keys, int nkeys, const int32_t* d_sel, int64_t n, const int64_t* d_n,
                                 const tqp_learned_cfg* cfg, int32_t* d_bucket, int32_t* d_rows, int64_t* d_offsets,
                                 float* d_train_x, float* d_train_y, tqp_cdf_model* d_model_out,
                                 tqp_learned_stats* d_stats, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || !cfg || n < 0 || n >= (1ll << 30) || nkeys < 1 || nkeys > TQP_MAX_KEYS || !keys)
    return TQP_ERR_INVALID;
  if (!valid_learned_cfg(cfg)) return TQP_ERR_INVALID;
  for (int k = 0; k < nkeys; ++k)
    if (!valid_dtype(keys[k].dtype)) return TQP_ERR_DTYPE;
  Carver c(ws);
  const LearnedWs w = carve_learned(c, n, cfg, 512, 0, nullptr, nullptr, false);
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int nb = w.B + kMaxHeavy;  // bucket ids: B light buckets, then one per heavy key
  int nbits = 1;
  while ((1 << nbits) < nb) ++nbits;
  int32_t* ids = c.take<int32_t>(nn);
  uint32_t* sids = c.take<uint32_t>(nn);
  int32_t* rows = c.take<int32_t>(nn);
  long long* off = c.take<long long>((size_t)nb + 1);
  SortWs sw = carve_sort(c, n, 4, (nbits + kRadixBits - 1) / kRadixBits);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  KeySet ks;
  std::memset(&ks, 0, sizeof(ks));
  ks.nkeys = nkeys;
  for (int k = 0; k < nkeys; ++k) {
    if (n > 0 && !keys[k].data) return TQP_ERR_INVALID;
    ks.col[k] = keys[k].data;
    ks.dt[k] = keys[k].dtype;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (d_offsets) TQP_CUDA(cudaMemsetAsync(d_offsets, 0, ((size_t)nb + 1) * sizeof(int64_t), s));
    if (d_stats) TQP_CUDA(cudaMemsetAsync(d_stats, 0, sizeof(tqp_learned_stats), s));
    return TQP_OK;
  }
  tqp_status st = run_learned_fit(w, ks, d_sel, n, d_n, cfg, cfg->heavy != 0, s);
  if (st != TQP_OK) return st;
  // every row's bucket id
  PartArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.ks = ks;
  pa.sel = d_sel;
  pa.n_max = n;
  pa.d_n = d_n;
  pa.gp = w.gp;
  pa.lp = w.lp;
  pa.thr = w.thr;
  pa.dir = w.dir;
  pa.heavy = w.heavy;
  int32_t* id_out = d_bucket ? d_bucket : ids;
  {
    const int mode = part_smem_bytes(w.B, 0, kThrShared) <= (size_t)kMaxSmemOptin ? kThrShared : kThrGlobal;
    const size_t sm = part_smem_bytes(w.B, 0, mode);
    auto k = mode == kThrShared ? lp_bucket_ids_kernel<kThrShared> : lp_bucket_ids_kernel<kThrGlobal>;
    TQP_CUDA(smem_optin(k, (int)sm));
    const int64_t tiles = (n + kPartThreads - 1) / kPartThreads;
    k<<<persistent_grid(k, kPartThreads, sm, tiles), kPartThreads, sm, s>>>(pa, id_out); note_launch();
    TQP_LAUNCHED();
  }
  // rows grouped by bucket id, in input order within a bucket (a stable
  // radix sort of the ids, the row ids as payload), and the offsets
  if (d_rows || d_offsets || d_stats) {
    int32_t* rows_out = d_rows ? d_rows : rows;
    st = run_sort(sw, kKeyU32, id_out, d_sel, sids, rows_out, n, d_n, 0, nbits, s);
    if (st != TQP_OK) return st;
    long long* off_out = d_offsets ? reinterpret_cast<long long*>(d_offsets) : off;
    lp_offsets_sorted_kernel<<<stride_grid(n, 256), 256, 0, s>>>(sids, n, d_n, nb, off_out); note_launch();
    if (d_stats) {
      lp_partition_stats_kernel<<<1, 1024, 0, s>>>(w.lp, off_out, w.loss, w.epochs, d_stats); note_launch();
    }
  }
  if (d_train_x) TQP_CUDA(cudaMemcpyAsync(d_train_x, w.tx, (size_t)w.S * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (d_train_y) TQP_CUDA(cudaMemcpyAsync(d_train_y, w.ty, (size_t)w.S * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (d_model_out) TQP_CUDA(cudaMemcpyAsync(d_model_out, w.model, sizeof(tqp_cdf_model), cudaMemcpyDeviceToDevice, s));
  return last_launch();
}

namespace {
struct StarDimWs {
  unsigned long long* fstatus;
  uint32_t* fcounter;
  int32_t* sel;
  int64_t* cnt;
  void* gkeys;
  void* skeys;
  int32_t* srows;
  SortWs ksort;
  bool learned;      // keys sorted through the learned range partitioner
  LearnedWs lws;
  // group ranks
  GroupPlan* gplan;
  void* packed;
  int32_t* prow;
  void* spacked;
  int32_t* sprow;
  SortWs gsort;
  unsigned long long* rstatus;
  uint32_t* rcounter;
  int32_t* rank_of_row;
  long long* gkey;
  long long* G;
  DomPlan* dom;          // group ranks over a small value domain
  int64_t* sort_n;       // rows the sort path ranks (0 when the domain path does)
  uint32_t* dbits;
  int* dpre;
  int dwords;
  int rank_payload;      // no value of the dimension is aggregated: the sort may carry ranks
  int32_t* payload;
  int32_t* rank_sorted;
  void* kr;
  long long* dval[TQP_MAX_VALS];
  uint32_t ftiles, rtiles;
  int gword;
  // key directory
  unsigned long long* krange;  // passing key images' min and max (dense-key check)
  int64_t* ksort_n;            // rows the key sort takes (0 for a dense dimension)
  DimDir* dplan;
  int* dir;
  uint32_t* bitmap;
  int log2cells;
  DirCell* table;
  int32_t* rank_cell;
  long long* dval_cell[TQP_MAX_VALS];
};

// The fused star aggregate; lcfg (nullable) sorts every large dimension's
// keys through the learned range partitioner instead of the radix sort.
tqp_status star_agg_impl(const tqp_col* fact_cols, int nfact_cols, int64_t n_fact, const tqp_pred* fact_preds,
                         int nfact_preds, const int* fk_col, const tqp_dim* dims, int ndims, const tqp_valref* vals,
                         int nvals, const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                         void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap, int64_t* d_out_groups, void* ws,
                         size_t* ws_bytes, tqp_stream_t stream, const tqp_learned_cfg* lcfg) {
  if (!ws_bytes || n_fact < 0 || n_fact > INT_MAX || ndims < 1 || ndims > kMaxDims || !dims || !fk_col ||
      !fact_cols || nfact_cols < 1)
    return TQP_ERR_INVALID;
  if (nfact_preds < 0 || nfact_preds > TQP_MAX_PREDS || (nfact_preds && !fact_preds)) return TQP_ERR_INVALID;
  if (nvals < 0 || nvals > TQP_MAX_VALS || (nvals && !vals)) return TQP_ERR_INVALID;
  if (nexprs < 0 || nexprs > TQP_MAX_EXPRS || (nexprs && !exprs) || naggs < 1 || naggs > TQP_MAX_AGGS - 1 || !aggs)
    return TQP_ERR_INVALID;
  // ---- host-side validation and slot bound
  long long slots_cap = 1;
  int nout_keys = 0;
  for (int d = 0; d < ndims; ++d) {
    const tqp_dim& D = dims[d];
    if (D.n < 0 || D.n >= (1ll << 30)) return TQP_ERR_INVALID;
    if (D.key.dtype != TQP_I32 && D.key.dtype != TQP_I64) return TQP_ERR_DTYPE;
    if (fk_col[d] < 0 || fk_col[d] >= nfact_cols) return TQP_ERR_INVALID;
    if (fact_cols[fk_col[d]].dtype != D.key.dtype) return TQP_ERR_DTYPE;
    if (D.npred < 0 || D.npred > TQP_MAX_PREDS || (D.npred && (!D.preds || !D.cols))) return TQP_ERR_INVALID;
    for (int p = 0; p < D.npred; ++p) {
      if (D.preds[p].col < 0 || D.preds[p].col >= D.ncols) return TQP_ERR_INVALID;
      if (!valid_dtype(D.cols[D.preds[p].col].dtype)) return TQP_ERR_DTYPE;
      if (D.preds[p].op < TQP_LT || D.preds[p].op > TQP_NE) return TQP_ERR_INVALID;
    }
    if (D.group.data) {
      if (!valid_dtype(D.group.dtype)) return TQP_ERR_DTYPE;
      long long dom = dtype_bytes(D.group.dtype) >= 4 ? (1ll << 40) : (1ll << (8 * dtype_bytes(D.group.dtype)));
      long long g = D.n < dom ? D.n : dom;
      if (g < 1) g = 1;
      slots_cap *= g;
      if (slots_cap > (1ll << 26)) return TQP_ERR_UNSUPPORTED;
      ++nout_keys;
    }
  }
  for (int p = 0; p < nfact_preds; ++p) {
    if (fact_preds[p].col < 0 || fact_preds[p].col >= nfact_cols) return TQP_ERR_INVALID;
    if (!valid_dtype(fact_cols[fact_preds[p].col].dtype)) return TQP_ERR_DTYPE;
    if (fact_preds[p].op < TQP_LT || fact_preds[p].op > TQP_NE) return TQP_ERR_INVALID;
  }
  for (int v = 0; v < nvals; ++v) {
    int src = vals[v].src;
    if (src < 0 || src > ndims) return TQP_ERR_INVALID;
    const tqp_col* cols = src == 0 ? fact_cols : dims[src - 1].cols;
    int nc = src == 0 ? nfact_cols : dims[src - 1].ncols;
    if (vals[v].col < 0 || vals[v].col >= nc || !cols) return TQP_ERR_INVALID;
    if (!valid_dtype(cols[vals[v].col].dtype)) return TQP_ERR_DTYPE;
  }
  StarAcc A;
  std::memset(&A, 0, sizeof(A));
  A.naggs = naggs;
  A.nexprs = nexprs;
  for (int e = 0; e < nexprs; ++e) {
    if (exprs[e].nterms < 1 || exprs[e].nterms > 3) return TQP_ERR_INVALID;
    A.nterms[e] = exprs[e].nterms;
    for (int t = 0; t < exprs[e].nterms; ++t) {
      if (exprs[e].term[t].col < 0 || exprs[e].term[t].col >= nvals) return TQP_ERR_INVALID;
      A.tval[e][t] = exprs[e].term[t].col;
      A.tmul[e][t] = exprs[e].term[t].mul;
      A.tadd[e][t] = exprs[e].term[t].add;
    }
  }
  for (int q = 0; q < naggs; ++q) {
    if (aggs[q].op < TQP_COUNT || aggs[q].op > TQP_MAX) return TQP_ERR_INVALID;
    if (aggs[q].op != TQP_COUNT && (aggs[q].expr < 0 || aggs[q].expr >= nexprs)) return TQP_ERR_INVALID;
    A.op[q] = aggs[q].op;
    A.expr[q] = aggs[q].op == TQP_COUNT ? 0 : aggs[q].expr;
  }
  A.cnt = naggs;
  for (int q = naggs - 1; q >= 0; --q)
    if (aggs[q].op == TQP_COUNT) A.cnt = q;
  // ---- workspace
  Carver c(ws);
  StarDimWs W[kMaxDims];
  for (int d = 0; d < ndims; ++d) {
    const tqp_dim& D = dims[d];
    StarDimWs& w = W[d];
    std::memset(&w, 0, sizeof(w));
    const size_t nn = (size_t)(D.n > 0 ? D.n : 1);
    const int eb = dtype_bytes(D.key.dtype);
    w.ftiles = (uint32_t)((D.n + kFilterT * kFilterI - 1) / (kFilterT * kFilterI));
    if (D.npred) {
      w.fstatus = c.take<unsigned long long>(w.ftiles ? w.ftiles : 1);
      w.fcounter = c.take<uint32_t>(1);
      w.sel = c.take<int32_t>(nn);
      w.cnt = c.take<int64_t>(1);
      w.gkeys = c.take<char>(nn * eb);
    }
    w.skeys = c.take<char>(nn * eb);
    w.srows = c.take<int32_t>(nn);
    // large dimensions' keys through the learned range partitioner when asked
    w.learned = lcfg && D.n >= kLearnedSortMinRows;
    if (w.learned) {
      tqp_learned_cfg lc = *lcfg;
      lc.heavy = 0;
      w.lws = carve_learned(c, D.n, &lc, kLearnedSortRowsPerBucket, 0, nullptr, w.srows);
    } else {
      w.ksort = carve_sort(c, D.n, eb, eb);
    }
    if (D.group.data) {
      w.gword = dtype_bytes(D.group.dtype) <= 4 ? 4 : 8;
      w.gplan = c.take<GroupPlan>(1);
      w.packed = c.take<char>(nn * w.gword);
      w.prow = c.take<int32_t>(nn);
      w.spacked = c.take<char>(nn * w.gword);
      w.sprow = c.take<int32_t>(nn);
      w.gsort = carve_sort(c, D.n, w.gword, w.gword);
      w.rtiles = (uint32_t)((D.n + kRankT * kRankI - 1) / (kRankT * kRankI));
      w.rstatus = c.take<unsigned long long>(w.rtiles ? w.rtiles : 1);
      w.rcounter = c.take<uint32_t>(1);
      w.rank_of_row = c.take<int32_t>(nn);
      w.gkey = c.take<long long>(nn);
      {
        const int b = 8 * dtype_bytes(D.group.dtype) < kDomBits ? 8 * dtype_bytes(D.group.dtype) : kDomBits;
        w.dwords = 1 << (b - 5);
      }
      w.rank_payload = 1;
      for (int v = 0; v < nvals; ++v)
        if (vals[v].src == d + 1) w.rank_payload = 0;
      w.payload = c.take<int32_t>(nn);
      w.dom = c.take<DomPlan>(1);
      w.sort_n = c.take<int64_t>(1);
      w.dbits = c.take<uint32_t>((size_t)w.dwords);
      w.dpre = c.take<int>((size_t)w.dwords);
      w.G = c.take<long long>(1);
    }
    w.rank_sorted = c.take<int32_t>(nn);
    w.kr = c.take<char>(nn * (eb == 4 ? sizeof(KeyRank32) : sizeof(KeyRank64)));
    for (int v = 0; v < nvals; ++v)
      if (vals[v].src == d + 1) w.dval[v] = c.take<long long>(nn);
    w.log2cells = 1;
    while (w.log2cells < 27 && (1ll << w.log2cells) < 8 * D.n) ++w.log2cells;
    w.dplan = c.take<DimDir>(1);
    w.krange = c.take<unsigned long long>(2);
    w.ksort_n = c.take<int64_t>(1);
    w.dir = c.take<int>((size_t)(1ll << w.log2cells) + 2);
    w.bitmap = c.take<uint32_t>((size_t)(1ll << w.log2cells) / 32 + 1);
    {
      // wide cells number at most 2^t with 2^t >= 2 x the dimension's rows
      int t = 1;
      while (t < w.log2cells && (1ll << t) < wide_cells_wanted(D.n, D.key.dtype)) ++t;
      w.table = c.take<DirCell>((size_t)(1ll << t) + 1);
    }
    w.rank_cell = c.take<int32_t>((size_t)(1ll << w.log2cells) + 1);
    for (int v = 0; v < nvals; ++v)
      if (vals[v].src == d + 1) w.dval_cell[v] = c.take<long long>((size_t)(1ll << w.log2cells) + 1);
  }
  StarPlan* plan = c.take<StarPlan>(1);
  const int nacc = naggs + 1;
  long long* acc = c.take<long long>((size_t)slots_cap * nacc);
  unsigned* wcounter = c.take<unsigned>(1);
  const int64_t ptiles = (n_fact + kProbeT * kProbeI - 1) / (kProbeT * kProbeI);
  const int64_t ctiles = (slots_cap + kCompactT * kCompactI - 1) / (kCompactT * kCompactI);
  unsigned long long* cstatus = c.take<unsigned long long>((size_t)ctiles);
  uint32_t* ccounter = c.take<uint32_t>(1);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  if (!d_out_groups || cap < 0 || (cap > 0 && (!d_out_aggs || (nout_keys && !d_out_keys)))) return TQP_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TQP_CUDA(cudaMemsetAsync(plan, 0, sizeof(StarPlan), s));
  // ---- dimensions
  for (int d = 0; d < ndims; ++d) {
    const tqp_dim& D = dims[d];
    StarDimWs& w = W[d];
    const int eb = dtype_bytes(D.key.dtype);
    const int64_t* dcnt = nullptr;
    const void* kin = D.key.data;
    const int32_t* vin = nullptr;
    if (D.npred && D.n > 0) {
      FilterArgs f;
      std::memset(&f, 0, sizeof(f));
      f.npred = D.npred;
      for (int p = 0; p < D.npred; ++p) {
        f.col[p] = D.cols[D.preds[p].col].data;
        f.dt[p] = D.cols[D.preds[p].col].dtype;
        f.op[p] = D.preds[p].op;
        f.lit[p] = D.preds[p].lit;
      }
      f.n_max = D.n;
      f.d_n = nullptr;
      f.out = w.sel;
      f.cap = D.n;
      f.d_out_n = w.cnt;
      f.status = w.fstatus;
      f.tile_counter = w.fcounter;
      f.num_tiles = w.ftiles;
      TQP_CUDA(cudaMemsetAsync(w.fstatus, 0, (size_t)w.ftiles * 8, s));
      TQP_CUDA(cudaMemsetAsync(w.fcounter, 0, 4, s));
      auto fk = filter_kernel<kFilterT, kFilterI>;
      fk<<<persistent_grid(fk, kFilterT, 0, w.ftiles), kFilterT, 0, s>>>(f); note_launch();
      int g = stride_grid(D.n, 256);
      if (eb == 4) {
        gather_kernel<int32_t><<<g, 256, 0, s>>>((const int32_t*)D.key.data, w.sel, D.n, w.cnt, (int32_t*)w.gkeys); note_launch();
      } else {
        gather_kernel<long long><<<g, 256, 0, s>>>((const long long*)D.key.data, w.sel, D.n, w.cnt,
                                                   (long long*)w.gkeys); note_launch();
      }
      dcnt = w.cnt;
      kin = w.gkeys;
      vin = w.sel;
    } else if (D.npred) {
      TQP_CUDA(cudaMemsetAsync(w.cnt, 0, 8, s));
      dcnt = w.cnt;
    }
    if (D.group.data && D.n > 0) {
      KeySet ks;
      std::memset(&ks, 0, sizeof(ks));
      ks.nkeys = 1;
      ks.col[0] = D.group.data;
      ks.dt[0] = D.group.dtype;
      gb_init_kernel<<<1, 32, 0, s>>>(w.gplan); note_launch();
      gb_keyrange_kernel<256><<<stride_grid(D.n, 256, 4), 256, 0, s>>>(ks, w.sel, D.n, dcnt, w.gplan); note_launch();
      gb_plan_kernel<<<1, 32, 0, s>>>(w.gplan, 1, w.gword * 8); note_launch();
      // a small value domain ranks through a bitmap; otherwise the packed
      // group keys are sorted and ranked (sort_n: the rows of that path)
      dom_plan_kernel<<<1, 32, 0, s>>>(w.gplan, D.n, dcnt, w.dom, w.sort_n); note_launch();
      const int64_t* gn = w.sort_n;
      // int8 and int16 group columns always rank through the bitmap: their
      // sort path is not launched (G stays 0 unless the bitmap counts groups)
      const bool small_domain = dtype_bytes(D.group.dtype) <= 2;
      TQP_CUDA(cudaMemsetAsync(w.G, 0, 8, s));
      if (!small_domain) {
        const int g = stride_grid(D.n, 256);
        if (w.gword == 4) {
          gb_encode_kernel<uint32_t><<<g, 256, 0, s>>>(ks, w.sel, D.n, gn, w.gplan, (uint32_t*)w.packed, w.prow);
        } else {
          gb_encode_kernel<unsigned long long><<<g, 256, 0, s>>>(ks, w.sel, D.n, gn, w.gplan,
                                                                 (unsigned long long*)w.packed, w.prow);
        }
        note_launch();
        const tqp_status st = run_sort(w.gsort, w.gword == 4 ? kKeyU32 : kKeyU64, w.packed, w.prow, w.spacked,
                                       w.sprow, D.n, gn, 0, w.gword * 8, s);
        if (st != TQP_OK) return st;
        TQP_CUDA(cudaMemsetAsync(w.rstatus, 0, (size_t)w.rtiles * 8, s));
        TQP_CUDA(cudaMemsetAsync(w.rcounter, 0, 4, s));
        if (w.gword == 4) {
          auto rk = rank_kernel<uint32_t, kRankT, kRankI>;
          rk<<<persistent_grid(rk, kRankT, 0, w.rtiles), kRankT, 0, s>>>(
              (const uint32_t*)w.spacked, w.sprow, D.n, gn, w.gplan, w.rank_of_row, w.gkey, w.G, w.rstatus,
              w.rcounter, w.rtiles);
        } else {
          auto rk = rank_kernel<unsigned long long, kRankT, kRankI>;
          rk<<<persistent_grid(rk, kRankT, 0, w.rtiles), kRankT, 0, s>>>(
              (const unsigned long long*)w.spacked, w.sprow, D.n, gn, w.gplan, w.rank_of_row, w.gkey, w.G,
              w.rstatus, w.rcounter, w.rtiles);
        }
        note_launch();
      }
      // after the sort path (which then counted no groups): the bitmap's ranks
      TQP_CUDA(cudaMemsetAsync(w.dbits, 0, (size_t)w.dwords * sizeof(uint32_t), s));
      const int gd = stride_grid((D.n + kDomItems - 1) / kDomItems, 256);
      dom_mark_kernel<<<gd, 256, 0, s>>>(D.group.data, D.group.dtype, w.sel, D.n, dcnt, w.dom, w.dbits); note_launch();
      dom_scan_kernel<1024><<<1, 1024, 0, s>>>(w.dom, w.dbits, w.dpre, w.gkey, w.G); note_launch();
      // the key sort's payload: the group rank itself when the bitmap ranks
      // and no value of this dimension is aggregated, else the row
      dom_payload_kernel<<<gd, 256, 0, s>>>(D.group.data, D.group.dtype, w.sel, D.n, dcnt, w.dom, w.dbits, w.dpre,
                                            w.rank_payload, w.payload);
      note_launch();
      vin = w.payload;
    } else if (D.group.data) {
      TQP_CUDA(cudaMemsetAsync(w.G, 0, 8, s));
    }
    // dense keys (a possible case up to the cell budget) skip the key sort:
    // kn counts the rows the sorted form takes
    const int64_t* kn = dcnt;
    prof_mark(12 + d, true, s);
    TQP_CUDA(cudaMemsetAsync(w.dplan, 0, sizeof(DimDir), s));
    if (D.n > 0 && D.n <= (1ll << w.log2cells)) {
      TQP_CUDA(cudaMemsetAsync(w.krange, 0xFF, 8, s));
      TQP_CUDA(cudaMemsetAsync(w.krange + 1, 0, 8, s));
      dim_range_kernel<<<stride_grid(D.n, 256, 4), 256, 0, s>>>(kin, D.key.dtype, D.n, dcnt, w.krange); note_launch();
      dim_direct_plan_kernel<<<1, 32, 0, s>>>(w.krange, D.n, dcnt, w.log2cells, w.dplan, w.ksort_n); note_launch();
      kn = w.ksort_n;
    }
    // no value of this dimension aggregated: the fused directory pass may
    // build it straight from the learned sort's packed keys and ranks
    bool dim_vals = false;
    for (int v = 0; v < nvals; ++v) dim_vals = dim_vals || vals[v].src == d + 1;
    tqp_status st;
    if (w.learned) {
      // the packed keys sorted (skeys only decoded when the fused pass does not run)
      st = run_sort_learned(w.lws, D.key.dtype, kin, vin, nullptr, D.n, kn, lcfg, s);
      if (st != TQP_OK) return st;
      dir_plan_packed_kernel<<<1, 32, 0, s>>>(w.lws.lpk, w.lws.gp, D.key.dtype, D.n, kn, D.n, w.log2cells,
                                              D.group.data ? w.G : nullptr, D.group.data ? w.dom : nullptr,
                                              dim_vals ? 0 : 1, w.dplan); note_launch();
      lp_decode_kernel<<<stride_grid(D.n, 256), 256, 0, s>>>(w.lws.lpk, w.lws.gp, D.key.dtype, D.n, kn, w.skeys,
                                                               &w.dplan->fused); note_launch();
    } else {
      st = run_sort(w.ksort, D.key.dtype, kin, vin, w.skeys, w.srows, D.n, kn, 0, eb * 8, s);
      if (st != TQP_OK) return st;
    }
    prof_mark(12 + d, false, s);
    prof_mark(14 + d, true, s);
    if (D.n > 0) {
      PregatherArgs pg;
      std::memset(&pg, 0, sizeof(pg));
      pg.skeys = w.skeys;
      pg.key_dt = D.key.dtype;
      pg.srows = w.srows;
      pg.n_max = D.n;
      pg.d_n = kn;
      pg.rank_of_row = D.group.data ? w.rank_of_row : nullptr;
      if (D.group.data) {
        pg.dom = w.dom;
        pg.gcol = D.group.data;
        pg.gdt = D.group.dtype;
        pg.dbits = w.dbits;
        pg.dpre = w.dpre;
        pg.rank_payload = w.rank_payload;
      }
      pg.rank_sorted = w.rank_sorted;
      pg.kr = w.kr;
      pg.plan = plan;
      pg.dd = w.dplan;
      for (int v = 0; v < nvals; ++v) {
        if (vals[v].src != d + 1) continue;
        pg.vcol[pg.nv] = D.cols[vals[v].col].data;
        pg.vdt[pg.nv] = D.cols[vals[v].col].dtype;
        pg.vout[pg.nv] = w.dval[v];
        ++pg.nv;
      }
      star_pregather_kernel<<<stride_grid(D.n, 256), 256, 0, s>>>(pg); note_launch();
    }
    dir_plan_kernel<<<1, 32, 0, s>>>(w.skeys, D.key.dtype, D.n, kn, D.n, w.log2cells,
                                     D.group.data ? w.G : nullptr, w.dplan); note_launch();
    if (D.n > 0) {
      TQP_CUDA(cudaMemsetAsync(w.bitmap, 0, ((size_t)(1ll << w.log2cells) / 32 + 1) * sizeof(uint32_t), s));
      if (w.learned) {
        EmitArgs ea;
        ea.packed = w.lws.lpk;
        ea.payload = w.srows;
        ea.has_group = D.group.data ? 1 : 0;
        ea.gp = w.lws.gp;
        ea.key_dt = D.key.dtype;
        ea.n_max = D.n;
        ea.d_n = kn;
        ea.dd = w.dplan;
        ea.kr = w.kr;
        ea.bitmap = w.bitmap;
        ea.table = w.table;
        ea.plan = plan;
        dir_emit_kernel<<<stride_grid(D.n, kEmitThreads), kEmitThreads, 0, s>>>(ea); note_launch();
      }
      dir_fill_kernel<<<stride_grid(D.n, 256), 256, 0, s>>>(w.skeys, D.key.dtype, D.n, kn, w.dplan, w.dir,
                                                             w.bitmap);
      note_launch();
      CellArgs ca;
      std::memset(&ca, 0, sizeof(ca));
      ca.skeys = w.skeys;
      ca.key_dt = D.key.dtype;
      ca.n_max = D.n;
      ca.d_n = kn;
      ca.dd = w.dplan;
      ca.rank_sorted = w.rank_sorted;
      ca.rank_cell = w.rank_cell;
      for (int v = 0; v < nvals; ++v) {
        if (vals[v].src != d + 1) continue;
        ca.dval[ca.nv] = w.dval[v];
        ca.dval_cell[ca.nv] = w.dval_cell[v];
        ++ca.nv;
      }
      dir_cells_kernel<<<stride_grid(D.n, 256), 256, 0, s>>>(ca); note_launch();
      {
        int t = 1;
        while (t < w.log2cells && (1ll << t) < wide_cells_wanted(D.n, D.key.dtype)) ++t;
        dir_table_kernel<<<stride_grid((1ll << t) + 1, 256), 256, 0, s>>>(w.kr, D.key.dtype, w.dplan, w.dir, w.table);
        note_launch();
      }
      DirectArgs da;
      std::memset(&da, 0, sizeof(da));
      da.keys = kin;
      da.key_dt = D.key.dtype;
      da.sel = D.npred ? w.sel : nullptr;
      da.n_max = D.n;
      da.d_n = dcnt;
      da.dd = w.dplan;
      da.bitmap = w.bitmap;
      da.rank_cell = w.rank_cell;
      if (D.group.data) {
        da.rank_of_row = w.rank_of_row;
        da.dom = w.dom;
        da.gcol = D.group.data;
        da.gdt = D.group.dtype;
        da.dbits = w.dbits;
        da.dpre = w.dpre;
      }
      for (int v = 0; v < nvals; ++v) {
        if (vals[v].src != d + 1) continue;
        da.vcol[da.nv] = D.cols[vals[v].col].data;
        da.vdt[da.nv] = D.cols[vals[v].col].dtype;
        da.dval_cell[da.nv] = w.dval_cell[v];
        ++da.nv;
      }
      da.plan = plan;
      dir_direct_kernel<<<stride_grid(D.n, 256), 256, 0, s>>>(da); note_launch();
    }
    prof_mark(14 + d, false, s);
  }
  // ---- slots, accumulators, probe, compaction
  star_slots_kernel<<<1, 32, 0, s>>>(plan, ndims, dims[0].group.data ? W[0].G : nullptr,
                                     (ndims > 1 && dims[1].group.data) ? W[1].G : nullptr, slots_cap, nacc); note_launch();
  star_init_acc_kernel<<<stride_grid(slots_cap * nacc, 256, 4), 256, 0, s>>>(plan, A, acc); note_launch();
  ProbeArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.wcounter = wcounter;
  TQP_CUDA(cudaMemsetAsync(wcounter, 0, 4, s));
  pa.ndims = ndims;
  pa.vec0 = dims[0].key.dtype == TQP_I32 && reinterpret_cast<uintptr_t>(fact_cols[fk_col[0]].data) % 16 == 0;
  for (int d = 0; d < ndims; ++d) {
    pa.dim[d].kr = W[d].kr;
    pa.dim[d].key_dt = dims[d].key.dtype;
    pa.dim[d].rank_cell = W[d].rank_cell;
    pa.dim[d].fk = fact_cols[fk_col[d]].data;
    pa.dim[d].dir_plan = W[d].dplan;
    pa.dim[d].table = W[d].table;
    pa.dim[d].bitmap = W[d].bitmap;
  }
  pa.npred = nfact_preds;
  for (int p = 0; p < nfact_preds; ++p) {
    pa.pcol[p] = fact_cols[fact_preds[p].col].data;
    pa.pdt[p] = fact_cols[fact_preds[p].col].dtype;
    pa.pop[p] = fact_preds[p].op;
    pa.plit[p] = fact_preds[p].lit;
  }
  pa.nvals = nvals;
  for (int v = 0; v < nvals; ++v) {
    pa.vsrc[v] = vals[v].src;
    if (vals[v].src == 0) {
      pa.vptr[v] = fact_cols[vals[v].col].data;
      pa.vdt[v] = fact_cols[vals[v].col].dtype;
    } else {
      pa.vptr[v] = W[vals[v].src - 1].dval[v];
      pa.vptr_cell[v] = W[vals[v].src - 1].dval_cell[v];
      pa.vdt[v] = TQP_I64;
    }
  }
  pa.n_fact = n_fact;
  pa.plan = plan;
  pa.acc = acc;
  if (ptiles > 0) {
    prof_mark(1, true, s);
    bool k32 = true;
    for (int d = 0; d < ndims; ++d) k32 = k32 && dims[d].key.dtype == TQP_I32;
    using ProbeFn = void (*)(ProbeArgs, StarAcc, int);
    if (dims[0].n <= kSmemBitmapDimRows) {
      // small first dimension: its bitmap can live in shared memory
      const ProbeFn v[2][2] = {{star_probe_kernel<1024, 4, true, false, 1>, star_probe_kernel<1024, 4, true, true, 1>},
                               {star_probe_kernel<1024, 4, true, false, 2>, star_probe_kernel<1024, 4, true, true, 2>}};
      const ProbeFn pk = v[ndims - 1][k32 ? 1 : 0];
      // the bitmap takes what the variant's static shared memory leaves of
      // the opt-in maximum, up to kSmemBitmapBytes
      int stat = 0;
      TQP_CUDA(static_smem(reinterpret_cast<const void*>(pk), &stat));
      int bytes = kMaxSmemOptin - stat;
      bytes = (bytes < kSmemBitmapBytes ? bytes : kSmemBitmapBytes) & ~255;
      TQP_CUDA(smem_optin(pk, bytes));
      const int64_t t1024 = (n_fact + 1024 * 4 - 1) / (1024 * 4);
      pk<<<persistent_grid(pk, 1024, bytes, t1024), 1024, bytes, s>>>(pa, A, bytes / 4);
      note_launch();
    } else {
      const ProbeFn v[2][2] = {
          {star_probe_kernel<kProbeT, kProbeI, false, false, 1>, star_probe_kernel<kProbeT, kProbeI, false, true, 1>},
          {star_probe_kernel<kProbeT, kProbeI, false, false, 2>, star_probe_kernel<kProbeT, kProbeI, false, true, 2>}};
      const ProbeFn pk = v[ndims - 1][k32 ? 1 : 0];
      pk<<<persistent_grid(pk, kProbeT, 0, ptiles), kProbeT, 0, s>>>(pa, A, 0); note_launch();
    }
    prof_mark(1, false, s);
  }
  CompactArgs ca;
  std::memset(&ca, 0, sizeof(ca));
  ca.plan = plan;
  ca.acc = acc;
  ca.naggs = naggs;
  ca.cnt = A.cnt;
  ca.ndims = ndims;
  int ok = 0;
  for (int d = 0; d < ndims; ++d) {
    if (dims[d].group.data) {
      ca.gkey[d] = W[d].gkey;
      ca.out_key_index[d] = ok;
      ca.out_keys[d] = cap > 0 ? d_out_keys[ok] : nullptr;
      ca.out_dt[d] = dims[d].group.dtype;
      ++ok;
    } else {
      ca.out_key_index[d] = -1;
    }
  }
  ca.out_aggs = reinterpret_cast<long long*>(d_out_aggs);
  ca.cap = cap;
  ca.d_out_groups = d_out_groups;
  ca.status = cstatus;
  ca.counter = ccounter;
  ca.num_tiles = (uint32_t)ctiles;
  TQP_CUDA(cudaMemsetAsync(cstatus, 0, (size_t)ctiles * 8, s));
  TQP_CUDA(cudaMemsetAsync(ccounter, 0, 4, s));
  auto ck = star_compact_kernel<kCompactT, kCompactI>;
  ck<<<persistent_grid(ck, kCompactT, 0, ctiles), kCompactT, 0, s>>>(ca); note_launch();
  return last_launch();
}
}  // namespace

tqp_status tqp_star_agg(const tqp_col* fact_cols, int nfact_cols, int64_t n_fact, const tqp_pred* fact_preds,
                        int nfact_preds, const int* fk_col, const tqp_dim* dims, int ndims, const tqp_valref* vals,
                        int nvals, const tqp_expr* exprs, int nexprs, const tqp_agg* aggs, int naggs,
                        void* const* d_out_keys, int64_t* d_out_aggs, int64_t cap, int64_t* d_out_groups, void* ws,
                        size_t* ws_bytes, tqp_stream_t stream) {
  return star_agg_impl(fact_cols, nfact_cols, n_fact, fact_preds, nfact_preds, fk_col, dims, ndims, vals, nvals, exprs,
                       nexprs, aggs, naggs, d_out_keys, d_out_aggs, cap, d_out_groups, ws, ws_bytes, stream, nullptr);
}

tqp_status tqp_star_agg_learned(const tqp_col* fact_cols, int nfact_cols, int64_t n_fact, const tqp_pred* fact_preds,
                                int nfact_preds, const int* fk_col, const tqp_dim* dims, int ndims,
                                const tqp_valref* vals, int nvals, const tqp_expr* exprs, int nexprs,
                                const tqp_agg* aggs, int naggs, void* const* d_out_keys, int64_t* d_out_aggs,
                                int64_t cap, int64_t* d_out_groups, const tqp_learned_cfg* cfg, void* ws,
                                size_t* ws_bytes, tqp_stream_t stream) {
  if (!valid_learned_cfg(cfg)) return TQP_ERR_INVALID;
  return star_agg_impl(fact_cols, nfact_cols, n_fact, fact_preds, nfact_preds, fk_col, dims, ndims, vals, nvals, exprs,
                       nexprs, aggs, naggs, d_out_keys, d_out_aggs, cap, d_out_groups, ws, ws_bytes, stream, cfg);
}

// ---------------------------------------------------------------------------
// Batched instances.
tqp_status tqp_star_agg_batched(const tqp_batch_shape* shape, const tqp_problem* probs, int nprob,
                                const tqp_batch_cfg* cfg, void* ws, size_t* ws_bytes, tqp_stream_t stream) {
  if (!ws_bytes || !shape || nprob < 1 || nprob > 65536 || !probs) return TQP_ERR_INVALID;
  const int items = (cfg && cfg->probe_items) ? cfg->probe_items : 8;
  if (items != 4 && items != 8 && items != 16) return TQP_ERR_INVALID;
  const tqp_batch_shape& sh = *shape;
  if (sh.nfact_cols < 1 || sh.nfact_cols > TQP_BATCH_MAX_COLS || sh.fk_col < 0 || sh.fk_col >= sh.nfact_cols)
    return TQP_ERR_INVALID;
  if (sh.key_dtype != TQP_I32 || sh.fact_dtype[sh.fk_col] != TQP_I32) return TQP_ERR_DTYPE;
  if (sh.group_dtype != TQP_I8 && sh.group_dtype != TQP_I16 && sh.group_dtype != TQP_I32) return TQP_ERR_DTYPE;
  for (int c = 0; c < sh.nfact_cols; ++c)
    if (!valid_dtype(sh.fact_dtype[c])) return TQP_ERR_DTYPE;
  if (sh.npred < 0 || sh.npred > TQP_MAX_PREDS || sh.nexprs < 0 || sh.nexprs > TQP_MAX_EXPRS || sh.naggs < 1 ||
      sh.naggs > TQP_MAX_AGGS - 1)
    return TQP_ERR_INVALID;
  BatchShape S;
  std::memset(&S, 0, sizeof(S));
  S.nfact_cols = sh.nfact_cols;
  for (int c = 0; c < sh.nfact_cols; ++c) S.fact_dt[c] = sh.fact_dtype[c];
  S.fk_col = sh.fk_col;
  S.group_dt = sh.group_dtype;
  S.npred = sh.npred;
  for (int q = 0; q < sh.npred; ++q) {
    if (sh.preds[q].col < 0 || sh.preds[q].col >= sh.nfact_cols || sh.preds[q].op < TQP_LT || sh.preds[q].op > TQP_NE)
      return TQP_ERR_INVALID;
    S.pcol[q] = sh.preds[q].col;
    S.pop[q] = sh.preds[q].op;
    S.plit[q] = sh.preds[q].lit;
  }
  S.nexprs = sh.nexprs;
  for (int e = 0; e < sh.nexprs; ++e) {
    if (sh.exprs[e].nterms < 1 || sh.exprs[e].nterms > 3) return TQP_ERR_INVALID;
    S.nterms[e] = sh.exprs[e].nterms;
    for (int t = 0; t < sh.exprs[e].nterms; ++t) {
      if (sh.exprs[e].term[t].col < 0 || sh.exprs[e].term[t].col >= sh.nfact_cols) return TQP_ERR_INVALID;
      S.tcol[e][t] = sh.exprs[e].term[t].col;
      S.tmul[e][t] = sh.exprs[e].term[t].mul;
      S.tadd[e][t] = sh.exprs[e].term[t].add;
    }
  }
  S.naggs = sh.naggs;
  for (int q = 0; q < sh.naggs; ++q) {
    if (sh.aggs[q].op < TQP_COUNT || sh.aggs[q].op > TQP_MAX) return TQP_ERR_INVALID;
    if (sh.aggs[q].op != TQP_COUNT && (sh.aggs[q].expr < 0 || sh.aggs[q].expr >= sh.nexprs)) return TQP_ERR_INVALID;
    S.op[q] = sh.aggs[q].op;
    S.expr[q] = sh.aggs[q].op == TQP_COUNT ? 0 : sh.aggs[q].expr;
  }
  // ---- host-side layout: offsets of dimension rows, probe tiles and slots
  const int TILE = 256 * items;
  std::vector<long long> dim_off(nprob), tile_off(nprob), slot_off(nprob), cell_off(nprob), word_off(nprob);
  std::vector<int> log2cells(nprob);
  long long total_dim = 0, total_tiles = 0, total_slots = 0, total_cells = 0, total_words = 0;
  const long long domain = sh.group_dtype == TQP_I8 ? 256 : sh.group_dtype == TQP_I16 ? 65536 : (1ll << 40);
  for (int p = 0; p < nprob; ++p) {
    const tqp_problem& P = probs[p];
    if (P.n_fact < 0 || P.n_fact > INT_MAX || P.n_dim < 0 || P.cap < 0) return TQP_ERR_INVALID;
    dim_off[p] = total_dim;
    tile_off[p] = total_tiles;
    slot_off[p] = total_slots;
    total_dim += P.n_dim;
    total_tiles += (P.n_fact + TILE - 1) / TILE;
    total_slots += P.n_dim < domain ? P.n_dim : domain;
    int l2 = 1;
    while (l2 < 30 && (1ll << l2) < 2 * P.n_dim) ++l2;
    log2cells[p] = l2;
    cell_off[p] = total_cells;
    word_off[p] = total_words;
    total_cells += (1ll << l2) + 2;
    total_words += (1ll << l2) / 32 + 1;
  }
  if (total_dim >= (1ll << 30) || total_tiles >= (1ll << 32)) return TQP_ERR_INVALID;
  const int nacc = S.naggs + 1;
  const size_t td = (size_t)(total_dim > 0 ? total_dim : 1);
  const int64_t seg_tiles = (total_dim + 256 * 8 - 1) / (256 * 8);
  Carver c(ws);
  BatchProb* dprobs = c.take<BatchProb>(nprob);
  long long* d_dim_off = c.take<long long>(nprob);
  long long* d_tile_off = c.take<long long>(nprob);
  unsigned long long* ckey = c.take<unsigned long long>(td);
  int32_t* crow = c.take<int32_t>(td);
  unsigned long long* cgrp = c.take<unsigned long long>(td);
  int32_t* grow = c.take<int32_t>(td);
  unsigned long long* skey = c.take<unsigned long long>(td);
  int32_t* srow = c.take<int32_t>(td);
  unsigned long long* sgrp = c.take<unsigned long long>(td);
  int32_t* sgrow = c.take<int32_t>(td);
  SortWs sw = carve_sort(c, total_dim, 8, 8);
  int32_t* seg = c.take<int32_t>(td);
  long long* gval = c.take<long long>(td);
  unsigned long long* sstatus = c.take<unsigned long long>((size_t)(seg_tiles > 0 ? seg_tiles : 1));
  uint32_t* scounter = c.take<uint32_t>(1);
  int32_t* rank_of_row = c.take<int32_t>(td);
  int32_t* key32 = c.take<int32_t>(td);
  int32_t* rank_sorted = c.take<int32_t>(td);
  long long* G = c.take<long long>(nprob);
  long long* first_seg = c.take<long long>(nprob);
  int* flag = c.take<int>(1);
  long long* acc = c.take<long long>((size_t)(total_slots > 0 ? total_slots : 1) * nacc);
  uint32_t* queue = c.take<uint32_t>(1);
  ProbDir* pdir = c.take<ProbDir>(nprob);
  int* dir = c.take<int>((size_t)total_cells);
  uint32_t* bitmap = c.take<uint32_t>((size_t)total_words);
  if (!ws) {
    *ws_bytes = c.off;
    return TQP_OK;
  }
  if (reinterpret_cast<uintptr_t>(ws) & 255) return TQP_ERR_INVALID;  // the carved arrays need it
  if (*ws_bytes < c.off) return TQP_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // ---- descriptors through kernel parameters (capturable, no host buffer kept)
  for (int first = 0; first < nprob; first += kUploadChunk) {
    UploadChunk ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.first = first;
    ch.count = nprob - first < kUploadChunk ? nprob - first : kUploadChunk;
    for (int i = 0; i < ch.count; ++i) {
      const tqp_problem& P = probs[first + i];
      if ((P.n_fact > 0 && (!P.fact_cols[sh.fk_col])) || (P.n_dim > 0 && (!P.dim_key || !P.dim_group)) ||
          !P.d_out_groups || (P.cap > 0 && (!P.out_keys || !P.out_aggs)))
        return TQP_ERR_INVALID;
      BatchProb& b = ch.p[i];
      b.n_fact = P.n_fact;
      for (int cc = 0; cc < TQP_BATCH_MAX_COLS; ++cc) b.fact[cc] = P.fact_cols[cc];
      b.n_dim = P.n_dim;
      b.key = P.dim_key;
      b.group = P.dim_group;
      b.out_keys = P.out_keys;
      b.out_aggs = reinterpret_cast<long long*>(P.out_aggs);
      b.cap = P.cap;
      b.d_out_groups = reinterpret_cast<long long*>(P.d_out_groups);
      b.dim_off = dim_off[first + i];
      b.tile_off = tile_off[first + i];
      b.slot_off = slot_off[first + i];
      b.cell_off = cell_off[first + i];
      b.word_off = word_off[first + i];
      b.log2cells = log2cells[first + i];
    }
    batch_upload_kernel<<<1, kUploadChunk, 0, s>>>(ch, dprobs); note_launch();
  }
  // offsets as separate arrays for the searches (uploaded the same way)
  for (int first = 0; first < nprob; first += kUploadChunk) {
    UploadChunk ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.first = first;
    ch.count = nprob - first < kUploadChunk ? nprob - first : kUploadChunk;
    for (int i = 0; i < ch.count; ++i) {
      ch.p[i].dim_off = dim_off[first + i];
      ch.p[i].tile_off = tile_off[first + i];
    }
    batch_offsets_kernel<<<1, kUploadChunk, 0, s>>>(ch, d_dim_off, d_tile_off); note_launch();
  }
  TQP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  batch_empty_groups_kernel<<<(nprob + 255) / 256, 256, 0, s>>>(dprobs, nprob, G); note_launch();
  if (total_dim > 0) {
    batch_dim_encode_kernel<<<stride_grid(total_dim, 256), 256, 0, s>>>(dprobs, d_dim_off, nprob, total_dim,
                                                                        sh.group_dtype, ckey, crow, cgrp, grow);
    note_launch();
    tqp_status st = run_sort(sw, kKeyU64, ckey, crow, skey, srow, total_dim, nullptr, 0, 64, s);
    if (st != TQP_OK) return st;
    st = run_sort(sw, kKeyU64, cgrp, grow, sgrp, sgrow, total_dim, nullptr, 0, 64, s);
    if (st != TQP_OK) return st;
    TQP_CUDA(cudaMemsetAsync(sstatus, 0, (size_t)seg_tiles * 8, s));
    TQP_CUDA(cudaMemsetAsync(scounter, 0, 4, s));
    auto sk = batch_seg_kernel<256, 8>;
    sk<<<persistent_grid(sk, 256, 0, seg_tiles), 256, 0, s>>>(sgrp, total_dim, sh.group_dtype, seg, gval, sstatus,
                                                              scounter, (uint32_t)seg_tiles);
    note_launch();
    batch_rank_kernel<<<stride_grid(total_dim, 256), 256, 0, s>>>(dprobs, d_dim_off, nprob, total_dim, sgrp, sgrow,
                                                                  seg, rank_of_row, G, first_seg);
    note_launch();
    batch_pregather_kernel<<<stride_grid(total_dim, 256), 256, 0, s>>>(skey, srow, d_dim_off, total_dim,
                                                                       rank_of_row, key32, rank_sorted, flag);
    note_launch();
  }
  batch_dir_plan_kernel<<<(nprob + 255) / 256, 256, 0, s>>>(dprobs, nprob, key32, pdir); note_launch();
  TQP_CUDA(cudaMemsetAsync(bitmap, 0, (size_t)total_words * sizeof(uint32_t), s));
  if (total_dim > 0) {
    batch_dir_fill_kernel<<<stride_grid(total_dim, 256), 256, 0, s>>>(dprobs, d_dim_off, nprob, total_dim, skey,
                                                                      key32, pdir, dir, bitmap);
    note_launch();
  }
  batch_init_acc_kernel<<<stride_grid(total_slots * nacc, 256, 4), 256, 0, s>>>(S, acc, total_slots); note_launch();
  TQP_CUDA(cudaMemsetAsync(queue, 0, 4, s));
  BatchProbeArgs pa;
  pa.pdir = pdir;
  pa.dir = dir;
  pa.bitmap = bitmap;
  pa.probs = dprobs;
  pa.tile_off = d_tile_off;
  pa.nprob = nprob;
  pa.num_tiles = total_tiles;
  pa.key32 = key32;
  pa.rank_sorted = rank_sorted;
  pa.G = G;
  pa.flag = flag;
  pa.acc = acc;
  pa.queue = queue;
  if (total_tiles > 0) {
    prof_mark(6, true, s);
    if (items == 4) {
      auto k = batch_probe_kernel<256, 4>;
      k<<<persistent_grid(k, 256, 0, total_tiles), 256, 0, s>>>(pa, S); note_launch();
    } else if (items == 8) {
      auto k = batch_probe_kernel<256, 8>;
      k<<<persistent_grid(k, 256, 0, total_tiles), 256, 0, s>>>(pa, S); note_launch();
    } else {
      auto k = batch_probe_kernel<256, 16>;
      k<<<persistent_grid(k, 256, 0, total_tiles), 256, 0, s>>>(pa, S); note_launch();
    }
    prof_mark(6, false, s);
  }
  batch_compact_kernel<<<nprob, 256, 0, s>>>(dprobs, G, first_seg, gval, acc, S.naggs, sh.group_dtype, flag);
  note_launch();
  return last_launch();
}

// ---------------------------------------------------------------------------
// Filter with a fixed, library-owned scratch array (for callers that cannot
// allocate a workspace).  One look-back status word per tile of
// 256 x 16 rows, then the tile counter.
}  // extern "C"

namespace {
constexpr int kNoAllocThreads = 256, kNoAllocItems = 16;
constexpr long long kNoAllocTiles = TQP_NOALLOC_MAX_ROWS / (kNoAllocThreads * kNoAllocItems);
}  // namespace

static __device__ __align__(256) unsigned long long g_filter_noalloc_scratch[kNoAllocTiles + 32];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[128] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a stand-in for the symbol).
tqp_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return TQP_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_filter_noalloc_scratch) != cudaSuccess || !p) return TQP_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return TQP_OK;
}
}  // namespace

extern "C" {

tqp_status tqp_filter_noalloc(const tqp_col* cols, int ncols, const tqp_pred* preds, int npred, int64_t n,
                              const int64_t* d_n, int32_t* d_out_idx, int64_t cap, int64_t* d_out_n,
                              tqp_stream_t stream) {
  if (n > TQP_NOALLOC_MAX_ROWS) return TQP_ERR_TOO_LARGE;
  if (n < 0 || npred < 0 || npred > TQP_MAX_PREDS || ncols < 0) return TQP_ERR_INVALID;
  if (npred && (!preds || !cols)) return TQP_ERR_INVALID;
  if (!d_out_n || cap < 0 || (cap > 0 && !d_out_idx)) return TQP_ERR_INVALID;
  FilterArgs a;
  std::memset(&a, 0, sizeof(a));
  a.npred = npred;
  for (int p = 0; p < npred; ++p) {
    int col = preds[p].col;
    if (col < 0 || col >= ncols || (n > 0 && !cols[col].data)) return TQP_ERR_INVALID;
    if (!valid_dtype(cols[col].dtype)) return TQP_ERR_DTYPE;
    if (preds[p].op < TQP_LT || preds[p].op > TQP_NE) return TQP_ERR_INVALID;
    a.col[p] = cols[col].data;
    a.dt[p] = cols[col].dtype;
    a.op[p] = preds[p].op;
    a.lit[p] = preds[p].lit;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 0) {
    TQP_CUDA(cudaMemsetAsync(d_out_n, 0, sizeof(int64_t), s));
    return TQP_OK;
  }
  void* scratch = nullptr;
  tqp_status st = noalloc_scratch(&scratch);
  if (st != TQP_OK) return st;
  const int64_t tiles = (n + kNoAllocThreads * kNoAllocItems - 1) / (kNoAllocThreads * kNoAllocItems);
  unsigned long long* status = static_cast<unsigned long long*>(scratch);
  uint32_t* counter = reinterpret_cast<uint32_t*>(status + kNoAllocTiles);
  // the array keeps the previous call's words: clear what this call uses
  TQP_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * sizeof(unsigned long long), s));
  TQP_CUDA(cudaMemsetAsync(counter, 0, sizeof(uint32_t), s));
  a.n_max = n;
  a.d_n = d_n;
  a.out = d_out_idx;
  a.cap = cap;
  a.d_out_n = d_out_n;
  a.status = status;
  a.tile_counter = counter;
  a.num_tiles = (uint32_t)tiles;
  auto k = filter_kernel<kNoAllocThreads, kNoAllocItems>;
  k<<<persistent_grid(k, kNoAllocThreads, 0, tiles), kNoAllocThreads, 0, s>>>(a); note_launch();
  return last_launch();
}

}  // extern "C"
