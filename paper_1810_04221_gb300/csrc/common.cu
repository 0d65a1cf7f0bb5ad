// common.cu -- error reporting, pool set-up and the int32 exclusive scan.
#include "common.cuh"

#include <atomic>
#include <cstdarg>
#include <mutex>
#include <vector>

#include "trace.cuh"

namespace cwm {

static thread_local std::string g_last_error;
thread_local bool g_sync_free = false;

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char *last_error() { return g_last_error.c_str(); }

amg_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  (void)cudaGetLastError();
  set_error("%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
}

amg_status status_from_device_bits(int bits, const char *where) {
  if (bits == 0) return AMG_OK;
  if (bits & kErrNotSpd) { set_error("%s: a diagonal entry is missing or not positive", where); return AMG_ERR_NOT_SPD; }
  if (bits & kErrInvalid) { set_error("%s: malformed or non-symmetric input", where); return AMG_ERR_INVALID_ARG; }
  if (bits & kErrUnsupported) { set_error("%s: a coarse row gathers more fine entries than supported", where); return AMG_ERR_UNSUPPORTED; }
  if (bits & kErrTimeout) { set_error("%s: a bounded device loop reached its iteration cap", where); return AMG_ERR_TIMEOUT; }
  if (bits & kErrBreakdown) { set_error("%s: FCG breakdown (rho <= 0 or not finite)", where); return AMG_ERR_BREAKDOWN; }
  set_error("%s: device error bits 0x%x", where, bits);
  return AMG_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

thread_local Tracer *g_tracer = nullptr;
thread_local int g_trace_level = -1;
thread_local int g_trace_sweep = 0;

TraceScope::TraceScope(const char *cat, double b, cudaStream_t st) : s(st), bytes(b) {
  if (!g_tracer || !g_tracer->on) return;
  char name[64];
  if (g_trace_level >= 0 && g_trace_sweep > 0)
    snprintf(name, sizeof(name), "%s@%d.%d", cat, g_trace_level, g_trace_sweep);
  else if (g_trace_level >= 0) snprintf(name, sizeof(name), "%s@%d", cat, g_trace_level);
  else snprintf(name, sizeof(name), "%s", cat);
  if (!g_tracer->wants(name)) return;
  t = g_tracer;
  idx = t->entry(name);
  a = t->event();
  // inside a stream capture an external record node is needed for replays to re-record it
  if (a) {
    if (t->capturing) cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
    else cudaEventRecord(a, s);
  }
}

TraceScope::~TraceScope() {
  if (!t || !a) return;
  cudaEvent_t b = t->event();
  if (!b) return;
  if (t->capturing) cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
  else cudaEventRecord(b, s);
  if (t->capturing) {
    t->graph_pending.push_back({idx, a, b, bytes});
    return;
  }
  t->pending.push_back({idx, a, b, bytes});
  if (t->pending.size() > 4096) t->flush();
}

void Tracer::collect(const std::vector<Pending> &scopes) {
  for (const Pending &p : scopes) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      TraceEntry &e = entries[p.idx];
      e.launches += 1;
      e.ms += ms;
      e.bytes += p.bytes;
    }
    (void)cudaGetLastError();
  }
}

void Tracer::release(std::vector<Pending> &scopes) {
  for (const Pending &p : scopes) {
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  scopes.clear();
}

Tracer::~Tracer() {
  flush();
  release(graph_pending);
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

bool Tracer::wants(const char *cat) const {
  return filter.empty() || std::strncmp(cat, filter.c_str(), filter.size()) == 0;
}

int Tracer::entry(const char *cat) {
  for (size_t i = 0; i < entries.size(); ++i)
    if (entries[i].name == cat) return (int)i;
  entries.push_back(TraceEntry{cat, 0, 0.0, 0.0});
  return (int)entries.size() - 1;
}

cudaEvent_t Tracer::event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

void Tracer::flush() {
  for (const Pending &p : pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      TraceEntry &e = entries[p.idx];
      e.launches += 1;
      e.ms += ms;
      e.bytes += p.bytes;
    }
    (void)cudaGetLastError();
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void retain_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  (void)cudaGetLastError();
}

int resident_blocks(const void *kernel, int block, size_t smem) {
  struct Key {
    int dev;
    const void *k;
    int block;
    size_t smem;
  };
  static std::mutex mu;
  static std::vector<std::pair<Key, int>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto &e : cache)
    if (e.first.dev == dev && e.first.k == kernel && e.first.block == block && e.first.smem == smem) return e.second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache.push_back({Key{dev, kernel, block, smem}, n});
  return n;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// ---------------------------------------------------------------- scans ----
// Three kernels: per-block sums, one-block scan of the block sums, per-block scan with
// the block's offset.  Each block covers kScanBlock * kScanItems inputs.
static constexpr int kScanBlock = 512;
static constexpr int kScanItems = 8;
static constexpr int kScanChunk = kScanBlock * kScanItems;

size_t scan_scratch_ints(long long n) { return (size_t)((n + kScanChunk - 1) / kScanChunk) + 2; }

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one int per thread; returns the exclusive prefix and the
// block total through *total.  blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
  __shared__ int warp_sums[33];  // [32] holds the block total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int s = lane < nw ? warp_sums[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) warp_sums[32] = si;
  }
  __syncthreads();
  int res = warp_sums[warp] + inc - v;
  *total = warp_sums[32];
  __syncthreads();
  return res;
}

__global__ void k_scan_reduce(const int *__restrict__ in, long long n, int *__restrict__ bsum) {
  long long base = (long long)blockIdx.x * kScanChunk;
  int s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long i = base + (long long)t * kScanBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  int total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block of 1024 threads scans nb block sums in place (exclusive); bsum[nb] = total.
__global__ void k_scan_top(int *bsum, int nb) {
  int carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    int total;
    int ex = block_excl_scan(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_down(const int *__restrict__ in, int *__restrict__ out, long long n,
                            const int *__restrict__ bsum, int nb) {
  long long base = (long long)blockIdx.x * kScanChunk;
  // each thread owns kScanItems consecutive inputs
  long long first = base + (long long)threadIdx.x * kScanItems;
  int vals[kScanItems];
  int s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long i = first + t;
    vals[t] = i < n ? in[i] : 0;
    s += vals[t];
  }
  int total;
  int ex = block_excl_scan(s, &total) + bsum[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long i = first + t;
    if (i < n) out[i] = ex;
    ex += vals[t];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = bsum[nb];
}

// Small inputs in one launch: one block of kScanOneThreads threads walks the input in
// chunks of kScanOneThreads * kScanOneItems (each thread a run of consecutive items),
// carrying the running total; out[n] = the total.  (The setup's small levels are bound
// by launch latency, where three launches per scan cost more than the scan.)
static constexpr int kScanOneThreads = 1024;
static constexpr int kScanOneItems = 16;
static constexpr long long kScanOneMax = 16384;  // one chunk: at 32K-64K the sequential chunks lost to three launches (measured)

// in and out may be the same array (each chunk is read before the block scan's barriers
// and written after them).
__global__ void __launch_bounds__(kScanOneThreads) k_scan_one(const int *in, int *out, int n) {
  int carry = 0;
  for (int base = 0; base < n; base += kScanOneThreads * kScanOneItems) {
    const int first = base + threadIdx.x * kScanOneItems;
    int vals[kScanOneItems];
    int sum = 0;
#pragma unroll
    for (int t = 0; t < kScanOneItems; ++t) {
      vals[t] = first + t < n ? in[first + t] : 0;
      sum += vals[t];
    }
    int total;
    int ex = carry + block_excl_scan(sum, &total);
#pragma unroll
    for (int t = 0; t < kScanOneItems; ++t) {
      if (first + t < n) out[first + t] = ex;
      ex += vals[t];
    }
    carry += total;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

amg_status exclusive_scan(const int *in, int *out, long long n, int *scratch, cudaStream_t s) {
  if (n <= 0) {
    CWM_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
    return AMG_OK;
  }
  if (n <= kScanOneMax) {
    k_scan_one<<<1, kScanOneThreads, 0, s>>>(in, out, (int)n);
    CWM_LAUNCH();
    return AMG_OK;
  }
  int nb = (int)((n + kScanChunk - 1) / kScanChunk);
  k_scan_reduce<<<nb, kScanBlock, 0, s>>>(in, n, scratch);
  CWM_LAUNCH();
  k_scan_top<<<1, 1024, 0, s>>>(scratch, nb);
  CWM_LAUNCH();
  k_scan_down<<<nb, kScanBlock, 0, s>>>(in, out, n, scratch, nb);
  CWM_LAUNCH();
  return AMG_OK;
}

}  // namespace cwm
