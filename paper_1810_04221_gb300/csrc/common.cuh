// common.cuh -- shared host/device utilities of the CUDA path (errors, buffers, scans).
#pragma once

#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>

#include "cwm_amg.h"

namespace cwm {

namespace cg = cooperative_groups;

// Device-side error word bits (OR-ed by kernels, read by the host after a sync).
enum : int {
  kErrTimeout = 1,      // a bounded retry loop hit its cap
  kErrNotSpd = 2,       // missing or non-positive diagonal
  kErrInvalid = 4,      // malformed CSR, asymmetric A, aggregate with > 2 members
  kErrUnsupported = 8,  // a Galerkin row beyond the long-row capacity
  kErrBreakdown = 16,   // FCG rho <= 0 or not finite
};

// ---------------------------------------------------------------- errors ----
void set_error(const char *fmt, ...);
amg_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
amg_status status_from_device_bits(int bits, const char *where);

#define CWM_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::cwm::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define CWM_TRY(expr)                        \
  do {                                       \
    amg_status s_ = (expr);                  \
    if (s_ != AMG_OK) return s_;             \
  } while (0)

// ---------------------------------------------------- programmatic dependent launch ----
// The solve-phase kernels run back to back on one stream (and in the FCG iteration graphs).
// Launched with programmatic stream serialization, a kernel may be scheduled while its
// predecessor drains; it waits in pdl_begin() (griddepcontrol.wait: the predecessor has
// completed and its writes are visible) before touching any data, then lets its own
// successor be scheduled.  Without the launch attribute both instructions are no-ops.
// Only grids of at most one wave (kPdlMaxBlocksPerSm blocks per SM) take the attribute:
// the launch latency it hides matters on the small coarse levels; on multi-wave grids it
// measured neutral to slightly slower.
#ifndef CWM_PDL
#define CWM_PDL 1
#endif
__device__ __forceinline__ void pdl_begin() {
#if CWM_PDL
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
#endif
}

int num_sms();
constexpr int kPdlMaxBlocksPerSm = 8;
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed =
      CWM_PDL && (long long)grid.x * grid.y * grid.z <= (long long)num_sms() * kPdlMaxBlocksPerSm;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Blocks of `block` threads of a kernel that fit on one SM at once (occupancy API, cached
// per device and kernel).  A grid-stride kernel whose grid assumes more resident blocks
// than its registers allow runs a second, partly empty wave; wave_cap bounds its grid.
int resident_blocks(const void *kernel, int block, size_t smem);
template <class K>
inline int wave_cap(K kernel, int grid, int block, size_t smem = 0) {
  const int r = resident_blocks(reinterpret_cast<const void *>(kernel), block, smem);
  const int cap = r > 0 ? r * num_sms() : grid;
  return grid < cap ? grid : cap;
}

// Launch-error check after a kernel launch; also counts the library's kernel launches.
void count_launch();
#define CWM_LAUNCH()         \
  do {                       \
    ::cwm::count_launch();   \
    CWM_CUDA(cudaGetLastError()); \
  } while (0)
long long launch_count();
// Kernels launched by a replay of a captured graph (counted once per replay).
void count_launches(long long k);

// ---------------------------------------------------------------- tracing ----
// Optional per-kernel-class timing with CUDA events recorded on the launching stream
// around each launch, plus the algorithmic bytes each launch moves.  Active only while a
// handle's tracer is installed for the calling thread (see amg_trace_enable).
struct Tracer;
extern thread_local Tracer *g_tracer;
extern thread_local int g_trace_level;  // appended to category names as @k when >= 0
extern thread_local int g_trace_sweep;  // s >= 1: the (s+1)-th matching sweep of a level, @k.s
struct TraceScope {
  Tracer *t = nullptr;
  int idx = -1;
  cudaEvent_t a = nullptr;
  cudaStream_t s = nullptr;
  double bytes = 0.0;
  TraceScope(const char *cat, double bytes, cudaStream_t s);
  ~TraceScope();
};
#define CWM_TRACE(cat, bytes, stream) ::cwm::TraceScope cwm_trace_scope_((cat), (double)(bytes), (stream))

// ---------------------------------------------------------------- buffers ----
// When set (while a handle is destroyed), buffers are freed synchronously instead of on
// the stream they were allocated on, which the caller may have destroyed meanwhile.
extern thread_local bool g_sync_free;

// A stream-ordered device buffer (cudaMallocAsync / cudaFreeAsync).
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  amg_status alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return AMG_OK;
    cudaError_t e = cudaMallocAsync((void **)&p, count * sizeof(T), stream);
    if (e != cudaSuccess) {
      p = nullptr;
      n = 0;
      (void)cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return AMG_ERR_OOM;
    }
    return AMG_OK;
  }
  void release() {
    if (p) {
      if (g_sync_free) cudaFree(p);
      else cudaFreeAsync(p, s);
    }
    p = nullptr;
    n = 0;
  }
  T *get() const { return p; }
};

// Makes the device's default memory pool keep freed memory (repeated setups reuse it).
void retain_pool_memory();

// ---------------------------------------------------------------- host arrays ----
// Where a caller's pointer lives: device (or managed) memory, page-locked host memory
// (with its device alias), or pageable host memory.
enum class MemKind { kDevice, kPinned, kPageable };
MemKind mem_kind(const void *p, void **dev_alias);
// bytes from src (device, page-locked or pageable host) into device memory d_dst, and from
// device memory d_src out to dst, ordered on s; page-locked host memory is moved by an SM
// kernel through its device mapping, pageable memory by cudaMemcpyAsync (which waits).
amg_status copy_in(void *d_dst, const void *src, size_t bytes, cudaStream_t s);
amg_status copy_out(void *dst, const void *d_src, size_t bytes, cudaStream_t s);

// ---------------------------------------------------------------- launch ----
int num_sms();
// Grid for `items` work items of `per_block` items each, capped at `waves` full waves.
inline int grid_for(long long items, int per_block, int cap_blocks) {
  long long b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap_blocks) b = cap_blocks;
  return (int)b;
}
// Sub-warp ("miniwarp") width for rows of `mean` stored entries: 4, 8, 16 or 32.
// FP64 comparisons against zero on the integer pipes.  GB300 retires FP64 instructions --
// compares included -- at a small fraction of its other rates, so a compare inside a
// latency-bound loop waits for that pipe; these give the IEEE results exactly.
//   pos_f64(x)     == (x > 0.0): positive sign bit clear, not +0.0, not NaN (+inf counts)
//   nonzero_f64(x) == (x != 0.0): any bits other than the sign bit (NaN counts)
__device__ __forceinline__ bool pos_f64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0ll && b <= 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool nonzero_f64(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}

inline int tile_for_mean(double mean) {
  if (mean <= 4.5) return 4;
  if (mean <= 9.0) return 8;
  if (mean <= 18.0) return 16;
  return 32;
}

// Sub-warp width for the solve kernels of a level: wide enough for the mean row, and for
// the longest row to take at most CWM_TILE_MAX_PER_LANE entries per lane (a long row on
// few lanes is a chain of gathers that sets the time of a small level; 32 measured best
// against 8 and 16, the row dot keeping four gathers per lane in flight).
#ifndef CWM_TILE_MAX_PER_LANE
#define CWM_TILE_MAX_PER_LANE 32
#endif
// The tile also gives each lane about CWM_TILE32_MEAN_PER_LANE entries of the mean row: the
// row walk keeps a predicated group of four per lane in flight, so narrower tiles put more
// rows in flight per warp.  Measured (binary32 cycles): 5 against ~1 (the earlier 4.5 /
// 9 / 18 steps) took Q1 elasticity 64^3 59.5 -> 58.9 ms (level-1 residual 49.3 -> 43.1 us,
// level-2 A P sweep 18.4 -> 14.3 us), lognormal 160^3 42.9 -> 41.4 ms, 3D Poisson 128^3
// 15.7 -> 15.4 ms; 2.5 gained half as much.
#ifndef CWM_TILE32_MEAN_PER_LANE
#define CWM_TILE32_MEAN_PER_LANE 5.0
#endif
inline int tile_for_rows(double mean, int max_row) {
  const int e = CWM_TILE_MAX_PER_LANE;
  const int t_max = max_row <= 4 * e ? 4 : max_row <= 8 * e ? 8 : max_row <= 16 * e ? 16 : 32;
  int t_mean = 4;
  while (t_mean < 32 && mean > CWM_TILE32_MEAN_PER_LANE * t_mean) t_mean <<= 1;
  return t_max > t_mean ? t_max : t_mean;
}

// ---------------------------------------------------------------- scans ----
// out[0..n] = exclusive prefix sums of in[0..n) with out[n] = total (int32; the total
// must fit).  scratch: at least scan_scratch_ints(n) ints.
size_t scan_scratch_ints(long long n);
amg_status exclusive_scan(const int *in, int *out, long long n, int *scratch, cudaStream_t s);

}  // namespace cwm
