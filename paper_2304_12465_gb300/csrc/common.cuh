// Shared device/host helpers of the sm_103a library: status handling, device
// buffers, the Philox4x64-10 generator and reductions.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <cmath>
#include <vector>

#include "krr.h"

namespace krr {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

#define KRR_CUDA_TRY(expr)                                                      \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::krr::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                       __FILE__, __LINE__);                                     \
      return (e_ == cudaErrorMemoryAllocation) ? KRR_ENOMEM : KRR_ECUDA;        \
    }                                                                           \
  } while (0)

// Counts this library's kernel launches (reported by krr_launch_count).
void count_launch();
void count_launches(unsigned long long n);
// Off while this thread captures a CUDA graph: its launches are counted when
// the graph is launched.
void set_launch_counting(bool on);

// Capture log of a launch sequence recorded into a CUDA graph by this thread
// (the PCG iteration chunks).  While it is active, count_launch() counts into
// the log instead of the process total, and the fused-product timers of
// krr_set_profiling record external event nodes into it; capture_replayed()
// adds both to the process totals after each replay of the graph completed.
struct CaptureTimer {
  cudaEvent_t a, b;
  int tag;
};
struct CaptureLog {
  unsigned long long launches = 0;
  std::vector<CaptureTimer> timers;
  CaptureLog() = default;
  CaptureLog(const CaptureLog &) = delete;
  CaptureLog &operator=(const CaptureLog &) = delete;
  ~CaptureLog();
};
// Makes `log` this thread's active capture log (nullptr: none).
void capture_log_begin(CaptureLog *log);
// After a replay of the graph has completed (its stream synchronised).
void capture_replayed(const CaptureLog &log);

#define KRR_LAUNCH_CHECK()          \
  do {                              \
    ::krr::count_launch();          \
    KRR_CUDA_TRY(cudaGetLastError()); \
  } while (0)

#define KRR_TRY(expr)                                                           \
  do {                                                                          \
    krr_status s_ = (expr);                                                     \
    if (s_ != KRR_OK) return s_;                                                \
  } while (0)

#define KRR_REQUIRE(cond, ...)                                                  \
  do {                                                                          \
    if (!(cond)) {                                                              \
      ::krr::set_error(__VA_ARGS__);                                            \
      return KRR_EINVAL;                                                        \
    }                                                                           \
  } while (0)

// Raises a kernel's dynamic shared memory limit to at least `bytes` and never
// lowers it: host threads that run in parallel (the serving engine's
// builders) launch the same kernels with different sizes, and a lower limit
// set by one thread would make another thread's larger launch fail.
krr_status raise_smem_limit_ptr(const void *func, size_t bytes);
template <typename F>
krr_status raise_smem_limit(F *func, size_t bytes) {
  return raise_smem_limit_ptr((const void *)func, bytes);
}

// ------------------------------------------------------- device buffers
// Stream-ordered scratch owned by one call (cudaMallocAsync / cudaFreeAsync).
template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  krr_status alloc(size_t count, cudaStream_t stream) {
    release();
    s = stream;
    n = count;
    if (count == 0) return KRR_OK;
    KRR_CUDA_TRY(cudaMallocAsync((void **)&p, count * sizeof(T), stream));
    return KRR_OK;
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  T *get() const { return p; }
};

// Stream for the persistent allocations made by this host thread (null:
// plain cudaMalloc).  A thread that builds handles while other streams keep
// the device busy (the serving engine's builder) sets it, so that neither the
// allocations nor the later frees synchronise the device.
void set_alloc_stream(cudaStream_t s);
cudaStream_t alloc_stream();

// Persistent device memory owned by a handle.
template <typename T>
krr_status dev_alloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return KRR_OK;
  cudaStream_t s = alloc_stream();
  if (s) KRR_CUDA_TRY(cudaMallocAsync((void **)p, count * sizeof(T), s));
  else KRR_CUDA_TRY(cudaMalloc((void **)p, count * sizeof(T)));
  return KRR_OK;
}

// Frees handle memory: stream-ordered on free_stream when the handle was
// built with an allocation stream (the owner has already seen every use
// complete), otherwise cudaFree.
inline void dev_free(void *p, cudaStream_t free_stream) {
  if (!p) return;
  if (free_stream) cudaFreeAsync(p, free_stream);
  else cudaFree(p);
}

bool is_device_ptr(const void *p);

// Makes a device-resident view of a caller array of `count` elements: the
// original pointer if it is device memory, otherwise a stream-ordered copy.
template <typename T>
krr_status device_view(const T *src, size_t count, cudaStream_t s, DevBuf<T> &tmp,
                       const T **out) {
  if (src == nullptr || is_device_ptr(src)) {
    *out = src;
    return KRR_OK;
  }
  KRR_TRY(tmp.alloc(count, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(tmp.p, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = tmp.p;
  return KRR_OK;
}

// ------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of the
// Philox S-box on a 4 x 64-bit counter with a 2 x 64-bit key bumped by the
// Weyl constants between rounds.
struct Philox4x64 {
  static constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ULL;
  static constexpr uint64_t kMulB = 0xCA5A826395121157ULL;
  static constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ULL;
  static constexpr uint64_t kWeylB = 0xBB67AE8584CAA73BULL;
};

__host__ __device__ inline void mul_wide_u64(uint64_t a, uint64_t b, uint64_t &hi,
                                             uint64_t &lo) {
#ifdef __CUDA_ARCH__
  lo = a * b;
  hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  hi = (uint64_t)(p >> 64);
  lo = (uint64_t)p;
#endif
}

__host__ __device__ inline void philox4x64_10(const uint64_t ctr[4], uint64_t key0,
                                              uint64_t key1, uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t h0, l0, h1, l1;
    mul_wide_u64(Philox4x64::kMulA, c0, h0, l0);
    mul_wide_u64(Philox4x64::kMulB, c2, h1, l1);
    const uint64_t n0 = h1 ^ c1 ^ key0;
    const uint64_t n2 = h0 ^ c3 ^ key1;
    c0 = n0;
    c1 = l1;
    c2 = n2;
    c3 = l0;
    key0 += Philox4x64::kWeylA;
    key1 += Philox4x64::kWeylB;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// floor(u * range / 2^64): an unbiased-enough map of a 64-bit word to [0, range).
__host__ __device__ inline uint64_t scale_u64(uint64_t u, uint64_t range) {
  uint64_t hi, lo;
  mul_wide_u64(u, range, hi, lo);
  return hi;
}

constexpr uint64_t kTagPivots = 0x5250434850495653ULL;
constexpr uint64_t kTagEmbedRows = 0x53534531524f5753ULL;
constexpr uint64_t kTagEmbedSigns = 0x535345325349474eULL;

// ---------------------------------------------------------- reductions
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

int num_sms();

// Kernel function codes (mirror of krr_kernel).
enum { KGAUSS = 0, KLAPLACE = 1, KMATERN = 2 };

// Profiling hooks for the fused product (see krr_set_profiling).
bool profiling_on();
struct KmvTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  int tag = 0;               // 0: float32, 1: float64, 2: float-float product
  explicit KmvTimer(int t = 0) : tag(t) {}
  void begin(cudaStream_t s);
  void end(cudaStream_t s);
};
void kmv_profile_reset();
// Sums the recorded launches with the given tag (and forgets them).
void kmv_profile_collect(int tag, double *ms, int *launches);

}  // namespace krr
