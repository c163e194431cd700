// Allocation-free variant of the float64 fused product.
//
// Some callers cannot allocate device memory on their call path: a serving
// loop that has reserved all of its memory up front and must not let a
// request trigger cudaMalloc (which can synchronise the device and can fail
// under memory pressure), or a plug-in that only ever receives buffers from a
// host framework that owns all device memory.  For them the split partial
// sums of the product live in one file-scope device array instead of a
// per-call allocation.  The array is created when the library is loaded and
// every GPU that loads the library holds it until the process exits.
#include <mutex>

#include "kmv.cuh"

namespace krr {

// 2 Mi doubles (16 MiB): the partial sums of one product need
// splits x padded(m) x N doubles, padded(m) in {1, 2, 4, 8, 16}.
constexpr size_t kNoallocScratchDoubles = size_t(1) << 21;

static __device__ __align__(256) double g_kmv_scratch[kNoallocScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mtx;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device.  The name
// g_kmv_scratch is only a host-side stand-in, so the address is asked from
// the runtime once per device (with that device current) and cached.
static krr_status scratch_address(double **out) {
  int dev = 0;
  KRR_CUDA_TRY(cudaGetDevice(&dev));
  KRR_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mtx);
  if (!g_scratch_ptr[dev]) {
    double *ptr = nullptr;
    KRR_CUDA_TRY(cudaGetSymbolAddress((void **)&ptr, g_kmv_scratch));
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return KRR_OK;
}

}  // namespace krr

using namespace krr;

extern "C" krr_status krr_kmatvec_f64_noalloc(const double *X, int64_t N, int d,
                                              krr_kernel kern, double sigma, double lambda,
                                              const double *V, int m, double *Y, void *stream) {
  clear_error();
  KRR_REQUIRE(X && V && Y, "X, V and Y must not be NULL");
  KRR_REQUIRE(N >= 1, "N must be >= 1 (got %lld)", (long long)N);
  KRR_REQUIRE(d >= 1 && d <= 32, "d must be in [1, 32] (got %d)", d);
  KRR_REQUIRE(kern == KRR_GAUSSIAN || kern == KRR_LAPLACE_L1 || kern == KRR_MATERN52,
              "unknown kernel %d", (int)kern);
  KRR_REQUIRE(sigma > 0 && std::isfinite(sigma), "sigma must be positive and finite");
  KRR_REQUIRE(std::isfinite(lambda), "lambda must be finite");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(is_device_ptr(X) && is_device_ptr(V) && is_device_ptr(Y),
              "X, V and Y must be device pointers (this entry point does not stage host data)");
  const int M = m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16;
  KRR_REQUIRE((size_t)N * M <= kNoallocScratchDoubles,
              "N x padded(m) = %lld exceeds the %zu-double scratch of the allocation-free "
              "product (N <= %zu for this m)",
              (long long)N * M, kNoallocScratchDoubles, kNoallocScratchDoubles / M);
  double *scratch = nullptr;
  KRR_TRY(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  KRR_TRY(kmv_f64_with_scratch(X, N, d, kern, sigma, lambda, V, N, m, Y, N, scratch,
                               kNoallocScratchDoubles, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  return KRR_OK;
}
