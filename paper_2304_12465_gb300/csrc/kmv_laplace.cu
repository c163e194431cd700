// Instantiates the fused product kernels for one kernel function.
#include "kmv_dispatch.cuh"

namespace krr {

cudaError_t launch_kmv32_laplace(int DP, int M, dim3 grid, cudaStream_t s, const Kmv32Args &a) {
  return launch_kmv32<KLAPLACE>(DP, M, grid, s, a);
}

cudaError_t launch_kmv64_laplace(int DP, int M, dim3 grid, cudaStream_t s, const Kmv64Args &a) {
  return launch_kmv64<KLAPLACE>(DP, M, grid, s, a);
}

}  // namespace krr
