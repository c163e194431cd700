// Instantiates the fused product kernels for one kernel function.
#include "kmv_dispatch.cuh"

namespace krr {

cudaError_t launch_kmv32_matern(int DP, int M, dim3 grid, cudaStream_t s, const Kmv32Args &a) {
  return launch_kmv32<KMATERN>(DP, M, grid, s, a);
}

cudaError_t launch_kmv64_matern(int DP, int M, dim3 grid, cudaStream_t s, const Kmv64Args &a) {
  return launch_kmv64<KMATERN>(DP, M, grid, s, a);
}

}  // namespace krr
