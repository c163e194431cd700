// Instantiates the fused product kernels for one kernel function.
#include "kmv_dispatch.cuh"

namespace krr {

cudaError_t launch_kmv32_gauss(int DP, int M, dim3 grid, cudaStream_t s, const Kmv32Args &a) {
  return launch_kmv32<KGAUSS>(DP, M, grid, s, a);
}

cudaError_t launch_kmv64_gauss(int DP, int M, dim3 grid, cudaStream_t s, const Kmv64Args &a) {
  return launch_kmv64<KGAUSS>(DP, M, grid, s, a);
}

}  // namespace krr
