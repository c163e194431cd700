// Instantiates the float-float fused product for one kernel function.
#include "kmv_dispatch.cuh"

namespace krr {

cudaError_t launch_kmvff_gauss(int DP, int M, dim3 grid, cudaStream_t s, const KmvFFArgs &a) {
  return launch_kmvff<KGAUSS>(DP, M, grid, s, a);
}

cudaError_t launch_kmvffsym_gauss(int DP, int M, int G, cudaStream_t s,
                                  const KmvFFSymArgs &a) {
  return launch_kmvffsym<KGAUSS>(DP, M, G, s, a);
}

}  // namespace krr
