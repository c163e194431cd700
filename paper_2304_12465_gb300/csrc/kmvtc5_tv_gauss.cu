// Instances of the tcgen05 product for the Gaussian kernel with the sums over
// the right-hand sides on the tensor cores (variants 8..11).
#include "kmvtc5_kernels.cuh"

namespace krr {

cudaError_t launch_kmvtc5_tv_gauss(int nh, int csep, int M, int variant, int G, size_t smem,
                                   cudaStream_t s, const CUtensorMap &rowmap,
                                   const CUtensorMap &colmap, const T5Args &a) {
  return launch_kmvtc5<KGAUSS, true>(nh, csep, M, variant, G, smem, s, rowmap, colmap, a);
}

}  // namespace krr
