// Instances of the tcgen05 product for the Matern-5/2 kernel with the sums
// over the right-hand sides on the tensor cores (variants 8..11).
#include "kmvtc5_kernels.cuh"

namespace krr {

cudaError_t launch_kmvtc5_tv_matern(int nh, int csep, int M, int variant, int G, size_t smem,
                                    cudaStream_t s, const CUtensorMap &rowmap,
                                    const CUtensorMap &colmap, const T5Args &a) {
  return launch_kmvtc5<KMATERN, true>(nh, csep, M, variant, G, smem, s, rowmap, colmap, a);
}

}  // namespace krr
