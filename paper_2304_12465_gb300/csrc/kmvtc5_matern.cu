// Instances of the tcgen05 product for the Matern-5/2 kernel.
#include "kmvtc5_kernels.cuh"

namespace krr {

cudaError_t launch_kmvtc5_matern(int nh, int csep, int M, int variant, int G, size_t smem,
                                cudaStream_t s,
                                 const CUtensorMap &rowmap, const CUtensorMap &colmap,
                                 const T5Args &a) {
  return launch_kmvtc5<KMATERN, false>(nh, csep, M, variant, G, smem, s, rowmap, colmap, a);
}

}  // namespace krr
