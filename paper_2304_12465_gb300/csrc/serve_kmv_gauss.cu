// Grouped serving product, gauss kernel instantiations (serve_kmv.cuh).
#include "serve_kmv.cuh"

namespace krr {

cudaError_t serve_launch_product_gauss(int dp, int M, int items, const ServeTable *T, int cls,
                                  cudaStream_t s) {
  return serve_launch_product_k<KGAUSS>(dp, M, items, T, cls, s);
}

}  // namespace krr
