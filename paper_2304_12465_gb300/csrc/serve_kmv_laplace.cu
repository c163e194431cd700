// Grouped serving product, laplace kernel instantiations (serve_kmv.cuh).
#include "serve_kmv.cuh"

namespace krr {

cudaError_t serve_launch_product_laplace(int dp, int M, int items, const ServeTable *T,
                                   int cls, cudaStream_t s) {
  return serve_launch_product_k<KLAPLACE>(dp, M, items, T, cls, s);
}

}  // namespace krr
