// Grouped fused product of the serving engine: one persistent launch computes
// the (A + lambda I) p partial sums of every iterating slot.  A fixed grid of
// two CTAs per SM pulls (slot, row tile, column split) work items from a
// device counter; each item runs the same tile code as the single-problem
// float32 product (kmv32_tile), instantiated for every (kernel, padded
// dimension 4/8/16/32, padded m 1/2/4/8/16) combination, so slots of any
// shape share the launch.  The item order does not change any result: each
// item writes its own partial-sum block.
#include "kmv_kernels.cuh"
#include "serve.cuh"

namespace krr {

template <int KERN, int DP, int M>
__device__ __forceinline__ void serve_tile(const ServeSlotDesc &d, int64_t rt, int64_t sp,
                                           unsigned char *smem) {
  kmv32_tile<KERN, DP, M>(d.xt, d.cn, d.N, d.xt, d.cn, d.p, d.N, d.N, d.m, d.chunk, d.part,
                          rt, sp, smem);
}

__global__ void __launch_bounds__(KMV_THREADS, 2)
serve_product_kernel(const ServeTable *__restrict__ T, int *__restrict__ counter) {
  extern __shared__ __align__(16) unsigned char serve_smem[];
  __shared__ int s_item;
  const int n = T->nslots;
  const int total = T->prod_off[n];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    // also orders the previous tile's shared-memory reads before the next
    // tile's stores
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) break;
    const int s = serve_find_slot(T->prod_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int local = item - T->prod_off[s];
    const int64_t rt = local % d.row_tiles, sp = local / d.row_tiles;
    switch (d.variant) {
#define KRR_SERVE_M(K, DI, DPV)                                   \
  case ((K) * 4 + (DI)) * 5 + 0: serve_tile<K, DPV, 1>(d, rt, sp, serve_smem); break;  \
  case ((K) * 4 + (DI)) * 5 + 1: serve_tile<K, DPV, 2>(d, rt, sp, serve_smem); break;  \
  case ((K) * 4 + (DI)) * 5 + 2: serve_tile<K, DPV, 4>(d, rt, sp, serve_smem); break;  \
  case ((K) * 4 + (DI)) * 5 + 3: serve_tile<K, DPV, 8>(d, rt, sp, serve_smem); break;  \
  case ((K) * 4 + (DI)) * 5 + 4: serve_tile<K, DPV, 16>(d, rt, sp, serve_smem); break;
#define KRR_SERVE_K(K) \
  KRR_SERVE_M(K, 0, 4) KRR_SERVE_M(K, 1, 8) KRR_SERVE_M(K, 2, 16) KRR_SERVE_M(K, 3, 32)
      KRR_SERVE_K(KGAUSS)
      KRR_SERVE_K(KLAPLACE)
      KRR_SERVE_K(KMATERN)
#undef KRR_SERVE_K
#undef KRR_SERVE_M
      default:
        break;
    }
  }
}

int serve_prod_smem_bytes() { return kmv32_smem_bytes(32, 16); }

krr_status serve_configure_product() {
  KRR_CUDA_TRY(cudaFuncSetAttribute(serve_product_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    serve_prod_smem_bytes()));
  return KRR_OK;
}

krr_status serve_launch_product(const ServeTable *T, int *counter, cudaStream_t s) {
  serve_product_kernel<<<num_sms() * 2, KMV_THREADS, serve_prod_smem_bytes(), s>>>(T, counter);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

}  // namespace krr
