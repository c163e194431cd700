// Grouped fused product of the serving engine: one launch per product
// variant (kernel, padded dimension 4/8/16/32, padded m 1/2/4/8/16) present
// in a step covers the (row tile, column split) items of every slot of that
// variant, one CTA per item.  Each item runs the same tile code as the
// single-problem float32 product (kmv32_tile) with the slot's own
// decomposition, so the result of a slot does not depend on the other slots.
// (A single persistent launch over all variants was measured 18% slower: the
// variant switch and the per-item arguments held in registers cost spills.)
#pragma once

#include "kmv_kernels.cuh"
#include "serve.cuh"

namespace krr {

template <int KERN, int DP, int M>
__global__ void __launch_bounds__(KMV_THREADS, 2)
serve_product_kernel(const ServeTable *__restrict__ T, int cls) {
  __shared__ __align__(16) unsigned char smem[kmv32_smem_bytes(DP, M)];
  const ServeClass &C = T->cls[cls];
  const int item = blockIdx.x;
  if (item >= C.off[C.nslots]) return;
  const int j = serve_find_slot(C.off, C.nslots, item);
  const ServeSlotDesc &d = T->slot[C.slot[j]];
  if (!d.sc->live) return;
  const int local = item - C.off[j];
  kmv32_tile<KERN, DP, M>(d.xt, d.cn, d.N, d.xt, d.cn, d.p, d.N, d.N, d.m, d.chunk, d.part,
                          local % d.row_tiles, local / d.row_tiles, smem);
}

template <int KERN, int DP>
cudaError_t serve_launch_product_m(int M, int items, const ServeTable *T, int cls,
                                   cudaStream_t s) {
  switch (M) {
#define KRR_CASE(MM)                                                              \
  case MM:                                                                        \
    serve_product_kernel<KERN, DP, MM><<<items, KMV_THREADS, 0, s>>>(T, cls);     \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8) KRR_CASE(16)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KERN>
cudaError_t serve_launch_product_k(int dp, int M, int items, const ServeTable *T, int cls,
                                   cudaStream_t s) {
  switch (dp) {
    case 4: return serve_launch_product_m<KERN, 4>(M, items, T, cls, s);
    case 8: return serve_launch_product_m<KERN, 8>(M, items, T, cls, s);
    case 16: return serve_launch_product_m<KERN, 16>(M, items, T, cls, s);
    case 32: return serve_launch_product_m<KERN, 32>(M, items, T, cls, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace krr
