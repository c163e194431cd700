// Grouped serving product, tensor-core variants: one launch per (kernel,
// coordinate blocks, padded m) present covers the (row tile, column split)
// items of every slot of that variant, one CTA per item, each running the
// single-problem tile code (kmvtc_tile) with the slot's own decomposition.
#include "kmvtc_kernels.cuh"
#include "serve.cuh"

namespace krr {

// A slot with m > 8 (M = 16) runs as two halves of 8 right-hand sides: item
// h * (row_tiles * splits) + r of the slot covers columns 8h .. 8h + 7 of its
// p, writing them into the slot's 16-column partial layout.
template <int KERN, int KC, int M>
__global__ void __launch_bounds__(KTC_THREADS, 1)
serve_product_tc_kernel(const ServeTable *__restrict__ T, int cls) {
  const ServeClass &C = T->cls[cls];
  const int item = blockIdx.x;
  if (item >= C.off[C.nslots]) return;
  const int j = serve_find_slot(C.off, C.nslots, item);
  const ServeSlotDesc &d = T->slot[C.slot[j]];
  if (!d.sc->live) return;
  const int local = item - C.off[j];
  const int per_half = d.row_tiles * d.splits;
  const int h = local / per_half, rem = local - h * per_half;
  const int mh = d.m - 8 * h < M ? d.m - 8 * h : M;
  kmvtc_tile<KERN, KC, M, kmvtc_frags(KC, M)>(
      d.xs, d.cs, d.p + (int64_t)8 * h * d.N, d.N, d.N, mh, d.chunk,
      d.part + (int64_t)8 * h * d.N, (int64_t)d.M * d.N, rem % d.row_tiles, rem / d.row_tiles);
}

template <int KERN, int KC>
static cudaError_t launch_m(int M, int items, const ServeTable *T, int cls, cudaStream_t s) {
  switch (M) {
#define KRR_CASE(MM)                                                                 \
  case MM:                                                                           \
    serve_product_tc_kernel<KERN, KC, MM><<<items, KTC_THREADS, 0, s>>>(T, cls);     \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8)
#undef KRR_CASE
    case 16:   // two halves of 8 right-hand sides
      serve_product_tc_kernel<KERN, KC, 8><<<items, KTC_THREADS, 0, s>>>(T, cls);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t serve_launch_product_tc(int kern, int kc, int M, int items, const ServeTable *T,
                                    int cls, cudaStream_t s) {
  if (kern == KGAUSS && kc == 1) return launch_m<KGAUSS, 1>(M, items, T, cls, s);
  if (kern == KGAUSS && kc == 2) return launch_m<KGAUSS, 2>(M, items, T, cls, s);
  if (kern == KMATERN && kc == 1) return launch_m<KMATERN, 1>(M, items, T, cls, s);
  if (kern == KMATERN && kc == 2) return launch_m<KMATERN, 2>(M, items, T, cls, s);
  return cudaErrorInvalidValue;
}

}  // namespace krr
