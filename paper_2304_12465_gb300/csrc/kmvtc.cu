// Host side of the tensor-core product (kmvtc_kernels.cuh): the half-split
// point layout and the launches, one instance per (kernel, coordinate
// blocks, padded m).
#include "kmv.cuh"
#include "kmvtc_kernels.cuh"

#include <cuda_fp16.h>

namespace krr {

__device__ __forceinline__ uint32_t pack_halves(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// One thread per point: centred, scaled coordinates split into h + l halves,
// stored in the fragment-group layout, and c = -|h + l|^2 / 2.  A coordinate
// outside the fp16-safe range sets *bad.
__global__ void prepare_tc_kernel(const double *__restrict__ X, int64_t N, int d, int kc_n,
                                  const double *__restrict__ mean, double scale,
                                  uint4 *__restrict__ xs, float *__restrict__ cs,
                                  int *__restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double nrm = 0.0;
  bool out_of_range = false;
  for (int kc = 0; kc < kc_n; ++kc) {
    for (int t = 0; t < 4; ++t) {
      const int ks[4] = {kc * 16 + 2 * t, kc * 16 + 2 * t + 1, kc * 16 + 2 * t + 8,
                         kc * 16 + 2 * t + 9};
      __half h[4], l[4];
      for (int q = 0; q < 4; ++q) {
        const int k = ks[q];
        const double v = (k < d) ? (X[i * d + k] - mean[k]) * scale : 0.0;
        if (!(fabs(v) <= (double)KTC_MAX_COORD)) out_of_range = true;
        h[q] = __float2half_rn((float)v);
        const double hv = (double)__half2float(h[q]);
        l[q] = __float2half_rn((float)(v - hv));
        const double e = hv + (double)__half2float(l[q]);
        nrm = fma(e, e, nrm);
      }
      uint4 w;
      w.x = pack_halves(h[0], h[1]);
      w.y = pack_halves(h[2], h[3]);
      w.z = pack_halves(l[0], l[1]);
      w.w = pack_halves(l[2], l[3]);
      xs[(i * kc_n + kc) * 4 + t] = w;
    }
  }
  cs[i] = (float)(-0.5 * nrm);
  if (out_of_range) *bad = 1;
}

krr_status prepare_points_tc(const double *Xd, cudaStream_t s, PointsF32 &P, bool with_tc5) {
  P.kc16 = 0;
  P.nh5 = 0;
  if (P.kern == KLAPLACE || P.d > 32 || P.N == 0) return KRR_OK;
  const int kc_n = (P.d + 15) / 16;
  const double log2e = 1.4426950408889634;
  const double scale = (P.kern == KGAUSS) ? std::sqrt(log2e) / P.sigma : std::sqrt(5.0) / P.sigma;
  KRR_TRY(P.xs16.alloc((size_t)P.N * kc_n * 4, s));
  KRR_TRY(P.cs16.alloc((size_t)P.N, s));
  DevBuf<int> bad;
  KRR_TRY(bad.alloc(1, s));
  KRR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  prepare_tc_kernel<<<ceil_div(P.N, 256), 256, 0, s>>>(Xd, P.N, P.d, kc_n, P.mean.p, scale,
                                                      P.xs16.p, P.cs16.p, bad.p);
  KRR_LAUNCH_CHECK();
  int h_bad = 0;
  KRR_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_bad) {
    // coordinates too large for the half split: keep the FMA product
    P.xs16.release();
    P.cs16.release();
    return KRR_OK;
  }
  P.kc16 = kc_n;
  if (with_tc5) {
    int bad5 = 0;
    KRR_TRY(prepare_points_tc5(Xd, s, P, &bad5));
  }
  return KRR_OK;
}

template <int KERN, int KC>
static cudaError_t launch_tc_m(int M, dim3 grid, cudaStream_t s, const KmvTcArgs &a) {
  switch (M) {
#define KRR_CASE(MM)                                                                        \
  case MM:                                                                                  \
    kmvtc_kernel<KERN, KC, MM><<<grid, KTC_THREADS, 0, s>>>(a.xs, a.cs, a.V, a.ldv, a.N, \
                                                              a.m, a.chunk, a.part);      \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_kmvtc(int kern, int KC, int M, dim3 grid, cudaStream_t s,
                         const KmvTcArgs &a) {
  if (kern == KGAUSS && KC == 1) return launch_tc_m<KGAUSS, 1>(M, grid, s, a);
  if (kern == KGAUSS && KC == 2) return launch_tc_m<KGAUSS, 2>(M, grid, s, a);
  if (kern == KMATERN && KC == 1) return launch_tc_m<KMATERN, 1>(M, grid, s, a);
  if (kern == KMATERN && KC == 2) return launch_tc_m<KMATERN, 2>(M, grid, s, a);
  return cudaErrorInvalidValue;
}

int kmvtc_rows_per_cta(int KC, int M) { return kmvtc_rows(KC, M); }

}  // namespace krr
