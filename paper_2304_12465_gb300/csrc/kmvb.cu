// Host driver of the batched multi-setting fused product (kmvb_kernels.cuh).
#include "kmv.cuh"
#include "kmvb_kernels.cuh"

namespace krr {

template <int DP, int MS>
static cudaError_t launch_kmvb_dp_ms(bool l2, bool l1, bool r, dim3 grid, cudaStream_t s,
                                     const float *xt, const float *V, int64_t N, int64_t chunk,
                                     const KmvbSettings &st, float *part) {
#define KRR_KMVB(L2, L1, R)                                                                  \
  kmvb_kernel<DP, MS, L2, L1, R><<<grid, KMVB_THREADS, 0, s>>>(xt, V, N, chunk, st, part)
  if (l2 && l1 && r) KRR_KMVB(true, true, true);
  else if (l2 && l1) KRR_KMVB(true, true, false);
  else if (l2 && r) KRR_KMVB(true, false, true);
  else if (l2) KRR_KMVB(true, false, false);
  else KRR_KMVB(false, true, false);
#undef KRR_KMVB
  return cudaGetLastError();
}

template <int MS>
static cudaError_t launch_kmvb_ms(int dp, bool l2, bool l1, bool r, dim3 grid, cudaStream_t s,
                                  const float *xt, const float *V, int64_t N, int64_t chunk,
                                  const KmvbSettings &st, float *part) {
  switch (dp) {
    case 4: return launch_kmvb_dp_ms<4, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 8: return launch_kmvb_dp_ms<8, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 12: return launch_kmvb_dp_ms<12, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 16: return launch_kmvb_dp_ms<16, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 20: return launch_kmvb_dp_ms<20, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 24: return launch_kmvb_dp_ms<24, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 28: return launch_kmvb_dp_ms<28, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
    case 32: return launch_kmvb_dp_ms<32, MS>(l2, l1, r, grid, s, xt, V, N, chunk, st, part);
  }
  return cudaErrorInvalidValue;
}

// Y[s*ms + c] = lambda[s*ms + c] V[s*ms + c] + sum_splits part
__global__ void kmvb_reduce_kernel(const float *__restrict__ part, int splits, int MT,
                                   int64_t N, int mt, const float *__restrict__ lambda,
                                   const float *__restrict__ V, float *__restrict__ Y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int c = 0; c < mt; ++c) {
    float acc = 0.0f;
    for (int sp = 0; sp < splits; ++sp) acc += part[((int64_t)sp * MT + c) * N + i];
    Y[(int64_t)c * N + i] = acc + lambda[c] * V[(int64_t)c * N + i];
  }
}

krr_status kmvb_prepare(const double *Xd, int64_t N, int d, cudaStream_t s, PointsF32 &P) {
  // centred, unscaled points: every setting applies its own scale
  return prepare_points_f32(Xd, N, d, KLAPLACE, 1.4426950408889634, s, P);
}

krr_status kmv_batched_f32(const PointsF32 &P, int S, const int *kerns, const double *sigmas,
                           int ms, const float *lambda_dev, const float *V, float *Y,
                           cudaStream_t s, DevBuf<float> &part) {
  const int64_t N = P.N;
  if (N == 0 || S == 0) return KRR_OK;
  KmvbSettings st{};
  st.S = S;
  bool l2 = false, l1 = false, r = false;
  const double log2e = 1.4426950408889634;
  for (int q = 0; q < S; ++q) {
    st.type[q] = kerns[q];
    const double sg = sigmas[q];
    if (kerns[q] == KGAUSS) {
      st.g[q] = (float)(-log2e / (2.0 * sg * sg));
      l2 = true;
    } else if (kerns[q] == KLAPLACE) {
      st.g[q] = (float)(-log2e / sg);
      l1 = true;
    } else {
      st.g[q] = (float)(std::sqrt(5.0) / sg);
      l2 = true;
      r = true;
    }
  }
  const int MT = KMVB_MAX_SETTINGS * ms;
  const int rows = KMVB_THREADS * 2 * KMVB_RP;
  const int64_t row_tiles = (N + rows - 1) / rows;
  int64_t target = (int64_t)num_sms() * 3 * 8;
  int64_t splits = (target + row_tiles - 1) / row_tiles;
  const int64_t maxs = (N + KMVB_TJ - 1) / KMVB_TJ;
  if (splits > maxs) splits = maxs;
  if (splits < 1) splits = 1;
  int64_t chunk = (N + splits - 1) / splits;
  chunk = (chunk + KMVB_TJ - 1) / KMVB_TJ * KMVB_TJ;
  const int nsplit = (int)((N + chunk - 1) / chunk);
  const size_t need = (size_t)nsplit * MT * N;
  if (part.n < need) KRR_TRY(part.alloc(need, s));
  cudaError_t e;
  dim3 grid((unsigned)row_tiles, nsplit);
  switch (ms) {
    case 1: e = launch_kmvb_ms<1>(P.dp, l2, l1, r, grid, s, P.xt.p, V, N, chunk, st, part.p); break;
    case 2: e = launch_kmvb_ms<2>(P.dp, l2, l1, r, grid, s, P.xt.p, V, N, chunk, st, part.p); break;
    default: e = cudaErrorInvalidValue;
  }
  count_launch();
  if (e != cudaSuccess) {
    set_error("batched product launch failed: %s", cudaGetErrorString(e));
    return KRR_ECUDA;
  }
  kmvb_reduce_kernel<<<ceil_div(N, 256), 256, 0, s>>>(part.p, nsplit, MT, N, S * ms, lambda_dev,
                                                      V, Y);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

}  // namespace krr
