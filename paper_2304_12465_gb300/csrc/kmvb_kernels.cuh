// Batched fused product: several kernel settings (kernel type, bandwidth)
// over one point set share each tile's distance computation.
//
//   Y_s = (A_s + Lambda_s) V_s,  s = 0..S-1,
// A_s the kernel matrix of setting s, V_s its MS right-hand-side columns
// (typically one per regularisation value mu) and Lambda_s the per-column
// shifts.  Per pair (i, j) the coordinate differences of the centred points
// are formed once and give the squared l2 distance and/or the l1 distance
// (direct differences: no cancellation for clustered or duplicated points);
// each setting then costs one kernel evaluation (one or two MUFU operations)
// and MS FMAs.  Rows are processed in packed float32x2 pairs.
#pragma once

#include "kmv_kernels.cuh"

namespace krr {

constexpr int KMVB_MAX_SETTINGS = 8;
constexpr int KMVB_THREADS = 256;
constexpr int KMVB_TJ = 64;
constexpr int KMVB_RP = 1;   // row pairs per thread

struct KmvbSettings {
  int S;                          // number of settings
  int type[KMVB_MAX_SETTINGS];    // KGAUSS / KLAPLACE / KMATERN
  float g[KMVB_MAX_SETTINGS];     // Gaussian: -log2e/(2 sigma^2) (times r^2)
                                  // Laplace : -log2e/sigma       (times l1)
                                  // Matern  : sqrt(5)/sigma      (times r)
};

// xt: N x DP centred, unscaled points; V: (S*MS) x N columns;
// part: splits x (S*MS) x N.
// Three CTAs per SM (80 registers): the per-setting MUFU -> FMA chains need
// the extra warps to hide their latency (measured 1.27x over two CTAs).
template <int DP, int MS, bool NEED_L2, bool NEED_L1, bool NEED_R>
__global__ void __launch_bounds__(KMVB_THREADS, 3)
kmvb_kernel(const float *__restrict__ xt, const float *__restrict__ V, int64_t N,
            int64_t chunk, KmvbSettings st, float *__restrict__ part) {
  constexpr int MT = KMVB_MAX_SETTINGS * MS;
  constexpr int ROWS = KMVB_THREADS * 2 * KMVB_RP;
  __shared__ __align__(16) float2 sx[KMVB_TJ][DP];
  __shared__ __align__(16) float2 sv[KMVB_TJ][MT];
  const int S = st.S;
  const int mt = S * MS;
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(N, j_begin + chunk);

  float2 xi[KMVB_RP][DP];
  float2 acc[KMVB_RP][MT];
#pragma unroll
  for (int p = 0; p < KMVB_RP; ++p) {
    const int64_t ra = row0 + tid + (int64_t)(2 * p) * KMVB_THREADS;
    const int64_t rb = ra + KMVB_THREADS;
    const bool va = ra < N, vb = rb < N;
#pragma unroll
    for (int k = 0; k < DP; ++k)
      xi[p][k] = f2(va ? xt[ra * DP + k] : 0.0f, vb ? xt[rb * DP + k] : 0.0f);
#pragma unroll
    for (int c = 0; c < MT; ++c) acc[p][c] = f2(0.0f, 0.0f);
  }

  for (int64_t j0 = j_begin; j0 < j_end; j0 += KMVB_TJ) {
    __syncthreads();
    for (int idx = tid; idx < KMVB_TJ * DP; idx += KMVB_THREADS) {
      const int64_t j = j0 + idx / DP;
      const float v = (j < j_end) ? -xt[j0 * DP + idx] : 0.0f;
      sx[idx / DP][idx % DP] = f2(v, v);
    }
    for (int idx = tid; idx < KMVB_TJ * MT; idx += KMVB_THREADS) {
      const int c = idx / KMVB_TJ;
      const int64_t j = j0 + idx % KMVB_TJ;
      const float v = (c < mt && j < j_end) ? V[(int64_t)c * N + j] : 0.0f;
      sv[idx % KMVB_TJ][c] = f2(v, v);
    }
    __syncthreads();
    const int jn = (int)min((int64_t)KMVB_TJ, j_end - j0);
#pragma unroll 1
    for (int jj = 0; jj < jn; ++jj) {
#pragma unroll
      for (int p = 0; p < KMVB_RP; ++p) {
        float2 r2 = f2(0.0f, 0.0f), l1 = f2(0.0f, 0.0f), r = f2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < DP; ++k) {
          const float2 dd = __fadd2_rn(xi[p][k], sx[jj][k]);   // sx holds -x_j
          if constexpr (NEED_L2) r2 = __ffma2_rn(dd, dd, r2);
          if constexpr (NEED_L1) {
            l1.x += fabsf(dd.x);
            l1.y += fabsf(dd.y);
          }
        }
        if constexpr (NEED_R) r = f2(sqrt_approx(r2.x), sqrt_approx(r2.y));
#pragma unroll
        for (int s = 0; s < KMVB_MAX_SETTINGS; ++s) {
          if (s < S) {
            const float g = st.g[s];
            float2 kv;
            const int ty = st.type[s];
            if (ty == KGAUSS) {
              kv = f2(ex2_approx(r2.x * g), ex2_approx(r2.y * g));
            } else if (ty == KLAPLACE) {
              kv = f2(ex2_approx(l1.x * g), ex2_approx(l1.y * g));
            } else {
              const float2 q = __fmul2_rn(r, f2(g, g));
              const float2 e = f2(ex2_approx(-1.4426950408889634f * q.x),
                                  ex2_approx(-1.4426950408889634f * q.y));
              const float2 poly = __ffma2_rn(q, __ffma2_rn(q, f2(0.33333334f, 0.33333334f),
                                                            f2(1.0f, 1.0f)),
                                             f2(1.0f, 1.0f));
              kv = __fmul2_rn(poly, e);
            }
#pragma unroll
            for (int c = 0; c < MS; ++c)
              acc[p][s * MS + c] = __ffma2_rn(kv, sv[jj][s * MS + c], acc[p][s * MS + c]);
          }
        }
      }
    }
  }
  float *out = part + (int64_t)blockIdx.y * MT * N;
#pragma unroll
  for (int p = 0; p < KMVB_RP; ++p) {
    const int64_t ra = row0 + tid + (int64_t)(2 * p) * KMVB_THREADS;
    const int64_t rb = ra + KMVB_THREADS;
#pragma unroll
    for (int c = 0; c < MT; ++c) {
      if (c < mt) {
        if (ra < N) out[(int64_t)c * N + ra] = acc[p][c].x;
        if (rb < N) out[(int64_t)c * N + rb] = acc[p][c].y;
      }
    }
  }
}

}  // namespace krr
