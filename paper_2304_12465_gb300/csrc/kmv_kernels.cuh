// Fused matrix-free product Y = (A + lambda I) V with A_ij = kappa(x_i, x_j)
// generated tile by tile in registers and never written to memory (the
// "Product" primitive of Alg. 1; the paper notes the kernel evaluations
// dominate its cost, Sec. 5.1).
//
// Work decomposition (both precisions): a CTA owns a block of rows and one
// column split; column points are staged through shared memory in tiles of
// KMV_TJ and broadcast to every thread, each thread keeps its rows' points
// and accumulators in registers.  Every (row block, split) pair writes its
// partial sums to part[split][c][row]; kmv_reduce adds the splits in a fixed
// order plus lambda V, so results are deterministic.
//
// float32 path: points are centred (stationary kernels are translation
// invariant) and pre-scaled so that
//   Gaussian : kappa = 2^(x_i.x_j + c_i + c_j),  x = (x - mean) sqrt(log2 e)/sigma,
//              c = -|x|^2/2
//   Matern   : acc = x_i.x_j + c_i + c_j = -q^2/2, x = (x - mean) sqrt(5)/sigma,
//              kappa = (1 + q + q^2/3) 2^(-q log2 e)
//   Laplace  : kappa = 2^(-sum_k |x_ik - x_jk|),  x = (x - mean) log2 e / sigma
// Pairs of rows are processed with packed float32x2 FMAs (FFMA2); column
// operands are stored duplicated ({v, v}) in shared memory so they feed the
// packed instructions directly.
#pragma once

#include "common.cuh"

namespace krr {

constexpr int KMV_THREADS = 256;
constexpr int KMV_TJ = 64;                        // columns per shared tile

// Rows per thread of the float32 kernel: four (two packed pairs) while the
// per-row registers (DP coordinates + M accumulators) fit two CTAs per SM,
// otherwise two.
__host__ __device__ constexpr int kmv32_rows_per_thread(int DP, int M) {
  return (DP + ((M + 1) / 2 * 2) <= 24) ? 4 : 2;
}

constexpr int KMV64_THREADS = 128;                // f64: one row per thread
constexpr int KMV64_TJ = 32;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KERN>
__device__ __forceinline__ float kappa_f32(float acc) {
  if constexpr (KERN == KMATERN) {
    const float q = sqrt_approx(fmaxf(-2.0f * acc, 0.0f));
    const float e = ex2_approx(-1.4426950408889634f * q);
    return fmaf(q, fmaf(q, 0.33333334f, 1.0f), 1.0f) * e;
  } else {
    return ex2_approx(acc);
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Shared memory of one float32 product tile: two column tiles of points
// (DP), right-hand sides (M rounded up to even) and per-point constants.
__host__ __device__ constexpr int kmv32_smem_bytes(int DP, int M) {
  return 2 * KMV_TJ * (DP + (M + 1) / 2 * 2 + 1) * (int)sizeof(float2);
}

// ------------------------------------------------------------------ f32
// xr, cr : Nr x DP, Nr  prepared row points and constants (the same arrays as
//          xt, cn for the square product; test points for prediction)
// xt : N x DP   prepared column points (zero padded beyond d)
// cn : N        per-point constant (c above; unused for Laplace)
// V  : m x ldv  right-hand sides (column c at V + c*ldv), float32
// part: splits x M x Nr partial products
// One (row tile, column split) work item of the float32 product; the
// single-problem kernel maps it from blockIdx, the grouped serving kernel
// from its work list.
template <int KERN, int DP, int M>
__device__ __forceinline__ void
kmv32_tile(const float *__restrict__ xr, const float *__restrict__ cr, int64_t Nr,
           const float *__restrict__ xt, const float *__restrict__ cn,
           const float *__restrict__ V, int64_t ldv, int64_t N, int m, int64_t chunk,
           float *__restrict__ part, int64_t row_tile, int64_t split,
           unsigned char *__restrict__ smem) {
  static_assert(DP % 4 == 0, "DP must be a multiple of 4");
  constexpr int RI = kmv32_rows_per_thread(DP, M);
  constexpr int RP = RI / 2;                      // row pairs per thread
  constexpr int MP = (M + 1) / 2 * 2;             // even number of columns
  constexpr int ROWS = KMV_THREADS * RI;          // rows per CTA
  // double-buffered column tiles, carved from the caller's shared buffer of
  // kmv32_smem_bytes(DP, M) bytes (16-byte aligned)
  auto sx = reinterpret_cast<float2 (*)[KMV_TJ][DP]>(smem);   // {x_jk, x_jk} (Laplace: -x_jk)
  auto sv = reinterpret_cast<float2 (*)[KMV_TJ][MP]>(smem + 2 * KMV_TJ * DP * sizeof(float2));
  auto sc = reinterpret_cast<float2 (*)[KMV_TJ]>(smem + 2 * KMV_TJ * (DP + MP) * sizeof(float2));

  const int tid = threadIdx.x;
  const int64_t row0 = row_tile * ROWS;
  const int64_t j_begin = split * chunk;
  const int64_t j_end = min(N, j_begin + chunk);

  // rows of this thread: row0 + tid + 256 r, paired (r = 2p, 2p + 1)
  float2 xi[RP][DP];
  float2 ci[RP];
  float2 acc[RP][MP];
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t ra = row0 + tid + (int64_t)(2 * p) * KMV_THREADS;
    const int64_t rb = ra + KMV_THREADS;
    const bool va = ra < Nr, vb = rb < Nr;
#pragma unroll
    for (int k = 0; k < DP; ++k)
      xi[p][k] = f2(va ? xr[ra * DP + k] : 0.0f, vb ? xr[rb * DP + k] : 0.0f);
    ci[p] = f2(va ? cr[ra] : 0.0f, vb ? cr[rb] : 0.0f);
#pragma unroll
    for (int c = 0; c < MP; ++c) acc[p][c] = f2(0.0f, 0.0f);
  }

  // register staging of the next tile
  constexpr int XE = KMV_TJ * DP;                 // x elements per tile
  constexpr int XPT = (XE + KMV_THREADS - 1) / KMV_THREADS;
  constexpr int VE = KMV_TJ * MP;
  constexpr int VPT = (VE + KMV_THREADS - 1) / KMV_THREADS;
  float rx[XPT], rv[VPT], rc = 0.0f;

  auto load_tile = [&](int64_t j0) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KMV_THREADS;
      float v = 0.0f;
      if (idx < XE) {
        const int64_t j = j0 + idx / DP;
        if (j < j_end) v = xt[j0 * DP + idx];
      }
      rx[e] = v;
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KMV_THREADS;
      float v = 0.0f;
      if (idx < VE) {
        const int c = idx / KMV_TJ;
        const int64_t j = j0 + idx % KMV_TJ;
        if (c < m && j < j_end) v = V[(int64_t)c * ldv + j];
      }
      rv[e] = v;
    }
    if (tid < KMV_TJ) {
      const int64_t j = j0 + tid;
      rc = (j < j_end) ? cn[j] : 0.0f;
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KMV_THREADS;
      if (idx < XE) {
        const float v = (KERN == KLAPLACE) ? -rx[e] : rx[e];
        sx[buf][idx / DP][idx % DP] = f2(v, v);
      }
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KMV_THREADS;
      if (idx < VE) sv[buf][idx % KMV_TJ][idx / KMV_TJ] = f2(rv[e], rv[e]);
    }
    if (tid < KMV_TJ) sc[buf][tid] = f2(rc, rc);
  };

  int buf = 0;
  if (j_begin < j_end) load_tile(j_begin);
  for (int64_t j0 = j_begin; j0 < j_end; j0 += KMV_TJ) {
    store_tile(buf);
    __syncthreads();
    if (j0 + KMV_TJ < j_end) load_tile(j0 + KMV_TJ);
    const int jn = (int)min((int64_t)KMV_TJ, j_end - j0);
#pragma unroll 1
    for (int jj = 0; jj < jn; ++jj) {
      float2 a[RP];
      if constexpr (KERN == KLAPLACE) {
#pragma unroll
        for (int p = 0; p < RP; ++p) a[p] = f2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < DP; k += 2) {
          const float4 q = *reinterpret_cast<const float4 *>(&sx[buf][jj][k]);
#pragma unroll
          for (int p = 0; p < RP; ++p) {
            const float2 d0 = __fadd2_rn(xi[p][k], f2(q.x, q.y));
            const float2 d1 = __fadd2_rn(xi[p][k + 1], f2(q.z, q.w));
            a[p].x = a[p].x - fabsf(d0.x) - fabsf(d1.x);
            a[p].y = a[p].y - fabsf(d0.y) - fabsf(d1.y);
          }
        }
      } else {
        const float2 cj = sc[buf][jj];
#pragma unroll
        for (int p = 0; p < RP; ++p) a[p] = __fadd2_rn(ci[p], cj);
#pragma unroll
        for (int k = 0; k < DP; k += 2) {
          const float4 q = *reinterpret_cast<const float4 *>(&sx[buf][jj][k]);
#pragma unroll
          for (int p = 0; p < RP; ++p) {
            a[p] = __ffma2_rn(xi[p][k], f2(q.x, q.y), a[p]);
            a[p] = __ffma2_rn(xi[p][k + 1], f2(q.z, q.w), a[p]);
          }
        }
      }
      float2 kk[RP];
#pragma unroll
      for (int p = 0; p < RP; ++p) kk[p] = f2(kappa_f32<KERN>(a[p].x), kappa_f32<KERN>(a[p].y));
#pragma unroll
      for (int c = 0; c < MP; c += 2) {
        const float4 q = *reinterpret_cast<const float4 *>(&sv[buf][jj][c]);
#pragma unroll
        for (int p = 0; p < RP; ++p) {
          acc[p][c] = __ffma2_rn(kk[p], f2(q.x, q.y), acc[p][c]);
          acc[p][c + 1] = __ffma2_rn(kk[p], f2(q.z, q.w), acc[p][c + 1]);
        }
      }
    }
    buf ^= 1;
  }

  float *out = part + split * M * Nr;
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    const int64_t ra = row0 + tid + (int64_t)(2 * p) * KMV_THREADS;
    const int64_t rb = ra + KMV_THREADS;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if (c < m) {
        if (ra < Nr) out[(int64_t)c * Nr + ra] = acc[p][c].x;
        if (rb < Nr) out[(int64_t)c * Nr + rb] = acc[p][c].y;
      }
    }
  }
}

template <int KERN, int DP, int M>
__global__ void __launch_bounds__(KMV_THREADS, 2)
kmv32_kernel(const float *__restrict__ xr, const float *__restrict__ cr, int64_t Nr,
             const float *__restrict__ xt, const float *__restrict__ cn,
             const float *__restrict__ V, int64_t ldv, int64_t N, int m,
             int64_t chunk, float *__restrict__ part) {
  __shared__ __align__(16) unsigned char smem[kmv32_smem_bytes(DP, M)];
  kmv32_tile<KERN, DP, M>(xr, cr, Nr, xt, cn, V, ldv, N, m, chunk, part, blockIdx.x,
                          blockIdx.y, smem);
}


// ------------------------------------------------------------------ f64
// Direct coordinate differences and the CUDA float64 exp, as in the
// definitions; X is N x d row-major float64, V m x ldv float64.
template <int KERN>
__device__ __forceinline__ double kappa_f64(double s, double inv_scale) {
  if constexpr (KERN == KLAPLACE) {
    return exp(-s * inv_scale);                    // inv_scale = 1/sigma
  } else if constexpr (KERN == KMATERN) {
    const double q = sqrt(5.0 * s) * inv_scale;    // inv_scale = 1/sigma
    return (1.0 + q + q * q / 3.0) * exp(-q);
  } else {
    return exp(-s * inv_scale);                    // inv_scale = 1/(2 sigma^2)
  }
}

// Xr (Nr x d) row points; X (N x d) column points; part: splits x M x Nr.
template <int KERN, int DP, int M>
__global__ void __launch_bounds__(KMV64_THREADS)
kmv64_kernel(const double *__restrict__ Xr, int64_t Nr, const double *__restrict__ X, int d,
             const double *__restrict__ V, int64_t ldv, int64_t N, int m, int64_t chunk,
             double inv_scale, double *__restrict__ part) {
  __shared__ double sx[KMV64_TJ][DP];
  __shared__ double sv[KMV64_TJ][M];
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * KMV64_THREADS + tid;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(N, j_begin + chunk);
  double xi[DP];
  double acc[M];
#pragma unroll
  for (int k = 0; k < DP; ++k) xi[k] = (i < Nr && k < d) ? Xr[i * d + k] : 0.0;
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0;

  for (int64_t j0 = j_begin; j0 < j_end; j0 += KMV64_TJ) {
    __syncthreads();
    for (int idx = tid; idx < KMV64_TJ * DP; idx += KMV64_THREADS) {
      const int jj = idx / DP, k = idx % DP;
      const int64_t j = j0 + jj;
      sx[jj][k] = (j < j_end && k < d) ? X[j * d + k] : 0.0;
    }
    for (int idx = tid; idx < KMV64_TJ * M; idx += KMV64_THREADS) {
      const int c = idx / KMV64_TJ, jj = idx % KMV64_TJ;
      const int64_t j = j0 + jj;
      sv[jj][c] = (j < j_end && c < m) ? V[(int64_t)c * ldv + j] : 0.0;
    }
    __syncthreads();
    const int jn = (int)min((int64_t)KMV64_TJ, j_end - j0);
#pragma unroll 1
    for (int jj = 0; jj < jn; ++jj) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        const double t = xi[k] - sx[jj][k];
        if constexpr (KERN == KLAPLACE) s += fabs(t);
        else s = fma(t, t, s);
      }
      const double kv = kappa_f64<KERN>(s, inv_scale);
#pragma unroll
      for (int c = 0; c < M; ++c) acc[c] = fma(kv, sv[jj][c], acc[c]);
    }
  }
  if (i < Nr) {
    double *out = part + (int64_t)blockIdx.y * M * Nr;
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < m) out[(int64_t)c * Nr + i] = acc[c];
  }
}

}  // namespace krr
