// KRILL (Alg. 2, Sec. 2.2.1) on the device.
//
// Build: H = lambda A(S,S) + N eps tr(A(S,S)) I; sparse sign embedding Phi
// (s x N, zeta nonzeros per column) from Philox; Phi transposed into per-row
// lists by a counting sort with a fixed within-row order; the
// sketch B = Phi A(:,S) gathered row by row with kernel entries regenerated
// in float32; P = B^T B + H and its Cholesky factor in float64.
// Solve: iterative refinement -- the right-hand side A(S,:) y and the outer
// residuals use float64-accurate kernel entries (float-float arithmetic on the
// float32 pipes); the inner PCG on k-vectors (float64)
// uses a product that regenerates the N x k block A(:,S) twice per
// application in float32 (u = A(:,S) beta, then A(S,:) u), with the
// preconditioner W^T W, W = L^{-1}, P = L L^T.
#include <chrono>

#include "dense.cuh"
#include "handles.cuh"
#include "kmv.cuh"
#include "kmv_kernels.cuh"
#include "krill.cuh"
#include "pcg.cuh"

namespace krr {

// ------------------------------------------------------ sparse sign
__global__ void sparse_sign_kernel(int64_t N, int s, int zeta, uint64_t seed,
                                   int32_t *__restrict__ rows, float *__restrict__ vals32,
                                   double *__restrict__ vals64) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int32_t kept[64];
  int nk = 0;
  for (uint64_t q = 0; nk < zeta; ++q) {
    uint64_t ctr[4] = {(uint64_t)n, q, 0ull, 0ull}, out[4];
    philox4x64_10(ctr, seed, kTagEmbedRows, out);
    for (int w = 0; w < 4 && nk < zeta; ++w) {
      const int32_t r = (int32_t)scale_u64(out[w], (uint64_t)s);
      bool dup = false;
      for (int t = 0; t < nk; ++t) dup = dup || (kept[t] == r);
      if (!dup) kept[nk++] = r;
    }
  }
  uint64_t ctr[4] = {(uint64_t)n, 0ull, 0ull, 0ull}, out[4];
  philox4x64_10(ctr, seed, kTagEmbedSigns, out);
  const double scale = 1.0 / sqrt((double)zeta);
  for (int t = 0; t < zeta; ++t) {
    rows[n * zeta + t] = kept[t];
    const double v = ((out[0] >> t) & 1ull) ? -scale : scale;
    if (vals32) vals32[n * zeta + t] = (float)v;
    if (vals64) vals64[n * zeta + t] = v;
  }
}

krr_status sparse_sign_device(int64_t N, int s, int zeta, uint64_t seed, int32_t *rows,
                              float *vals32, double *vals64, cudaStream_t st) {
  if (N == 0) return KRR_OK;
  sparse_sign_kernel<<<ceil_div(N, 128), 128, 0, st>>>(N, s, zeta, seed, rows, vals32, vals64);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ------------------------------------------- stable transpose to rows
constexpr int TR_CHUNK = 1024;

__global__ void row_hist_kernel(const int32_t *__restrict__ rows, int64_t N, int zeta, int s,
                                int *__restrict__ hist) {
  extern __shared__ int sh[];
  for (int r = threadIdx.x; r < s; r += blockDim.x) sh[r] = 0;
  __syncthreads();
  const int64_t n0 = (int64_t)blockIdx.x * TR_CHUNK;
  const int64_t n1 = min(N, n0 + TR_CHUNK);
  for (int64_t e = n0 * zeta + threadIdx.x; e < n1 * zeta; e += blockDim.x)
    atomicAdd(&sh[rows[e]], 1);
  __syncthreads();
  for (int r = threadIdx.x; r < s; r += blockDim.x) hist[(int64_t)blockIdx.x * s + r] = sh[r];
}

// total[r] = sum over chunks
__global__ void row_total_kernel(const int *__restrict__ hist, int nch, int s,
                                 int64_t *__restrict__ total) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  int64_t t = 0;
  for (int c = 0; c < nch; ++c) t += hist[(int64_t)c * s + r];
  total[r] = t;
}

// rowptr[r] = exclusive prefix of total (single block, sequential chunks)
__global__ void row_scan_kernel(const int64_t *__restrict__ total, int s,
                                int64_t *__restrict__ rowptr) {
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int r = 0; r < s; ++r) {
      rowptr[r] = run;
      run += total[r];
    }
    rowptr[s] = run;
  }
}

// off[c][r] = rowptr[r] + sum_{c' < c} hist[c'][r]
__global__ void row_offsets_kernel(const int *__restrict__ hist, int nch, int s,
                                   const int64_t *__restrict__ rowptr,
                                   int64_t *__restrict__ off) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  int64_t run = rowptr[r];
  for (int c = 0; c < nch; ++c) {
    off[(int64_t)c * s + r] = run;
    run += hist[(int64_t)c * s + r];
  }
}

// One warp per chunk: groups of 32 consecutive points, one slot t at a time;
// lanes that hit the same row are ranked by lane (__match_any_sync), so the
// order inside each row list is fixed: (point group, slot, lane).
__global__ void __launch_bounds__(32)
row_fill_kernel(const int32_t *__restrict__ rows, const float *__restrict__ vals, int64_t N,
                int zeta, int s, const int64_t *__restrict__ off,
                int32_t *__restrict__ col_n, float *__restrict__ col_v) {
  extern __shared__ int64_t so[];
  const int c = blockIdx.x;
  const int lane = threadIdx.x;
  for (int r = lane; r < s; r += 32) so[r] = off[(int64_t)c * s + r];
  __syncwarp();
  const int64_t n0 = (int64_t)c * TR_CHUNK;
  const int64_t n1 = min(N, n0 + TR_CHUNK);
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t g = n0; g < n1; g += 32) {
    const int64_t n = g + lane;
    const bool valid = n < n1;
    for (int t = 0; t < zeta; ++t) {
      const int32_t r = valid ? rows[n * zeta + t] : -1 - lane;
      const unsigned same = __match_any_sync(0xffffffffu, r);
      const int rank = __popc(same & lt);
      if (valid) {
        const int64_t pos = so[r] + rank;
        col_n[pos] = (int32_t)n;
        col_v[pos] = vals[n * zeta + t];
      }
      __syncwarp();
      if (valid && rank == 0) so[r] += __popc(same);
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------ sketch
// Bsk[r + c s] (float32 accumulation, float64 output) = sum over the list of
// row r of v * kappa(x_n, x_{S_c}).  CTA: one sketch row x 256 centers.
template <int KERN, int DP>
__global__ void __launch_bounds__(256)
sketch_kernel(const float *__restrict__ xt, const float *__restrict__ cn,
              const int64_t *__restrict__ S, int k, const int64_t *__restrict__ rowptr,
              const int32_t *__restrict__ col_n, const float *__restrict__ col_v, int s,
              double *__restrict__ Bsk) {
  constexpr int TE = 64;
  __shared__ float sx[TE][DP];
  __shared__ float sc[TE];
  __shared__ float sv[TE];
  const int r = blockIdx.x;
  const int c = blockIdx.y * 256 + threadIdx.x;
  float xc[DP];
  float cc = 0.0f;
  if (c < k) {
    const int64_t p = S[c];
#pragma unroll
    for (int q = 0; q < DP; ++q) xc[q] = xt[p * DP + q];
    cc = cn[p];
  } else {
#pragma unroll
    for (int q = 0; q < DP; ++q) xc[q] = 0.0f;
  }
  const int64_t e0 = rowptr[r], e1 = rowptr[r + 1];
  double acc64 = 0.0;
  for (int64_t b = e0; b < e1; b += TE) {
    const int ne = (int)min((int64_t)TE, e1 - b);
    __syncthreads();
    for (int idx = threadIdx.x; idx < TE * DP; idx += 256) {
      const int e = idx / DP, q = idx % DP;
      sx[e][q] = (e < ne) ? xt[(int64_t)col_n[b + e] * DP + q] : 0.0f;
    }
    if (threadIdx.x < TE) {
      const int e = threadIdx.x;
      sc[e] = (e < ne) ? cn[col_n[b + e]] : 0.0f;
      sv[e] = (e < ne) ? col_v[b + e] : 0.0f;
    }
    __syncthreads();
    float acc = 0.0f;
    for (int e = 0; e < ne; ++e) {
      float a;
      if constexpr (KERN == KLAPLACE) {
        a = 0.0f;
#pragma unroll
        for (int q = 0; q < DP; ++q) a -= fabsf(xc[q] - sx[e][q]);
      } else {
        a = cc + sc[e];
#pragma unroll
        for (int q = 0; q < DP; ++q) a = fmaf(xc[q], sx[e][q], a);
      }
      acc = fmaf(sv[e], kappa_f32<KERN>(a), acc);
    }
    acc64 += (double)acc;
  }
  if (c < k) Bsk[(int64_t)r + (int64_t)c * s] = acc64;
}

// ------------------------------------------------------- H = lam A(S,S) + ...
__global__ void kss_kernel(const double *__restrict__ X, int d, int kern, double sigma,
                           const int64_t *__restrict__ S, int k, double *__restrict__ H) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int i = (int)(e % k), j = (int)(e / k);
  H[e] = kappa_point_f64(X + S[i] * d, X + S[j] * d, d, kern, sigma);
}

__global__ void h_finish_kernel(double *__restrict__ H, int k, double lambda, double shift_scale) {
  // trace by one block, then H = lambda A + shift I
  __shared__ double red[32];
  __shared__ double tr;
  double t = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) t += H[i + (int64_t)i * k];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    tr = s;
  }
  __syncthreads();
  const double shift = shift_scale * tr;
  for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    H[e] = lambda * H[e] + ((i == j) ? shift : 0.0);
  }
}

// ---------------------------------------------------- block products
// u[c][n] = sum_l kappa(x_n, x_{S_l}) beta[c][l]   (float32 entries)
template <int KERN, int DP, int M>
__global__ void __launch_bounds__(256)
kcols_kernel(const float *__restrict__ xt, const float *__restrict__ cn, int64_t N,
             const int64_t *__restrict__ S, int k, const double *__restrict__ beta, int m,
             float *__restrict__ u) {
  constexpr int TL = 128;
  __shared__ float sx[TL][DP];
  __shared__ float sc[TL];
  __shared__ float sb[TL][M];
  const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
  float xn[DP];
  float cnn = 0.0f;
#pragma unroll
  for (int q = 0; q < DP; ++q) xn[q] = (n < N) ? xt[n * DP + q] : 0.0f;
  if (n < N) cnn = cn[n];
  float acc[M];
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0f;
  for (int l0 = 0; l0 < k; l0 += TL) {
    const int nl = min(TL, k - l0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < TL * DP; idx += 256) {
      const int l = idx / DP, q = idx % DP;
      sx[l][q] = (l < nl) ? xt[S[l0 + l] * DP + q] : 0.0f;
    }
    for (int idx = threadIdx.x; idx < TL * M; idx += 256) {
      const int l = idx / M, c = idx % M;
      sb[l][c] = (l < nl && c < m) ? (float)beta[(int64_t)c * k + l0 + l] : 0.0f;
    }
    if (threadIdx.x < TL) sc[threadIdx.x] = (threadIdx.x < nl) ? cn[S[l0 + threadIdx.x]] : 0.0f;
    __syncthreads();
    for (int l = 0; l < nl; ++l) {
      float a;
      if constexpr (KERN == KLAPLACE) {
        a = 0.0f;
#pragma unroll
        for (int q = 0; q < DP; ++q) a -= fabsf(xn[q] - sx[l][q]);
      } else {
        a = cnn + sc[l];
#pragma unroll
        for (int q = 0; q < DP; ++q) a = fmaf(xn[q], sx[l][q], a);
      }
      const float kv = kappa_f32<KERN>(a);
#pragma unroll
      for (int c = 0; c < M; ++c) acc[c] = fmaf(kv, sb[l][c], acc[c]);
    }
  }
  if (n < N)
    for (int c = 0; c < m; ++c) u[(int64_t)c * N + n] = acc[c];
}

// part[ch][c][l] = sum_{n in chunk ch} kappa(x_{S_l}, x_n) u[c][n]
constexpr int KR_CHUNK = 2048;
template <int KERN, int DP, int M>
__global__ void __launch_bounds__(256)
krows_kernel(const float *__restrict__ xt, const float *__restrict__ cn, int64_t N,
             const int64_t *__restrict__ S, int k, const float *__restrict__ u, int m,
             double *__restrict__ part) {
  constexpr int TN = 128;
  __shared__ float sx[TN][DP];
  __shared__ float sc[TN];
  __shared__ float su[TN][M];
  const int l = blockIdx.y * 256 + threadIdx.x;
  const int64_t n_begin = (int64_t)blockIdx.x * KR_CHUNK;
  const int64_t n_end = min(N, n_begin + KR_CHUNK);
  float xl[DP];
  float cl = 0.0f;
#pragma unroll
  for (int q = 0; q < DP; ++q) xl[q] = (l < k) ? xt[S[l] * DP + q] : 0.0f;
  if (l < k) cl = cn[S[l]];
  float acc[M];
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0f;
  for (int64_t n0 = n_begin; n0 < n_end; n0 += TN) {
    const int nn = (int)min((int64_t)TN, n_end - n0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < TN * DP; idx += 256) {
      const int e = idx / DP, q = idx % DP;
      sx[e][q] = (e < nn) ? xt[(n0 + e) * DP + q] : 0.0f;
    }
    for (int idx = threadIdx.x; idx < TN * M; idx += 256) {
      const int e = idx % TN, c = idx / TN;
      su[e][c] = (e < nn && c < m) ? u[(int64_t)c * N + n0 + e] : 0.0f;
    }
    if (threadIdx.x < TN) sc[threadIdx.x] = (threadIdx.x < nn) ? cn[n0 + threadIdx.x] : 0.0f;
    __syncthreads();
    for (int e = 0; e < nn; ++e) {
      float a;
      if constexpr (KERN == KLAPLACE) {
        a = 0.0f;
#pragma unroll
        for (int q = 0; q < DP; ++q) a -= fabsf(xl[q] - sx[e][q]);
      } else {
        a = cl + sc[e];
#pragma unroll
        for (int q = 0; q < DP; ++q) a = fmaf(xl[q], sx[e][q], a);
      }
      const float kv = kappa_f32<KERN>(a);
#pragma unroll
      for (int c = 0; c < M; ++c) acc[c] = fmaf(kv, su[e][c], acc[c]);
    }
  }
  if (l < k)
    for (int c = 0; c < m; ++c) part[((int64_t)blockIdx.x * m + c) * k + l] = (double)acc[c];
}

__global__ void krows_reduce_kernel(const double *__restrict__ part, int nch, int k, int m,
                                    double *__restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * m) return;
  double acc = 0.0;
  for (int c = 0; c < nch; ++c) acc += part[(int64_t)c * k * m + e];
  out[e] = acc;
}

// y[c][i] = H[i, :] beta[c] + add[c][i]   (H symmetric, one warp per row)
__global__ void sym_gemv_add_kernel(const double *__restrict__ H, int k,
                                    const double *__restrict__ beta, int m,
                                    const double *__restrict__ add, double *__restrict__ y) {
  const int warps = blockDim.x >> 5;
  const int i = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= k) return;
  const double *col = H + (int64_t)i * k;
  for (int c = 0; c < m; ++c) {
    double acc = 0.0;
    for (int j = lane; j < k; j += 32) acc = fma(col[j], beta[(int64_t)c * k + j], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[(int64_t)c * k + i] = acc + add[(int64_t)c * k + i];
  }
}

// ---------------------------------------------------- dispatch helpers
#define KRR_DP_SWITCH(DPV, ...)                         \
  switch (DPV) {                                        \
    case 4: { constexpr int DP = 4; __VA_ARGS__; break; } \
    case 8: { constexpr int DP = 8; __VA_ARGS__; break; } \
    case 12: { constexpr int DP = 12; __VA_ARGS__; break; } \
    case 16: { constexpr int DP = 16; __VA_ARGS__; break; } \
    case 20: { constexpr int DP = 20; __VA_ARGS__; break; } \
    case 24: { constexpr int DP = 24; __VA_ARGS__; break; } \
    case 28: { constexpr int DP = 28; __VA_ARGS__; break; } \
    case 32: { constexpr int DP = 32; __VA_ARGS__; break; } \
    default: return KRR_EINVAL;                         \
  }

#define KRR_KERN_SWITCH(KV, ...)                                      \
  switch (KV) {                                                       \
    case KGAUSS: { constexpr int KERN = KGAUSS; __VA_ARGS__; break; }   \
    case KLAPLACE: { constexpr int KERN = KLAPLACE; __VA_ARGS__; break; } \
    case KMATERN: { constexpr int KERN = KMATERN; __VA_ARGS__; break; } \
    default: return KRR_EINVAL;                                       \
  }

#define KRR_M_SWITCH(MV, ...)                            \
  switch (MV) {                                          \
    case 1: { constexpr int M = 1; __VA_ARGS__; break; }   \
    case 2: { constexpr int M = 2; __VA_ARGS__; break; }   \
    case 4: { constexpr int M = 4; __VA_ARGS__; break; }   \
    default: { constexpr int M = 16; __VA_ARGS__; break; } \
  }

static int pad_m_krill(int m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : 16; }

krr_status krill_kcols(const krill_precond *P, const double *beta, int m, float *u,
                       cudaStream_t s) {
  const int M = pad_m_krill(m);
  KRR_KERN_SWITCH(P->kern, KRR_DP_SWITCH(P->dp, KRR_M_SWITCH(M, {
    kcols_kernel<KERN, DP, M><<<ceil_div(P->N, 256), 256, 0, s>>>(P->xt, P->cn, P->N, P->S,
                                                                  P->k, beta, m, u);
  })));
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status krill_krows(const krill_precond *P, const float *u, int m, double *out,
                       cudaStream_t s) {
  const int M = pad_m_krill(m);
  const int nch = ceil_div(P->N, KR_CHUNK);
  DevBuf<double> part;
  KRR_TRY(part.alloc((size_t)nch * P->k * m, s));
  dim3 grid(nch, ceil_div(P->k, 256));
  KRR_KERN_SWITCH(P->kern, KRR_DP_SWITCH(P->dp, KRR_M_SWITCH(M, {
    krows_kernel<KERN, DP, M><<<grid, 256, 0, s>>>(P->xt, P->cn, P->N, P->S, P->k, u, m,
                                                   part.p);
  })));
  KRR_LAUNCH_CHECK();
  krows_reduce_kernel<<<ceil_div((int64_t)P->k * m, 256), 256, 0, s>>>(part.p, nch, P->k, m,
                                                                     out);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ------------------------------------------------------------- build
krr_status krill_build_device(krill_precond *P, cudaStream_t s) {
  auto t0 = std::chrono::steady_clock::now();
  const int64_t N = P->N;
  const int k = P->k, sr = P->s, zeta = P->zeta;
  // prepared float32 points (shared with the product kernels)
  {
    PointsF32 pts;
    KRR_TRY(prepare_points_f32(P->X, N, P->d, P->kern, P->sigma, s, pts));
    P->dp = pts.dp;
    KRR_TRY(dev_alloc(&P->xt, (size_t)N * pts.dp));
    KRR_TRY(dev_alloc(&P->cn, (size_t)N));
    KRR_CUDA_TRY(cudaMemcpyAsync(P->xt, pts.xt.p, sizeof(float) * N * pts.dp,
                                 cudaMemcpyDeviceToDevice, s));
    KRR_CUDA_TRY(cudaMemcpyAsync(P->cn, pts.cn.p, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
  }
  // H
  KRR_TRY(dev_alloc(&P->H, (size_t)k * k));
  kss_kernel<<<ceil_div((int64_t)k * k, 256), 256, 0, s>>>(P->X, P->d, P->kern, P->sigma, P->S,
                                                          k, P->H);
  KRR_LAUNCH_CHECK();
  h_finish_kernel<<<1, 1024, 0, s>>>(P->H, k, P->lambda, (double)N * 2.220446049250313e-16);
  KRR_LAUNCH_CHECK();
  // Phi and its row lists
  DevBuf<int32_t> rows, col_n;
  DevBuf<float> vals, col_v;
  KRR_TRY(rows.alloc((size_t)N * zeta, s));
  KRR_TRY(vals.alloc((size_t)N * zeta, s));
  KRR_TRY(col_n.alloc((size_t)N * zeta, s));
  KRR_TRY(col_v.alloc((size_t)N * zeta, s));
  KRR_TRY(sparse_sign_device(N, sr, zeta, P->seed, rows.p, vals.p, nullptr, s));
  const int nch = ceil_div(N, TR_CHUNK);
  DevBuf<int> hist;
  DevBuf<int64_t> total, rowptr, off;
  KRR_TRY(hist.alloc((size_t)nch * sr, s));
  KRR_TRY(total.alloc(sr, s));
  KRR_TRY(rowptr.alloc(sr + 1, s));
  KRR_TRY(off.alloc((size_t)nch * sr, s));
  const size_t hsm = (size_t)sr * sizeof(int);
  KRR_TRY(raise_smem_limit(row_hist_kernel, hsm));
  row_hist_kernel<<<nch, 256, hsm, s>>>(rows.p, N, zeta, sr, hist.p);
  KRR_LAUNCH_CHECK();
  row_total_kernel<<<ceil_div(sr, 256), 256, 0, s>>>(hist.p, nch, sr, total.p);
  KRR_LAUNCH_CHECK();
  row_scan_kernel<<<1, 32, 0, s>>>(total.p, sr, rowptr.p);
  KRR_LAUNCH_CHECK();
  row_offsets_kernel<<<ceil_div(sr, 256), 256, 0, s>>>(hist.p, nch, sr, rowptr.p, off.p);
  KRR_LAUNCH_CHECK();
  const size_t fsm = (size_t)sr * sizeof(int64_t);
  KRR_TRY(raise_smem_limit(row_fill_kernel, fsm));
  row_fill_kernel<<<nch, 32, fsm, s>>>(rows.p, vals.p, N, zeta, sr, off.p, col_n.p, col_v.p);
  KRR_LAUNCH_CHECK();
  // sketch
  KRR_TRY(dev_alloc(&P->Bsk, (size_t)sr * k));
  {
    dim3 grid(sr, ceil_div(k, 256));
    KRR_KERN_SWITCH(P->kern, KRR_DP_SWITCH(P->dp, {
      sketch_kernel<KERN, DP><<<grid, 256, 0, s>>>(P->xt, P->cn, P->S, k, rowptr.p, col_n.p,
                                                   col_v.p, sr, P->Bsk);
    }));
    KRR_LAUNCH_CHECK();
  }
  // P = B^T B + H
  KRR_TRY(dev_alloc(&P->P, (size_t)k * k));
  KRR_CUDA_TRY(cudaMemcpyAsync(P->P, P->H, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, s));
  {
    Gemm<double> g;
    g.M = k; g.N = k; g.K = sr;
    g.A = P->Bsk; g.sai = sr; g.sak = 1;
    g.B = P->Bsk; g.sbk = 1; g.sbj = sr;
    g.alpha = 1.0; g.beta = 1.0; g.C = P->P; g.ldc = k;
    KRR_TRY(gemm(g, s, gemm_auto_split(k, k, sr)));
  }
  KRR_TRY(dev_alloc(&P->L, (size_t)k * k));
  KRR_CUDA_TRY(cudaMemcpyAsync(P->L, P->P, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, s));
  KRR_TRY(potrf_lower(P->L, k, k, s));
  KRR_TRY(dev_alloc(&P->Winv, (size_t)k * k));
  KRR_TRY(trinv_lower(P->L, k, k, P->Winv, s));
  KRR_TRY(dev_alloc(&P->Winv_t, (size_t)k * k));
  KRR_TRY(transpose_square(P->Winv, k, P->Winv_t, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  P->build_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return KRR_OK;
}

// M beta = A(S,:)(A(:,S) beta) + H beta   (k x m blocks, float64)
krr_status krill_product(const krill_precond *P, const double *beta, int m, double *out,
                         cudaStream_t s, DevBuf<float> &u, DevBuf<double> &v) {
  if (u.n < (size_t)P->N * m) KRR_TRY(u.alloc((size_t)P->N * m, s));
  if (v.n < (size_t)P->k * m) KRR_TRY(v.alloc((size_t)P->k * m, s));
  KRR_TRY(krill_kcols(P, beta, m, u.p, s));
  KRR_TRY(krill_krows(P, u.p, m, v.p, s));
  sym_gemv_add_kernel<<<ceil_div(P->k, 8), 256, 0, s>>>(P->H, P->k, beta, m, v.p, out);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// out = C^{-1} C^{-T} in = W^T (W in), W = L^{-1}, P = L L^T, C = L^T.
krr_status krill_precond_apply(const krill_precond *P, const double *in, int m, double *tmp,
                               double *out, cudaStream_t s) {
  KRR_TRY(tri_apply_lower(P->Winv_t, P->k, in, m, tmp, s));
  KRR_TRY(tri_apply_lower_t(P->Winv, P->k, tmp, m, out, s));
  return KRR_OK;
}

__global__ void gather_points_kernel(const double *__restrict__ X, int d,
                                     const int64_t *__restrict__ S, int k,
                                     double *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * d) return;
  out[e] = X[S[e / d] * d + e % d];
}

// float-float point sets of a solve: all points and the centers, split with
// the same centre and scale.
krr_status krill_points_ff(const krill_precond *P, cudaStream_t s, KrillFF &Q) {
  KRR_TRY(prepare_points_ff(P->X, P->N, P->d, P->kern, P->sigma, s, Q.all));
  DevBuf<double> xc;
  KRR_TRY(xc.alloc((size_t)P->k * P->d, s));
  gather_points_kernel<<<ceil_div((int64_t)P->k * P->d, 256), 256, 0, s>>>(P->X, P->d, P->S,
                                                                          P->k, xc.p);
  KRR_LAUNCH_CHECK();
  KRR_TRY(prepare_points_ff(xc.p, P->k, P->d, P->kern, P->sigma, s, Q.centers, Q.all.mean.p));
  return KRR_OK;
}

// Right-hand side A(S,:) y, y N x m float64, float64-accurate (float-float).
krr_status krill_rhs(const krill_precond *P, KrillFF &Q, const double *y, int m, double *b,
                     cudaStream_t s) {
  return kff_cross(Q.centers, Q.all, 0.0, y, P->N, m, b, P->k, s, Q.part, Q.vsplit);
}

// float64-accurate product M beta = A(S,:)(A(:,S) beta) + H beta for the
// refinement residual (float-float block products).
krr_status krill_product64(const krill_precond *P, KrillFF &Q, const double *beta, int m,
                           double *out, cudaStream_t s, DevBuf<double> &u, DevBuf<double> &v) {
  if (u.n < (size_t)P->N * m) KRR_TRY(u.alloc((size_t)P->N * m, s));
  if (v.n < (size_t)P->k * m) KRR_TRY(v.alloc((size_t)P->k * m, s));
  KRR_TRY(kff_cross(Q.all, Q.centers, 0.0, beta, P->k, m, u.p, P->N, s, Q.part, Q.vsplit));
  KRR_TRY(kff_cross(Q.centers, Q.all, 0.0, u.p, P->N, m, v.p, P->k, s, Q.part, Q.vsplit));
  sym_gemv_add_kernel<<<ceil_div(P->k, 8), 256, 0, s>>>(P->H, P->k, beta, m, v.p, out);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ------------------------------------------- tcgen05 block products
krr_status krill_points_tc5(const krill_precond *P, cudaStream_t s, KrillTC5 &T) {
  T.ok = false;
  if (P->kern == KLAPLACE || product_path() == 1 || P->d > 32) return KRR_OK;
  KRR_TRY(prepare_points_f32(P->X, P->N, P->d, P->kern, P->sigma, s, T.all));
  DevBuf<double> xc;
  KRR_TRY(xc.alloc((size_t)P->k * P->d, s));
  gather_points_kernel<<<ceil_div((int64_t)P->k * P->d, 256), 256, 0, s>>>(P->X, P->d, P->S,
                                                                          P->k, xc.p);
  KRR_LAUNCH_CHECK();
  KRR_TRY(prepare_points_f32(xc.p, P->k, P->d, P->kern, P->sigma, s, T.centers, T.all.mean.p));
  int bad_all = 0, bad_c = 0;
  KRR_TRY(prepare_points_tc5(P->X, s, T.all, &bad_all));
  KRR_TRY(prepare_points_tc5(xc.p, s, T.centers, &bad_c));
  T.ok = !bad_all && !bad_c && T.all.nh5 > 0 && T.centers.nh5 > 0;
  return KRR_OK;
}

krr_status krill_product_tc5(const krill_precond *P, KrillTC5 &T, const double *beta, int m,
                             double *out, cudaStream_t s, DevBuf<float> &u) {
  const int64_t N = P->N;
  const int k = P->k;
  if (u.n < (size_t)N * m) KRR_TRY(u.alloc((size_t)N * m, s));
  if (T.b32.n < (size_t)k * m) KRR_TRY(T.b32.alloc((size_t)k * m, s));
  if (T.v32.n < (size_t)k * m) KRR_TRY(T.v32.alloc((size_t)k * m, s));
  if (T.v64.n < (size_t)k * m) KRR_TRY(T.v64.alloc((size_t)k * m, s));
  KRR_TRY(convert_f64_to_f32(beta, T.b32.p, (int64_t)k * m, s));
  // u = A(:, S) beta: rows are all points, columns the centers
  KRR_TRY(kmv_tc5(T.all, T.centers, 0.0f, false, T.b32.p, k, m, u.p, N, s, T.part));
  // v = A(S, :) u: rows are the centers, columns all points
  KRR_TRY(kmv_tc5(T.centers, T.all, 0.0f, false, u.p, N, m, T.v32.p, k, s, T.part));
  KRR_TRY(convert_f32_to_f64(T.v32.p, T.v64.p, (int64_t)k * m, s));
  sym_gemv_add_kernel<<<ceil_div(k, 8), 256, 0, s>>>(P->H, k, beta, m, T.v64.p, out);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

}  // namespace krr
