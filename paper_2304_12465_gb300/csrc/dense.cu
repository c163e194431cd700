// Dense building blocks: strided SIMT GEMM (float32 / float64), blocked
// float64 Cholesky and blocked lower-triangular inverse.  Used for the k x k
// cores of Alg. 1 (lambda I + F^T F) and Alg. 2 (B^T B + H), the Schur update
// of Alg. 3 and the triangular solves of both preconditioners.
#include "dense.cuh"

namespace krr {

constexpr int GB_M = 64, GB_N = 64, GB_K = 16, G_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(G_THREADS)
gemm_kernel(int M, int N, int K, const T *__restrict__ A, int64_t sai, int64_t sak,
            const T *__restrict__ B, int64_t sbk, int64_t sbj, T *__restrict__ out,
            int64_t ldo, int64_t slice_stride, int kslice, T alpha, T beta, int direct) {
  __shared__ T As[GB_K][GB_M + 1];
  __shared__ T Bs[GB_K][GB_N + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.x * GB_M, j0 = blockIdx.y * GB_N;
  const int kb = blockIdx.z * kslice;
  const int ke = min(K, kb + kslice);
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0;
  const bool a_kfast = (sak == 1 && sai != 1);
  const bool b_kfast = (sbk == 1 && sbj != 1);
  for (int k0 = kb; k0 < ke; k0 += GB_K) {
#pragma unroll
    for (int e = 0; e < (GB_M * GB_K) / G_THREADS; ++e) {
      const int idx = tid + e * G_THREADS;
      int ii, kk;
      if (a_kfast) { kk = idx % GB_K; ii = idx / GB_K; }
      else { ii = idx % GB_M; kk = idx / GB_M; }
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < ke) ? A[(int64_t)gi * sai + (int64_t)gk * sak] : T(0);
    }
#pragma unroll
    for (int e = 0; e < (GB_N * GB_K) / G_THREADS; ++e) {
      const int idx = tid + e * G_THREADS;
      int jj, kk;
      if (b_kfast) { kk = idx % GB_K; jj = idx / GB_K; }
      else { jj = idx % GB_N; kk = idx / GB_N; }
      const int gj = j0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < ke) ? B[(int64_t)gk * sbk + (int64_t)gj * sbj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  T *o = out + (int64_t)blockIdx.z * slice_stride;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < M && gj < N) {
        T *dst = o + (int64_t)gi + (int64_t)gj * ldo;
        if (direct) *dst = (beta == T(0)) ? alpha * acc[r][c] : fma(alpha, acc[r][c], beta * *dst);
        else *dst = acc[r][c];
      }
    }
}

// C = beta C + alpha * sum_z P_z, P_z (M x N, ld M) in slices.
template <typename T>
__global__ void gemm_combine_kernel(int M, int N, const T *__restrict__ P, int slices,
                                    T alpha, T beta, T *__restrict__ C, int64_t ldc) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % M), j = (int)(e / M);
    T acc = 0;
    for (int z = 0; z < slices; ++z) acc += P[(int64_t)z * total + e];
    T *c = C + (int64_t)i + (int64_t)j * ldc;
    *c = (beta == T(0)) ? alpha * acc : beta * (*c) + alpha * acc;
  }
}

int gemm_auto_split(int M, int N, int K) {
  const int64_t tiles = (int64_t)((M + GB_M - 1) / GB_M) * ((N + GB_N - 1) / GB_N);
  const int64_t want = (int64_t)num_sms() * 4;
  if (tiles >= want || K < 4 * GB_K) return 1;
  int64_t sk = (want + tiles - 1) / tiles;
  const int64_t maxk = K / (8 * GB_K);
  if (sk > maxk) sk = maxk;
  if (sk > 64) sk = 64;
  return (int)(sk < 1 ? 1 : sk);
}

template <typename T>
krr_status gemm(const Gemm<T> &g, cudaStream_t s, int split_k) {
  if (g.M <= 0 || g.N <= 0) return KRR_OK;
  if (g.K <= 0) {
    // C = beta C
    DevBuf<T> z;
    KRR_TRY(z.alloc((size_t)g.M * g.N, s));
    KRR_CUDA_TRY(cudaMemsetAsync(z.p, 0, sizeof(T) * (size_t)g.M * g.N, s));
    gemm_combine_kernel<T><<<ceil_div((int64_t)g.M * g.N, 256), 256, 0, s>>>(
        g.M, g.N, z.p, 1, g.alpha, g.beta, g.C, g.ldc);
    KRR_LAUNCH_CHECK();
    return KRR_OK;
  }
  if (split_k < 1) split_k = 1;
  int kslice = (g.K + split_k - 1) / split_k;
  kslice = (kslice + GB_K - 1) / GB_K * GB_K;
  const int slices = (g.K + kslice - 1) / kslice;
  dim3 grid((g.M + GB_M - 1) / GB_M, (g.N + GB_N - 1) / GB_N, slices);
  if (slices == 1) {
    gemm_kernel<T><<<grid, G_THREADS, 0, s>>>(g.M, g.N, g.K, g.A, g.sai, g.sak, g.B, g.sbk,
                                             g.sbj, g.C, g.ldc, 0, kslice, g.alpha, g.beta, 1);
    KRR_LAUNCH_CHECK();
    return KRR_OK;
  }
  DevBuf<T> P;
  KRR_TRY(P.alloc((size_t)slices * g.M * g.N, s));
  gemm_kernel<T><<<grid, G_THREADS, 0, s>>>(g.M, g.N, g.K, g.A, g.sai, g.sak, g.B, g.sbk,
                                           g.sbj, P.p, g.M, (int64_t)g.M * g.N, kslice,
                                           T(1), T(0), 0);
  KRR_LAUNCH_CHECK();
  int64_t total = (int64_t)g.M * g.N;
  int blocks = ceil_div(total, 256);
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  gemm_combine_kernel<T><<<blocks, 256, 0, s>>>(g.M, g.N, P.p, slices, g.alpha, g.beta,
                                                g.C, g.ldc);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ------------------------------------------- float-float Schur update
// C(M x N) -= A(M x K) B(K x N) for float64 data, with the products and sums
// in float-float arithmetic on the float32 pipes (float64 runs at a small
// fraction of the float32 rate on this GPU).  Each float64 input is split
// into hi = fl32(a) and lo = fl32(a - hi) (48 bits) when its tile is staged;
// a product is hi_a hi_b, split exactly into p + e with an FMA (Dekker's
// TwoProduct), plus the cross terms hi_a lo_b + lo_a hi_b (lo_a lo_b, below
// 2^-48 |a b|, is dropped); p enters the running sum through Knuth's
// error-free TwoSum, the rounding error and e through a float32 correction.
// The pair (sum, correction) is renormalised once per K tile.  Intrinsics
// keep the compiler from contracting or reassociating the error-free steps.
// Error: about 2^-48 sqrt(K) max_k |sum_{l<=k} a_il b_lj| per entry.
__global__ void __launch_bounds__(G_THREADS)
gemm_sub_ff_kernel(int M, int N, int K, const double *__restrict__ A, int64_t sai,
                   int64_t sak, const double *__restrict__ B, int64_t sbk, int64_t sbj,
                   double *__restrict__ C, int64_t ldc) {
  __shared__ float Ah[GB_K][GB_M + 1], Al[GB_K][GB_M + 1];
  __shared__ float Bh[GB_K][GB_N + 1], Bl[GB_K][GB_N + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.x * GB_M, j0 = blockIdx.y * GB_N;
  // outputs (row ty + 16 r, columns tx + 16 (2 h) and tx + 16 (2 h + 1)) as
  // packed pairs: every step below is one FMUL2 / FFMA2 / FADD2 for two
  // outputs, x - y written as fma(y, -1, x) (the same single rounding)
  float2 sh[4][2], sl[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) sh[r][h] = sl[r][h] = make_float2(0.0f, 0.0f);
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const bool a_kfast = (sak == 1 && sai != 1);
  const bool b_kfast = (sbk == 1 && sbj != 1);
  for (int k0 = 0; k0 < K; k0 += GB_K) {
#pragma unroll
    for (int e = 0; e < (GB_M * GB_K) / G_THREADS; ++e) {
      const int idx = tid + e * G_THREADS;
      int ii, kk;
      if (a_kfast) { kk = idx % GB_K; ii = idx / GB_K; }
      else { ii = idx % GB_M; kk = idx / GB_M; }
      const int gi = i0 + ii, gk = k0 + kk;
      const double v = (gi < M && gk < K) ? A[(int64_t)gi * sai + (int64_t)gk * sak] : 0.0;
      const float h = __double2float_rn(v);
      Ah[kk][ii] = h;
      Al[kk][ii] = __double2float_rn(v - (double)h);
    }
#pragma unroll
    for (int e = 0; e < (GB_N * GB_K) / G_THREADS; ++e) {
      const int idx = tid + e * G_THREADS;
      int jj, kk;
      if (b_kfast) { kk = idx % GB_K; jj = idx / GB_K; }
      else { jj = idx % GB_N; kk = idx / GB_N; }
      const int gj = j0 + jj, gk = k0 + kk;
      const double v = (gj < N && gk < K) ? B[(int64_t)gk * sbk + (int64_t)gj * sbj] : 0.0;
      const float h = __double2float_rn(v);
      Bh[kk][jj] = h;
      Bl[kk][jj] = __double2float_rn(v - (double)h);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GB_K; ++kk) {
      float2 ah[4], nah[4], nal[4], bh[2], bl[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float a = Ah[kk][ty + 16 * r], al = Al[kk][ty + 16 * r];
        ah[r] = make_float2(a, a);
        nah[r] = make_float2(-a, -a);
        nal[r] = make_float2(-al, -al);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        bh[h] = make_float2(Bh[kk][tx + 32 * h], Bh[kk][tx + 32 * h + 16]);
        bl[h] = make_float2(Bl[kk][tx + 32 * h], Bl[kk][tx + 32 * h + 16]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // p = hi_a hi_b; en = -(hi_a hi_b - p) - hi_a lo_b - lo_a hi_b (the
          // negated product error and cross terms, each step exact or
          // rounded once as in the scalar form)
          const float2 p = __fmul2_rn(ah[r], bh[h]);
          float2 en = __ffma2_rn(nah[r], bh[h], p);
          en = __ffma2_rn(nah[r], bl[h], en);
          en = __ffma2_rn(nal[r], bh[h], en);
          // TwoSum(sh, p)
          const float2 t = __fadd2_rn(sh[r][h], p);
          const float2 z = __ffma2_rn(sh[r][h], m1, t);
          const float2 tz = __ffma2_rn(z, m1, t);
          const float2 err = __fadd2_rn(__ffma2_rn(tz, m1, sh[r][h]), __ffma2_rn(z, m1, p));
          sh[r][h] = t;
          sl[r][h] = __fadd2_rn(sl[r][h], __ffma2_rn(en, m1, err));
        }
    }
    __syncthreads();
    // renormalise once per tile (TwoSum): the correction stays below an ulp
    // of the sum, so its own roundings stay at the float-float level
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 t = __fadd2_rn(sh[r][h], sl[r][h]);
        const float2 z = __ffma2_rn(sh[r][h], m1, t);
        sl[r][h] = __fadd2_rn(__ffma2_rn(__ffma2_rn(z, m1, t), m1, sh[r][h]),
                              __ffma2_rn(z, m1, sl[r][h]));
        sh[r][h] = t;
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int gi = i0 + ty + 16 * r, gj = j0 + tx + 32 * h + 16 * e;
        if (gi < M && gj < N) {
          double *dst = C + (int64_t)gi + (int64_t)gj * ldc;
          const float hi = e ? sh[r][h].y : sh[r][h].x, lo = e ? sl[r][h].y : sl[r][h].x;
          *dst = *dst - ((double)hi + (double)lo);
        }
      }
}

krr_status gemm_sub_ff(const Gemm<double> &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return KRR_OK;
  KRR_REQUIRE(g.alpha == -1.0 && g.beta == 1.0, "gemm_sub_ff: C -= A B only");
  dim3 grid((g.M + GB_M - 1) / GB_M, (g.N + GB_N - 1) / GB_N, 1);
  gemm_sub_ff_kernel<<<grid, G_THREADS, 0, s>>>(g.M, g.N, g.K, g.A, g.sai, g.sak, g.B, g.sbk,
                                                g.sbj, g.C, g.ldc);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ------------------------------------------------------------ Gram (F^T F)
// Lower-triangular output tiles only.  float input: each K tile of GB_K
// products is summed in float32, then added to a float-float accumulator
// (Knuth's TwoSum, the rounding errors gathered in a float32 correction that
// is folded back every 8 tiles) -- float64 adds, at a small fraction of the
// float32 rate on this GPU, bounded the kernel; double input: float64
// throughout.
template <typename T>
__global__ void __launch_bounds__(G_THREADS)
gram_lower_kernel(const T *__restrict__ F, int64_t N, int r, int kslice,
                  double *__restrict__ part) {
  __shared__ T As[GB_K][GB_M + 1];
  __shared__ T Bs[GB_K][GB_N + 1];
  // map blockIdx.x to a lower-triangular (ti, tj) tile pair, tj <= ti
  int t = blockIdx.x, ti = 0;
  while (t > ti) { t -= ti + 1; ++ti; }
  const int tj = t;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = ti * GB_M, j0 = tj * GB_N;
  const int64_t kb = (int64_t)blockIdx.y * kslice;
  const int64_t ke = min(N, kb + kslice);
  constexpr bool FLT = sizeof(T) == 4;
  double acc[4][4];
  float sh[4][4], sl[4][4];   // float-float accumulators (float input)
  T acc32[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0.0;
      sh[a][b] = sl[a][b] = 0.0f;
    }
  int chunk = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += GB_K) {
#pragma unroll
    for (int e = 0; e < (GB_M * GB_K) / G_THREADS; ++e) {
      const int idx = tid + e * G_THREADS;
      const int kk = idx % GB_K, ii = idx / GB_K;
      const int64_t gk = k0 + kk;
      As[kk][ii] = (i0 + ii < r && gk < ke) ? F[gk + (int64_t)(i0 + ii) * N] : T(0);
      Bs[kk][ii] = (j0 + ii < r && gk < ke) ? F[gk + (int64_t)(j0 + ii) * N] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc32[a][b] = T(0);
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc32[a][b] = fma(av[a], bv[b], acc32[a][b]);
    }
    if constexpr (FLT) {
      ++chunk;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float c = (float)acc32[a][b];
          const float t = __fadd_rn(sh[a][b], c);
          const float z = __fsub_rn(t, sh[a][b]);
          const float err = __fadd_rn(__fsub_rn(sh[a][b], __fsub_rn(t, z)), __fsub_rn(c, z));
          sh[a][b] = t;
          sl[a][b] = __fadd_rn(sl[a][b], err);
          if ((chunk & 7) == 0) {
            // fold the correction back (TwoSum), keeping it below an ulp of the sum
            const float t2 = __fadd_rn(sh[a][b], sl[a][b]);
            const float z2 = __fsub_rn(t2, sh[a][b]);
            sl[a][b] = __fadd_rn(__fsub_rn(sh[a][b], __fsub_rn(t2, z2)), __fsub_rn(sl[a][b], z2));
            sh[a][b] = t2;
          }
        }
    } else {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += (double)acc32[a][b];
    }
    __syncthreads();
  }
  double *o = part + (int64_t)blockIdx.y * r * r;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
      if (gi < r && gj <= gi)
        o[(int64_t)gi + (int64_t)gj * r] =
            FLT ? (double)sh[a][b] + (double)sl[a][b] : acc[a][b];
    }
}

__global__ void gram_combine_kernel(const double *__restrict__ part, int slices, int r,
                                    double *__restrict__ C) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r), j = (int)(e / r);
    if (j > i) continue;
    double acc = 0.0;
    for (int z = 0; z < slices; ++z) acc += part[(int64_t)z * total + e];
    C[e] = acc;
  }
}

template <typename T>
krr_status gram_lower(const T *F, int64_t N, int r, double *C, cudaStream_t s) {
  if (r <= 0) return KRR_OK;
  const int tiles = (r + GB_M - 1) / GB_M;
  const int ntri = tiles * (tiles + 1) / 2;
  int64_t slices = ((int64_t)num_sms() * 4 + ntri - 1) / ntri;
  const int64_t maxs = (N + 1023) / 1024;
  if (slices > maxs) slices = maxs;
  if (slices < 1) slices = 1;
  int64_t kslice = (N + slices - 1) / slices;
  kslice = (kslice + GB_K - 1) / GB_K * GB_K;
  slices = (N + kslice - 1) / kslice;
  DevBuf<double> part;
  KRR_TRY(part.alloc((size_t)slices * r * r, s));
  gram_lower_kernel<T><<<dim3(ntri, (unsigned)slices), G_THREADS, 0, s>>>(F, N, r, (int)kslice,
                                                                         part.p);
  KRR_LAUNCH_CHECK();
  int blocks = ceil_div((int64_t)r * r, 256);
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  gram_combine_kernel<<<blocks, 256, 0, s>>>(part.p, (int)slices, r, C);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

template krr_status gram_lower<float>(const float *, int64_t, int, double *, cudaStream_t);
template krr_status gram_lower<double>(const double *, int64_t, int, double *, cudaStream_t);

template krr_status gemm<double>(const Gemm<double> &, cudaStream_t, int);
template krr_status gemm<float>(const Gemm<float> &, cudaStream_t, int);

// ------------------------------------------------------------ Cholesky
constexpr int CH_NB = 64;

// Factors the w x w diagonal block at A (lda) in place (lower) and writes the
// inverse of its factor to Dinv (CH_NB x CH_NB, column-major, zero padded).
// factor == 0: the block already holds a lower factor; only invert it.
__global__ void __launch_bounds__(256)
potrf_diag_kernel(double *__restrict__ A, int w, int64_t lda, double *__restrict__ Dinv,
                  int *__restrict__ status, int factor) {
  extern __shared__ double smem[];
  double *sA = smem;                        // CH_NB x (CH_NB+1)
  double *sW = smem + CH_NB * (CH_NB + 1);  // CH_NB x (CH_NB+1)
  const int tid = threadIdx.x;
  constexpr int LD = CH_NB + 1;
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e % w, j = e / w;
    sA[i * LD + j] = (i >= j) ? A[i + (int64_t)j * lda] : 0.0;
  }
  __syncthreads();
  if (factor) {
    for (int j = 0; j < w; ++j) {
      if (tid == 0) {
        const double p = sA[j * LD + j];
        if (!(p > 0.0)) atomicExch(status, 1);
        sA[j * LD + j] = sqrt(p);
      }
      __syncthreads();
      const double dj = sA[j * LD + j];
      for (int i = j + 1 + tid; i < w; i += blockDim.x) sA[i * LD + j] /= dj;
      __syncthreads();
      const int rem = w - j - 1;
      for (int e = tid; e < rem * rem; e += blockDim.x) {
        const int i = j + 1 + e % rem, l = j + 1 + e / rem;
        if (l <= i) sA[i * LD + l] -= sA[i * LD + j] * sA[l * LD + j];
      }
      __syncthreads();
    }
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = e % w, j = e / w;
      if (i >= j) A[i + (int64_t)j * lda] = sA[i * LD + j];
    }
  }
  // inverse of the lower factor, one column per thread (forward substitution)
  if (tid < CH_NB) {
    const int c = tid;
    for (int i = 0; i < CH_NB; ++i) {
      double v = 0.0;
      if (c < w && i < w && i >= c) {
        v = (i == c) ? 1.0 : 0.0;
        for (int l = c; l < i; ++l) v -= sA[i * LD + l] * sW[l * LD + c];
        v /= sA[i * LD + i];
      }
      sW[i * LD + c] = v;
    }
  }
  __syncthreads();
  for (int e = tid; e < CH_NB * CH_NB; e += blockDim.x) {
    const int i = e % CH_NB, j = e / CH_NB;
    Dinv[i + j * CH_NB] = sW[i * LD + j];
  }
}

static krr_status diag_block(double *A, int w, int64_t lda, double *Dinv, int *status,
                             int factor, cudaStream_t s) {
  const size_t smem = 2 * CH_NB * (CH_NB + 1) * sizeof(double);
  KRR_TRY(raise_smem_limit(potrf_diag_kernel, smem));
  potrf_diag_kernel<<<1, 256, smem, s>>>(A, w, lda, Dinv, status, factor);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

__global__ void copy_block_kernel(const double *__restrict__ src, int64_t lds, int rows,
                                  int cols, double *__restrict__ dst, int64_t ldd) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    dst[i + j * ldd] = src[i + j * lds];
  }
}

krr_status potrf_lower(double *A, int n, int64_t lda, cudaStream_t s) {
  if (n <= 0) return KRR_OK;
  DevBuf<int> status;
  KRR_TRY(status.alloc(1, s));
  KRR_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  DevBuf<double> dinv, T;
  KRR_TRY(dinv.alloc(CH_NB * CH_NB, s));
  KRR_TRY(T.alloc((size_t)n * CH_NB, s));
  for (int o = 0; o < n; o += CH_NB) {
    const int w = (n - o < CH_NB) ? n - o : CH_NB;
    double *Abb = A + o + (int64_t)o * lda;
    KRR_TRY(diag_block(Abb, w, lda, dinv.p, status.p, 1, s));
    const int r = n - o - w;
    if (r <= 0) break;
    double *A21 = Abb + w;
    // T (r x w) = A21 Dinv^T
    Gemm<double> g;
    g.M = r; g.N = w; g.K = w;
    g.A = A21; g.sai = 1; g.sak = lda;
    g.B = dinv.p; g.sbk = CH_NB; g.sbj = 1;
    g.alpha = 1.0; g.beta = 0.0; g.C = T.p; g.ldc = r;
    KRR_TRY(gemm(g, s));
    copy_block_kernel<<<ceil_div((int64_t)r * w, 256), 256, 0, s>>>(T.p, r, r, w, A21, lda);
    KRR_LAUNCH_CHECK();
    // A22 -= T T^T
    Gemm<double> u;
    u.M = r; u.N = r; u.K = w;
    u.A = T.p; u.sai = 1; u.sak = r;
    u.B = T.p; u.sbk = r; u.sbj = 1;
    u.alpha = -1.0; u.beta = 1.0; u.C = A21 + (int64_t)w * lda; u.ldc = lda;
    KRR_TRY(gemm(u, s, gemm_auto_split(r, r, w)));
  }
  int h = 0;
  KRR_CUDA_TRY(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    set_error("Cholesky factorisation met a non-positive pivot (matrix not numerically "
              "positive definite)");
    return KRR_ECHOL;
  }
  return KRR_OK;
}

krr_status trinv_lower(const double *L, int n, int64_t lda, double *W, cudaStream_t s) {
  if (n <= 0) return KRR_OK;
  KRR_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * n, s));
  DevBuf<int> status;
  KRR_TRY(status.alloc(1, s));
  KRR_CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(int), s));
  const int nb = (n + CH_NB - 1) / CH_NB;
  DevBuf<double> dinv, T;
  KRR_TRY(dinv.alloc((size_t)nb * CH_NB * CH_NB, s));
  KRR_TRY(T.alloc((size_t)CH_NB * n, s));
  for (int b = 0; b < nb; ++b) {
    const int o = b * CH_NB;
    const int w = (n - o < CH_NB) ? n - o : CH_NB;
    KRR_TRY(diag_block(const_cast<double *>(L) + o + (int64_t)o * lda, w, lda,
                       dinv.p + (size_t)b * CH_NB * CH_NB, status.p, 0, s));
    copy_block_kernel<<<ceil_div((int64_t)w * w, 256), 256, 0, s>>>(
        dinv.p + (size_t)b * CH_NB * CH_NB, CH_NB, w, w, W + o + (int64_t)o * n, n);
    KRR_LAUNCH_CHECK();
  }
  for (int b = 1; b < nb; ++b) {
    const int o = b * CH_NB;
    const int w = (n - o < CH_NB) ? n - o : CH_NB;
    // T (w x o) = L(o:o+w, 0:o) W(0:o, 0:o)
    Gemm<double> g;
    g.M = w; g.N = o; g.K = o;
    g.A = L + o; g.sai = 1; g.sak = lda;
    g.B = W; g.sbk = 1; g.sbj = n;
    g.alpha = 1.0; g.beta = 0.0; g.C = T.p; g.ldc = w;
    KRR_TRY(gemm(g, s));
    // W(o:o+w, 0:o) = -Dinv_b T
    Gemm<double> h;
    h.M = w; h.N = o; h.K = w;
    h.A = dinv.p + (size_t)b * CH_NB * CH_NB; h.sai = 1; h.sak = CH_NB;
    h.B = T.p; h.sbk = 1; h.sbj = w;
    h.alpha = -1.0; h.beta = 0.0; h.C = W + o; h.ldc = n;
    KRR_TRY(gemm(h, s));
  }
  return KRR_OK;
}

__global__ void add_diag_kernel(double *A, int n, int64_t lda, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + (int64_t)i * lda] += v;
}

krr_status add_diagonal(double *A, int n, int64_t lda, double v, cudaStream_t s) {
  if (n <= 0) return KRR_OK;
  add_diag_kernel<<<ceil_div(n, 256), 256, 0, s>>>(A, n, lda, v);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

__global__ void transpose_kernel(const double *__restrict__ A, int n, double *__restrict__ B) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = bx + threadIdx.x, c = by + j;
    if (r < n && c < n) tile[j][threadIdx.x] = A[r + (int64_t)c * n];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + threadIdx.x, c = bx + j;
    if (r < n && c < n) B[r + (int64_t)c * n] = tile[threadIdx.x][j];
  }
}

krr_status transpose_square(const double *A, int n, double *B, cudaStream_t s) {
  if (n <= 0) return KRR_OK;
  dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  transpose_kernel<<<grid, block, 0, s>>>(A, n, B);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

__global__ void symmetrize_kernel(double *A, int n, int64_t lda) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (j > i) A[i + (int64_t)j * lda] = A[j + (int64_t)i * lda];
  }
}

krr_status symmetrize_lower(double *A, int n, int64_t lda, cudaStream_t s) {
  if (n <= 0) return KRR_OK;
  int blocks = ceil_div((int64_t)n * n, 256);
  if (blocks > num_sms() * 16) blocks = num_sms() * 16;
  symmetrize_kernel<<<blocks, 256, 0, s>>>(A, n, lda);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

}  // namespace krr
