// Host drivers of the fused product (Alg. 1 "Product"), point preparation,
// split reduction and kernel-column evaluation.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "kmv.cuh"
#include "kmv_dispatch.cuh"
#include "kmvtc_kernels.cuh"

namespace krr {

cudaError_t launch_kmv32_gauss(int DP, int M, dim3 g, cudaStream_t s, const Kmv32Args &a);
cudaError_t launch_kmv32_laplace(int DP, int M, dim3 g, cudaStream_t s, const Kmv32Args &a);
cudaError_t launch_kmv32_matern(int DP, int M, dim3 g, cudaStream_t s, const Kmv32Args &a);
cudaError_t launch_kmv64_gauss(int DP, int M, dim3 g, cudaStream_t s, const Kmv64Args &a);
cudaError_t launch_kmvff_gauss(int DP, int M, dim3 g, cudaStream_t s, const KmvFFArgs &a);
cudaError_t launch_kmvff_laplace(int DP, int M, dim3 g, cudaStream_t s, const KmvFFArgs &a);
cudaError_t launch_kmvff_matern(int DP, int M, dim3 g, cudaStream_t s, const KmvFFArgs &a);
cudaError_t launch_kmv64_laplace(int DP, int M, dim3 g, cudaStream_t s, const Kmv64Args &a);
cudaError_t launch_kmvffsym_gauss(int DP, int M, int G, cudaStream_t s, const KmvFFSymArgs &a);
cudaError_t launch_kmvffsym_laplace(int DP, int M, int G, cudaStream_t s, const KmvFFSymArgs &a);
cudaError_t launch_kmvffsym_matern(int DP, int M, int G, cudaStream_t s, const KmvFFSymArgs &a);
cudaError_t launch_kmv64_matern(int DP, int M, dim3 g, cudaStream_t s, const Kmv64Args &a);

cudaError_t launch_kmv32_any(int kern, int DP, int M, dim3 g, cudaStream_t s,
                             const Kmv32Args &a) {
  switch (kern) {
    case KGAUSS: return launch_kmv32_gauss(DP, M, g, s, a);
    case KLAPLACE: return launch_kmv32_laplace(DP, M, g, s, a);
    case KMATERN: return launch_kmv32_matern(DP, M, g, s, a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kmv64_any(int kern, int DP, int M, dim3 g, cudaStream_t s,
                             const Kmv64Args &a) {
  switch (kern) {
    case KGAUSS: return launch_kmv64_gauss(DP, M, g, s, a);
    case KLAPLACE: return launch_kmv64_laplace(DP, M, g, s, a);
    case KMATERN: return launch_kmv64_matern(DP, M, g, s, a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kmvff_any(int kern, int DP, int M, dim3 g, cudaStream_t s,
                             const KmvFFArgs &a) {
  switch (kern) {
    case KGAUSS: return launch_kmvff_gauss(DP, M, g, s, a);
    case KLAPLACE: return launch_kmvff_laplace(DP, M, g, s, a);
    case KMATERN: return launch_kmvff_matern(DP, M, g, s, a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_kmvffsym_any(int kern, int DP, int M, int G, cudaStream_t s,
                                const KmvFFSymArgs &a) {
  switch (kern) {
    case KGAUSS: return launch_kmvffsym_gauss(DP, M, G, s, a);
    case KLAPLACE: return launch_kmvffsym_laplace(DP, M, G, s, a);
    case KMATERN: return launch_kmvffsym_matern(DP, M, G, s, a);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------- preparation
__global__ void column_mean_kernel(const double *__restrict__ X, int64_t N, int d,
                                   double *__restrict__ mean) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += X[i * d + k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) mean[k] = v / (double)N;
  }
}

__global__ void prepare_f32_kernel(const double *__restrict__ X, int64_t N, int d, int dp,
                                   const double *__restrict__ mean, double scale,
                                   int with_norm, float *__restrict__ xt,
                                   float *__restrict__ cn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double nrm = 0.0;
  for (int k = 0; k < dp; ++k) {
    float v = 0.0f;
    if (k < d) v = (float)((X[i * d + k] - mean[k]) * scale);
    xt[i * dp + k] = v;
    nrm += (double)v * (double)v;
  }
  cn[i] = with_norm ? (float)(-0.5 * nrm) : 0.0f;
}

krr_status prepare_points_f32(const double *Xd, int64_t N, int d, int kern, double sigma,
                              cudaStream_t s, PointsF32 &P, const double *mean_dev, int dp) {
  P.dp = dp > 0 ? dp : (d + 3) / 4 * 4;
  KRR_REQUIRE(P.dp >= d && P.dp % 4 == 0 && P.dp <= 32, "bad padded dimension %d", P.dp);
  P.d = d;
  P.N = N;
  P.kern = kern;
  P.sigma = sigma;
  KRR_TRY(P.xt.alloc((size_t)N * P.dp, s));
  KRR_TRY(P.cn.alloc((size_t)N, s));
  KRR_TRY(P.mean.alloc(d, s));
  if (mean_dev) {
    KRR_CUDA_TRY(cudaMemcpyAsync(P.mean.p, mean_dev, sizeof(double) * d,
                                 cudaMemcpyDeviceToDevice, s));
  } else {
    column_mean_kernel<<<d, 256, 0, s>>>(Xd, N, d, P.mean.p);
    KRR_LAUNCH_CHECK();
  }
  const double log2e = 1.4426950408889634;
  double scale;
  int with_norm = 1;
  if (kern == KGAUSS) {
    scale = std::sqrt(log2e) / sigma;
  } else if (kern == KMATERN) {
    scale = std::sqrt(5.0) / sigma;
  } else {
    scale = log2e / sigma;
    with_norm = 0;
  }
  prepare_f32_kernel<<<ceil_div(N, 256), 256, 0, s>>>(Xd, N, d, P.dp, P.mean.p, scale,
                                                      with_norm, P.xt.p, P.cn.p);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// float-float split of centred, scaled points: x = xh + xl (float), and the
// constant c = -|xh + xl|^2 / 2 split as ch + cl.
__global__ void prepare_ff_kernel(const double *__restrict__ X, int64_t N, int d, int dp,
                                  const double *__restrict__ mean, double scale, int with_norm,
                                  float *__restrict__ xh, float *__restrict__ xl,
                                  float *__restrict__ ch, float *__restrict__ cl) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double nrm = 0.0;
  for (int k = 0; k < dp; ++k) {
    double v = (k < d) ? (X[i * d + k] - mean[k]) * scale : 0.0;
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    xh[i * dp + k] = h;
    xl[i * dp + k] = l;
    const double e = (double)h + (double)l;
    nrm = fma(e, e, nrm);
  }
  const double c = with_norm ? -0.5 * nrm : 0.0;
  const float c_h = (float)c;
  ch[i] = c_h;
  cl[i] = (float)(c - (double)c_h);
}

krr_status prepare_points_ff(const double *Xd, int64_t N, int d, int kern, double sigma,
                             cudaStream_t s, PointsFF &P, const double *mean_dev) {
  P.dp = (d + 3) / 4 * 4;
  P.d = d;
  P.N = N;
  P.kern = kern;
  KRR_TRY(P.xh.alloc((size_t)N * P.dp, s));
  KRR_TRY(P.xl.alloc((size_t)N * P.dp, s));
  KRR_TRY(P.ch.alloc((size_t)N, s));
  KRR_TRY(P.cl.alloc((size_t)N, s));
  KRR_TRY(P.mean.alloc(d, s));
  if (mean_dev) {
    KRR_CUDA_TRY(cudaMemcpyAsync(P.mean.p, mean_dev, sizeof(double) * d,
                                 cudaMemcpyDeviceToDevice, s));
  } else {
    column_mean_kernel<<<d, 256, 0, s>>>(Xd, N, d, P.mean.p);
    KRR_LAUNCH_CHECK();
  }
  const double scale = (kern == KMATERN) ? std::sqrt(5.0) / sigma : 1.0 / sigma;
  const int with_norm = 0;   // the float-float distance uses direct differences
  prepare_ff_kernel<<<ceil_div(N, 256), 256, 0, s>>>(Xd, N, d, P.dp, P.mean.p, scale,
                                                     with_norm, P.xh.p, P.xl.p, P.ch.p, P.cl.p);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

__global__ void split_ff_kernel(const double *__restrict__ V, int64_t ldv, int64_t N, int m,
                                float *__restrict__ vh, float *__restrict__ vl) {
  const int64_t total = N * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / N);
    const int64_t i = e % N;
    const double v = V[(int64_t)c * ldv + i];
    const float h = (float)v;
    vh[e] = h;
    vl[e] = (float)(v - (double)h);
  }
}

// Host-side constants of the float-float exponential (see kmvff_kernels.cuh):
// ln2/32 split into floats (the first with 8 significant bits) and the table
// 2^(j/32), j < 32, as hi + lo floats.  Mathematical constants from the host
// C library in double precision.
static ExpFFConsts make_exp_consts() {
  ExpFFConsts e;
  const double ln2 = 0.69314718055994530942;
  const double c = ln2 / 32.0;
  e.c[0] = (float)(32.0 / ln2);
  int ex = 0;
  const double fr = std::frexp(c, &ex);
  const double c1 = std::ldexp(std::nearbyint(std::ldexp(fr, 8)), ex - 8);
  const double rem = c - c1;
  const float c2 = (float)rem;
  e.c[1] = (float)c1;
  e.c[2] = c2;
  e.c[3] = (float)(rem - (double)c2);
  for (int j = 0; j < 32; ++j) {
    const double t = std::exp2(j / 32.0);
    const float h = (float)t;
    e.tab[2 * j] = h;
    e.tab[2 * j + 1] = (float)(t - (double)h);
  }
  return e;
}

// ---------------------------------------------------------- reduction
template <typename T, int MAXM>
__global__ void kmv_reduce_kernel(const T *__restrict__ part, int splits, int M,
                                  int64_t N, int m, T lambda, const T *__restrict__ V,
                                  int64_t ldv, T *__restrict__ Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int c = 0; c < m; ++c) {
    T acc = 0;
    for (int sp = 0; sp < splits; ++sp) acc += part[((int64_t)sp * M + c) * N + i];
    Y[(int64_t)c * ldy + i] = V ? acc + lambda * V[(int64_t)c * ldv + i] : acc;
  }
}

static int pad_m(int m) {
  if (m <= 1) return 1;
  if (m <= 2) return 2;
  if (m <= 4) return 4;
  if (m <= 8) return 8;
  return 16;
}

// Column splits so the grid is about `waves` full waves of `per_sm` CTAs.
static int choose_splits(int64_t row_tiles, int64_t N, int tj, int per_sm, int waves) {
  const int64_t target = (int64_t)num_sms() * per_sm * waves;
  int64_t splits = (target + row_tiles - 1) / row_tiles;
  const int64_t max_splits = (N + tj - 1) / tj;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  return (int)splits;
}

// ------------------------------------------------------------ autotuner
// The column tile of the float32 products (the columns one CTA covers, set by
// the number of column splits) is chosen per (path, kernel, padded
// dimension, padded m, N) by timing candidate split counts -- the grid at 2,
// 4, 8, 16 and 32 waves -- once, on the caller's stream and data, when
// autotuning is on.  The choice is cached for the process; the default rule
// is 8 waves.  Summation order depends on the split count, so a tuned
// product can differ from an untuned one at the rounding level.
static std::atomic<bool> g_autotune{false};
static std::atomic<int> g_product_path{0};
static std::mutex g_tune_mtx;
static std::map<std::tuple<int, int, int, int, int64_t>, int> g_tuned;

void set_autotune(bool on) { g_autotune.store(on); }
bool autotune_on() { return g_autotune.load(); }
void set_product_path(int path) { g_product_path.store(path); }
int product_path() { return g_product_path.load(); }

// Path a float32 product of this shape takes: 1 tensor cores, 0 FMA.
static int path_of(int kern, int dp) {
  return (g_product_path.load() != 1 && kern != KLAPLACE && dp <= 32) ? 1 : 0;
}

int tuned_splits(int kern, int dp, int M, int64_t N) {
  const int path = path_of(kern, dp);
  const int dim = path ? (dp + 15) / 16 : dp;
  const int Mk = path ? (M > 8 ? 8 : M) : M;
  std::lock_guard<std::mutex> lk(g_tune_mtx);
  auto it = g_tuned.find(std::make_tuple(path, kern, dim, Mk, N));
  return it == g_tuned.end() ? 0 : it->second;
}

// chunk (a multiple of tj) and split count for `splits` requested splits
static void split_shape(int64_t N, int splits, int tj, int64_t *chunk, int *nsplit) {
  int64_t c = (N + splits - 1) / splits;
  c = (c + tj - 1) / tj * tj;
  *chunk = c;
  *nsplit = (int)((N + c - 1) / c);
}

// launch(chunk, nsplit, part) issues one product with that column split.
template <typename Launch>
static int choose_product_splits(int path, int kern, int dim, int M, int64_t N,
                                 int64_t row_tiles, int tj, int per_sm, DevBuf<float> &part,
                                 cudaStream_t s, Launch launch) {
  const int dflt = choose_splits(row_tiles, N, tj, per_sm, 8);
  if (!g_autotune.load()) return dflt;
  const auto key = std::make_tuple(path, kern, dim, M, N);
  {
    std::lock_guard<std::mutex> lk(g_tune_mtx);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return dflt;   // timing would synchronise a capturing stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return dflt;
  }
  int best = dflt;
  float best_ms = 1e30f;
  int last = -1;
  for (int waves : {2, 4, 8, 16, 32}) {
    const int splits = choose_splits(row_tiles, N, tj, per_sm, waves);
    if (splits == last) continue;
    last = splits;
    int64_t chunk;
    int nsplit;
    split_shape(N, splits, tj, &chunk, &nsplit);
    const size_t need = (size_t)nsplit * M * N;
    if (part.n < need && part.alloc(need, s) != KRR_OK) break;
    float ms = 0.0f;
    bool ok = cudaEventRecord(e0, s) == cudaSuccess;
    ok = ok && launch(chunk, nsplit, part.p) == cudaSuccess;
    count_launch();
    ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = splits;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mtx);
  g_tuned[key] = best;
  return best;
}

// Tensor-core product over right-hand-side groups of at most 8.
static krr_status kmv_tc(const PointsF32 &P, float lambda, const float *V, int64_t ldv, int m,
                         float *Y, int64_t ldy, cudaStream_t s, DevBuf<float> &part) {
  const int64_t N = P.N;
  const int KC = P.kc16;
  for (int c0 = 0; c0 < m; c0 += 8) {
    const int mg = (m - c0 < 8) ? (m - c0) : 8;
    const int M = pad_m(mg);
    const int64_t row_tiles = (N + kmvtc_rows_per_cta(KC, M) - 1) / kmvtc_rows_per_cta(KC, M);
    const float *Vg = V + (int64_t)c0 * ldv;
    auto launch = [&](int64_t chunk, int nsplit, float *pp) {
      const KmvTcArgs a{P.xs16.p, P.cs16.p, Vg, ldv, N, mg, chunk, pp};
      return launch_kmvtc(P.kern, KC, M, dim3((unsigned)row_tiles, nsplit), s, a);
    };
    const int splits =
        choose_product_splits(1, P.kern, KC, M, N, row_tiles, KTC_TJ, 1, part, s, launch);
    int64_t chunk;
    int nsplit;
    split_shape(N, splits, KTC_TJ, &chunk, &nsplit);
    const size_t need = (size_t)nsplit * M * N;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    KmvTimer tm;
    tm.begin(s);
    cudaError_t e = launch(chunk, nsplit, part.p);
    tm.end(s);
    count_launch();
    if (e != cudaSuccess) {
      set_error("tensor-core product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<float, 16><<<ceil_div(N, 256), 256, 0, s>>>(
        part.p, nsplit, M, N, mg, lambda, Vg, ldv, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

krr_status kmv_f32(const PointsF32 &P, float lambda, const float *V, int64_t ldv, int m,
                   float *Y, int64_t ldy, cudaStream_t s, DevBuf<float> &part) {
  const int64_t N = P.N;
  if (N == 0 || m == 0) return KRR_OK;
  if (P.nh5 > 0 && g_product_path.load() == 0)
    return kmv_tc5(P, P, lambda, true, V, ldv, m, Y, ldy, s, part);
  if (P.kc16 > 0 && path_of(P.kern, P.dp) == 1)
    return kmv_tc(P, lambda, V, ldv, m, Y, ldy, s, part);
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    const int rows = KMV_THREADS * kmv32_rows_per_thread(P.dp, M);
    const int64_t row_tiles = (N + rows - 1) / rows;
    const float *Vg = V + (int64_t)c0 * ldv;
    auto launch = [&](int64_t chunk, int nsplit, float *pp) {
      const Kmv32Args a{P.xt.p, P.cn.p, N, P.xt.p, P.cn.p, Vg, ldv, N, mg, chunk, pp};
      return launch_kmv32_any(P.kern, P.dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    };
    const int splits =
        choose_product_splits(0, P.kern, P.dp, M, N, row_tiles, KMV_TJ, 2, part, s, launch);
    int64_t chunk;
    int nsplit;
    split_shape(N, splits, KMV_TJ, &chunk, &nsplit);
    const size_t need = (size_t)nsplit * M * N;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    KmvTimer tm;
    tm.begin(s);
    cudaError_t e = launch(chunk, nsplit, part.p);
    tm.end(s);
    count_launch();
    if (e != cudaSuccess) {
      set_error("fused product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<float, 16><<<ceil_div(N, 256), 256, 0, s>>>(
        part.p, nsplit, M, N, mg, lambda, Vg, ldv, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

krr_status kmv_f64(const double *Xd, int64_t N, int d, int kern, double sigma,
                   double lambda, const double *V, int64_t ldv, int m, double *Y,
                   int64_t ldy, cudaStream_t s, DevBuf<double> &part) {
  if (N == 0 || m == 0) return KRR_OK;
  const int dp = (d + 3) / 4 * 4;
  double inv_scale = (kern == KGAUSS) ? 1.0 / (2.0 * sigma * sigma) : 1.0 / sigma;
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    const int64_t row_tiles = (N + KMV64_THREADS - 1) / KMV64_THREADS;
    const int splits = choose_splits(row_tiles, N, KMV64_TJ, 4, 4);
    int64_t chunk = (N + splits - 1) / splits;
    chunk = (chunk + KMV64_TJ - 1) / KMV64_TJ * KMV64_TJ;
    const int nsplit = (int)((N + chunk - 1) / chunk);
    const size_t need = (size_t)nsplit * M * N;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    Kmv64Args a{Xd, N, Xd, d, V + (int64_t)c0 * ldv, ldv, N, mg, chunk, inv_scale, part.p};
    KmvTimer tm(1);
    tm.begin(s);
    cudaError_t e = launch_kmv64_any(kern, dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    tm.end(s);
    count_launch();
    if (e != cudaSuccess) {
      set_error("float64 product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<double, 16><<<ceil_div(N, 256), 256, 0, s>>>(
        part.p, nsplit, M, N, mg, lambda, V + (int64_t)c0 * ldv, ldv,
        Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

__global__ void kmvffsym_reduce_kernel(const double *__restrict__ rowpart,
                                       const double *__restrict__ colpart,
                                       const int *__restrict__ seg0, int64_t N, int m, int M,
                                       int RT, int nt, int64_t T, int G, int J, double lambda,
                                       const double *__restrict__ V, int64_t ldv,
                                       double *__restrict__ Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int t = (int)(i / RT), r = (int)(i % RT);
  const int64_t st = ffsym_start(t, nt);
  const int b_lo = ffsym_cta_of(st, T, G), b_hi = ffsym_cta_of(st + (nt - t) - 1, T, G);
  for (int c = 0; c < m; ++c) {
    double acc = 0.0;
    for (int b = b_lo; b <= b_hi; ++b)
      acc += rowpart[(((int64_t)b * J + (t - seg0[b])) * M + c) * RT + r];
    for (int I = 0; I < t; ++I)
      acc += colpart[((ffsym_start(I, nt) + (t - I)) * M + c) * RT + r];
    Y[(int64_t)c * ldy + i] = acc + lambda * V[(int64_t)c * ldv + i];
  }
}

// Geometry of the symmetric float-float product: nt tiles of RT points, T
// pairs of the upper triangle over G CTAs, J segments per CTA at most.
struct FFSymGeometry {
  int RT = 0, nt = 0, G = 0, J = 1;
  int64_t T = 0;
};

static FFSymGeometry ffsym_geometry(int64_t N, int DP) {
  FFSymGeometry g;
  g.RT = KFF_THREADS * kmvff_rows_per_thread(DP);
  g.nt = (int)((N + g.RT - 1) / g.RT);
  g.T = (int64_t)g.nt * (g.nt + 1) / 2;
  g.G = (int)std::min<int64_t>((int64_t)num_sms() * kmvff_min_blocks(DP), g.T);
  for (int b = 0; b < g.G; ++b) {
    const int64_t p0 = (int64_t)b * g.T / g.G, p1 = (int64_t)(b + 1) * g.T / g.G;
    if (p1 > p0) g.J = std::max(g.J, ffsym_row(p1 - 1, g.nt) - ffsym_row(p0, g.nt) + 1);
  }
  return g;
}

// The symmetric product serves square products with up to 4 right-hand sides
// per launch when there are at least 4 pairs per CTA (smaller problems keep
// the column-split kernel, which fills the GPU better) and its column sums
// (8 T M RT bytes) stay within 4 GiB.
static bool ffsym_fits(const FFSymGeometry &g, int M) {
  return M <= 4 && g.T >= 4 * (int64_t)g.G &&
         (double)g.T * M * g.RT * 8.0 <= 4.0 * 1024 * 1024 * 1024;
}

// Y (Nr x m) = K(R, P) V (+ lambda V when R is P and lambda != 0): the
// float-float product between a row point set R and a column set P prepared
// with the same centre and scale.
krr_status kff_cross(const PointsFF &R, const PointsFF &P, double lambda, const double *V,
                     int64_t ldv, int m, double *Y, int64_t ldy, cudaStream_t s,
                     DevBuf<double> &part, DevBuf<float> &vsplit) {
  const int64_t N = P.N, Nr = R.N;
  if (N == 0 || Nr == 0 || m == 0) return KRR_OK;
  static const ExpFFConsts ec = make_exp_consts();
  if (vsplit.n < (size_t)2 * N * m) KRR_TRY(vsplit.alloc((size_t)2 * N * m, s));
  float *vh = vsplit.p, *vl = vsplit.p + (size_t)N * m;
  {
    int64_t g = (N * m + 255) / 256;
    if (g > num_sms() * 16) g = num_sms() * 16;
    split_ff_kernel<<<(unsigned)g, 256, 0, s>>>(V, ldv, N, m, vh, vl);
    KRR_LAUNCH_CHECK();
  }
  const bool square = (&R == &P);
  const FFSymGeometry sg = ffsym_geometry(N, P.dp);
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    if (square && ffsym_fits(sg, M)) {
      // rowpart | colpart | seg0
      const size_t nrow = (size_t)sg.G * sg.J * M * sg.RT, ncol = (size_t)sg.T * M * sg.RT;
      const size_t need = nrow + ncol + (sg.G + 1) / 2;
      if (part.n < need) KRR_TRY(part.alloc(need, s));
      int *seg0 = reinterpret_cast<int *>(part.p + nrow + ncol);
      KmvFFSymArgs a{P.xh.p, P.xl.p, vh + (int64_t)c0 * N, vl + (int64_t)c0 * N, N, mg, sg.nt,
                     sg.T, sg.J, ec, part.p, part.p + nrow, seg0};
      KmvTimer tm(2);
      tm.begin(s);
      cudaError_t e = launch_kmvffsym_any(P.kern, P.dp, M, sg.G, s, a);
      tm.end(s);
      count_launch();
      if (e != cudaSuccess) {
        set_error("float-float product launch failed: %s", cudaGetErrorString(e));
        return KRR_ECUDA;
      }
      kmvffsym_reduce_kernel<<<ceil_div(N, 256), 256, 0, s>>>(
          part.p, part.p + nrow, seg0, N, mg, M, sg.RT, sg.nt, sg.T, sg.G, sg.J, lambda,
          V + (int64_t)c0 * ldv, ldv, Y + (int64_t)c0 * ldy, ldy);
      KRR_LAUNCH_CHECK();
      continue;
    }
    const int rows = KFF_THREADS * kmvff_rows_per_thread(P.dp);
    const int64_t row_tiles = (Nr + rows - 1) / rows;
    const int splits = choose_splits(row_tiles, N, KFF_TJ, 4, 6);
    int64_t chunk = (N + splits - 1) / splits;
    chunk = (chunk + KFF_TJ - 1) / KFF_TJ * KFF_TJ;
    const int nsplit = (int)((N + chunk - 1) / chunk);
    const size_t need = (size_t)nsplit * M * Nr;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    KmvFFArgs a{R.xh.p, R.xl.p, Nr, P.xh.p, P.xl.p, P.ch.p, P.cl.p, vh + (int64_t)c0 * N,
                vl + (int64_t)c0 * N, N, mg, chunk, ec, part.p};
    KmvTimer tm(2);
    tm.begin(s);
    cudaError_t e = launch_kmvff_any(P.kern, P.dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    tm.end(s);
    count_launch();
    if (e != cudaSuccess) {
      set_error("float-float product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<double, 16><<<ceil_div(Nr, 256), 256, 0, s>>>(
        part.p, nsplit, M, Nr, mg, square ? lambda : 0.0,
        square ? V + (int64_t)c0 * ldv : nullptr, ldv, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

krr_status kmv_ff(const PointsFF &P, double lambda, const double *V, int64_t ldv, int m,
                  double *Y, int64_t ldy, cudaStream_t s, DevBuf<double> &part,
                  DevBuf<float> &vsplit) {
  return kff_cross(P, P, lambda, V, ldv, m, Y, ldy, s, part, vsplit);
}

// Prediction products Y (Nr x m) = K(Xr, X) V, V N x m (no shift).
krr_status kcross_f32(const PointsF32 &R, const PointsF32 &P, const float *V, int64_t ldv,
                      int m, float *Y, int64_t ldy, cudaStream_t s, DevBuf<float> &part) {
  const int64_t N = P.N, Nr = R.N;
  if (N == 0 || Nr == 0 || m == 0) return KRR_OK;
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    const int rows = KMV_THREADS * kmv32_rows_per_thread(P.dp, M);
    const int64_t row_tiles = (Nr + rows - 1) / rows;
    const int splits = choose_splits(row_tiles, N, KMV_TJ, 2, 8);
    int64_t chunk = (N + splits - 1) / splits;
    chunk = (chunk + KMV_TJ - 1) / KMV_TJ * KMV_TJ;
    const int nsplit = (int)((N + chunk - 1) / chunk);
    const size_t need = (size_t)nsplit * M * Nr;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    Kmv32Args a{R.xt.p, R.cn.p, Nr, P.xt.p, P.cn.p, V + (int64_t)c0 * ldv, ldv, N, mg, chunk,
                part.p};
    cudaError_t e = launch_kmv32_any(P.kern, P.dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    count_launch();
    if (e != cudaSuccess) {
      set_error("prediction product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<float, 16><<<ceil_div(Nr, 256), 256, 0, s>>>(
        part.p, nsplit, M, Nr, mg, 0.0f, nullptr, 0, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

krr_status kcross_f64(const double *Xr, int64_t Nr, const double *Xd, int64_t N, int d,
                      int kern, double sigma, const double *V, int64_t ldv, int m, double *Y,
                      int64_t ldy, cudaStream_t s, DevBuf<double> &part) {
  if (N == 0 || Nr == 0 || m == 0) return KRR_OK;
  const int dp = (d + 3) / 4 * 4;
  double inv_scale = (kern == KGAUSS) ? 1.0 / (2.0 * sigma * sigma) : 1.0 / sigma;
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    const int64_t row_tiles = (Nr + KMV64_THREADS - 1) / KMV64_THREADS;
    const int splits = choose_splits(row_tiles, N, KMV64_TJ, 4, 4);
    int64_t chunk = (N + splits - 1) / splits;
    chunk = (chunk + KMV64_TJ - 1) / KMV64_TJ * KMV64_TJ;
    const int nsplit = (int)((N + chunk - 1) / chunk);
    const size_t need = (size_t)nsplit * M * Nr;
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    Kmv64Args a{Xr, Nr, Xd, d, V + (int64_t)c0 * ldv, ldv, N, mg, chunk, inv_scale, part.p};
    cudaError_t e = launch_kmv64_any(kern, dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    count_launch();
    if (e != cudaSuccess) {
      set_error("prediction product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<double, 16><<<ceil_div(Nr, 256), 256, 0, s>>>(
        part.p, nsplit, M, Nr, mg, 0.0, nullptr, 0, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

// Same product with caller-provided split scratch of `scratch_elems` doubles:
// the column split count is reduced until the partial sums fit.  Launches
// only the product and reduction kernels (no allocation).
krr_status kmv_f64_with_scratch(const double *Xd, int64_t N, int d, int kern, double sigma,
                                double lambda, const double *V, int64_t ldv, int m, double *Y,
                                int64_t ldy, double *scratch, size_t scratch_elems,
                                cudaStream_t s) {
  if (N == 0 || m == 0) return KRR_OK;
  const int dp = (d + 3) / 4 * 4;
  double inv_scale = (kern == KGAUSS) ? 1.0 / (2.0 * sigma * sigma) : 1.0 / sigma;
  for (int c0 = 0; c0 < m; c0 += 16) {
    const int mg = (m - c0 < 16) ? (m - c0) : 16;
    const int M = pad_m(mg);
    if ((size_t)M * (size_t)N > scratch_elems) {
      set_error("scratch of %zu doubles cannot hold N x %d = %lld partial sums", scratch_elems,
                M, (long long)N * M);
      return KRR_EINVAL;
    }
    const int64_t row_tiles = (N + KMV64_THREADS - 1) / KMV64_THREADS;
    int splits = choose_splits(row_tiles, N, KMV64_TJ, 4, 4);
    const int64_t fit = (int64_t)(scratch_elems / ((size_t)M * (size_t)N));
    if (splits > fit) splits = (int)fit;
    int64_t chunk = (N + splits - 1) / splits;
    chunk = (chunk + KMV64_TJ - 1) / KMV64_TJ * KMV64_TJ;
    const int nsplit = (int)((N + chunk - 1) / chunk);
    Kmv64Args a{Xd, N, Xd, d, V + (int64_t)c0 * ldv, ldv, N, mg, chunk, inv_scale, scratch};
    cudaError_t e = launch_kmv64_any(kern, dp, M, dim3((unsigned)row_tiles, nsplit), s, a);
    count_launch();
    if (e != cudaSuccess) {
      set_error("float64 product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    kmv_reduce_kernel<double, 16><<<ceil_div(N, 256), 256, 0, s>>>(
        scratch, nsplit, M, N, mg, lambda, V + (int64_t)c0 * ldv, ldv,
        Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

// ------------------------------------------------------- conversions
__global__ void f64_to_f32_kernel(const double *__restrict__ a, float *__restrict__ b,
                                  int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f32_to_f64_kernel(const float *__restrict__ a, double *__restrict__ b,
                                  int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

krr_status convert_f64_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s) {
  if (n == 0) return KRR_OK;
  f64_to_f32_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status convert_f32_to_f64(const float *src, double *dst, int64_t n, cudaStream_t s) {
  if (n == 0) return KRR_OK;
  f32_to_f64_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ---------------------------------------------------- kernel columns
// One thread per (row, column) pair; the selected points are staged in
// shared memory (nc <= 128 points of <= 32 coordinates).
__global__ void kernel_columns_kernel(const double *__restrict__ X, int64_t N, int d,
                                      int kern, double sigma,
                                      const int64_t *__restrict__ cols, int nc,
                                      double *__restrict__ G, int64_t ldg) {
  extern __shared__ double sp[];
  for (int idx = threadIdx.x; idx < nc * d; idx += blockDim.x)
    sp[idx] = X[cols[idx / d] * d + idx % d];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double xi[32];
  for (int k = 0; k < d; ++k) xi[k] = X[i * d + k];
  for (int c = 0; c < nc; ++c)
    G[(int64_t)c * ldg + i] = kappa_point_f64(xi, sp + c * d, d, kern, sigma);
}

krr_status kernel_columns_f64(const double *Xd, int64_t N, int d, int kern, double sigma,
                              const int64_t *cols, int nc, double *G, int64_t ldg,
                              cudaStream_t s) {
  if (nc == 0 || N == 0) return KRR_OK;
  for (int c0 = 0; c0 < nc; c0 += 128) {
    const int ncg = (nc - c0 < 128) ? nc - c0 : 128;
    const size_t smem = (size_t)ncg * d * sizeof(double);
    KRR_TRY(raise_smem_limit(kernel_columns_kernel, smem));
    kernel_columns_kernel<<<ceil_div(N, 128), 128, smem, s>>>(
        Xd, N, d, kern, sigma, cols + c0, ncg, G + (int64_t)c0 * ldg, ldg);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

__global__ void kernel_diag_kernel(const double *__restrict__ X, int64_t N, int d,
                                   int kern, double sigma, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  out[i] = kappa_point_f64(X + i * d, X + i * d, d, kern, sigma);
}

krr_status kernel_diag_f64(const double *Xd, int64_t N, int d, int kern, double sigma,
                           double *out, cudaStream_t s) {
  if (N == 0) return KRR_OK;
  kernel_diag_kernel<<<ceil_div(N, 256), 256, 0, s>>>(Xd, N, d, kern, sigma, out);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

}  // namespace krr
