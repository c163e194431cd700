// Alg. 1 preconditioner (Woodbury form of the paper's SVD form) and PCG
// (Sec. 3: zero initial iterate, stop on the recursive relative residual),
// plus the mixed-precision iterative refinement around a float32 inner PCG.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>

#include "dense.cuh"
#include "kmv.cuh"
#include "pcg.cuh"
#include "rpc.cuh"

namespace krr {

// ------------------------------------------------ tall skinny products
// The Woodbury apply streams F (N x rank) twice: t = F^T r and z = r - F v.
// Both are HBM-bound; products and in-block sums use the precision of the
// data (float32 in the mixed path, float64 otherwise), sums across blocks are
// float64, in a fixed order.
constexpr int TT_ROWS = 512;   // rows per block of the transposed product
constexpr int RED_BLOCKS = 512;

// part[b][l][c] = sum_{n in block b} F[n + l N] R[c][n]
// Block (b, g) covers rows [b TT_ROWS, (b + 1) TT_ROWS) and the columns
// [g TT_COLS, (g + 1) TT_COLS) (column groups give enough blocks to stream F
// at HBM speed).  One warp per column; each lane holds TT_ROWS/32 rows, all
// loaded before any arithmetic so that many loads are in flight.  M is m
// rounded up to 1, 2, 4, 8 or 16 (specialised: a runtime column count costs
// the unrolled loops several times their work).
constexpr int TT_COLS = 64;

template <typename T, int M>
__global__ void __launch_bounds__(256)
tall_t_kernel(const T *__restrict__ F, int64_t N, int rank, const T *__restrict__ R, int m,
              double *__restrict__ part) {
  constexpr int PER_LANE = TT_ROWS / 32;
  __shared__ T sR[M][TT_ROWS];
  const int64_t n0 = (int64_t)blockIdx.x * TT_ROWS;
  const int nr = (int)min((int64_t)TT_ROWS, N - n0);
  for (int e = threadIdx.x; e < m * TT_ROWS; e += blockDim.x) {
    const int c = e / TT_ROWS, n = e % TT_ROWS;
    sR[c][n] = (n < nr) ? R[(int64_t)c * N + n0 + n] : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int l1 = min(rank, (int)(blockIdx.y + 1) * TT_COLS);
  // two columns per pass: each R value read from shared memory serves both
  for (int l = (int)blockIdx.y * TT_COLS + warp; l < l1; l += 2 * nw) {
    const bool two = l + nw < l1;
    const T *col = F + (int64_t)l * N + n0;
    const T *col2 = col + (int64_t)nw * N;
    T f[PER_LANE], g[PER_LANE];
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
      const int n = lane + 32 * q;
      f[q] = (n < nr) ? col[n] : T(0);
      g[q] = (two && n < nr) ? col2[n] : T(0);
    }
    T acc[M], acc2[M];
#pragma unroll
    for (int c = 0; c < M; ++c) acc[c] = acc2[c] = T(0);
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        if (c < m) {
          const T r = sR[c][lane + 32 * q];
          acc[c] = fma(f[q], r, acc[c]);
          acc2[c] = fma(g[q], r, acc2[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if (c < m) {
        const T v = warp_sum(acc[c]);
        const T v2 = warp_sum(acc2[c]);
        if (lane == 0) {
          part[((int64_t)blockIdx.x * rank + l) * m + c] = (double)v;
          if (two) part[((int64_t)blockIdx.x * rank + l + nw) * m + c] = (double)v2;
        }
      }
    }
  }
}

// t[c][l] = sum_b part[b][l][c], one warp per (l, c), blocks summed in a
// fixed lane-strided order then a fixed shuffle tree.
__global__ void tall_t_reduce_kernel(const double *__restrict__ part, int nb, int rank, int m,
                                     double *__restrict__ t) {
  const int warps = blockDim.x >> 5;
  const int e = blockIdx.x * warps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= rank * m) return;
  const int l = e / m, c = e % m;
  double acc = 0.0;
  for (int b = lane; b < nb; b += 32) acc += part[((int64_t)b * rank + l) * m + c];
  acc = warp_sum(acc);
  if (lane == 0) t[(int64_t)c * rank + l] = acc;
}

// Triangular products with one block of TRI_THREADS threads per output row,
// reading contiguous columns of a column-major rank x rank matrix Mt:
//   UPPER == false: out[c][i] = sum_{l <= i} Mt[l + i rank] x[c][l]
//   UPPER == true : out[c][i] = sum_{l >= i} Mt[l + i rank] x[c][l]
// With Mt = W^T (W lower) the first is W x; with Mt = W the second is W^T x.
// A row is split across four warps (a row of about rank / 2 entries per warp
// would leave too few loads in flight to stream Mt); per column the warps'
// sums are added in warp order.
constexpr int TRI_THREADS = 128;

template <bool UPPER, int M>
__global__ void __launch_bounds__(TRI_THREADS)
tri_gemv_kernel(const double *__restrict__ Mt, int rank, const double *__restrict__ x, int m,
                double *__restrict__ out) {
  __shared__ double red[TRI_THREADS / 32][M];
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[M];
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0;
  const double *col = Mt + (int64_t)i * rank;
  const int lo = UPPER ? i : 0, hi = UPPER ? rank : i + 1;
  for (int l = lo + threadIdx.x; l < hi; l += TRI_THREADS) {
    const double w = col[l];
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < m) acc[c] = fma(w, x[(int64_t)c * rank + l], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < M; ++c) {
    if (c < m) {
      const double v = warp_sum(acc[c]);
      if (lane == 0) red[warp][c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < TRI_THREADS / 32; ++w) t += red[w][threadIdx.x];
    out[(int64_t)threadIdx.x * rank + i] = t;
  }
}

// Launches tri_gemv_kernel specialised on m rounded up to 1, 2, 4, 8 or 16
// (a runtime column count costs the unrolled loops their full 16-wide work).
template <bool UPPER>
static void launch_tri_gemv(const double *Mt, int rank, const double *x, int m, double *out,
                            cudaStream_t s) {
  const int p = m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16;
  switch (p) {
    case 1: tri_gemv_kernel<UPPER, 1><<<rank, TRI_THREADS, 0, s>>>(Mt, rank, x, m, out); break;
    case 2: tri_gemv_kernel<UPPER, 2><<<rank, TRI_THREADS, 0, s>>>(Mt, rank, x, m, out); break;
    case 4: tri_gemv_kernel<UPPER, 4><<<rank, TRI_THREADS, 0, s>>>(Mt, rank, x, m, out); break;
    case 8: tri_gemv_kernel<UPPER, 8><<<rank, TRI_THREADS, 0, s>>>(Mt, rank, x, m, out); break;
    default: tri_gemv_kernel<UPPER, 16><<<rank, TRI_THREADS, 0, s>>>(Mt, rank, x, m, out); break;
  }
}

// Z[c][n] = (R[c][n] - sum_l F[n + l N] v[c][l]) / lambda
// One thread per row (blocks of TN_THREADS); the column loop loads LU
// values of F before using them so that enough loads are in flight to stream
// F at HBM speed.  M as above.
template <typename T, int M>
__global__ void __launch_bounds__(256)
tall_n_kernel(const T *__restrict__ F, int64_t N, int rank, const double *__restrict__ v,
              int m, const T *__restrict__ R, double inv_lambda, T *__restrict__ Z) {
  constexpr int LCH = 256;
  constexpr int LU = 32;
  __shared__ T sv[LCH][M];
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = n < N;
  T acc[M];
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = T(0);
  for (int l0 = 0; l0 < rank; l0 += LCH) {
    const int nl = min(LCH, rank - l0);
    __syncthreads();
    for (int e = threadIdx.x; e < M * LCH; e += blockDim.x) {
      const int c = e / LCH, l = e % LCH;
      sv[l][c] = (l < nl && c < m) ? (T)v[(int64_t)c * rank + l0 + l] : T(0);
    }
    __syncthreads();
    for (int lb = 0; lb < nl; lb += LU) {
      T f[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u)
        f[u] = (ok && lb + u < nl) ? F[n + (int64_t)(l0 + lb + u) * N] : T(0);
#pragma unroll
      for (int u = 0; u < LU; ++u) {
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = fma(f[u], sv[lb + u][c], acc[c]);
      }
    }
  }
  if (ok) {
#pragma unroll
    for (int c = 0; c < M; ++c)
      if (c < m)
        Z[(int64_t)c * N + n] =
            (T)(((double)R[(int64_t)c * N + n] - (double)acc[c]) * inv_lambda);
  }
}

static int tall_pad_m(int m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16; }

template <typename T>
static krr_status launch_tall_t(const T *F, int64_t N, int rank, const T *R, int m,
                                double *part, cudaStream_t s) {
  const dim3 grid(ceil_div(N, TT_ROWS), ceil_div(rank, TT_COLS));
  switch (tall_pad_m(m)) {
    case 1: tall_t_kernel<T, 1><<<grid, 256, 0, s>>>(F, N, rank, R, m, part); break;
    case 2: tall_t_kernel<T, 2><<<grid, 256, 0, s>>>(F, N, rank, R, m, part); break;
    case 4: tall_t_kernel<T, 4><<<grid, 256, 0, s>>>(F, N, rank, R, m, part); break;
    case 8: tall_t_kernel<T, 8><<<grid, 256, 0, s>>>(F, N, rank, R, m, part); break;
    default: tall_t_kernel<T, 16><<<grid, 256, 0, s>>>(F, N, rank, R, m, part); break;
  }
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// Blocks of 64 threads: about ten per SM at N = 1e5, so the last wave of
// blocks leaves few SMs idle (256-thread blocks left 2.6 per SM).
constexpr int TN_THREADS = 64;

template <typename T>
static krr_status launch_tall_n(const T *F, int64_t N, int rank, const double *v, int m,
                                const T *R, double inv_lambda, T *Z, cudaStream_t s) {
  const unsigned grid = ceil_div(N, TN_THREADS);
  constexpr int B = TN_THREADS;
  switch (tall_pad_m(m)) {
    case 1: tall_n_kernel<T, 1><<<grid, B, 0, s>>>(F, N, rank, v, m, R, inv_lambda, Z); break;
    case 2: tall_n_kernel<T, 2><<<grid, B, 0, s>>>(F, N, rank, v, m, R, inv_lambda, Z); break;
    case 4: tall_n_kernel<T, 4><<<grid, B, 0, s>>>(F, N, rank, v, m, R, inv_lambda, Z); break;
    case 8: tall_n_kernel<T, 8><<<grid, B, 0, s>>>(F, N, rank, v, m, R, inv_lambda, Z); break;
    default: tall_n_kernel<T, 16><<<grid, B, 0, s>>>(F, N, rank, v, m, R, inv_lambda, Z); break;
  }
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

template <typename T>
static krr_status nystrom_apply_impl(const T *F, int64_t N, int rank, const double *W,
                                     const double *Wt, double lambda, const T *R, int m, T *Z,
                                     cudaStream_t s, PrecondWs *ws) {
  if (rank == 0) {
    // P = lambda I
    return launch_tall_n<T>(F, N, 0, nullptr, m, R, 1.0 / lambda, Z, s);
  }
  const int nb = ceil_div(N, TT_ROWS);
  PrecondWs local;
  PrecondWs &w = ws ? *ws : local;
  auto grow = [&](DevBuf<double> &b, size_t n) {
    return b.n < n ? b.alloc(n, s) : KRR_OK;
  };
  KRR_TRY(grow(w.part, (size_t)nb * rank * m));
  KRR_TRY(grow(w.t, (size_t)rank * m));
  KRR_TRY(grow(w.u, (size_t)rank * m));
  KRR_TRY(grow(w.v, (size_t)rank * m));
  KRR_TRY(launch_tall_t<T>(F, N, rank, R, m, w.part.p, s));
  tall_t_reduce_kernel<<<ceil_div((int64_t)rank * m, 8), 256, 0, s>>>(w.part.p, nb, rank, m,
                                                                    w.t.p);
  KRR_LAUNCH_CHECK();
  KRR_TRY(tri_apply_lower(Wt, rank, w.t.p, m, w.u.p, s));
  KRR_TRY(tri_apply_lower_t(W, rank, w.u.p, m, w.v.p, s));
  return launch_tall_n<T>(F, N, rank, w.v.p, m, R, 1.0 / lambda, Z, s);
}

krr_status nystrom_apply_f64(const krr_factor *f, const NystromCore *c, const double *R,
                             int m, double *Z, cudaStream_t s, PrecondWs *ws) {
  return nystrom_apply_impl<double>(f->F, f->N, c->rank, c->W, c->Wt, c->lambda, R, m, Z, s,
                                    ws);
}

krr_status nystrom_apply_f32(const krr_factor *f, const NystromCore *c, const float *R,
                             int m, float *Z, cudaStream_t s, PrecondWs *ws) {
  return nystrom_apply_impl<float>(c->F32, f->N, c->rank, c->W, c->Wt, c->lambda, R, m, Z, s,
                                   ws);
}

// ------------------------------------------------------- core build
krr_status nystrom_core(const krr_factor *f, double mu, int prec, cudaStream_t s,
                        const NystromCore **out) {
  std::lock_guard<std::mutex> lk(f->mtx);
  for (const auto &c : f->cores)
    if (c.mu == mu && c.prec == prec) {
      *out = &c;
      return KRR_OK;
    }
  auto t0 = std::chrono::steady_clock::now();
  NystromCore c;
  c.mu = mu;
  c.prec = prec;
  c.lambda = mu * (double)f->N;
  c.rank = f->rank;
  const int r = f->rank;
  const int64_t N = f->N;
  if (r > 0) {
    DevBuf<double> Gm;
    KRR_TRY(Gm.alloc((size_t)r * r, s));
    if (prec == KRR_PREC_MIXED) {
      // the mixed preconditioner is built from F rounded to float32, so that
      // it is exactly P^{-1} for that factor (up to the Gram accumulation)
      KRR_TRY(dev_alloc(&c.F32, (size_t)N * r));
      KRR_TRY(convert_f64_to_f32(f->F, c.F32, N * r, s));
      KRR_TRY(gram_lower<float>(c.F32, N, r, Gm.p, s));
    } else {
      KRR_TRY(gram_lower<double>(f->F, N, r, Gm.p, s));
    }
    KRR_TRY(add_diagonal(Gm.p, r, r, c.lambda, s));
    krr_status st = potrf_lower(Gm.p, r, r, s);
    if (st != KRR_OK) {
      dev_free(c.F32, f->free_stream);
      return st;
    }
    KRR_TRY(dev_alloc(&c.W, (size_t)r * r));
    KRR_TRY(trinv_lower(Gm.p, r, r, c.W, s));
    KRR_TRY(dev_alloc(&c.Wt, (size_t)r * r));
    KRR_TRY(transpose_square(c.W, r, c.Wt, s));
    KRR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  c.build_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  f->cores.push_back(c);
  *out = &f->cores.back();
  return KRR_OK;
}

// ---------------------------------------------------------- PCG kernels
template <typename T>
__global__ void dots_kernel(const T *__restrict__ a, const T *__restrict__ b, int64_t N,
                            int m, double *__restrict__ part) {
  __shared__ double red[32];
  for (int c = 0; c < m; ++c) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
      s = fma((double)a[(int64_t)c * N + i], (double)b[(int64_t)c * N + i], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      part[(int64_t)c * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// Sum of the nb block partials of column c by one warp: lane l adds partials
// l, l + 32, ... in order, then a fixed shuffle tree (every lane gets the same
// bits).  The scalar kernels below run one warp per column (32 m threads).
__device__ double sum_parts(const double *part, int nb, int c, int lane) {
  double t = 0.0;
  for (int b = lane; b < nb; b += 32) t += part[(int64_t)c * nb + b];
  return warp_sum(t);
}

// alpha_c = rz_c / (p_c . q_c) for active columns; breakdown flag otherwise.
__global__ void pcg_alpha_kernel(const double *__restrict__ part, int nb, int m,
                                 PcgScalars *__restrict__ sc) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= m) return;
  const double pq = sum_parts(part, nb, c, lane);
  if (lane != 0) return;
  double a = 0.0;
  if (sc->active[c]) {
    if (!(pq > 0.0)) {
      sc->breakdown = 1;
      sc->active[c] = 0;
    } else {
      a = sc->rz[c] / pq;
    }
  }
  sc->alpha[c] = a;
}

// Convergence test on the recursive residual; advances the iteration
// counter (every thread reads it before thread 0 writes it).
__global__ void pcg_resid_kernel(const double *__restrict__ part, int nb, int m,
                                 PcgScalars *__restrict__ sc) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it = sc->it + 1;
  __syncthreads();
  if (threadIdx.x == 0) sc->it = it;
  if (c >= m) return;
  const double rr = sum_parts(part, nb, c, lane);
  if (lane == 0 && sc->active[c]) {
    const double rel = sqrt(rr / sc->bb[c]);
    sc->relres[c] = rel;
    sc->iters[c] = it;
    if (rel <= sc->tol[c]) sc->active[c] = 0;
  }
}

__global__ void pcg_beta_kernel(const double *__restrict__ part, int nb, int m,
                                PcgScalars *__restrict__ sc) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= m) return;
  const double rz = sum_parts(part, nb, c, lane);
  if (lane != 0) return;
  double b = 0.0;
  if (sc->active[c]) {
    b = rz / sc->rz[c];
    sc->rz[c] = rz;
  }
  sc->beta[c] = b;
}

__global__ void pcg_init_kernel(const double *__restrict__ part_bb,
                                const double *__restrict__ part_rz, int nb, int m,
                                const double *__restrict__ tol, PcgScalars *__restrict__ sc) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= m) return;
  const double bb = sum_parts(part_bb, nb, c, lane);
  const double rz = sum_parts(part_rz, nb, c, lane);
  if (lane != 0) return;
  sc->bb[c] = bb;
  sc->rz[c] = rz;
  sc->tol[c] = tol[c];
  sc->iters[c] = 0;
  sc->relres[c] = (bb > 0.0) ? 1.0 : 0.0;
  sc->active[c] = (bb > 0.0) ? 1 : 0;
  if (c == 0) {
    sc->breakdown = 0;
    sc->it = 0;
  }
}

// x += alpha p; r -= alpha q (column by column: no per-element division)
template <typename T>
__global__ void pcg_update_kernel(T *__restrict__ x, T *__restrict__ r,
                                  const T *__restrict__ p, const T *__restrict__ q, int64_t N,
                                  int m, const PcgScalars *__restrict__ sc) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c = 0; c < m; ++c) {
    const double a = sc->alpha[c];
    if (a == 0.0) continue;
    const int64_t off = (int64_t)c * N;
    for (int64_t i = i0; i < N; i += stride) {
      const int64_t e = off + i;
      x[e] = (T)((double)x[e] + a * (double)p[e]);
      r[e] = (T)((double)r[e] - a * (double)q[e]);
    }
  }
}

// p = z + beta p (active columns)
template <typename T>
__global__ void pcg_dir_kernel(T *__restrict__ p, const T *__restrict__ z, int64_t N, int m,
                               const PcgScalars *__restrict__ sc) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c = 0; c < m; ++c) {
    if (!sc->active[c]) continue;
    const double b = sc->beta[c];
    const int64_t off = (int64_t)c * N;
    for (int64_t i = i0; i < N; i += stride) {
      const int64_t e = off + i;
      p[e] = (T)((double)z[e] + b * (double)p[e]);
    }
  }
}

static unsigned vec_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------ PCG driver
static std::atomic<bool> g_pcg_graphs{true};
void set_pcg_graphs(bool on) { g_pcg_graphs.store(on); }
bool pcg_graphs_on() { return g_pcg_graphs.load(); }
static thread_local int t_pcg_replays = 0, t_pcg_checks = 0;
void pcg_counters_take(int *replays, int *checks) {
  if (replays) *replays = t_pcg_replays;
  if (checks) *checks = t_pcg_checks;
  t_pcg_replays = t_pcg_checks = 0;
}

namespace {
// One captured chunk of PCG iterations.
struct PcgChunk {
  cudaGraphExec_t exec = nullptr;
  CaptureLog log;
  ~PcgChunk() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// Iterations still needed by the slowest active column, estimated from its
// residual's rate since the previous check (a large count when unknown).
int pcg_remaining(const PcgScalars &h, const double *prev_rel, int prev_it, int m) {
  double worst = 0.0;
  for (int c = 0; c < m; ++c) {
    if (!h.active[c]) continue;
    const double rel = h.relres[c], tol = h.tol[c];
    const int di = h.it - prev_it;
    if (!(rel > 0.0) || !(prev_rel[c] > rel) || di <= 0 || !(tol > 0.0)) return 1 << 20;
    const double rate = std::pow(rel / prev_rel[c], 1.0 / di);
    const double need = std::log(tol / rel) / std::log(rate);
    worst = std::max(worst, need);
  }
  return worst > (double)(1 << 20) ? (1 << 20) : (int)worst;
}
}  // namespace

template <typename T>
krr_status pcg_run(const PcgOps<T> &ops, int64_t N, int m, const T *b, T *x,
                   const double *tol_host, int maxit, cudaStream_t s, PcgStats *stats) {
  KRR_REQUIRE(m >= 1 && m <= PCG_MAX_M, "PCG: 1 to %d columns (got %d)", PCG_MAX_M, m);
  DevBuf<T> r, z, p, q;
  KRR_TRY(r.alloc((size_t)N * m, s));
  KRR_TRY(z.alloc((size_t)N * m, s));
  KRR_TRY(p.alloc((size_t)N * m, s));
  KRR_TRY(q.alloc((size_t)N * m, s));
  DevBuf<double> part1, part2, dtol;
  KRR_TRY(part1.alloc((size_t)RED_BLOCKS * m, s));
  KRR_TRY(part2.alloc((size_t)RED_BLOCKS * m, s));
  KRR_TRY(dtol.alloc(m, s));
  DevBuf<PcgScalars> sc;
  KRR_TRY(sc.alloc(1, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(dtol.p, tol_host, sizeof(double) * m, cudaMemcpyHostToDevice, s));
  KRR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * (size_t)N * m, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(r.p, b, sizeof(T) * (size_t)N * m, cudaMemcpyDeviceToDevice, s));
  KRR_TRY(ops.precond(r.p, z.p, s));
  dots_kernel<T><<<RED_BLOCKS, 256, 0, s>>>(r.p, r.p, N, m, part1.p);
  KRR_LAUNCH_CHECK();
  dots_kernel<T><<<RED_BLOCKS, 256, 0, s>>>(r.p, z.p, N, m, part2.p);
  KRR_LAUNCH_CHECK();
  pcg_init_kernel<<<1, 32 * m, 0, s>>>(part1.p, part2.p, RED_BLOCKS, m, dtol.p, sc.p);
  KRR_LAUNCH_CHECK();
  KRR_CUDA_TRY(cudaMemcpyAsync(p.p, z.p, sizeof(T) * (size_t)N * m, cudaMemcpyDeviceToDevice, s));

  // q = A p, alpha, x += alpha p, r -= alpha q, convergence test
  auto step_a = [&](cudaStream_t st) -> krr_status {
    KRR_TRY(ops.product(p.p, q.p, st));
    dots_kernel<T><<<RED_BLOCKS, 256, 0, st>>>(p.p, q.p, N, m, part1.p);
    KRR_LAUNCH_CHECK();
    pcg_alpha_kernel<<<1, 32 * m, 0, st>>>(part1.p, RED_BLOCKS, m, sc.p);
    KRR_LAUNCH_CHECK();
    pcg_update_kernel<T><<<vec_grid(N), 256, 0, st>>>(x, r.p, p.p, q.p, N, m, sc.p);
    KRR_LAUNCH_CHECK();
    dots_kernel<T><<<RED_BLOCKS, 256, 0, st>>>(r.p, r.p, N, m, part1.p);
    KRR_LAUNCH_CHECK();
    pcg_resid_kernel<<<1, 32 * m, 0, st>>>(part1.p, RED_BLOCKS, m, sc.p);
    KRR_LAUNCH_CHECK();
    return KRR_OK;
  };
  // z = M^-1 r, beta, p = z + beta p
  auto step_b = [&](cudaStream_t st) -> krr_status {
    KRR_TRY(ops.precond(r.p, z.p, st));
    dots_kernel<T><<<RED_BLOCKS, 256, 0, st>>>(r.p, z.p, N, m, part1.p);
    KRR_LAUNCH_CHECK();
    pcg_beta_kernel<<<1, 32 * m, 0, st>>>(part1.p, RED_BLOCKS, m, sc.p);
    KRR_LAUNCH_CHECK();
    pcg_dir_kernel<T><<<vec_grid(N), 256, 0, st>>>(p.p, z.p, N, m, sc.p);
    KRR_LAUNCH_CHECK();
    return KRR_OK;
  };
  PcgScalars h;
  int checks = 0;
  auto read_back = [&]() -> krr_status {
    KRR_CUDA_TRY(cudaMemcpyAsync(&h, sc.p, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    KRR_CUDA_TRY(cudaStreamSynchronize(s));
    ++checks;
    return KRR_OK;
  };
  auto any_active = [&]() {
    bool any = false;
    for (int c = 0; c < m; ++c) any = any || h.active[c];
    return any;
  };
  KRR_TRY(read_back());
  double prev_rel[PCG_MAX_M];
  int prev_it = 0;
  for (int c = 0; c < m; ++c) prev_rel[c] = h.relres[c];
  // the first iteration runs eagerly: it makes the operator's and the
  // preconditioner's first calls (allocations, the product's autotuning)
  if (any_active() && maxit > 0) {
    KRR_TRY(step_a(s));
    KRR_TRY(read_back());
  }
  int replays = 0;
  bool graphs = pcg_graphs_on();
  PcgChunk chunks[3];   // 16, 4 and 1 iterations
  struct CaptureStream {
    cudaStream_t s = nullptr;
    ~CaptureStream() {
      if (s) cudaStreamDestroy(s);
    }
  } capture_stream;
  cudaStream_t &cs = capture_stream.s;
  while (any_active() && h.it < maxit) {
    const int left = maxit - h.it;
    const int need = pcg_remaining(h, prev_rel, prev_it, m);
    // replays may overshoot convergence (wasted but harmless iterations of
    // frozen columns): aim at half the estimated need
    const int want = std::min(left, std::max(1, need / 2));
    const int ci = want >= 16 ? 0 : want >= 4 ? 1 : 2;
    const int U = ci == 0 ? 16 : ci == 1 ? 4 : 1;
    for (int c = 0; c < m; ++c) prev_rel[c] = h.relres[c];
    prev_it = h.it;
    if (graphs && !chunks[ci].exec) {
      if (!cs) KRR_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      capture_log_begin(&chunks[ci].log);
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      krr_status st = KRR_OK;
      if (e == cudaSuccess) {
        for (int u = 0; u < U && st == KRR_OK; ++u) {
          st = step_b(cs);
          if (st == KRR_OK) st = step_a(cs);
        }
        e = cudaStreamEndCapture(cs, &g);
      }
      capture_log_begin(nullptr);
      if (e == cudaSuccess && st == KRR_OK && g) e = cudaGraphInstantiate(&chunks[ci].exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess || st != KRR_OK || !chunks[ci].exec) {
        // not capturable (an operator that synchronises or allocates on
        // every call): step one launch at a time
        cudaGetLastError();
        clear_error();
        graphs = false;
      }
    }
    if (graphs) {
      KRR_CUDA_TRY(cudaGraphLaunch(chunks[ci].exec, s));
      ++replays;
      KRR_TRY(read_back());
      capture_replayed(chunks[ci].log);
    } else {
      KRR_TRY(step_b(s));
      KRR_TRY(step_a(s));
      KRR_TRY(read_back());
    }
  }
  t_pcg_replays += replays;
  t_pcg_checks += checks;
  if (stats) {
    stats->products += h.it;
    stats->graph_replays += replays;
    stats->host_checks += checks;
    int mx = 0;
    double worst = 0.0;
    bool conv = true;
    for (int c = 0; c < m; ++c) {
      mx = (h.iters[c] > mx) ? h.iters[c] : mx;
      worst = (h.relres[c] > worst) ? h.relres[c] : worst;
      if (h.relres[c] > tol_host[c]) conv = false;
    }
    stats->iters_max = mx;
    stats->relres_max = worst;
    stats->converged = conv;
    stats->breakdown = h.breakdown != 0;
    for (int c = 0; c < m; ++c) {
      stats->col_iters[c] = h.iters[c];
      stats->col_relres[c] = h.relres[c];
    }
  }
  return KRR_OK;
}

template krr_status pcg_run<double>(const PcgOps<double> &, int64_t, int, const double *,
                                    double *, const double *, int, cudaStream_t, PcgStats *);
template krr_status pcg_run<float>(const PcgOps<float> &, int64_t, int, const float *,
                                   float *, const double *, int, cudaStream_t, PcgStats *);

// ----------------------------------------------------- vector helpers
__global__ void residual_kernel(const double *__restrict__ y, const double *__restrict__ mx,
                                double *__restrict__ r, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    r[e] = y[e] - mx[e];
}

__global__ void add_f32_kernel(double *__restrict__ x, const float *__restrict__ d, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)d[e];
}

krr_status tri_apply_lower(const double *Wt, int rank, const double *t, int m, double *u,
                           cudaStream_t s) {
  if (rank == 0) return KRR_OK;
  launch_tri_gemv<false>(Wt, rank, t, m, u, s);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status tri_apply_lower_t(const double *W, int rank, const double *u, int m, double *v,
                             cudaStream_t s) {
  if (rank == 0) return KRR_OK;
  launch_tri_gemv<true>(W, rank, u, m, v, s);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status residual_f64(const double *y, const double *mx, double *r, int64_t n,
                        cudaStream_t s) {
  residual_kernel<<<vec_grid(n), 256, 0, s>>>(y, mx, r, n);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status add_f32_to_f64(double *x, const float *d, int64_t n, cudaStream_t s) {
  add_f32_kernel<<<vec_grid(n), 256, 0, s>>>(x, d, n);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

krr_status column_norms(const double *a, int64_t N, int m, double *out_host, cudaStream_t s) {
  DevBuf<double> part;
  KRR_TRY(part.alloc((size_t)RED_BLOCKS * m, s));
  dots_kernel<double><<<RED_BLOCKS, 256, 0, s>>>(a, a, N, m, part.p);
  KRR_LAUNCH_CHECK();
  std::vector<double> h((size_t)RED_BLOCKS * m);
  KRR_CUDA_TRY(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * h.size(),
                               cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  for (int c = 0; c < m; ++c) {
    double t = 0.0;
    for (int b = 0; b < RED_BLOCKS; ++b) t += h[(size_t)c * RED_BLOCKS + b];
    out_host[c] = std::sqrt(t);
  }
  return KRR_OK;
}

}  // namespace krr
