// Serving engine: continuous batching of Alg. 1 solves on one GPU.
//
// Requests are admitted in arrival order while their estimated device
// footprint fits the HBM budget and a slot is free.  A builder thread (its own
// low-priority stream) copies X and Y to the device, runs RPCholesky (Alg. 3),
// factors the mixed-precision Woodbury core and prepares the points.  The solve
// then follows the mixed-precision refinement of the single-solve driver:
// x = 0, r = y; repeat { float32 PCG on M d = r to a loose per-column
// tolerance; x += d; r = y - M x with the float-float product } until every
// column's relative residual is <= tol.  The inner PCG iterations of all
// iterating slots advance together, one grouped launch per phase (serve.cuh);
// inner-solve set-up and refinement residuals run on each slot's own stream,
// so they overlap with the other slots' iterations.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kmv.cuh"
#include "kmv_kernels.cuh"
#include "pcg.cuh"
#include "rpc.cuh"
#include "serve.cuh"
#include "solve.cuh"

namespace krr {

// ======================================================= device kernels
constexpr int SERVE_COL_THREADS = 1024;   // single-CTA per-column kernels
constexpr int SERVE_KERNELS_PER_ITER = 12;

// Fixed-order sum of a column's block partials by one warp (lane-strided,
// then a butterfly whose result is the same in every lane).
__device__ __forceinline__ double serve_col_sum(const double *part, int nbv, int c,
                                                int lane) {
  double acc = 0.0;
  for (int b = lane; b < nbv; b += 32) acc += part[(int64_t)c * nbv + b];
  return warp_sum(acc);
}

// Block partial of one column: every thread passes its value, the warp sums
// go to red[warp][c]; serve_block_flush then writes out[c * nbv + b].
__device__ __forceinline__ void serve_block_put(double (*red)[SERVE_MAX_M], int c, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
}

__device__ __forceinline__ void serve_block_flush(double (*red)[SERVE_MAX_M], int m,
                                                  double *out, int nbv, int b) {
  __syncthreads();
  if ((int)threadIdx.x < m) {
    double t = 0.0;
    for (int w = 0; w < SERVE_VB / 32; ++w) t += red[w][threadIdx.x];
    out[(int64_t)threadIdx.x * nbv + b] = t;
  }
  __syncthreads();
}

// q = sum of the product's split partials + lambda p; block partials of p.q
__global__ void __launch_bounds__(SERVE_VB) serve_reduce_kernel(const ServeTable *__restrict__ T) {
  __shared__ double red[SERVE_VB / 32][SERVE_MAX_M];
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int b = item - T->vec_off[s];
    const int64_t N = d.N, i = (int64_t)b * SERVE_VB + threadIdx.x;
    for (int c = 0; c < d.m; ++c) {
      double pq = 0.0;
      if (i < N) {
        float acc = 0.0f;
        for (int sp = 0; sp < d.splits; ++sp) acc += d.part[((int64_t)sp * d.M + c) * N + i];
        const float pv = d.p[(int64_t)c * N + i];
        const float qv = acc + d.lam32 * pv;
        d.q[(int64_t)c * N + i] = qv;
        pq = (double)pv * (double)qv;
      }
      serve_block_put(red, c, pq);
    }
    serve_block_flush(red, d.m, d.dpart0, d.nbv, b);
  }
}

// alpha_c = rz_c / (p_c . q_c) for active columns; breakdown otherwise.
__global__ void __launch_bounds__(SERVE_COL_THREADS)
serve_alpha_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->col_off[n];
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (int g = threadIdx.x >> 5; g < total; g += warps) {
    const int s = serve_find_slot(T->col_off, n, g);
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    if (!sc->live) continue;
    const int c = g - T->col_off[s];
    const double pq = serve_col_sum(d.dpart0, d.nbv, c, lane);
    if (lane == 0) {
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
  }
}

// x += alpha p, r -= alpha q; block partials of r.r
__global__ void __launch_bounds__(SERVE_VB) serve_update_kernel(const ServeTable *__restrict__ T) {
  __shared__ double red[SERVE_VB / 32][SERVE_MAX_M];
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int b = item - T->vec_off[s];
    const int64_t N = d.N, i = (int64_t)b * SERVE_VB + threadIdx.x;
    for (int c = 0; c < d.m; ++c) {
      double rr = 0.0;
      if (i < N) {
        const int64_t e = (int64_t)c * N + i;
        const double a = d.sc->alpha[c];
        float rv = d.r[e];
        if (a != 0.0) {
          d.x[e] = (float)((double)d.x[e] + a * (double)d.p[e]);
          rv = (float)((double)rv - a * (double)d.q[e]);
          d.r[e] = rv;
        }
        rr = (double)rv * (double)rv;
      }
      serve_block_put(red, c, rr);
    }
    serve_block_flush(red, d.m, d.dpart0, d.nbv, b);
  }
}

// Convergence test on the recursive residual and the iteration limit; then
// the slot flags (one thread per slot) and the host-visible status.
__global__ void __launch_bounds__(SERVE_COL_THREADS)
serve_resid_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->col_off[n];
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (int g = threadIdx.x >> 5; g < total; g += warps) {
    const int s = serve_find_slot(T->col_off, n, g);
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    if (!sc->live) continue;
    const int c = g - T->col_off[s];
    const double rr = serve_col_sum(d.dpart0, d.nbv, c, lane);
    if (lane == 0 && sc->active[c]) {
      const double rel = sqrt(rr / sc->bb[c]);
      sc->relres[c] = rel;
      sc->iters[c] += 1;
      if (rel <= sc->ctl.tol[c] || sc->iters[c] >= sc->ctl.limit) sc->active[c] = 0;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    if (!sc->live) continue;
    int live = 0, imax = 0;
    for (int c = 0; c < d.m; ++c) {
      live |= sc->active[c];
      imax = max(imax, sc->iters[c]);
    }
    sc->live = live;
    d.status->live = live;
    d.status->breakdown = sc->breakdown;
    d.status->iters_max = imax;
  }
}

// part[b][l][c] = sum over the rows n of block b of F[n + l N] r[c][n], for
// the columns l of group g (SERVE_TT_COLS of them): one warp per column, the
// lanes' rows loaded before the arithmetic.  M is the slot's padded m.
template <int M>
__device__ __forceinline__ void serve_tt_item(const ServeSlotDesc &d, int b, int g,
                                              float (*sR)[SERVE_TT_ROWS]) {
  constexpr int PER_LANE = SERVE_TT_ROWS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = d.N, n0 = (int64_t)b * SERVE_TT_ROWS;
  const int nr = (int)min((int64_t)SERVE_TT_ROWS, N - n0);
  const int m = d.m, rank = d.rank;
  __syncthreads();
  for (int e = threadIdx.x; e < m * SERVE_TT_ROWS; e += blockDim.x) {
    const int c = e / SERVE_TT_ROWS, r = e % SERVE_TT_ROWS;
    sR[c][r] = (r < nr) ? d.r[(int64_t)c * N + n0 + r] : 0.0f;
  }
  __syncthreads();
  const int l1 = min(rank, (g + 1) * SERVE_TT_COLS);
  for (int l = g * SERVE_TT_COLS + warp; l < l1; l += blockDim.x >> 5) {
    const float *col = d.F + (int64_t)l * N + n0;
    float f[PER_LANE];
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
      const int r = lane + 32 * q;
      f[q] = (r < nr) ? col[r] : 0.0f;
    }
    float acc[M];
#pragma unroll
    for (int c = 0; c < M; ++c) acc[c] = 0.0f;
#pragma unroll
    for (int q = 0; q < PER_LANE; ++q) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        if (c < m) acc[c] = fmaf(f[q], sR[c][lane + 32 * q], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if (c < m) {
        const float v = warp_sum(acc[c]);
        if (lane == 0) d.ttpart[((int64_t)b * rank + l) * m + c] = (double)v;
      }
    }
  }
}

__global__ void __launch_bounds__(256) serve_tt_kernel(const ServeTable *__restrict__ T) {
  __shared__ float sR[SERVE_MAX_M][SERVE_TT_ROWS];
  const int n = T->nslots, total = T->tt_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->tt_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int local = item - T->tt_off[s];
    const int b = local % d.nbt, g = local / d.nbt;
    switch (d.M) {
      case 1: serve_tt_item<1>(d, b, g, sR); break;
      case 2: serve_tt_item<2>(d, b, g, sR); break;
      case 4: serve_tt_item<4>(d, b, g, sR); break;
      case 8: serve_tt_item<8>(d, b, g, sR); break;
      default: serve_tt_item<16>(d, b, g, sR); break;
    }
  }
}

// t[c][l] = sum over blocks of part[b][l][c] (one warp per (l, c))
__global__ void __launch_bounds__(256) serve_ttred_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->ttr_off[n];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < total; w += gridDim.x * wpb) {
    const int s = serve_find_slot(T->ttr_off, n, w);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int e = w - T->ttr_off[s];
    const int l = e / d.m, c = e % d.m;
    double acc = 0.0;
    for (int b = lane; b < d.nbt; b += 32) acc += d.ttpart[((int64_t)b * d.rank + l) * d.m + c];
    acc = warp_sum(acc);
    if (lane == 0) d.t[(int64_t)c * d.rank + l] = acc;
  }
}

// UPPER == false: u = W t (rows of W read from Wt); UPPER == true: v = W^T u.
template <bool UPPER>
__global__ void __launch_bounds__(256) serve_tri_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->tri_off[n];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int w = blockIdx.x * wpb + (threadIdx.x >> 5); w < total; w += gridDim.x * wpb) {
    const int s = serve_find_slot(T->tri_off, n, w);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int i = w - T->tri_off[s];
    const int rank = d.rank, m = d.m;
    const double *Mt = UPPER ? d.W : d.Wt;
    const double *x = UPPER ? d.u : d.t;
    double *out = UPPER ? d.v : d.u;
    double acc[SERVE_MAX_M];
#pragma unroll
    for (int c = 0; c < SERVE_MAX_M; ++c) acc[c] = 0.0;
    const double *col = Mt + (int64_t)i * rank;
    const int lo = UPPER ? i : 0, hi = UPPER ? rank : i + 1;
    for (int l = lo + lane; l < hi; l += 32) {
      const double wv = col[l];
#pragma unroll
      for (int c = 0; c < SERVE_MAX_M; ++c)
        if (c < m) acc[c] = fma(wv, x[(int64_t)c * rank + l], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < SERVE_MAX_M; ++c) {
      if (c < m) {
        const double v = warp_sum(acc[c]);
        if (lane == 0) out[(int64_t)c * rank + i] = v;
      }
    }
  }
}

// z = (r - F v) / lambda for one block of SERVE_VB rows; block partials of r.z
template <int M>
__device__ __forceinline__ void serve_tn_item(const ServeSlotDesc &d, int b,
                                              float (*sv)[SERVE_MAX_M],
                                              double (*red)[SERVE_MAX_M]) {
  constexpr int LCH = 256;
  constexpr int LU = 16;
  const int64_t N = d.N, i = (int64_t)b * SERVE_VB + threadIdx.x;
  const bool ok = i < N;
  const int m = d.m, rank = d.rank;
  float acc[M];
#pragma unroll
  for (int c = 0; c < M; ++c) acc[c] = 0.0f;
  for (int l0 = 0; l0 < rank; l0 += LCH) {
    const int nl = min(LCH, rank - l0);
    __syncthreads();
    for (int e = threadIdx.x; e < M * LCH; e += blockDim.x) {
      const int c = e / LCH, l = e % LCH;
      sv[l][c] = (l < nl && c < m) ? (float)d.v[(int64_t)c * rank + l0 + l] : 0.0f;
    }
    __syncthreads();
    for (int lb = 0; lb < nl; lb += LU) {
      float f[LU];
#pragma unroll
      for (int u = 0; u < LU; ++u)
        f[u] = (ok && lb + u < nl) ? d.F[i + (int64_t)(l0 + lb + u) * N] : 0.0f;
#pragma unroll
      for (int u = 0; u < LU; ++u) {
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = fmaf(f[u], sv[lb + u][c], acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < M; ++c) {
    if (c < m) {
      double rz = 0.0;
      if (ok) {
        const int64_t e = (int64_t)c * N + i;
        const float rv = d.r[e];
        const float zv = (float)(((double)rv - (double)acc[c]) * d.inv_lam);
        d.z[e] = zv;
        rz = (double)rv * (double)zv;
      }
      serve_block_put(red, c, rz);
    }
  }
  serve_block_flush(red, m, d.dpart1, d.nbv, b);
}

__global__ void __launch_bounds__(SERVE_VB) serve_tn_kernel(const ServeTable *__restrict__ T) {
  __shared__ float sv[256][SERVE_MAX_M];
  __shared__ double red[SERVE_VB / 32][SERVE_MAX_M];
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    if (!d.sc->live) continue;
    const int b = item - T->vec_off[s];
    switch (d.M) {
      case 1: serve_tn_item<1>(d, b, sv, red); break;
      case 2: serve_tn_item<2>(d, b, sv, red); break;
      case 4: serve_tn_item<4>(d, b, sv, red); break;
      case 8: serve_tn_item<8>(d, b, sv, red); break;
      default: serve_tn_item<16>(d, b, sv, red); break;
    }
  }
}

// beta_c = rz_new / rz for active columns
__global__ void __launch_bounds__(SERVE_COL_THREADS)
serve_beta_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->col_off[n];
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (int g = threadIdx.x >> 5; g < total; g += warps) {
    const int s = serve_find_slot(T->col_off, n, g);
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    if (!sc->live) continue;
    const int c = g - T->col_off[s];
    const double rz = serve_col_sum(d.dpart1, d.nbv, c, lane);
    if (lane == 0) {
      double bt = 0.0;
      if (sc->active[c]) {
        bt = rz / sc->rz[c];
        sc->rz[c] = rz;
      }
      sc->beta[c] = bt;
    }
  }
}

// p = z + beta p for active columns
__global__ void __launch_bounds__(SERVE_VB) serve_dir_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    const ServeScalars *sc = d.sc;
    if (!sc->live) continue;
    const int64_t N = d.N, i = (int64_t)(item - T->vec_off[s]) * SERVE_VB + threadIdx.x;
    if (i >= N) continue;
    for (int c = 0; c < d.m; ++c) {
      if (sc->active[c]) {
        const int64_t e = (int64_t)c * N + i;
        d.p[e] = (float)((double)d.z[e] + sc->beta[c] * (double)d.p[e]);
      }
    }
  }
}

// Inner-solve start (one-slot table): x = 0, r = float32(r64) on the columns
// that take part (zero elsewhere), block partials of r.r; marks the slot live
// for the preconditioner launches that follow.
__global__ void __launch_bounds__(SERVE_VB) serve_init_vec_kernel(const ServeTable *__restrict__ T) {
  __shared__ double red[SERVE_VB / 32][SERVE_MAX_M];
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    if (item == T->vec_off[s] && threadIdx.x == 0) sc->live = 1;
    const int b = item - T->vec_off[s];
    const int64_t N = d.N, i = (int64_t)b * SERVE_VB + threadIdx.x;
    for (int c = 0; c < d.m; ++c) {
      double rr = 0.0;
      if (i < N) {
        const int64_t e = (int64_t)c * N + i;
        const float rv = sc->ctl.need[c] ? (float)d.r64[e] : 0.0f;
        d.r[e] = rv;
        d.x[e] = 0.0f;
        rr = (double)rv * (double)rv;
      }
      serve_block_put(red, c, rr);
    }
    serve_block_flush(red, d.m, d.dpart0, d.nbv, b);
  }
}

__global__ void __launch_bounds__(SERVE_COL_THREADS)
serve_init_scalars_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->col_off[n];
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (int g = threadIdx.x >> 5; g < total; g += warps) {
    const int s = serve_find_slot(T->col_off, n, g);
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    const int c = g - T->col_off[s];
    const double bb = serve_col_sum(d.dpart0, d.nbv, c, lane);
    const double rz = serve_col_sum(d.dpart1, d.nbv, c, lane);
    if (lane == 0) {
      sc->bb[c] = bb;
      sc->rz[c] = rz;
      sc->iters[c] = 0;
      sc->alpha[c] = 0.0;
      sc->beta[c] = 0.0;
      sc->relres[c] = (bb > 0.0) ? 1.0 : 0.0;
      sc->active[c] = (sc->ctl.need[c] && bb > 0.0) ? 1 : 0;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const ServeSlotDesc &d = T->slot[s];
    ServeScalars *sc = d.sc;
    int live = 0;
    for (int c = 0; c < d.m; ++c) live |= sc->active[c];
    sc->breakdown = 0;
    sc->live = live;
    d.status->live = live;
    d.status->breakdown = 0;
    d.status->iters_max = 0;
  }
}

// p = z (all columns)
__global__ void __launch_bounds__(SERVE_VB) serve_pinit_kernel(const ServeTable *__restrict__ T) {
  const int n = T->nslots, total = T->vec_off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = serve_find_slot(T->vec_off, n, item);
    const ServeSlotDesc &d = T->slot[s];
    const int64_t N = d.N, i = (int64_t)(item - T->vec_off[s]) * SERVE_VB + threadIdx.x;
    if (i >= N) continue;
    for (int c = 0; c < d.m; ++c) d.p[(int64_t)c * N + i] = d.z[(int64_t)c * N + i];
  }
}

// out[c] = sum_n a[c][n]^2 (one CTA per column, fixed order)
__global__ void __launch_bounds__(1024) serve_sumsq_kernel(const double *__restrict__ a, int64_t N,
                                                           double *__restrict__ out) {
  __shared__ double red[32];
  const double *col = a + (int64_t)blockIdx.x * N;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc = fma(col[i], col[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

static unsigned serve_vec_grid() { return (unsigned)(num_sms() * 4); }

// Optional per-kernel timing of a step (events after every launch).
struct PhaseEvents {
  std::vector<cudaEvent_t> ev;   // U * SERVE_KERNELS_PER_ITER + 1
  size_t next = 0;
  krr_status mark(cudaStream_t s) {
    if (ev.empty()) return KRR_OK;
    KRR_CUDA_TRY(cudaEventRecord(ev[next++], s));
    return KRR_OK;
  }
};

static krr_status serve_launch_precond(const ServeTable *T, cudaStream_t s,
                                       PhaseEvents *pe = nullptr) {
  const unsigned g = serve_vec_grid();
  serve_tt_kernel<<<g, 256, 0, s>>>(T);
  KRR_LAUNCH_CHECK();
  if (pe) KRR_TRY(pe->mark(s));
  serve_ttred_kernel<<<g, 256, 0, s>>>(T);
  KRR_LAUNCH_CHECK();
  if (pe) KRR_TRY(pe->mark(s));
  serve_tri_kernel<false><<<g, 256, 0, s>>>(T);
  KRR_LAUNCH_CHECK();
  if (pe) KRR_TRY(pe->mark(s));
  serve_tri_kernel<true><<<g, 256, 0, s>>>(T);
  KRR_LAUNCH_CHECK();
  if (pe) KRR_TRY(pe->mark(s));
  serve_tn_kernel<<<g, SERVE_VB, 0, s>>>(T);
  KRR_LAUNCH_CHECK();
  if (pe) KRR_TRY(pe->mark(s));
  return KRR_OK;
}

// U inner PCG iterations of every slot in T (SERVE_KERNELS_PER_ITER kernels
// each), in the order of the single-solve loop: product, alpha, update,
// convergence test, preconditioner, beta, direction.
// Streams and events of the product's parallel branches.
constexpr int SERVE_BRANCHES = 8;
struct ProductBranches {
  cudaStream_t side[SERVE_BRANCHES] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[SERVE_BRANCHES] = {};
};

// The product of one slot that runs as its own tcgen05 launch (ServeSlotDesc::
// tc5): y = K p without the shift, written as the slot's single split of
// partial sums, so the grouped reduction adds lambda p as for the others.
struct Tc5Job {
  const PointsF32 *P;
  const float *p;
  float *y;
  int m;
  DevBuf<float> *scratch;
};

// Kernels one tcgen05 job launches per iteration (right-hand-side staging,
// product, segment reduction per group of 8 right-hand sides).
static int tc5_job_kernels(const Tc5Job &j) { return 3 * ((j.m + 7) / 8); }

// (A + lambda I) p partial sums of every slot of T: one launch per variant
// present (Th: host copy of the table at T) and one tcgen05 product per job,
// forked onto parallel branches and joined back into s.
static krr_status serve_launch_product(const ServeTable *T, const ServeTable *Th,
                                       const ProductBranches &B,
                                       const std::vector<Tc5Job> &jobs, cudaStream_t s) {
  const int nc = Th->nclasses, nj = (int)jobs.size();
  if (nc + nj == 0) return KRR_OK;
  const int nb = nc + nj < SERVE_BRANCHES ? nc + nj : SERVE_BRANCHES;
  KRR_CUDA_TRY(cudaEventRecord(B.fork, s));
  for (int b = 0; b < nb; ++b) KRR_CUDA_TRY(cudaStreamWaitEvent(B.side[b], B.fork, 0));
  for (int c = 0; c < nc; ++c) {
    const ServeClass &C = Th->cls[c];
    const ServeSlotDesc &d0 = Th->slot[C.slot[0]];
    const int items = C.off[C.nslots];
    cudaStream_t bs = B.side[c % nb];
    cudaError_t e = cudaErrorInvalidValue;
    if (d0.kc > 0) e = serve_launch_product_tc(d0.kern, d0.kc, d0.M, items, T, c, bs);
    else if (d0.kern == KGAUSS) e = serve_launch_product_gauss(d0.dp, d0.M, items, T, c, bs);
    else if (d0.kern == KLAPLACE) e = serve_launch_product_laplace(d0.dp, d0.M, items, T, c, bs);
    else if (d0.kern == KMATERN) e = serve_launch_product_matern(d0.dp, d0.M, items, T, c, bs);
    count_launch();
    KRR_CUDA_TRY(e);
  }
  for (int j = 0; j < nj; ++j) {
    const Tc5Job &J = jobs[j];
    KRR_TRY(kmv_tc5(*J.P, *J.P, 0.0f, false, J.p, J.P->N, J.m, J.y, J.P->N,
                    B.side[(nc + j) % nb], *J.scratch, true));
  }
  for (int b = 0; b < nb; ++b) {
    KRR_CUDA_TRY(cudaEventRecord(B.join[b], B.side[b]));
    KRR_CUDA_TRY(cudaStreamWaitEvent(s, B.join[b], 0));
  }
  return KRR_OK;
}

// U inner PCG iterations of every slot in T, in the order of the
// single-solve loop: product, alpha, update, convergence test,
// preconditioner, beta, direction.
static krr_status serve_launch_iterations(const ServeTable *T, const ServeTable *Th,
                                          const ProductBranches &B,
                                          const std::vector<Tc5Job> &jobs, int U,
                                          cudaStream_t s, PhaseEvents *pe = nullptr) {
  const unsigned g = serve_vec_grid();
  if (pe) KRR_TRY(pe->mark(s));
  for (int it = 0; it < U; ++it) {
    KRR_TRY(serve_launch_product(T, Th, B, jobs, s));
    if (pe) KRR_TRY(pe->mark(s));
    serve_reduce_kernel<<<g, SERVE_VB, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
    serve_alpha_kernel<<<1, SERVE_COL_THREADS, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
    serve_update_kernel<<<g, SERVE_VB, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
    serve_resid_kernel<<<1, SERVE_COL_THREADS, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
    KRR_TRY(serve_launch_precond(T, s, pe));
    serve_beta_kernel<<<1, SERVE_COL_THREADS, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
    serve_dir_kernel<<<g, SERVE_VB, 0, s>>>(T);
    KRR_LAUNCH_CHECK();
    if (pe) KRR_TRY(pe->mark(s));
  }
  return KRR_OK;
}

static krr_status serve_launch_inner_start(const ServeTable *T1, cudaStream_t s) {
  const unsigned g = serve_vec_grid();
  serve_init_vec_kernel<<<g, SERVE_VB, 0, s>>>(T1);
  KRR_LAUNCH_CHECK();
  KRR_TRY(serve_launch_precond(T1, s));
  serve_init_scalars_kernel<<<1, SERVE_COL_THREADS, 0, s>>>(T1);
  KRR_LAUNCH_CHECK();
  serve_pinit_kernel<<<g, SERVE_VB, 0, s>>>(T1);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// ============================================================ host side
static int serve_pad_m(int m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16; }

// Columns per split of a slot's product: at least SERVE_MIN_CHUNK, at most
// SERVE_MAX_SPLITS splits, a multiple of the column tile.
static int64_t serve_chunk(int64_t N) {
  int64_t chunk = (N + SERVE_MAX_SPLITS - 1) / SERVE_MAX_SPLITS;
  if (chunk < SERVE_MIN_CHUNK) chunk = SERVE_MIN_CHUNK;
  return (chunk + KMV_TJ - 1) / KMV_TJ * KMV_TJ;
}

// Estimated peak device bytes of one solve (build and solve phases together).
double serve_footprint(int64_t N, int d, int m, int k) {
  const double n = (double)N;
  const int M = serve_pad_m(m);
  const int dp = serve_dp_class(d), dpff = (d + 3) / 4 * 4;
  const int B = std::min(100, std::max(1, (k + 9) / 10));
  const int64_t chunk = serve_chunk(N);
  const double splits = (double)((N + chunk - 1) / chunk);
  const double nbt = (double)((N + SERVE_TT_ROWS - 1) / SERVE_TT_ROWS);
  const double nbv = (double)((N + SERVE_VB - 1) / SERVE_VB);
  double b = 0.0;
  // build: X, the float64 factor and its scratch, float32 factor, core
  b += n * d * 8 + n * k * 8 + n * k * 4 + n * 8 + k * 8.0;
  b += 2.0 * n * B * 8 + (double)B * k * 8 + 3.0 * k * k * 8;
  // prepared points (float32, half split of the tensor-core product, float-float)
  b += n * dp * 4 + n * 4 + n * 64.0 * ((d + 15) / 16) + n * 4 + 2.0 * n * dpff * 4 +
       2.0 * n * 4;
  // float64 blocks (y, x, r, M x) and float32 CG vectors
  b += 4.0 * n * m * 8 + 5.0 * n * m * 4;
  // product partials, preconditioner partials, reductions
  b += splits * M * n * 4 + nbt * k * m * 8 + 3.0 * k * m * 8 + 2.0 * nbv * m * 8;
  // float-float residual product: split partials and split right-hand sides
  const double rows_ff = 128.0 * (dpff <= 16 ? 2 : 1);
  const double tiles_ff = std::ceil(n / rows_ff);
  const double ffsplits = std::min(std::ceil(3648.0 / tiles_ff) + 1.0, std::ceil(n / 32.0));
  b += ffsplits * M * n * 8 + 2.0 * n * m * 4;
  return b * 1.05 + 16.0 * 1024 * 1024;
}

}  // namespace krr

using krr::ServeControl;
using krr::ServeScalars;
using krr::ServeSlotDesc;
using krr::ServeStatus;
using krr::ServeTable;
using Clock = std::chrono::steady_clock;

namespace {

enum class Phase { Queued, Building, Norms, Init, Inner, Refine, Escalated, Final };

struct Slot {
  // request
  int64_t req_id = 0;
  const double *X = nullptr;
  const double *Y = nullptr;
  double *alpha_out = nullptr;
  int64_t N = 0;
  int d = 0, kern = 0, m = 0, k = 0, maxit = 0;
  double sigma = 0, mu = 0, tol = 0;
  int64_t bytes = 0;
  uint64_t seed = 0;
  double t_submit = 0, t_admit = 0, t_built = 0;
  // engine state
  int id = -1;
  int lane = 1;                // stepping lane (0: fast, 1: bulk)
  Phase phase = Phase::Queued;
  krr_status build_status = KRR_OK;
  std::string error;
  krr_factor *f = nullptr;
  const krr::NystromCore *core = nullptr;
  krr::PointsF32 P32;
  krr::PointsFF Pff;
  void *arena = nullptr;
  krr::DevBuf<double> ffpart;
  krr::DevBuf<float> ffvsplit;
  krr::DevBuf<float> t5scratch;   // segment partials and staged p of a tcgen05 product
  double *Y64 = nullptr, *alpha64 = nullptr, *r64 = nullptr, *mx64 = nullptr;
  ServeSlotDesc desc{};
  // refinement bookkeeping (as the single-solve driver)
  std::vector<double> yn, rn;
  int outer = 0, iters = 0, budget = 0;
  double prev_worst = 1e300, relres = 1.0, entries = 0.0;
  bool breakdown = false, first_norms = true;
  int inner_limit = 0;
  bool inner_capped = false;   // the last inner solve stopped at its limit
  bool escalated = false;      // finished with float-float inner products
  krr_status status = KRR_OK;
  // eviction / checkpoint
  bool evict_req = false;      // leave the device at the next refinement boundary
  bool resume = false;         // continue from saved_alpha / saved_r when built
  std::vector<double> saved_alpha, saved_r;
};

// Checkpoint of a parked request: this header, then yn[m], rn[m], alpha
// (m x N) and the float64 residual r (m x N), all native-endian.
struct Checkpoint {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t N;
  int32_t d, kern, m, k;
  double sigma, mu, tol;
  uint64_t seed;
  int32_t maxit, outer, iters, budget;
  double prev_worst, relres, entries;
};
constexpr char kCheckpointMagic[8] = {'K', 'R', 'R', 'C', 'K', 'P', 'T', '1'};

}  // namespace

namespace krr {
// Slots step in two lanes that advance independently: a fast lane for slots
// whose float32 product is cheap and a bulk lane for the rest, so a small
// solve's steps are not paced by the largest slot's iterations.
constexpr int SERVE_LANES = 2;
constexpr double SERVE_FAST_LANE_FLOP = 4e10;   // float32 product flop per iteration
// Smallest N whose Gaussian / Matern product runs as the slot's own tcgen05
// launch (one CTA per SM over the slot's tiles) instead of a grouped launch.
constexpr int64_t SERVE_TC5_MIN_N = 32768;

struct Lane {
  cudaStream_t s = nullptr;
  ServeTable *table_dev = nullptr;      // work table of the lane's steps
  ServeTable *table_host = nullptr;     // pinned
  ServeStatus *status_host = nullptr;   // pinned copy of the status array
  ProductBranches branches;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev_done = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  PhaseEvents phase_ev;
  bool dirty = true;                    // slot set changed since the table was written
  bool busy = false;                    // a step is in flight
  std::vector<Slot *> members;          // slots of the step in flight
  std::vector<Tc5Job> tc5;              // tcgen05 products of the table's slots
};
}  // namespace krr

struct krr_server {
  krr_server_config cfg{};
  int device = 0;
  Clock::time_point t0;
  cudaStream_t s_free = nullptr;
  krr::Lane lanes[krr::SERVE_LANES];
  cudaStream_t s_build[krr::SERVE_MAX_BUILDERS] = {};
  int nbuilders = 0;
  cudaStream_t s_slot[krr::SERVE_MAX_SLOTS] = {};
  cudaEvent_t ev_slot[krr::SERVE_MAX_SLOTS] = {};
  // device
  ServeTable *init_dev = nullptr;      // one single-slot table per slot index
  ServeScalars *scalars_dev = nullptr;
  ServeStatus *status_dev = nullptr;
  int64_t captures = 0;
  // pinned host
  ServeTable *init_host = nullptr;
  ServeControl *ctl_host = nullptr;
  double *sumsq_host = nullptr;
  // slots
  std::unique_ptr<Slot> slots[krr::SERVE_MAX_SLOTS];
  std::deque<std::unique_ptr<Slot>> queue;
  std::vector<std::unique_ptr<Slot>> parked;   // evicted, waiting for resume / export
  std::vector<krr_request_result> done;
  // builders
  std::vector<std::thread> builders;
  std::mutex mtx;
  std::condition_variable cv;
  std::deque<Slot *> build_q;
  std::vector<Slot *> built;
  bool stop = false;
  // accounting
  int64_t budget = 0, reserved = 0, peak_reserved = 0;
  double entries_total = 0;
  int64_t next_id = 0, submitted = 0, completed = 0, steps = 0, step_kernels = 0;
  int max_concurrent = 0;
  double step_ms = 0, build_s = 0, escalate_s = 0;
  double phase_ms[krr::SERVE_KERNELS_PER_ITER] = {};
  int64_t escalations = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace krr {

static size_t table_bytes(int nslots) {
  return offsetof(ServeTable, slot) + sizeof(ServeSlotDesc) * (size_t)(nslots > 0 ? nslots : 0);
}

static void table_add(ServeTable *T, const ServeSlotDesc &d) {
  const int s = T->nslots;
  if (s == 0) {
    T->vec_off[0] = T->tt_off[0] = T->ttr_off[0] = T->tri_off[0] = T->col_off[0] = 0;
    T->nclasses = 0;
  }
  T->slot[s] = d;
  T->vec_off[s + 1] = T->vec_off[s] + d.nbv;
  T->tt_off[s + 1] = T->tt_off[s] + d.nbt * ((d.rank + SERVE_TT_COLS - 1) / SERVE_TT_COLS);
  T->ttr_off[s + 1] = T->ttr_off[s] + (d.rank > 0 ? d.rank * d.m : 0);
  T->tri_off[s + 1] = T->tri_off[s] + d.rank;
  T->col_off[s + 1] = T->col_off[s] + d.m;
  T->nslots = s + 1;
  // a tcgen05 slot's product is a launch of its own (Tc5Job)
  if (d.tc5) return;
  // the slot joins the product launch of its variant
  int c = 0;
  while (c < T->nclasses && T->cls[c].variant != d.variant) ++c;
  if (c == T->nclasses) {
    T->cls[c].variant = d.variant;
    T->cls[c].nslots = 0;
    T->cls[c].off[0] = 0;
    T->nclasses += 1;
  }
  ServeClass &C = T->cls[c];
  C.slot[C.nslots] = s;
  C.off[C.nslots + 1] = C.off[C.nslots] + d.row_tiles * d.splits * d.halves;
  C.nslots += 1;
}

template <typename T>
static void rebind(DevBuf<T> &b, cudaStream_t s) { b.s = s; }

// ------------------------------------------------------------- build
static krr_status build_slot(krr_server *S, Slot *sl, cudaStream_t s) {
  const int64_t N = sl->N;
  const int d = sl->d, m = sl->m;
  DevBuf<double> xtmp;
  const double *Xd = nullptr;
  KRR_TRY(device_view(sl->X, (size_t)N * d, s, xtmp, &Xd));
  sl->f = new (std::nothrow) krr_factor();
  if (!sl->f) return KRR_ENOMEM;
  sl->f->free_stream = S->s_free;
  sl->f->N = N;
  sl->f->d = d;
  sl->f->kern = sl->kern;
  sl->f->sigma = sl->sigma;
  if (sl->k > 0) {
    const int B = std::min(100, (sl->k + 9) / 10);
    KRR_TRY(rpcholesky_device(Xd, N, d, sl->kern, sl->sigma, sl->k, B, sl->seed, s, sl->f));
  }
  if (sl->f->rank > 0) KRR_TRY(nystrom_core(sl->f, sl->mu, KRR_PREC_MIXED, s, &sl->core));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  // the float64 factor only served the core; the solve uses its float32 copy
  dev_free(sl->f->F, S->s_free);
  sl->f->F = nullptr;
  const int dp = serve_dp_class(d);
  KRR_TRY(prepare_points_f32(Xd, N, d, sl->kern, sl->sigma, s, sl->P32, nullptr, dp));
  KRR_TRY(prepare_points_ff(Xd, N, d, sl->kern, sl->sigma, s, sl->Pff));

  ServeSlotDesc &D = sl->desc;
  const int M = serve_pad_m(m);
  // inner products on the tensor cores where the tile code has a variant and
  // the coordinates fit the half split
  // large slots take the single-problem tcgen05 product as a launch of their own
  const bool want_tc5 = product_path() == 0 && N >= SERVE_TC5_MIN_N;
  if (product_path() != 1) KRR_TRY(prepare_points_tc(Xd, s, sl->P32, want_tc5));
  const bool tc5 = want_tc5 && sl->P32.nh5 > 0;
  const int kc = sl->P32.kc16;
  const int rank = sl->core ? sl->core->rank : 0;
  const int64_t chunk = serve_chunk(N);
  // a tensor-core M = 16 slot runs its product as two halves of 8 columns
  const int rows = kc > 0 ? kmvtc_rows_per_cta(kc, M > 8 ? 8 : M)
                          : KMV_THREADS * kmv32_rows_per_thread(dp, M);
  D.halves = (kc > 0 && M > 8 && !tc5) ? 2 : 1;
  D.tc5 = tc5 ? 1 : 0;
  D.xt = sl->P32.xt.p;
  D.cn = sl->P32.cn.p;
  D.xs = kc > 0 ? sl->P32.xs16.p : nullptr;
  D.cs = kc > 0 ? sl->P32.cs16.p : nullptr;
  D.kc = kc;
  D.N = N;
  D.chunk = chunk;
  D.m = m;
  D.M = M;
  D.dp = dp;
  D.kern = sl->kern;
  D.variant = tc5 ? -1 : kc > 0 ? serve_variant_tc(sl->kern, kc, M) : serve_variant(sl->kern, dp, M);
  D.row_tiles = tc5 ? 0 : (int)((N + rows - 1) / rows);
  D.splits = tc5 ? 1 : (int)((N + chunk - 1) / chunk);
  const double lambda = sl->mu * (double)N;
  D.lam32 = (float)lambda;
  D.inv_lam = 1.0 / lambda;
  D.rank = rank;
  D.nbt = rank > 0 ? (int)((N + SERVE_TT_ROWS - 1) / SERVE_TT_ROWS) : 0;
  D.nbv = (int)((N + SERVE_VB - 1) / SERVE_VB);
  D.F = sl->core ? sl->core->F32 : nullptr;
  D.W = sl->core ? sl->core->W : nullptr;
  D.Wt = sl->core ? sl->core->Wt : nullptr;
  D.sc = S->scalars_dev + sl->id;
  D.status = S->status_dev + sl->id;
  sl->lane = (double)N * (double)N * (2.0 * dp + 2.0 * M + 5.0) <= SERVE_FAST_LANE_FLOP ? 0 : 1;

  // one arena for the slot's solve state, 256-byte aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t nm = (size_t)N * m;
  const size_t oY = take(nm * 8), oA = take(nm * 8), oR = take(nm * 8), oMx = take(nm * 8);
  const size_t ox = take(nm * 4), orr = take(nm * 4), oz = take(nm * 4), op = take(nm * 4),
               oq = take(nm * 4);
  const size_t opart = take((size_t)D.splits * M * N * 4);
  const size_t ott = take((size_t)D.nbt * rank * m * 8);
  const size_t ot = take((size_t)rank * m * 8), ou = take((size_t)rank * m * 8),
               ov = take((size_t)rank * m * 8);
  const size_t od0 = take((size_t)D.nbv * m * 8), od1 = take((size_t)D.nbv * m * 8);
  KRR_CUDA_TRY(cudaMallocAsync(&sl->arena, off, s));
  char *base = (char *)sl->arena;
  sl->Y64 = (double *)(base + oY);
  sl->alpha64 = (double *)(base + oA);
  sl->r64 = (double *)(base + oR);
  sl->mx64 = (double *)(base + oMx);
  D.x = (float *)(base + ox);
  D.r = (float *)(base + orr);
  D.z = (float *)(base + oz);
  D.p = (float *)(base + op);
  D.q = (float *)(base + oq);
  D.part = (float *)(base + opart);
  D.ttpart = (double *)(base + ott);
  D.t = (double *)(base + ot);
  D.u = (double *)(base + ou);
  D.v = (double *)(base + ov);
  D.dpart0 = (double *)(base + od0);
  D.dpart1 = (double *)(base + od1);
  D.r64 = sl->r64;
  KRR_CUDA_TRY(cudaMemcpyAsync(sl->Y64, sl->Y, nm * 8, cudaMemcpyDefault, s));
  if (sl->resume) {
    // continue a parked or imported solve where it left off
    KRR_CUDA_TRY(cudaMemcpyAsync(sl->alpha64, sl->saved_alpha.data(), nm * 8,
                                 cudaMemcpyHostToDevice, s));
    KRR_CUDA_TRY(cudaMemcpyAsync(sl->r64, sl->saved_r.data(), nm * 8, cudaMemcpyHostToDevice,
                                 s));
  } else {
    KRR_CUDA_TRY(cudaMemsetAsync(sl->alpha64, 0, nm * 8, s));
    KRR_CUDA_TRY(cudaMemcpyAsync(sl->r64, sl->Y64, nm * 8, cudaMemcpyDeviceToDevice, s));
  }
  KRR_CUDA_TRY(cudaMemsetAsync(D.p, 0, nm * 4, s));
  // a first tcgen05 product here sizes its scratch and raises the kernel's
  // shared-memory limit, so that the lane's captured steps allocate nothing
  if (D.tc5)
    KRR_TRY(kmv_tc5(sl->P32, sl->P32, 0.0f, false, D.p, N, m, D.part, N, s, sl->t5scratch,
                    true));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (sl->resume) {
    std::vector<double>().swap(sl->saved_alpha);
    std::vector<double>().swap(sl->saved_r);
  }
  // from here on the slot's memory is released on the free stream
  rebind(sl->P32.xt, S->s_free);
  rebind(sl->P32.cn, S->s_free);
  rebind(sl->P32.mean, S->s_free);
  rebind(sl->P32.xs16, S->s_free);
  rebind(sl->P32.cs16, S->s_free);
  rebind(sl->P32.xa5, S->s_free);
  rebind(sl->P32.xb5, S->s_free);
  rebind(sl->t5scratch, S->s_free);
  rebind(sl->Pff.xh, S->s_free);
  rebind(sl->Pff.xl, S->s_free);
  rebind(sl->Pff.ch, S->s_free);
  rebind(sl->Pff.cl, S->s_free);
  rebind(sl->Pff.mean, S->s_free);
  return KRR_OK;
}

static double worst_rel(const Slot *sl);

// Higher-precision continuation of a solve whose float32 inner iterations
// stopped making progress (escalate_refine: float64 CG vectors, float-float
// products, float64 residuals if needed).  Runs on a worker thread; the
// slot's data are not used by anything else meanwhile.
static krr_status escalate_slot(krr_server *S, Slot *sl, cudaStream_t s) {
  (void)S;
  Escalation e;
  e.Pff = &sl->Pff;
  e.X = sl->X;
  e.N = sl->N;
  e.d = sl->d;
  e.kern = sl->kern;
  e.m = sl->m;
  e.sigma = sl->sigma;
  e.lambda = sl->mu * (double)sl->N;
  e.tol = sl->tol;
  e.core = sl->core;
  e.Y = sl->Y64;
  e.alpha = sl->alpha64;
  e.r64 = sl->r64;
  e.mx = sl->mx64;
  e.yn = sl->yn;
  e.rn = sl->rn;
  e.budget = sl->budget;
  e.iters = sl->iters;
  e.outer = sl->outer;
  e.entries = sl->entries;
  e.ffpart = &sl->ffpart;
  e.ffvsplit = &sl->ffvsplit;
  sl->escalated = true;
  const krr_status st = escalate_refine(e, s);
  sl->rn = e.rn;
  sl->budget = e.budget;
  sl->iters = e.iters;
  sl->outer = e.outer;
  sl->entries = e.entries;
  sl->relres = e.relres;
  sl->status = e.status;
  return st;
}

static void builder_main(krr_server *S, int b) {
  cudaSetDevice(S->device);
  cudaStream_t s = S->s_build[b];
  set_alloc_stream(s);
  for (;;) {
    Slot *sl = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mtx);
      S->cv.wait(lk, [&] { return S->stop || !S->build_q.empty(); });
      if (S->stop) break;
      sl = S->build_q.front();
      S->build_q.pop_front();
    }
    clear_error();
    const bool esc = sl->phase == Phase::Escalated;
    const auto t0 = Clock::now();
    const krr_status st = esc ? escalate_slot(S, sl, s) : build_slot(S, sl, s);
    cudaStreamSynchronize(s);
    const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
    {
      std::lock_guard<std::mutex> lk(S->mtx);
      if (esc) {
        S->escalate_s += dt;
        S->escalations += 1;
      } else {
        S->build_s += dt;
      }
      if (esc) {
        // a failure of the launches themselves ends the request with it
        if (st != KRR_OK) sl->status = st;
      } else {
        sl->build_status = st;
      }
      if (st != KRR_OK) sl->error = krr_last_error();
      S->built.push_back(sl);
    }
  }
  set_alloc_stream(nullptr);
}

// ------------------------------------------------------------ phases
// Releases a slot's device memory (every use of it has completed: the host
// has seen the slot's last event).
static void release_device(krr_server *S, Slot *sl) {
  free_factor(sl->f);
  sl->f = nullptr;
  sl->core = nullptr;
  if (sl->arena) cudaFreeAsync(sl->arena, S->s_free);
  sl->arena = nullptr;
  sl->P32.xt.release();
  sl->P32.cn.release();
  sl->P32.mean.release();
  sl->P32.xs16.release();
  sl->P32.cs16.release();
  sl->P32.kc16 = 0;
  sl->P32.xa5.release();
  sl->P32.xb5.release();
  sl->P32.nh5 = 0;
  sl->t5scratch.release();
  sl->Pff.xh.release();
  sl->Pff.xl.release();
  sl->Pff.ch.release();
  sl->Pff.cl.release();
  sl->Pff.mean.release();
  sl->ffpart.release();
  sl->ffvsplit.release();
}

static void complete(krr_server *S, Slot *sl, krr_status st) {
  krr_request_result r{};
  r.id = sl->req_id;
  r.status = st;
  r.iters = sl->iters;
  r.outer_refinements = sl->outer;
  r.rank = sl->desc.rank;
  r.m = sl->m;
  r.escalated = sl->escalated ? 1 : 0;
  r.rel_residual = sl->relres;
  r.kernel_entries = sl->entries;
  r.t_submit = sl->t_submit;
  r.t_admit = sl->t_admit;
  r.t_built = sl->t_built;
  r.t_done = S->now();
  std::snprintf(r.error, sizeof(r.error), "%s", sl->error.c_str());
  S->done.push_back(r);
  S->completed += 1;
  S->entries_total += sl->entries;
  S->reserved -= sl->bytes;
  // every use of the slot's memory has completed (its last event was seen)
  release_device(S, sl);
  const int id = sl->id;
  if (id >= 0) S->slots[id].reset();
}

// Eviction at a refinement boundary: alpha and the float64 residual move to
// host memory, the slot and its budget are released, and the request waits
// in the parked list (krr_server_resume / krr_server_export).
static krr_status park(krr_server *S, Slot *sl) {
  const size_t nm = (size_t)sl->N * sl->m;
  cudaStream_t ss = S->s_slot[sl->id];
  sl->saved_alpha.resize(nm);
  sl->saved_r.resize(nm);
  KRR_CUDA_TRY(cudaMemcpyAsync(sl->saved_alpha.data(), sl->alpha64, nm * 8,
                               cudaMemcpyDeviceToHost, ss));
  KRR_CUDA_TRY(cudaMemcpyAsync(sl->saved_r.data(), sl->r64, nm * 8, cudaMemcpyDeviceToHost, ss));
  KRR_CUDA_TRY(cudaStreamSynchronize(ss));
  release_device(S, sl);
  S->reserved -= sl->bytes;
  const int id = sl->id;
  sl->id = -1;
  sl->phase = Phase::Queued;
  sl->evict_req = false;
  sl->resume = true;
  S->parked.push_back(std::move(S->slots[id]));
  return KRR_OK;
}

static krr_status start_norms(krr_server *S, Slot *sl) {
  cudaStream_t ss = S->s_slot[sl->id];
  ServeScalars *sc = S->scalars_dev + sl->id;
  serve_sumsq_kernel<<<sl->m, 1024, 0, ss>>>(sl->r64, sl->N, sc->resid_sq);
  KRR_LAUNCH_CHECK();
  KRR_CUDA_TRY(cudaMemcpyAsync(S->sumsq_host + (size_t)sl->id * SERVE_MAX_M, sc->resid_sq,
                               sizeof(double) * sl->m, cudaMemcpyDeviceToHost, ss));
  KRR_CUDA_TRY(cudaEventRecord(S->ev_slot[sl->id], ss));
  return KRR_OK;
}

static krr_status finalize(krr_server *S, Slot *sl, krr_status st) {
  sl->status = st;
  cudaStream_t ss = S->s_slot[sl->id];
  KRR_CUDA_TRY(cudaMemcpyAsync(sl->alpha_out, sl->alpha64, sizeof(double) * sl->N * sl->m,
                               cudaMemcpyDefault, ss));
  KRR_CUDA_TRY(cudaEventRecord(S->ev_slot[sl->id], ss));
  sl->phase = Phase::Final;
  return KRR_OK;
}

static double worst_rel(const Slot *sl) {
  double w = 0.0;
  for (int c = 0; c < sl->m; ++c)
    w = std::max(w, sl->yn[c] > 0 ? sl->rn[c] / sl->yn[c] : 0.0);
  return w;
}

static void escalate(krr_server *S, Slot *sl) {
  sl->phase = Phase::Escalated;
  {
    std::lock_guard<std::mutex> lk(S->mtx);
    S->build_q.push_back(sl);
  }
  S->cv.notify_one();
}

// One decision of the refinement loop after a float64 residual is known.
static krr_status decide(krr_server *S, Slot *sl) {
  constexpr int kMaxOuter = 12;
  constexpr double kInnerFloor = 1e-4;
  constexpr int kInnerCap = 1000;   // iterations of one float32 inner solve
  const double worst = worst_rel(sl);
  sl->relres = worst;
  if (worst <= sl->tol) return finalize(S, sl, KRR_OK);
  // float32 inner solves that break down, run into their cap or stop
  // reducing the residual hand the solve to the float-float continuation
  if (sl->breakdown || sl->inner_capped || sl->outer >= kMaxOuter || sl->budget <= 0 ||
      (sl->outer > 0 && worst > 0.5 * sl->prev_worst)) {
    escalate(S, sl);
    return KRR_OK;
  }
  if (sl->evict_req) return park(S, sl);
  sl->prev_worst = worst;
  ServeControl &ctl = S->ctl_host[sl->id];
  std::memset(&ctl, 0, sizeof(ctl));
  for (int c = 0; c < sl->m; ++c) {
    const double rel = sl->yn[c] > 0 ? sl->rn[c] / sl->yn[c] : 0.0;
    ctl.need[c] = rel > sl->tol ? 1 : 0;
    ctl.tol[c] = ctl.need[c] ? std::max(0.3 * sl->tol / rel, kInnerFloor) : 1.0;
  }
  ctl.limit = std::min(sl->budget, kInnerCap);
  sl->inner_limit = ctl.limit;
  cudaStream_t ss = S->s_slot[sl->id];
  KRR_CUDA_TRY(cudaMemcpyAsync(&S->scalars_dev[sl->id].ctl, &ctl, sizeof(ServeControl),
                               cudaMemcpyHostToDevice, ss));
  KRR_TRY(serve_launch_inner_start(S->init_dev + sl->id, ss));
  KRR_CUDA_TRY(cudaEventRecord(S->ev_slot[sl->id], ss));
  sl->phase = Phase::Init;
  return KRR_OK;
}

// Inner solve finished: x += d, r = y - M x (float-float product), norms.
static krr_status start_refine(krr_server *S, Slot *sl) {
  cudaStream_t ss = S->s_slot[sl->id];
  const int64_t nm = sl->N * sl->m;
  KRR_TRY(add_f32_to_f64(sl->alpha64, sl->desc.x, nm, ss));
  KRR_TRY(kmv_ff(sl->Pff, sl->mu * (double)sl->N, sl->alpha64, sl->N, sl->m, sl->mx64, sl->N,
                 ss, sl->ffpart, sl->ffvsplit));
  sl->entries += kmv_entries(sl->N);
  KRR_TRY(residual_f64(sl->Y64, sl->mx64, sl->r64, nm, ss));
  KRR_TRY(start_norms(S, sl));
  sl->phase = Phase::Refine;
  return KRR_OK;
}

static krr_status on_built(krr_server *S, Slot *sl) {
  if (sl->phase == Phase::Escalated) return finalize(S, sl, sl->status);
  sl->t_built = S->now();
  if (sl->build_status != KRR_OK) {
    sl->relres = 1.0;
    complete(S, sl, sl->build_status);
    return KRR_OK;
  }
  // the slot's one-slot table for its inner-solve starts
  ServeTable *T1 = S->init_host + sl->id;
  T1->nslots = 0;
  table_add(T1, sl->desc);
  cudaStream_t ss = S->s_slot[sl->id];
  KRR_CUDA_TRY(cudaMemcpyAsync(S->init_dev + sl->id, T1, table_bytes(1), cudaMemcpyHostToDevice,
                               ss));
  if (sl->resume) {
    sl->resume = false;
    return decide(S, sl);
  }
  sl->budget = sl->maxit;
  sl->first_norms = true;
  KRR_TRY(start_norms(S, sl));
  sl->phase = Phase::Norms;
  return KRR_OK;
}

static krr_status on_event(krr_server *S, Slot *sl) {
  const double *sq = S->sumsq_host + (size_t)sl->id * SERVE_MAX_M;
  switch (sl->phase) {
    case Phase::Norms:
      sl->yn.assign(sl->m, 0.0);
      for (int c = 0; c < sl->m; ++c) sl->yn[c] = std::sqrt(sq[c]);
      sl->rn = sl->yn;
      return decide(S, sl);
    case Phase::Init:
      sl->phase = Phase::Inner;
      S->lanes[sl->lane].dirty = true;
      return KRR_OK;
    case Phase::Refine:
      sl->rn.assign(sl->m, 0.0);
      for (int c = 0; c < sl->m; ++c) sl->rn[c] = std::sqrt(sq[c]);
      sl->outer += 1;
      return decide(S, sl);
    case Phase::Final:
      complete(S, sl, sl->status);
      return KRR_OK;
    default:
      return KRR_OK;
  }
}

static void admit(krr_server *S) {
  while (!S->queue.empty()) {
    Slot *front = S->queue.front().get();
    int active = 0, free_id = -1;
    for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
      if (S->slots[i]) ++active;
      else if (free_id < 0) free_id = i;
    }
    if (active >= S->cfg.max_slots || free_id < 0) return;
    if (S->reserved + front->bytes > S->budget) return;
    std::unique_ptr<Slot> sl = std::move(S->queue.front());
    S->queue.pop_front();
    sl->id = free_id;
    sl->t_admit = S->now();
    sl->phase = Phase::Building;
    S->reserved += sl->bytes;
    S->peak_reserved = std::max(S->peak_reserved, S->reserved);
    Slot *raw = sl.get();
    S->slots[free_id] = std::move(sl);
    {
      std::lock_guard<std::mutex> lk(S->mtx);
      S->build_q.push_back(raw);
    }
    S->cv.notify_one();
  }
}

static krr_status launch_step(krr_server *S, Lane &L) {
  const int U = S->cfg.iters_per_step;
  const ServeTable *Th = L.table_host;
  unsigned long long per_iter = SERVE_KERNELS_PER_ITER - 1 + Th->nclasses;
  for (const Tc5Job &j : L.tc5) per_iter += tc5_job_kernels(j);
  const unsigned long long kernels = (unsigned long long)U * per_iter;
  if (S->cfg.use_graph) {
    if (!L.graph) {
      // the launch sequence depends on the variants present: captured again
      // whenever the lane's slot set changes
      cudaGraph_t g = nullptr;
      set_launch_counting(false);
      KRR_CUDA_TRY(cudaStreamBeginCapture(L.s, cudaStreamCaptureModeThreadLocal));
      krr_status st = serve_launch_iterations(L.table_dev, Th, L.branches, L.tc5, U, L.s);
      cudaError_t e = cudaStreamEndCapture(L.s, &g);
      set_launch_counting(true);
      if (st != KRR_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      KRR_CUDA_TRY(e);
      e = cudaGraphInstantiate(&L.graph, g, 0);
      cudaGraphDestroy(g);
      KRR_CUDA_TRY(e);
      S->captures += 1;
    }
    KRR_CUDA_TRY(cudaGraphLaunch(L.graph, L.s));
    count_launches(kernels);
  } else if (profiling_on()) {
    PhaseEvents &pe = L.phase_ev;
    const size_t need = (size_t)U * SERVE_KERNELS_PER_ITER + 1;
    while (pe.ev.size() < need) {
      cudaEvent_t e;
      KRR_CUDA_TRY(cudaEventCreate(&e));
      pe.ev.push_back(e);
    }
    pe.next = 0;
    KRR_TRY(serve_launch_iterations(L.table_dev, Th, L.branches, L.tc5, U, L.s, &pe));
  } else {
    KRR_TRY(serve_launch_iterations(L.table_dev, Th, L.branches, L.tc5, U, L.s));
  }
  S->steps += 1;
  S->step_kernels += (int64_t)kernels;
  return KRR_OK;
}

// A lane's step has completed: device times, then every slot whose inner
// solve ended goes on to its refinement residual.
static krr_status finish_step(krr_server *S, Lane &L) {
  L.busy = false;
  float ms = 0.0f;
  KRR_CUDA_TRY(cudaEventElapsedTime(&ms, L.ev_t0, L.ev_t1));
  S->step_ms += ms;
  if (L.phase_ev.next > 1) {
    for (size_t e = 1; e < L.phase_ev.next; ++e) {
      float pm = 0.0f;
      KRR_CUDA_TRY(cudaEventElapsedTime(&pm, L.phase_ev.ev[e - 1], L.phase_ev.ev[e]));
      S->phase_ms[(e - 1) % SERVE_KERNELS_PER_ITER] += pm;
    }
    L.phase_ev.next = 0;
  }
  for (Slot *sl : L.members) {
    const ServeStatus &st = L.status_host[sl->id];
    if (st.live) continue;
    sl->iters += st.iters_max;
    sl->budget -= st.iters_max;
    sl->entries += kmv_entries(sl->N) * st.iters_max;
    sl->breakdown = st.breakdown != 0;
    sl->inner_capped = st.iters_max >= sl->inner_limit;
    L.dirty = true;
    KRR_TRY(start_refine(S, sl));
  }
  L.members.clear();
  return KRR_OK;
}

// Admission, finished builds and the slot streams' events: everything that
// does not touch the slots of a running step.
static krr_status service(krr_server *S) {
  admit(S);
  std::vector<Slot *> built;
  {
    std::lock_guard<std::mutex> lk(S->mtx);
    built.swap(S->built);
  }
  for (Slot *sl : built) KRR_TRY(on_built(S, sl));
  for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
    Slot *sl = S->slots[i].get();
    if (!sl) continue;
    if (sl->phase == Phase::Norms || sl->phase == Phase::Init || sl->phase == Phase::Refine ||
        sl->phase == Phase::Final) {
      const cudaError_t e = cudaEventQuery(S->ev_slot[i]);
      if (e == cudaErrorNotReady) continue;
      KRR_CUDA_TRY(e);
      KRR_TRY(on_event(S, sl));
    }
  }
  // freed slots may admit more
  admit(S);
  return KRR_OK;
}

static krr_status server_step(krr_server *S, int64_t *unfinished) {
  KRR_TRY(service(S));
  // launch a step in every idle lane that has iterating slots
  int iterating = 0;
  for (int i = 0; i < SERVE_MAX_SLOTS; ++i)
    if (S->slots[i] && S->slots[i]->phase == Phase::Inner) ++iterating;
  bool launched = false;
  for (int l = 0; l < SERVE_LANES; ++l) {
    Lane &L = S->lanes[l];
    if (L.busy) continue;
    std::vector<Slot *> inner;
    for (int i = 0; i < SERVE_MAX_SLOTS; ++i)
      if (S->slots[i] && S->slots[i]->phase == Phase::Inner && S->slots[i]->lane == l)
        inner.push_back(S->slots[i].get());
    if (inner.empty()) continue;
    if (L.dirty) {
      ServeTable *T = L.table_host;
      T->nslots = 0;
      L.tc5.clear();
      for (Slot *sl : inner) {
        table_add(T, sl->desc);
        if (sl->desc.tc5)
          L.tc5.push_back({&sl->P32, sl->desc.p, sl->desc.part, sl->m, &sl->t5scratch});
      }
      KRR_CUDA_TRY(cudaMemcpyAsync(L.table_dev, T, table_bytes(T->nslots),
                                   cudaMemcpyHostToDevice, L.s));
      L.dirty = false;
      if (L.graph) {
        KRR_CUDA_TRY(cudaGraphExecDestroy(L.graph));
        L.graph = nullptr;
      }
    }
    KRR_CUDA_TRY(cudaEventRecord(L.ev_t0, L.s));
    KRR_TRY(launch_step(S, L));
    KRR_CUDA_TRY(cudaEventRecord(L.ev_t1, L.s));
    KRR_CUDA_TRY(cudaMemcpyAsync(L.status_host, S->status_dev,
                                 sizeof(ServeStatus) * SERVE_MAX_SLOTS, cudaMemcpyDeviceToHost,
                                 L.s));
    KRR_CUDA_TRY(cudaEventRecord(L.ev_done, L.s));
    L.busy = true;
    L.members = inner;
    launched = true;
  }
  S->max_concurrent = std::max(S->max_concurrent, iterating);
  bool any_busy = false;
  for (int l = 0; l < SERVE_LANES; ++l) any_busy = any_busy || S->lanes[l].busy;
  if (any_busy) {
    // keep the other slots moving until a lane's step completes
    for (;;) {
      bool finished = false;
      for (int l = 0; l < SERVE_LANES; ++l) {
        Lane &L = S->lanes[l];
        if (!L.busy) continue;
        const cudaError_t e = cudaEventQuery(L.ev_done);
        if (e == cudaErrorNotReady) continue;
        KRR_CUDA_TRY(e);
        KRR_TRY(finish_step(S, L));
        finished = true;
      }
      if (finished) break;
      KRR_TRY(service(S));
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  } else if (!launched) {
    bool busy = false;
    for (int i = 0; i < SERVE_MAX_SLOTS; ++i) busy = busy || (bool)S->slots[i];
    if (busy) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (unfinished) {
    int64_t n = (int64_t)S->queue.size();
    for (int i = 0; i < SERVE_MAX_SLOTS; ++i) n += S->slots[i] ? 1 : 0;
    *unfinished = n;
  }
  return KRR_OK;
}

static void server_free(krr_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mtx);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto &t : S->builders)
    if (t.joinable()) t.join();
  cudaDeviceSynchronize();
  for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
    if (S->slots[i]) {
      free_factor(S->slots[i]->f);
      S->slots[i]->f = nullptr;
      if (S->slots[i]->arena) cudaFreeAsync(S->slots[i]->arena, S->s_free);
      S->slots[i].reset();
    }
  }
  cudaDeviceSynchronize();
  S->queue.clear();
  S->parked.clear();
  for (int l = 0; l < SERVE_LANES; ++l) {
    Lane &L = S->lanes[l];
    if (L.graph) cudaGraphExecDestroy(L.graph);
    cudaFree(L.table_dev);
    cudaFreeHost(L.table_host);
    cudaFreeHost(L.status_host);
    for (int b = 0; b < SERVE_BRANCHES; ++b) {
      if (L.branches.side[b]) cudaStreamDestroy(L.branches.side[b]);
      if (L.branches.join[b]) cudaEventDestroy(L.branches.join[b]);
    }
    if (L.branches.fork) cudaEventDestroy(L.branches.fork);
    for (cudaEvent_t e : L.phase_ev.ev) cudaEventDestroy(e);
    if (L.ev_done) cudaEventDestroy(L.ev_done);
    if (L.ev_t0) cudaEventDestroy(L.ev_t0);
    if (L.ev_t1) cudaEventDestroy(L.ev_t1);
    if (L.s) cudaStreamDestroy(L.s);
  }
  cudaFree(S->init_dev);
  cudaFree(S->scalars_dev);
  cudaFree(S->status_dev);
  cudaFreeHost(S->init_host);
  cudaFreeHost(S->ctl_host);
  cudaFreeHost(S->sumsq_host);
  for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
    if (S->ev_slot[i]) cudaEventDestroy(S->ev_slot[i]);
    if (S->s_slot[i]) cudaStreamDestroy(S->s_slot[i]);
  }
  for (int b = 0; b < SERVE_MAX_BUILDERS; ++b)
    if (S->s_build[b]) cudaStreamDestroy(S->s_build[b]);
  if (S->s_free) cudaStreamDestroy(S->s_free);
  delete S;
}

static krr_status server_init(krr_server *S) {
  KRR_CUDA_TRY(cudaGetDevice(&S->device));
  int lo = 0, hi = 0;
  KRR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  for (int l = 0; l < SERVE_LANES; ++l) {
    Lane &L = S->lanes[l];
    // the fast lane gets the highest priority, the bulk lane the next one
    const int prio = (l == 0 || hi == lo) ? hi : hi + 1;
    KRR_CUDA_TRY(cudaStreamCreateWithPriority(&L.s, cudaStreamNonBlocking, prio));
    KRR_CUDA_TRY(cudaEventCreateWithFlags(&L.ev_done, cudaEventDisableTiming));
    KRR_CUDA_TRY(cudaEventCreate(&L.ev_t0));
    KRR_CUDA_TRY(cudaEventCreate(&L.ev_t1));
    KRR_CUDA_TRY(cudaMalloc(&L.table_dev, sizeof(ServeTable)));
    KRR_CUDA_TRY(cudaMemset(L.table_dev, 0, sizeof(ServeTable)));
    KRR_CUDA_TRY(cudaMallocHost(&L.table_host, sizeof(ServeTable)));
    std::memset(L.table_host, 0, sizeof(ServeTable));
    KRR_CUDA_TRY(cudaMallocHost(&L.status_host, sizeof(ServeStatus) * SERVE_MAX_SLOTS));
    for (int b = 0; b < SERVE_BRANCHES; ++b) {
      KRR_CUDA_TRY(cudaStreamCreateWithPriority(&L.branches.side[b], cudaStreamNonBlocking, prio));
      KRR_CUDA_TRY(cudaEventCreateWithFlags(&L.branches.join[b], cudaEventDisableTiming));
    }
    KRR_CUDA_TRY(cudaEventCreateWithFlags(&L.branches.fork, cudaEventDisableTiming));
  }
  S->nbuilders = S->cfg.build_threads > 0 ? S->cfg.build_threads : 4;
  for (int b = 0; b < S->nbuilders; ++b)
    KRR_CUDA_TRY(cudaStreamCreateWithPriority(&S->s_build[b], cudaStreamNonBlocking, lo));
  KRR_CUDA_TRY(cudaStreamCreateWithFlags(&S->s_free, cudaStreamNonBlocking));
  for (int i = 0; i < SERVE_MAX_SLOTS; ++i) {
    KRR_CUDA_TRY(cudaStreamCreateWithPriority(&S->s_slot[i], cudaStreamNonBlocking, hi));
    KRR_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_slot[i], cudaEventDisableTiming));
  }
  KRR_CUDA_TRY(cudaMalloc(&S->init_dev, sizeof(ServeTable) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMalloc(&S->scalars_dev, sizeof(ServeScalars) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMalloc(&S->status_dev, sizeof(ServeStatus) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMemset(S->scalars_dev, 0, sizeof(ServeScalars) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMemset(S->status_dev, 0, sizeof(ServeStatus) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMallocHost(&S->init_host, sizeof(ServeTable) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMallocHost(&S->ctl_host, sizeof(ServeControl) * SERVE_MAX_SLOTS));
  KRR_CUDA_TRY(cudaMallocHost(&S->sumsq_host, sizeof(double) * SERVE_MAX_SLOTS * SERVE_MAX_M));
  if (S->cfg.hbm_budget_bytes > 0) {
    S->budget = (int64_t)S->cfg.hbm_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    KRR_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    S->budget = (int64_t)(0.9 * (double)fr);
  }
  KRR_CUDA_TRY(cudaDeviceSynchronize());
  S->t0 = Clock::now();
  for (int b = 0; b < S->nbuilders; ++b) S->builders.emplace_back(builder_main, S, b);
  return KRR_OK;
}

}  // namespace krr

// ============================================================= C ABI
extern "C" {

krr_status krr_server_footprint(int64_t N, int d, int m, int k, double *bytes) {
  krr::clear_error();
  KRR_REQUIRE(bytes, "bytes is NULL");
  KRR_REQUIRE(N >= 1 && d >= 1 && d <= 32 && m >= 1 && m <= 16 && k >= 0 && k <= N,
              "bad request shape");
  *bytes = krr::serve_footprint(N, d, m, k);
  return KRR_OK;
}

krr_status krr_server_create(const krr_server_config *cfg, krr_server **out) {
  krr::clear_error();
  KRR_REQUIRE(cfg && out, "NULL argument");
  *out = nullptr;
  KRR_REQUIRE(cfg->max_slots >= 1 && cfg->max_slots <= KRR_SERVE_MAX_SLOTS,
              "max_slots must be in [1, %d]", KRR_SERVE_MAX_SLOTS);
  KRR_REQUIRE(cfg->iters_per_step >= 1 && cfg->iters_per_step <= 64,
              "iters_per_step must be in [1, 64]");
  KRR_REQUIRE(cfg->hbm_budget_bytes >= 0 && std::isfinite(cfg->hbm_budget_bytes),
              "hbm_budget_bytes must be >= 0");
  KRR_REQUIRE(cfg->build_threads >= 0 && cfg->build_threads <= KRR_SERVE_MAX_BUILDERS,
              "build_threads must be in [0, %d]", KRR_SERVE_MAX_BUILDERS);
  krr_server *S = new (std::nothrow) krr_server();
  if (!S) return KRR_ENOMEM;
  S->cfg = *cfg;
  const krr_status st = krr::server_init(S);
  if (st != KRR_OK) {
    krr::server_free(S);
    return st;
  }
  *out = S;
  return KRR_OK;
}

krr_status krr_server_submit(krr_server *S, const double *X, int64_t N, int d, krr_kernel kern,
                             double sigma, const double *Y, int m, double mu, int k,
                             uint64_t seed, double tol, int maxit, double *alpha_out,
                             int64_t *id_out) {
  krr::clear_error();
  KRR_REQUIRE(S && X && Y && alpha_out, "NULL argument");
  KRR_REQUIRE(N >= 1 && N <= (int64_t)1 << 26, "N must be in [1, 2^26]");
  KRR_REQUIRE(d >= 1 && d <= 32, "d must be in [1, 32]");
  KRR_REQUIRE(kern == KRR_GAUSSIAN || kern == KRR_LAPLACE_L1 || kern == KRR_MATERN52,
              "unknown kernel %d", (int)kern);
  KRR_REQUIRE(sigma > 0 && std::isfinite(sigma), "sigma must be positive");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(mu > 0 && std::isfinite(mu), "mu must be positive");
  KRR_REQUIRE(k >= 0 && k <= N && k <= 4096, "k must be in [0, min(N, 4096)]");
  KRR_REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
  KRR_REQUIRE(maxit >= 1, "maxit must be >= 1");
  const int64_t bytes = (int64_t)std::ceil(krr::serve_footprint(N, d, m, k));
  if (bytes > S->budget) {
    krr::set_error("request needs about %.3g bytes, more than the server's budget %.3g",
                   (double)bytes, (double)S->budget);
    return KRR_ENOMEM;
  }
  std::unique_ptr<Slot> sl(new (std::nothrow) Slot());
  if (!sl) return KRR_ENOMEM;
  sl->req_id = S->next_id++;
  sl->X = X;
  sl->Y = Y;
  sl->alpha_out = alpha_out;
  sl->N = N;
  sl->d = d;
  sl->kern = (int)kern;
  sl->sigma = sigma;
  sl->m = m;
  sl->mu = mu;
  sl->k = k;
  sl->seed = seed;
  sl->tol = tol;
  sl->maxit = maxit;
  sl->bytes = bytes;
  sl->t_submit = S->now();
  if (id_out) *id_out = sl->req_id;
  S->queue.push_back(std::move(sl));
  S->submitted += 1;
  return KRR_OK;
}

krr_status krr_server_step(krr_server *S, int64_t *unfinished) {
  krr::clear_error();
  KRR_REQUIRE(S, "server is NULL");
  return krr::server_step(S, unfinished);
}

krr_status krr_server_poll(krr_server *S, krr_request_result *out, int max_results, int *n_out) {
  krr::clear_error();
  KRR_REQUIRE(S && n_out, "NULL argument");
  KRR_REQUIRE(max_results >= 0 && (out || max_results == 0), "bad result buffer");
  const int n = std::min<int>(max_results, (int)S->done.size());
  for (int i = 0; i < n; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + n);
  *n_out = n;
  return KRR_OK;
}

krr_status krr_server_get_stats(const krr_server *S, krr_server_stats *out) {
  krr::clear_error();
  KRR_REQUIRE(S && out, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->queued = (int64_t)S->queue.size();
  int64_t adm = 0;
  for (int i = 0; i < krr::SERVE_MAX_SLOTS; ++i) adm += S->slots[i] ? 1 : 0;
  out->admitted = adm;
  out->steps = S->steps;
  out->step_kernels = S->step_kernels;
  out->max_concurrent = S->max_concurrent;
  out->reserved_bytes = (double)S->reserved;
  out->peak_reserved_bytes = (double)S->peak_reserved;
  out->budget_bytes = (double)S->budget;
  out->kernel_entries = S->entries_total;
  out->step_ms = S->step_ms;
  for (int k = 0; k < krr::SERVE_KERNELS_PER_ITER; ++k) out->phase_ms[k] = S->phase_ms[k];
  {
    std::lock_guard<std::mutex> lk(const_cast<krr_server *>(S)->mtx);
    out->build_s = S->build_s;
    out->escalate_s = S->escalate_s;
    out->escalations = S->escalations;
  }
  return KRR_OK;
}

double krr_server_clock(const krr_server *S) { return S ? S->now() : 0.0; }

krr_status krr_server_progress(const krr_server *S, int64_t id, krr_request_progress *out) {
  krr::clear_error();
  KRR_REQUIRE(S && out, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->id = id;
  auto fill = [&](const Slot *sl, int state) {
    out->state = state;
    out->iters = sl->iters;
    out->outer_refinements = sl->outer;
    out->rel_residual = sl->relres;
  };
  for (int i = 0; i < krr::SERVE_MAX_SLOTS; ++i) {
    const Slot *sl = S->slots[i].get();
    if (!sl || sl->req_id != id) continue;
    int st = KRR_REQ_ITERATING;
    if (sl->phase == Phase::Building) st = KRR_REQ_BUILDING;
    else if (sl->phase == Phase::Escalated) st = KRR_REQ_ESCALATED;
    else if (sl->phase == Phase::Final) st = KRR_REQ_FINISHING;
    fill(sl, st);
    return KRR_OK;
  }
  for (const auto &sl : S->queue)
    if (sl->req_id == id) { fill(sl.get(), KRR_REQ_QUEUED); return KRR_OK; }
  for (const auto &sl : S->parked)
    if (sl->req_id == id) { fill(sl.get(), KRR_REQ_PARKED); return KRR_OK; }
  for (const auto &r : S->done)
    if (r.id == id) {
      out->state = KRR_REQ_DONE;
      out->iters = r.iters;
      out->outer_refinements = r.outer_refinements;
      out->rel_residual = r.rel_residual;
      return KRR_OK;
    }
  krr::set_error("request %lld is not known to the server (or was already polled)",
                 (long long)id);
  return KRR_EINVAL;
}

krr_status krr_server_evict(krr_server *S, int64_t id) {
  krr::clear_error();
  KRR_REQUIRE(S, "server is NULL");
  for (int i = 0; i < krr::SERVE_MAX_SLOTS; ++i) {
    Slot *sl = S->slots[i].get();
    if (!sl || sl->req_id != id) continue;
    KRR_REQUIRE(sl->phase != Phase::Escalated && sl->phase != Phase::Final,
                "request %lld is finishing and cannot be evicted", (long long)id);
    sl->evict_req = true;
    return KRR_OK;
  }
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
    if ((*it)->req_id != id) continue;
    // not started: nothing on the device, parked as it is
    S->parked.push_back(std::move(*it));
    S->queue.erase(it);
    return KRR_OK;
  }
  krr::set_error("request %lld is not queued or running", (long long)id);
  return KRR_EINVAL;
}

krr_status krr_server_resume(krr_server *S, int64_t id) {
  krr::clear_error();
  KRR_REQUIRE(S, "server is NULL");
  for (auto it = S->parked.begin(); it != S->parked.end(); ++it) {
    if ((*it)->req_id != id) continue;
    S->queue.push_front(std::move(*it));
    S->parked.erase(it);
    return KRR_OK;
  }
  krr::set_error("request %lld is not parked", (long long)id);
  return KRR_EINVAL;
}

krr_status krr_server_export(krr_server *S, int64_t id, void *buf, size_t *size) {
  krr::clear_error();
  KRR_REQUIRE(S && size, "NULL argument");
  for (auto it = S->parked.begin(); it != S->parked.end(); ++it) {
    Slot *sl = it->get();
    if (sl->req_id != id) continue;
    const size_t nm = sl->resume ? (size_t)sl->N * sl->m : 0;
    const size_t need = sizeof(Checkpoint) + sizeof(double) * (2 * (size_t)sl->m + 2 * nm);
    if (!buf) {
      *size = need;
      return KRR_OK;
    }
    KRR_REQUIRE(*size >= need, "checkpoint needs %zu bytes, buffer has %zu", need, *size);
    Checkpoint h{};
    std::memcpy(h.magic, kCheckpointMagic, sizeof(h.magic));
    h.version = 1;
    h.header_bytes = (uint32_t)sizeof(Checkpoint);
    h.N = sl->N;
    h.d = sl->d;
    h.kern = sl->kern;
    h.m = sl->m;
    h.k = sl->k;
    h.sigma = sl->sigma;
    h.mu = sl->mu;
    h.tol = sl->tol;
    h.seed = sl->seed;
    h.maxit = sl->maxit;
    h.outer = sl->resume ? sl->outer : -1;   // -1: not started
    h.iters = sl->iters;
    h.budget = sl->budget;
    h.prev_worst = sl->prev_worst;
    h.relres = sl->relres;
    h.entries = sl->entries;
    char *p = (char *)buf;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    std::vector<double> zeros(sl->m, 0.0);
    const std::vector<double> &yn = sl->resume ? sl->yn : zeros;
    const std::vector<double> &rn = sl->resume ? sl->rn : zeros;
    std::memcpy(p, yn.data(), sizeof(double) * sl->m);
    p += sizeof(double) * sl->m;
    std::memcpy(p, rn.data(), sizeof(double) * sl->m);
    p += sizeof(double) * sl->m;
    if (nm) {
      std::memcpy(p, sl->saved_alpha.data(), sizeof(double) * nm);
      p += sizeof(double) * nm;
      std::memcpy(p, sl->saved_r.data(), sizeof(double) * nm);
    }
    *size = need;
    S->parked.erase(it);
    return KRR_OK;
  }
  krr::set_error("request %lld is not parked", (long long)id);
  return KRR_EINVAL;
}

krr_status krr_server_import(krr_server *S, const void *buf, size_t size, const double *X,
                             const double *Y, double *alpha_out, int64_t *id_out) {
  krr::clear_error();
  KRR_REQUIRE(S && buf && X && Y && alpha_out, "NULL argument");
  KRR_REQUIRE(size >= sizeof(Checkpoint), "checkpoint too short");
  Checkpoint h;
  std::memcpy(&h, buf, sizeof(h));
  KRR_REQUIRE(std::memcmp(h.magic, kCheckpointMagic, sizeof(h.magic)) == 0 && h.version == 1 &&
                  h.header_bytes == sizeof(Checkpoint),
              "not a checkpoint of this library");
  KRR_REQUIRE(h.N >= 1 && h.N <= (int64_t)1 << 26 && h.d >= 1 && h.d <= 32 && h.m >= 1 &&
                  h.m <= 16 && h.k >= 0 && h.k <= h.N && h.kern >= 0 && h.kern <= 2,
              "corrupt checkpoint header");
  const bool started = h.outer >= 0;
  const size_t nm = started ? (size_t)h.N * h.m : 0;
  const size_t need = sizeof(Checkpoint) + sizeof(double) * (2 * (size_t)h.m + 2 * nm);
  KRR_REQUIRE(size >= need, "checkpoint truncated (%zu of %zu bytes)", size, need);
  int64_t id = -1;
  KRR_TRY(krr_server_submit(S, X, h.N, h.d, (krr_kernel)h.kern, h.sigma, Y, h.m, h.mu, h.k,
                            h.seed, h.tol, h.maxit, alpha_out, &id));
  if (started) {
    Slot *sl = S->queue.back().get();
    const char *p = (const char *)buf + sizeof(Checkpoint);
    sl->yn.assign((const double *)p, (const double *)p + h.m);
    p += sizeof(double) * h.m;
    sl->rn.assign((const double *)p, (const double *)p + h.m);
    p += sizeof(double) * h.m;
    sl->saved_alpha.assign((const double *)p, (const double *)p + nm);
    p += sizeof(double) * nm;
    sl->saved_r.assign((const double *)p, (const double *)p + nm);
    sl->outer = h.outer;
    sl->iters = h.iters;
    sl->budget = h.budget;
    sl->prev_worst = h.prev_worst;
    sl->relres = h.relres;
    sl->entries = h.entries;
    sl->resume = true;
  }
  if (id_out) *id_out = id;
  return KRR_OK;
}

void krr_server_destroy(krr_server *S) { krr::server_free(S); }

}  // extern "C"
