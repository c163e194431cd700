// Blocked RPCholesky (Alg. 3) on the device, float64.
//
// Per block: (1) fixed-point pivot sampling from the residual diagonal
// (residuals at or below the drop threshold carry no weight) and
// Unique in first-occurrence order; (2) G = A(:,S') from the kernel function
// minus the Schur term F(:,1:i) F(S',1:i)^T (GEMM); (3) Cholesky of G(S',S')
// pivot by pivot with the drop rule; (4) the new columns G R^{-1} by forward
// substitution, fused with the residual-diagonal downdate.
#include "dense.cuh"
#include "handles.cuh"
#include "kmv.cuh"
#include "rpc.cuh"

namespace krr {

// ------------------------------------------------------------- sampler
__device__ __forceinline__ uint64_t fixed_weight(double v, double dfloor, int fbits) {
  if (!(v > 0.0) || !(v > dfloor)) return 0ull;
  if (v > 1.0) v = 1.0;
  return __double2ull_rz(ldexp(v, fbits));
}

int fixed_point_bits(int64_t N) {
  int c = 0;
  while (((int64_t)1 << c) < N) ++c;
  return 62 - c;
}

constexpr int SMP_THREADS = 256;
constexpr int SMP_MAX_CHUNKS = 4096;

static int64_t sampler_chunk(int64_t N) {
  int64_t ch = 2048;
  while ((N + ch - 1) / ch > SMP_MAX_CHUNKS) ch *= 2;
  return ch;
}

__global__ void __launch_bounds__(SMP_THREADS)
sample_chunk_sums_kernel(const double *__restrict__ dres, int64_t N, double dfloor,
                         int fbits, int64_t chunk, uint64_t *__restrict__ csum) {
  __shared__ uint64_t red[SMP_THREADS / 32];
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = min(N, b0 + chunk);
  uint64_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += SMP_THREADS) s += fixed_weight(dres[i], dfloor, fbits);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < SMP_THREADS / 32; ++w) t += red[w];
    csum[blockIdx.x] = t;
  }
}

// One CTA: prefix of chunk sums, ndraw draws (one warp per draw), then Unique
// (first-occurrence order) by one thread.
__global__ void __launch_bounds__(SMP_THREADS)
sample_draw_kernel(const double *__restrict__ dres, int64_t N, double dfloor, int fbits,
                   int64_t chunk,
                   const uint64_t *__restrict__ csum, int nchunks, uint64_t seed,
                   uint64_t t, int ndraw, int64_t *__restrict__ draws,
                   int64_t *__restrict__ cand, int *__restrict__ counts) {
  __shared__ uint64_t cpre[SMP_MAX_CHUNKS];
  __shared__ uint64_t total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    for (int c = 0; c < nchunks; ++c) {
      run += csum[c];
      cpre[c] = run;
    }
    total = run;
  }
  __syncthreads();
  if (total == 0) {
    if (threadIdx.x == 0) {
      counts[0] = 0;
      counts[1] = 0;
    }
    return;
  }
  for (int j = warp; j < ndraw; j += SMP_THREADS / 32) {
    uint64_t ctr[4] = {t, (uint64_t)j, 0ull, 0ull}, out[4];
    philox4x64_10(ctr, seed, kTagPivots, out);
    const uint64_t target = scale_u64(out[0], total);
    // smallest chunk whose inclusive prefix exceeds the target
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cpre[mid] > target) hi = mid; else lo = mid + 1;
    }
    const uint64_t base = cpre[lo] - csum[lo];
    const uint64_t tl = target - base;
    const int64_t b0 = (int64_t)lo * chunk, b1 = min(N, b0 + chunk);
    uint64_t run = 0;
    int64_t pick = b1 - 1;
    for (int64_t off = b0; off < b1; off += 32) {
      const int64_t i = off + lane;
      const uint64_t w = (i < b1) ? fixed_weight(dres[i], dfloor, fbits) : 0ull;
      uint64_t incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint64_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (run + tot > tl) {
        const unsigned hit = __ballot_sync(0xffffffffu, run + incl > tl);
        pick = off + (__ffs(hit) - 1);
        break;
      }
      run += tot;
    }
    if (lane == 0) draws[j] = pick;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nc = 0;
    for (int j = 0; j < ndraw; ++j) {
      const int64_t v = draws[j];
      bool seen = false;
      for (int c = 0; c < nc; ++c)
        if (cand[c] == v) { seen = true; break; }
      if (!seen) cand[nc++] = v;
    }
    counts[0] = ndraw;
    counts[1] = nc;
  }
}

krr_status rpc_sample_device(const double *dres, int64_t N, double dfloor, uint64_t seed,
                             uint64_t t, int ndraw, int64_t *draws, int64_t *cand, int *counts,
                             cudaStream_t s) {
  const int fbits = fixed_point_bits(N);
  const int64_t chunk = sampler_chunk(N);
  const int nchunks = (int)((N + chunk - 1) / chunk);
  DevBuf<uint64_t> csum;
  KRR_TRY(csum.alloc(nchunks, s));
  sample_chunk_sums_kernel<<<nchunks, SMP_THREADS, 0, s>>>(dres, N, dfloor, fbits, chunk,
                                                           csum.p);
  KRR_LAUNCH_CHECK();
  sample_draw_kernel<<<1, SMP_THREADS, 0, s>>>(dres, N, dfloor, fbits, chunk, csum.p, nchunks,
                                               seed, t, ndraw, draws, cand, counts);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// --------------------------------------------- uniform and greedy rules
// The pivot rules the paper compares RPCholesky with (Sec. 4).
//
// Uniform: a uniformly random k-subset of the columns, drawn independently
// of A: draw q takes word 0 of Philox(counter (q, 0, 1, 0), key (seed, pivot
// tag)) as floor(u N / 2^64), keeping first occurrences (a bitmap of the
// columns seen) until k distinct indices are found.  One thread; the loop is
// bounded (far above the expected k + k^2 / (2N) draws for k <= N) and
// reports failure through out_count.
__global__ void uniform_pivots_kernel(int64_t N, int k, uint64_t seed, unsigned *__restrict__ seen,
                                      int64_t *__restrict__ S, int *__restrict__ out_count) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int got = 0;
  const uint64_t qmax = 64ull * (uint64_t)k + 4096ull;
  for (uint64_t q = 0; got < k && q < qmax; ++q) {
    uint64_t ctr[4] = {q, 0ull, 1ull, 0ull}, out[4];
    philox4x64_10(ctr, seed, kTagPivots, out);
    const int64_t i = (int64_t)scale_u64(out[0], (uint64_t)N);
    const unsigned bit = 1u << (i & 31);
    if (seen[i >> 5] & bit) continue;
    seen[i >> 5] |= bit;
    S[got++] = i;
  }
  *out_count = got;
}

// Greedy: the npick largest residuals above dfloor in descending order (ties:
// the smallest index); npick = 1 is the paper's rule.  One CTA; pick j is the
// largest (value, -index) strictly below pick j - 1 in that order.
constexpr int GREEDY_THREADS = 1024;

// Smallest N whose Schur updates take the float-float GEMM: the drop
// threshold N 2^-52 max A_ii is then at least 7e-12, about 70 times the
// float-float rounding of a partial sum of magnitude 1 over 1000 terms.
constexpr int64_t kSchurFFMinN = 32768;
__global__ void __launch_bounds__(GREEDY_THREADS)
greedy_pick_kernel(const double *__restrict__ dres, int64_t N, double dfloor, int npick,
                   int64_t *__restrict__ cand, int *__restrict__ counts) {
  __shared__ double sv[GREEDY_THREADS / 32];
  __shared__ int64_t si[GREEDY_THREADS / 32];
  __shared__ double prev_v;
  __shared__ int64_t prev_i;
  __shared__ int got;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    prev_v = INFINITY;
    prev_i = -1;
    got = 0;
  }
  __syncthreads();
  for (int j = 0; j < npick; ++j) {
    const double pv = prev_v;
    const int64_t pi = prev_i;
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < N; i += GREEDY_THREADS) {
      const double v = dres[i];
      if (!(v > 0.0) || !(v > dfloor)) continue;
      // strictly after the previous pick in (value desc, index asc) order
      if (v > pv || (v == pv && i <= pi)) continue;
      if (bi < 0 || v > bv) {
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      sv[warp] = bv;
      si[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = -1.0;
      int64_t b = -1;
      for (int w = 0; w < GREEDY_THREADS / 32; ++w) {
        if (si[w] >= 0 && (b < 0 || sv[w] > v || (sv[w] == v && si[w] < b))) {
          v = sv[w];
          b = si[w];
        }
      }
      if (b >= 0) {
        cand[got] = b;
        got = got + 1;
        prev_v = v;
        prev_i = b;
      }
    }
    __syncthreads();
    if (got <= j) break;   // nothing eligible left
  }
  if (threadIdx.x == 0) {
    counts[0] = got > 0 ? npick : 0;
    counts[1] = got;
  }
}

// ------------------------------------------------------- block kernels
// Fs (nc x rank, column-major) = F(cand, 0:rank)
__global__ void gather_rows_kernel(const double *__restrict__ F, int64_t N, int rank,
                                   const int64_t *__restrict__ cand, int nc,
                                   double *__restrict__ Fs) {
  const int64_t total = (int64_t)nc * rank;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nc);
    const int l = (int)(e / nc);
    Fs[e] = F[cand[c] + (int64_t)l * N];
  }
}

// Right-looking Cholesky of T = G(S', S') (nc x nc) in candidate order; a
// candidate whose current Schur value is <= thr is dropped and does not
// update the rest.  Outputs the factor entries Lb (nc x nc, column-major,
// lower, rows/columns of dropped candidates unused), the kept positions in
// order, and their count.
__global__ void __launch_bounds__(256)
block_chol_kernel(const double *__restrict__ G, int64_t ldg, const int64_t *__restrict__ cand,
                  int nc, double thr, double *__restrict__ Lb, int *__restrict__ kept,
                  int *__restrict__ nkept) {
  extern __shared__ double sT[];  // nc x nc, row-major
  __shared__ int s_keep;
  __shared__ int s_list[RPC_MAX_BLOCK];
  __shared__ int s_na;
  const int tid = threadIdx.x;
  for (int e = tid; e < nc * nc; e += blockDim.x) {
    const int a = e / nc, c = e % nc;
    sT[a * nc + c] = G[cand[a] + (int64_t)c * ldg];
  }
  if (tid == 0) s_na = 0;
  __syncthreads();
  for (int c = 0; c < nc; ++c) {
    if (tid == 0) {
      const double p = sT[c * nc + c];
      s_keep = (p > thr) ? 1 : 0;
      if (s_keep) {
        sT[c * nc + c] = sqrt(p);
        s_list[s_na] = c;
        s_na = s_na + 1;
      }
    }
    __syncthreads();
    if (s_keep) {
      const double dc = sT[c * nc + c];
      for (int a = c + 1 + tid; a < nc; a += blockDim.x) sT[a * nc + c] /= dc;
      __syncthreads();
      const int rem = nc - c - 1;
      for (int e = tid; e < rem * rem; e += blockDim.x) {
        const int a = c + 1 + e / rem, b = c + 1 + e % rem;
        if (b <= a) sT[a * nc + b] -= sT[a * nc + c] * sT[b * nc + c];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nc * nc; e += blockDim.x) {
    const int a = e % nc, c = e / nc;
    Lb[a + (int64_t)c * nc] = (a >= c) ? sT[a * nc + c] : 0.0;
  }
  for (int e = tid; e < s_na; e += blockDim.x) kept[e] = s_list[e];
  if (tid == 0) *nkept = s_na;
}

// New columns: row n solves x L_kk^T = G(n, kept) by forward substitution and
// writes x to F(n, rank : rank + na); dres(n) -= |x|^2.
__global__ void __launch_bounds__(128)
block_trsm_kernel(const double *__restrict__ G, int64_t ldg, const double *__restrict__ Lb,
                  int nc, const int *__restrict__ kept, const int *__restrict__ nkept,
                  double *__restrict__ F, int64_t N, int rank, double *__restrict__ dres) {
  extern __shared__ double sL[];  // na x na, row-major, kept rows/cols only
  const int na = *nkept;
  for (int e = threadIdx.x; e < na * na; e += blockDim.x) {
    const int a = e / na, b = e % na;
    sL[e] = (b <= a) ? Lb[kept[a] + (int64_t)kept[b] * nc] : 0.0;
  }
  __syncthreads();
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s2 = 0.0;
  double *Fn = F + n + (int64_t)rank * N;
  for (int a = 0; a < na; ++a) {
    double v = G[n + (int64_t)kept[a] * ldg];
    for (int b = 0; b < a; ++b) v -= Fn[(int64_t)b * N] * sL[a * na + b];
    v /= sL[a * na + a];
    Fn[(int64_t)a * N] = v;
    s2 = fma(v, v, s2);
  }
  dres[n] -= s2;
}

__global__ void block_finish_kernel(const int64_t *__restrict__ cand, int nc,
                                    const int *__restrict__ kept, const int *__restrict__ nkept,
                                    int64_t *__restrict__ S, int rank,
                                    double *__restrict__ dres) {
  const int na = *nkept;
  for (int e = threadIdx.x; e < na; e += blockDim.x) S[rank + e] = cand[kept[e]];
  for (int c = threadIdx.x; c < nc; c += blockDim.x) dres[cand[c]] = 0.0;
}

__global__ void max_reduce_kernel(const double *__restrict__ v, int64_t n,
                                  double *__restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    *out = r;
  }
}

// ----------------------------------------------------------- driver
krr_status rpcholesky_device(const double *Xd, int64_t N, int d, int kern, double sigma,
                             int k, int B, uint64_t seed, cudaStream_t s, krr_factor *f,
                             int rule) {
  f->N = N;
  f->d = d;
  f->kern = kern;
  f->sigma = sigma;
  f->k = k;
  f->seed = seed;
  KRR_TRY(dev_alloc(&f->F, (size_t)N * k));
  KRR_TRY(dev_alloc(&f->S, (size_t)k));
  KRR_TRY(dev_alloc(&f->dres, (size_t)N));
  KRR_CUDA_TRY(cudaMemsetAsync(f->F, 0, sizeof(double) * (size_t)N * k, s));
  KRR_TRY(kernel_diag_f64(Xd, N, d, kern, sigma, f->dres, s));

  DevBuf<double> maxd;
  KRR_TRY(maxd.alloc(1, s));
  max_reduce_kernel<<<1, 1024, 0, s>>>(f->dres, N, maxd.p);
  KRR_LAUNCH_CHECK();
  double maxdiag = 0.0;
  KRR_CUDA_TRY(cudaMemcpyAsync(&maxdiag, maxd.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  const double thr = (double)N * 2.220446049250313e-16 * maxdiag;

  DevBuf<int64_t> draws, cand;
  DevBuf<int> counts, kept;
  DevBuf<double> G, Fs, Lb;
  KRR_TRY(draws.alloc(B, s));
  KRR_TRY(cand.alloc(B, s));
  KRR_TRY(counts.alloc(4, s));
  KRR_TRY(kept.alloc(B, s));
  KRR_TRY(G.alloc((size_t)N * B, s));
  KRR_TRY(Fs.alloc((size_t)B * k, s));
  KRR_TRY(Lb.alloc((size_t)B * B, s));

  const size_t chol_smem = (size_t)B * B * sizeof(double);
  KRR_TRY(raise_smem_limit(block_chol_kernel, chol_smem));
  KRR_TRY(raise_smem_limit(block_trsm_kernel, chol_smem));

  // the uniform rule's k pivots are drawn before the first block
  DevBuf<int64_t> upiv;
  int nupiv = 0, used = 0;
  if (rule == KRR_PIVOT_UNIFORM) {
    DevBuf<unsigned> seen;
    KRR_TRY(seen.alloc((size_t)(N + 31) / 32, s));
    KRR_TRY(upiv.alloc(k, s));
    KRR_CUDA_TRY(cudaMemsetAsync(seen.p, 0, sizeof(unsigned) * (size_t)((N + 31) / 32), s));
    uniform_pivots_kernel<<<1, 32, 0, s>>>(N, k, seed, seen.p, upiv.p, counts.p);
    KRR_LAUNCH_CHECK();
    KRR_CUDA_TRY(cudaMemcpyAsync(&nupiv, counts.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    KRR_CUDA_TRY(cudaStreamSynchronize(s));
    if (nupiv < k) {
      set_error("uniform pivot draw ended early (%d of %d)", nupiv, k);
      return KRR_ECUDA;
    }
  }

  int rank = 0;
  uint64_t t = 0;
  int hcounts[4];
  while (rule == KRR_PIVOT_UNIFORM ? used < nupiv : rank < k) {
    int nc;
    if (rule == KRR_PIVOT_UNIFORM) {
      nc = (nupiv - used < B) ? (nupiv - used) : B;
      KRR_CUDA_TRY(cudaMemcpyAsync(cand.p, upiv.p + used, sizeof(int64_t) * nc,
                                   cudaMemcpyDeviceToDevice, s));
      used += nc;
      ++t;
    } else {
      const int nd = (k - rank < B) ? (k - rank) : B;
      if (rule == KRR_PIVOT_GREEDY) {
        greedy_pick_kernel<<<1, GREEDY_THREADS, 0, s>>>(f->dres, N, thr, nd, cand.p, counts.p);
        KRR_LAUNCH_CHECK();
      } else {
        KRR_TRY(rpc_sample_device(f->dres, N, thr, seed, t, nd, draws.p, cand.p, counts.p, s));
      }
      ++t;
      KRR_CUDA_TRY(cudaMemcpyAsync(hcounts, counts.p, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                   s));
      KRR_CUDA_TRY(cudaStreamSynchronize(s));
      if (hcounts[0] == 0) break;
      nc = hcounts[1];
    }
    // G = A(:, S') - F(:, 0:rank) F(S', 0:rank)^T
    KRR_TRY(kernel_columns_f64(Xd, N, d, kern, sigma, cand.p, nc, G.p, N, s));
    if (rank > 0) {
      gather_rows_kernel<<<ceil_div((int64_t)nc * rank, 256), 256, 0, s>>>(f->F, N, rank,
                                                                         cand.p, nc, Fs.p);
      KRR_LAUNCH_CHECK();
      Gemm<double> g;
      g.M = (int)N; g.N = nc; g.K = rank;
      g.A = f->F; g.sai = 1; g.sak = N;
      g.B = Fs.p; g.sbk = nc; g.sbj = 1;
      g.alpha = -1.0; g.beta = 1.0; g.C = G.p; g.ldc = N;
      // float-float on the float32 pipes where its rounding (about 1e-13 of
      // the partial sums) stays two orders below the drop threshold
      // N 2^-52 max A_ii; float64 below that size
      if (N >= kSchurFFMinN) KRR_TRY(gemm_sub_ff(g, s));
      else KRR_TRY(gemm(g, s));
    }
    block_chol_kernel<<<1, 256, (size_t)nc * nc * sizeof(double), s>>>(G.p, N, cand.p, nc, thr,
                                                                     Lb.p, kept.p, counts.p + 2);
    KRR_LAUNCH_CHECK();
    block_trsm_kernel<<<ceil_div(N, 128), 128, (size_t)nc * nc * sizeof(double), s>>>(
        G.p, N, Lb.p, nc, kept.p, counts.p + 2, f->F, N, rank, f->dres);
    KRR_LAUNCH_CHECK();
    block_finish_kernel<<<1, 128, 0, s>>>(cand.p, nc, kept.p, counts.p + 2, f->S, rank, f->dres);
    KRR_LAUNCH_CHECK();
    int na = 0;
    KRR_CUDA_TRY(cudaMemcpyAsync(&na, counts.p + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    KRR_CUDA_TRY(cudaStreamSynchronize(s));
    rank += na;
  }
  f->rank = rank;
  f->nblocks = (int)t;
  return KRR_OK;
}

}  // namespace krr
