// Float64-accurate fused product on the float32 pipes ("double-float").
//
// The mixed-precision refinement needs its residual y - (A + lambda I)x with
// kernel entries accurate far beyond float32, but this part's float64 pipe
// runs at 1/73 of its float32 rate.  Here every value is an unevaluated sum
// hi + lo of two floats (about 48 significant bits) and all arithmetic uses
// error-free transformations: TwoSum (Knuth), TwoProd by FMA (Dekker's
// product with a fused multiply-add), and renormalisation by FastTwoSum.
// Intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from
// contracting or reassociating them.
//
// Per entry (i, j):
//   distance   from direct coordinate differences of pre-scaled points split
//              as x = xh + xl: xh_i - xh_j exactly by TwoSum, squares exactly
//              by TwoProd, the sum compensated by TwoSum (Gaussian, Matern:
//              S = |x_i - x_j|^2; Laplace: S = sum |x_i - x_j|).  Direct
//              differences keep every intermediate the size of S, so the
//              exponent is accurate to ~2^-48 S rather than 2^-48 |x|^2 (the
//              norm expansion the float32 product uses loses that for near
//              points).
//   exp        arg -> k = round(arg 32 / ln 2), r = arg - k ln2/32 (Cody-Waite
//              with a three-float ln2/32), exp(r) = 1 + r + r^2/2 + r^3 p(r)
//              (Taylor; the cubic tail in float is below 2^-46 for
//              |r| <= ln2/64), times the table value 2^(j/32) (hi + lo floats
//              computed on the host) and 2^(k div 32).
//   accumulate  acc_c += kappa v_jc with TwoProd + TwoSum per right-hand side.
// Partial sums are written as float64 and reduced with lambda V in float64.
#pragma once

#include "common.cuh"

namespace krr {

struct FF {
  float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  FF p = two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return fast_two_sum(p.h, p.l);
}

// Constants of the exponential (filled on the host, see kmv_ff.cu):
//   c[0] = 32 / ln 2 (float), c[1..3] = ln2/32 split into three floats with
//   c[1] carrying 8 significant bits (so k c[1] is exact for |k| < 2^16),
//   tab[2 j], tab[2 j + 1] = hi, lo of 2^(j/32).
struct ExpFFConsts {
  float c[4];
  float tab[64];
};

// exp(a) for a = a.h + a.l <= 0 (tiny positive values from rounding are fine).
__device__ __forceinline__ FF exp_ff(FF a, const float *__restrict__ cst,
                                     const float *__restrict__ tab) {
  if (a.h < -87.0f) return {0.0f, 0.0f};
  const float kf = rintf(__fmul_rn(a.h, cst[0]));
  const int k = (int)kf;
  // r = a - k ln2/32
  const float t1 = __fmaf_rn(-kf, cst[1], a.h);           // exact (Sterbenz / few bits)
  FF kc2 = two_prod(kf, cst[2]);
  FF r = two_sum(t1, -kc2.h);
  r.l = __fadd_rn(r.l, __fadd_rn(__fsub_rn(a.l, kc2.l), -__fmul_rn(kf, cst[3])));
  r = fast_two_sum(r.h, r.l);
  // exp(r) - 1 = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720)
  const float rh = r.h;
  float q = __fmaf_rn(rh, 1.0f / 720.0f, 1.0f / 120.0f);
  q = __fmaf_rn(rh, q, 1.0f / 24.0f);
  q = __fmaf_rn(rh, q, 1.0f / 6.0f);
  q = __fmul_rn(q, __fmul_rn(rh, __fmul_rn(rh, rh)));
  FF r2 = two_prod(rh, rh);
  r2.l = __fmaf_rn(2.0f * rh, r.l, r2.l);
  r2.h *= 0.5f;
  r2.l *= 0.5f;
  FF em1 = ff_add(r, r2);
  em1.l = __fadd_rn(em1.l, q);
  // kappa = T_j (1 + em1) = T_j + T_j em1
  const int j = k & 31;
  const int n = (k - j) / 32;  // exact: k - j is a multiple of 32
  const FF T = {tab[2 * j], tab[2 * j + 1]};
  FF v = ff_add(T, ff_mul(T, em1));
  if (n < -125) {
    const float s1 = __int_as_float((n + 64 + 127) << 23);   // 2^(n + 64)
    const float s2 = __int_as_float((127 - 64) << 23);        // 2^-64
    v.h = __fmul_rn(__fmul_rn(v.h, s1), s2);
    v.l = __fmul_rn(__fmul_rn(v.l, s1), s2);
  } else {
    const float sc = __int_as_float((n + 127) << 23);
    v.h = __fmul_rn(v.h, sc);
    v.l = __fmul_rn(v.l, sc);
  }
  return v;
}

// ff square root of a positive ff value (one Newton correction).
__device__ __forceinline__ FF sqrt_ff(FF a) {
  if (!(a.h > 0.0f)) return {0.0f, 0.0f};
  const float s = __fsqrt_rn(a.h);
  const FF ss = two_prod(s, s);
  const float corr = __fdiv_rn(__fadd_rn(__fsub_rn(a.h, ss.h), __fsub_rn(a.l, ss.l)),
                               __fmul_rn(2.0f, s));
  return fast_two_sum(s, corr);
}

// kappa(x_i, x_j) in float-float from split points (xh + xl, pre-scaled):
// direct coordinate differences, float-float exponential (and the Matern
// polynomial).
template <int KERN, int DP>
__device__ __forceinline__ FF ff_kernel_value(const float (&ih)[DP], const float (&il)[DP],
                                              const float *jh, const float *jl,
                                              const float *__restrict__ cst,
                                              const float *__restrict__ tab) {
  FF arg;
  if constexpr (KERN == KLAPLACE) {
    FF s = {0.0f, 0.0f};
    float lo = 0.0f;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      FF dd = two_sum(ih[k], -jh[k]);
      dd.l = __fadd_rn(dd.l, __fsub_rn(il[k], jl[k]));
      // sign of the unevaluated sum (dd.h is 0 when the high parts agree)
      if (__fadd_rn(dd.h, dd.l) < 0.0f) {
        dd.h = -dd.h;
        dd.l = -dd.l;
      }
      const FF t = two_sum(s.h, dd.h);
      s.h = t.h;
      lo = __fadd_rn(lo, __fadd_rn(t.l, dd.l));
    }
    s = fast_two_sum(s.h, __fadd_rn(s.l, lo));
    arg = {-s.h, -s.l};
  } else {
    // S = sum_k (x_ik - x_jk)^2 with exact differences (TwoSum) and exact
    // squares (TwoProd): intermediates stay the size of S.
    FF s = {0.0f, 0.0f};
    float lo = 0.0f;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      FF dd = two_sum(ih[k], -jh[k]);
      dd.l = __fadd_rn(dd.l, __fsub_rn(il[k], jl[k]));
      const FF p = two_prod(dd.h, dd.h);
      // d^2 = dh^2 + 2 dh dl + dl^2 (dl^2 matters when dh is 0 or tiny)
      const float cross = __fmaf_rn(__fadd_rn(dd.h, dd.h), dd.l, __fmaf_rn(dd.l, dd.l, p.l));
      const FF t = two_sum(s.h, p.h);
      s.h = t.h;
      lo = __fadd_rn(lo, __fadd_rn(t.l, cross));
    }
    s = fast_two_sum(s.h, lo);
    if constexpr (KERN == KMATERN) {
      // q = sqrt(S);  kappa = (1 + q + q^2/3) exp(-q)
      const FF q = sqrt_ff(s);
      arg = {-q.h, -q.l};
    } else {
      arg = {-0.5f * s.h, -0.5f * s.l};  // Gaussian: -|x - y|^2 / (2 sigma^2)
    }
  }
  FF kv = exp_ff(arg, cst, tab);
  if constexpr (KERN == KMATERN) {
    const FF q = {-arg.h, -arg.l};
    FF q2 = ff_mul(q, q);
    const FF third = {0.3333333433f, -9.9341077e-09f};  // 1/3 = hi + lo
    FF poly = ff_add({1.0f, 0.0f}, ff_add(q, ff_mul(q2, third)));
    kv = ff_mul(poly, kv);
  }
  return kv;
}

// acc += a b for float-float acc and a, b = bh + bl (TwoProd + TwoSum, the
// low-order products folded into the low part).
__device__ __forceinline__ void ff_fma_acc(FF &acc, FF a, float bh, float bl) {
  const FF p = two_prod(a.h, bh);
  const float cross = __fmaf_rn(a.h, bl, __fmaf_rn(a.l, bh, p.l));
  const FF t = two_sum(acc.h, p.h);
  acc.h = t.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t.l, cross));
}

constexpr int KFF_THREADS = 128;
constexpr int KFF_TJ = 32;                // columns per shared tile

// Rows per thread: two independent compensated chains while the split points
// fit the register budget, one otherwise.
__host__ __device__ constexpr int kmvff_rows_per_thread(int DP) { return DP <= 16 ? 2 : 1; }

// CTAs per SM the register budget is sized for: with two rows per thread,
// three CTAs (up to 170 registers, no spills) measured 7.6% faster than four
// (128 registers) at N = 1e5, d = 16, m = 4.
__host__ __device__ constexpr int kmvff_min_blocks(int DP) { return DP <= 16 ? 3 : 4; }

// rh, rl : Nr x DP split row points (the column arrays for the square
// product); xh, xl : N x DP split column points; ch, cl: N split constants
// (not used by the direct-difference distance).  Vh, Vl: m x N split RHS.
// part: splits x M x Nr float64.
template <int KERN, int DP, int M>
__global__ void __launch_bounds__(KFF_THREADS, kmvff_min_blocks(DP))
kmvff_kernel(const float *__restrict__ rh, const float *__restrict__ rl, int64_t Nr,
             const float *__restrict__ xh, const float *__restrict__ xl,
             const float *__restrict__ ch, const float *__restrict__ cl,
             const float *__restrict__ Vh, const float *__restrict__ Vl, int64_t N, int m,
             int64_t chunk, ExpFFConsts ec, double *__restrict__ part) {
  __shared__ float sxh[KFF_TJ][DP], sxl[KFF_TJ][DP];
  __shared__ float sch[KFF_TJ], scl[KFF_TJ];
  __shared__ float svh[KFF_TJ][M], svl[KFF_TJ][M];
  __shared__ float s_cst[4], s_tab[64];
  const int tid = threadIdx.x;
  if (tid < 4) s_cst[tid] = ec.c[tid];
  if (tid < 64) s_tab[tid] = ec.tab[tid];
  constexpr int KFF_RI = kmvff_rows_per_thread(DP);
  const int64_t row0 = (int64_t)blockIdx.x * KFF_THREADS * KFF_RI;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(N, j_begin + chunk);

  float ih[KFF_RI][DP], il[KFF_RI][DP];
  FF ic[KFF_RI];
  FF acc[KFF_RI][M];
#pragma unroll
  for (int r = 0; r < KFF_RI; ++r) {
    const int64_t i = row0 + tid + (int64_t)r * KFF_THREADS;
    const bool ok = i < Nr;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      ih[r][k] = ok ? rh[i * DP + k] : 0.0f;
      il[r][k] = ok ? rl[i * DP + k] : 0.0f;
    }
    ic[r] = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < M; ++c) acc[r][c] = {0.0f, 0.0f};
  }

  for (int64_t j0 = j_begin; j0 < j_end; j0 += KFF_TJ) {
    __syncthreads();
    for (int idx = tid; idx < KFF_TJ * DP; idx += KFF_THREADS) {
      const int jj = idx / DP, k = idx % DP;
      const int64_t j = j0 + jj;
      const bool ok = j < j_end;
      sxh[jj][k] = ok ? xh[j * DP + k] : 0.0f;
      sxl[jj][k] = ok ? xl[j * DP + k] : 0.0f;
    }
    for (int idx = tid; idx < KFF_TJ * M; idx += KFF_THREADS) {
      const int c = idx / KFF_TJ, jj = idx % KFF_TJ;
      const int64_t j = j0 + jj;
      const bool ok = (j < j_end) && (c < m);
      svh[jj][c] = ok ? Vh[(int64_t)c * N + j] : 0.0f;
      svl[jj][c] = ok ? Vl[(int64_t)c * N + j] : 0.0f;
    }
    if (tid < KFF_TJ) {
      const int64_t j = j0 + tid;
      const bool ok = j < j_end;
      sch[tid] = ok ? ch[j] : 0.0f;
      scl[tid] = ok ? cl[j] : 0.0f;
    }
    __syncthreads();
    const int jn = (int)min((int64_t)KFF_TJ, j_end - j0);
#pragma unroll 1
    for (int jj = 0; jj < jn; ++jj) {
#pragma unroll
      for (int r = 0; r < KFF_RI; ++r) {
        const FF kv = ff_kernel_value<KERN, DP>(ih[r], il[r], sxh[jj], sxl[jj], s_cst, s_tab);
#pragma unroll
        for (int c = 0; c < M; ++c) ff_fma_acc(acc[r][c], kv, svh[jj][c], svl[jj][c]);
      }
    }
  }
  double *out = part + (int64_t)blockIdx.y * M * Nr;
#pragma unroll
  for (int r = 0; r < KFF_RI; ++r) {
    const int64_t i = row0 + tid + (int64_t)r * KFF_THREADS;
    if (i < Nr) {
#pragma unroll
      for (int c = 0; c < M; ++c)
        if (c < m) out[(int64_t)c * Nr + i] = (double)acc[r][c].h + (double)acc[r][c].l;
    }
  }
}


// ---------------------------------------------------------------------------
// Symmetric square product: K is symmetric, so each pair of row tiles (I, J),
// J > I, is evaluated once and serves both (K V)_I (row sums, in registers)
// and (K V)_J (column sums); a diagonal pair (I, I) gives row sums only.
// The pairs of the upper triangle are numbered row-major (pair (I, J) is
// ffsym_start(I, nt) + J - I) and CTA b of G takes the contiguous range
// [b T / G, (b + 1) T / G); its pairs fall into segments of one row tile
// each.  Row sums go to rowpart[b][segment][c][RT rows], the column sums of
// pair p to colpart[p][c][RT columns], both as float64 (hi + lo), and
// kmvffsym_reduce_kernel adds, for every row, its segments' row sums and
// the column sums of the pairs above it, each in a fixed order.  About half
// of the entries of the plain product, each with one more float-float
// multiply-add per right-hand side and two shuffles per right-hand side per
// column step (a rotating column accumulator, below).

// Pairs before row tile I in the row-major upper triangle of nt tiles.
__host__ __device__ inline int64_t ffsym_start(int64_t I, int64_t nt) {
  return I * nt - I * (I - 1) / 2;
}
// Row tile of pair p: the largest I with ffsym_start(I) <= p.
__host__ __device__ inline int ffsym_row(int64_t p, int nt) {
  int lo = 0, hi = nt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (ffsym_start(mid, nt) <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// CTA whose pair range contains pair p.
__host__ __device__ inline int ffsym_cta_of(int64_t p, int64_t T, int G) {
  return (int)(((p + 1) * (int64_t)G + T - 1) / T) - 1;
}

template <int KERN, int DP, int M>
__global__ void __launch_bounds__(KFF_THREADS, kmvff_min_blocks(DP))
kmvffsym_kernel(const float *__restrict__ xh, const float *__restrict__ xl,
                const float *__restrict__ Vh, const float *__restrict__ Vl, int64_t N, int m,
                int nt, int64_t T, int J, ExpFFConsts ec, double *__restrict__ rowpart,
                double *__restrict__ colpart, int *__restrict__ seg0) {
  constexpr int RI = kmvff_rows_per_thread(DP);
  constexpr int RT = KFF_THREADS * RI;            // points per tile
  constexpr int NW = KFF_THREADS / 32;
  static_assert(KFF_TJ == 32, "one staged column per lane");
  // rows padded by one float: lanes read 32 different staged columns at once
  __shared__ float sxh[KFF_TJ][DP + 1], sxl[KFF_TJ][DP + 1];
  __shared__ float svh[KFF_TJ][M + 1], svl[KFF_TJ][M + 1];
  __shared__ float s_cst[4], s_tab[64];
  __shared__ FF scol[NW][KFF_TJ][M];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 4) s_cst[tid] = ec.c[tid];
  if (tid < 64) s_tab[tid] = ec.tab[tid];
  const int G = gridDim.x, b = blockIdx.x;
  const int64_t p_begin = (int64_t)b * T / G, p_end = (int64_t)(b + 1) * T / G;
  if (p_begin >= p_end) return;
  int I = ffsym_row(p_begin, nt);
  int Jt = I + (int)(p_begin - ffsym_start(I, nt));
  const int I_first = I;
  if (tid == 0) seg0[b] = I_first;

  float ih[RI][DP], il[RI][DP];
  float vih[RI][M], vil[RI][M];
  FF acc[RI][M];
  auto load_rows = [&]() {
#pragma unroll
    for (int r = 0; r < RI; ++r) {
      const int64_t i = (int64_t)I * RT + tid + (int64_t)r * KFF_THREADS;
      const bool ok = i < N;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        ih[r][k] = ok ? xh[i * DP + k] : 0.0f;
        il[r][k] = ok ? xl[i * DP + k] : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const bool okc = ok && c < m;
        vih[r][c] = okc ? Vh[(int64_t)c * N + i] : 0.0f;
        vil[r][c] = okc ? Vl[(int64_t)c * N + i] : 0.0f;
        acc[r][c] = {0.0f, 0.0f};
      }
    }
  };
  load_rows();

  for (int64_t p = p_begin; p < p_end; ++p) {
    const bool diag = (Jt == I);
    const int64_t jt0 = (int64_t)Jt * RT, jt1 = min(N, jt0 + RT);
    for (int64_t j0 = jt0; j0 < jt1; j0 += KFF_TJ) {
      __syncthreads();
      for (int idx = tid; idx < KFF_TJ * DP; idx += KFF_THREADS) {
        const int jj = idx / DP, k = idx % DP;
        const int64_t j = j0 + jj;
        const bool ok = j < jt1;
        sxh[jj][k] = ok ? xh[j * DP + k] : 0.0f;
        sxl[jj][k] = ok ? xl[j * DP + k] : 0.0f;
      }
      for (int idx = tid; idx < KFF_TJ * M; idx += KFF_THREADS) {
        const int c = idx / KFF_TJ, jj = idx % KFF_TJ;
        const int64_t j = j0 + jj;
        const bool ok = (j < jt1) && (c < m);
        svh[jj][c] = ok ? Vh[(int64_t)c * N + j] : 0.0f;
        svl[jj][c] = ok ? Vl[(int64_t)c * N + j] : 0.0f;
      }
      __syncthreads();
      const int jn = (int)min((int64_t)KFF_TJ, jt1 - j0);
      if (diag) {
#pragma unroll 1
        for (int jj = 0; jj < jn; ++jj) {
#pragma unroll
          for (int r = 0; r < RI; ++r) {
            const FF kv = ff_kernel_value<KERN, DP>(ih[r], il[r], sxh[jj], sxl[jj], s_cst, s_tab);
#pragma unroll
            for (int c = 0; c < M; ++c) ff_fma_acc(acc[r][c], kv, svh[jj][c], svl[jj][c]);
          }
        }
      } else {
        // Lane l takes the staged columns in the order (l + s) mod 32 and
        // carries the column sum of its current column; after each step it
        // passes that sum to lane l - 1, which takes the same column next.
        // After 32 steps lane l holds the warp's sum for column (l + 31) mod
        // 32.  Columns beyond the tile are zero points with zero right-hand
        // sides: their row terms vanish and their column sums are dropped.
        FF col[M];
#pragma unroll
        for (int c = 0; c < M; ++c) col[c] = {0.0f, 0.0f};
#pragma unroll 1
        for (int st = 0; st < KFF_TJ; ++st) {
          const int jj = (lane + st) & (KFF_TJ - 1);
#pragma unroll
          for (int r = 0; r < RI; ++r) {
            const FF kv = ff_kernel_value<KERN, DP>(ih[r], il[r], sxh[jj], sxl[jj], s_cst, s_tab);
#pragma unroll
            for (int c = 0; c < M; ++c) {
              ff_fma_acc(acc[r][c], kv, svh[jj][c], svl[jj][c]);
              ff_fma_acc(col[c], kv, vih[r][c], vil[r][c]);
            }
          }
          if (st + 1 < KFF_TJ)
#pragma unroll
            for (int c = 0; c < M; ++c) {
              col[c].h = __shfl_sync(0xffffffffu, col[c].h, (lane + 1) & 31);
              col[c].l = __shfl_sync(0xffffffffu, col[c].l, (lane + 1) & 31);
            }
        }
#pragma unroll
        for (int c = 0; c < M; ++c) scol[warp][(lane + KFF_TJ - 1) & (KFF_TJ - 1)][c] = col[c];
        __syncthreads();
        // the warps' shares in warp order, one (column, rhs) per thread
        for (int idx = tid; idx < KFF_TJ * M; idx += KFF_THREADS) {
          const int jj = idx / M, c = idx % M;
          if (jj < jn) {
            FF t = scol[0][jj][c];
#pragma unroll
            for (int w = 1; w < NW; ++w) t = ff_add(t, scol[w][jj][c]);
            colpart[(p * M + c) * RT + (j0 - jt0) + jj] = (double)t.h + (double)t.l;
          }
        }
      }
    }
    if (Jt + 1 == nt || p + 1 == p_end) {
      // end of this row tile's segment
      double *out = rowpart + (((int64_t)b * J + (I - I_first)) * M) * RT;
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int c = 0; c < M; ++c)
          out[c * RT + tid + r * KFF_THREADS] = (double)acc[r][c].h + (double)acc[r][c].l;
      if (p + 1 < p_end) {
        ++I;
        Jt = I;
        load_rows();
      }
    } else {
      ++Jt;
    }
  }
}

// Y[c][i] = the row sums of the segments covering row i's tile (CTA order)
// + the column sums of every pair (I, t) above it (I order) + lambda V[c][i].
__global__ void kmvffsym_reduce_kernel(const double *__restrict__ rowpart,
                                       const double *__restrict__ colpart,
                                       const int *__restrict__ seg0, int64_t N, int m, int M,
                                       int RT, int nt, int64_t T, int G, int J, double lambda,
                                       const double *__restrict__ V, int64_t ldv,
                                       double *__restrict__ Y, int64_t ldy);

}  // namespace krr
