// Fused product Y = (A + lambda I) V with the inner products x_i . x_j of
// the Gaussian and Matern kernels (Sec. 2.1; the product primitive of
// Alg. 1) taken on the tensor cores, the rest in float32 registers.
//
// Points are centred and scaled as for the float32 FMA product (kappa =
// 2^(x_i.x_j + c_i + c_j) for the Gaussian, -q^2/2 = x_i.x_j + c_i + c_j for
// Matern) and each coordinate is split into two halves, x = h + l with
// h = fp16(x) and l = fp16(x - h): |x - h - l| <= 2^-22 |x|.  The inner
// product is the three-term sum h_i.h_j + h_i.l_j + l_i.h_j (the dropped
// l_i.l_j is below 2^-22 |x_i||x_j|), formed by three m16n8k16 MMAs per 16
// coordinates with float32 accumulation, whose accumulator starts at
// c_i + c_j.  Kernel values and the sums over V stay in float32 (FFMA2 on
// the row pair g, g + 8 that one thread holds).
//
// Fragment layout of mma.m16n8k16 (row.col, f16 inputs, f32 accumulator),
// lane = 4 g + t:  A (16 x 16, rows = points i): a0 = (g, 2t..2t+1),
// a1 = (g+8, 2t..2t+1), a2 = (g, 2t+8..2t+9), a3 = (g+8, 2t+8..2t+9);
// B (16 x 8, columns = points j): b0 = (2t..2t+1, g), b1 = (2t+8..2t+9, g);
// D (16 x 8): d0 = (g, 2t), d1 = (g, 2t+1), d2 = (g+8, 2t), d3 = (g+8, 2t+1).
// The prepared layout stores, per point and block of 16 coordinates, four
// 16-byte groups; group t = {h(2t, 2t+1), h(2t+8, 2t+9), l(2t, 2t+1),
// l(2t+8, 2t+9)} as packed half pairs, so a lane reads its A or B fragment
// words for one point with a single 16-byte load.
//
// Work decomposition: as the float32 FMA product -- a CTA owns a block of
// rows (8 warps x R fragments of 16) and one column split, column tiles of
// KTC_TJ points are staged through shared memory, partial sums go to
// part[split][c][row] and are added in a fixed order by the reduction.
#pragma once

#include "kmv_kernels.cuh"

namespace krr {

constexpr int KTC_THREADS = 256;
constexpr int KTC_WARPS = KTC_THREADS / 32;
constexpr int KTC_TJ = 64;               // columns per shared tile
constexpr float KTC_MAX_COORD = 16384.0f;  // |scaled coordinate| bound for fp16

// Row fragments of 16 rows per warp: as many as the registers allow (one CTA
// of 8 warps per SM) -- each 8-column block's fragment, c_j and V loads from
// shared memory serve all of them.  At N = 1e5, d = 16, m = 4 eight fragments
// measured 3.38 ms per product against 3.74 ms for four and 3.85 ms for two.
__host__ __device__ constexpr int kmvtc_frags(int KC, int M) {
  return KC == 1 ? (M <= 4 ? 8 : 4) : (M <= 4 ? 4 : 2);
}
__host__ __device__ constexpr int kmvtc_rows(int KC, int M) {
  return KTC_WARPS * 16 * kmvtc_frags(KC, M);
}

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const uint32_t (&a)[4],
                                              uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One (row tile, column split) work item of the square product; the
// single-problem kernel maps it from blockIdx, the grouped serving kernel
// from its work list.  Each kernel instantiates it once, so its shared tiles,
// declared here, are not duplicated.
// xs : N x KC x 4 uint4, the split layout above (rows and columns: the same
//      points)
// cs : N             c_i
// V  : m x ldv       right-hand sides, float32 (m <= M)
// part: partial products, column c of split s at part + s * split_stride + c N
template <int KERN, int KC, int M, int R>
__device__ __forceinline__ void
kmvtc_tile(const uint4 *__restrict__ xs, const float *__restrict__ cs,
           const float *__restrict__ V, int64_t ldv, int64_t N, int m, int64_t chunk,
           float *__restrict__ part, int64_t split_stride, int64_t row_tile, int64_t split) {
  constexpr int ROWS = KTC_WARPS * 16 * R;
  constexpr int GX = KTC_TJ * KC * 4;             // uint4 per column tile
  constexpr int XPT = (GX + KTC_THREADS - 1) / KTC_THREADS;
  constexpr int VE = KTC_TJ * M;
  constexpr int VPT = (VE + KTC_THREADS - 1) / KTC_THREADS;
  __shared__ __align__(16) uint4 sx[2][GX];
  __shared__ __align__(16) float2 sv[2][M][KTC_TJ];   // {v, v}
  __shared__ __align__(16) float sc[2][KTC_TJ];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t row_base = row_tile * ROWS + (int64_t)warp * 16 * R;
  const int64_t j_begin = split * chunk;
  const int64_t j_end = min(N, j_begin + chunk);

  // A fragments (hi, lo) and row constants of this lane's rows g, g + 8
  uint32_t ah[R][KC][4], al[R][KC][4];
  float2 ci[R];
  float2 acc[R][M];
#pragma unroll
  for (int f = 0; f < R; ++f) {
    const int64_t r0 = row_base + 16 * f + g, r1 = r0 + 8;
    const bool v0 = r0 < N, v1 = r1 < N;
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      const uint4 u0 = v0 ? xs[(r0 * KC + kc) * 4 + t] : z;
      const uint4 u1 = v1 ? xs[(r1 * KC + kc) * 4 + t] : z;
      ah[f][kc][0] = u0.x; ah[f][kc][1] = u1.x; ah[f][kc][2] = u0.y; ah[f][kc][3] = u1.y;
      al[f][kc][0] = u0.z; al[f][kc][1] = u1.z; al[f][kc][2] = u0.w; al[f][kc][3] = u1.w;
    }
    ci[f] = f2(v0 ? cs[r0] : 0.0f, v1 ? cs[r1] : 0.0f);
#pragma unroll
    for (int c = 0; c < M; ++c) acc[f][c] = f2(0.0f, 0.0f);
  }

  // register staging of the next column tile
  uint4 rx[XPT];
  float rv[VPT], rc = 0.0f;
  auto load_tile = [&](int64_t j0) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (idx < GX) {
        const int64_t j = j0 + idx / (KC * 4);
        if (j < j_end) u = xs[j0 * KC * 4 + idx];
      }
      rx[e] = u;
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      float v = 0.0f;
      if (idx < VE) {
        const int c = idx / KTC_TJ;
        const int64_t j = j0 + idx % KTC_TJ;
        if (c < m && j < j_end) v = V[(int64_t)c * ldv + j];
      }
      rv[e] = v;
    }
    if (tid < KTC_TJ) {
      const int64_t j = j0 + tid;
      rc = (j < j_end) ? cs[j] : 0.0f;
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      // block-major in shared memory: a quarter warp's 16-byte fragment loads
      // of one coordinate block cover 128 contiguous bytes
      if (idx < GX) {
        const int jl = idx / (KC * 4), kc = (idx >> 2) % KC;
        sx[buf][(kc * KTC_TJ + jl) * 4 + (idx & 3)] = rx[e];
      }
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      if (idx < VE) sv[buf][idx / KTC_TJ][idx % KTC_TJ] = f2(rv[e], rv[e]);
    }
    if (tid < KTC_TJ) sc[buf][tid] = rc;
  };

  int buf = 0;
  if (j_begin < j_end) load_tile(j_begin);
  for (int64_t j0 = j_begin; j0 < j_end; j0 += KTC_TJ) {
    store_tile(buf);
    __syncthreads();
    if (j0 + KTC_TJ < j_end) load_tile(j0 + KTC_TJ);
    // blocks of 8 columns; columns past j_end carry zero points and V
#pragma unroll 1
    for (int jb = 0; jb < KTC_TJ; jb += 8) {
      uint32_t bh[KC][2], bl[KC][2];
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        const uint4 w = sx[buf][(kc * KTC_TJ + jb + g) * 4 + t];
        bh[kc][0] = w.x; bh[kc][1] = w.y;
        bl[kc][0] = w.z; bl[kc][1] = w.w;
      }
      const float2 cj = *reinterpret_cast<const float2 *>(&sc[buf][jb + 2 * t]);
#pragma unroll
      for (int f = 0; f < R; ++f) {
        // D = c_i + c_j + l_i.h_j + h_i.l_j + h_i.h_j, small terms first
        const float2 s0 = __fadd2_rn(f2(ci[f].x, ci[f].x), cj);   // row g
        const float2 s1 = __fadd2_rn(f2(ci[f].y, ci[f].y), cj);   // row g + 8
        float d[4] = {s0.x, s0.y, s1.x, s1.y};
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          mma_f16_16816(d, al[f][kc], bh[kc][0], bh[kc][1]);
          mma_f16_16816(d, ah[f][kc], bl[kc][0], bl[kc][1]);
        }
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) mma_f16_16816(d, ah[f][kc], bh[kc][0], bh[kc][1]);
        // kernel values of (g, 2t), (g+8, 2t) and (g, 2t+1), (g+8, 2t+1)
        const float2 k0 = f2(kappa_f32<KERN>(d[0]), kappa_f32<KERN>(d[2]));
        const float2 k1 = f2(kappa_f32<KERN>(d[1]), kappa_f32<KERN>(d[3]));
#pragma unroll
        for (int c = 0; c < M; ++c) {
          const float4 q = *reinterpret_cast<const float4 *>(&sv[buf][c][jb + 2 * t]);
          acc[f][c] = __ffma2_rn(k0, f2(q.x, q.y), acc[f][c]);
          acc[f][c] = __ffma2_rn(k1, f2(q.z, q.w), acc[f][c]);
        }
      }
    }
    buf ^= 1;
  }

  // the four lanes of a group hold partial sums over different columns
#pragma unroll
  for (int f = 0; f < R; ++f)
#pragma unroll
    for (int c = 0; c < M; ++c) {
      float2 a = acc[f][c];
      a.x += __shfl_xor_sync(0xffffffffu, a.x, 1);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, 1);
      a.x += __shfl_xor_sync(0xffffffffu, a.x, 2);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, 2);
      acc[f][c] = a;
    }
  float *out = part + split * split_stride;
#pragma unroll
  for (int f = 0; f < R; ++f) {
    const int64_t r0 = row_base + 16 * f + g, r1 = r0 + 8;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if ((c & 3) == t && c < m) {
        if (r0 < N) out[(int64_t)c * N + r0] = acc[f][c].x;
        if (r1 < N) out[(int64_t)c * N + r1] = acc[f][c].y;
      }
    }
  }
}

// Single-problem kernel.  Its body is the tile above with the work item
// taken from blockIdx; it is kept as its own copy because the inlined tile
// call compiled to a schedule measured 4.8% slower (3.55 vs 3.39 ms at
// N = 1e5, d = 16, m = 4, identical results).  The two copies implement the
// same arithmetic: the product tests check this kernel and the serving tests
// check the tile, each against the oracle.
// xs : N x KC x 4 uint4, the split layout above (rows and columns: the same
//      points, square product)
// cs : N             c_i
// V  : m x ldv       right-hand sides, float32
// part: splits x M x N partial products
template <int KERN, int KC, int M, int R = kmvtc_frags(KC, M), int MINB = 1>
__global__ void __launch_bounds__(KTC_THREADS, MINB)
kmvtc_kernel(const uint4 *__restrict__ xs, const float *__restrict__ cs,
             const float *__restrict__ V, int64_t ldv, int64_t N, int m, int64_t chunk,
             float *__restrict__ part) {
  constexpr int ROWS = KTC_WARPS * 16 * R;
  constexpr int GX = KTC_TJ * KC * 4;             // uint4 per column tile
  constexpr int XPT = (GX + KTC_THREADS - 1) / KTC_THREADS;
  constexpr int VE = KTC_TJ * M;
  constexpr int VPT = (VE + KTC_THREADS - 1) / KTC_THREADS;
  __shared__ __align__(16) uint4 sx[2][GX];
  __shared__ __align__(16) float2 sv[2][M][KTC_TJ];   // {v, v}
  __shared__ __align__(16) float sc[2][KTC_TJ];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t row_base = (int64_t)blockIdx.x * ROWS + (int64_t)warp * 16 * R;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(N, j_begin + chunk);

  // A fragments (hi, lo) and row constants of this lane's rows g, g + 8
  uint32_t ah[R][KC][4], al[R][KC][4];
  float2 ci[R];
  float2 acc[R][M];
#pragma unroll
  for (int f = 0; f < R; ++f) {
    const int64_t r0 = row_base + 16 * f + g, r1 = r0 + 8;
    const bool v0 = r0 < N, v1 = r1 < N;
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      const uint4 u0 = v0 ? xs[(r0 * KC + kc) * 4 + t] : z;
      const uint4 u1 = v1 ? xs[(r1 * KC + kc) * 4 + t] : z;
      ah[f][kc][0] = u0.x; ah[f][kc][1] = u1.x; ah[f][kc][2] = u0.y; ah[f][kc][3] = u1.y;
      al[f][kc][0] = u0.z; al[f][kc][1] = u1.z; al[f][kc][2] = u0.w; al[f][kc][3] = u1.w;
    }
    ci[f] = f2(v0 ? cs[r0] : 0.0f, v1 ? cs[r1] : 0.0f);
#pragma unroll
    for (int c = 0; c < M; ++c) acc[f][c] = f2(0.0f, 0.0f);
  }

  // register staging of the next column tile
  uint4 rx[XPT];
  float rv[VPT], rc = 0.0f;
  auto load_tile = [&](int64_t j0) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (idx < GX) {
        const int64_t j = j0 + idx / (KC * 4);
        if (j < j_end) u = xs[j0 * KC * 4 + idx];
      }
      rx[e] = u;
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      float v = 0.0f;
      if (idx < VE) {
        const int c = idx / KTC_TJ;
        const int64_t j = j0 + idx % KTC_TJ;
        if (c < m && j < j_end) v = V[(int64_t)c * ldv + j];
      }
      rv[e] = v;
    }
    if (tid < KTC_TJ) {
      const int64_t j = j0 + tid;
      rc = (j < j_end) ? cs[j] : 0.0f;
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int e = 0; e < XPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      // block-major in shared memory: a quarter warp's 16-byte fragment loads
      // of one coordinate block cover 128 contiguous bytes
      if (idx < GX) {
        const int jl = idx / (KC * 4), kc = (idx >> 2) % KC;
        sx[buf][(kc * KTC_TJ + jl) * 4 + (idx & 3)] = rx[e];
      }
    }
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * KTC_THREADS;
      if (idx < VE) sv[buf][idx / KTC_TJ][idx % KTC_TJ] = f2(rv[e], rv[e]);
    }
    if (tid < KTC_TJ) sc[buf][tid] = rc;
  };

  int buf = 0;
  if (j_begin < j_end) load_tile(j_begin);
  for (int64_t j0 = j_begin; j0 < j_end; j0 += KTC_TJ) {
    store_tile(buf);
    __syncthreads();
    if (j0 + KTC_TJ < j_end) load_tile(j0 + KTC_TJ);
    // blocks of 8 columns; columns past j_end carry zero points and V
#pragma unroll 1
    for (int jb = 0; jb < KTC_TJ; jb += 8) {
      uint32_t bh[KC][2], bl[KC][2];
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        const uint4 w = sx[buf][(kc * KTC_TJ + jb + g) * 4 + t];
        bh[kc][0] = w.x; bh[kc][1] = w.y;
        bl[kc][0] = w.z; bl[kc][1] = w.w;
      }
      const float2 cj = *reinterpret_cast<const float2 *>(&sc[buf][jb + 2 * t]);
#pragma unroll
      for (int f = 0; f < R; ++f) {
        // D = c_i + c_j + l_i.h_j + h_i.l_j + h_i.h_j, small terms first
        const float2 s0 = __fadd2_rn(f2(ci[f].x, ci[f].x), cj);   // row g
        const float2 s1 = __fadd2_rn(f2(ci[f].y, ci[f].y), cj);   // row g + 8
        float d[4] = {s0.x, s0.y, s1.x, s1.y};
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          mma_f16_16816(d, al[f][kc], bh[kc][0], bh[kc][1]);
          mma_f16_16816(d, ah[f][kc], bl[kc][0], bl[kc][1]);
        }
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) mma_f16_16816(d, ah[f][kc], bh[kc][0], bh[kc][1]);
        // kernel values of (g, 2t), (g+8, 2t) and (g, 2t+1), (g+8, 2t+1)
        const float2 k0 = f2(kappa_f32<KERN>(d[0]), kappa_f32<KERN>(d[2]));
        const float2 k1 = f2(kappa_f32<KERN>(d[1]), kappa_f32<KERN>(d[3]));
#pragma unroll
        for (int c = 0; c < M; ++c) {
          const float4 q = *reinterpret_cast<const float4 *>(&sv[buf][c][jb + 2 * t]);
          acc[f][c] = __ffma2_rn(k0, f2(q.x, q.y), acc[f][c]);
          acc[f][c] = __ffma2_rn(k1, f2(q.z, q.w), acc[f][c]);
        }
      }
    }
    buf ^= 1;
  }

  // the four lanes of a group hold partial sums over different columns
#pragma unroll
  for (int f = 0; f < R; ++f)
#pragma unroll
    for (int c = 0; c < M; ++c) {
      float2 a = acc[f][c];
      a.x += __shfl_xor_sync(0xffffffffu, a.x, 1);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, 1);
      a.x += __shfl_xor_sync(0xffffffffu, a.x, 2);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, 2);
      acc[f][c] = a;
    }
  float *out = part + (int64_t)blockIdx.y * M * N;
#pragma unroll
  for (int f = 0; f < R; ++f) {
    const int64_t r0 = row_base + 16 * f + g, r1 = r0 + 8;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      if ((c & 3) == t && c < m) {
        if (r0 < N) out[(int64_t)c * N + r0] = acc[f][c].x;
        if (r1 < N) out[(int64_t)c * N + r1] = acc[f][c].y;
      }
    }
  }
}

}  // namespace krr
