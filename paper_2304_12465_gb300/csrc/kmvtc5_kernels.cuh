// Fused product Y = K(rows, columns) V (+ lambda V for the square product)
// for the Gaussian and Matern kernels (Sec. 2.1; the "Product" primitive of
// Alg. 1), with the inner products x_i . x_j on the fifth-generation tensor
// cores (tcgen05.mma, accumulators in Tensor Memory) and the kernel values
// and sums over V in float32 registers.
//
// Arithmetic.  Points are centred and scaled as for the float32 FMA product,
// so that kappa = 2^D (Gaussian) or D = -q^2/2 (Matern) with
// D = x_i . x_j + c_i + c_j and c = -|x|^2 / 2; the Gaussian's operands carry
// c + 7 instead of c, so that its D is log2 kappa + 14 and ex2 gives the
// kernel value scaled by 2^14 (the FMA variants multiply by V scaled by
// 2^-14, exactly; the TV variants need the headroom).  Each coordinate is split
// into two halves x = h + l (h = fp16(x), l = fp16(x - h), |x - h - l| <=
// 2^-22 |x|) and c into three fp16 pieces c1 + c2 + c3.  Each point has
// 16-wide K-blocks [H_0..H_{NH-1} | L_0..L_{NH-1} | C], stored K-block-major
// (kb x N x 16 halves) so that one column tile is a single 3-D TMA box of
// contiguous 4 KB slabs:
// the row operand's c-part is (c1, c2, c3, 1, 1, 1) and the column operand's
// (1, 1, 1, c1, c2, c3), so the product of the two c-parts is c_i + c_j.  The
// c-part sits in a block of its own (CSEP = 1) or in the unused positions
// 10..15 of the last H block (CSEP = 0, when d mod 16 is 1..10).  D is then
// the float32 sum of the MMAs (L_i, H_j), (H_i, L_j), (C_i, C_j), (H_i, H_j)
// over the coordinate blocks, small terms first; the dropped l_i . l_j is
// below 2^-22 |x_i| |x_j|.
//
// Decomposition.  A row block is 256 rows (two row tiles of 128 = the TMEM
// lanes), a column tile 128 columns (the MMA's N).  The (row block, column
// tile) pairs are numbered row-block-major and CTA b of G persistent CTAs
// (one per SM) takes the contiguous range [b T / G, (b + 1) T / G), so the
// load is balanced to one tile.  Its pairs fall into segments, one per row
// block it touches; each segment's partial sums go to part[b][j] (j the
// segment's index within the CTA) and t5_reduce_kernel adds, for every row,
// the segments of the CTAs that cover its row block in CTA order (a fixed
// order: results are deterministic for a given grid).
//
// Warp roles (320 threads):
//   warp 8 (producer): one lane issues the TMA loads of the row operand (both
//     row tiles, once per segment) and of each column tile's operand into a
//     ring of t5_stages(kb, M) stages (up to 8), plus a bulk copy of the tile's right-hand sides,
//     prepared once per product as {v_c, v_c, v_c+1, v_c+1} quadruples
//     (t5_vdup_kernel), all completing on the stage's barrier.
//   warp 9 (MMA): allocates all 512 TMEM columns; one lane issues, per column
//     tile and row tile, the MMAs of D into one of two accumulator buffers
//     (2 buffers x 2 row tiles x 128 columns), and commits them to the
//     barriers that release the column stage and hand the buffer to the
//     epilogue.
//   warps 0-7 (epilogue): warp w reads TMEM lanes 32 (w % 4) .. + 31 of both
//     row tiles for columns 64 (w / 4) .. + 63 of the tile with tcgen05.ld
//     16x256b (a lane holds rows g, g + 8, g + 16, g + 24 of each row tile and
//     two columns of every 8), forms kappa with ex2 on the MUFU, and
//     accumulates V with packed FFMA2 on row pairs; each quadruple of V read
//     from shared memory serves eight rows.
//
// Every mbarrier wait is bounded (T5_WAIT_BUDGET cycles); a wait that gives
// up sets *fault, raises a CTA-wide abort flag so the other roles leave too,
// and the CTA waits (bounded) for its own TMA copies and MMAs in flight and
// frees its Tensor Memory before returning.
#pragma once

#include <cuda_fp16.h>

#include "blackwell.cuh"
#include "kmv_kernels.cuh"

namespace krr {

constexpr int T5_TM = 128;                   // rows of a row tile (TMEM lanes)
constexpr int T5_RT = 2;                     // row tiles per row block
constexpr int T5_RB = T5_TM * T5_RT;         // rows per row block
constexpr int T5_TN = 128;                   // columns per column tile (MMA N)
constexpr int T5_BLK = T5_TM * 32;           // bytes of one 16-wide K-block of 128 points
constexpr int T5_TMEM_COLS = 512;
constexpr long long T5_WAIT_BUDGET = 1LL << 32;   // about 2 s at 2 GHz
constexpr float T5_MAX_COORD = 16384.0f;     // |scaled coordinate| bound of the split
constexpr float T5_MAX_C = 32768.0f;         // |c| bound of its fp16 pieces

// K-blocks of the split layout for dimension d.
__host__ __device__ constexpr int t5_nh(int d) { return (d + 15) / 16; }
__host__ __device__ constexpr int t5_csep(int d) { return (d % 16 == 0 || d % 16 > 10) ? 1 : 0; }
__host__ __device__ constexpr int t5_kb(int nh, int csep) { return 2 * nh + csep; }

// Floats of shared memory that hold the epilogue's running totals (the second
// accumulation level) for the FMA variants whose registers would not hold
// them (16 epilogue warps, or the software-pipelined variant, at M = 4): 8
// per right-hand side per thread (2 row tiles x 2 row halves x a row pair).
// 0 (totals in registers) otherwise.  At M = 8 with 8 warps the registers
// spill about 270 bytes, which measured faster (4.49 ms against 4.64 ms at
// N = 1e5) than the totals in shared memory and the two stages they cost.
__host__ __device__ constexpr int t5_tot_floats(int EW, int M, int LAG, int TV) {
  return (!TV && M == 4 && (EW == 16 || LAG)) ? EW * 32 * 8 * M : 0;
}

// Column-tile pipeline stages: as many as fit (at most 8) in about 200 KB of
// shared memory beside the row operand and the totals, so that TMA latency is
// hidden.
__host__ __device__ constexpr int t5_stages(int kb, int M, int tot_floats = 0) {
  return ((204800 - 1024 - T5_RT * kb * T5_BLK - 4 * tot_floats) /
          (kb * T5_BLK + (M / 2) * T5_TN * 16)) > 8
             ? 8
             : ((204800 - 1024 - T5_RT * kb * T5_BLK - 4 * tot_floats) /
                (kb * T5_BLK + (M / 2) * T5_TN * 16));
}

// Barrier indices in shared memory for ST stages.
__host__ __device__ constexpr int t5_bar_a_full() { return 0; }
__host__ __device__ constexpr int t5_bar_a_empty() { return 1; }
__host__ __device__ constexpr int t5_bar_b_full(int) { return 2; }
__host__ __device__ constexpr int t5_bar_b_empty(int st) { return 2 + st; }
__host__ __device__ constexpr int t5_bar_v_empty(int st) { return 2 + 2 * st; }
__host__ __device__ constexpr int t5_bar_d_full(int st) { return 2 + 3 * st; }
__host__ __device__ constexpr int t5_bar_d_empty(int st) { return 4 + 3 * st; }
__host__ __device__ constexpr int t5_bar_fin(int st) { return 6 + 3 * st; }
__host__ __device__ constexpr int t5_nbar(int st) { return 7 + 3 * st; }

// Shared memory of one CTA (bytes, including 1024 bytes of alignment slack).
__host__ __device__ constexpr int t5_smem_bytes(int kb, int M, int tot_floats = 0) {
  return 1024 + T5_RT * kb * T5_BLK +
         t5_stages(kb, M, tot_floats) * (kb * T5_BLK + (M / 2) * T5_TN * 16) + 4 * tot_floats +
         8 * t5_nbar(t5_stages(kb, M, tot_floats)) + 16;
}

struct T5Args {
  const float4 *vdup;   // C x (M/2) x TN right-hand-side quadruples (t5_vdup_kernel)
  int64_t Nc;           // column points
  float *part;          // G x J x (EW / 4) x M x T5_RB partial sums
  int C;            // column tiles
  int64_t T;        // row blocks x column tiles
  int J;            // segments per CTA (maximum)
  int *fault;       // set to 1 when a bounded wait gives up
};

// Kernel values of the MMA accumulator D.
template <int KERN>
__device__ __forceinline__ float t5_kappa(uint32_t d) {
  return kappa_f32<KERN>(__uint_as_float(d));
}

// 2^14 kappa for the tensor-core sums (TV variants): the Gaussian's operands
// carry the factor in their c-parts (D = log2 kappa + 14), the Matern
// polynomial is scaled instead.
template <int KERN>
__device__ __forceinline__ float t5_kappa_scaled(uint32_t d) {
  if constexpr (KERN == KMATERN) {
    const float q = sqrt_approx(fmaxf(-2.0f * __uint_as_float(d), 0.0f));
    const float e = ex2_approx(-1.4426950408889634f * q);
    return fmaf(q, fmaf(q, 5461.3335f, 16384.0f), 16384.0f) * e;
  } else {
    return ex2_approx(__uint_as_float(d));
  }
}

// Splits two non-negative values k0, k1 into fp16 halves k = hi + lo: hi keeps
// the leading 11 significant bits (exact in fp16 for k >= 2^-14), lo = k - hi
// (exact in float32) rounded to fp16; packed with k0 in the low half.
__device__ __forceinline__ void t5_split_pair(float k0, float k1, uint32_t &hi, uint32_t &lo) {
  const float h0 = __uint_as_float(__float_as_uint(k0) & 0xFFFFE000u);
  const float h1 = __uint_as_float(__float_as_uint(k1) & 0xFFFFE000u);
  const float2 l = __ffma2_rn(f2(h0, h1), f2(-1.0f, -1.0f), f2(k0, k1));
  const __half2 hh = __floats2half2_rn(h0, h1), ll = __floats2half2_rn(l.x, l.y);
  hi = *reinterpret_cast<const uint32_t *>(&hh);
  lo = *reinterpret_cast<const uint32_t *>(&ll);
}

__device__ __forceinline__ void t5_mma_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Epilogue variants: EW epilogue warps (8, 12 or 16; EW / 4 column groups of
// TN / (EW / 4) columns per tile, TN the column tile: 128, or 96 for 12
// warps), PIPE = 1 keeps the TMEM loads of the
// next 16 columns in flight while the current ones are computed, LAG = 1
// (with PIPE) software-pipelines the epilogue by one batch of 16 columns:
// the kernel values (ex2 on the MUFU) of batch b are formed while the FFMA2
// accumulation of batch b - 1 runs on the FMA pipe, across tile boundaries,
// so that the two pipes work at the same time instead of in turn.  TV = 1
// takes the sums over the right-hand sides on the tensor cores instead of the
// FMA pipe: the 16x256b TMEM layout of a batch of 16 columns is the A-operand
// fragment layout of mma.sync m16n8k16, so each kernel value, scaled by 2^14
// and split into fp16 halves hi + lo, enters two MMAs (A = hi, A = lo) whose
// B operand holds the right-hand sides split likewise, v s_c = v_hi + v_lo
// with a power-of-two scale s_c per right-hand side (t5_vfrag_kernel): B
// slots 0..M-1 the v_hi, M..2M-1 the v_lo (M <= 4), or one fragment of each
// (M = 8).  Products of fp16 halves are exact in float32, so the result is
// (hi + lo)(v_hi + v_lo) summed in float32 per tile, then added to the
// segment total (two levels, as the FMA variants).
template <int KERN, int NH, int CSEP, int M, int EW, int PIPE, int LAG, int TN, int TV = 0>
__global__ void __launch_bounds__((EW + 2) * 32, 1)
kmvtc5_kernel(const __grid_constant__ CUtensorMap rowmap,
              const __grid_constant__ CUtensorMap colmap, const T5Args a) {
  // column tile of this variant (the MMA's N; the TMA box stays 128 points,
  // of which the first TN are used)
  constexpr int T5_TN = TN;
  constexpr int KB = 2 * NH + CSEP;
  constexpr int MP = M / 2;   // right-hand-side pairs
  constexpr int NB = (M == 8) ? 2 : 1;   // B fragments per batch (TV)
  constexpr int VQ = TV ? NB : MP;       // 16-byte right-hand-side words per column
  constexpr int TOTF = t5_tot_floats(EW, M, LAG, TV);   // running totals in shared memory
  constexpr int T5_ST = t5_stages(KB, M, TOTF);
  constexpr int T5_BAR_A_FULL = t5_bar_a_full();
  constexpr int T5_BAR_A_EMPTY = t5_bar_a_empty();
  constexpr int T5_BAR_B_FULL = t5_bar_b_full(T5_ST);
  constexpr int T5_BAR_B_EMPTY = t5_bar_b_empty(T5_ST);
  constexpr int T5_BAR_V_EMPTY = t5_bar_v_empty(T5_ST);
  constexpr int T5_BAR_D_FULL = t5_bar_d_full(T5_ST);
  constexpr int T5_BAR_D_EMPTY = t5_bar_d_empty(T5_ST);
  constexpr int T5_BAR_FIN = t5_bar_fin(T5_ST);
  constexpr int T5_NBAR = t5_nbar(T5_ST);
  constexpr int T5_EPI_WARPS = EW;
  constexpr int T5_CG = EW / 4;                 // column groups of the epilogue
  constexpr int T5_WCOLS = T5_TN / T5_CG;       // columns per epilogue warp per tile
  constexpr int T5_PRODUCER_WARP = EW;
  constexpr int T5_MMA_WARP = EW + 1;
  extern __shared__ uint8_t t5_smem[];
  const uint32_t raw = bw::smem_u32(t5_smem);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t *gbase = t5_smem + (base - raw);
  const uint32_t sA = base;                                   // [rt][kb][128 x 32 B]
  const uint32_t sB = sA + T5_RT * KB * T5_BLK;               // [stage][kb][128 x 32 B]
  const uint32_t vOff = sB + T5_ST * KB * T5_BLK - base;
  float4 *sV = reinterpret_cast<float4 *>(gbase + vOff);       // [stage][MP][128]
  const uint32_t totOff = vOff + T5_ST * MP * 128 * 16;
  float4 *sTot = reinterpret_cast<float4 *>(gbase + totOff);   // [warp][2M][32 lanes]
  const uint32_t sBar = base + totOff + 4 * TOTF;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(gbase + (sBar - base) + 8 * T5_NBAR);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
  auto bar = [&](int i) -> uint32_t { return sBar + 8u * (uint32_t)i; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int64_t p_begin = (int64_t)b * a.T / G, p_end = (int64_t)(b + 1) * a.T / G;
  const int64_t rb_first = p_begin / a.C;
  const int ct_first = (int)(p_begin - rb_first * a.C);
  // (row block, column tile) of pair p are kept incrementally along the range
  // (no per-tile 64-bit division)

  if (threadIdx.x == 0) {
    bw::mbar_init(bar(T5_BAR_A_FULL), 1);
    bw::mbar_init(bar(T5_BAR_A_EMPTY), 1);
    for (int s = 0; s < T5_ST; ++s) {
      bw::mbar_init(bar(T5_BAR_B_FULL + s), 1);
      bw::mbar_init(bar(T5_BAR_B_EMPTY + s), 1);
      bw::mbar_init(bar(T5_BAR_V_EMPTY + s), T5_EPI_WARPS);   // one arrival per warp
    }
    for (int i = 0; i < 2; ++i) {
      bw::mbar_init(bar(T5_BAR_D_FULL + i), 1);
      bw::mbar_init(bar(T5_BAR_D_EMPTY + i), T5_EPI_WARPS);
    }
    bw::mbar_init(bar(T5_BAR_FIN), 1);
    *abort_flag = 0;
    bw::fence_mbar_init();
  }
  if (warp == T5_MMA_WARP) {
    bw::tmem_alloc(bw::smem_u32(tslot), T5_TMEM_COLS);
    bw::tmem_relinquish();
  }
  if (warp == T5_PRODUCER_WARP && lane == 0) {
    bw::prefetch_tensormap(&rowmap);
    bw::prefetch_tensormap(&colmap);
  }
  bw::tc_fence_before();
  __syncthreads();
  bw::tc_fence_after();
  const uint32_t tmem = *tslot;

  // bounded wait; on timeout records the fault and aborts the CTA
  auto wait = [&](int i, uint32_t parity) -> bool {
    if (bw::mbar_wait_abortable(bar(i), parity, T5_WAIT_BUDGET, abort_flag)) return true;
    *abort_flag = 1;
    atomicOr(a.fault, 1);
    return false;
  };

  if (warp == T5_PRODUCER_WARP) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      constexpr uint32_t VBYTES = VQ * T5_TN * 16;
      int64_t kt = 0, issued_b = 0;
      int issued_a = 0;
      int64_t rb = rb_first;
      int ct = ct_first;
      for (int64_t p = p_begin; p < p_end; ++p, ++kt, (++ct == a.C ? (ct = 0, ++rb) : 0)) {
        if (p == p_begin || ct == 0) {
          if (!wait(T5_BAR_A_EMPTY, (uint32_t)(issued_a & 1) ^ 1u)) break;
          bw::mbar_arrive_expect_tx(bar(T5_BAR_A_FULL), T5_RT * KB * T5_BLK);
#pragma unroll
          for (int rt = 0; rt < T5_RT; ++rt)
            bw::tma_load_3d(sA + rt * KB * T5_BLK, &rowmap, bar(T5_BAR_A_FULL), 0,
                            (int)(rb * T5_RB + rt * T5_TM), 0);
          ++issued_a;
        }
        const int s = (int)(kt % T5_ST);
        const uint32_t ph = (uint32_t)((kt / T5_ST) & 1);
        if (!wait(T5_BAR_B_EMPTY + s, ph ^ 1u) || !wait(T5_BAR_V_EMPTY + s, ph ^ 1u)) break;
        bw::mbar_arrive_expect_tx(bar(T5_BAR_B_FULL + s), KB * T5_BLK + VBYTES);
        bw::tma_load_3d(sB + s * KB * T5_BLK, &colmap, bar(T5_BAR_B_FULL + s), 0, ct * T5_TN, 0);
        bw::bulk_load(base + vOff + (uint32_t)s * VBYTES, a.vdup + (size_t)ct * VQ * T5_TN,
                      VBYTES, bar(T5_BAR_B_FULL + s));
        ++issued_b;
      }
      // wait (bounded, quietly) for this lane's own copies: the last one of
      // each stage and of the row operand.  After a normal run all have been
      // consumed and every wait returns at once.
      for (int64_t q = (issued_b > T5_ST ? issued_b - T5_ST : 0); q < issued_b; ++q)
        bw::mbar_wait(bar(T5_BAR_B_FULL + (int)(q % T5_ST)), (uint32_t)((q / T5_ST) & 1),
                      T5_WAIT_BUDGET >> 4);
      if (issued_a > 0)
        bw::mbar_wait(bar(T5_BAR_A_FULL), (uint32_t)((issued_a - 1) & 1), T5_WAIT_BUDGET >> 4);
    }
    __syncwarp();
  } else if (warp == T5_MMA_WARP) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t IDESC = bw::idesc_f16_f32(T5_TM, T5_TN);
      int64_t kt = 0;
      int seg = 0;
      int ct = ct_first;
      for (int64_t p = p_begin; p < p_end; ++p, ++kt, (++ct == a.C ? ct = 0 : 0)) {
        if (p == p_begin || ct == 0) {
          if (!wait(T5_BAR_A_FULL, (uint32_t)(seg & 1))) break;
          ++seg;
        }
        const int s = (int)(kt % T5_ST);
        const int buf = (int)(kt & 1);
        if (!wait(T5_BAR_B_FULL + s, (uint32_t)((kt / T5_ST) & 1))) break;
        if (!wait(T5_BAR_D_EMPTY + buf, (uint32_t)((kt >> 1) & 1) ^ 1u)) break;
        bw::tc_fence_after();
#pragma unroll
        for (int rt = 0; rt < T5_RT; ++rt) {
          const uint32_t d = tmem + (uint32_t)((buf * T5_RT + rt) * T5_TN);
          const uint32_t aBase = sA + rt * KB * T5_BLK, bBase = sB + s * KB * T5_BLK;
          uint32_t acc = 0;
#pragma unroll
          for (int kc = 0; kc < NH; ++kc) {
            bw::mma_f16(d, bw::sdesc_kmajor_sw32(aBase + (NH + kc) * T5_BLK),
                        bw::sdesc_kmajor_sw32(bBase + kc * T5_BLK), IDESC, acc);
            acc = 1;
            bw::mma_f16(d, bw::sdesc_kmajor_sw32(aBase + kc * T5_BLK),
                        bw::sdesc_kmajor_sw32(bBase + (NH + kc) * T5_BLK), IDESC, 1);
          }
          if (CSEP)
            bw::mma_f16(d, bw::sdesc_kmajor_sw32(aBase + 2 * NH * T5_BLK),
                        bw::sdesc_kmajor_sw32(bBase + 2 * NH * T5_BLK), IDESC, 1);
#pragma unroll
          for (int kc = 0; kc < NH; ++kc)
            bw::mma_f16(d, bw::sdesc_kmajor_sw32(aBase + kc * T5_BLK),
                        bw::sdesc_kmajor_sw32(bBase + kc * T5_BLK), IDESC, 1);
        }
        bw::mma_commit(bar(T5_BAR_D_FULL + buf));
        bw::mma_commit(bar(T5_BAR_B_EMPTY + s));
        if (p + 1 == p_end || ct + 1 == a.C) bw::mma_commit(bar(T5_BAR_A_EMPTY));
      }
      // every MMA issued so far has completed once FIN flips
      bw::mma_commit(bar(T5_BAR_FIN));
      bw::mbar_wait(bar(T5_BAR_FIN), 0, T5_WAIT_BUDGET >> 4);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int qd = warp & 3;        // TMEM lane quarter
    const int cg = warp >> 2;       // column group
    const int g = lane >> 2, tq = lane & 3;
    // sums over the current tile's columns (acc) and over the segment's
    // finished tiles (tot): two-level float32 accumulation, so a long segment
    // (up to about 1e5 columns per row) adds one tile sum at a time to its
    // running total instead of one entry at a time
    float2 acc[T5_RT][2][M];        // [row tile][rows g,g+8 | g+16,g+24][rhs]
    // running totals: registers, or (TOTF > 0) this thread's 2M float4 in
    // shared memory, float4 q holding acc entries 2q and 2q + 1 (flattened)
    float2 tot[TOTF ? 1 : T5_RT][2][M];
    float4 *mytot = sTot + warp * (2 * M) * 32 + lane;
#pragma unroll
    for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf)
#pragma unroll
        for (int c = 0; c < M; ++c) acc[rt][hf][c] = f2(0.0f, 0.0f);
    if constexpr (TOTF > 0) {
#pragma unroll
      for (int q = 0; q < 2 * M; ++q) mytot[q * 32] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
#pragma unroll
      for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf)
#pragma unroll
          for (int c = 0; c < M; ++c) tot[rt][hf][c] = f2(0.0f, 0.0f);
    }
    auto fold_tile = [&]() {
      if constexpr (TOTF > 0) {
        float2 *af = &acc[0][0][0];
#pragma unroll
        for (int q = 0; q < 2 * M; ++q) {
          const float4 t = mytot[q * 32];
          const float2 lo = __fadd2_rn(f2(t.x, t.y), af[2 * q]);
          const float2 hi = __fadd2_rn(f2(t.z, t.w), af[2 * q + 1]);
          mytot[q * 32] = make_float4(lo.x, lo.y, hi.x, hi.y);
          af[2 * q] = af[2 * q + 1] = f2(0.0f, 0.0f);
        }
      } else {
#pragma unroll
        for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf)
#pragma unroll
            for (int c = 0; c < M; ++c) {
              tot[rt][hf][c] = __fadd2_rn(tot[rt][hf][c], acc[rt][hf][c]);
              acc[rt][hf][c] = f2(0.0f, 0.0f);
            }
      }
    };
    // running total of (rt, hf, c), cleared as it is read (segment end)
    auto take_tot = [&](int rt, int hf, int c) -> float2 {
      if constexpr (TOTF > 0) {
        const int i = (rt * 2 + hf) * M + c;
        float4 *t = mytot + (i >> 1) * 32;
        const float4 v = *t;
        if (i & 1) {
          t->z = 0.0f;
          t->w = 0.0f;
          return f2(v.z, v.w);
        }
        t->x = 0.0f;
        t->y = 0.0f;
        return f2(v.x, v.y);
      } else {
        const float2 v = tot[rt][hf][c];
        tot[rt][hf][c] = f2(0.0f, 0.0f);
        return v;
      }
    };
    constexpr int NBT = T5_WCOLS / 16;   // batches of 16 columns per tile
    if constexpr (TV) {
      constexpr int NG = T5_RT * 2;      // m16 row groups of a warp: (row tile, half)
      float yacc[NG][NB][4], ytot[NG][NB][4];
#pragma unroll
      for (int gr = 0; gr < NG; ++gr)
#pragma unroll
        for (int f = 0; f < NB; ++f)
#pragma unroll
          for (int i = 0; i < 4; ++i) yacc[gr][f][i] = ytot[gr][f][i] = 0.0f;
      int64_t kt = 0, rb = rb_first;
      int ct = ct_first;
      for (int64_t p = p_begin; p < p_end; ++p, ++kt, (++ct == a.C ? (ct = 0, ++rb) : 0)) {
        const int s = (int)(kt % T5_ST);
        const int buf = (int)(kt & 1);
        const bool ok = __all_sync(0xffffffffu, wait(T5_BAR_D_FULL + buf, (uint32_t)((kt >> 1) & 1)) &&
                                                    wait(T5_BAR_B_FULL + s, (uint32_t)((kt / T5_ST) & 1)));
        if (!ok) break;
        bw::tc_fence_after();
        const uint2 *vf = reinterpret_cast<const uint2 *>(sV + (size_t)s * VQ * T5_TN);
        const uint32_t tcol = tmem + (uint32_t)(buf * T5_RT * T5_TN + cg * T5_WCOLS);
        uint32_t r[PIPE ? 2 : 1][32];   // [batch parity][row group][8]
        auto load_batch = [&](int bt, uint32_t *rr) {
#pragma unroll
          for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
              bw::tmem_ld_16x256b_x2(tcol + ((uint32_t)(32 * qd + 16 * hf) << 16) +
                                         (uint32_t)(rt * T5_TN + bt * 16),
                                     &rr[(rt * 2 + hf) * 8]);
        };
        auto release_buffer = [&]() {
          bw::tc_fence_before();
          __syncwarp();
          if (lane == 0) bw::mbar_arrive(bar(T5_BAR_D_EMPTY + buf));
        };
        if (PIPE) {
          load_batch(0, r[0]);
          bw::tmem_wait_ld32(r[0]);
          if (NBT == 1) release_buffer();
        }
#pragma unroll
        for (int bt = 0; bt < NBT; ++bt) {
          uint32_t *cur = r[PIPE ? (bt & 1) : 0];
          if (PIPE) {
            if (bt + 1 < NBT) load_batch(bt + 1, r[(bt + 1) & 1]);
          } else {
            load_batch(bt, cur);
            bw::tmem_wait_ld32(cur);
            if (bt + 1 == NBT) release_buffer();
          }
          uint2 bf[NB];
#pragma unroll
          for (int f = 0; f < NB; ++f) bf[f] = vf[((cg * NBT + bt) * NB + f) * 32 + lane];
#pragma unroll
          for (int gr = 0; gr < NG; ++gr) {
            // registers (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), then the
            // same for columns 8..15: fragments a0..a3 in order
            const uint32_t *q = &cur[gr * 8];
            uint32_t ah[4], al[4];
#pragma unroll
            for (int pr = 0; pr < 4; ++pr)
              t5_split_pair(t5_kappa_scaled<KERN>(q[2 * pr]), t5_kappa_scaled<KERN>(q[2 * pr + 1]),
                            ah[pr], al[pr]);
#pragma unroll
            for (int f = 0; f < NB; ++f) {
              t5_mma_16816(yacc[gr][f], al, bf[f]);
              t5_mma_16816(yacc[gr][f], ah, bf[f]);
            }
          }
          if (PIPE && bt + 1 < NBT) {
            bw::tmem_wait_ld32(r[(bt + 1) & 1]);
            if (bt + 2 == NBT) release_buffer();
          }
        }
#pragma unroll
        for (int gr = 0; gr < NG; ++gr)
#pragma unroll
          for (int f = 0; f < NB; ++f)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              ytot[gr][f][i] += yacc[gr][f][i];
              yacc[gr][f][i] = 0.0f;
            }
        __syncwarp();
        if (lane == 0) bw::mbar_arrive(bar(T5_BAR_V_EMPTY + s));
        if (p + 1 == p_end || ct + 1 == a.C) {
          // end of a segment: accumulator (g, 2t + e) / (g + 8, 2t + e) holds
          // B slot 2t + e; add each v_hi slot's v_lo partner and write this
          // warp's partial sums (scaled by 2^14 s_c; t5_reduce_kernel undoes it)
          const int j = (int)(rb - rb_first);
          float *out = a.part + (((int64_t)b * a.J + j) * T5_CG + cg) * (int64_t)M * T5_RB;
#pragma unroll
          for (int gr = 0; gr < NG; ++gr) {
            float y[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              if constexpr (NB == 2)
                y[i] = ytot[gr][0][i] + ytot[gr][1][i];
              else
                y[i] = ytot[gr][0][i] + __shfl_xor_sync(0xffffffffu, ytot[gr][0][i], M / 2);
#pragma unroll
              for (int f = 0; f < NB; ++f) ytot[gr][f][i] = 0.0f;
            }
            const int c0 = 2 * tq;
            if (c0 < M) {
              const int row = (gr >> 1) * T5_TM + 32 * qd + 16 * (gr & 1) + g;
              out[c0 * T5_RB + row] = y[0];
              out[(c0 + 1) * T5_RB + row] = y[1];
              out[c0 * T5_RB + row + 8] = y[2];
              out[(c0 + 1) * T5_RB + row + 8] = y[3];
            }
          }
        }
      }
    } else if constexpr (LAG) {
      // segment end: the four lanes of a row group hold sums over different
      // columns; add them and write this warp's partial sums
      auto flush = [&](int64_t rbq) {
        const int j = (int)(rbq - rb_first);
        float *out = a.part + (((int64_t)b * a.J + j) * T5_CG + cg) * (int64_t)M * T5_RB;
#pragma unroll
        for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf)
#pragma unroll
            for (int c = 0; c < M; ++c) {
              float2 v = take_tot(rt, hf, c);
              v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
              v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
              v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
              v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
              if ((c & 3) == tq) {
                const int row = rt * T5_TM + 32 * qd + 16 * hf + g;
                out[c * T5_RB + row] = v.x;
                out[c * T5_RB + row + 8] = v.y;
              }
            }
      };
      // kernel values of one batch: [ch][e][rt][hf] -> rows (g, g + 8) pair
      auto kappa_batch = [&](const uint32_t *cur, float2 *kq) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
          for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
              for (int hf = 0; hf < 2; ++hf) {
                const uint32_t *q = &cur[(rt * 2 + hf) * 8 + ch * 4];
                kq[((ch * 2 + e) * 2 + rt) * 2 + hf] =
                    f2(t5_kappa<KERN>(q[e]), t5_kappa<KERN>(q[2 + e]));
              }
      };
      auto ffma_batch = [&](const float2 *kq, const float4 *vq, int col0) {
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int jl = col0 + ch * 8 + 2 * tq + e;
#pragma unroll
            for (int cp = 0; cp < MP; ++cp) {
              const float4 v = vq[cp * T5_TN + jl];
#pragma unroll
              for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                  const float2 k2 = kq[((ch * 2 + e) * 2 + rt) * 2 + hf];
                  acc[rt][hf][2 * cp] = __ffma2_rn(k2, f2(v.x, v.y), acc[rt][hf][2 * cp]);
                  acc[rt][hf][2 * cp + 1] = __ffma2_rn(k2, f2(v.z, v.w), acc[rt][hf][2 * cp + 1]);
                }
            }
          }
      };
      // the batch whose accumulation is pending
      float2 kp[16];
      const float4 *vp = sV;
      int colp = 0, sp = 0;
      bool havep = false, p_last = false, p_segend = false;
      int64_t p_rb = 0;
      auto retire_pending = [&]() {
        ffma_batch(kp, vp, colp);
        if (p_last) {
          fold_tile();
          __syncwarp();
          if (lane == 0) bw::mbar_arrive(bar(T5_BAR_V_EMPTY + sp));
          if (p_segend) flush(p_rb);
        }
      };
      int64_t kt = 0, rb = rb_first;
      int ct = ct_first;
      for (int64_t p = p_begin; p < p_end; ++p, ++kt, (++ct == a.C ? (ct = 0, ++rb) : 0)) {
        const int s = (int)(kt % T5_ST);
        const int buf = (int)(kt & 1);
        const bool ok =
            __all_sync(0xffffffffu, wait(T5_BAR_D_FULL + buf, (uint32_t)((kt >> 1) & 1)) &&
                                        wait(T5_BAR_B_FULL + s, (uint32_t)((kt / T5_ST) & 1)));
        if (!ok) break;
        bw::tc_fence_after();
        const float4 *vt = sV + (size_t)s * MP * T5_TN;
        const uint32_t tcol = tmem + (uint32_t)(buf * T5_RT * T5_TN + cg * T5_WCOLS);
        const bool segend = (p + 1 == p_end) || (ct + 1 == a.C);
        uint32_t r[2][32];
        auto load_batch = [&](int bt, uint32_t *rr) {
#pragma unroll
          for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
              bw::tmem_ld_16x256b_x2(tcol + ((uint32_t)(32 * qd + 16 * hf) << 16) +
                                         (uint32_t)(rt * T5_TN + bt * 16),
                                     &rr[(rt * 2 + hf) * 8]);
        };
        auto release_buffer = [&]() {
          bw::tc_fence_before();
          __syncwarp();
          if (lane == 0) bw::mbar_arrive(bar(T5_BAR_D_EMPTY + buf));
        };
        load_batch(0, r[0]);
        bw::tmem_wait_ld32(r[0]);
        if (NBT == 1) release_buffer();
#pragma unroll
        for (int bt = 0; bt < NBT; ++bt) {
          if (bt + 1 < NBT) load_batch(bt + 1, r[(bt + 1) & 1]);
          float2 kc[16];
          kappa_batch(r[bt & 1], kc);
          if (havep) retire_pending();
          if (bt + 1 < NBT) {
            bw::tmem_wait_ld32(r[(bt + 1) & 1]);
            if (bt + 2 == NBT) release_buffer();
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) kp[i] = kc[i];
          vp = vt;
          colp = cg * T5_WCOLS + bt * 16;
          sp = s;
          havep = true;
          p_last = (bt + 1 == NBT);
          p_segend = p_last && segend;
          p_rb = rb;
        }
      }
      if (havep) retire_pending();
    } else {
    int64_t kt = 0, rb = rb_first;
    int ct = ct_first;
    for (int64_t p = p_begin; p < p_end; ++p, ++kt, (++ct == a.C ? (ct = 0, ++rb) : 0)) {
      const int s = (int)(kt % T5_ST);
      const int buf = (int)(kt & 1);
      // D of this tile, and (for the visibility of the bulk-copied V) the
      // stage's arrival
      const bool ok = __all_sync(0xffffffffu, wait(T5_BAR_D_FULL + buf, (uint32_t)((kt >> 1) & 1)) &&
                                                  wait(T5_BAR_B_FULL + s, (uint32_t)((kt / T5_ST) & 1)));
      if (!ok) break;
      bw::tc_fence_after();
      const float4 *vt = sV + (size_t)s * MP * T5_TN;
      const uint32_t tcol = tmem + (uint32_t)(buf * T5_RT * T5_TN + cg * T5_WCOLS);
      // with PIPE, the TMEM loads of batch bt + 1 are in flight while batch bt
      // is computed
      uint32_t r[PIPE ? 2 : 1][32];   // [batch parity][rt][hf][8]
      auto load_batch = [&](int bt, uint32_t *rr) {
#pragma unroll
        for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf)
            bw::tmem_ld_16x256b_x2(tcol + ((uint32_t)(32 * qd + 16 * hf) << 16) +
                                       (uint32_t)(rt * T5_TN + bt * 16),
                                   &rr[(rt * 2 + hf) * 8]);
      };
      auto release_buffer = [&]() {
        // every TMEM load of this buffer has landed: hand it back
        bw::tc_fence_before();
        __syncwarp();
        if (lane == 0) bw::mbar_arrive(bar(T5_BAR_D_EMPTY + buf));
      };
      if (PIPE) {
        load_batch(0, r[0]);
        bw::tmem_wait_ld32(r[0]);
        if (NBT == 1) release_buffer();
      }
#pragma unroll
      for (int bt = 0; bt < NBT; ++bt) {
        uint32_t *cur = r[PIPE ? (bt & 1) : 0];
        if (PIPE) {
          if (bt + 1 < NBT) load_batch(bt + 1, r[(bt + 1) & 1]);
        } else {
          load_batch(bt, cur);
          bw::tmem_wait_ld32(cur);
          if (bt + 1 == NBT) release_buffer();
        }
        const int col0 = cg * T5_WCOLS + bt * 16;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int jl = col0 + ch * 8 + 2 * tq + e;
            float2 kk[T5_RT][2];
#pragma unroll
            for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
              for (int hf = 0; hf < 2; ++hf) {
                const uint32_t *q = &cur[(rt * 2 + hf) * 8 + ch * 4];
                kk[rt][hf] = f2(t5_kappa<KERN>(q[e]), t5_kappa<KERN>(q[2 + e]));
              }
#pragma unroll
            for (int cp = 0; cp < MP; ++cp) {
              const float4 v = vt[cp * T5_TN + jl];
#pragma unroll
              for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                  acc[rt][hf][2 * cp] = __ffma2_rn(kk[rt][hf], f2(v.x, v.y), acc[rt][hf][2 * cp]);
                  acc[rt][hf][2 * cp + 1] =
                      __ffma2_rn(kk[rt][hf], f2(v.z, v.w), acc[rt][hf][2 * cp + 1]);
                }
            }
          }
        }
        if (PIPE && bt + 1 < NBT) {
          bw::tmem_wait_ld32(r[(bt + 1) & 1]);
          if (bt + 2 == NBT) release_buffer();
        }
      }
      fold_tile();
      __syncwarp();
      if (lane == 0) bw::mbar_arrive(bar(T5_BAR_V_EMPTY + s));
      if (p + 1 == p_end || ct + 1 == a.C) {
        // end of a segment: the four lanes of a row group hold sums over
        // different columns; add them and write this warp's partial sums
        const int j = (int)(rb - rb_first);
        float *out = a.part + (((int64_t)b * a.J + j) * T5_CG + cg) * (int64_t)M * T5_RB;
#pragma unroll
        for (int rt = 0; rt < T5_RT; ++rt)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf)
#pragma unroll
            for (int c = 0; c < M; ++c) {
              float2 v = take_tot(rt, hf, c);
              v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
              v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
              v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
              v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
              if ((c & 3) == tq) {
                const int row = rt * T5_TM + 32 * qd + 16 * hf + g;
                out[c * T5_RB + row] = v.x;
                out[c * T5_RB + row + 8] = v.y;
              }
            }
      }
    }
    }
}

  bw::tc_fence_before();
  __syncthreads();
  if (warp == T5_MMA_WARP) {
    bw::tc_fence_after();
    bw::tmem_dealloc(tmem, T5_TMEM_COLS);
  }
}

// CTA whose pair range contains pair p: the largest b with floor(b T / G) <= p.
__host__ __device__ inline int t5_cta_of(int64_t p, int64_t T, int G) {
  return (int)(((p + 1) * (int64_t)G + T - 1) / T) - 1;
}

// Y[c][i] = sum of the partial sums of row i over the CTAs covering its row
// block (CTA order) and column groups, + lambda V[c][i] when V is given.
// With vexp (TV variants) the partial sums of right-hand side c carry the
// factor 2^(14 + vexp[c]), which is divided out in float64.
__global__ void t5_reduce_kernel(const float *__restrict__ part, int64_t Nr, int m, int M, int C,
                                 int64_t T, int G, int J, int CG, const int *__restrict__ vexp,
                                 float lambda, const float *__restrict__ V, int64_t ldv,
                                 float *__restrict__ Y, int64_t ldy);

}  // namespace krr

namespace krr {

// Epilogue variants of the tcgen05 product: 1 = 8 warps with pipelined TMEM
// loads, 2 = 16 warps, 3 = 8 warps without the pipelining, 4 = 16 warps with
// it, 5 = 8 warps, pipelined and software-pipelined by one batch, 6 = 12 warps
// on 96-column tiles with pipelined loads, 7 = the same without; 8..11 take
// the sums over V on the tensor cores (TV): 8 = 8 warps with pipelined loads,
// 9 = 8 warps without, 10 = 16 warps without, 11 = 16 warps with.  The 12-
// and 16-warp and software-pipelined variants serve M <= 4 only.
constexpr int T5_NVARIANTS = 11;
__host__ __device__ constexpr bool t5_variant_tv(int v) { return v >= 8; }
__host__ __device__ constexpr int t5_variant_ew(int v) {
  return (v == 2 || v == 4 || v == 10 || v == 11) ? 16 : ((v == 6 || v == 7) ? 12 : 8);
}
__host__ __device__ constexpr int t5_variant_tn(int v) { return (v == 6 || v == 7) ? 96 : 128; }
// The tensor-core sums serve square products only: there every row's largest
// kernel value is kappa_ii = 1, while a rectangular product (prediction,
// restricted KRR) may have rows whose kernel values all lie below 2^-20,
// where their fp16 halves (even scaled by 2^14) keep too few bits.
inline bool t5_variant_valid(int v, int M, bool square) {
  return v >= 1 && v <= T5_NVARIANTS && (v == 1 || v == 3 || v == 8 || v == 9 || M <= 4) &&
         (square || !t5_variant_tv(v));
}

// Launches the instance for (nh, csep, M, variant); cudaErrorInvalidValue for
// a shape without one.  Defined per kernel function and family (TV or not) in
// kmvtc5_gauss.cu, kmvtc5_matern.cu, kmvtc5_tv_gauss.cu, kmvtc5_tv_matern.cu.
cudaError_t launch_kmvtc5_gauss(int nh, int csep, int M, int variant, int G, size_t smem,
                                cudaStream_t s, const CUtensorMap &rowmap,
                                const CUtensorMap &colmap, const T5Args &a);
cudaError_t launch_kmvtc5_matern(int nh, int csep, int M, int variant, int G, size_t smem,
                                 cudaStream_t s, const CUtensorMap &rowmap,
                                 const CUtensorMap &colmap, const T5Args &a);
cudaError_t launch_kmvtc5_tv_gauss(int nh, int csep, int M, int variant, int G, size_t smem,
                                   cudaStream_t s, const CUtensorMap &rowmap,
                                   const CUtensorMap &colmap, const T5Args &a);
cudaError_t launch_kmvtc5_tv_matern(int nh, int csep, int M, int variant, int G, size_t smem,
                                    cudaStream_t s, const CUtensorMap &rowmap,
                                    const CUtensorMap &colmap, const T5Args &a);

template <int KERN, int NH, int CS, int M, int EW, int PIPE, int LAG = 0, int TN = 128, int TV = 0>
cudaError_t launch_kmvtc5_one(int G, size_t smem, cudaStream_t s, const CUtensorMap &rowmap,
                              const CUtensorMap &colmap, const T5Args &a) {
  auto k = kmvtc5_kernel<KERN, NH, CS, M, EW, PIPE, LAG, TN, TV>;
  if (raise_smem_limit(k, smem) != KRR_OK) return cudaErrorInvalidValue;
  k<<<G, (EW + 2) * 32, smem, s>>>(rowmap, colmap, a);
  return cudaGetLastError();
}

template <int KERN, int NH, int CS, int M, bool TVSET>
cudaError_t launch_kmvtc5_m(int variant, int G, size_t smem, cudaStream_t s,
                            const CUtensorMap &rowmap, const CUtensorMap &colmap,
                            const T5Args &a) {
  if constexpr (TVSET) {
    switch (variant) {
      case 8: return launch_kmvtc5_one<KERN, NH, CS, M, 8, 1, 0, 128, 1>(G, smem, s, rowmap, colmap, a);
      case 9: return launch_kmvtc5_one<KERN, NH, CS, M, 8, 0, 0, 128, 1>(G, smem, s, rowmap, colmap, a);
      case 10:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 16, 0, 0, 128, 1>(G, smem, s, rowmap, colmap, a);
        break;
      case 11:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 16, 1, 0, 128, 1>(G, smem, s, rowmap, colmap, a);
        break;
    }
  } else {
    switch (variant) {
      case 1: return launch_kmvtc5_one<KERN, NH, CS, M, 8, 1>(G, smem, s, rowmap, colmap, a);
      case 3: return launch_kmvtc5_one<KERN, NH, CS, M, 8, 0>(G, smem, s, rowmap, colmap, a);
      case 2:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 16, 0>(G, smem, s, rowmap, colmap, a);
        break;
      case 4:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 16, 1>(G, smem, s, rowmap, colmap, a);
        break;
      case 5:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 8, 1, 1>(G, smem, s, rowmap, colmap, a);
        break;
      case 6:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 12, 1, 0, 96>(G, smem, s, rowmap, colmap, a);
        break;
      case 7:
        if constexpr (M <= 4) return launch_kmvtc5_one<KERN, NH, CS, M, 12, 0, 0, 96>(G, smem, s, rowmap, colmap, a);
        break;
    }
  }
  return cudaErrorInvalidValue;
}

template <int KERN, bool TVSET>
cudaError_t launch_kmvtc5(int nh, int csep, int M, int variant, int G, size_t smem,
                          cudaStream_t s, const CUtensorMap &rowmap, const CUtensorMap &colmap,
                          const T5Args &a) {
#define KRR_T5_CASE(NH, CS, MM)                                                         \
  if (nh == NH && csep == CS && M == MM)                                              \
    return launch_kmvtc5_m<KERN, NH, CS, MM, TVSET>(variant, G, smem, s, rowmap, colmap, a);
  KRR_T5_CASE(1, 0, 2) KRR_T5_CASE(1, 0, 4) KRR_T5_CASE(1, 0, 8)
  KRR_T5_CASE(1, 1, 2) KRR_T5_CASE(1, 1, 4) KRR_T5_CASE(1, 1, 8)
  KRR_T5_CASE(2, 0, 2) KRR_T5_CASE(2, 0, 4) KRR_T5_CASE(2, 0, 8)
  KRR_T5_CASE(2, 1, 2) KRR_T5_CASE(2, 1, 4) KRR_T5_CASE(2, 1, 8)
#undef KRR_T5_CASE
  return cudaErrorInvalidValue;
}

}  // namespace krr
