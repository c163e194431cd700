// Host side of the tcgen05 product (kmvtc5_kernels.cuh): the split operands
// and their TMA tensor maps, the launch over right-hand-side groups of at
// most 8, and the reduction of the per-CTA segment partial sums.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "kmv.cuh"
#include "kmvtc5_kernels.cuh"

namespace krr {

// ------------------------------------------------------------ preparation
// One thread per point: centred, scaled coordinates split as h + l, c split
// as c1 + c2 + c3; writes the row operand xa and the column operand xb
// (kb = 2 nh + csep blocks of 16 halves each, stored K-block-major: block q
// of point i at (q N + i) 16).  A coordinate or c outside the split's range
// sets *bad.
// cshift is added to c on both sides (7 for the Gaussian: D = log2 kappa + 14).
__global__ void prepare_tc5_kernel(const double *__restrict__ X, int64_t N, int d, int nh,
                                   int csep, const double *__restrict__ mean, double scale,
                                   double cshift, __half *__restrict__ xa,
                                   __half *__restrict__ xb, int *__restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // element t of block q of this point
  auto at = [&](__half *base, int q, int t) -> __half & { return base[((int64_t)q * N + i) * 16 + t]; };
  double nrm = 0.0;
  bool out_of_range = false;
  for (int k = 0; k < nh * 16; ++k) {
    const double v = (k < d) ? (X[i * d + k] - mean[k]) * scale : 0.0;
    if (!(fabs(v) <= (double)T5_MAX_COORD)) out_of_range = true;
    const __half h = __double2half(v);
    const double hv = (double)__half2float(h);
    const __half l = __double2half(v - hv);
    const double e = hv + (double)__half2float(l);
    nrm = fma(e, e, nrm);
    at(xa, k / 16, k % 16) = h;
    at(xb, k / 16, k % 16) = h;
    at(xa, nh + k / 16, k % 16) = l;
    at(xb, nh + k / 16, k % 16) = l;
  }
  const double c = -0.5 * nrm + cshift;
  if (!(fabs(c) <= (double)T5_MAX_C)) out_of_range = true;
  const __half c1 = __double2half(c);
  const double r1 = c - (double)__half2float(c1);
  const __half c2 = __double2half(r1);
  const __half c3 = __double2half(r1 - (double)__half2float(c2));
  const __half one = __double2half(1.0), zero = __double2half(0.0);
  // c-part: its own block, or positions 10..15 of the last H block (those
  // coordinates are beyond d, so their H and L entries are zero)
  const int qc = csep ? 2 * nh : nh - 1, off = csep ? 0 : 10;
  if (csep)
    for (int t = 6; t < 16; ++t) {
      at(xa, qc, t) = zero;
      at(xb, qc, t) = zero;
    }
  const __half pa_c[6] = {c1, c2, c3, one, one, one};
  const __half pb_c[6] = {one, one, one, c1, c2, c3};
  for (int t = 0; t < 6; ++t) {
    at(xa, qc, off + t) = pa_c[t];
    at(xb, qc, off + t) = pb_c[t];
  }
  if (out_of_range) *bad = 1;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensormap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 3-D map over a kb x N x 16 fp16 operand (K-block-major): boxes of 16 halves
// (one K-block row, 32 bytes) x 128 points x kb blocks, 32-byte swizzle, zero
// fill beyond N.  Each block of a box is a contiguous 4 KB range.
static krr_status encode_operand_map(CUtensorMap *map, const uint16_t *ptr, int64_t N, int kb) {
  auto enc = tensormap_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return KRR_ECUDA;
  }
  const cuuint64_t dims[3] = {16, (cuuint64_t)N, (cuuint64_t)kb};
  const cuuint64_t strides[2] = {32, (cuuint64_t)N * 32};
  const cuuint32_t box[3] = {16, (cuuint32_t)T5_TM, (cuuint32_t)kb};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void *)ptr, dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return KRR_ECUDA;
  }
  return KRR_OK;
}

// Builds P's tcgen05 operands (P.nh5 > 0 on success; left at 0 when a point is
// outside the split's range).  P was prepared by prepare_points_f32.
krr_status prepare_points_tc5(const double *Xd, cudaStream_t s, PointsF32 &P, int *h_bad_out) {
  P.nh5 = 0;
  *h_bad_out = 0;
  if (P.kern == KLAPLACE || P.d > 32 || P.N == 0) return KRR_OK;
  const int nh = t5_nh(P.d), csep = t5_csep(P.d), kb = t5_kb(nh, csep);
  const double log2e = 1.4426950408889634;
  const double scale = (P.kern == KGAUSS) ? std::sqrt(log2e) / P.sigma : std::sqrt(5.0) / P.sigma;
  KRR_TRY(P.xa5.alloc((size_t)P.N * kb * 16, s));
  KRR_TRY(P.xb5.alloc((size_t)P.N * kb * 16, s));
  DevBuf<int> bad;
  KRR_TRY(bad.alloc(1, s));
  KRR_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  prepare_tc5_kernel<<<ceil_div(P.N, 256), 256, 0, s>>>(
      Xd, P.N, P.d, nh, csep, P.mean.p, scale, P.kern == KGAUSS ? 7.0 : 0.0,
      reinterpret_cast<__half *>(P.xa5.p),
      reinterpret_cast<__half *>(P.xb5.p), bad.p);
  KRR_LAUNCH_CHECK();
  int h_bad = 0;
  KRR_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_bad) {
    P.xa5.release();
    P.xb5.release();
    *h_bad_out = 1;
    return KRR_OK;
  }
  KRR_TRY(encode_operand_map(&P.ma5, P.xa5.p, P.N, kb));
  KRR_TRY(encode_operand_map(&P.mb5, P.xb5.p, P.N, kb));
  P.nh5 = nh;
  P.csep5 = csep;
  return KRR_OK;
}

// --------------------------------------------------------------- faults
// Set by a CTA whose bounded wait gave up (one flag per device, read and
// cleared by tc5_check_fault).
__device__ int g_t5_fault;

static int *fault_ptr() {
  static std::mutex mtx;
  static int *ptrs[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mtx);
  if (!ptrs[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_t5_fault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs[dev] = static_cast<int *>(p);
  }
  return ptrs[dev];
}

krr_status tc5_check_fault(cudaStream_t s) {
  int *f = fault_ptr();
  if (!f) return KRR_OK;
  int h = 0;
  KRR_CUDA_TRY(cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, s));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    KRR_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(int), s));
    set_error("a bounded wait of the tensor-core product gave up (device-side timeout)");
    return KRR_ETIMEOUT;
  }
  return KRR_OK;
}

// Diagnostic of the bounded waits: one thread waits on an mbarrier that no
// arrival ever completes, for `budget` SM clock cycles, with the routine the
// product's roles use, then takes the timeout path (the fault flag).
__global__ void t5_wait_selftest_kernel(int *fault, long long budget) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  const uint32_t b = bw::smem_u32(&bar);
  bw::mbar_init(b, 1);
  abort_flag = 0;
  bw::fence_mbar_init();
  if (!bw::mbar_wait_abortable(b, 0, budget, &abort_flag)) atomicOr(fault, 1);
}

krr_status tc5_wait_selftest(long long budget, cudaStream_t s) {
  KRR_REQUIRE(budget >= 0 && budget <= (1LL << 31), "wait budget: 0 to 2^31 cycles");
  int *f = fault_ptr();
  KRR_REQUIRE(f != nullptr, "no fault flag on this device");
  t5_wait_selftest_kernel<<<1, 32, 0, s>>>(f, budget);
  KRR_LAUNCH_CHECK();
  return tc5_check_fault(s);
}

// ------------------------------------------------------------ reduction
__global__ void t5_reduce_kernel(const float *__restrict__ part, int64_t Nr, int m, int M, int C,
                                 int64_t T, int G, int J, int CG, const int *__restrict__ vexp,
                                 float lambda, const float *__restrict__ V, int64_t ldv,
                                 float *__restrict__ Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nr) return;
  const int64_t rb = i / T5_RB;
  const int r = (int)(i % T5_RB);
  const int b_lo = t5_cta_of(rb * C, T, G);
  const int b_hi = t5_cta_of(rb * C + C - 1, T, G);
  for (int c = 0; c < m; ++c) {
    double acc = 0.0;   // a row block's segments may come from many CTAs
    for (int b = b_lo; b <= b_hi; ++b) {
      const int64_t j = rb - ((int64_t)b * T / G) / C;
      for (int cg = 0; cg < CG; ++cg)
        acc += (double)part[((((int64_t)b * J + j) * CG + cg) * M + c) * T5_RB + r];
    }
    if (vexp) acc = ldexp(acc, -14 - vexp[c]);
    Y[(int64_t)c * ldy + i] =
        V ? (float)(acc + (double)lambda * (double)V[(int64_t)c * ldv + i]) : (float)acc;
  }
}

// Right-hand sides of the column points as the kernel's shared tiles hold
// them: for column tile t (of TN points), pair cp and column jl, {v_2cp,
// v_2cp, v_2cp+1, v_2cp+1} of point t TN + jl times vscale (zero beyond Nc
// or m); vscale = 2^-14 for the Gaussian, whose kernel values come scaled by
// 2^14.
__global__ void t5_vdup_kernel(const float *__restrict__ V, int64_t ldv, int64_t Nc, int m,
                               int MP, int C, int TN, float vscale, float4 *__restrict__ vdup) {
  const int64_t total = (int64_t)C * MP * TN;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int jl = (int)(e % TN);
    const int cp = (int)((e / TN) % MP);
    const int64_t t = e / ((int64_t)TN * MP);
    const int64_t j = t * TN + jl;
    float va = 0.0f, vb = 0.0f;
    if (j < Nc) {
      if (2 * cp < m) va = V[(int64_t)(2 * cp) * ldv + j] * vscale;
      if (2 * cp + 1 < m) vb = V[(int64_t)(2 * cp + 1) * ldv + j] * vscale;
    }
    vdup[e] = make_float4(va, va, vb, vb);
  }
}

// Largest |v| of each right-hand side (m <= 8) over this block's grid-stride
// share of the Nc points: bmax[block][c].
constexpr int T5_VMAX_BLOCKS = 256;
__global__ void t5_vmax_kernel(const float *__restrict__ V, int64_t ldv, int64_t Nc, int m,
                               float *__restrict__ bmax) {
  __shared__ float red[8][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < 8; ++c) {
    float mx = 0.0f;
    if (c < m)
      for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < Nc;
           j += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(V[(int64_t)c * ldv + j]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp][c] = mx;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    float mx = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w][threadIdx.x]);
    bmax[blockIdx.x * 8 + threadIdx.x] = mx;
  }
}

__device__ __forceinline__ uint32_t t5_pack_halves(__half lo, __half hi) {
  return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

// Right-hand sides as mma.sync B fragments for the TV variants.  Column c is
// scaled by s_c = 2^vexp[c], the power of two that brings its largest |v|
// into [2^13, 2^14), and split into fp16 halves v s_c = v_hi + v_lo.  B slot n
// of fragment f: v_hi of column n (n < M) and v_lo of column n - M (M <= n <
// 2M) for M <= 4; v_hi (f = 0) or v_lo (f = 1) of column n for M = 8.  For
// column tile t, batch bt of 16 columns, fragment f and lane 4 g + q, frag
// holds {B(2q, g), B(2q + 1, g)}, {B(2q + 8, g), B(2q + 9, g)} over the
// batch's columns (zero beyond Nc, m or 2M).  Every block derives the scales
// from bmax (gmax blocks); block 0 also stores vexp for the reduction.
__global__ void t5_vfrag_kernel(const float *__restrict__ V, int64_t ldv, int64_t Nc, int m,
                                int M, int C, int TN, const float *__restrict__ bmax, int gmax,
                                uint2 *__restrict__ frag, int *__restrict__ vexp) {
  __shared__ float sc[8];
  if (threadIdx.x < 8) {
    float mx = 0.0f;
    for (int q = 0; q < gmax; ++q) mx = fmaxf(mx, bmax[q * 8 + threadIdx.x]);
    int e = 0;
    if (mx > 0.0f && mx <= 3.4028234663852886e38f) {
      int E = 0;
      frexpf(mx, &E);   // mx < 2^E
      e = min(max(14 - E, -126), 126);
    }
    sc[threadIdx.x] = ldexpf(1.0f, e);
    if (blockIdx.x == 0) vexp[threadIdx.x] = e;
  }
  __syncthreads();
  const int NB = (M == 8) ? 2 : 1;
  const int nbat = TN / 16;
  const int64_t total = (int64_t)C * nbat * NB * 32;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int lane = (int)(e % 32);
    const int f = (int)((e / 32) % NB);
    const int bt = (int)((e / (32 * NB)) % nbat);
    const int64_t t = e / ((int64_t)32 * NB * nbat);
    const int g = lane >> 2, q = lane & 3;
    int c = g;
    bool lo = (f == 1), live = true;
    if (NB == 1) {
      lo = g >= M;
      c = lo ? g - M : g;
      live = g < 2 * M;
    }
    const int64_t j0 = t * TN + bt * 16;
    auto slot = [&](int k) -> __half {
      const int64_t j = j0 + k;
      if (!live || c >= m || j >= Nc) return __float2half_rn(0.0f);
      const float vs = V[(int64_t)c * ldv + j] * sc[c];
      const __half h = __float2half_rn(vs);
      return lo ? __float2half_rn(vs - __half2float(h)) : h;
    };
    frag[e] = make_uint2(t5_pack_halves(slot(2 * q), slot(2 * q + 1)),
                         t5_pack_halves(slot(2 * q + 8), slot(2 * q + 9)));
  }
}

// ----------------------------------------------------------- variants
// Epilogue variant of the product: forced process-wide (1..T5_NVARIANTS), or
// 0: chosen per shape by timing every valid variant on the caller's stream at
// the first product of that shape while autotuning is on, else the default.
// Results of different variants differ only in the summation order of the
// column groups (rounding level).
static_assert(T5_NVARIANTS == KRR_PRODUCT_VARIANTS, "variant count of the ABI");
// Untuned default: the FMA sums (3) up to 4 right-hand sides per launch, the
// tensor-core sums (9) for 5..8, where they measured 2.96 ms against 4.35 ms
// per product at N = 1e5, d = 16.
static int t5_default_variant(int M, bool square) { return (M == 8 && square) ? 9 : 3; }
static std::atomic<int> g_t5_variant{0};
static std::mutex g_t5_mtx;
struct T5Tune {
  int best = 0;
  float ms[T5_NVARIANTS + 1] = {};
};
static std::map<std::tuple<int, int, int, int, int64_t, int64_t, bool>, T5Tune> g_t5_tuned;

krr_status set_tc5_variant(int v) {
  KRR_REQUIRE(v >= 0 && v <= T5_NVARIANTS, "unknown product variant %d", v);
  g_t5_variant.store(v);
  return KRR_OK;
}

bool tc5_tuned(int kern, int d, int M, int64_t N, int *best, float *ms) {
  const int nh = t5_nh(d), csep = t5_csep(d);
  std::lock_guard<std::mutex> lk(g_t5_mtx);
  auto it = g_t5_tuned.find(std::make_tuple(kern, nh, csep, M, N, N, true));
  if (it == g_t5_tuned.end()) return false;
  *best = it->second.best;
  if (ms)
    for (int v = 1; v <= T5_NVARIANTS; ++v) ms[v - 1] = it->second.ms[v];
  return true;
}

// ------------------------------------------------------------------ launch
// Work geometry of one variant: column tiles of TN points, pairs (row block,
// column tile), grid and segments per CTA.
struct T5Geometry {
  int TN = 128, C = 0, G = 0, J = 1;
  int64_t T = 0;
};

static T5Geometry t5_geometry(int64_t Nr, int64_t Nc, int TN) {
  T5Geometry g;
  g.TN = TN;
  const int64_t Rb = (Nr + T5_RB - 1) / T5_RB;
  g.C = (int)((Nc + TN - 1) / TN);
  g.T = Rb * g.C;
  g.G = (int)std::min<int64_t>(num_sms(), g.T);
  for (int b = 0; b < g.G; ++b) {
    const int64_t p0 = (int64_t)b * g.T / g.G, p1 = (int64_t)(b + 1) * g.T / g.G;
    g.J = std::max<int>(g.J, (int)((p1 - 1) / g.C - p0 / g.C + 1));
  }
  return g;
}

// Scratch of one launch: partial sums (room for 4 column groups), the
// right-hand-side quadruples or B fragments (16-byte aligned), the block
// maxima of V and the scale exponents (TV variants).
static size_t t5_npart(const T5Geometry &g, int M) { return (size_t)g.G * g.J * 4 * M * T5_RB; }
static size_t t5_nvdup(const T5Geometry &g, int M) {
  return (size_t)g.C * g.TN * 4 * (M / 2);   // quadruples, or (fewer) B fragments
}
static size_t t5_scratch_floats(const T5Geometry &g, int M) {
  return t5_npart(g, M) + t5_nvdup(g, M) + T5_VMAX_BLOCKS * 8 + 8;
}
static int *t5_vexp(float *part, const T5Geometry &g, int M) {
  return reinterpret_cast<int *>(part + t5_npart(g, M) + t5_nvdup(g, M) + T5_VMAX_BLOCKS * 8);
}

// Stages V for this geometry and launches the product; returns the launch's
// error.  part must hold t5_scratch_floats(g, M) floats.
static cudaError_t t5_launch(const PointsF32 &R, const PointsF32 &P, int M, int variant,
                             const T5Geometry &g, const float *Vg, int64_t ldv, int mg,
                             float *part, int *fault, cudaStream_t s, bool timed) {
  float *vbuf = part + t5_npart(g, M);
  cudaError_t e = cudaSuccess;
  if (t5_variant_tv(variant)) {
    float *bmax = vbuf + t5_nvdup(g, M);
    const int gmax = (int)std::min<int64_t>((P.N + 255) / 256, T5_VMAX_BLOCKS);
    t5_vmax_kernel<<<gmax, 256, 0, s>>>(Vg, ldv, P.N, mg, bmax);
    count_launch();
    const int NB = (M == 8) ? 2 : 1;
    const int64_t total = (int64_t)g.C * (g.TN / 16) * NB * 32;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    t5_vfrag_kernel<<<blocks, 256, 0, s>>>(Vg, ldv, P.N, mg, M, g.C, g.TN, bmax, gmax,
                                           reinterpret_cast<uint2 *>(vbuf), t5_vexp(part, g, M));
    count_launch();
  } else {
    const int64_t total = (int64_t)g.C * (M / 2) * g.TN;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    t5_vdup_kernel<<<blocks, 256, 0, s>>>(Vg, ldv, P.N, mg, M / 2, g.C, g.TN,
                                          P.kern == KGAUSS ? 0x1p-14f : 1.0f,
                                          reinterpret_cast<float4 *>(vbuf));
    count_launch();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const T5Args args{reinterpret_cast<const float4 *>(vbuf), P.N, part, g.C, g.T, g.J, fault};
  const int nh = P.nh5, csep = P.csep5, kb = t5_kb(nh, csep);
  // at least half of an SM's shared memory: one CTA per SM (each takes all
  // 512 TMEM columns)
  const int ew = t5_variant_ew(variant);
  const size_t smem = std::max<size_t>(
      t5_smem_bytes(kb, M, t5_tot_floats(ew, M, variant == 5, t5_variant_tv(variant))),
      116 * 1024);
  const bool tv = t5_variant_tv(variant), gauss = P.kern == KGAUSS;
  KmvTimer tm;
  if (timed) tm.begin(s);
  if (tv)
    e = gauss ? launch_kmvtc5_tv_gauss(nh, csep, M, variant, g.G, smem, s, R.ma5, P.mb5, args)
              : launch_kmvtc5_tv_matern(nh, csep, M, variant, g.G, smem, s, R.ma5, P.mb5, args);
  else
    e = gauss ? launch_kmvtc5_gauss(nh, csep, M, variant, g.G, smem, s, R.ma5, P.mb5, args)
              : launch_kmvtc5_matern(nh, csep, M, variant, g.G, smem, s, R.ma5, P.mb5, args);
  if (timed) tm.end(s);
  count_launch();
  return e;
}

// Variant for this product: forced, cached, tuned now, or the default.
static int choose_variant(const PointsF32 &R, const PointsF32 &P, bool square, int M,
                          const float *Vg,
                          int64_t ldv, int mg, DevBuf<float> &part, int *fault, cudaStream_t s,
                          bool quiet) {
  const int forced = g_t5_variant.load();
  if (forced > 0 && t5_variant_valid(forced, M, square)) return forced;
  if (quiet) return t5_default_variant(M, square);
  const auto key = std::make_tuple(P.kern, P.nh5, P.csep5, M, R.N, P.N, square);
  {
    std::lock_guard<std::mutex> lk(g_t5_mtx);
    auto it = g_t5_tuned.find(key);
    if (it != g_t5_tuned.end()) return it->second.best;
  }
  if (!autotune_on()) return t5_default_variant(M, square);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return t5_default_variant(M, square);   // timing would synchronise a capturing stream
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return t5_default_variant(M, square);
  }
  T5Tune tune;
  float best_ms = 1e30f;
  tune.best = t5_default_variant(M, square);
  for (int v = 1; v <= T5_NVARIANTS; ++v) {
    if (!t5_variant_valid(v, M, square)) continue;
    const T5Geometry g = t5_geometry(R.N, P.N, t5_variant_tn(v));
    const size_t need = t5_scratch_floats(g, M);
    if (part.n < need && part.alloc(need, s) != KRR_OK) break;
    float ms = 0.0f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {   // the second launch is timed
      ok = t5_launch(R, P, M, v, g, Vg, ldv, mg, part.p, fault, s, false) == cudaSuccess &&
           cudaEventRecord(e0, s) == cudaSuccess &&
           t5_launch(R, P, M, v, g, Vg, ldv, mg, part.p, fault, s, false) == cudaSuccess &&
           cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    }
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    tune.ms[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      tune.best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_t5_mtx);
  g_t5_tuned[key] = tune;
  return tune.best;
}

krr_status kmv_tc5(const PointsF32 &R, const PointsF32 &P, float lambda, bool square,
                   const float *V, int64_t ldv, int m, float *Y, int64_t ldy, cudaStream_t s,
                   DevBuf<float> &part, bool quiet) {
  const int64_t Nr = R.N, Nc = P.N;
  if (Nr == 0 || Nc == 0 || m == 0) return KRR_OK;
  KRR_REQUIRE(R.nh5 > 0 && P.nh5 == R.nh5 && P.csep5 == R.csep5 && R.kern == P.kern,
              "tcgen05 product: operands missing or of different layouts");
  int *fault = fault_ptr();
  KRR_REQUIRE(fault != nullptr, "tcgen05 product: no fault flag on this device");
  for (int c0 = 0; c0 < m; c0 += 8) {
    const int mg = std::min(8, m - c0);
    const int M = mg <= 2 ? 2 : mg <= 4 ? 4 : 8;
    const float *Vg = V + (int64_t)c0 * ldv;
    const int variant = choose_variant(R, P, square, M, Vg, ldv, mg, part, fault, s, quiet);
    const T5Geometry g = t5_geometry(Nr, Nc, t5_variant_tn(variant));
    const size_t need = t5_scratch_floats(g, M);
    if (part.n < need) KRR_TRY(part.alloc(need, s));
    cudaError_t e = t5_launch(R, P, M, variant, g, Vg, ldv, mg, part.p, fault, s, !quiet);
    if (e != cudaSuccess) {
      set_error("tcgen05 product launch failed: %s", cudaGetErrorString(e));
      return KRR_ECUDA;
    }
    const int CG = t5_variant_ew(variant) / 4;
    t5_reduce_kernel<<<ceil_div(Nr, 256), 256, 0, s>>>(
        part.p, Nr, mg, M, g.C, g.T, g.G, g.J, CG,
        t5_variant_tv(variant) ? t5_vexp(part.p, g, M) : nullptr, lambda, square ? Vg : nullptr,
        ldv, Y + (int64_t)c0 * ldy, ldy);
    KRR_LAUNCH_CHECK();
  }
  return KRR_OK;
}

}  // namespace krr
