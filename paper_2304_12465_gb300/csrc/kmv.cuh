// Host-side interface of the fused product (kmatvec.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace krr {

// Points prepared for the float32 product: centred, scaled, padded to DP
// (a multiple of 4) coordinates, plus the per-point constant c_i.
struct PointsF32 {
  DevBuf<float> xt;   // N x dp
  DevBuf<float> cn;   // N
  DevBuf<double> mean;  // d, the centre subtracted from every point
  int dp = 0;
  int d = 0;
  int64_t N = 0;
  int kern = 0;
  double sigma = 0.0;
  // half-split layout of the tensor-core product (kmvtc_kernels.cuh), present
  // when kc16 > 0: N x kc16 x 4 groups of 16 bytes, and c_i
  DevBuf<uint4> xs16;
  DevBuf<float> cs16;
  int kc16 = 0;
  // operands of the tcgen05 product (kmvtc5_kernels.cuh), present when
  // nh5 > 0: N x kb x 16 fp16 each, row operand (c-part c1, c2, c3, 1, 1, 1)
  // and column operand (1, 1, 1, c1, c2, c3), and their TMA tensor maps
  DevBuf<uint16_t> xa5, xb5;
  CUtensorMap ma5{}, mb5{};
  int nh5 = 0, csep5 = 0;
};

// mean_dev (optional, d doubles on the device): centre to use instead of the
// points' own mean (prediction prepares test points with the training mean).
// dp (optional): padded dimension (a multiple of 4 in [d, 32]) instead of the
// smallest multiple of 4 >= d.
krr_status prepare_points_f32(const double *Xd, int64_t N, int d, int kern,
                              double sigma, cudaStream_t s, PointsF32 &P,
                              const double *mean_dev = nullptr, int dp = 0);

// Adds the half-split layouts of the tensor-core products to P (prepared by
// prepare_points_f32 from the same Xd) for the Gaussian and Matern kernels:
// the mma.sync layout (kc16 > 0) and, when with_tc5, the tcgen05 operands
// (nh5 > 0).  Leaves both absent (FMA product) for Laplace or when a centred,
// scaled coordinate (or c) exceeds the half-precision split's range.
// Synchronises s.
krr_status prepare_points_tc(const double *Xd, cudaStream_t s, PointsF32 &P,
                             bool with_tc5 = true);

// Builds only the tcgen05 operands of P (P.nh5 > 0); *bad = 1 (and nh5 = 0)
// when a point is outside the split's range.  Synchronises s.
krr_status prepare_points_tc5(const double *Xd, cudaStream_t s, PointsF32 &P, int *bad);

// tcgen05 product Y (R.N x m) = K(R, P) V, + lambda V when square (R is P);
// both point sets carry tcgen05 operands prepared with the same centre and
// scale.  V: m x ldv over P's points; Y: m x ldy over R's points.  quiet:
// the process's forced variant or the default one, never tuned or timed (the
// serving engine's products, launched into captured graphs).
krr_status kmv_tc5(const PointsF32 &R, const PointsF32 &P, float lambda, bool square,
                   const float *V, int64_t ldv, int m, float *Y, int64_t ldy, cudaStream_t s,
                   DevBuf<float> &part, bool quiet = false);

// Epilogue variant of the tcgen05 product (see krr_set_product_variant), and
// the autotuner's choice and per-variant times for a square shape.
krr_status set_tc5_variant(int v);
bool tc5_tuned(int kern, int d, int M, int64_t N, int *best, float *ms);
bool autotune_on();

// Raises KRR_ETIMEOUT (and clears the flag) when a bounded device-side wait
// of the tcgen05 product gave up since the last check; synchronises s.
krr_status tc5_check_fault(cudaStream_t s);
// Runs a bounded wait that cannot complete; KRR_ETIMEOUT once it gave up.
krr_status tc5_wait_selftest(long long budget, cudaStream_t s);

struct KmvTcArgs {
  const uint4 *xs;
  const float *cs;
  const float *V;
  int64_t ldv, N;
  int m;
  int64_t chunk;
  float *part;
};
cudaError_t launch_kmvtc(int kern, int KC, int M, dim3 grid, cudaStream_t s,
                         const KmvTcArgs &a);
int kmvtc_rows_per_cta(int KC, int M);

// Product path of kmv_f32 when P has the half-split layouts: 0 tcgen05
// tensor cores (default), 1 the FMA kernel, 2 the mma.sync tensor-core kernel
// (see krr_set_product_path).
void set_product_path(int path);
int product_path();

// Prediction products (no shift): Y (Nr x m) = K(rows, columns) V.
krr_status kcross_f32(const PointsF32 &R, const PointsF32 &P, const float *V, int64_t ldv,
                      int m, float *Y, int64_t ldy, cudaStream_t s, DevBuf<float> &part);
krr_status kcross_f64(const double *Xr, int64_t Nr, const double *Xd, int64_t N, int d,
                      int kern, double sigma, const double *V, int64_t ldv, int m, double *Y,
                      int64_t ldy, cudaStream_t s, DevBuf<double> &part);

// Points split for the float-float product: centred, scaled x = xh + xl and
// c = -|x|^2/2 = ch + cl (unused for Laplace).
struct PointsFF {
  DevBuf<float> xh, xl;   // N x dp
  DevBuf<float> ch, cl;   // N
  DevBuf<double> mean;    // d
  int dp = 0;
  int d = 0;
  int64_t N = 0;
  int kern = 0;
};

krr_status prepare_points_ff(const double *Xd, int64_t N, int d, int kern, double sigma,
                             cudaStream_t s, PointsFF &P, const double *mean_dev = nullptr);

// Rectangular float-float product Y (R.N x m) = K(R, P) V; when &R == &P the
// shift lambda V is added (square product).
krr_status kff_cross(const PointsFF &R, const PointsFF &P, double lambda, const double *V,
                     int64_t ldv, int m, double *Y, int64_t ldy, cudaStream_t s,
                     DevBuf<double> &part, DevBuf<float> &vsplit);

// Y (float64) = (A + lambda I) V (float64) with float64-accurate kernel
// entries computed in float-float arithmetic on the float32 pipes.
krr_status kmv_ff(const PointsFF &P, double lambda, const double *V, int64_t ldv, int m,
                  double *Y, int64_t ldy, cudaStream_t s, DevBuf<double> &part,
                  DevBuf<float> &vsplit);

// Autotuning of the float32 product's column tile (see krr_set_autotune);
// tuned_splits returns the cached split count of a shape, 0 if not tuned.
void set_autotune(bool on);
int tuned_splits(int kern, int dp, int M, int64_t N);

// Y (m x ldy, float32) = (A + lambda I) V (m x ldv, float32).
krr_status kmv_f32(const PointsF32 &P, float lambda, const float *V, int64_t ldv,
                   int m, float *Y, int64_t ldy, cudaStream_t s, DevBuf<float> &part);

// Y (m x ldy, float64) = (A + lambda I) V (m x ldv, float64); Xd N x d float64.
krr_status kmv_f64(const double *Xd, int64_t N, int d, int kern, double sigma,
                   double lambda, const double *V, int64_t ldv, int m, double *Y,
                   int64_t ldy, cudaStream_t s, DevBuf<double> &part);

// kmv_f64 with caller-provided scratch for the split partial sums (no
// allocation); KRR_EINVAL if N x padded(m) exceeds scratch_elems.
krr_status kmv_f64_with_scratch(const double *Xd, int64_t N, int d, int kern, double sigma,
                                double lambda, const double *V, int64_t ldv, int m, double *Y,
                                int64_t ldy, double *scratch, size_t scratch_elems,
                                cudaStream_t s);

// Batched multi-setting float32 product (kmvb.cu): S settings (kernel type,
// sigma) with ms columns each, column s*ms + c shifted by lambda_dev[s*ms+c];
// V, Y: (S ms) x N.  Points prepared by kmvb_prepare (centred, unscaled).
krr_status kmvb_prepare(const double *Xd, int64_t N, int d, cudaStream_t s, PointsF32 &P);
krr_status kmv_batched_f32(const PointsF32 &P, int S, const int *kerns, const double *sigmas,
                           int ms, const float *lambda_dev, const float *V, float *Y,
                           cudaStream_t s, DevBuf<float> &part);

// Number of kernel entries one product evaluates (N^2).
inline double kmv_entries(int64_t N) { return (double)N * (double)N; }

// Element-wise conversions between float64 and float32 blocks.
krr_status convert_f64_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s);
krr_status convert_f32_to_f64(const float *src, double *dst, int64_t n, cudaStream_t s);

// Kernel function value on device, float64, from direct coordinate
// differences (the definitions of Sec. 2.1.2 / Sec. 5.1 / textbook Matern).
__device__ __forceinline__ double kappa_point_f64(const double *a, const double *b,
                                                  int d, int kern, double sigma) {
  double s = 0.0;
  if (kern == KLAPLACE) {
    for (int k = 0; k < d; ++k) s += fabs(a[k] - b[k]);
    return exp(-s / sigma);
  }
  for (int k = 0; k < d; ++k) {
    const double t = a[k] - b[k];
    s = fma(t, t, s);
  }
  if (kern == KMATERN) {
    const double q = sqrt(5.0 * s) / sigma;
    return (1.0 + q + q * q / 3.0) * exp(-q);
  }
  return exp(-s / (2.0 * sigma * sigma));
}

// G (nc x ldg column-major, rows 0..N-1) = A(:, cols), float64.
krr_status kernel_columns_f64(const double *Xd, int64_t N, int d, int kern,
                              double sigma, const int64_t *cols, int nc, double *G,
                              int64_t ldg, cudaStream_t s);

// out[i] = kappa(x_i, x_i) for all i (float64).
krr_status kernel_diag_f64(const double *Xd, int64_t N, int d, int kern, double sigma,
                           double *out, cudaStream_t s);

}  // namespace krr
