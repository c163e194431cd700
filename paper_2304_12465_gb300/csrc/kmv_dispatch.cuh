// Compile-time dispatch of the fused product kernels over the padded point
// dimension DP (multiple of 4, <= 32) and the padded right-hand-side count M
// (1, 2, 4, 8, 16).  Each kernel type is instantiated in its own translation
// unit (kmv_gauss.cu, kmv_laplace.cu, kmv_matern.cu) to keep builds parallel.
#pragma once

#include "kmv_kernels.cuh"
#include "kmvff_kernels.cuh"

namespace krr {

struct Kmv32Args {
  const float *xr;   // row points (== xt for the square product)
  const float *cr;
  int64_t Nr;
  const float *xt;
  const float *cn;
  const float *V;
  int64_t ldv, N;
  int m;
  int64_t chunk;
  float *part;
};

struct Kmv64Args {
  const double *Xr;  // row points (== X for the square product)
  int64_t Nr;
  const double *X;
  int d;
  const double *V;
  int64_t ldv, N;
  int m;
  int64_t chunk;
  double inv_scale;
  double *part;
};

template <int KERN, int DP>
cudaError_t launch_kmv32_m(int M, dim3 grid, cudaStream_t s, const Kmv32Args &a) {
  switch (M) {
#define KRR_CASE(MM)                                                              \
  case MM:                                                                        \
    kmv32_kernel<KERN, DP, MM><<<grid, KMV_THREADS, 0, s>>>(a.xr, a.cr, a.Nr, a.xt,    \
                                                           a.cn, a.V, a.ldv, a.N, \
                                                           a.m, a.chunk, a.part); \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8) KRR_CASE(16)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KERN>
cudaError_t launch_kmv32(int DP, int M, dim3 grid, cudaStream_t s, const Kmv32Args &a) {
  switch (DP) {
    case 4: return launch_kmv32_m<KERN, 4>(M, grid, s, a);
    case 8: return launch_kmv32_m<KERN, 8>(M, grid, s, a);
    case 12: return launch_kmv32_m<KERN, 12>(M, grid, s, a);
    case 16: return launch_kmv32_m<KERN, 16>(M, grid, s, a);
    case 20: return launch_kmv32_m<KERN, 20>(M, grid, s, a);
    case 24: return launch_kmv32_m<KERN, 24>(M, grid, s, a);
    case 28: return launch_kmv32_m<KERN, 28>(M, grid, s, a);
    case 32: return launch_kmv32_m<KERN, 32>(M, grid, s, a);
    default: return cudaErrorInvalidValue;
  }
}

template <int KERN, int DP>
cudaError_t launch_kmv64_m(int M, dim3 grid, cudaStream_t s, const Kmv64Args &a) {
  switch (M) {
#define KRR_CASE(MM)                                                                \
  case MM:                                                                          \
    kmv64_kernel<KERN, DP, MM><<<grid, KMV64_THREADS, 0, s>>>(a.Xr, a.Nr, a.X, a.d,  \
                                                             a.V, a.ldv, a.N, a.m,  \
                                                             a.chunk, a.inv_scale,  \
                                                             a.part);               \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8) KRR_CASE(16)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KERN>
cudaError_t launch_kmv64(int DP, int M, dim3 grid, cudaStream_t s, const Kmv64Args &a) {
  switch (DP) {
    case 4: return launch_kmv64_m<KERN, 4>(M, grid, s, a);
    case 8: return launch_kmv64_m<KERN, 8>(M, grid, s, a);
    case 12: return launch_kmv64_m<KERN, 12>(M, grid, s, a);
    case 16: return launch_kmv64_m<KERN, 16>(M, grid, s, a);
    case 20: return launch_kmv64_m<KERN, 20>(M, grid, s, a);
    case 24: return launch_kmv64_m<KERN, 24>(M, grid, s, a);
    case 28: return launch_kmv64_m<KERN, 28>(M, grid, s, a);
    case 32: return launch_kmv64_m<KERN, 32>(M, grid, s, a);
    default: return cudaErrorInvalidValue;
  }
}

struct KmvFFArgs {
  const float *rh, *rl;  // row points (== xh, xl for the square product)
  int64_t Nr;
  const float *xh, *xl, *ch, *cl, *Vh, *Vl;
  int64_t N;
  int m;
  int64_t chunk;
  ExpFFConsts ec;
  double *part;
};

template <int KERN, int DP>
cudaError_t launch_kmvff_m(int M, dim3 grid, cudaStream_t s, const KmvFFArgs &a) {
  switch (M) {
#define KRR_CASE(MM)                                                                 \
  case MM:                                                                           \
    kmvff_kernel<KERN, DP, MM><<<grid, KFF_THREADS, 0, s>>>(                             \
        a.rh, a.rl, a.Nr, a.xh, a.xl, a.ch, a.cl, a.Vh, a.Vl, a.N, a.m, a.chunk, a.ec,  \
        a.part);                                                                        \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4) KRR_CASE(8) KRR_CASE(16)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

struct KmvFFSymArgs {
  const float *xh, *xl, *Vh, *Vl;
  int64_t N;
  int m;
  int nt;      // row tiles
  int64_t T;   // pairs of the upper triangle
  int J;       // segments per CTA (maximum)
  ExpFFConsts ec;
  double *rowpart, *colpart;
  int *seg0;   // first row tile of each CTA (written by the kernel)
};

template <int KERN, int DP>
cudaError_t launch_kmvffsym_m(int M, int G, cudaStream_t s, const KmvFFSymArgs &a) {
  switch (M) {
#define KRR_CASE(MM)                                                                     \
  case MM:                                                                               \
    kmvffsym_kernel<KERN, DP, MM><<<G, KFF_THREADS, 0, s>>>(                             \
        a.xh, a.xl, a.Vh, a.Vl, a.N, a.m, a.nt, a.T, a.J, a.ec, a.rowpart, a.colpart,    \
        a.seg0);                                                                         \
    break;
    KRR_CASE(1) KRR_CASE(2) KRR_CASE(4)
#undef KRR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KERN>
cudaError_t launch_kmvffsym(int DP, int M, int G, cudaStream_t s, const KmvFFSymArgs &a) {
  switch (DP) {
    case 4: return launch_kmvffsym_m<KERN, 4>(M, G, s, a);
    case 8: return launch_kmvffsym_m<KERN, 8>(M, G, s, a);
    case 12: return launch_kmvffsym_m<KERN, 12>(M, G, s, a);
    case 16: return launch_kmvffsym_m<KERN, 16>(M, G, s, a);
    case 20: return launch_kmvffsym_m<KERN, 20>(M, G, s, a);
    case 24: return launch_kmvffsym_m<KERN, 24>(M, G, s, a);
    case 28: return launch_kmvffsym_m<KERN, 28>(M, G, s, a);
    case 32: return launch_kmvffsym_m<KERN, 32>(M, G, s, a);
    default: return cudaErrorInvalidValue;
  }
}

template <int KERN>
cudaError_t launch_kmvff(int DP, int M, dim3 grid, cudaStream_t s, const KmvFFArgs &a) {
  switch (DP) {
    case 4: return launch_kmvff_m<KERN, 4>(M, grid, s, a);
    case 8: return launch_kmvff_m<KERN, 8>(M, grid, s, a);
    case 12: return launch_kmvff_m<KERN, 12>(M, grid, s, a);
    case 16: return launch_kmvff_m<KERN, 16>(M, grid, s, a);
    case 20: return launch_kmvff_m<KERN, 20>(M, grid, s, a);
    case 24: return launch_kmvff_m<KERN, 24>(M, grid, s, a);
    case 28: return launch_kmvff_m<KERN, 28>(M, grid, s, a);
    case 32: return launch_kmvff_m<KERN, 32>(M, grid, s, a);
    default: return cudaErrorInvalidValue;
  }
}

// Per-kernel entry points, defined in kmv_{gauss,laplace,matern}.cu and
// kmvff_{gauss,laplace,matern}.cu.
cudaError_t launch_kmv32_any(int kern, int DP, int M, dim3 grid, cudaStream_t s,
                             const Kmv32Args &a);
cudaError_t launch_kmv64_any(int kern, int DP, int M, dim3 grid, cudaStream_t s,
                             const Kmv64Args &a);
cudaError_t launch_kmvff_any(int kern, int DP, int M, dim3 grid, cudaStream_t s,
                             const KmvFFArgs &a);
cudaError_t launch_kmvffsym_any(int kern, int DP, int M, int G, cudaStream_t s,
                                const KmvFFSymArgs &a);

}  // namespace krr
