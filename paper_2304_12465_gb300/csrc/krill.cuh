// KRILL internals (krill.cu).
#pragma once

#include "common.cuh"
#include "handles.cuh"
#include "kmv.cuh"

namespace krr {

krr_status sparse_sign_device(int64_t N, int s, int zeta, uint64_t seed, int32_t *rows,
                              float *vals32, double *vals64, cudaStream_t st);
krr_status krill_build_device(krill_precond *P, cudaStream_t s);
krr_status krill_product(const krill_precond *P, const double *beta, int m, double *out,
                         cudaStream_t s, DevBuf<float> &u, DevBuf<double> &v);
krr_status krill_precond_apply(const krill_precond *P, const double *in, int m, double *tmp,
                               double *out, cudaStream_t s);
// float-float point sets and scratch of one KRILL solve
struct KrillFF {
  PointsFF all, centers;
  DevBuf<double> part;
  DevBuf<float> vsplit;
};
krr_status krill_points_ff(const krill_precond *P, cudaStream_t s, KrillFF &Q);
krr_status krill_product64(const krill_precond *P, KrillFF &Q, const double *beta, int m,
                           double *out, cudaStream_t s, DevBuf<double> &u, DevBuf<double> &v);
krr_status krill_rhs(const krill_precond *P, KrillFF &Q, const double *y, int m, double *b,
                     cudaStream_t s);

// tcgen05 operands of one KRILL solve (Gaussian and Matern on the tensor-core
// product path): all points and the centers, split with the same centre and
// scale, and the scratch of the rectangular products.  ok is false when the
// FMA block products serve the solve (Laplace, the FMA product path, or
// coordinates outside the split's range).
struct KrillTC5 {
  PointsF32 all, centers;
  DevBuf<float> part, b32, v32;
  DevBuf<double> v64;
  bool ok = false;
};
krr_status krill_points_tc5(const krill_precond *P, cudaStream_t s, KrillTC5 &T);
// M beta = A(S,:)(A(:,S) beta) + H beta with both block products on the
// tcgen05 product (float32 entries and sums, float64 H beta).
krr_status krill_product_tc5(const krill_precond *P, KrillTC5 &T, const double *beta, int m,
                             double *out, cudaStream_t s, DevBuf<float> &u);

}  // namespace krr
