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

}  // namespace krr
