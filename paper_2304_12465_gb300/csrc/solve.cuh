// Solve drivers (solve.cu).
#pragma once

#include "common.cuh"
#include "handles.cuh"

namespace krr {

// Alg. 1 PCG on (A + mu N I) alpha = Y; Xd, Y, alpha are device arrays.
krr_status pcg_solve_device(const double *Xd, int64_t N, int d, int kern, double sigma,
                            const double *Y, int m, double mu, const krr_factor *F,
                            double tol, int maxit, int prec, double *alpha, cudaStream_t s,
                            krr_info *info);

// Batched Alg. 1 PCG over S settings x ms regularisations (mixed precision):
// column q*ms + c solves (A_q + mus[c] N I) x = Y column; factors[q] may be
// NULL.  Device arrays.
krr_status pcg_solve_batched_device(const double *Xd, int64_t N, int d, int S,
                                    const int *kerns, const double *sigmas,
                                    const krr_factor *const *factors, int ms,
                                    const double *mus, const double *Y, double tol, int maxit,
                                    double *alpha, cudaStream_t s, krr_info *info);

// Alg. 2 PCG; Y (N x m) and beta (k x m) are device arrays.
krr_status krill_solve_device(const krill_precond *P, const double *Y, int m, double tol,
                              int maxit, double *beta, cudaStream_t s, krr_info *info);

}  // namespace krr
