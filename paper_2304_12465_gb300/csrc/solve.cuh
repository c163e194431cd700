// Solve drivers (solve.cu).
#pragma once

#include <vector>

#include "common.cuh"
#include "handles.cuh"
#include "kmv.cuh"

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

// Continuation of a mixed-precision refinement whose float32 inner
// iterations stalled (very small mu with smooth kernels: the float32
// product's rounding then exceeds lambda): the same refinement with float64
// CG vectors, the float-float product inside PCG and the Woodbury
// preconditioner applied in float64 to the float32 factor it was built from;
// when even the float-float residuals stall, the residuals come from the
// float64 product on X.  alpha, r64 (= Y - M alpha) and the host-side norms
// and counters are updated in place.
struct Escalation {
  const PointsFF *Pff = nullptr;      // float-float prepared points
  const double *X = nullptr;          // N x d float64 points (host or device)
  int64_t N = 0;
  int d = 0, kern = 0, m = 0;
  double sigma = 0.0, lambda = 0.0, tol = 0.0;
  const NystromCore *core = nullptr;  // mixed core (F32, W, Wt) or null: P = lambda I
  const double *Y = nullptr;          // m x N right-hand sides
  double *alpha = nullptr;            // m x N iterate
  double *r64 = nullptr;              // m x N residual Y - M alpha
  double *mx = nullptr;               // m x N scratch
  std::vector<double> yn, rn;         // column norms of Y and of r64
  int budget = 0, iters = 0, outer = 0;
  double entries = 0.0, relres = 0.0;
  DevBuf<double> *ffpart = nullptr;   // float-float product scratch
  DevBuf<float> *ffvsplit = nullptr;
  krr_status status = KRR_ENOCONV;    // outcome
};
krr_status escalate_refine(Escalation &e, cudaStream_t s);

// Alg. 2 PCG; Y (N x m) and beta (k x m) are device arrays.
krr_status krill_solve_device(const krill_precond *P, const double *Y, int m, double tol,
                              int maxit, double *beta, cudaStream_t s, krr_info *info);

}  // namespace krr
