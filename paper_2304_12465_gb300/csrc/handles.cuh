// Library-owned handle layouts shared by the translation units.
#pragma once

#include <deque>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace krr {

// Woodbury core of the Alg. 1 preconditioner for one (lambda, precision):
// W = L^{-1}, L L^T = lambda I + Fp^T Fp, where Fp is F (float64) or F
// rounded to float32 (mixed); P^{-1} = lambda^{-1}(I - Fp W^T W Fp^T).
struct NystromCore {
  double mu = 0.0;
  double lambda = 0.0;
  int prec = 0;
  int rank = 0;
  double *W = nullptr;    // rank x rank, column-major, lower
  double *Wt = nullptr;   // W^T (row access of W)
  float *F32 = nullptr;   // N x rank float32 copy (mixed only)
  double build_s = 0.0;
};

}  // namespace krr

struct krr_factor {
  int64_t N = 0;
  int d = 0;
  int kern = 0;
  double sigma = 0.0;
  int k = 0;
  int rank = 0;
  int nblocks = 0;
  uint64_t seed = 0;
  double *F = nullptr;      // N x k column-major (first `rank` columns valid)
  int64_t *S = nullptr;     // pivots, column order
  double *dres = nullptr;   // residual diagonal
  // non-null when the factor was built with a thread allocation stream: its
  // memory is then released with cudaFreeAsync on this stream
  cudaStream_t free_stream = nullptr;
  mutable std::mutex mtx;
  // a deque keeps the address of every core stable while more are added, so
  // pointers handed out by nystrom_core stay valid for the factor's lifetime
  mutable std::deque<krr::NystromCore> cores;
};

struct krill_precond {
  int64_t N = 0;
  int d = 0;
  int kern = 0;
  double sigma = 0.0;
  int k = 0;
  int s = 0;
  int zeta = 0;
  double mu = 0.0, lambda = 0.0;
  uint64_t seed = 0;
  double *X = nullptr;        // N x d float64 copy
  int64_t *S = nullptr;       // centers
  double *H = nullptr;        // k x k
  double *Bsk = nullptr;      // s x k, column-major
  double *P = nullptr;        // k x k (B^T B + H)
  double *L = nullptr;        // k x k lower factor, P = L L^T (C = L^T)
  double *Winv = nullptr;     // k x k, L^{-1}
  double *Winv_t = nullptr;   // (L^{-1})^T
  float *xt = nullptr;        // prepared float32 points for the product
  float *cn = nullptr;
  int dp = 0;
  double build_s = 0.0;
};
