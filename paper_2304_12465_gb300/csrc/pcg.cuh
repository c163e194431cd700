// PCG driver interface (pcg.cu).
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace krr {

constexpr int PCG_MAX_M = 16;

// Device-resident per-column CG scalars (float64).
struct PcgScalars {
  double rz[PCG_MAX_M];
  double bb[PCG_MAX_M];
  double alpha[PCG_MAX_M];
  double beta[PCG_MAX_M];
  double relres[PCG_MAX_M];
  double tol[PCG_MAX_M];
  int active[PCG_MAX_M];
  int iters[PCG_MAX_M];
  int breakdown;
  int it;   // iterations taken (counted on the device)
};

// Operator and preconditioner of one PCG run, on m x N column-major blocks.
template <typename T>
struct PcgOps {
  std::function<krr_status(const T *in, T *out, cudaStream_t)> product;
  std::function<krr_status(const T *in, T *out, cudaStream_t)> precond;
};

struct PcgStats {
  int products = 0;       // operator applications
  int iters_max = 0;
  double relres_max = 0;  // recursive residual at exit
  bool converged = false;
  bool breakdown = false;
  int col_iters[PCG_MAX_M] = {0};
  double col_relres[PCG_MAX_M] = {0};
  int graph_replays = 0;  // CUDA-graph chunks replayed
  int host_checks = 0;    // convergence flags read back by the host
};

// CUDA-graph replay of the PCG iterations (krr_set_pcg_graphs; on by default).
void set_pcg_graphs(bool on);
bool pcg_graphs_on();
// Graph replays and host read-backs of the convergence flags made by this
// thread's pcg_run calls since the last call (which resets both).
void pcg_counters_take(int *replays, int *checks);

// Standard PCG with zero initial iterate; column c stops when its recursive
// relative residual is <= tol_host[c] (each column has its own scalars).
// After the first iteration the iterations run as replays of CUDA graphs of
// 16, 4 or 1 iterations (their launches captured once per run), the
// convergence flags read back once per replay; converged columns freeze on
// the device, so the iterates are those of one-iteration-at-a-time stepping.
// The operator and preconditioner must launch only on the stream they are
// given and allocate only on their first call.
template <typename T>
krr_status pcg_run(const PcgOps<T> &ops, int64_t N, int m, const T *b, T *x,
                   const double *tol_host, int maxit, cudaStream_t s, PcgStats *stats);

// u (m x rank) = W t (given Wt = W^T) and v = W^T u (given W), W lower
// triangular rank x rank, column-major.
krr_status tri_apply_lower(const double *Wt, int rank, const double *t, int m, double *u,
                           cudaStream_t s);
krr_status tri_apply_lower_t(const double *W, int rank, const double *u, int m, double *v,
                             cudaStream_t s);

krr_status residual_f64(const double *y, const double *mx, double *r, int64_t n,
                        cudaStream_t s);
krr_status add_f32_to_f64(double *x, const float *d, int64_t n, cudaStream_t s);
krr_status column_norms(const double *a, int64_t N, int m, double *out_host, cudaStream_t s);

}  // namespace krr
