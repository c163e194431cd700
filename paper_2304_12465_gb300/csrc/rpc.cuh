// Internal interface of the RPCholesky, preconditioner, PCG and KRILL units.
#pragma once

#include "common.cuh"
#include "handles.cuh"

namespace krr {

constexpr int RPC_MAX_BLOCK = 128;

int fixed_point_bits(int64_t N);

// Draws of block t (see krr_rpc_sample); counts[0] = ndraw or 0 if every
// weight is zero, counts[1] = number of distinct draws written to cand.
krr_status rpc_sample_device(const double *dres, int64_t N, double dfloor, uint64_t seed,
                             uint64_t t, int ndraw, int64_t *draws, int64_t *cand, int *counts,
                             cudaStream_t s);

// Alg. 3 with the pivot rule of krr_pivot_rule (RPCholesky sampling by
// default; uniform and greedy are the comparison rules of Sec. 4).
krr_status rpcholesky_device(const double *Xd, int64_t N, int d, int kern, double sigma,
                             int k, int B, uint64_t seed, cudaStream_t s, krr_factor *f,
                             int rule = KRR_PIVOT_RPCHOLESKY);

// Woodbury core for (mu, prec), built on first use and cached in the factor.
krr_status nystrom_core(const krr_factor *f, double mu, int prec, cudaStream_t s,
                        const NystromCore **out);

// Scratch of the preconditioner apply, kept by a caller that applies it
// repeatedly (a PCG run): grown on first use, then reused, so the launches of
// later applies touch fixed addresses and can be captured in a CUDA graph.
struct PrecondWs {
  DevBuf<double> part, t, u, v;
};

// Z = P^{-1} R for float64 blocks (m x N column-major, ld N); ws = nullptr
// allocates the scratch for this call.
krr_status nystrom_apply_f64(const krr_factor *f, const NystromCore *c, const double *R,
                             int m, double *Z, cudaStream_t s, PrecondWs *ws = nullptr);
// Same with float32 blocks (mixed core).
krr_status nystrom_apply_f32(const krr_factor *f, const NystromCore *c, const float *R,
                             int m, float *Z, cudaStream_t s, PrecondWs *ws = nullptr);

void free_factor(krr_factor *f);

}  // namespace krr
