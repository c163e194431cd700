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

// Z = P^{-1} R for float64 blocks (m x N column-major, ld N).
krr_status nystrom_apply_f64(const krr_factor *f, const NystromCore *c, const double *R,
                             int m, double *Z, cudaStream_t s);
// Same with float32 blocks (mixed core).
krr_status nystrom_apply_f32(const krr_factor *f, const NystromCore *c, const float *R,
                             int m, float *Z, cudaStream_t s);

void free_factor(krr_factor *f);

}  // namespace krr
