// Device-side layout of the serving engine (serve.cu, serve_kmv.cu).
//
// Every admitted solve ("slot") keeps its prepared points, its Nystrom
// preconditioner and its float32 CG state resident in HBM.  A step advances
// the inner PCG iteration of the iterating slots of one lane with one product
// launch per variant present and one grouped launch per other phase of
// Alg. 1's loop: each is a grid of CTAs that walks a work list spanning the
// slots (product tiles, row blocks, triangular rows, CG columns).  The work
// list lives in a device table; the launch sequence only changes with the
// set of variants present, and is captured as a CUDA graph.
//
// A slot's work decomposition (tile shape, column splits, row blocks) is a
// function of that slot alone, and every sum is taken in a fixed order, so a
// solve produces the same bits whether it runs alone or among other solves.
#pragma once

#include "common.cuh"

namespace krr {

constexpr int SERVE_MAX_SLOTS = 64;     // slots per table (== KRR_SERVE_MAX_SLOTS)
constexpr int SERVE_MAX_BUILDERS = 8;   // builder threads (== KRR_SERVE_MAX_BUILDERS)
constexpr int SERVE_MAX_M = 16;         // right-hand sides per solve
constexpr int SERVE_VB = 256;           // rows per vector block (one per thread)
constexpr int SERVE_TT_ROWS = 512;      // rows per block of F^T r
constexpr int SERVE_TT_COLS = 64;       // columns of F per block of F^T r
constexpr int SERVE_MAX_SPLITS = 32;    // column splits of one slot's product
constexpr int SERVE_MIN_CHUNK = 256;    // columns per split at least

// Per-slot CG scalars (float64), one entry per right-hand side.  The control
// block is written by the host before an inner solve starts.
struct ServeControl {
  double tol[SERVE_MAX_M];   // inner relative tolerance per column
  int need[SERVE_MAX_M];     // column takes part in this inner solve
  int limit;                 // iteration limit of this inner solve
  int pad;
};

struct ServeScalars {
  ServeControl ctl;
  double rz[SERVE_MAX_M];
  double bb[SERVE_MAX_M];
  double alpha[SERVE_MAX_M];
  double beta[SERVE_MAX_M];
  double relres[SERVE_MAX_M];
  int active[SERVE_MAX_M];
  int iters[SERVE_MAX_M];
  int live;        // some column still iterating
  int breakdown;
  double resid_sq[SERVE_MAX_M];   // squared norms of the float64 residual
};

// Compact per-slot status read back by the host after every step.
struct ServeStatus {
  int live;
  int breakdown;
  int iters_max;
  int pad;
};

struct ServeSlotDesc {
  // fused float32 product (A + lambda I) p
  const float *xt;   // N x dp prepared points
  const float *cn;   // N per-point constants
  // tensor-core product (kc > 0): half-split points and their constants
  const uint4 *xs;   // N x kc x 4 fragment groups
  const float *cs;   // N
  int kc;            // 16-coordinate blocks, 0 for the FMA product
  int halves;        // product items per (row tile, split): 2 for a tensor-core M = 16
  int tc5;           // 1: the slot's product is its own tcgen05 launch (large
                     // Gaussian / Matern slots), writing part as one split
  float *part;       // splits x M x N partial sums
  int64_t N;
  int64_t chunk;     // columns per split
  int m, M, dp, kern;
  int variant;       // product dispatch index (kernel, DP class, M class)
  int row_tiles, splits;
  float lam32;
  double inv_lam;
  // CG vectors, float32, column c at base + c N
  float *x, *r, *z, *p, *q;
  const double *r64;   // float64 residual, source of an inner right-hand side
  // Woodbury preconditioner P^{-1} = lambda^{-1}(I - F W^T W F^T)
  const float *F;      // N x rank (float32)
  const double *W;     // rank x rank lower
  const double *Wt;    // W^T
  int rank;
  int nbt;             // ceil(N / SERVE_TT_ROWS)
  double *ttpart;      // nbt x rank x m
  double *t, *u, *v;   // m x rank each
  // fixed-order reductions
  int nbv;             // ceil(N / SERVE_VB)
  double *dpart0, *dpart1;   // m x nbv block partial dot products
  ServeScalars *sc;
  ServeStatus *status;
};

// FMA products: 3 kernels x 4 DP classes x 5 M classes; tensor-core products:
// (Gaussian, Matern) x 1 or 2 coordinate blocks x 5 M classes (M = 16 runs as
// two halves of 8)
constexpr int SERVE_NUM_FMA_VARIANTS = 60;
constexpr int SERVE_NUM_VARIANTS = SERVE_NUM_FMA_VARIANTS + 20;

// The slots of one product variant: the product launch of that variant
// covers their (row tile, split) items, item i of slot slot[j] being
// i - off[j] for off[j] <= i < off[j + 1].
struct ServeClass {
  int variant;
  int nslots;
  int slot[SERVE_MAX_SLOTS];          // indices into ServeTable::slot
  int off[SERVE_MAX_SLOTS + 1];
};

// Work list of one launch sequence: cumulative item counts per phase.
struct ServeTable {
  int nslots;
  int nclasses;
  ServeClass cls[SERVE_NUM_VARIANTS];  // product launches, one per variant present
  int vec_off[SERVE_MAX_SLOTS + 1];    // vector blocks of SERVE_VB rows
  int tt_off[SERVE_MAX_SLOTS + 1];     // F^T r blocks (row block, column group)
  int ttr_off[SERVE_MAX_SLOTS + 1];    // rank x m reductions
  int tri_off[SERVE_MAX_SLOTS + 1];    // triangular rows (rank)
  int col_off[SERVE_MAX_SLOTS + 1];    // CG columns
  ServeSlotDesc slot[SERVE_MAX_SLOTS];
};

// Slot owning `item` in a cumulative offset array (last s with off[s] <= item).
__device__ __forceinline__ int serve_find_slot(const int *off, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Product dispatch index of (kernel, padded dimension, padded m); -1 when the
// combination has no grouped variant.
__host__ __device__ inline int serve_dp_class(int d) {
  return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : -1;
}
__host__ __device__ inline int serve_variant(int kern, int dp, int M) {
  const int di = dp == 4 ? 0 : dp == 8 ? 1 : dp == 16 ? 2 : dp == 32 ? 3 : -1;
  const int mi = M == 1 ? 0 : M == 2 ? 1 : M == 4 ? 2 : M == 8 ? 3 : M == 16 ? 4 : -1;
  if (di < 0 || mi < 0 || kern < 0 || kern > 2) return -1;
  return (kern * 4 + di) * 5 + mi;
}
__host__ __device__ inline int serve_variant_tc(int kern, int kc, int M) {
  const int ki = kern == KGAUSS ? 0 : kern == KMATERN ? 1 : -1;
  const int mi = M == 1 ? 0 : M == 2 ? 1 : M == 4 ? 2 : M == 8 ? 3 : M == 16 ? 4 : -1;
  if (ki < 0 || mi < 0 || kc < 1 || kc > 2) return -1;
  return SERVE_NUM_FMA_VARIANTS + (ki * 2 + kc - 1) * 5 + mi;
}

// Grouped product of class `cls` of the table at T (device pointer): one CTA
// per item, `items` of them (serve_kmv_*.cu, one file per kernel function).
cudaError_t serve_launch_product_gauss(int dp, int M, int items, const ServeTable *T, int cls,
                                       cudaStream_t s);
cudaError_t serve_launch_product_laplace(int dp, int M, int items, const ServeTable *T, int cls,
                                         cudaStream_t s);
cudaError_t serve_launch_product_matern(int dp, int M, int items, const ServeTable *T, int cls,
                                        cudaStream_t s);
// Tensor-core variants (serve_kmv_tc.cu): kern KGAUSS or KMATERN, kc 1 or 2,
// M 1, 2, 4, 8 or 16 (items: row tiles x splits, twice for M = 16).
cudaError_t serve_launch_product_tc(int kern, int kc, int M, int items, const ServeTable *T,
                                    int cls, cudaStream_t s);

}  // namespace krr
