/*
 * krr.h -- C ABI of the GB300 (sm_103a) kernel ridge regression library.
 *
 * Method: "Robust, randomized preconditioning for kernel ridge regression"
 * (Diaz, Epperly, Frangella, Tropp, Webber).
 *   full-data KRR   (A + lambda I) alpha = y                     Sec. 2.1
 *   RPCholesky preconditioned CG                                 Alg. 1, Alg. 3
 *   restricted KRR  [A(S,:)A(:,S) + lambda A(S,S)] beta = A(S,:) y   Sec. 2.2
 *   KRILL preconditioned CG                                      Alg. 2
 * with A_ij = kappa(x_i, x_j) generated on the fly and never stored.
 *
 * Conventions shared by every call
 * --------------------------------
 * - X is N x d, row-major float64 (point i is X[i*d .. i*d+d-1]), 1 <= d <= 32.
 * - Right-hand-side / solution blocks are N x m (or k x m) column-major
 *   float64: column c starts at c*N (c*k).  1 <= m <= 16.
 * - mu is the regularisation per data point; the shift is lambda = mu * N
 *   (the paper's mu, Sec. 2.1.2, quoted there as mu / N).
 * - Array arguments may be host or device pointers: the library asks the CUDA
 *   runtime which one it got and copies host data in / out itself.  Device
 *   pointers must belong to the current device.  The caller owns every array
 *   it passes; handles (krr_factor, krill_precond) own their device memory.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Work is enqueued on it; calls return after their results are complete
 *   (each call synchronises the stream before returning).
 * - No call aborts, traps or exits.  Invalid arguments return KRR_EINVAL
 *   before any launch; CUDA failures return KRR_ECUDA.  krr_last_error()
 *   describes the last failure of the calling thread.
 * - The library is built for sm_103a only and never falls back to the CPU.
 */
#ifndef KRR_GB300_H
#define KRR_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define KRR_API __attribute__((visibility("default")))
#else
#define KRR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KRR_OK = 0,
    KRR_EINVAL = 1,      /* bad argument (checked before any launch)          */
    KRR_ENOMEM = 2,      /* device allocation failed                          */
    KRR_ECUDA = 3,       /* CUDA runtime error                                */
    KRR_ECHOL = 4,       /* non-positive pivot in a k x k Cholesky factor     */
    KRR_EBREAKDOWN = 5,  /* p^T M p <= 0 or NaN in PCG                        */
    KRR_ENOCONV = 6,     /* maxit reached before the tolerance                */
    KRR_ETIMEOUT = 7     /* a bounded device-side wait gave up                */
} krr_status;

typedef enum {
    KRR_GAUSSIAN = 0,    /* exp(-||x-y||^2 / (2 sigma^2)), Sec. 2.1.2          */
    KRR_LAPLACE_L1 = 1,  /* exp(-||x-y||_1 / sigma), l1 distance, Sec. 5.1     */
    KRR_MATERN52 = 2     /* (1 + q + q^2/3) exp(-q), q = sqrt(5)||x-y||/sigma;
                            not in the paper: textbook Matern, nu = 5/2        */
} krr_kernel;

typedef enum {
    KRR_PREC_FP64 = 0,   /* every step in float64                             */
    KRR_PREC_MIXED = 1,  /* float32 kernel tiles and inner PCG, float64-accurate
                            outer iterative refinement, float64 CG scalars and
                            k x k core                                         */
    KRR_PREC_FLOAT_FLOAT = 2  /* krr_kmatvec and krr_pcg_solve: float64-accurate
                            product (about 2^-46 per entry) evaluated in
                            float-float arithmetic on the float32 pipes; the
                            product the mixed path uses for its refinement
                            residuals                                         */
} krr_precision;

/* Pivot rule of the partial Cholesky factorization: RPCholesky (Alg. 3)    */
/* and the two rules the paper compares it with in Sec. 4.                   */
typedef enum {
    KRR_PIVOT_RPCHOLESKY = 0,  /* pivots ~ residual diagonal (Alg. 3)          */
    KRR_PIVOT_UNIFORM = 1,     /* a uniformly random k-subset of the columns   */
    KRR_PIVOT_GREEDY = 2       /* the largest residual diagonal entry          */
} krr_pivot_rule;

typedef struct krr_factor krr_factor;        /* RPCholesky factor F, pivots S */
typedef struct krill_precond krill_precond;  /* KRILL preconditioner          */

typedef struct {
    int iters;               /* PCG iterations (max over columns; for the
                                mixed path, summed over refinement steps)    */
    int outer_refinements;   /* float64 residual recomputations (mixed path)  */
    int rank;                /* factor rank used                              */
    int escalated;           /* mixed path: 1 if the float32 inner iterations
                                stalled (an inner solve ran into half the
                                iteration budget or refinement stopped
                                improving) and the solve finished with float64
                                CG vectors and float-float products           */
    double rel_residual;     /* max over columns of ||y - M x|| / ||y||,
                                recomputed in float64 after the solve         */
    double kernel_entries;   /* kernel entries kappa(x_i, x_j) evaluated      */
    double t_build_s;        /* preconditioner core build time (s)            */
    double t_solve_s;        /* PCG time (s)                                  */
    double kmv_ms;           /* summed device time of the float32 fused
                                product kernel (CUDA events on `stream`);
                                filled only while krr_set_profiling(1) is on  */
    int kmv_launches;        /* number of float32 fused-product launches      */
    int kmv64_launches;      /* number of float64 fused-product launches      */
    double kmv64_ms;         /* summed device time of the float64 product     */
    double kmvff_ms;         /* summed device time of the float-float product */
    int kmvff_launches;      /* number of float-float fused-product launches  */
    int graph_replays;       /* CUDA-graph replays of PCG iteration chunks
                                (see krr_set_pcg_graphs)                      */
    int host_checks;         /* convergence flags read back by the host       */
} krr_info;

/* ------------------------------------------------------------------------ */
/* Fused matrix-free product (Alg. 1 "Product"):                             */
/*   Y = (A + lambda I) V,  A_ij = kappa(x_i, x_j), never stored.            */
/* precision KRR_PREC_FP64 evaluates in float64 with direct differences;     */
/* KRR_PREC_MIXED evaluates kernel tiles in float32 (distances from row      */
/* norms of centred points) and accumulates in float32 -- for the Gaussian   */
/* and Matern kernels by default with the inner products on the tensor cores */
/* (see krr_set_product_path), prepared once per call (synchronises stream);  */
/* KRR_PREC_FLOAT_FLOAT evaluates entries and sums in float-float arithmetic */
/* (error-free transformations on the float32 pipes, ~2^-46 per entry).     */
/* V, Y: N x m column-major float64.  Y may not alias V.                     */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_kmatvec(const double *X, int64_t N, int d, krr_kernel kern,
                       double sigma, double lambda, const double *V, int m,
                       double *Y, krr_precision prec, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched fused product over several hyperparameter settings sharing one     */
/* tile generation (the paper applies its solvers across bandwidths and      */
/* regularisations, Sec. 2.1.2, Sec. 2.2.2, Sec. 5; batching them is this   */
/* library's design):                                                         */
/*   Y_{s,c} = (A_s + lambda_{s,c} I) V_{s,c},  s < S, c < ms,                */
/* A_s the kernel matrix of (kerns[s], sigmas[s]).  V, Y: N x (S ms)          */
/* column-major, column s*ms + c; lambdas: S*ms.  Per point pair the          */
/* coordinate differences are formed once (l2 and/or l1 distance), then each  */
/* setting costs one kernel evaluation.  float32 tiles, float32 accumulation. */
/* 1 <= S <= KRR_MAX_SETTINGS, ms in {1, 2}.                                  */
/* ------------------------------------------------------------------------ */
#define KRR_MAX_SETTINGS 8
KRR_API krr_status krr_kmatvec_batched(const double *X, int64_t N, int d, int S,
                                       const int *kerns, const double *sigmas, int ms,
                                       const double *lambdas, const double *V, double *Y,
                                       void *stream);

/* ------------------------------------------------------------------------ */
/* Prediction at test points (Sec. 2.1: f(x) = sum_i alpha_i K(x_i, x)):      */
/*   out (Nt x m) = K(Xtest, Xtrain) alpha,  alpha N x m.                     */
/* Xtrain N x d and Xtest Nt x d row-major.  KRR_PREC_FP64 evaluates entries  */
/* in float64; KRR_PREC_MIXED in float32 tiles with float32 accumulation     */
/* (both point sets centred on the training mean).                           */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_predict(const double *Xtrain, int64_t N, int d, krr_kernel kern,
                               double sigma, const double *alpha, int m,
                               const double *Xtest, int64_t Nt, double *out,
                               krr_precision prec, void *stream);

/* ------------------------------------------------------------------------ */
/* Pivot sampling of Alg. 3: ndraw i.i.d. indices with probability           */
/* proportional to the residual diagonal dres (length N).  Weights are the    */
/* fixed-point integers floor(min(dres_i, 1) * 2^F) for dres_i > dfloor and   */
/* 0 otherwise, F = 62 - ceil(log2 N); draw j of block t uses word 0 of       */
/* Philox4x64-10 with counter (t, j, 0, 0) and key (seed,                     */
/* 0x5250434850495653), target = floor(u W / 2^64), and picks the smallest i  */
/* whose inclusive prefix sum exceeds the target.  Writes ndraw indices to    */
/* `draws` and sets *ndraw_out = ndraw, or *ndraw_out = 0 (and no draws) when */
/* every weight is zero.  0 < ndraw <= 1024; dres entries must be <= 1 in     */
/* meaning (larger values count as 1).                                        */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_rpc_sample(const double *dres, int64_t N, double dfloor,
                                  uint64_t seed, uint64_t t, int ndraw, int64_t *draws,
                                  int *ndraw_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Blocked RPCholesky (Alg. 3) with block size `block` (0 = Alg. 1's rule     */
/* min(100, ceil(k/10))), rank k <= min(N, 4096), block <= 128.  Each block   */
/* draws min(block, k - i) pivots (krr_rpc_sample with t = block counter and  */
/* dfloor = the drop threshold N * 2^-52 * max_i A_ii),                       */
/* keeps the first occurrence of each, forms G = A(:,S') - F F(S',:)^T,       */
/* factors G(S',S') pivot by pivot dropping any candidate whose Schur value   */
/* is <= N * 2^-52 * max_i A_ii, appends G R^{-1} to F and subtracts its      */
/* squared row norms from the residual diagonal; every candidate of a block   */
/* gets residual 0.  Stops early (rank < k) if every weight becomes zero.     */
/* All arithmetic is float64.  *F_out receives a new handle (free with        */
/* krr_factor_free).                                                          */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_rpcholesky(const double *X, int64_t N, int d, krr_kernel kern,
                          double sigma, int k, int block, uint64_t seed,
                          void *stream, krr_factor **F_out);

/* ------------------------------------------------------------------------ */
/* The partial Cholesky factorization of krr_rpcholesky with another pivot    */
/* rule (Sec. 4, the comparison strategies): the blocks, the Schur update,    */
/* the drop rule and the handle are the same; only the pivots of each block   */
/* differ.                                                                    */
/*   KRR_PIVOT_RPCHOLESKY: krr_rpcholesky itself.                             */
/*   KRR_PIVOT_UNIFORM: the k pivots are a uniformly random k-subset of the   */
/*     N columns drawn before the first block, independently of A: draw       */
/*     q = 0, 1, ... takes word 0 of Philox4x64-10 with counter (q, 0, 1, 0)  */
/*     and key (seed, 0x5250434850495653) as floor(u N / 2^64), keeping first */
/*     occurrences; blocks take them in that order.  A pivot the factor       */
/*     already spans is dropped and still counts, so the rank can be < k.     */
/*   KRR_PIVOT_GREEDY: each block takes the `block` largest residual diagonal */
/*     entries above the drop threshold, in descending order (ties: smaller   */
/*     index); block 0 means 1, one pivot at a time, which is the paper's     */
/*     greedy rule (Cholesky with complete diagonal pivoting); larger blocks  */
/*     are a blocked variant.                                                 */
/* block 0 otherwise means min(100, ceil(k/10)).  Arguments and errors as     */
/* krr_rpcholesky, plus KRR_EINVAL for an unknown rule.                       */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_pivoted_cholesky(const double *X, int64_t N, int d, krr_kernel kern,
                                        double sigma, int k, int block, uint64_t seed,
                                        krr_pivot_rule rule, void *stream,
                                        krr_factor **F_out);

/* Rank reached, number of blocks drawn and N of a factor. */
KRR_API krr_status krr_factor_info(const krr_factor *F, int64_t *N, int *rank,
                           int *nblocks);

/* Copy a factor out: F_out N x rank column-major float64, pivots int64[rank]
 * in column order, dres float64[N] (the final residual diagonal).  Any output
 * pointer may be NULL to skip it. */
KRR_API krr_status krr_factor_export(const krr_factor *F, double *F_out, int64_t *pivots,
                             double *dres);

KRR_API void krr_factor_free(krr_factor *F);

/* ------------------------------------------------------------------------ */
/* Preconditioner of Alg. 1 in Woodbury form (identical in exact arithmetic   */
/* to the paper's SVD form):                                                  */
/*   Z = P^{-1} R,  P = F F^T + lambda I,                                    */
/*   P^{-1} = lambda^{-1} (I - F (lambda I + F^T F)^{-1} F^T).               */
/* The k x k core lambda I + F^T F is factored in float64 (KRR_ECHOL if it is */
/* not numerically positive definite) and cached in the factor per (mu,       */
/* precision).  KRR_PREC_MIXED streams F in float32.  R, Z: N x m.           */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_precond_apply(const krr_factor *F, double mu, const double *R,
                             int m, double *Z, krr_precision prec, void *stream);

/* ------------------------------------------------------------------------ */
/* RPCholesky-preconditioned CG (Alg. 1; PCG as in Sec. 3: zero initial      */
/* iterate, each column stops when its recursive relative residual            */
/* ||r|| / ||y|| <= tol).                                                     */
/*   KRR_PREC_FP64 : float64 throughout.                                      */
/*   KRR_PREC_MIXED: iterative refinement -- an outer float64 loop x += d,    */
/*     r = y - (A + lambda I) x recomputed with the float-float product       */
/*     (KRR_PREC_FLOAT_FLOAT of krr_kmatvec, float64-accurate), around        */
/*     an inner float32 PCG (float32 kernel tiles, float64 CG scalars) that   */
/*     solves (A + lambda I) d = r to a loose tolerance; stops when the       */
/*     float64 relative residual is <= tol.                                   */
/*   KRR_PREC_FLOAT_FLOAT: float64 PCG as KRR_PREC_FP64 with the float-float  */
/*     product in place of the float64 one: the same iterates up to rounding  */
/*     (entries within about 2^-46), at the float32 pipes' speed.             */
/* F may be NULL (no preconditioner beyond lambda^{-1} I).  maxit bounds the  */
/* PCG iterations per column (<= 0 selects 1000).  Y, alpha_out: N x m.       */
/* info (optional) receives iteration counts, the float64 residual and times. */
/* Returns KRR_ENOCONV (with the best iterate in alpha_out) if the tolerance  */
/* was not reached.                                                           */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_pcg_solve(const double *X, int64_t N, int d, krr_kernel kern,
                         double sigma, const double *Y, int m, double mu,
                         const krr_factor *F, double tol, int maxit,
                         krr_precision prec, double *alpha_out, void *stream,
                         krr_info *info);

/* ------------------------------------------------------------------------ */
/* Batched RPCholesky-preconditioned CG over S hyperparameter settings x ms   */
/* regularisations (mixed precision with float64-accurate refinement, as     */
/* krr_pcg_solve with KRR_PREC_MIXED).  System q*ms + c solves                */
/*   (A_q + mus[c] N I) alpha = Y(:, q*ms + c),                               */
/* A_q the kernel matrix of (kerns[q], sigmas[q]), preconditioned by the      */
/* Alg. 1 preconditioner of factors[q] and mus[c] (factors or factors[q] may  */
/* be NULL: lambda^{-1} I).  All systems advance together: one batched fused  */
/* product (krr_kmatvec_batched) per iteration; each column keeps its own CG  */
/* scalars and stops at its own tolerance.  Y, alpha_out: N x (S ms).        */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_pcg_solve_batched(const double *X, int64_t N, int d, int S,
                                         const int *kerns, const double *sigmas,
                                         const krr_factor *const *factors, int ms,
                                         const double *mus, const double *Y, double tol,
                                         int maxit, double *alpha_out, void *stream,
                                         krr_info *info);

/* ------------------------------------------------------------------------ */
/* Sparse sign embedding of Alg. 2 (Sec. 2.2.1): Phi is s x N; column n has   */
/* zeta distinct rows, entries +-zeta^{-1/2}.  Rows of column n are drawn from */
/* Philox4x64-10 words (counter (n, q, 0, 0), key (seed, 0x53534531524f5753), */
/* q = 0, 1, ..., words 0..3 in order) as floor(u s / 2^64), rejecting        */
/* repeats; the sign of the t-th kept row is bit t of word 0 of counter       */
/* (n, 0, 0, 0), key (seed, 0x535345325349474e), bit 1 meaning negative.      */
/* rows: int32 N x zeta, vals: float64 N x zeta (row-major, acceptance order).*/
/* 1 <= zeta <= min(s, 64).                                                   */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_sparse_sign(int64_t N, int s, int zeta, uint64_t seed,
                           int32_t *rows, double *vals, void *stream);

/* ------------------------------------------------------------------------ */
/* KRILL build (Alg. 2):                                                      */
/*   H = lambda A(S,S) + N 2^-52 tr(A(S,S)) I,  Phi = SparseSign(s, N, zeta), */
/*   B = Phi A(:,S),  P = B^T B + H,  C = Cholesky(P) (float64).              */
/* centers: int64[k], distinct, in [0, N) (the paper samples them uniformly). */
/* sketch_rows s (0 = 2k), zeta (0 = ceil(ln(k+1))).  The handle keeps a      */
/* device copy of X and the centers.  k <= 8192.                              */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krill_build(const double *X, int64_t N, int d, krr_kernel kern,
                       double sigma, const int64_t *centers, int k, double mu,
                       int sketch_rows, int zeta, uint64_t seed, void *stream,
                       krill_precond **P_out);

/* Copy KRILL intermediates out (any pointer may be NULL): H, P and the upper
 * Cholesky factor C (P = C^T C) as k x k column-major float64, and the sketch
 * B as s x k column-major float64; *s_out receives s. */
KRR_API krr_status krill_export(const krill_precond *P, double *H, double *Bsk,
                        double *Pm, double *Cu, int *s_out);

/* ------------------------------------------------------------------------ */
/* KRILL PCG (Alg. 2): solves [A(S,:)A(:,S) + H] beta = A(S,:) y with the     */
/* preconditioner beta -> C^{-1}(C^{-T} beta).  Iterative refinement: the     */
/* right-hand side and each outer residual use float64 kernel entries; the    */
/* inner PCG (float64 k-vectors and CG scalars) regenerates the N x k block   */
/* A(:,S) in float32 for its products.  Stops when the float64 relative       */
/* residual is <= tol.  Y: N x m, beta_out: k x m.                            */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krill_solve(const krill_precond *P, const double *Y, int m,
                       double tol, int maxit, double *beta_out, void *stream,
                       krr_info *info);

KRR_API void krill_free(krill_precond *P);

/* ------------------------------------------------------------------------ */
/* Allocation-free float64 fused product (the paper has no counterpart: this  */
/* entry point exists for callers that cannot allocate device memory on their */
/* call path -- e.g. a serving loop that reserved all its memory up front and */
/* must not let a request trigger cudaMalloc, or a plug-in that only receives */
/* buffers from a framework that owns all device memory).                    */
/*   Y = (A + lambda I) V, the same product as krr_kmatvec with               */
/*   KRR_PREC_FP64, computed with no allocation of any kind.                  */
/* X (N x d), V and Y (N x m, column-major) must be device pointers on the    */
/* current device; host pointers are rejected with KRR_EINVAL (staging them   */
/* would allocate).  The split partial sums live in one 16 MiB static device  */
/* array owned by the library (held by every GPU that uses it until the       */
/* process exits), so N x padded(m) must be <= 2^21, padded(m) being m        */
/* rounded up to 1, 2, 4, 8 or 16; larger sizes return KRR_EINVAL with a      */
/* message.  With CUDA's lazy module loading the array is created on a device */
/* when the library's device code is first loaded there -- at the latest by   */
/* the first call of this entry point on that device, which looks up the      */
/* array's address and caches it.  That first call can therefore allocate     */
/* (and fail with KRR_ENOMEM on a full device): make it at set-up time, and   */
/* before any stream capture.  Every call shares the one array and overwrites */
/* the partial sums it reads (nothing needs to start at zero), so calls that  */
/* overlap on the GPU race: serialise them (one stream, or events).  Returns  */
/* after the stream is synchronised.                                          */
/* ------------------------------------------------------------------------ */
KRR_API krr_status krr_kmatvec_f64_noalloc(const double *X, int64_t N, int d,
                                           krr_kernel kern, double sigma, double lambda,
                                           const double *V, int m, double *Y, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving engine: continuous batching of Alg. 1 solves (the paper solves one */
/* problem at a time; this is the serving layer around the same method).     */
/*                                                                            */
/* A request is one mixed-precision krr_pcg_solve with its own RPCholesky     */
/* factor: (A + mu N I) alpha = Y for points X (N x d, row-major float64),    */
/* kernel kern with bandwidth sigma, Y with m columns (m x N, column c at     */
/* Y + c N), RPCholesky rank k (Alg. 3, block min(100, ceil(k/10)), seed),    */
/* tolerance tol on the float64-accurate relative residual of every column    */
/* and at most maxit inner PCG iterations over all refinements.               */
/*                                                                            */
/* Requests wait in a queue and are admitted in arrival order while a slot is */
/* free and the sum of the admitted requests' estimated footprints           */
/* (krr_server_footprint) stays within the server's HBM budget.  Builder      */
/* threads, each with its own stream, copy X and Y to the device and build the*/
/* factor, the Woodbury core and the prepared points; the solve then keeps    */
/* them and its CG state resident.  Iterating requests step in two lanes     */
/* that advance independently: a fast lane for requests whose float32 product */
/* costs at most 4e10 flop per iteration (N^2 (2 d' + 2 m' + 5), d' and m'   */
/* the padded sizes) and a bulk lane for the rest.  A step of a lane advances */
/* each of its requests by iters_per_step inner PCG iterations with one       */
/* grouped launch per phase for all of them (replayed as one CUDA graph when  */
/* use_graph is set), while inner-solve starts, float-float refinement        */
/* residuals and result copies run on per-slot streams.  A result does not    */
/* depend on which other requests are being served: every per-request work    */
/* decomposition and sum order is fixed by that request alone.                */
/*                                                                            */
/* Ownership: X, Y and alpha_out (m x N float64, host or device memory) stay  */
/* owned by the caller and must stay valid until the request is reported by   */
/* krr_server_poll (or the server is destroyed, which abandons unfinished     */
/* requests).  alpha_out is written once, when the request finishes.  Device */
/* arrays must hold their data when submitted: the server reads them later   */
/* on its own streams, without waiting on the caller's.                       */
/* Threading: one host thread at a time may call a server's functions.        */
/* ------------------------------------------------------------------------ */
#define KRR_SERVE_MAX_SLOTS 64
#define KRR_SERVE_MAX_BUILDERS 8

typedef struct krr_server krr_server;

typedef struct {
  int max_slots;            /* concurrent requests, 1..KRR_SERVE_MAX_SLOTS    */
  int iters_per_step;       /* inner PCG iterations per step, 1..64           */
  int use_graph;            /* replay each step as one CUDA graph launch      */
  int build_threads;        /* builder threads (own streams), 0..8; 0: 4      */
  double hbm_budget_bytes;  /* admission budget; 0: 90% of the free HBM at    */
                            /* creation                                       */
} krr_server_config;

typedef struct {
  int64_t id;               /* from krr_server_submit                         */
  krr_status status;        /* KRR_OK, KRR_ENOCONV, KRR_EBREAKDOWN, or the    */
                            /* error of a failed build (KRR_ENOMEM, ...)      */
  int iters;                /* inner PCG iterations over all refinements      */
  int outer_refinements;
  int rank;                 /* RPCholesky rank                                */
  int m;
  int escalated;            /* 1: the float32 inner iterations stalled and    */
                            /* the solve finished with float64 CG vectors and */
                            /* float-float products                           */
  int reserved;
  double rel_residual;      /* worst column's relative residual, float64-     */
                            /* accurate product                               */
  double kernel_entries;    /* kernel entries evaluated by this request       */
  double t_submit, t_admit, t_built, t_done;   /* seconds on krr_server_clock */
  char error[160];          /* message of a failed build ("" otherwise)       */
} krr_request_result;

typedef struct {
  int64_t submitted, completed, queued, admitted;   /* request counts         */
  int64_t steps;            /* steps launched                                 */
  int64_t step_kernels;     /* kernels those steps launched                   */
  int max_concurrent;       /* most requests iterating in one step            */
  int reserved;
  double reserved_bytes;    /* footprint of the admitted requests             */
  double peak_reserved_bytes;
  double budget_bytes;
  double kernel_entries;    /* over the completed requests                    */
  double step_ms;           /* device time of the steps (CUDA events)         */
  double build_s;           /* builder-thread wall time spent on builds       */
  double escalate_s;        /* worker wall time spent on escalated solves     */
  int64_t escalations;      /* requests handed to the float-float continuation */
  /* device ms per kernel of the step, summed over steps, recorded only while */
  /* krr_set_profiling is on and use_graph is 0: product, reduce, alpha,      */
  /* update, resid, F^T r, its reduction, W t, W^T u, z, beta, direction      */
  double phase_ms[12];
} krr_server_stats;

/* Estimated peak device bytes of one request (host-only; no GPU needed).     */
KRR_API krr_status krr_server_footprint(int64_t N, int d, int m, int k, double *bytes);

/* Creates a server on the current device (streams, builder threads, the     */
/* device tables).  KRR_EINVAL for a config outside the documented ranges.    */
KRR_API krr_status krr_server_create(const krr_server_config *cfg, krr_server **out);

/* Queues a request (see above); returns at once.  N <= 2^26, 1 <= d <= 32,   */
/* 1 <= m <= 16, 0 <= k <= min(N, 4096), 0 < tol < 1, maxit >= 1.            */
/* KRR_ENOMEM (not queued) when the request alone exceeds the budget.         */
KRR_API krr_status krr_server_submit(krr_server *S, const double *X, int64_t N, int d,
                                     krr_kernel kern, double sigma, const double *Y, int m,
                                     double mu, int k, uint64_t seed, double tol, int maxit,
                                     double *alpha_out, int64_t *id_out);

/* Admits what fits, takes finished builds and slot events, launches a step  */
/* in every idle lane that has iterating requests, and returns when a lane's  */
/* step has completed (at once when nothing is in flight).                    */
/* *unfinished (optional): queued plus admitted requests not yet reported.    */
KRR_API krr_status krr_server_step(krr_server *S, int64_t *unfinished);

/* Copies up to max_results finished requests (each reported once).           */
KRR_API krr_status krr_server_poll(krr_server *S, krr_request_result *out, int max_results,
                                   int *n_out);

KRR_API krr_status krr_server_get_stats(const krr_server *S, krr_server_stats *out);

/* Seconds since the server was created (the clock of the result times).      */
KRR_API double krr_server_clock(const krr_server *S);

/* ------------------------------------------------------------------------ */
/* Eviction and checkpoint/resume of served requests (the paper has no        */
/* counterpart; a server uses it to free HBM for other work, and a caller to  */
/* move a solve between servers or processes).                                */
/* A running request is evicted at its next refinement boundary: when its     */
/* float64 residual is known and another inner PCG solve would start, alpha   */
/* and the residual move to host memory, its device memory and budget are     */
/* released, and it is parked.  A queued request is parked at once.  A        */
/* request that meets the tolerance (or is handed to the float-float          */
/* continuation) before a boundary finishes instead.  A parked request is     */
/* resumed at the head of the queue (krr_server_resume) or exported as a      */
/* checkpoint (krr_server_export) and then leaves this server.  On resume or  */
/* import its factor, core and points are rebuilt (the build is               */
/* deterministic for a fixed seed) and the refinement continues from the      */
/* saved state, so the result is bit-identical to an uninterrupted solve.     */
/* ------------------------------------------------------------------------ */
typedef enum {
    KRR_REQ_QUEUED = 0, KRR_REQ_BUILDING = 1, KRR_REQ_ITERATING = 2,
    KRR_REQ_ESCALATED = 3, KRR_REQ_FINISHING = 4, KRR_REQ_PARKED = 5, KRR_REQ_DONE = 6
} krr_request_state;

typedef struct {
    int64_t id;
    int state;                /* krr_request_state                              */
    int iters;                /* inner PCG iterations so far                    */
    int outer_refinements;    /* float64 residuals computed so far              */
    int reserved;
    double rel_residual;      /* worst column, after the last refinement        */
} krr_request_progress;

/* Progress of a request that is queued, running, parked, or finished and not */
/* yet returned by krr_server_poll; KRR_EINVAL for other ids.                 */
KRR_API krr_status krr_server_progress(const krr_server *S, int64_t id,
                                       krr_request_progress *out);

/* Marks a queued or running request for eviction (see above).                */
KRR_API krr_status krr_server_evict(krr_server *S, int64_t id);

/* Puts a parked request back at the head of the admission queue.             */
KRR_API krr_status krr_server_resume(krr_server *S, int64_t id);

/* Checkpoint of a parked request.  buf NULL: *size receives the bytes needed */
/* (a header, 2 m norms and, once started, alpha and the float64 residual,    */
/* 2 N m doubles).  Otherwise writes it into buf (*size bytes available,      */
/* KRR_EINVAL if too small) and removes the request from this server: it is   */
/* not reported by krr_server_poll, and its caller buffers are released.      */
KRR_API krr_status krr_server_export(krr_server *S, int64_t id, void *buf, size_t *size);

/* Queues a request from a checkpoint (checked for its magic, version, sizes  */
/* and shapes; KRR_EINVAL otherwise) with the caller's X and Y -- the same    */
/* data the checkpointed request was submitted with -- and a new output       */
/* buffer; ownership and admission as krr_server_submit.                      */
KRR_API krr_status krr_server_import(krr_server *S, const void *buf, size_t size,
                                     const double *X, const double *Y, double *alpha_out,
                                     int64_t *id_out);

/* Waits for the device, stops the builders and frees everything.             */
KRR_API void krr_server_destroy(krr_server *S);

/* Autotuning of the float32 fused product (not in the paper).  While on     */
/* (non-zero), the first float32 product of each (path, kernel, d rounded up  */
/* to 4 -- or to 16 on the tensor path --, m rounded up to 1/2/4/8/16, N)     */
/* times candidate column tiles -- the split counts that make the grid 2, 4,  */
/* 8, 16 and 32 waves of the path's CTAs per SM --                            */
/* once on the caller's stream (it synchronises that stream; a stream that is */
/* being captured is not tuned) and keeps the fastest for the process.  Off   */
/* (the default): 8 waves.  The split count sets the summation order, so a    */
/* tuned product can differ from an untuned one at the rounding level; with   */
/* a fixed choice, results are reproducible.                                  */
KRR_API void krr_set_autotune(int on);

/* CUDA-graph replay of the PCG iterations (engineering, not in the paper).  */
/* While on (non-zero, the default) every PCG run of krr_pcg_solve,          */
/* krr_pcg_solve_batched and krill_solve takes its first iteration one       */
/* launch at a time, then captures chunks of 16, 4 and 1 whole iterations    */
/* (preconditioner, PCG scalars and vectors, fused product) as CUDA graphs   */
/* on a private stream and replays them on the caller's stream, reading the  */
/* per-column convergence flags back once per replay (one host read per      */
/* iteration when off).  Chunk lengths follow the residual's observed rate;  */
/* iterations a replay runs after every column converged change nothing      */
/* (converged columns freeze on the device) and are counted in the kernel    */
/* entries.  Results are identical with and without graphs.  An operator    */
/* that cannot be captured falls back to launch-at-a-time stepping.          */
KRR_API void krr_set_pcg_graphs(int on);

/* Split count chosen by the autotuner for a float32 product shape, or 0 if   */
/* that shape has not been tuned (for the path krr_set_product_path selects). */
KRR_API krr_status krr_autotune_choice(krr_kernel kern, int d, int m, int64_t N,
                                       int *splits);

/* Path of the float32 fused product (the product of Alg. 1 inside the mixed  */
/* solve, and krr_kmatvec with KRR_PREC_MIXED) for the Gaussian and Matern    */
/* kernels (Sec. 2.1: both are functions of |x_i - x_j|^2):                   */
/*   KRR_PRODUCT_TENSOR (0, default): the inner products x_i . x_j on the     */
/*     fifth-generation tensor cores (tcgen05.mma into Tensor Memory, operands */
/*     staged by TMA) from a two-half split of each centred, scaled           */
/*     coordinate (x = h + l, |x - h - l| <= 2^-22 |x|; fp16 MMAs with float32 */
/*     accumulation, c_i + c_j folded in as three fp16 pieces), kernel values */
/*     and sums over V in float32.  Points whose centred, scaled coordinates  */
/*     exceed 16384 in magnitude (or |x|^2 / 2 exceeds 32768), and the        */
/*     Laplace kernel, take the FMA path.                                     */
/*   KRR_PRODUCT_FMA (1): every entry on the float32 FMA pipe.                */
/*   KRR_PRODUCT_MMA_SYNC (2): the same split on the register-operand         */
/*     mma.sync tensor path (kept for comparison).                            */
/* All paths meet the float32 error bound of krr_kmatvec; their results       */
/* differ at the rounding level.  Process-wide; not thread-safe with solves   */
/* in flight.  KRR_EINVAL for another value.                                  */
typedef enum {
  KRR_PRODUCT_TENSOR = 0,
  KRR_PRODUCT_FMA = 1,
  KRR_PRODUCT_MMA_SYNC = 2
} krr_product_path;
KRR_API krr_status krr_set_product_path(int path);

/* Epilogue variant of the tcgen05 product (KRR_PRODUCT_TENSOR): 0 (default)  */
/* = chosen per shape by the autotuner while krr_set_autotune is on (every    */
/* valid variant timed once on the caller's stream at the first product of    */
/* the shape), else variant 3 (9 for 5..8 right-hand sides per launch of a    */
/* square product).  Variants 1..7 sum over the right-hand sides with FFMA2   */
/* on the FMA pipe: 1 = 8 epilogue warps with the next columns' Tensor Memory */
/* loads in flight while the current ones are computed; 2 = 16 epilogue       */
/* warps; 3 = 8 warps without that overlap; 4 = 16 warps with it; 5 = 8       */
/* warps, software-pipelined by one batch of columns (the ex2 of one batch on */
/* the MUFU while the FFMA2 sums of the previous batch run); 6 = 12 epilogue  */
/* warps on 96-column tiles with the overlap; 7 = the same without.  Variants */
/* 8..11 take those sums on the tensor cores (mma.sync m16n8k16 on the kernel */
/* values, scaled by 2^14 and split into fp16 halves, times the right-hand    */
/* sides, scaled per column by a power of two and split likewise): 8 = 8      */
/* warps with the overlap, 9 = 8 warps without, 10 = 16 warps without, 11 =   */
/* 16 warps with.  Their error is 2^-22 of each term plus 2^-39 of the        */
/* column's largest |v| per term (the FMA variants: 2^-24 of each term), so   */
/* they serve square products (krr_kmatvec, the solvers) only; prediction and */
/* the restricted products keep 1..7.  Variants 2, 4..7, 10 and 11 serve m <= */
/* 4 per launch.  A forced variant that does not serve a launch leaves that   */
/* launch to the autotuner or the default.  Results differ between variants   */
/* at the rounding level only.  Process-wide.  KRR_EINVAL outside             */
/* 0..KRR_PRODUCT_VARIANTS.                                                   */
#define KRR_PRODUCT_VARIANTS 11
KRR_API krr_status krr_set_product_variant(int variant);

/* The autotuner's choice for the square tcgen05 product of a shape (kernel,  */
/* d, m, N): *variant (0 if the shape has not been tuned) and, when ms is not */
/* NULL, the measured launch time of each of the KRR_PRODUCT_VARIANTS         */
/* variants in milliseconds (ms[v - 1] for variant v; 0 for a variant that    */
/* was not timed).                                                            */
KRR_API krr_status krr_autotune_variant(krr_kernel kern, int d, int m, int64_t N, int *variant,
                                        float *ms);

/* Timing instrumentation: while on (non-zero), solves record CUDA events
 * around every fused-product launch on the caller's stream and report the
 * summed device time in krr_info.kmv_ms / kmv_launches. */
KRR_API void krr_set_profiling(int on);

/* Summed device time (ms) and number of the fused-product launches recorded  */
/* while profiling was on and not yet collected by a solve: which = 0 the     */
/* float32 product, 1 the float64 product, 2 the float-float product.  The    */
/* collected launches are forgotten.  Synchronises the recorded events.       */
/* KRR_EINVAL for another which or NULL outputs.                              */
KRR_API krr_status krr_profile_collect(int which, double *ms, int *launches);

/* Diagnostic of the device-side timeout path (engineering, not in the        */
/* paper).  Launches one thread that waits, with the bounded mbarrier wait of */
/* the tcgen05 product's roles, on a barrier that no arrival completes, for   */
/* budget_cycles SM clock cycles (0 .. 2^31; 1e6 is about half a             */
/* millisecond), then raises the device fault flag as a real timeout does.    */
/* Synchronises stream.  Returns KRR_ETIMEOUT once the wait gave up and the   */
/* flag was read and cleared -- the expected result; the context stays       */
/* usable -- and KRR_EINVAL for a budget out of range.                        */
KRR_API krr_status krr_check_bounded_wait(int64_t budget_cycles, void *stream);

/* Message for the last failure on the calling thread ("" if none). */
KRR_API const char *krr_last_error(void);

/* Library version string. */
KRR_API const char *krr_version(void);

/* Number of kernels this library has launched in the process so far. */
KRR_API uint64_t krr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* KRR_GB300_H */
