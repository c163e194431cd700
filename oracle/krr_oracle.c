/*
 * krr_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * A plain, slow, double-precision CPU statement of what the GPU path computes,
 * following "Robust, randomized preconditioning for kernel ridge regression"
 * (Diaz, Epperly, Frangella, Tropp, Webber).  It is used only by the tests,
 * by the package smoke check and by the benchmark's CPU-baseline leg.  It
 * shares no code, header, table or constant generator with the CUDA library.
 *
 * Everything is straight loops in the order the paper states the steps.  The
 * only parallelism is an OpenMP loop over independent output rows or columns,
 * each of which is summed sequentially, so results do not depend on the
 * thread count.
 *
 * Conventions: X is N x d row-major; right-hand-side and factor blocks are
 * column-major (column c of an N x m block starts at c * N).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define ORC_GAUSSIAN 0
#define ORC_LAPLACE_L1 1
#define ORC_MATERN52 2

/* ------------------------------------------------------------------------ */
/* Kernel functions.                                                         */
/*  Gaussian: exp(-||x-y||^2 / (2 sigma^2))           (Sec. 2.1.2, squared   */
/*            exponential kernel)                                            */
/*  Laplace:  exp(-||x-y||_1 / sigma), l1 distance    (Sec. 5.1)             */
/*  Matern-5/2: (1 + q + q^2/3) exp(-q), q = sqrt(5) ||x-y||_2 / sigma       */
/*            (not in the paper; the textbook Matern form with nu = 5/2,     */
/*            sigma the length scale)                                        */
/* Distances are formed from direct coordinate differences.                  */
/* ------------------------------------------------------------------------ */
double orc_kappa(const double *a, const double *b, int d, int kern, double sigma)
{
    if (kern == ORC_LAPLACE_L1) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s += fabs(a[j] - b[j]);
        return exp(-s / sigma);
    }
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = a[j] - b[j];
        s += t * t;
    }
    if (kern == ORC_MATERN52) {
        double q = sqrt(5.0) * sqrt(s) / sigma;
        return (1.0 + q + q * q / 3.0) * exp(-q);
    }
    return exp(-s / (2.0 * sigma * sigma));
}

/* out (nr x nc, row-major) = A(rows, cols), A_ij = kappa(x_i, x_j).
 * rows / cols may be NULL, meaning 0..nr-1 / 0..nc-1. */
void orc_kernel_block(const double *X, int64_t N, int d, int kern, double sigma,
                      const int64_t *rows, int64_t nr, const int64_t *cols,
                      int64_t nc, double *out)
{
    (void)N;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < nr; ++a) {
        int64_t i = rows ? rows[a] : a;
        for (int64_t b = 0; b < nc; ++b) {
            int64_t j = cols ? cols[b] : b;
            out[a * nc + b] = orc_kappa(X + i * d, X + j * d, d, kern, sigma);
        }
    }
}

/* Matrix-free product of Alg. 1 ("Product"): Y = (A + lambda I) V for the
 * requested output rows.  V is N x m column-major; Y is nr x m column-major
 * (Y[c * nr + a] belongs to row rows[a]).  rows == NULL means all N rows. */
void orc_kmatvec(const double *X, int64_t N, int d, int kern, double sigma,
                 double lambda, const double *V, int m, const int64_t *rows,
                 int64_t nr, double *Y)
{
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < nr; ++a) {
            int64_t i = rows ? rows[a] : a;
            for (int c = 0; c < m; ++c) acc[c] = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                double kij = orc_kappa(X + i * d, X + j * d, d, kern, sigma);
                for (int c = 0; c < m; ++c) acc[c] += kij * V[c * N + j];
            }
            for (int c = 0; c < m; ++c) Y[c * nr + a] = acc[c] + lambda * V[c * N + i];
        }
        free(acc);
    }
}

/* Prediction (Sec. 2.1): out (Nt x m, col-major) = K(T, X) V, i.e.
 * out[c][t] = sum_n kappa(t_t, x_n) V[c][n], V N x m col-major. */
void orc_kcross_matvec(const double *X, int64_t N, const double *T, int64_t Nt, int d,
                       int kern, double sigma, const double *V, int m, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < Nt; ++t) {
        for (int c = 0; c < m; ++c) {
            double acc = 0.0;
            for (int64_t n = 0; n < N; ++n)
                acc += orc_kappa(T + t * d, X + n * d, d, kern, sigma) * V[c * N + n];
            out[c * Nt + t] = acc;
        }
    }
}

/* u (N x m, col-major) = A(:, S) beta, beta k x m col-major. */
void orc_kcols_matvec(const double *X, int64_t N, int d, int kern, double sigma,
                      const int64_t *S, int k, const double *beta, int m, double *u)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        for (int c = 0; c < m; ++c) u[c * N + n] = 0.0;
        for (int l = 0; l < k; ++l) {
            double v = orc_kappa(X + n * d, X + S[l] * d, d, kern, sigma);
            for (int c = 0; c < m; ++c) u[c * N + n] += v * beta[c * k + l];
        }
    }
}

/* out (k x m, col-major) = A(S, :) u, u N x m col-major. */
void orc_krows_matvec(const double *X, int64_t N, int d, int kern, double sigma,
                      const int64_t *S, int k, const double *u, int m, double *out)
{
#pragma omp parallel for schedule(static)
    for (int l = 0; l < k; ++l) {
        for (int c = 0; c < m; ++c) out[c * k + l] = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double v = orc_kappa(X + S[l] * d, X + n * d, d, kern, sigma);
            for (int c = 0; c < m; ++c) out[c * k + l] += v * u[c * N + n];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator, written from its published        */
/* definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC 2011): ten rounds of two 64x64->128 multiplies with the   */
/* Philox multipliers, xor with the key, and a Weyl-sequence key bump.       */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags that separate the random streams drawn from one seed. */
#define ORC_TAG_PIVOTS 0x5250434850495653ULL /* pivot draws of Alg. 3 */
#define ORC_TAG_EMBED_ROWS 0x53534531524f5753ULL /* sparse sign rows */
#define ORC_TAG_EMBED_SIGNS 0x535345325349474eULL /* sparse sign signs */

/* ------------------------------------------------------------------------ */
/* Pivot sampling of Alg. 3: i.i.d. draws s ~ d / Sum(d).                     */
/* Reading used for bit reproducibility: weights are the fixed-point values  */
/* w_i = floor(min(d_i, 1) * 2^F) for d_i > dfloor and 0 otherwise (dfloor  */
/* is the drop threshold below, so numerically zero residuals are never     */
/* drawn), F = 62 - ceil(log2 N), summed as                                 */
/* 64-bit integers; draw j of block t takes u = Philox(counter (t, j, 0, 0), */
/* key (seed, pivot tag)) word 0, target = floor(u * W / 2^64), and returns  */
/* the smallest i whose inclusive prefix sum exceeds target.  The diagonal    */
/* of every supported kernel is 1, so 0 <= d_i <= 1.                          */
/* Returns the number of draws written, 0 if every weight is zero.            */
/* ------------------------------------------------------------------------ */
static int ceil_log2_i64(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n) ++c;
    return c;
}

int orc_fixed_point_bits(int64_t N) { return 62 - ceil_log2_i64(N); }

uint64_t orc_fixed_point_weight(double dres, double dfloor, int fbits)
{
    double v = dres;
    if (!(v > 0.0) || !(v > dfloor)) return 0;   /* at or below the floor, or NaN */
    if (v > 1.0) v = 1.0;
    return (uint64_t)floor(ldexp(v, fbits));
}

int orc_rpc_sample(const double *dres, int64_t N, double dfloor, uint64_t seed,
                   uint64_t t, int ndraw, int64_t *draws)
{
    int fbits = orc_fixed_point_bits(N);
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t run = 0;
    for (int64_t i = 0; i < N; ++i) {
        run += orc_fixed_point_weight(dres[i], dfloor, fbits);
        W[i] = run;
    }
    if (run == 0) { free(W); return 0; }
    const uint64_t key[2] = {seed, ORC_TAG_PIVOTS};
    for (int j = 0; j < ndraw; ++j) {
        uint64_t ctr[4] = {t, (uint64_t)j, 0, 0}, out[4];
        orc_philox4x64(ctr, key, out);
        uint64_t target = (uint64_t)(((unsigned __int128)out[0] * run) >> 64);
        /* smallest i with W[i] > target, by bisection over the prefix sums */
        int64_t lo = 0, hi = N - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (W[mid] > target) hi = mid; else lo = mid + 1;
        }
        draws[j] = lo;
    }
    free(W);
    return ndraw;
}

/* ------------------------------------------------------------------------ */
/* The two pivot rules the paper compares RPCholesky with (Sec. 4, "Failure  */
/* of uniform sampling" / "Failure of greedy selection").                    */
/* Uniform: the k pivots are a uniformly random k-subset of the N columns,   */
/* drawn independently of A.  Reading: draw q = 0, 1, ... takes word 0 of     */
/* Philox(counter (q, 0, 1, 0), key (seed, pivot tag)) as the index           */
/* floor(u * N / 2^64), keeping first occurrences until k distinct indices   */
/* are found; the pivots enter the blocked Cholesky in that order, so a     */
/* column the factor already spans is dropped and still counts as a pivot.   */
/* Writes min(k, N) indices.                                                 */
/* ------------------------------------------------------------------------ */
int orc_uniform_pivots(int64_t N, int k, uint64_t seed, int64_t *S)
{
    if ((int64_t)k > N) k = (int)N;
    unsigned char *seen = (unsigned char *)calloc((size_t)N, 1);
    const uint64_t key[2] = {seed, ORC_TAG_PIVOTS};
    int got = 0;
    for (uint64_t q = 0; got < k; ++q) {
        uint64_t ctr[4] = {q, 0, 1, 0}, out[4];
        orc_philox4x64(ctr, key, out);
        int64_t i = (int64_t)(((unsigned __int128)out[0] * (uint64_t)N) >> 64);
        if (seen[i]) continue;
        seen[i] = 1;
        S[got++] = i;
    }
    free(seen);
    return got;
}

/* Greedy: each pivot is the largest entry of the residual diagonal after    */
/* the previous steps (ties: the smallest index).  With a block of b > 1 the */
/* b largest entries of the block's residual diagonal are taken (in          */
/* descending order), a blocked variant; b = 1 is the paper's rule.          */
/* Returns the number of picks (fewer than npick if fewer are eligible).     */
int orc_greedy_pick(const double *dres, int64_t N, double dfloor, int npick, int64_t *picks)
{
    int got = 0;
    for (int j = 0; j < npick; ++j) {
        int64_t best = -1;
        for (int64_t i = 0; i < N; ++i) {
            if (!(dres[i] > 0.0 && dres[i] > dfloor)) continue;
            int taken = 0;
            for (int q = 0; q < got; ++q) if (picks[q] == i) { taken = 1; break; }
            if (taken) continue;
            if (best < 0 || dres[i] > dres[best]) best = i;
        }
        if (best < 0) break;
        picks[got++] = best;
    }
    return got;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3, blocked RPCholesky.                                               */
/*   F <- 0, S <- {}, d <- diag(A), i <- 0                                    */
/*   while i < k:                                                            */
/*     draw min(B, k - i) i.i.d. pivots ~ d / Sum(d); S' <- Unique (first-   */
/*     occurrence order)                                                      */
/*     G <- A(:, S') - F(:, 1:i) F(S', 1:i)^T                                 */
/*     R <- Cholesky(G(S', :)),  G(S', :) = R^T R                            */
/*     F(:, i+1 : i+|S'|) <- G R^{-1}                                         */
/*     d <- d - SquaredRowNorms(new columns);  i <- i + |S'|                  */
/* Reading for a numerically singular G(S', S') (the paper is silent): the   */
/* Cholesky runs pivot by pivot in S' order; a candidate whose Schur value   */
/* is <= N * eps * max_i A_ii is dropped from S' (not resampled).  The scale */
/* is the initial diagonal, so a block whose candidates all have rounding-   */
/* level residuals cannot pass the test.  The same threshold is the floor    */
/* below which residuals carry no sampling weight.                           */
/* Every candidate drawn in a block, kept or dropped, gets d = 0 exactly.    */
/* F is N x k column-major and must be zeroed by the caller; S receives the  */
/* kept pivots in column order; dres receives the final residual diagonal.   */
/* trace_hist (optional, >= k + N + 1 entries) receives Sum(d) before the    */
/* first block and after every block.                                        */
/* Returns the rank reached (< k only if every weight became zero).           */
/* ------------------------------------------------------------------------ */
/* rule selects the pivots of each block: 0 RPCholesky (the sampler above),  */
/* 1 uniform (the next B of orc_uniform_pivots; the loop ends when all k are */
/* used, whatever the rank), 2 greedy (orc_greedy_pick); the rest of the     */
/* block is the same for every rule.                                         */
int orc_pivoted_cholesky(const double *X, int64_t N, int d, int kern, double sigma,
                         int k, int B, uint64_t seed, int rule, double *F, int64_t *S,
                         double *dres, int64_t *nblocks_out, double *trace_hist)
{
    double maxdiag = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        dres[n] = orc_kappa(X + n * d, X + n * d, d, kern, sigma);
        if (dres[n] > maxdiag) maxdiag = dres[n];
    }
    if (trace_hist) {
        double tr = 0.0;
        for (int64_t n = 0; n < N; ++n) tr += dres[n];
        trace_hist[0] = tr;
    }

    int64_t *draws = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int *acc = (int *)malloc(sizeof(int) * (size_t)B);
    double *G = (double *)malloc(sizeof(double) * (size_t)N * (size_t)B);
    double *R = (double *)malloc(sizeof(double) * (size_t)B * (size_t)B);
    double *Fn = (double *)malloc(sizeof(double) * (size_t)N * (size_t)B);

    const double thr = (double)N * DBL_EPSILON * maxdiag;
    int64_t *upiv = NULL;
    int nupiv = 0, used = 0;
    if (rule == 1) {
        upiv = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        nupiv = orc_uniform_pivots(N, k, seed, upiv);
    }
    int rank = 0;
    uint64_t t = 0;
    while (rule == 1 ? used < nupiv : rank < k) {
        int nd, got;
        if (rule == 1) {
            nd = (nupiv - used < B) ? (nupiv - used) : B;
            memcpy(draws, upiv + used, sizeof(int64_t) * (size_t)nd);
            used += nd;
            got = nd;
        } else {
            nd = (k - rank < B) ? (k - rank) : B;
            if (rule == 2) got = orc_greedy_pick(dres, N, thr, nd, draws);
            else got = orc_rpc_sample(dres, N, thr, seed, t, nd, draws);
        }
        ++t;
        if (got == 0) break;
        nd = got;

        /* Unique, first-occurrence order */
        int nc = 0;
        for (int j = 0; j < nd; ++j) {
            int seen = 0;
            for (int c = 0; c < nc; ++c) if (cand[c] == draws[j]) { seen = 1; break; }
            if (!seen) cand[nc++] = draws[j];
        }

        /* G = A(:, S') - F(:, 1:i) F(S', 1:i)^T, N x nc column-major */
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            for (int c = 0; c < nc; ++c) {
                double g = orc_kappa(X + n * d, X + cand[c] * d, d, kern, sigma);
                for (int l = 0; l < rank; ++l) g -= F[(int64_t)l * N + n] * F[(int64_t)l * N + cand[c]];
                G[(int64_t)c * N + n] = g;
            }
        }

        /* R = Cholesky(G(S', S')), upper triangular, with the drop rule */
        memset(R, 0, sizeof(double) * (size_t)B * (size_t)B);
        int na = 0;
        for (int c = 0; c < nc; ++c) {
            /* off-diagonal entries R[a, c] for the kept candidates a < c */
            for (int ia = 0; ia < na; ++ia) {
                int a = acc[ia];
                double v = G[(int64_t)c * N + cand[a]];
                for (int ib = 0; ib < ia; ++ib) {
                    int b = acc[ib];
                    v -= R[b * B + a] * R[b * B + c];
                }
                R[a * B + c] = v / R[a * B + a];
            }
            double p = G[(int64_t)c * N + cand[c]];
            for (int ia = 0; ia < na; ++ia) {
                int a = acc[ia];
                p -= R[a * B + c] * R[a * B + c];
            }
            if (!(p > thr)) continue;            /* dropped */
            R[c * B + c] = sqrt(p);
            acc[na++] = c;
        }

        /* new columns G(:, kept) R^{-1}, by forward substitution per row */
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            for (int ia = 0; ia < na; ++ia) {
                int a = acc[ia];
                double v = G[(int64_t)a * N + n];
                for (int ib = 0; ib < ia; ++ib) {
                    int b = acc[ib];
                    v -= Fn[(int64_t)ib * N + n] * R[b * B + a];
                }
                Fn[(int64_t)ia * N + n] = v / R[a * B + a];
            }
        }
        for (int ia = 0; ia < na; ++ia) {
            memcpy(F + (int64_t)(rank + ia) * N, Fn + (int64_t)ia * N, sizeof(double) * (size_t)N);
            S[rank + ia] = cand[acc[ia]];
        }
        /* residual diagonal: d <- d - SquaredRowNorms(new columns) */
        for (int64_t n = 0; n < N; ++n) {
            double s2 = 0.0;
            for (int ia = 0; ia < na; ++ia) s2 += Fn[(int64_t)ia * N + n] * Fn[(int64_t)ia * N + n];
            dres[n] -= s2;
        }
        for (int c = 0; c < nc; ++c) dres[cand[c]] = 0.0;
        rank += na;
        if (trace_hist) {
            double tr = 0.0;
            for (int64_t n = 0; n < N; ++n) tr += dres[n];
            trace_hist[t] = tr;
        }
    }
    if (nblocks_out) *nblocks_out = (int64_t)t;
    free(draws); free(cand); free(acc); free(G); free(R); free(Fn); free(upiv);
    return rank;
}

int orc_rpcholesky(const double *X, int64_t N, int d, int kern, double sigma,
                   int k, int B, uint64_t seed, double *F, int64_t *S,
                   double *dres, int64_t *nblocks_out, double *trace_hist)
{
    return orc_pivoted_cholesky(X, N, d, kern, sigma, k, B, seed, 0, F, S, dres,
                                nblocks_out, trace_hist);
}

/* ------------------------------------------------------------------------ */
/* Sparse sign embedding of Alg. 2 (Sec. 2.2.1): Phi is s x N; independently */
/* for each column, zeta distinct row indices uniformly without replacement, */
/* each entry an independent Rademacher sign times zeta^{-1/2}.              */
/* Reading for reproducibility: column n draws candidate rows from           */
/* Philox(counter (n, q, 0, 0), key (seed, row tag)), words 0..3 of q = 0,   */
/* 1, ... in order, row = floor(u * s / 2^64), rejecting repeats until zeta  */
/* rows are kept; the sign of the t-th kept row is bit t of word 0 of        */
/* Philox(counter (n, 0, 0, 0), key (seed, sign tag)), bit 1 meaning -1.      */
/* rows / vals are N x zeta row-major, in acceptance order.                  */
/* ------------------------------------------------------------------------ */
void orc_sparse_sign(int64_t N, int s, int zeta, uint64_t seed, int32_t *rows,
                     double *vals)
{
    const uint64_t krow[2] = {seed, ORC_TAG_EMBED_ROWS};
    const uint64_t ksgn[2] = {seed, ORC_TAG_EMBED_SIGNS};
    const double scale = 1.0 / sqrt((double)zeta);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        int32_t *r = rows + n * zeta;
        int kept = 0;
        for (uint64_t q = 0; kept < zeta; ++q) {
            uint64_t ctr[4] = {(uint64_t)n, q, 0, 0}, out[4];
            orc_philox4x64(ctr, krow, out);
            for (int w = 0; w < 4 && kept < zeta; ++w) {
                int32_t cand = (int32_t)(((unsigned __int128)out[w] * (uint64_t)s) >> 64);
                int dup = 0;
                for (int t = 0; t < kept; ++t) if (r[t] == cand) { dup = 1; break; }
                if (!dup) r[kept++] = cand;
            }
        }
        uint64_t ctr[4] = {(uint64_t)n, 0, 0, 0}, out[4];
        orc_philox4x64(ctr, ksgn, out);
        for (int t = 0; t < zeta; ++t)
            vals[n * zeta + t] = ((out[0] >> t) & 1ULL) ? -scale : scale;
    }
}

/* Sketch of Alg. 2: Bsk (s x k, row-major) = Phi A(:, S), accumulated over  */
/* data points n = 0..N-1 in order, one output column per thread.             */
void orc_krill_sketch(const double *X, int64_t N, int d, int kern, double sigma,
                      const int64_t *S, int k, const int32_t *rows,
                      const double *vals, int zeta, int s, double *Bsk)
{
    memset(Bsk, 0, sizeof(double) * (size_t)s * (size_t)k);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < k; ++c) {
        for (int64_t n = 0; n < N; ++n) {
            double a = orc_kappa(X + n * d, X + S[c] * d, d, kern, sigma);
            for (int t = 0; t < zeta; ++t)
                Bsk[(int64_t)rows[n * zeta + t] * k + c] += vals[n * zeta + t] * a;
        }
    }
}
