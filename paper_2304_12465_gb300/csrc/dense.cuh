// Dense building blocks (dense.cu): a strided SIMT GEMM, the blocked float64
// Cholesky factorisation and the blocked inverse of a lower-triangular factor.
#pragma once

#include "common.cuh"

namespace krr {

// C(MxN, column-major, ldc) = alpha * A(MxK) B(KxN) + beta * C, where element
// (i, k) of A is A[i*sai + k*sak] and element (k, j) of B is B[k*sbk + j*sbj].
// split_k > 1 sums K in slices through a workspace, in a fixed order.
template <typename T>
struct Gemm {
  int M = 0, N = 0, K = 0;
  T alpha = 1;
  const T *A = nullptr;
  int64_t sai = 0, sak = 0;
  const T *B = nullptr;
  int64_t sbk = 0, sbj = 0;
  T beta = 0;
  T *C = nullptr;
  int64_t ldc = 0;
};

template <typename T>
krr_status gemm(const Gemm<T> &g, cudaStream_t s, int split_k = 1);

// C -= A B (alpha = -1, beta = 1) for float64 data with float-float products
// and sums on the float32 pipes: about 2^-48 sqrt(K) times the largest
// partial sum per entry.
krr_status gemm_sub_ff(const Gemm<double> &g, cudaStream_t s);

// Lower triangle of C (r x r, column-major) = F^T F for F N x r column-major.
// float F: float32 products summed in float32 over 16-term chunks, the chunk
// sums in float-float (slices added in float64); double F: float64.  The
// strict upper triangle of C is untouched.
template <typename T>
krr_status gram_lower(const T *F, int64_t N, int r, double *C, cudaStream_t s);

// Picks a split-K count that fills the machine for a long, thin reduction.
int gemm_auto_split(int M, int N, int K);

// In-place lower Cholesky of the n x n column-major matrix A (lda): on return
// the lower triangle holds L with A = L L^T (the upper triangle is scratch).
// Returns KRR_ECHOL if a pivot is not positive (NaN included).
krr_status potrf_lower(double *A, int n, int64_t lda, cudaStream_t s);

// W (n x n, column-major) = L^{-1} for the lower-triangular L (lda); the upper
// triangle of W is zero.
krr_status trinv_lower(const double *L, int n, int64_t lda, double *W, cudaStream_t s);

// A(i, i) += v for i < n.
krr_status add_diagonal(double *A, int n, int64_t lda, double v, cudaStream_t s);

// B = A^T for n x n column-major matrices (no aliasing).
krr_status transpose_square(const double *A, int n, double *B, cudaStream_t s);

// Mirror the lower triangle into the upper one.
krr_status symmetrize_lower(double *A, int n, int64_t lda, cudaStream_t s);

}  // namespace krr
