// Batched small dense linear algebra used by the basis extraction and the online
// factorisation: per-matrix descriptors, one launch per batch.
#pragma once

#include <cuda_runtime.h>

namespace msp {

// C (M x N) = alpha op(A) op(B) + beta C, column-major; op(X) = X or X^T.
// op(A) is M x K, op(B) is K x N.  With beta == 0, C is not read.
// lower != 0: only output tiles that reach the diagonal or below it are computed
// (symmetric updates whose upper triangle is never read); the others keep C.
// b_lower != 0: op(B) is lower triangular (op(B)[k][j] = 0 for k < j), so the
// K loop of an output tile starting at column j0 begins at j0.
// a_lower != 0: op(A) is lower triangular (op(A)[i][k] = 0 for k > i), so the K
// loop of an output tile ending at row i1 stops after i1.
// a_k_lo (device, per row of op(A), nondecreasing): op(A)[i][k] = 0 for
// k < a_k_lo[i], so the K loop of an output tile starting at row i0 begins there.
template <class T>
struct GemmDescT {
    const T* A;
    const T* B;
    T* C;
    int M, N, K;
    int lda, ldb, ldc;
    T alpha, beta;
    int lower = 0;
    int b_lower = 0;
    int a_lower = 0;
    const int* a_k_lo = nullptr;
    int b_upper = 0;   // op(B) upper triangular (op(B)[k][j] = 0 for k > j): K stops after the tile's last column
};
using GemmDesc = GemmDescT<double>;

// Launch flags of gemm_batched.
//   kGemmInPlace: C aliases A (allowed only with N <= 64): every CTA then covers
//     all of N, so each output tile reads its rows of A before writing them.
//   kGemmStructured: the descriptors use lower / b_lower / a_lower / b_upper /
//     a_k_lo; FP64 launches then take tiles of at most 32 x 32, whose finer
//     skipping of zero blocks saves more work than the smaller tile costs.
enum : unsigned { kGemmInPlace = 1u, kGemmStructured = 2u };

// Launch a batched GEMM over descriptors in device memory.  max_m, max_n bound
// the batch's M and N (grid size).
template <class T>
void gemm_batched(const GemmDescT<T>* descs_dev, int batch, int max_m, int max_n, bool transA, bool transB,
                  cudaStream_t s, unsigned flags = 0);

// One GEMM, descriptor passed by value (no device-side descriptor array); both
// flags are read off the descriptor.
template <class T>
void gemm_one(const GemmDescT<T>& d, bool transA, bool transB, cudaStream_t s);

// Backwards-compatible FP64 entry (op(B) = B).
inline void gemm_batched(const GemmDesc* descs_dev, int batch, int max_m, int max_n, bool transA, cudaStream_t s,
                         unsigned flags = 0) {
    gemm_batched<double>(descs_dev, batch, max_m, max_n, transA, false, s, flags);
}

}  // namespace msp
