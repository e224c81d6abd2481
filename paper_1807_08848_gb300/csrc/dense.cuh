// Batched small dense linear algebra in FP64 used by the basis extraction and
// the online preconditioner: per-matrix descriptors, one launch per batch.
#pragma once

#include <cuda_runtime.h>

namespace msp {

// C (M x N) = op(A) (M x K) * B (K x N), column-major, op(A) = A or A^T.
struct GemmDesc {
    const double* A;
    const double* B;
    double* C;
    int M, N, K;
    int lda, ldb, ldc;
};

// Launch a batched GEMM.  transA selects op(A) = A^T.  max_m, max_n bound the
// batch's M and N (grid size).  Descriptors live in device memory.
void gemm_batched(const GemmDesc* descs_dev, int batch, int max_m, int max_n, bool transA, cudaStream_t s);

}  // namespace msp
