// Batched FP64 GEMM: 64x64 output tile per CTA, 16-deep K slices staged in shared
// memory, 4x4 register tile per thread.
#include "dense.cuh"
#include "internal.h"

namespace msp {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <bool TRANS_A>
__global__ void __launch_bounds__(256) gemm_batched_kernel(const GemmDesc* descs) {
    const GemmDesc D = descs[blockIdx.z];
    const int tiles_m = (D.M + TM - 1) / TM;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    if (blockIdx.x >= tiles_m * ((D.N + TN - 1) / TN)) return;
    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    const int m0 = tm * TM, n0 = tn * TN;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < D.K; k0 += TK) {
        // stage A slice: op(A)[m0 .. m0+63][k0 .. k0+15]
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            int mm, kk;
            double v = 0.0;
            if (TRANS_A) {   // A^T(m, k) = A[k + m*lda]: read along k (contiguous)
                kk = e % TK; mm = e / TK;
                const int gm = m0 + mm, gk = k0 + kk;
                if (gm < D.M && gk < D.K) v = D.A[(long long)gm * D.lda + gk];
            } else {         // A(m, k) = A[m + k*lda]: read along m (contiguous)
                mm = e % TM; kk = e / TM;
                const int gm = m0 + mm, gk = k0 + kk;
                if (gm < D.M && gk < D.K) v = D.A[(long long)gk * D.lda + gm];
            }
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < TN * TK; e += 256) {
            const int kk = e % TK, nn = e / TK;
            const int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < D.K && gn < D.N) ? D.B[(long long)gn * D.ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
            if (gm < D.M && gn < D.N) D.C[(long long)gn * D.ldc + gm] = acc[i][j];
        }
}

}  // namespace

void gemm_batched(const GemmDesc* descs_dev, int batch, int max_m, int max_n, bool transA, cudaStream_t s) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return;
    const int tiles = ((max_m + TM - 1) / TM) * ((max_n + TN - 1) / TN);
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid(tiles, 1, nb);
        if (transA)
            gemm_batched_kernel<true><<<grid, 256, 0, s>>>(descs_dev + b0);
        else
            gemm_batched_kernel<false><<<grid, 256, 0, s>>>(descs_dev + b0);
        count_launches(1);
    }
}

}  // namespace msp
