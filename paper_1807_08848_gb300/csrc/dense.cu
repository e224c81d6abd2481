// Batched GEMM on CUDA cores (FP64 and FP32): 64x64 output tile per CTA, 16-deep
// K slices staged in shared memory, 4x4 register tile per thread.
#include "dense.cuh"
#include "internal.h"

namespace msp {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <class T, bool TRANS_A, bool TRANS_B>
__device__ __forceinline__ void gemm_tile(const GemmDescT<T>& D) {
    const int tiles_m = (D.M + TM - 1) / TM;
    if (blockIdx.x >= tiles_m * ((D.N + TN - 1) / TN)) return;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    if (D.lower && tn * TN > tm * TM + TM - 1) return;   // tile strictly above the diagonal
    __shared__ T As[TK][TM + 1];
    __shared__ T Bs[TK][TN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    const int m0 = tm * TM, n0 = tn * TN;
    T acc[4][4] = {};
    int k_begin = D.b_lower ? (n0 / TK) * TK : 0;
    if (D.a_k_lo && m0 < D.M) k_begin = max(k_begin, (D.a_k_lo[m0] / TK) * TK);
    int k_end = D.a_lower ? min(D.K, m0 + TM) : D.K;
    if (D.b_upper) k_end = min(k_end, n0 + TN);
    for (int k0 = k_begin; k0 < k_end; k0 += TK) {
        // stage op(A)[m0 .. m0+63][k0 .. k0+15], reading along the contiguous index
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            int mm, kk;
            if (TRANS_A) { kk = e % TK; mm = e / TK; }
            else { mm = e % TM; kk = e / TM; }
            const int gm = m0 + mm, gk = k0 + kk;
            T v = 0;
            if (gm < D.M && gk < D.K) v = TRANS_A ? D.A[(long long)gm * D.lda + gk] : D.A[(long long)gk * D.lda + gm];
            As[kk][mm] = v;
        }
        // stage op(B)[k0 .. k0+15][n0 .. n0+63]
        for (int e = threadIdx.x; e < TN * TK; e += 256) {
            int kk, nn;
            if (TRANS_B) { nn = e % TN; kk = e / TN; }
            else { kk = e % TK; nn = e / TK; }
            const int gk = k0 + kk, gn = n0 + nn;
            T v = 0;
            if (gk < D.K && gn < D.N) v = TRANS_B ? D.B[(long long)gk * D.ldb + gn] : D.B[(long long)gn * D.ldb + gk];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
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
            if (gm < D.M && gn < D.N) {
                T* c = D.C + (long long)gn * D.ldc + gm;
                *c = (D.beta == T(0)) ? D.alpha * acc[i][j] : D.alpha * acc[i][j] + D.beta * (*c);
            }
        }
}

template <class T, bool TRANS_A, bool TRANS_B>
__global__ void __launch_bounds__(256) gemm_batched_kernel(const GemmDescT<T>* descs) {
    gemm_tile<T, TRANS_A, TRANS_B>(descs[blockIdx.z]);
}

// one GEMM whose descriptor travels as a kernel parameter (no device copy)
template <class T, bool TRANS_A, bool TRANS_B>
__global__ void __launch_bounds__(256) gemm_one_kernel(const GemmDescT<T> D) {
    gemm_tile<T, TRANS_A, TRANS_B>(D);
}

template <class T, bool TA, bool TB>
void launch(const GemmDescT<T>* d, int nb, dim3 grid, cudaStream_t s) {
    gemm_batched_kernel<T, TA, TB><<<grid, 256, 0, s>>>(d);
}

}  // namespace

template <class T>
void gemm_batched(const GemmDescT<T>* descs_dev, int batch, int max_m, int max_n, bool transA, bool transB,
                  cudaStream_t s) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return;
    const int tiles = ((max_m + TM - 1) / TM) * ((max_n + TN - 1) / TN);
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid(tiles, 1, nb);
        if (transA && transB) launch<T, true, true>(descs_dev + b0, nb, grid, s);
        else if (transA) launch<T, true, false>(descs_dev + b0, nb, grid, s);
        else if (transB) launch<T, false, true>(descs_dev + b0, nb, grid, s);
        else launch<T, false, false>(descs_dev + b0, nb, grid, s);
        count_launches(1);
    }
}

template <class T>
void gemm_one(const GemmDescT<T>& d, bool transA, bool transB, cudaStream_t s) {
    if (d.M <= 0 || d.N <= 0) return;
    const dim3 grid(((d.M + TM - 1) / TM) * ((d.N + TN - 1) / TN));
    if (transA && transB) gemm_one_kernel<T, true, true><<<grid, 256, 0, s>>>(d);
    else if (transA) gemm_one_kernel<T, true, false><<<grid, 256, 0, s>>>(d);
    else if (transB) gemm_one_kernel<T, false, true><<<grid, 256, 0, s>>>(d);
    else gemm_one_kernel<T, false, false><<<grid, 256, 0, s>>>(d);
    count_launches(1);
}

template void gemm_one<float>(const GemmDescT<float>&, bool, bool, cudaStream_t);
template void gemm_one<double>(const GemmDescT<double>&, bool, bool, cudaStream_t);
template void gemm_batched<double>(const GemmDescT<double>*, int, int, int, bool, bool, cudaStream_t);
template void gemm_batched<float>(const GemmDescT<float>*, int, int, int, bool, bool, cudaStream_t);

}  // namespace msp
