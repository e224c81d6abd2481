// Batched GEMM on CUDA cores (FP64 and FP32): TM x TN output tile per CTA of 256
// threads, 16-deep K slices staged in shared memory, (TM/16) x (TN/16) register
// tile per thread.  FP64 launches whose 64 x 64 grid would leave SMs idle take
// 32 x 32 or 16 x 16 tiles: on GB300 the FP64 pipe, not the shared-memory
// traffic of a small register tile, bounds every tile size, so smaller tiles
// cost little per flop and spread short launches over the whole GPU.  Every
// output element is accumulated by FMA over the same K order whatever the tile
// (the skipped K ranges hold exact zeros), so the tile size does not change the
// result.
#include "dense.cuh"
#include "internal.h"

namespace msp {

namespace {

constexpr int TK = 16;

template <class T, bool TRANS_A, bool TRANS_B, int TM, int TN>
__device__ __forceinline__ void gemm_tile(const GemmDescT<T>& D) {
    constexpr int RM = TM / 16, RN = TN / 16;
    const int tiles_m = (D.M + TM - 1) / TM;
    if (blockIdx.x >= tiles_m * ((D.N + TN - 1) / TN)) return;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    if (D.lower && tn * TN > tm * TM + TM - 1) return;   // tile strictly above the diagonal
    __shared__ T As[TK][TM + 1];
    __shared__ T Bs[TK][TN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads
    const int m0 = tm * TM, n0 = tn * TN;
    T acc[RM][RN] = {};
    int k_begin = D.b_lower ? (n0 / TK) * TK : 0;
    if (D.a_k_lo && m0 < D.M) k_begin = max(k_begin, (D.a_k_lo[m0] / TK) * TK);
    int k_end = D.a_lower ? min(D.K, m0 + TM) : D.K;
    if (D.b_upper) k_end = min(k_end, n0 + TN);
    for (int k0 = k_begin; k0 < k_end; k0 += TK) {
        // stage op(A)[m0 .. m0+TM-1][k0 .. k0+15], reading along the contiguous index
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            int mm, kk;
            if (TRANS_A) { kk = e % TK; mm = e / TK; }
            else { mm = e % TM; kk = e / TM; }
            const int gm = m0 + mm, gk = k0 + kk;
            T v = 0;
            if (gm < D.M && gk < D.K) v = TRANS_A ? D.A[(long long)gm * D.lda + gk] : D.A[(long long)gk * D.lda + gm];
            As[kk][mm] = v;
        }
        // stage op(B)[k0 .. k0+15][n0 .. n0+TN-1]
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
            T a[RM], b[RN];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < RN; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) {
            const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
            if (gm < D.M && gn < D.N) {
                T* c = D.C + (long long)gn * D.ldc + gm;
                *c = (D.beta == T(0)) ? D.alpha * acc[i][j] : D.alpha * acc[i][j] + D.beta * (*c);
            }
        }
}

template <class T, bool TRANS_A, bool TRANS_B, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_batched_kernel(const GemmDescT<T>* descs) {
    gemm_tile<T, TRANS_A, TRANS_B, TM, TN>(descs[blockIdx.z]);
}

// one GEMM whose descriptor travels as a kernel parameter (no device copy)
template <class T, bool TRANS_A, bool TRANS_B, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_one_kernel(const GemmDescT<T> D) {
    gemm_tile<T, TRANS_A, TRANS_B, TM, TN>(D);
}

long long tiles_of(int m, int n, int tm, int tn) { return (long long)((m + tm - 1) / tm) * ((n + tn - 1) / tn); }

struct TileShape {
    int tm, tn;
};

// Output tile: 64 x 64 unless an FP64 launch would then give fewer than three
// CTAs per SM, then the largest of 32 x 32 and 16 x 16 that does (16 x 16 if
// neither does); structured FP64 launches take at most 32 x 32.  A product
// written in place over A (N <= 64) needs every CTA to cover all of N, so it
// takes 16 x 64 where a smaller tile is wanted.
template <class T>
TileShape pick_tile(int max_m, int max_n, long long batch, unsigned flags) {
    if (sizeof(T) != sizeof(double)) return {64, 64};
    const long long want = 3LL * num_sms();
    const bool big = tiles_of(max_m, max_n, 64, 64) * batch >= want;
    if (flags & kGemmInPlace) return big ? TileShape{64, 64} : TileShape{16, 64};
    if (big) return (flags & kGemmStructured) ? TileShape{32, 32} : TileShape{64, 64};
    if (tiles_of(max_m, max_n, 32, 32) * batch >= want) return {32, 32};
    return {16, 16};
}

template <class T, bool TA, bool TB>
void launch_batched(const GemmDescT<T>* d, TileShape t, dim3 grid, cudaStream_t s) {
    if constexpr (sizeof(T) == sizeof(double)) {
        if (t.tm == 32) { gemm_batched_kernel<T, TA, TB, 32, 32><<<grid, 256, 0, s>>>(d); return; }
        if (t.tm == 16 && t.tn == 16) { gemm_batched_kernel<T, TA, TB, 16, 16><<<grid, 256, 0, s>>>(d); return; }
        if (t.tm == 16) { gemm_batched_kernel<T, TA, TB, 16, 64><<<grid, 256, 0, s>>>(d); return; }
    }
    gemm_batched_kernel<T, TA, TB, 64, 64><<<grid, 256, 0, s>>>(d);
}

template <class T, bool TA, bool TB>
void launch_one(const GemmDescT<T>& d, TileShape t, dim3 grid, cudaStream_t s) {
    if constexpr (sizeof(T) == sizeof(double)) {
        if (t.tm == 32) { gemm_one_kernel<T, TA, TB, 32, 32><<<grid, 256, 0, s>>>(d); return; }
        if (t.tm == 16 && t.tn == 16) { gemm_one_kernel<T, TA, TB, 16, 16><<<grid, 256, 0, s>>>(d); return; }
        if (t.tm == 16) { gemm_one_kernel<T, TA, TB, 16, 64><<<grid, 256, 0, s>>>(d); return; }
    }
    gemm_one_kernel<T, TA, TB, 64, 64><<<grid, 256, 0, s>>>(d);
}

}  // namespace

template <class T>
void gemm_batched(const GemmDescT<T>* descs_dev, int batch, int max_m, int max_n, bool transA, bool transB,
                  cudaStream_t s, unsigned flags) {
    if (batch <= 0 || max_m <= 0 || max_n <= 0) return;
    const TileShape tile = pick_tile<T>(max_m, max_n, batch, flags);
    const int tiles = (int)tiles_of(max_m, max_n, tile.tm, tile.tn);
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid(tiles, 1, nb);
        if (transA && transB) launch_batched<T, true, true>(descs_dev + b0, tile, grid, s);
        else if (transA) launch_batched<T, true, false>(descs_dev + b0, tile, grid, s);
        else if (transB) launch_batched<T, false, true>(descs_dev + b0, tile, grid, s);
        else launch_batched<T, false, false>(descs_dev + b0, tile, grid, s);
        count_launches(1);
    }
}

template <class T>
void gemm_one(const GemmDescT<T>& d, bool transA, bool transB, cudaStream_t s) {
    if (d.M <= 0 || d.N <= 0) return;
    const bool structured = d.lower || d.b_lower || d.a_lower || d.b_upper || d.a_k_lo;
    const TileShape tile =
        pick_tile<T>(d.M, d.N, 1, (d.C == d.A ? kGemmInPlace : 0u) | (structured ? kGemmStructured : 0u));
    const dim3 grid((unsigned)tiles_of(d.M, d.N, tile.tm, tile.tn));
    if (transA && transB) launch_one<T, true, true>(d, tile, grid, s);
    else if (transA) launch_one<T, true, false>(d, tile, grid, s);
    else if (transB) launch_one<T, false, true>(d, tile, grid, s);
    else launch_one<T, false, false>(d, tile, grid, s);
    count_launches(1);
}

template void gemm_one<float>(const GemmDescT<float>&, bool, bool, cudaStream_t);
template void gemm_one<double>(const GemmDescT<double>&, bool, bool, cudaStream_t);
template void gemm_batched<double>(const GemmDescT<double>*, int, int, int, bool, bool, cudaStream_t, unsigned);
template void gemm_batched<float>(const GemmDescT<float>*, int, int, int, bool, bool, cudaStream_t, unsigned);

}  // namespace msp
