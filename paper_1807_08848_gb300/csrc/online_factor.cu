// Preconditioner of the online least-squares iteration: a block-tridiagonal
// Cholesky factorisation of the normal matrix H = P~^T P~ (Eq.
// elliptic_cond_reduced), ordered by rows of patches.
//
// H couples a patch only with its eight neighbours, so with the unknowns of one
// row of patches as a block, H is block tridiagonal: diagonal blocks D_q and
// sub-diagonal blocks E_q = H_{q+1,q}.  The factor is computed on the patch-block
// scaled matrix Hs = R^{-T} H R^{-1} (R = blockdiag(R_m), H_mm = R_m^T R_m, so the
// diagonal patch blocks of Hs are identities):
//     L_q L_q^T = D_q - C_{q-1} C_{q-1}^T,   C_q = E_q L_q^{-T}
// with explicit inverses Li_q = L_q^{-1}; in FP32 when every pivot of that attempt is
// positive, else in FP64 (the large products on the tensor cores), repeated with a
// growing diagonal shift on a non-positive pivot.  Each D_q is factorised by 64-wide
// tiles (tile Cholesky, panel solve, trailing update) with a lookahead of one tile:
// the next tile column is updated first, the rest of the trailing update runs on a
// second stream while the next tile is factorised.  Applying
// M^{-1} = R^{-1} (L L^T)^{-1} R^{-T} is then a per-patch triangular product, a
// forward and a backward sweep, and a second per-patch product.  The FP64 CGLS
// iteration around it keeps the least-squares solution at FP64 accuracy.
#include "internal.h"

#include <mutex>

#include <array>
#include "dense.cuh"
#include "device_util.cuh"

#include <algorithm>
#include <utility>

namespace msp {

namespace {

constexpr int kTile = 64;

// ---- assembly of the FP64 blocks: one CTA per (m_a, m_b) patch pair
struct PairBlock {
    int ma, mb;          // patches (row unknowns from ma, column unknowns from mb)
    int list_begin, list_end;
    long long dst;       // first element of the (ma, mb) sub-block in its dense block
    int ld;              // leading dimension of that dense block
};

__global__ void assemble_kernel(const PairBlock* pb, const int* list_sa, const int* list_sb, const signed char* list_sg,
                                const int* k, const long long* e_off, const int* slot_off, const double* E,
                                double* dst_base) {
    // one warp per (column j, 128 rows): lanes own rows i, i + 32, i + 64, i + 96 and
    // accumulate them from one broadcast E_b value per list entry, in list order
    const PairBlock b = pb[blockIdx.x];
    const int ka = k[b.ma], kb = k[b.mb];
    const double* Ea = E + e_off[b.ma];
    const double* Eb = E + e_off[b.mb];
    const int ga = slot_off[b.ma], gb = slot_off[b.mb];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nib = (ka + 127) / 128;
    for (int task = threadIdx.x >> 5; task < kb * nib; task += nw) {
        const int j = task / nib, i0 = (task - j * nib) * 128 + lane;
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int t = b.list_begin; t < b.list_end; ++t) {
            const double* ea = Ea + (long long)(list_sa[t] - ga) * ka;
            double e = Eb[(long long)(list_sb[t] - gb) * kb + j];
            if (list_sg[t] < 0) e = -e;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + 32 * u < ka) a[u] = fma(ea[i0 + 32 * u], e, a[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + 32 * u < ka) dst_base[b.dst + (i0 + 32 * u) + (long long)j * b.ld] = a[u];
    }
}

// FP32 copy of one dense block of the scaled matrix, plus a shift on the diagonal
// of a diagonal block
template <class T>
__global__ void scale_convert_kernel(const double* src, T* dst, int nr, int nc, double shift, int diag) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nr * nc;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nr), j = (int)(t / nr);
        double v = src[t];
        if (diag && i == j) v += shift;
        dst[t] = (T)v;
    }
}

__global__ void round_kernel(const double* src, float* dst, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

// per-patch products with R_m^{-1} = F_m (upper, k x k column-major):
// y = F^T s (FP64 in, FP32 out) before the sweeps, z = F x (FP32 in, FP64 out) after
template <class T>
__global__ void patch_pre_kernel(const double* F, const long long* f_off, const int* k, const int* c_off,
                                 const double* s, T* y, int B) {
    const int m = blockIdx.x, km = k[m];
    const double* Fm = F + f_off[m];
    const double* sm = s + (long long)c_off[m] * B;
    T* ym = y + (long long)c_off[m] * B;
    for (int w = threadIdx.x; w < km * B; w += blockDim.x) {
        const int i = w / B, b = w - i * B;
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a += Fm[j + (long long)i * km] * sm[(long long)j * B + b];
        ym[w] = (T)a;
    }
}
template <class T>
__global__ void patch_post_kernel(const double* F, const long long* f_off, const int* k, const int* c_off,
                                  const T* x, double* z, int B) {
    const int m = blockIdx.x, km = k[m];
    const double* Fm = F + f_off[m];
    const T* xm = x + (long long)c_off[m] * B;
    double* zm = z + (long long)c_off[m] * B;
    for (int w = threadIdx.x; w < km * B; w += blockDim.x) {
        const int i = w / B, b = w - i * B;
        double a = 0.0;
        for (int j = i; j < km; ++j) a += Fm[i + (long long)j * km] * (double)xm[(long long)j * B + b];
        zm[w] = a;
    }
}

// Cholesky of one <= 64 x 64 diagonal tile in shared memory; writes L (lower,
// strict upper zeroed) in place.  One CTA of 256 threads on the factorisation's
// critical path, in the LDL^T form so that each column costs one barrier: at step
// k every thread (i, g) (row i = tid mod 64, g = tid / 64) updates
// L[i][j] -= (L[i][k] / d_k) L[j][k] for j = k+1+g, k+5+g, ... up to i, with the
// reciprocal 1 / d_k of the pivot taken in step k-1 by the thread that made the
// last update of L[k][k] (while the others finish theirs).  At the end the columns
// are scaled, L[i][j] / sqrt(d_j) below the diagonal and sqrt(d_j) on it.  A
// non-positive pivot sets *fail (and continues with d = 1).  The inverse of the
// factor is left to tile_inverse_kernel, off the critical path.
template <class T>
__device__ __forceinline__ T checked_pivot(T d, int* s_ok) {
    if (!(d > T(0)) || !isfinite(d)) {
        *s_ok = 0;
        return T(1);
    }
    return d;
}

template <class T>
__global__ void __launch_bounds__(256) potrf_tile_kernel(T* A, int lda, int nb, int* fail) {
    static_assert(kTile == 64, "thread layout assumes 64-wide tiles and 256 threads");
    __shared__ T L[kTile][kTile + 1];
    __shared__ T s_inv[2];
    __shared__ T s_sq[kTile];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        L[i][j] = (i >= j) ? A[i + (long long)j * lda] : T(0);
    }
    __syncthreads();
    if (tid == 0) {
        s_ok = 1;
        if (nb > 0) {
            const T d = checked_pivot(L[0][0], &s_ok);
            L[0][0] = d;
            s_inv[0] = T(1) / d;
        }
    }
    __syncthreads();
    const int ri = tid & (kTile - 1), g = tid >> 6;
    for (int k = 0; k < nb; ++k) {
        if (ri > k && ri < nb) {
            const T t = L[ri][k] * s_inv[k & 1];
            for (int j = k + 1 + g; j <= ri; j += 4) L[ri][j] = fma(-t, L[j][k], L[ri][j]);
            if (g == 0 && ri == k + 1) {   // L[k+1][k+1] is final: the next pivot
                const T d = checked_pivot(L[ri][ri], &s_ok);
                L[ri][ri] = d;
                s_inv[(k + 1) & 1] = T(1) / d;
            }
        }
        __syncthreads();
    }
    if (!s_ok && tid == 0) atomicExch(fail, 1);
    for (int j = tid; j < nb; j += blockDim.x) s_sq[j] = sqrt(L[j][j]);
    __syncthreads();
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        A[i + (long long)j * lda] = i > j ? L[i][j] / s_sq[j] : (i == j ? s_sq[j] : T(0));
    }
}

// Inverses of the factored diagonal tiles of one n x n block (one CTA per tile kt,
// rows/columns 64 kt ..): four lanes of a warp per column j of inv(L) run down its
// rows, each summing every fourth term of the forward substitution, combined by
// shuffles; column j is kept in the free strict upper part (inv(L)[i][j] at
// L[j][i + 1]); written to inv + kt 64^2 (ld 64, zero outside the tile).
template <class T>
__global__ void __launch_bounds__(256) tile_inverse_kernel(const T* D, int n, T* inv) {
    __shared__ T L[kTile][kTile + 1];
    __shared__ T rdiag[kTile];
    const int tid = threadIdx.x, r0 = blockIdx.x * kTile, nb = min(kTile, n - r0);
    const T* A = D + r0 + (long long)r0 * n;
    T* out = inv + (size_t)blockIdx.x * kTile * kTile;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        L[i][j] = (i >= j) ? A[i + (long long)j * n] : T(0);
    }
    __syncthreads();
    for (int i = tid; i < nb; i += blockDim.x) rdiag[i] = T(1) / L[i][i];
    __syncthreads();
    {
        const int j = tid >> 2, part = tid & 3;
        const bool col = j < nb;
        for (int i = (tid >> 5) * 8; i < nb; ++i) {   // warp-uniform rows: lanes with i < j add nothing
            T acc = T(0);
            if (col && i > j)
                for (int q = j + part; q < i; q += 4) acc = fma(L[i][q], L[j][q + 1], acc);
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (col && i >= j && part == 0) L[j][i + 1] = ((i == j ? T(1) : T(0)) - acc) * rdiag[i];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < kTile * kTile; e += blockDim.x) {
        const int i = e % kTile, j = e / kTile;
        out[i + j * kTile] = (i < nb && j < nb && i >= j) ? L[j][i + 1] : T(0);
    }
}

// Panel of the block Cholesky: P <- P L^{-T} for the m x nb panel P (ld ldp) under
// the factored diagonal tile L (nb x nb lower, ld ldl): every row x solves
// L x^T = p^T by column-oriented forward substitution, x_j = x_j / L[j][j], then
// x_l -= L[l][j] x_j for l > j.  One warp per row, lane l holding x_l and x_{l+32}
// in registers, x_j passed by one shuffle per column, so the chain of a column is
// one product, one shuffle and one FMA; eight rows per CTA share L in shared memory.
constexpr int kTrsmRows = 8;
template <class T>
__global__ void __launch_bounds__(32 * kTrsmRows) trsm_panel_kernel(const T* Lkk, int ldl, T* P, int ldp, int m,
                                                                  int nb) {
    __shared__ T L[kTile][kTile + 1];
    __shared__ T rd[kTile];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        L[i][j] = (i >= j) ? Lkk[i + (long long)j * ldl] : T(0);
    }
    __syncthreads();
    for (int i = tid; i < nb; i += blockDim.x) rd[i] = T(1) / L[i][i];
    __syncthreads();
    const int row = blockIdx.x * kTrsmRows + (tid >> 5);
    if (row >= m) return;   // warp-uniform; no barrier follows
    T* pr = P + row;
    const int l1 = lane + 32;
    T x0 = lane < nb ? pr[(long long)lane * ldp] : T(0);
    T x1 = l1 < nb ? pr[(long long)l1 * ldp] : T(0);
    for (int j = 0; j < nb; ++j) {
        T v = j < 32 ? x0 : x1;
        if (lane == (j & 31)) {
            v *= rd[j];
            if (j < 32) x0 = v;
            else x1 = v;
        }
        const T xj = __shfl_sync(0xffffffffu, v, j & 31);
        if (lane > j && lane < nb) x0 = fma(-L[lane][j], xj, x0);
        if (l1 > j && l1 < nb) x1 = fma(-L[l1][j], xj, x1);
    }
    if (lane < nb) pr[(long long)lane * ldp] = x0;
    if (l1 < nb) pr[(long long)l1 * ldp] = x1;
}

template <class T>
__global__ void zero_upper_kernel(T* A, int n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (i < j) A[t] = T(0);
    }
}

template <class T>
__global__ void copy_tile_kernel(const T* src, int lds, T* dst, int ldd, int nr, int nc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nr * nc;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nr), j = (int)(e / nr);
        dst[i + (long long)j * ldd] = src[i + (long long)j * lds];
    }
}

// Y[j][b] = alpha sum_k X[k][b] M[k + j ldm] + beta Y[j][b] for b < B: one warp per
// output column j reading column j of M contiguously; per (j, b) the sum runs in
// a fixed order, independent of B.
constexpr int kSbBatch = 8;
template <class T>
__global__ void sb_gemm_kernel(const T* X, const T* M, int ldm, T* Y, int K, int ncols, int B, T alpha, T beta) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ncols) return;
    const T* mj = M + (long long)j * ldm;
    for (int b0 = 0; b0 < B; b0 += kSbBatch) {
        T acc[kSbBatch];
#pragma unroll
        for (int t = 0; t < kSbBatch; ++t) acc[t] = T(0);
        for (int k = lane; k < K; k += 32) {
            const T m = mj[k];
            const T* xk = X + (long long)k * B + b0;
#pragma unroll
            for (int t = 0; t < kSbBatch; ++t)
                if (b0 + t < B) acc[t] = fma(m, xk[t], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < kSbBatch; ++t) {
            const T v = warp_sum(acc[t]);
            if (lane == 0 && b0 + t < B) {
                T* y = Y + (long long)j * B + b0 + t;
                *y = (beta == T(0)) ? alpha * v : alpha * v + beta * (*y);
            }
        }
    }
}

// Both triangular sweeps of the block-row factor in one persistent cooperative
// launch.  Each sweep is a chain of products Y = alpha X M + beta Y (X: [K][B]
// rows of the work vector, M: K x ncols column-major) whose steps depend on one
// another, so every product is spread over all warps of the grid (one output
// column per warp at a time, lanes along K) and a grid barrier separates the
// steps.  The barrier spins with a bound: on timeout it raises *err and every
// CTA leaves at its next barrier.
template <class T>
struct SweepArgs {
    int Qn, B;
    const int* off;            // [Qn + 1] element offsets of the blocks
    const long long* d_off;    // [Qn] offsets of L_q^{-1} (and its transpose)
    const long long* e_off;    // [Qn - 1] offsets of C_q (and its transpose)
    const T* LiT;
    const T* FT;
    const T* Li;
    const T* F;
    T* y;
    T* x;
    unsigned int* bar;         // [0] arrivals, [1] generation
    int* err;
    long long spin_limit;      // polls of the generation word before a CTA gives up
};

// Every thread of a CTA returns the same verdict: thread 0 reads the error word
// once and hands it to the others through shared memory (another CTA may raise
// the word at any moment, so per-thread reads could split the CTA).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned int& gen, int* err,
                                             long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int target = gen + 1;
        if (atomicAdd(&bar[0], 1u) == nblocks - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], target);
        } else {
            const volatile unsigned int* g = bar + 1;
            const volatile int* e = err;
            long long spins = 0;
            while (*g != target) {
                if (++spins > spin_limit || *e != 0) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = *((volatile int*)err) == 0;
    }
    ++gen;
    __syncthreads();
    return s_ok != 0;
}

// Y[j][b] = alpha sum_k M[k][j] X[k][b] + beta Y[j][b] for b < B, spread over the
// whole grid: one output column per warp and round, lanes along K.  The rows of X
// needed by a K chunk are staged in shared memory by every CTA (all CTAs run the
// same rounds and chunks, so the block barriers are uniform).
constexpr int kSweepKC = 1024;
template <class T, int BT>
__device__ __forceinline__ void sweep_product(const T* X, const T* M, int ldm, T* Y, int K, int ncols, int B, T alpha,
                                              T beta, int gw, int nw, int lane, T* xs) {
    for (int j0 = 0; j0 < ncols; j0 += nw) {
        const int j = j0 + gw;
        const bool live = j < ncols;
        const T* mj = M + (long long)(live ? j : 0) * ldm;
        for (int b0 = 0; b0 < B; b0 += BT) {
            const int bt = min(BT, B - b0);
            T acc[BT];
#pragma unroll
            for (int t = 0; t < BT; ++t) acc[t] = T(0);
            for (int kc = 0; kc < K; kc += kSweepKC) {
                const int kn = min(kSweepKC, K - kc);
                __syncthreads();
                for (int e = threadIdx.x; e < kn * bt; e += blockDim.x) {
                    const int kk = e / bt, t = e - kk * bt;
                    xs[t * kSweepKC + kk] = __ldcg(X + (long long)(kc + kk) * B + b0 + t);
                }
                __syncthreads();
                if (live) {
#pragma unroll 8
                    for (int kk = lane; kk < kn; kk += 32) {
                        const T m = mj[kc + kk];
#pragma unroll
                        for (int t = 0; t < BT; ++t) acc[t] = fma(m, xs[t * kSweepKC + kk], acc[t]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < BT; ++t) {
                const T v = warp_sum(acc[t]);
                if (live && lane == 0 && t < bt) {
                    T* yp = Y + (long long)j * B + b0 + t;
                    *yp = (beta == T(0)) ? alpha * v : alpha * v + beta * __ldcg(yp);
                }
            }
        }
    }
}

template <class T, int BT>
__global__ void __launch_bounds__(512) sweep_kernel(SweepArgs<T> A) {
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    T* xs = reinterpret_cast<T*>(sweep_smem);   // kSweepKC x BT
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    unsigned int gen = atomicAdd(&A.bar[1], 0u);
    const int B = A.B;
    // forward: y_q -= x_{q-1} C_{q-1}^T;  x_q = y_q Li_q^T
    for (int q = 0; q < A.Qn; ++q) {
        const int o = A.off[q], nq = A.off[q + 1] - o;
        if (nq == 0) continue;
        if (q > 0) {
            const int o0 = A.off[q - 1], n0 = o - o0;
            if (n0 > 0) {
                sweep_product<T, BT>(A.x + (long long)o0 * B, A.FT + A.e_off[q - 1], n0, A.y + (long long)o * B, n0, nq,
                                     B, T(-1), T(1), gw, nw, lane, xs);
                if (!grid_barrier(A.bar, gridDim.x, gen, A.err, A.spin_limit)) return;
            }
        }
        sweep_product<T, BT>(A.y + (long long)o * B, A.LiT + A.d_off[q], nq, A.x + (long long)o * B, nq, nq, B, T(1),
                             T(0), gw, nw, lane, xs);
        if (!grid_barrier(A.bar, gridDim.x, gen, A.err, A.spin_limit)) return;
    }
    // backward: x_q -= z_{q+1} C_q;  z_q = x_q Li_q   (z into y)
    for (int q = A.Qn - 1; q >= 0; --q) {
        const int o = A.off[q], nq = A.off[q + 1] - o;
        if (nq == 0) continue;
        if (q + 1 < A.Qn) {
            const int o1 = A.off[q + 1], n1 = A.off[q + 2] - o1;
            if (n1 > 0) {
                sweep_product<T, BT>(A.y + (long long)o1 * B, A.F + A.e_off[q], n1, A.x + (long long)o * B, n1, nq, B,
                                     T(-1), T(1), gw, nw, lane, xs);
                if (!grid_barrier(A.bar, gridDim.x, gen, A.err, A.spin_limit)) return;
            }
        }
        sweep_product<T, BT>(A.x + (long long)o * B, A.Li + A.d_off[q], nq, A.y + (long long)o * B, nq, nq, B, T(1), T(0),
                             gw, nw, lane, xs);
        if (!grid_barrier(A.bar, gridDim.x, gen, A.err, A.spin_limit)) return;
    }
}

// dst (nc x nr, col-major) = src^T (src nr x nc, col-major)
template <class T>
__global__ void transpose_kernel(const T* src, T* dst, int nr, int nc) {
    __shared__ T t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bx + threadIdx.x, j = by + y;
        if (i < nr && j < nc) t[y][threadIdx.x] = src[i + (long long)j * nr];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = by + threadIdx.x, i = bx + y;
        if (i < nr && j < nc) dst[j + (long long)i * nc] = t[threadIdx.x][y];
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

}  // namespace

// Block-tridiagonal Cholesky in precision T of the scaled matrix Hs64 (+ shift on
// the diagonal), with explicit inverses of the diagonal factors and transposed
// copies for the sweeps.  *fail_out = 1 on a non-positive pivot.
template <class T>
msp_status factorize(Basis& B, const double* Hs64p, long long total, double shift, int* fail_out, BtStore<T>& S,
                     bool early_exit, cudaStream_t s) {
    const int Qn = B.bt_q;
    struct { const double* p; } Hs64{Hs64p};
    MSP_TRY(S.F.alloc(std::max<long long>(total, 1), s));
    MSP_TRY(S.Li.alloc(std::max<long long>(B.bt_diag_elems, 1), s));
    int max_n = 0;
    for (int q = 0; q < Qn; ++q) max_n = std::max(max_n, B.bt_off[q + 1] - B.bt_off[q]);
    const int max_nt = (max_n + kTile - 1) / kTile;
    DevBuf<T> tinv, trow;
    DevBuf<int> fail;
    MSP_TRY(tinv.alloc((size_t)std::max(max_nt, 1) * kTile * kTile, s));
    MSP_TRY(trow.alloc((size_t)std::max(max_n, 1) * std::max(max_n, 1), s));
    MSP_TRY(fail.alloc(1, s));
    // temporary for C_q (E_q is read by every output tile of the product)
    long long max_e = 1;
    for (int q = 0; q + 1 < Qn; ++q)
        max_e = std::max<long long>(max_e, (long long)(B.bt_off[q + 2] - B.bt_off[q + 1]) * (B.bt_off[q + 1] - B.bt_off[q]));
    DevBuf<T> ctmp;
    MSP_TRY(ctmp.alloc((size_t)max_e, s));
    OzakiWork ozw;   // the large FP64 products on the tensor cores
    int hfail = 1;
    {
        MSP_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), s));
        MSP_CUDA(cudaMemsetAsync(S.Li.p, 0, sizeof(T) * std::max<long long>(B.bt_diag_elems, 1), s));
        // scaled copies in precision T
        for (int q = 0; q < Qn; ++q) {
            const int n = B.bt_off[q + 1] - B.bt_off[q];
            if (n == 0) continue;
            scale_convert_kernel<T><<<grid_for((long long)n * n), 256, 0, s>>>(Hs64.p + B.bt_d_off[q], S.F.p + B.bt_d_off[q],
                                                                             n, n, shift, 1);
            count_launches(1);
            if (q + 1 < Qn) {
                const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
                if (n1 == 0) continue;
                scale_convert_kernel<T><<<grid_for((long long)n1 * n), 256, 0, s>>>(Hs64.p + B.bt_e_off[q], S.F.p + B.bt_e_off[q],
                                                                                  n1, n, T(0), 0);
                count_launches(1);
            }
        }
        MSP_CUDA(cudaGetLastError());
        // Collect the whole factorisation's GEMMs in order, then launch them in order
        // with their descriptors resident in one device array.
        struct Step {
            int kind;        // 0 gemm, 1 potrf tile, 2 zero upper, 3 copy tile, 4 zero fill, 5 pivot check,
                             // 6 panel triangular solve, 7 inverses of the diagonal tiles, 8 join of
                             // the side stream into the main one
            int stream = 0;  // 0 the caller's stream, 1 the side stream of the trailing updates
            int wait_ev = -1, rec_ev = -1;   // event waited on before the step, recorded after it
            bool chain = false;  // a product on the chain of tile steps: CUDA cores (no slicing launches)
            GemmDescT<T> g;
            bool tA, tB;
            T* ptr;
            int ld, nb, nr, nc;
            T* inv;
            const T* src;
            int lds;
            int group;
        };
        std::vector<Step> steps;
        int group_id = 0;
        auto add_gemm = [&](const T* A, int lda, const T* Bm, int ldb, T* C, int ldc, int M, int N, int K,
                            T alpha, T beta, bool tA, bool tB, int lower = 0, int b_lower = 0, int group = 0,
                            int a_lower = 0, const int* a_k_lo = nullptr) {
            if (M <= 0 || N <= 0 || K <= 0) return;
            Step st{};
            st.kind = 0;
            st.group = group;
            st.g = GemmDescT<T>{A, Bm, C, M, N, K, lda, ldb, ldc, alpha, beta, lower, b_lower, a_lower, a_k_lo};
            st.tA = tA;
            st.tB = tB;
            steps.push_back(st);
        };
        for (int q = 0; q < Qn; ++q) {
            const int n = B.bt_off[q + 1] - B.bt_off[q];
            if (n == 0) continue;
            T* Dq = S.F.p + B.bt_d_off[q];
            T* Li = S.Li.p + B.bt_d_off[q];
            if (q > 0) {   // D_q -= C_{q-1} C_{q-1}^T
                const int n0 = B.bt_off[q] - B.bt_off[q - 1];
                const T* Cp = S.F.p + B.bt_e_off[q - 1];
                add_gemm(Cp, n, Cp, n, Dq, n, n, n, n0, T(-1), T(1), false, true, 1, 0, 0, 0,
                         B.d_bt_rowlo.p + B.bt_off[q]);
            }
            const int nt = (n + kTile - 1) / kTile;
            for (int kt = 0; kt < nt; ++kt) {
                const int r0 = kt * kTile, nb = std::min(kTile, n - r0), m = n - r0 - nb;
                Step st{};
                st.kind = 1;
                st.ptr = Dq + r0 + (long long)r0 * n;
                st.ld = n;
                st.nb = nb;
                steps.push_back(st);
                if (m > 0) {
                    T* panel = Dq + (r0 + nb) + (long long)r0 * n;
                    // panel <- panel L_kk^{-T} (in place: one column tile)
                    Step ts{};
                    ts.kind = 6;
                    ts.src = st.ptr;
                    ts.lds = n;
                    ts.ptr = panel;
                    ts.ld = n;
                    ts.nr = m;
                    ts.nb = nb;
                    steps.push_back(ts);
                    steps.back().rec_ev = 0;          // panel kt final
                    // trailing -= panel panel^T, with a lookahead of one tile: the next tile
                    // column first, on the caller's stream (after the previous rest, which
                    // also writes it), so that the next tile's factorisation and panel solve
                    // run while the rest of the update runs on the side stream
                    const int nb1 = std::min(kTile, m);
                    add_gemm(panel, n, panel, n, Dq + (r0 + nb) + (long long)(r0 + nb) * n, n, m, nb1, nb, T(-1), T(1),
                             false, true);
                    steps.back().wait_ev = 1;
                    steps.back().chain = true;
                    if (m > nb1) {
                        add_gemm(panel + nb1, n, panel + nb1, n, Dq + (r0 + nb + nb1) + (long long)(r0 + nb + nb1) * n, n,
                                 m - nb1, m - nb1, nb, T(-1), T(1), false, true, 1);
                        steps.back().stream = 1;
                        steps.back().wait_ev = 0;
                        steps.back().rec_ev = 1;
                    }
                }
            }
            Step jn{};   // the side stream's trailing updates end before the block's other steps
            jn.kind = 8;
            steps.push_back(jn);
            Step ti{};   // inverses of the diagonal tiles, off the chain of the tile factorisations
            ti.kind = 7;
            ti.ptr = Dq;
            ti.nb = n;
            ti.nr = nt;
            ti.inv = tinv.p;
            steps.push_back(ti);
            Step zu{};
            zu.kind = 2;
            zu.ptr = Dq;
            zu.nb = n;
            steps.push_back(zu);
            Step pc{};
            pc.kind = 5;
            steps.push_back(pc);
            // Li = L^{-1}: diagonal tiles from the tile inverses, then blocks of
            // doubling size, inv([A 0; B C]) = [inv(A) 0; -inv(C) B inv(A) inv(C)],
            // all pairs of one level in one batched launch per product.
            for (int it = 0; it < nt; ++it) {
                const int r0 = it * kTile, nb = std::min(kTile, n - r0);
                Step ct{};
                ct.kind = 3;
                ct.src = tinv.p + (size_t)it * kTile * kTile;
                ct.lds = kTile;
                ct.ptr = Li + r0 + (long long)r0 * n;
                ct.ld = n;
                ct.nr = nb;
                ct.nc = nb;
                steps.push_back(ct);
            }
            for (int w = 1; w < nt; w *= 2) {
                const int g1 = ++group_id, g2 = ++group_id;
                std::vector<std::array<int, 5>> prs;   // a0, a1 (= c0), c1, offset in the work buffer
                long long wo = 0;
                for (int t0 = 0; t0 + w < nt; t0 += 2 * w) {
                    const int a0 = t0 * kTile, a1 = std::min((t0 + w) * kTile, n), c1 = std::min((t0 + 2 * w) * kTile, n);
                    prs.push_back({a0, a1, c1, (int)wo, 0});
                    wo += (long long)(c1 - a1) * (a1 - a0);
                }
                for (auto& pr : prs) {   // Wk = L[C, A] inv(A)   (inv(A) lower triangular)
                    const int a0 = pr[0], a1 = pr[1], c1 = pr[2];
                    add_gemm(Dq + a1 + (long long)a0 * n, n, Li + a0 + (long long)a0 * n, n, trow.p + pr[3], c1 - a1, c1 - a1,
                             a1 - a0, a1 - a0, T(1), T(0), false, false, 0, 1, g1);
                }
                for (auto& pr : prs) {   // Li[C, A] = -inv(C) Wk   (inv(C) lower triangular)
                    const int a0 = pr[0], a1 = pr[1], c1 = pr[2];
                    add_gemm(Li + a1 + (long long)a1 * n, n, trow.p + pr[3], c1 - a1, Li + a1 + (long long)a0 * n, n, c1 - a1,
                             a1 - a0, c1 - a1, T(-1), T(0), false, false, 0, 0, g2, 1);
                }
            }
            if (q + 1 < Qn) {   // C_q = E_q Li^T
                const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
                T* Eq = S.F.p + B.bt_e_off[q];
                // C_q overwrites E_q: go through a temporary (E_q is read by every output
                // tile).  E_q couples a patch of row q+1 only with a contiguous range of
                // patches of row q (its neighbours), so each patch's rows of C_q take a
                // product over that range only; Li is lower triangular, so the columns
                // left of the range stay zero.
                Step z{};
                z.kind = 4;
                z.ptr = ctmp.p;
                z.nr = n1;
                z.nc = n;
                steps.push_back(z);
                const int egroup = ++group_id;
                for (int p = 0; p < B.mx; ++p) {
                    const int ma = (q + 1) * B.mx + p;
                    if (ma >= (int)B.bt_elo.size() || B.bt_elo[ma] < 0 || B.k[ma] == 0) continue;
                    const int r0 = B.c_off[ma] - B.bt_off[q + 1];
                    const int c0 = B.c_off[B.bt_elo[ma]] - B.bt_off[q];
                    const int c1 = B.c_off[B.bt_ehi[ma] + 1] - B.bt_off[q];
                    add_gemm(Eq + r0 + (long long)c0 * n1, n1, Li + c0 + (long long)c0 * n, n, ctmp.p + r0 + (long long)c0 * n1,
                             n1, B.k[ma], n - c0, c1 - c0, T(1), T(0), false, true, 0, 0, egroup);
                }
                Step cp{};
                cp.kind = 3;
                cp.src = ctmp.p;
                cp.lds = n1;
                cp.ptr = Eq;
                cp.ld = n1;
                cp.nr = n1;
                cp.nc = n;
                steps.push_back(cp);
            }
        }
        // descriptors of all GEMM steps in one device array
        std::vector<GemmDescT<T>> gds;
        for (auto& st : steps)
            if (st.kind == 0) gds.push_back(st.g);
        DevBuf<GemmDescT<T>> d_all;
        MSP_TRY(upload(d_all, gds, s));
        size_t gi = 0;
        // the tensor-core products of the side stream have their own workspace; declared
        // before the stream, so that on every way out the stream is synchronised first
        OzakiWork ozw_side;
        // side stream of the trailing updates and its events (panel final, rest of a
        // trailing update done, join), released on every way out
        struct SideStream {
            cudaStream_t st = nullptr;
            cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
            ~SideStream() {
                if (st) cudaStreamSynchronize(st);
                for (cudaEvent_t e : ev)
                    if (e) cudaEventDestroy(e);
                if (st) cudaStreamDestroy(st);
            }
        } side;
        MSP_CUDA(cudaStreamCreateWithFlags(&side.st, cudaStreamNonBlocking));
        for (cudaEvent_t& e : side.ev) MSP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (size_t si = 0; si < steps.size(); ++si) {
            const Step& st = steps[si];
            const cudaStream_t ss = st.stream ? side.st : s;
            if (st.wait_ev >= 0) MSP_CUDA(cudaStreamWaitEvent(ss, side.ev[st.wait_ev], 0));
            if (st.kind == 8) {
                MSP_CUDA(cudaEventRecord(side.ev[2], side.st));
                MSP_CUDA(cudaStreamWaitEvent(s, side.ev[2], 0));
                continue;
            }
            if (st.kind == 0) {
                // consecutive GEMMs of one group (independent outputs) go out as one batch
                size_t sj = si + 1;
                int mm = st.g.M, nn = st.g.N;
                while (st.group && sj < steps.size() && steps[sj].kind == 0 && steps[sj].group == st.group) {
                    mm = std::max(mm, steps[sj].g.M);
                    nn = std::max(nn, steps[sj].g.N);
                    ++sj;
                }
                const GemmDescT<T>& g0 = st.g;
                const bool structured = g0.lower || g0.b_lower || g0.a_lower || g0.b_upper || g0.a_k_lo;
                bool on_tc = false;
                if constexpr (sizeof(T) == sizeof(double)) {
                    // a group worth at least ~2^23 multiply-adds goes to the tensor cores
                    double work = 0.0;
                    for (size_t k = si; k < sj; ++k) work += (double)steps[k].g.M * steps[k].g.N * steps[k].g.K;
                    if (fp64_gemm_engine() == MSP_GEMM_TENSOR_CORES && work >= 8388608.0 && !st.chain) {
                        std::vector<GemmDesc> hg;
                        for (size_t k = si; k < sj; ++k) hg.push_back(steps[k].g);
                        if (ozaki_gemm_supported(hg)) {
                            MSP_TRY(ozaki_gemm_batched(hg, reinterpret_cast<const GemmDesc*>(d_all.p + gi), st.tA, st.tB,
                                                       ss, st.stream ? ozw_side : ozw));
                            on_tc = true;
                        }
                    }
                }
                if (!on_tc)
                    gemm_batched<T>(d_all.p + gi, (int)(sj - si), mm, nn, st.tA, st.tB, ss,
                                    (sj - si == 1 && g0.C == g0.A ? kGemmInPlace : 0u) | (structured ? kGemmStructured : 0u));
                gi += sj - si;
                si = sj - 1;
                if (steps[si].rec_ev >= 0) MSP_CUDA(cudaEventRecord(side.ev[steps[si].rec_ev], ss));
                continue;
            } else if (st.kind == 1) {
                potrf_tile_kernel<T><<<1, 256, 0, s>>>(st.ptr, st.ld, st.nb, fail.p);
                count_launches(1);
            } else if (st.kind == 6) {
                trsm_panel_kernel<T><<<(st.nr + kTrsmRows - 1) / kTrsmRows, 32 * kTrsmRows, 0, s>>>(
                    st.src, st.lds, st.ptr, st.ld, st.nr, st.nb);
                count_launches(1);
            } else if (st.kind == 7) {
                tile_inverse_kernel<T><<<st.nr, 256, 0, s>>>(st.ptr, st.nb, st.inv);
                count_launches(1);
            } else if (st.kind == 2) {
                zero_upper_kernel<T><<<grid_for((long long)st.nb * st.nb), 256, 0, s>>>(st.ptr, st.nb);
                count_launches(1);
            } else if (st.kind == 3) {
                copy_tile_kernel<T><<<std::max(1, std::min(1024, (st.nr * st.nc + 255) / 256)), 256, 0, s>>>(st.src, st.lds, st.ptr,
                                                                                                          st.ld, st.nr, st.nc);
                count_launches(1);
            } else if (st.kind == 4) {
                MSP_CUDA(cudaMemsetAsync(st.ptr, 0, sizeof(T) * (size_t)st.nr * st.nc, s));
            } else if (early_exit) {   // pivot check after a diagonal block: stop at the first breakdown
                MSP_CUDA(cudaGetLastError());
                MSP_CUDA(cudaMemcpyAsync(&hfail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
                MSP_CUDA(cudaStreamSynchronize(s));
                if (hfail) break;
            }
            if (st.rec_ev >= 0) MSP_CUDA(cudaEventRecord(side.ev[st.rec_ev], ss));
        }
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaMemcpyAsync(&hfail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        MSP_CUDA(cudaStreamSynchronize(side.st));
        MSP_TRY(ozaki_check(ozw, s));
        MSP_TRY(ozaki_check(ozw_side, side.st));
        B.bt_shift = shift;
    }
    *fail_out = hfail;
    if (hfail) return MSP_OK;
    // transposed copies for the sweeps (each product then reads contiguous columns)
    MSP_TRY(S.FT.alloc(std::max<long long>(total, 1), s));
    MSP_TRY(S.LiT.alloc(std::max<long long>(B.bt_diag_elems, 1), s));
    for (int q = 0; q < Qn; ++q) {
        const int n = B.bt_off[q + 1] - B.bt_off[q];
        if (n == 0) continue;
        dim3 g1((n + 31) / 32, (n + 31) / 32);
        transpose_kernel<T><<<g1, dim3(32, 8), 0, s>>>(S.Li.p + B.bt_d_off[q], S.LiT.p + B.bt_d_off[q], n, n);
        count_launches(1);
        if (q + 1 < Qn) {
            const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
            dim3 g2((n1 + 31) / 32, (n + 31) / 32);
            transpose_kernel<T><<<g2, dim3(32, 8), 0, s>>>(S.F.p + B.bt_e_off[q], S.FT.p + B.bt_e_off[q], n1, n);
            count_launches(1);
        }
    }
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}


msp_status build_online_factor(Basis& B, const std::vector<int>& row_ptr, const std::vector<int>& row_slot,
                               cudaStream_t s) {
    const int np = (int)B.patches.size();
    const int Qn = B.my, mx = B.mx;
    B.bt_q = Qn;
    B.bt_off.assign(Qn + 1, 0);
    for (int q = 0; q <= Qn; ++q) B.bt_off[q] = B.c_off[std::min(q * mx, np)];
    // slot -> patch
    std::vector<int> slot_patch(B.n_slots);
    for (int m = 0; m < np; ++m)
        for (int g = B.slot_off[m]; g < B.slot_off[m + 1]; ++g) slot_patch[g] = m;
    // dense block layout (FP64 assembly and FP32 factors)
    B.bt_d_off.assign(Qn, 0);
    B.bt_e_off.assign(std::max(Qn - 1, 0), 0);
    long long off = 0;
    for (int q = 0; q < Qn; ++q) {
        const long long n = B.bt_off[q + 1] - B.bt_off[q];
        B.bt_d_off[q] = off;
        off += n * n;
    }
    B.bt_diag_elems = off;
    for (int q = 0; q + 1 < Qn; ++q) {
        const long long n0 = B.bt_off[q + 1] - B.bt_off[q], n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
        B.bt_e_off[q] = off;
        off += n1 * n0;
    }
    const long long total = off;
    // pair lists: for every row and ordered pair of its entries in the same or the
    // next-lower patch row, the (slot a, slot b, sign) triple, grouped by patch pair
    // (ma, mb) in ascending order and in row order inside a pair.  Patches sharing a
    // skeleton node are grid neighbours, so mb is one of six positions relative to
    // ma (one row down or the same row, one column left, the same or one right),
    // numbered in ascending mb; two counting passes build the groups.
    auto pair_slot = [&](int ma, int mb) {
        const int dq = ma / mx - mb / mx, dp = ma % mx - mb % mx;   // dq in {0, 1}, dp in {-1, 0, 1}
        return ma * 6 + (1 - dq) * 3 + (1 - dp);
    };
    std::vector<int> pcount((size_t)np * 6 + 1, 0);
    auto for_pairs = [&](auto&& fn) {
        for (int r = 0; r + 1 < (int)row_ptr.size(); ++r)
            for (int a = row_ptr[r]; a < row_ptr[r + 1]; ++a) {
                const unsigned va = (unsigned)row_slot[a];
                const int sa = (int)(va & 0x7fffffffu), ma = slot_patch[sa];
                for (int b = row_ptr[r]; b < row_ptr[r + 1]; ++b) {
                    const unsigned vb = (unsigned)row_slot[b];
                    const int sb = (int)(vb & 0x7fffffffu), mb = slot_patch[sb];
                    const int qa = ma / mx, qb = mb / mx;
                    if (!(qa == qb || qa == qb + 1)) continue;
                    fn(ma, mb, sa, sb, (signed char)(((va ^ vb) & 0x80000000u) ? -1 : 1));
                }
            }
    };
    bool adjacency_ok = true;
    for_pairs([&](int ma, int mb, int, int, signed char) {
        const int dp = ma % mx - mb % mx;
        if (dp < -1 || dp > 1) adjacency_ok = false;
        else ++pcount[pair_slot(ma, mb) + 1];
    });
    if (!adjacency_ok) {
        set_error("msp_extract_basis: a skeleton row couples patches that are not grid neighbours");
        return MSP_ERR_INVALID_ARG;
    }
    for (size_t t = 0; t + 1 < pcount.size(); ++t) pcount[t + 1] += pcount[t];
    std::vector<int> lsa(pcount.back()), lsb(pcount.back());
    std::vector<signed char> lsg(pcount.back());
    {
        std::vector<int> cur(pcount.begin(), pcount.end() - 1);
        for_pairs([&](int ma, int mb, int sa, int sb, signed char sg) {
            const int at = cur[pair_slot(ma, mb)]++;
            lsa[at] = sa;
            lsb[at] = sb;
            lsg[at] = sg;
        });
    }
    std::vector<PairBlock> pb;
    B.bt_elo.assign(np, -1);
    B.bt_ehi.assign(np, -1);
    for (int ma = 0; ma < np; ++ma)
        for (int c = 0; c < 6; ++c) {
            const int t = ma * 6 + c;
            if (pcount[t] == pcount[t + 1]) continue;
            const int dq = 1 - c / 3, dp = 1 - c % 3;
            const int mb = ma - dq * mx - dp;
            if (B.k[ma] == 0 || B.k[mb] == 0) continue;
            const int qa = ma / mx, qb = mb / mx;
            PairBlock p{};
            p.ma = ma;
            p.mb = mb;
            p.list_begin = pcount[t];
            p.list_end = pcount[t + 1];
            if (qa == qb) {
                const int n = B.bt_off[qa + 1] - B.bt_off[qa];
                p.dst = B.bt_d_off[qa] + (B.c_off[ma] - B.bt_off[qa]) + (long long)(B.c_off[mb] - B.bt_off[qb]) * n;
                p.ld = n;
            } else {   // E_qb: rows from block qb+1, columns from block qb
                const int n1 = B.bt_off[qa + 1] - B.bt_off[qa];
                p.dst = B.bt_e_off[qb] + (B.c_off[ma] - B.bt_off[qa]) + (long long)(B.c_off[mb] - B.bt_off[qb]) * n1;
                p.ld = n1;
            }
            pb.push_back(p);
            if (qa == qb + 1) {   // patch ma (row qb+1) couples with patch mb of row qb
                B.bt_elo[ma] = B.bt_elo[ma] < 0 ? mb : std::min(B.bt_elo[ma], mb);
                B.bt_ehi[ma] = std::max(B.bt_ehi[ma], mb);
            }
        }
    DevBuf<PairBlock> d_pb;
    DevBuf<int> d_lsa, d_lsb;
    DevBuf<signed char> d_lsg;
    MSP_TRY(upload(d_pb, pb, s));
    MSP_TRY(upload(d_lsa, lsa, s));
    MSP_TRY(upload(d_lsb, lsb, s));
    MSP_TRY(upload(d_lsg, lsg, s));
    DevBuf<double> H64;
    MSP_TRY(H64.alloc(std::max<long long>(total, 1), s));
    MSP_CUDA(cudaMemsetAsync(H64.p, 0, sizeof(double) * std::max<long long>(total, 1), s));
    if (!pb.empty()) {
        assemble_kernel<<<(int)pb.size(), 256, 0, s>>>(d_pb.p, d_lsa.p, d_lsb.p, d_lsg.p, B.d_k.p, B.d_e_off.p,
                                                       B.d_slot_off.p, B.E.p, H64.p);
        count_launches(1);
    }
    // Hs_ab = F_a^T H_ab F_b for every nonzero patch pair (F = L_m^{-T} of the patch blocks)
    DevBuf<double> Hs64, Tp;
    MSP_TRY(Hs64.alloc(std::max<long long>(total, 1), s));
    MSP_CUDA(cudaMemsetAsync(Hs64.p, 0, sizeof(double) * std::max<long long>(total, 1), s));
    {
        long long tsz = 0;
        std::vector<long long> toff(pb.size());
        int maxk = 1;
        for (size_t t = 0; t < pb.size(); ++t) {
            toff[t] = tsz;
            tsz += (long long)B.k[pb[t].ma] * B.k[pb[t].mb];
            maxk = std::max(maxk, std::max(B.k[pb[t].ma], B.k[pb[t].mb]));
        }
        MSP_TRY(Tp.alloc(std::max<long long>(tsz, 1), s));
        std::vector<GemmDesc> g1(pb.size()), g2(pb.size());
        for (size_t t = 0; t < pb.size(); ++t) {
            const int ka = B.k[pb[t].ma], kb = B.k[pb[t].mb];
            const double* Fa = B.bt_Fi.p + B.binv_off[pb[t].ma];
            const double* Fb = B.bt_Fi.p + B.binv_off[pb[t].mb];
            g1[t] = GemmDesc{H64.p + pb[t].dst, Fb, Tp.p + toff[t], ka, kb, kb, pb[t].ld, kb, ka, 1.0, 0.0};
            g2[t] = GemmDesc{Fa, Tp.p + toff[t], Hs64.p + pb[t].dst, ka, kb, ka, ka, ka, pb[t].ld, 1.0, 0.0};
        }
        DevBuf<GemmDesc> d1, d2;
        MSP_TRY(upload(d1, g1, s));
        MSP_TRY(upload(d2, g2, s));
        if (!pb.empty()) {
            gemm_batched<double>(d1.p, (int)pb.size(), maxk, maxk, false, false, s);
            gemm_batched<double>(d2.p, (int)pb.size(), maxk, maxk, true, false, s);
        }
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaStreamSynchronize(s));   // descriptor buffers go out of scope
    }
    H64.free_now();
    // first nonzero column of each row of C_{q-1} = E_{q-1} L_{q-1}^{-T} (in block q-1
    // coordinates), as a suffix minimum so that it is nondecreasing along the rows
    {
        std::vector<int> rowlo(std::max(B.Np, 1), 0);
        for (int q = 1; q < Qn; ++q) {
            const int n0 = B.bt_off[q] - B.bt_off[q - 1];
            for (int p = 0; p < mx; ++p) {
                const int ma = q * mx + p;
                if (ma >= np) continue;
                const int lo = B.bt_elo[ma] < 0 ? n0 : B.c_off[B.bt_elo[ma]] - B.bt_off[q - 1];
                for (int r = B.c_off[ma]; r < B.c_off[ma + 1]; ++r) rowlo[r] = lo;
            }
            for (int r = B.bt_off[q + 1] - 2; r >= B.bt_off[q]; --r) rowlo[r] = std::min(rowlo[r], rowlo[r + 1]);
        }
        MSP_TRY(upload(B.d_bt_rowlo, rowlo, s));
    }
    // factorise in FP32; if a pivot fails, in FP64
    int fail = 0;
    MSP_TRY(factorize<float>(B, Hs64.p, total, 0.0, &fail, B.bt32, true, s));
    if (!fail) {
        B.bt_prec = 1;
        return MSP_OK;
    }
    B.bt32.free_all();
    const double shifts[3] = {0.0, 1e-12, 1e-9};
    for (int a = 0; a < 3; ++a) {
        MSP_TRY(factorize<double>(B, Hs64.p, total, shifts[a], &fail, B.bt64, false, s));
        if (!fail) {
            B.bt_prec = 2;
            B.bt_shift = (float)shifts[a];
            // FP32 rounded copy of the factor for the sweeps: the rounded factor is a
            // preconditioner within about u32 kappa(L) = u32 kappa(H)^(1/2) of the
            // exact one, so the FP64 iteration needs a few more steps, each sweep at
            // the FP32 rate
            const long long nd = std::max<long long>(B.bt_diag_elems, 1), nt = std::max<long long>(total, 1);
            MSP_TRY(B.bt32.F.alloc(nt, s));
            MSP_TRY(B.bt32.FT.alloc(nt, s));
            MSP_TRY(B.bt32.Li.alloc(nd, s));
            MSP_TRY(B.bt32.LiT.alloc(nd, s));
            round_kernel<<<grid_for(nt), 256, 0, s>>>(B.bt64.F.p, B.bt32.F.p, nt);
            round_kernel<<<grid_for(nt), 256, 0, s>>>(B.bt64.FT.p, B.bt32.FT.p, nt);
            round_kernel<<<grid_for(nd), 256, 0, s>>>(B.bt64.Li.p, B.bt32.Li.p, nd);
            round_kernel<<<grid_for(nd), 256, 0, s>>>(B.bt64.LiT.p, B.bt32.LiT.p, nd);
            count_launches(4);
            MSP_CUDA(cudaGetLastError());
            return MSP_OK;
        }
    }
    set_error("msp_extract_basis: online preconditioner factorisation broke down in FP64");
    return MSP_ERR_BREAKDOWN;
}

// z = S (L L^T)^{-1} S s for a batch of Bsz vectors ([element][B] layout, FP64 in and out)
// Cooperative launch of sweep_kernel: the grid is as many CTAs as are resident
// at once (at most two per SM), so the grid barrier cannot wait on an unscheduled CTA.
// The grid size and the shared-memory attribute are set up once per device and
// instance, under a lock (several host threads may make their first call at once).
template <class T, int BT>
msp_status launch_sweeps_bt(SweepArgs<T> A, cudaStream_t s) {
    static std::mutex mu;
    static std::vector<int> grids;   // per device; 0 = not set up yet
    const size_t smem = sizeof(T) * kSweepKC * BT;
    int dev = 0, grid = 0;
    MSP_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(mu);
        if ((int)grids.size() <= dev) grids.resize(dev + 1, 0);
        if (grids[dev] == 0) {
            MSP_CUDA(cudaFuncSetAttribute(sweep_kernel<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int occ = 0;
            MSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sweep_kernel<T, BT>, 512, smem));
            if (occ < 1) {
                set_error("online sweeps: the sweep kernel does not fit on an SM");
                return MSP_ERR_CUDA;
            }
            grids[dev] = num_sms() * std::min(occ, 2);
        }
        grid = grids[dev];
    }
    A.spin_limit = wait_limit();
    void* params[] = {&A};
    MSP_CUDA(cudaLaunchCooperativeKernel((const void*)sweep_kernel<T, BT>, dim3(grid), dim3(512), params, smem, s));
    count_launches(1);
    return MSP_OK;
}

template <class T>
msp_status launch_sweeps(Basis& B, BtStore<T>& S, T* y, T* x, int Bsz, cudaStream_t s) {
    if (B.bt_q <= 0) return MSP_OK;
    if (!B.d_bt_off.p) {
        std::vector<long long> eo(B.bt_e_off);
        if (eo.empty()) eo.push_back(0);
        MSP_TRY(upload(B.d_bt_off, B.bt_off, s));
        MSP_TRY(upload(B.d_bt_d_off, B.bt_d_off, s));
        MSP_TRY(upload(B.d_bt_e_off, eo, s));
        MSP_TRY(B.d_bt_bar.alloc(4, s));
        MSP_CUDA(cudaMemsetAsync(B.d_bt_bar.p, 0, sizeof(unsigned int) * 4, s));
    }
    SweepArgs<T> A{};
    A.Qn = B.bt_q;
    A.B = Bsz;
    A.off = B.d_bt_off.p;
    A.d_off = B.d_bt_d_off.p;
    A.e_off = B.d_bt_e_off.p;
    A.LiT = S.LiT.p;
    A.FT = S.FT.p;
    A.Li = S.Li.p;
    A.F = S.F.p;
    A.y = y;
    A.x = x;
    A.bar = B.d_bt_bar.p;
    A.err = reinterpret_cast<int*>(B.d_bt_bar.p + 2);
    if (Bsz <= 1) return launch_sweeps_bt<T, 1>(A, s);
    if (Bsz <= 2) return launch_sweeps_bt<T, 2>(A, s);
    if (Bsz <= 4) return launch_sweeps_bt<T, 4>(A, s);
    return launch_sweeps_bt<T, 8>(A, s);
}

template <class T>
msp_status apply_factor(Basis& B, BtStore<T>& S, const double* s_in, double* z_out, int Bsz, cudaStream_t s) {
    const long long n = B.Np;
    if (n == 0) return MSP_OK;
    if ((long long)S.w1.n < n * Bsz) {
        MSP_TRY(S.w1.alloc((size_t)n * std::max(Bsz, 1), s));
        MSP_TRY(S.w2.alloc((size_t)n * std::max(Bsz, 1), s));
    }
    T* y = S.w1.p;   // right-hand side, then the forward sweep's result
    T* x = S.w2.p;   // backward sweep's result
    const int np = (int)B.patches.size();
    patch_pre_kernel<T><<<np, 256, 0, s>>>(B.bt_Fi.p, B.d_binv_off.p, B.d_k.p, B.d_c_off.p, s_in, y, Bsz);
    count_launches(1);
    MSP_TRY(launch_sweeps<T>(B, S, y, x, Bsz, s));
    patch_post_kernel<T><<<np, 256, 0, s>>>(B.bt_Fi.p, B.d_binv_off.p, B.d_k.p, B.d_c_off.p, y, z_out, Bsz);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}


constexpr int kApply32MinBatch = 4;

msp_status apply_online_factor(Basis& B, const double* s_in, double* z_out, int Bsz, cudaStream_t s) {
    // an FP64 factor: applied in FP64 for small batches (fewest iterations, the
    // sweeps are latency-bound there), through its FP32 copy for larger ones (the
    // sweeps become arithmetic-bound)
    if (B.bt_prec == 2 && (B.bt_apply_mode == 1 || (B.bt_apply_mode == 0 && Bsz < kApply32MinBatch)))
        return apply_factor<double>(B, B.bt64, s_in, z_out, Bsz, s);
    return apply_factor<float>(B, B.bt32, s_in, z_out, Bsz, s);
}

}  // namespace msp
