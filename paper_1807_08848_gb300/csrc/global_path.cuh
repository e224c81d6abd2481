// The global-scratch form of the offline local solves (Algorithm alg:summary,
// RanLocalSolu; Eq. elliptic_random): ring data of the buffered patch,
// Jacobi-preconditioned CG for the 5-point operator on a tile held in a per-CTA
// slot of global memory, restriction to K_m.  Used by local_solve_global and, for
// the tiles that do not fit on chip, by the fused persistent tile kernel.
#pragma once

#include "internal.h"
#include "device_util.cuh"

namespace msp {
namespace gpath {

struct SolveArgs {
    int N;
    const double* aE;   // (N+1) x N
    const double* aN;   // N x (N+1)
    const float* aE32;
    const float* aN32;
    const PatchDev* patches;
    const int* bpos;
    const int2* items;
    int n_items;
    double* snaps;
    uint64_t seed;
    double tol, inner_tol;
    int max_iter, max_ref;
    double* scratch;
    long long slot_bytes;   // bytes per CTA slot (multiple of 256)
    int* stats;             // per item: [iters, refinements, not_converged]
};

// Ring datum of column `col` at ring position t (Gaussian or a boundary delta).
__device__ __forceinline__ void fill_ring(const SolveArgs& A, const PatchDev& P, int m, int col, double* x,
                                          int W) {
    if (col < P.samples) {
        const int npairs = (P.n_ring + 1) >> 1;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            const double2 z = gaussian_pair(A.seed, (uint32_t)q, (uint32_t)col, (uint32_t)m, kTagElliptic);
            int i, j;
            ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q, i, j);
            x[(i - P.X0) + (j - P.Y0) * W] = z.x;
            if (2 * q + 1 < P.n_ring) {
                ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q + 1, i, j);
                x[(i - P.X0) + (j - P.Y0) * W] = z.y;
            }
        }
    } else {
        const int t0 = A.bpos[P.bpos_offset + (col - P.samples)];
        for (int t = threadIdx.x; t < P.n_ring; t += blockDim.x) {
            int i, j;
            ring_node(P.X0, P.X1, P.Y0, P.Y1, t, i, j);
            x[(i - P.X0) + (j - P.Y0) * W] = (t == t0) ? 1.0 : 0.0;
        }
    }
}

template <class T>
struct Coefs;
template <>
struct Coefs<double> {
    __device__ static const double* E(const SolveArgs& A) { return A.aE; }
    __device__ static const double* Nn(const SolveArgs& A) { return A.aN; }
};
template <>
struct Coefs<float> {
    __device__ static const float* E(const SolveArgs& A) { return A.aE32; }
    __device__ static const float* Nn(const SolveArgs& A) { return A.aN32; }
};

// Solve A d = r on the interior of a W x H tile by Jacobi-preconditioned CG in
// precision T, from d = 0, until |r| <= rtol |r0|.  Vectors are full tiles with a
// zero ring (p and d); r, Ap, dinv use only interior entries.  Returns the
// iteration count (negative if max_iter was hit).
template <class T>
__device__ int block_pcg(const SolveArgs& A, const PatchDev& P, int W, int H, T* d, T* r, T* p, T* Ap,
                         const T* dinv, double rtol, int max_iter, T* red) {
    const int nx = W - 2, ny = H - 2, nint = nx * ny;
    const int N = A.N;
    const T* aE = Coefs<T>::E(A);
    const T* aN = Coefs<T>::Nn(A);
    T rz, rr0;
    {
        T v[2] = {0, 0};
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            const T z = dinv[k] * r[k];
            p[k] = z;
            d[k] = 0;
            v[0] += r[k] * z;
            v[1] += r[k] * r[k];
        }
        block_sum<T, 2>(v, red);
        rz = v[0];
        rr0 = v[1];
    }
    if (rr0 == T(0)) return 0;
    const T stop = (T)(rtol * rtol) * rr0;
    int it = 0;
    for (; it < max_iter;) {
        // Ap = A p, pAp
        T v1[1] = {0};
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            const int gi = P.X0 + ii + 1, gj = P.Y0 + jj + 1;
            const T ae = aE[(long long)gj * N + gi], aw = aE[(long long)gj * N + gi - 1];
            const T an = aN[(long long)gj * (N + 1) + gi], as = aN[(long long)(gj - 1) * (N + 1) + gi];
            const T q = (ae + aw + an + as) * p[k] - ae * p[k + 1] - aw * p[k - 1] - an * p[k + W] - as * p[k - W];
            Ap[k] = q;
            v1[0] += p[k] * q;
        }
        block_sum<T, 1>(v1, red + 64);
        const T alpha = rz / v1[0];
        T v2[2] = {0, 0};
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            d[k] += alpha * p[k];
            const T rk = r[k] - alpha * Ap[k];
            r[k] = rk;
            v2[0] += rk * dinv[k] * rk;
            v2[1] += rk * rk;
        }
        block_sum<T, 2>(v2, red);
        ++it;
        if (v2[1] <= stop) break;
        const T beta = v2[0] / rz;
        rz = v2[0];
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            p[k] = dinv[k] * r[k] + beta * p[k];
        }
        __syncthreads();
    }
    return (it >= max_iter) ? -it : it;
}

// r = -(A x)_interior in FP64 (x holds the ring data), stored in T; returns |r|^2.
template <class T>
__device__ double residual64(const SolveArgs& A, const PatchDev& P, int W, int H, const double* x, T* r,
                             double* red) {
    const int nx = W - 2, ny = H - 2, nint = nx * ny;
    const int N = A.N;
    double v[1] = {0.0};
    for (int t = threadIdx.x; t < nint; t += blockDim.x) {
        const int jj = t / nx, ii = t - jj * nx;
        const int k = (ii + 1) + (jj + 1) * W;
        const int gi = P.X0 + ii + 1, gj = P.Y0 + jj + 1;
        const double ae = A.aE[(long long)gj * N + gi], aw = A.aE[(long long)gj * N + gi - 1];
        const double an = A.aN[(long long)gj * (N + 1) + gi], as = A.aN[(long long)(gj - 1) * (N + 1) + gi];
        const double q = -((ae + aw + an + as) * x[k] - ae * x[k + 1] - aw * x[k - 1] - an * x[k + W] - as * x[k - W]);
        r[k] = (T)q;
        v[0] += q * q;
    }
    block_sum<double, 1>(v, red);
    return v[0];
}

// One local solve (patch, column) of item `item` of A.items in the CTA's global
// scratch slot: ring data, FP64 iterate, CG in precision T (FP32 CG inside FP64
// iterative refinement when T = float), restriction to K_m, statistics.
template <class T>
__device__ void global_item(const SolveArgs& A, int item, char* slot, double* red64, T* redT) {
        const int2 it = A.items[item];
    const int m = it.x, col = it.y;
    const PatchDev P = A.patches[m];
    const int W = P.X1 - P.X0 + 1, H = P.Y1 - P.Y0 + 1, WH = W * H;
    double* x = reinterpret_cast<double*>(slot);
    T* d = reinterpret_cast<T*>(x + WH);
    T* r = d + WH;
    T* p = r + WH;
    T* Ap = p + WH;
    T* dinv = Ap + WH;
    // x = 0 inside, ring data on the ring; d, p zero everywhere (zero ring)
    for (int k = threadIdx.x; k < WH; k += blockDim.x) {
        x[k] = 0.0;
        d[k] = 0;
        p[k] = 0;
    }
    __syncthreads();
    fill_ring(A, P, m, col, x, W);
    {
        const int nx = W - 2, nint = nx * (H - 2);
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            const int gi = P.X0 + ii + 1, gj = P.Y0 + jj + 1;
            const double diag = A.aE[(long long)gj * A.N + gi] + A.aE[(long long)gj * A.N + gi - 1] +
                                A.aN[(long long)gj * (A.N + 1) + gi] + A.aN[(long long)(gj - 1) * (A.N + 1) + gi];
            dinv[k] = (T)(1.0 / diag);
        }
    }
    __syncthreads();
    int total_it = 0, refs = 0, bad = 0;
    double b2 = -1.0;
    const int passes = (sizeof(T) == 8) ? 1 : A.max_ref;
    for (int pass = 0; pass < passes; ++pass) {
        const double r2 = residual64<T>(A, P, W, H, x, r, red64);
        if (b2 < 0) b2 = r2;
        if (b2 == 0.0 || r2 <= A.tol * A.tol * b2) break;
        double scale = 1.0;
        if (sizeof(T) == 4) {   // normalise the FP32 right-hand side
            scale = sqrt(r2);
            const int nx = W - 2, nint = nx * (H - 2);
            const T inv = (T)(1.0 / scale);
            for (int t = threadIdx.x; t < nint; t += blockDim.x) {
                const int jj = t / nx, ii = t - jj * nx;
                const int k = (ii + 1) + (jj + 1) * W;
                r[k] *= inv;
            }
            __syncthreads();
        }
        const double rtol = (sizeof(T) == 8) ? A.tol : A.inner_tol;
        int its = block_pcg<T>(A, P, W, H, d, r, p, Ap, dinv, rtol, A.max_iter, redT);
        if (its < 0) { bad = 1; its = -its; }
        total_it += its;
        ++refs;
        const int nx = W - 2, nint = nx * (H - 2);
        for (int t = threadIdx.x; t < nint; t += blockDim.x) {
            const int jj = t / nx, ii = t - jj * nx;
            const int k = (ii + 1) + (jj + 1) * W;
            x[k] += scale * (double)d[k];
        }
        __syncthreads();
        if (bad) break;
    }
    if (sizeof(T) == 4 && !bad && b2 > 0.0) {   // did the refinement reach tol?
        const double r2 = residual64<T>(A, P, W, H, x, r, red64);
        if (r2 > A.tol * A.tol * b2) bad = 1;
    }
    // restriction to K_m (Sec. 3.3): column `col` of the snapshot block
    const int wk = P.x1 - P.x0 + 1;
    double* out = A.snaps + P.snap_offset + (long long)col * P.n_k;
    for (int t = threadIdx.x; t < P.n_k; t += blockDim.x) {
        const int jj = t / wk, ii = t - jj * wk;
        out[t] = x[(P.x0 - P.X0 + ii) + (P.y0 - P.Y0 + jj) * W];
    }
    if (threadIdx.x == 0) {
        A.stats[3 * item + 0] = total_it;
        A.stats[3 * item + 1] = refs;
        A.stats[3 * item + 2] = bad;
    }
    __syncthreads();
}

}  // namespace gpath
}  // namespace msp
