// Basis extraction (Sec. 3.2, Eq. svd; the QR remark of Sec. 3.3) and the
// online operators built from it (Eq. elliptic_cond_tilde).
//
// Per patch, with R_m the n_k x c snapshot block:
//   shifted Cholesky-QR3  R = Q3 T   (Fukaya, Kannan, Nakatsukasa, Yamamoto,
//                                     Yanagisawa, SIAM J. Sci. Comput. 2020)
//   one-sided Jacobi SVD of T^T     T = U_T S V_T^T   (Hestenes' method)
//   truncation                       k = #{s_i > tau s_1},  Q_m = Q3 U_T[:, :k]
// then the value/flux rows of Q_m on the ring of K_m and the inverse of every
// patch block of P~^T P~ (the additive-Schwarz preconditioner of the online
// iteration).
#include "internal.h"
#include "dense.cuh"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>
#include <utility>

namespace msp {

namespace {

struct SmallMat {
    long long off;   // offset of this patch's c x c block
    int c;           // order
    int n;           // rows of the tall matrix
    int idx;         // patch index (the Jacobi kernels run the blocks largest first)
};

// Cholesky of (G + shift I) = L L^T in global memory (one CTA per matrix),
// then F = L^T and Fi = L^{-T} (upper triangular), column-major order c.
// shift0 > 0 requests a shifted factorisation; on a non-positive pivot the
// shift grows (to 1e-14 trace if it was zero, else x100) up to 6 tries.
// status[b]: number of tries used, or -1 on failure.
__global__ void __launch_bounds__(256) chol_factor_kernel(const SmallMat* mats, const double* G, double* L,
                                                          double* F, double* Fi, const double* shift_scale,
                                                          int shifted, int* status) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    if (c <= 0) return;
    const double* g = G + S.off;
    double* l = L + S.off;
    double* f = F + S.off;
    double* fi = Fi + S.off;
    __shared__ double s_trace;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < c; ++i) t += g[i + (long long)i * c];
        s_trace = t;
    }
    __syncthreads();
    const double trace = s_trace;
    double shift = 0.0;
    if (shifted) shift = shift_scale[blockIdx.x] * trace;
    int tries = 0;
    bool ok = false;
    for (; tries < 6 && !ok; ++tries) {
        for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
            const int i = (int)(e % c), j = (int)(e / c);
            l[e] = (i >= j) ? g[e] + (i == j ? shift : 0.0) : 0.0;
        }
        __syncthreads();
        ok = true;
        for (int k = 0; k < c; ++k) {
            if (threadIdx.x == 0) {
                const double d = l[k + (long long)k * c];
                s_ok = (d > 0.0 && isfinite(d)) ? 1 : 0;
                if (s_ok) l[k + (long long)k * c] = sqrt(d);
            }
            __syncthreads();
            if (!s_ok) { ok = false; break; }
            const double piv = l[k + (long long)k * c];
            for (int i = k + 1 + threadIdx.x; i < c; i += blockDim.x) l[i + (long long)k * c] /= piv;
            __syncthreads();
            // trailing update of the lower triangle: a warp per column j, lanes along
            // the rows i >= j (contiguous in the column-major block)
            {
                const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
                for (int j = k + 1 + (threadIdx.x >> 5); j < c; j += nw) {
                    const double ljk = l[j + (long long)k * c];
                    double* lj = l + (long long)j * c;
                    const double* lk = l + (long long)k * c;
                    for (int i = j + lane; i < c; i += 32) lj[i] -= lk[i] * ljk;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (!ok) shift = (shift == 0.0) ? 1e-14 * trace : shift * 100.0;
    }
    if (!ok) {
        if (threadIdx.x == 0) status[blockIdx.x] = -1;
        return;
    }
    if (threadIdx.x == 0) status[blockIdx.x] = tries;
    // F = L^T
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        f[e] = (i <= j) ? l[j + (long long)i * c] : 0.0;
    }
    // Fi = (L^{-1})^T, X = L^{-1} with X(i, j) stored at Fi(j, i) = fi[j + i c]: row i
    // of X, X(i, j) = (delta_ij - sum_{q<i} l_iq X(q, j)) / l_ii, for all j <= i at
    // once -- one barrier per row, a warp per column j, lanes along q, the partial
    // sums of a warp combined by shuffles in a fixed order
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) fi[e] = 0.0;
    __syncthreads();
    {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = 0; i < c; ++i) {
            const double rli = 1.0 / l[i + (long long)i * c];
            const double* li = l + i;   // l_iq at li[q c]
            for (int j = threadIdx.x >> 5; j <= i; j += nw) {
                double a = 0.0;
                for (int q = j + lane; q < i; q += 32) a += li[(long long)q * c] * fi[j + (long long)q * c];
                a = warp_sum(a);
                if (lane == 0) fi[j + (long long)i * c] = ((i == j ? 1.0 : 0.0) - a) * rli;
            }
            __syncthreads();
        }
    }
}

// W = T^T, V = I (per patch, order c).
__global__ void jacobi_init_kernel(const SmallMat* mats, const double* T, double* W, double* V) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        W[S.off + e] = T[S.off + j + (long long)i * c];
        V[S.off + e] = (i == j) ? 1.0 : 0.0;
    }
}

constexpr int kJacGroup = 8;       // threads per column pair
constexpr int kJacMaxPairs = 512;  // c <= 1024

// One-sided (Hestenes) Jacobi on the columns of w (c x c, leading dimension ldw):
// rotate column pairs (p, q) until every pair is orthogonal to relative level
// tol; v (leading dimension ldv) accumulates the same rotations.  Started from
// w = T^T V0 with V0 orthogonal, it ends with w = Z S and T = (V0 J) S Z^T, J the
// product of the rotations: the singular values are the column norms of w and
// v = V0 J holds the left singular vectors of T.  (On T^T the sweeps converge in
// about a third of the sweeps needed on the columns of T.)  Pairs follow the
// round-robin tournament order, c/2 disjoint pairs per round.  Each round has
// three phases: groups of kJacGroup threads take one pair each and form its
// three inner products; one thread per pair decides whether to rotate and takes
// the angle (the square roots and divisions are done once per pair, not once per
// lane of a group); then the whole block applies the round's rotations to the
// columns of w and v with row-wise accesses.
// Skips: columns below u |T|_F are numerically zero; a pair orthogonal to the
// rounding floor of its inner product is left alone; and a pair whose columns
// are both below small_rel |T|_F (far under the truncation level) is left alone,
// since rotating it only mixes directions that are dropped.  Returns the sweeps
// taken (max_sweeps if it did not converge).  fro2 = |T|_F^2, u = unit roundoff
// of T.  Called by all threads of the block.
template <class T>
__device__ int jacobi_sweeps(T* w, int ldw, T* v, int ldv, int c, int max_sweeps, T tol, T small_rel, T fro2, T u) {
    __shared__ T s_cs[kJacMaxPairs], s_sn[kJacMaxPairs], s_ga[kJacMaxPairs];
    __shared__ int s_p[kJacMaxPairs], s_q[kJacMaxPairs];
    __shared__ int s_rot;
    const T negligible = u * u * fro2;   // (u |T|_F)^2
    // rounding floor of an inner product of columns of norms a and b: the columns
    // carry absolute errors ~ c u |T|_F, so orthogonality below that is noise
    const T floor_abs = T(2) * c * u * sqrt(fro2);
    const T small2 = small_rel * small_rel * fro2;
    const int np = c + (c & 1);   // players, even
    const int npairs = np / 2;
    const int g = threadIdx.x % kJacGroup;
    const int groups = blockDim.x / kJacGroup;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            // phase 1: one group per pair, its three inner products; every thread
            // runs the same number of iterations so that the group shuffles see
            // full warps
            for (int base = 0; base < npairs; base += groups) {
                const int pr = base + threadIdx.x / kJacGroup;
                const bool live = pr < npairs;
                int p = 0, q = 0;
                if (live) {
                    int a, b;
                    if (pr == 0) { a = r; b = np - 1; }
                    else { a = (r + pr) % (np - 1); b = (r - pr + (np - 1)) % (np - 1); }
                    p = min(a, b);
                    q = max(a, b);
                }
                const bool real = live && q < c;
                const T* wp = w + (long long)p * ldw;
                const T* wq = w + (long long)q * ldw;
                T al = 0, be = 0, ga = 0;
                if (real) {
                    for (int i = g; i < c; i += kJacGroup) {
                        const T x = wp[i], y = wq[i];
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                        ga = fma(x, y, ga);
                    }
                }
#pragma unroll
                for (int o = kJacGroup / 2; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (live && g == 0) {
                    s_p[pr] = real ? p : -1;
                    s_q[pr] = q;
                    s_cs[pr] = al;   // the angle phase overwrites these with cos, sin
                    s_sn[pr] = be;
                    s_ga[pr] = ga;
                }
            }
            __syncthreads();
            // phase 2: one thread per pair, the decision and the rotation angle
            for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
                if (s_p[pr] < 0) continue;
                const T al = s_cs[pr], be = s_sn[pr], ga = s_ga[pr];
                const T na = sqrt(al), nb = sqrt(be);
                if (al <= negligible || be <= negligible || (al < small2 && be < small2) ||
                    fabs(ga) <= tol * na * nb + floor_abs * (na + nb)) {
                    s_p[pr] = -1;
                    continue;
                }
                const T zeta = (be - al) / (T(2) * ga);
                const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                const T cs = T(1) / sqrt(T(1) + t * t);
                s_cs[pr] = cs;
                s_sn[pr] = cs * t;
                s_rot = 1;
            }
            __syncthreads();
            // phase 3: the round's rotations applied to the columns of w and v, rows
            // fastest
            for (int e = threadIdx.x; e < npairs * c; e += blockDim.x) {
                const int pr = e / c, i = e - pr * c;
                const int p = s_p[pr];
                if (p < 0) continue;
                const int q = s_q[pr];
                const T cs = s_cs[pr], sn = s_sn[pr];
                T* wp = w + (long long)p * ldw;
                T* wq = w + (long long)q * ldw;
                const T x = wp[i], y = wq[i];
                wp[i] = cs * x - sn * y;
                wq[i] = sn * x + cs * y;
                T* vp = v + (long long)p * ldv;
                T* vq = v + (long long)q * ldv;
                const T xv = vp[i], yv = vq[i];
                vp[i] = cs * xv - sn * yv;
                vq[i] = sn * xv + cs * yv;
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();
    }
    return sweep;
}

template <class T>
__device__ T block_sum_sq(const T* w, int ldw, int c, T* red) {
    T a = 0;
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        const T x = w[i + (long long)j * ldw];
        a += x * x;
    }
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    T t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;
}

// FP64 Jacobi of W (global, c x c per patch; copied to shared memory with leading
// dimension c + 1 when c <= smem_c), V (global) accumulating.
__global__ void __launch_bounds__(512) jacobi_svd_kernel(const SmallMat* mats, double* W, double* V, int max_sweeps,
                                                         double tol, double small_rel, int smem_c, int* sweeps_out) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    __shared__ double s_red[32];
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    if (c <= 1 || c > 2 * kJacMaxPairs) {
        if (threadIdx.x == 0) sweeps_out[S.idx] = 0;
        return;
    }
    const bool in_smem = c <= smem_c;
    const int ldw = in_smem ? c + 1 : c;
    double* w = in_smem ? reinterpret_cast<double*>(jac_smem) : W + S.off;
    if (in_smem) {
        for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
            const int i = (int)(e % c), j = (int)(e / c);
            w[i + (long long)j * ldw] = W[S.off + e];
        }
        __syncthreads();
    }
    const double fro2 = block_sum_sq(w, ldw, c, s_red);
    const int sweep = jacobi_sweeps<double>(w, ldw, V + S.off, c, c, max_sweeps, tol, small_rel, fro2,
                                            1.1102230246251565e-16);
    if (in_smem) {
        for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
            const int i = (int)(e % c), j = (int)(e / c);
            W[S.off + e] = w[i + (long long)j * ldw];
        }
    }
    if (threadIdx.x == 0) sweeps_out[S.idx] = sweep;
}

// FP32 Jacobi of (float) T^T with V = I, both in shared memory (leading dimension
// c + 1) when c <= smem_c, else in the scratch (2 c^2 floats per patch at 2 off).
// Writes V (FP64 copy of the FP32 rotations, orthogonal to about 1e-6), the
// starting point of the FP64 sweeps after re-orthogonalisation.
__global__ void __launch_bounds__(512) jacobi_svd32_kernel(const SmallMat* mats, const double* Tm, float* scratch,
                                                           double* V, int max_sweeps, float tol, float small_rel,
                                                           int smem_c, int* sweeps_out) {
    extern __shared__ __align__(16) unsigned char jac_smem[];
    __shared__ float s_red[32];
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    if (c < 1 || c > 2 * kJacMaxPairs) {
        if (threadIdx.x == 0) sweeps_out[S.idx] = 0;
        return;
    }
    const bool in_smem = c <= smem_c;
    const int ld = in_smem ? c + 1 : c;
    float* w = in_smem ? reinterpret_cast<float*>(jac_smem) : scratch + 2 * S.off;
    float* v = w + (long long)c * ld;
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        w[i + (long long)j * ld] = (float)Tm[S.off + j + (long long)i * c];
        v[i + (long long)j * ld] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    const float fro2 = block_sum_sq(w, ld, c, s_red);
    int sweep = 0;
    if (c > 1) sweep = jacobi_sweeps<float>(w, ld, v, ld, c, max_sweeps, tol, small_rel, fro2, 5.9604645e-8f);
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        V[S.off + e] = (double)v[i + (long long)j * ld];
    }
    if (threadIdx.x == 0) sweeps_out[S.idx] = sweep;
}

// Newton-Schulz scaling for X (3 I - X^T X) / 2 in place of G = X^T X: the
// multiplier M = (3 I - G) / 2, so that X M is the next iterate (c x c).
__global__ void newton_schulz_kernel(const SmallMat* mats, double* G) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        G[S.off + e] = ((i == j) ? 1.5 : 0.0) - 0.5 * G[S.off + e];
    }
}


// Householder QR with column pivoting of T (c x c, column-major; one CTA of 512
// threads per patch), the preconditioner of the one-sided Jacobi SVD in the
// manner of Drmac and Veselic (2008): with T P = Q R, the Jacobi sweeps run on
// the columns of W = R^T, whose rows decay with the pivots, and V starts at Q, so
// that the rotations J of the sweeps leave V = Q J, the left singular vectors of
// T (the permutation only acts on the right).  Step j: squared norms of the
// trailing columns over rows j.. (recomputed, no downdating), the largest swapped
// into place, the reflector H_j = I - tau v v^T (v_0 = 1) that maps it onto
// R(j, j) e_0, applied to the trailing columns.  Q = H_0 H_1 ... H_{c-1} is then
// formed backwards in V.  A lives in shared memory (leading dimension c + 1) when
// c <= smem_c, else in W, which is overwritten by R^T at the end either way.
__global__ void __launch_bounds__(512) qrcp_kernel(const SmallMat* mats, const double* Tm, double* W, double* V,
                                                   int smem_c) {
    extern __shared__ __align__(16) unsigned char qr_smem[];
    __shared__ double s_nrm[2 * kJacMaxPairs];
    __shared__ double s_tau[2 * kJacMaxPairs];
    __shared__ int s_piv;
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    if (c < 1 || c > 2 * kJacMaxPairs) return;
    const bool in_smem = c <= smem_c;
    const int lda = in_smem ? c + 1 : c;
    double* a = in_smem ? reinterpret_cast<double*>(qr_smem) : W + S.off;
    double* q = V + S.off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        a[i + (long long)j * lda] = Tm[S.off + e];
    }
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        // squared norms of columns j.. over rows j..
        for (int col = j + warp; col < c; col += nw) {
            const double* ac = a + (long long)col * lda;
            double t = 0.0;
            for (int i = j + lane; i < c; i += 32) t = fma(ac[i], ac[i], t);
            t = warp_sum(t);
            if (lane == 0) s_nrm[col] = t;
        }
        __syncthreads();
        if (warp == 0) {
            double best = -1.0;
            int bi = j;
            for (int col = j + lane; col < c; col += 32)
                if (s_nrm[col] > best) { best = s_nrm[col]; bi = col; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) s_piv = bi;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != j) {
            for (int i = threadIdx.x; i < c; i += blockDim.x) {
                const double x = a[i + (long long)j * lda];
                a[i + (long long)j * lda] = a[i + (long long)p * lda];
                a[i + (long long)p * lda] = x;
            }
        }
        __syncthreads();
        // reflector of column j: beta = -sign(alpha) |x|, tau = (beta - alpha) / beta,
        // v = x(1:) / (alpha - beta) below the diagonal, R(j, j) = beta; the squared
        // norm below the diagonal is summed afresh (a difference of the column norm
        // and alpha^2 could cancel, and tau must match v for H_j to be orthogonal)
        double* aj = a + (long long)j * lda;
        if (warp == 0) {
            double t = 0.0;
            for (int i = j + 1 + lane; i < c; i += 32) t = fma(aj[i], aj[i], t);
            t = warp_sum(t);
            if (lane == 0) s_nrm[j] = t;
        }
        __syncthreads();
        const double alpha = aj[j];
        const double xn2 = s_nrm[j];
        double tau = 0.0, scal = 0.0, beta = alpha;
        if (xn2 > 0.0) {
            beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
        }
        __syncthreads();
        if (tau != 0.0) {
            for (int i = j + 1 + threadIdx.x; i < c; i += blockDim.x) aj[i] *= scal;
        }
        if (threadIdx.x == 0) {
            aj[j] = beta;
            s_tau[j] = tau;
        }
        __syncthreads();
        if (tau != 0.0) {
            // A(j:, col) -= tau v (v^T A(j:, col)) for the trailing columns, a warp each
            for (int col = j + 1 + warp; col < c; col += nw) {
                double* ac = a + (long long)col * lda;
                double t = (lane == 0) ? ac[j] : 0.0;
                for (int i = j + 1 + lane; i < c; i += 32) t = fma(aj[i], ac[i], t);
                t = warp_sum(t) * tau;
                if (lane == 0) ac[j] -= t;
                for (int i = j + 1 + lane; i < c; i += 32) ac[i] = fma(-t, aj[i], ac[i]);
            }
        }
        __syncthreads();
    }
    // Q = H_0 ... H_{c-1}: from the identity, H_j applied to rows j.. of columns j..
    for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        q[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = c - 1; j >= 0; --j) {
        const double tau = s_tau[j];
        if (tau != 0.0) {
            const double* aj = a + (long long)j * lda;
            for (int col = j + warp; col < c; col += nw) {
                double* qc = q + (long long)col * c;
                double t = (lane == 0) ? qc[j] : 0.0;
                for (int i = j + 1 + lane; i < c; i += 32) t = fma(aj[i], qc[i], t);
                t = warp_sum(t) * tau;
                if (lane == 0) qc[j] -= t;
                for (int i = j + 1 + lane; i < c; i += 32) qc[i] = fma(-t, aj[i], qc[i]);
            }
        }
        __syncthreads();
    }
    // W = R^T (lower triangular); in the global case R is read before W is written
    // over it, column by column of W = row by row of R, through registers
    if (in_smem) {
        for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
            const int i = (int)(e % c), j = (int)(e / c);
            W[S.off + e] = (i >= j) ? a[j + (long long)i * lda] : 0.0;
        }
    } else {
        // transpose in place: swap (i, j) and (j, i) for i > j, zero the upper part
        for (long long e = threadIdx.x; e < (long long)c * c; e += blockDim.x) {
            const int i = (int)(e % c), j = (int)(e / c);
            if (i > j) {
                const double r = a[j + (long long)i * lda];   // R(j, i), upper part
                a[i + (long long)j * lda] = r;                // W(i, j)
                a[j + (long long)i * lda] = 0.0;
            }
        }
    }
}

// Column norms of W = singular values; sort descending (rank by comparison);
// keep k = #{s_i > tau s_1}.  Writes sigma (sorted), order, k.
__global__ void sort_truncate_kernel(const SmallMat* mats, const double* W, double tau, double* sig_tmp,
                                     double* sigma, const long long* sig_off, int* order, int* k_out) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    double* st = sig_tmp + sig_off[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < c; i += nw) {
        const double* col = W + S.off + (long long)i * c;
        double a = 0.0;
        for (int r = lane; r < c; r += 32) a += col[r] * col[r];
        a = warp_sum(a);
        if (lane == 0) st[i] = sqrt(a);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
        const double si = st[i];
        int rank = 0;
        for (int j = 0; j < c; ++j) {
            const double sj = st[j];
            rank += (sj > si) || (sj == si && j < i);
        }
        sigma[sig_off[blockIdx.x] + rank] = si;
        order[sig_off[blockIdx.x] + rank] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double s1 = sigma[sig_off[blockIdx.x]];
        int k = 0;
        for (int i = 0; i < c; ++i) k += (sigma[sig_off[blockIdx.x] + i] > tau * s1) ? 1 : 0;
        if (s1 == 0.0) k = 0;
        k_out[blockIdx.x] = k;
    }
}

// Uk = V[:, order[0..k)] (c x k, ld c).
__global__ void gather_uk_kernel(const SmallMat* mats, const double* V, const int* order, const long long* sig_off,
                                 const int* k, double* Uk) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c, kk = k[blockIdx.x];
    for (long long e = threadIdx.x; e < (long long)c * kk; e += blockDim.x) {
        const int i = (int)(e % c), j = (int)(e / c);
        Uk[S.off + e] = V[S.off + i + (long long)order[sig_off[blockIdx.x] + j] * c];
    }
}

__global__ void copy_kernel(const double* src, double* dst, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = src[t];
}

// Edge operators of patch m: for every ring node t of K_m, value row
// E[2t] = Q_m[node] and flux row E[2t+1] = (1/h) sum over faces f at the node
// inside the closed K_m of (a_f / nu_f)(Q_m[node] - Q_m[nbr_f]), nu_f = 2 on a
// face lying on a patch break (held by two patches), else 1.
__global__ void edge_ops_kernel(int N, const double* aE, const double* aN, const PatchDev* patches, const int* kk,
                                const long long* q_off, const long long* e_off, const double* Q, double* E,
                                const unsigned char* xbreak, const unsigned char* ybreak) {
    const int m = blockIdx.x;
    const PatchDev P = patches[m];
    const int k = kk[m];
    const int ne = 2 * (P.x1 - P.x0) + 2 * (P.y1 - P.y0);
    const int wk = P.x1 - P.x0 + 1;
    const double* q = Q + q_off[m];
    double* e = E + e_off[m];
    const double invh = (double)N;
    for (long long w = threadIdx.x; w < (long long)ne * k; w += blockDim.x) {
        const int t = (int)(w / k), col = (int)(w % k);
        int i, j;
        ring_node(P.x0, P.x1, P.y0, P.y1, t, i, j);
        const double* qc = q + (long long)col * P.n_k;
        const int loc = (i - P.x0) + (j - P.y0) * wk;
        const double u0 = qc[loc];
        double fl = 0.0;
        const double nuh = ybreak[j] ? 0.5 : 1.0;   // x-faces lie on row j
        const double nuv = xbreak[i] ? 0.5 : 1.0;   // y-faces lie on column i
        if (i + 1 <= P.x1) fl += aE[(long long)j * N + i] * nuh * (u0 - qc[loc + 1]);
        if (i - 1 >= P.x0) fl += aE[(long long)j * N + i - 1] * nuh * (u0 - qc[loc - 1]);
        if (j + 1 <= P.y1) fl += aN[(long long)j * (N + 1) + i] * nuv * (u0 - qc[loc + wk]);
        if (j - 1 >= P.y0) fl += aN[(long long)(j - 1) * (N + 1) + i] * nuv * (u0 - qc[loc - wk]);
        e[(long long)(2 * t) * k + col] = u0;
        e[(long long)(2 * t + 1) * k + col] = invh * fl;
    }
}

// Patch block of the normal equations: B_m = sum_s cnt_s E[s]^T E[s] (k x k).
__global__ void precond_block_kernel(const int* kk, const int* ne, const long long* e_off, const double* E,
                                     const int* slot_off, const int* tr_ptr, const SmallMat* mats, double* Bm) {
    const int m = blockIdx.x;
    const int k = kk[m], ns = 2 * ne[m];
    const double* e = E + e_off[m];
    for (long long w = threadIdx.x; w < (long long)k * k; w += blockDim.x) {
        const int i = (int)(w % k), j = (int)(w / k);
        double a = 0.0;
        for (int s = 0; s < ns; ++s) {
            const int g = slot_off[m] + s;
            const int cnt = tr_ptr[g + 1] - tr_ptr[g];
            if (cnt) a += cnt * e[(long long)s * k + i] * e[(long long)s * k + j];
        }
        Bm[mats[m].off + w] = a;
    }
}

// Binv = Fi Fi^T (Fi = L^{-T}, so Binv = (L L^T)^{-1}); stored at binv_off.
__global__ void precond_inverse_kernel(const SmallMat* mats, const double* Fi, const long long* binv_off,
                                       double* Binv) {
    const SmallMat S = mats[blockIdx.x];
    const int c = S.c;
    const double* f = Fi + S.off;
    for (long long w = threadIdx.x; w < (long long)c * c; w += blockDim.x) {
        const int i = (int)(w % c), j = (int)(w / c);
        double a = 0.0;
        for (int l = max(i, j); l < c; ++l) a += f[i + (long long)l * c] * f[j + (long long)l * c];
        Binv[binv_off[blockIdx.x] + w] = a;
    }
}

}  // namespace

// position of domain-boundary node (i, j) on the global ring (counter-clockwise
// from (0, 0)), the index of its value in phi
int domain_ring_pos(int N, int i, int j) {
    if (j == 0 && i < N) return i;
    if (i == N && j < N) return N + j;
    if (j == N && i > 0) return 2 * N + (N - i);
    return 3 * N + (N - j);
}

// Orthonormal bases of the snapshot blocks (n_rows[m] x cols[m], column-major at
// snaps + snap_off[m]): shifted Cholesky-QR3, SVD of the triangular factor,
// truncation at tau sigma_1.  Outputs the kept counts, all singular values
// (descending) and the bases (n_rows x k blocks at q_off) in Q.
msp_status svd_bases(const double* snaps, long long snap_elems, const std::vector<long long>& snap_off,
                     const std::vector<int>& n_rows, const std::vector<int>& cols, double tau, cudaStream_t s,
                     DevBuf<double>& Q, std::vector<int>& k, std::vector<double>& sigma,
                     std::vector<long long>& sigma_off, std::vector<long long>& q_off, int& max_sweeps, int& max_tries,
                     float* mean_sweeps, std::vector<cudaEvent_t>* marks, std::vector<int>* sweeps_out) {
    const int np = (int)cols.size();
    max_sweeps = 0;
    max_tries = 0;
    MSP_TRY(phase_mark(marks, s));
    // ---- small-matrix layout
    std::vector<SmallMat> mats(np);
    std::vector<long long> sig_off(np);
    long long mo = 0, so = 0;
    int maxc = 0, maxn = 0;
    for (int m = 0; m < np; ++m) {
        mats[m] = SmallMat{mo, cols[m], n_rows[m], m};
        mo += (long long)cols[m] * cols[m];
        sig_off[m] = so;
        so += cols[m];
        maxc = std::max(maxc, cols[m]);
        maxn = std::max(maxn, n_rows[m]);
    }
    DevBuf<SmallMat> d_mats;
    DevBuf<long long> d_sig_off;
    MSP_TRY(upload(d_mats, mats, s));
    MSP_TRY(upload(d_sig_off, sig_off, s));
    DevBuf<double> G, L, F, Fi, T0, T1, W, V, ping, pong, sig_tmp, sig;
    DevBuf<int> order, kdev, status, sweeps, sweeps32;
    DevBuf<double> shift_scale;
    MSP_TRY(G.alloc(mo, s)); MSP_TRY(L.alloc(mo, s)); MSP_TRY(F.alloc(mo, s)); MSP_TRY(Fi.alloc(mo, s));
    MSP_TRY(T0.alloc(mo, s)); MSP_TRY(T1.alloc(mo, s));
    MSP_TRY(ping.alloc(snap_elems, s)); MSP_TRY(pong.alloc(snap_elems, s));
    MSP_TRY(sig_tmp.alloc(so, s)); MSP_TRY(sig.alloc(so, s));
    MSP_TRY(order.alloc(so, s)); MSP_TRY(kdev.alloc(np, s)); MSP_TRY(status.alloc(np, s)); MSP_TRY(sweeps.alloc(np, s));
    MSP_TRY(sweeps32.alloc(np, s));
    {
        // shift of the first pass: 11 (n c + c (c+1)) u, times |R|_F^2 (= trace of the Gram)
        std::vector<double> sc(np);
        for (int m = 0; m < np; ++m) {
            const double c = mats[m].c, n = mats[m].n;
            sc[m] = 11.0 * (n * c + c * (c + 1.0)) * 1.1102230246251565e-16;
        }
        MSP_TRY(upload(shift_scale, sc, s));
    }
    std::vector<GemmDesc> gd(np);
    DevBuf<GemmDesc> d_gd;
    MSP_TRY(d_gd.alloc(np, s));
    OzakiWork ozw;
    const bool tc = fp64_gemm_engine() == MSP_GEMM_TENSOR_CORES;
    auto run_gemm = [&](bool transA, int max_m, int max_n, unsigned flags = 0) -> msp_status {
        MSP_CUDA(cudaMemcpyAsync(d_gd.p, gd.data(), sizeof(GemmDesc) * np, cudaMemcpyHostToDevice, s));
        if (tc && ozaki_gemm_supported(gd)) {
            MSP_TRY(ozaki_gemm_batched(gd, d_gd.p, transA, false, s, ozw));
            MSP_TRY(ozaki_check(ozw, s));   // synchronises
        } else {
            gemm_batched(d_gd.p, np, max_m, max_n, transA, s, flags);
        }
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaStreamSynchronize(s));   // descriptors are reused
        return MSP_OK;
    };
    const double* X = snaps;
    double* Tacc = T0.p;
    double* Tnew = T1.p;
    double* outs[3] = {ping.p, pong.p, ping.p};
    std::vector<int> hstat(np);
    for (int pass = 0; pass < 3; ++pass) {
        double* Y = outs[pass];
        // Gram G = X^T X
        for (int m = 0; m < np; ++m) {
            const long long so_ = snap_off[m];
            gd[m] = GemmDesc{X + so_, X + so_, G.p + mats[m].off, mats[m].c, mats[m].c, mats[m].n,
                             mats[m].n, mats[m].n, mats[m].c, 1.0, 0.0};
            gd[m].lower = 1;   // the Cholesky reads the lower triangle only
        }
        MSP_TRY(run_gemm(true, maxc, maxc, kGemmStructured));
        chol_factor_kernel<<<np, 256, 0, s>>>(d_mats.p, G.p, L.p, F.p, Fi.p, shift_scale.p, pass == 0, status.p);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaMemcpyAsync(hstat.data(), status.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        for (int m = 0; m < np; ++m) max_tries = std::max(max_tries, hstat[m]);
        for (int m = 0; m < np; ++m)
            if (hstat[m] < 0) {
                set_error("basis extraction: Cholesky-QR breakdown on patch " + std::to_string(m) + " (pass " +
                          std::to_string(pass) + ")");
                return MSP_ERR_BREAKDOWN;
            }
        // Y = X Fi
        for (int m = 0; m < np; ++m) {
            const long long so_ = snap_off[m];
            gd[m] = GemmDesc{X + so_, Fi.p + mats[m].off, Y + so_, mats[m].n, mats[m].c, mats[m].c,
                             mats[m].n, mats[m].c, mats[m].n, 1.0, 0.0};
            gd[m].b_upper = 1;   // Fi = L^{-T} is upper triangular
        }
        MSP_TRY(run_gemm(false, maxn, maxc, kGemmStructured));
        // T accumulation: Tacc <- F Tacc
        if (pass == 0) {
            copy_kernel<<<1024, 256, 0, s>>>(F.p, Tacc, mo);
            count_launches(1);
            MSP_CUDA(cudaGetLastError());
        } else {
            for (int m = 0; m < np; ++m)
                gd[m] = GemmDesc{F.p + mats[m].off, Tacc + mats[m].off, Tnew + mats[m].off, mats[m].c, mats[m].c,
                                 mats[m].c, mats[m].c, mats[m].c, mats[m].c, 1.0, 0.0};
            MSP_TRY(run_gemm(false, maxc, maxc));
            std::swap(Tacc, Tnew);
        }
        X = Y;
    }
    MSP_TRY(phase_mark(marks, s));
    // ---- SVD of the triangular factor
    MSP_TRY(W.alloc(mo, s));
    MSP_TRY(V.alloc(mo, s));
    if (maxc > 2 * kJacMaxPairs) {
        set_error("basis extraction: more than " + std::to_string(2 * kJacMaxPairs) + " snapshot columns on a patch");
        return MSP_ERR_INVALID_ARG;
    }
    {
        int dev = 0, optin = 0;
        MSP_CUDA(cudaGetDevice(&dev));
        MSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // pairs of columns both below 1e-3 tau sigma_1 (|T|_F / sqrt(c) <= sigma_1) are not rotated
        const double small_rel = 1e-3 * tau / std::sqrt((double)std::max(maxc, 1));
        // the largest blocks first (their sweeps cost the most), so the last wave is short
        std::vector<SmallMat> by_size(mats);
        std::stable_sort(by_size.begin(), by_size.end(), [](const SmallMat& a, const SmallMat& b) { return a.c > b.c; });
        DevBuf<SmallMat> d_by_size;
        MSP_TRY(upload(d_by_size, by_size, s));
        if (svd_mixed()) {
            // FP32 sweeps on (float) T^T from V = I, then V re-orthogonalised in FP64
            // by two Newton-Schulz steps (orthogonal to ~1e-6 -> ~1e-12 -> rounding),
            // W = T^T V; the FP64 sweeps below then start from nearly orthogonal
            // columns and converge in a few sweeps.
            cudaFuncAttributes fa{};
            MSP_CUDA(cudaFuncGetAttributes(&fa, jacobi_svd32_kernel));
            const long long dyn_max = (long long)optin - (long long)fa.sharedSizeBytes - 1024;
            int c32 = 0;
            while (2LL * (c32 + 1) * (c32 + 2) * (long long)sizeof(float) <= dyn_max) ++c32;
            c32 = std::min(c32, maxc);
            const size_t sm32 = 2 * (size_t)c32 * (c32 + 1) * sizeof(float);
            MSP_CUDA(cudaFuncSetAttribute(jacobi_svd32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32));
            // FP32 scratch of the blocks too large for shared memory (2 c^2 floats
            // each): the second Cholesky-QR output buffer, free now, when it holds
            // them all (sum of c^2 <= sum of n c doubles)
            DevBuf<float> scratch32;
            float* scr = reinterpret_cast<float*>(pong.p);
            if (maxc > c32 && snap_elems < mo) {
                MSP_TRY(scratch32.alloc(2 * (size_t)mo, s));
                scr = scratch32.p;
            }
            jacobi_svd32_kernel<<<np, 512, sm32, s>>>(d_by_size.p, Tacc, scr, V.p, 30,
                                                      (float)(maxc * 5.96e-8), (float)small_rel, c32, sweeps32.p);
            count_launches(1);
            MSP_CUDA(cudaGetLastError());
            double* Vp = V.p;
            double* Vq = L.p;
            for (int it = 0; it < 2; ++it) {
                for (int m = 0; m < np; ++m) {
                    const int c = mats[m].c;
                    gd[m] = GemmDesc{Vp + mats[m].off, Vp + mats[m].off, G.p + mats[m].off, c, c, c, c, c, c, 1.0, 0.0};
                }
                MSP_TRY(run_gemm(true, maxc, maxc));
                newton_schulz_kernel<<<np, 256, 0, s>>>(d_mats.p, G.p);
                count_launches(1);
                MSP_CUDA(cudaGetLastError());
                for (int m = 0; m < np; ++m) {
                    const int c = mats[m].c;
                    gd[m] = GemmDesc{Vp + mats[m].off, G.p + mats[m].off, Vq + mats[m].off, c, c, c, c, c, c, 1.0, 0.0};
                }
                MSP_TRY(run_gemm(false, maxc, maxc));
                std::swap(Vp, Vq);
            }
            // two swaps: the re-orthogonalised V is back in V
            for (int m = 0; m < np; ++m) {
                const int c = mats[m].c;
                gd[m] = GemmDesc{Tacc + mats[m].off, V.p + mats[m].off, W.p + mats[m].off, c, c, c, c, c, c, 1.0, 0.0};
            }
            MSP_TRY(run_gemm(true, maxc, maxc));
        } else if (svd_qr()) {
            cudaFuncAttributes fq{};
            MSP_CUDA(cudaFuncGetAttributes(&fq, qrcp_kernel));
            const long long dyn_max = (long long)optin - (long long)fq.sharedSizeBytes - 1024;
            int cq = 0;
            while ((long long)(cq + 1) * (cq + 2) * (long long)sizeof(double) <= dyn_max) ++cq;
            cq = std::min(cq, maxc);
            const size_t smq = (size_t)cq * (cq + 1) * sizeof(double);
            MSP_CUDA(cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
            qrcp_kernel<<<np, 512, smq, s>>>(d_by_size.p, Tacc, W.p, V.p, cq);
            count_launches(1);
            MSP_CUDA(cudaGetLastError());
        } else {
            jacobi_init_kernel<<<np, 256, 0, s>>>(d_mats.p, Tacc, W.p, V.p);
            count_launches(1);
            MSP_CUDA(cudaGetLastError());
        }
        MSP_TRY(phase_mark(marks, s));
        // largest order whose W is held in shared memory: the opt-in limit per
        // block less the kernel's static shared memory
        cudaFuncAttributes fa{};
        MSP_CUDA(cudaFuncGetAttributes(&fa, jacobi_svd_kernel));
        const long long dyn_max = (long long)optin - (long long)fa.sharedSizeBytes - 1024;
        int c64 = 0;
        while ((long long)(c64 + 1) * (c64 + 2) * (long long)sizeof(double) <= dyn_max) ++c64;
        c64 = std::min(c64, maxc);
        const size_t sm64 = (size_t)c64 * (c64 + 1) * sizeof(double);
        MSP_CUDA(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64));
        jacobi_svd_kernel<<<np, 512, sm64, s>>>(d_by_size.p, W.p, V.p, 40, maxc * 1.12e-16, small_rel, c64, sweeps.p);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        MSP_TRY(phase_mark(marks, s));
    }
    sort_truncate_kernel<<<np, 256, 0, s>>>(d_mats.p, W.p, tau, sig_tmp.p, sig.p, d_sig_off.p, order.p, kdev.p);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    k.resize(np);
    sigma.resize(so);
    sigma_off = sig_off;
    {
        std::vector<int> sw(np);
        MSP_CUDA(cudaMemcpyAsync(sw.data(), sweeps.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        for (int v : sw) max_sweeps = std::max(max_sweeps, v);
        if (sweeps_out) *sweeps_out = sw;
        if (mean_sweeps) {
            double t = 0.0;
            for (int v : sw) t += v;
            *mean_sweeps = np > 0 ? (float)(t / np) : 0.f;
        }
    }
    MSP_CUDA(cudaMemcpyAsync(k.data(), kdev.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaMemcpyAsync(sigma.data(), sig.p, sizeof(double) * so, cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    // ---- Q_m = Q3 U_T[:, :k]
    q_off.resize(np);
    long long qo = 0;
    int maxk = 0;
    for (int m = 0; m < np; ++m) {
        q_off[m] = qo;
        qo += (long long)n_rows[m] * k[m];
        maxk = std::max(maxk, k[m]);
    }
    MSP_TRY(Q.alloc(std::max<long long>(qo, 1), s));
    gather_uk_kernel<<<np, 256, 0, s>>>(d_mats.p, V.p, order.p, d_sig_off.p, kdev.p, G.p);   // Uk into G
    MSP_CUDA(cudaGetLastError());
    count_launches(1);
    for (int m = 0; m < np; ++m) {
        const long long so_ = snap_off[m];
        gd[m] = GemmDesc{X + so_, G.p + mats[m].off, Q.p + q_off[m], mats[m].n, k[m], mats[m].c,
                         mats[m].n, mats[m].c, mats[m].n, 1.0, 0.0};
    }
    MSP_TRY(run_gemm(false, maxn, std::max(maxk, 1)));
    MSP_TRY(phase_mark(marks, s));
    return MSP_OK;
}

msp_status build_basis(Medium& M, double tau, int precision, cudaStream_t s, Basis& B) {
    (void)precision;
    const int np = (int)M.patches.size();
    B.N = M.N; B.mx = M.mx; B.my = M.my; B.xb = M.xb; B.yb = M.yb; B.patches = M.patches;
    B.device = M.device;
    {
        std::vector<long long> snap_off(np);
        std::vector<int> n_rows(np), cols(np);
        for (int m = 0; m < np; ++m) {
            snap_off[m] = M.patches[m].snap_offset;
            n_rows[m] = M.patches[m].n_k;
            cols[m] = M.patches[m].cols;
        }
        MSP_TRY(svd_bases(M.snaps.p, M.snap_elems, snap_off, n_rows, cols, tau, s, B.Q, B.k, B.sigma, B.sigma_off, B.q_off,
                          B.max_jacobi_sweeps, B.max_cholqr_tries, &B.mean_jacobi_sweeps, &B.ext_ev, &B.jac_sweeps));
        B.jac_cols.assign(cols.begin(), cols.end());
    }
    return finish_basis(B, M.aE.p, M.aN.p, s);
}

// Online operators of a basis whose geometry (N, patches, breaks), Q_m, k_m and
// sigma are set: coefficient offsets, skeleton and row tables, edge operators (from
// the FP64 face coefficients aE, aN on the device), patch-block preconditioner and
// the block-row factor.  Shared by the extraction and by msp_load_basis.
msp_status finish_basis(Basis& B, const double* aE_dev, const double* aN_dev, cudaStream_t s) {
    const int np = (int)B.patches.size();
    {
        const size_t nf = (size_t)(B.N + 1) * B.N;
        MSP_TRY(B.aE.alloc(nf, s));
        MSP_TRY(B.aN.alloc(nf, s));
        MSP_CUDA(cudaMemcpyAsync(B.aE.p, aE_dev, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(B.aN.p, aN_dev, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
    }
    B.c_off.resize(np + 1);
    int co = 0;
    for (int m = 0; m < np; ++m) {
        B.c_off[m] = co;
        co += B.k[m];
    }
    B.c_off[np] = co;
    B.Np = co;
    // G as scratch for the precondtioner blocks below
    long long mo = 0;
    for (int m = 0; m < np; ++m) mo += (long long)B.patches[m].cols * B.patches[m].cols;
    DevBuf<double> G, L, F, Fi, shift_scale;
    DevBuf<int> status;
    MSP_TRY(G.alloc(mo, s)); MSP_TRY(L.alloc(mo, s)); MSP_TRY(F.alloc(mo, s)); MSP_TRY(Fi.alloc(mo, s));
    MSP_TRY(shift_scale.alloc(np, s));
    MSP_TRY(status.alloc(np, s));
    std::vector<int> hstat(np);


    // ---- online tables (host): skeleton nodes, rows of P~, transpose lists
    const int N = B.N;
    B.n_e.resize(np);
    B.slot_off.resize(np + 1);
    B.e_off.resize(np);
    int slots = 0;
    long long eo = 0;
    for (int m = 0; m < np; ++m) {
        const PatchDev& P = B.patches[m];
        B.n_e[m] = 2 * (P.x1 - P.x0) + 2 * (P.y1 - P.y0);
        B.slot_off[m] = slots;
        slots += 2 * B.n_e[m];
        B.e_off[m] = eo;
        eo += (long long)2 * B.n_e[m] * B.k[m];
    }
    B.slot_off[np] = slots;
    B.n_slots = slots;
    // skeleton nodes in row-major node order, each with the (patch, ring position)
    // pairs that hold it in patch order: a counting pass over the nodes of the grid
    const long long nn = (long long)(N + 1) * (N + 1);
    std::vector<int> node_cnt(nn + 1, 0);
    for (int m = 0; m < np; ++m) {
        const PatchDev& P = B.patches[m];
        for (int t = 0; t < B.n_e[m]; ++t) {
            int i, j;
            ring_node(P.x0, P.x1, P.y0, P.y1, t, i, j);
            ++node_cnt[(long long)j * (N + 1) + i + 1];
        }
    }
    for (long long v = 0; v < nn; ++v) node_cnt[v + 1] += node_cnt[v];
    std::vector<int> holder(node_cnt[nn]);   // slot of (m, t), grouped by node, patches ascending
    {
        std::vector<int> cur(node_cnt.begin(), node_cnt.end() - 1);
        for (int m = 0; m < np; ++m) {
            const PatchDev& P = B.patches[m];
            for (int t = 0; t < B.n_e[m]; ++t) {
                int i, j;
                ring_node(P.x0, P.x1, P.y0, P.y1, t, i, j);
                holder[cur[(long long)j * (N + 1) + i]++] = B.slot_off[m] + 2 * t;
            }
        }
    }
    std::vector<int> row_ptr{0}, row_slot, row_bnd, sk_ptr{0}, sk_slot, sk_node, sk_ring;
    const unsigned neg = 0x80000000u;
    for (long long v = 0; v < nn; ++v) {
        const int h0 = node_cnt[v], h1 = node_cnt[v + 1];
        if (h0 == h1) continue;
        const int j = (int)(v / (N + 1)), i = (int)(v % (N + 1));
        const bool bnd = (i == 0 || i == N || j == 0 || j == N);
        for (int h = h0; h < h1; ++h) sk_slot.push_back(holder[h]);
        sk_ptr.push_back((int)sk_slot.size());
        sk_node.push_back((int)v);
        sk_ring.push_back(bnd ? domain_ring_pos(N, i, j) : -1);
        if (bnd) {
            if (B.no_boundary_rows) continue;   // constrained variant: the boundary data hold exactly
            for (int h = h0; h < h1; ++h) {
                row_slot.push_back(holder[h]);
                row_ptr.push_back((int)row_slot.size());
                row_bnd.push_back(domain_ring_pos(N, i, j));
            }
        } else {
            for (int h = h0 + 1; h < h1; ++h) {
                row_slot.push_back(holder[h0]);
                row_slot.push_back((int)((unsigned)holder[h] | neg));
                row_ptr.push_back((int)row_slot.size());
                row_bnd.push_back(-1);
            }
            for (int h = h0; h < h1; ++h) row_slot.push_back(holder[h] + 1);
            row_ptr.push_back((int)row_slot.size());
            row_bnd.push_back(-1);
        }
    }
    B.n_rows = (int)row_bnd.size();
    B.n_skel = (int)sk_node.size();
    // transpose: per slot, the rows touching it (rows ascending), by a counting pass
    std::vector<int> tr_ptr(slots + 1, 0), tr_ent(row_slot.size());
    for (size_t e = 0; e < row_slot.size(); ++e) ++tr_ptr[((unsigned)row_slot[e] & 0x7fffffffu) + 1];
    for (int g = 0; g < slots; ++g) tr_ptr[g + 1] += tr_ptr[g];
    {
        std::vector<int> cur(tr_ptr.begin(), tr_ptr.end() - 1);
        for (int r = 0; r < B.n_rows; ++r)
            for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                const unsigned v = (unsigned)row_slot[e];
                tr_ent[cur[v & 0x7fffffffu]++] = (int)((unsigned)r | (v & neg));
            }
    }
    MSP_TRY(upload(B.row_ptr, row_ptr, s)); MSP_TRY(upload(B.row_slot, row_slot, s)); MSP_TRY(upload(B.row_bnd, row_bnd, s));
    MSP_TRY(upload(B.tr_ptr, tr_ptr, s)); MSP_TRY(upload(B.tr_ent, tr_ent, s));
    MSP_TRY(upload(B.sk_ptr, sk_ptr, s)); MSP_TRY(upload(B.sk_slot, sk_slot, s)); MSP_TRY(upload(B.sk_node, sk_node, s));
    MSP_TRY(upload(B.sk_ring, sk_ring, s));
    MSP_TRY(upload(B.d_c_off, B.c_off, s)); MSP_TRY(upload(B.d_k, B.k, s)); MSP_TRY(upload(B.d_slot_off, B.slot_off, s));
    MSP_TRY(upload(B.d_ne, B.n_e, s)); MSP_TRY(upload(B.d_q_off, B.q_off, s)); MSP_TRY(upload(B.d_e_off, B.e_off, s));
    MSP_TRY(upload(B.d_patches, B.patches, s));
    std::vector<unsigned char> xbr(N + 1, 0), ybr(N + 1, 0);
    for (size_t i = 1; i + 1 < B.xb.size(); ++i) xbr[B.xb[i]] = 1;
    for (size_t i = 1; i + 1 < B.yb.size(); ++i) ybr[B.yb[i]] = 1;
    DevBuf<unsigned char> d_xbr, d_ybr;
    MSP_TRY(upload(d_xbr, xbr, s)); MSP_TRY(upload(d_ybr, ybr, s));
    MSP_TRY(B.E.alloc(std::max<long long>(eo, 1), s));
    edge_ops_kernel<<<np, 256, 0, s>>>(N, aE_dev, aN_dev, B.d_patches.p, B.d_k.p, B.d_q_off.p, B.d_e_off.p, B.Q.p,
                                       B.E.p, d_xbr.p, d_ybr.p);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    // ---- preconditioner blocks (k x k) and their inverses
    std::vector<SmallMat> kmats(np);
    B.binv_off.resize(np);
    long long ko = 0;
    for (int m = 0; m < np; ++m) {
        kmats[m] = SmallMat{ko, B.k[m], 0};
        B.binv_off[m] = ko;
        ko += (long long)B.k[m] * B.k[m];
    }
    DevBuf<SmallMat> d_kmats;
    MSP_TRY(upload(d_kmats, kmats, s));
    MSP_TRY(upload(B.d_binv_off, B.binv_off, s));
    MSP_TRY(B.Binv.alloc(std::max<long long>(ko, 1), s));
    precond_block_kernel<<<np, 256, 0, s>>>(B.d_k.p, B.d_ne.p, B.d_e_off.p, B.E.p, B.d_slot_off.p, B.tr_ptr.p,
                                            d_kmats.p, G.p);
    count_launches(1);
    chol_factor_kernel<<<np, 256, 0, s>>>(d_kmats.p, G.p, L.p, F.p, Fi.p, shift_scale.p, 0, status.p);
    count_launches(1);
    precond_inverse_kernel<<<np, 256, 0, s>>>(d_kmats.p, Fi.p, B.d_binv_off.p, B.Binv.p);
    // keep L_m^{-T} of every patch block: the scaling of the online factor
    MSP_TRY(B.bt_Fi.alloc(std::max<long long>(ko, 1), s));
    if (ko > 0) MSP_CUDA(cudaMemcpyAsync(B.bt_Fi.p, Fi.p, sizeof(double) * ko, cudaMemcpyDeviceToDevice, s));
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    MSP_CUDA(cudaMemcpyAsync(hstat.data(), status.p, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    for (int m = 0; m < np; ++m)
        if (hstat[m] < 0 && B.k[m] > 0) {
            set_error("msp_extract_basis: preconditioner block of patch " + std::to_string(m) + " is not positive definite");
            return MSP_ERR_BREAKDOWN;
        }
    // ---- block-tridiagonal factor of the scaled normal matrix (online preconditioner)
    MSP_TRY(phase_mark(B.ext_ev.empty() ? nullptr : &B.ext_ev, s));
    MSP_TRY(build_online_factor(B, row_ptr, row_slot, s));
    MSP_TRY(phase_mark(B.ext_ev.empty() ? nullptr : &B.ext_ev, s));
    return MSP_OK;
}

}  // namespace msp
