// Direct local solver of the kinetic slab (Sec. 4, Eq. RTE with the
// Henyey-Greenstein collision of Eq. HG; the offline local problem of
// Eq. rte_random on a buffered patch).
//
// Discrete operator on the nodes i = 0..nn-1 of a buffered patch, unknowns
// f_i in R^{n_v} at every node (the incoming components at the two ends carry
// identity rows whose right-hand side is the random datum):
//
//   D_i f_i + L_i f_{i-1} + U_i f_{i+1} = b_i,
//   D_i = diag(a_l + sigma_l/eps) - Kw/eps,    a_l = |v_l|/dx,
//   L_i = -diag(a_l [v_l > 0]),  U_i = -diag(a_l [v_l < 0]).
//
// Block LU over the nodes: S_0 = D_0, S_i = D_i - L_i S_{i-1}^{-1} U_{i-1}; the
// coupling touches only the (v>0 rows, v<0 columns) quadrant.  Every S_i is a
// nonsingular M-matrix (weakly row-diagonally dominant since the gain row sums
// equal the loss rates, strictly at the identity rows), so neither the block
// elimination nor the Gauss-Jordan inversion of each S_i needs pivoting.  The
// factor kernel keeps W_i = S_i^{-1} for every node (one CTA per patch, the
// n_v x n_v block in registers over a 16 x 16 thread grid).
//
// The solve kernel takes one CTA per (patch, 32 samples), one sample per lane,
// and refines in FP64: r = b - A f (FP64, sweeping a three-node window of f
// through shared memory), forward y_i = W_i (r_i - L_i y_{i-1}), backward
// x_i = y_i - W_i U_i x_{i+1}, f += x.  With the FP64 factor one pass solves
// and a second confirms; with the FP32 factor each pass gains about seven
// digits.  Stop when max |r_l| / D_ll <= tol max |f|.
#include "kinetic_internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>

namespace msp {
namespace {

constexpr int kKdThreads = 256;
constexpr int kKdG = 32;        // samples per CTA of the solve, one per lane
constexpr int kKdLd = 33;       // padded row stride of the [velocity][sample] tiles
constexpr int kKdMaxNv = 128;
constexpr int kKdMaxPasses = 16;   // corrections per solve at most

struct KdArgs {
    int N, n_v, S, max_passes;
    double eps, tol;
    uint64_t seed;
    const double* v;
    const double* Kw;
    const double* sigma;
    const KPatchDev* patches;
    const long long* node_off;
    double* f;
    double* snaps;
    int* stats;
};

__device__ __forceinline__ bool kd_identity(int i, int nn, double vl) {
    return (i == 0 && vl > 0.0) || (i == nn - 1 && vl < 0.0);
}

// One CTA per patch.  Thread (ty, tx) of the 16 x 16 grid owns the entries
// (ty + 16 a, tx + 16 b), a, b < RA, of the n_v x n_v block (n_v <= 16 RA).
template <class T, int RA>
__global__ void __launch_bounds__(kKdThreads) kd_factor_kernel(KdArgs A, T* W) {
    __shared__ T colk[2][kKdMaxNv];
    __shared__ T rowk[2][kKdMaxNv];
    const int m = blockIdx.x, nv = A.n_v;
    const KPatchDev P = A.patches[m];
    const int nn = P.X1 - P.X0 + 1;
    const long long n2 = (long long)nv * nv;
    const double dx = 1.0 / A.N, ie = 1.0 / A.eps;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T x[RA][RA];
    T* Wm = W + A.node_off[m] * n2;
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RA; ++b) x[a][b] = T(0);
    int par = 0;
    for (int i = 0; i < nn; ++i) {
        // S_i over W_{i-1}: each entry depends only on the previous value at the same place
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int r = ty + 16 * a;
            if (r >= nv) continue;
            const double vr = A.v[r], ar = fabs(vr) / dx;
            const bool ident = kd_identity(i, nn, vr);
#pragma unroll
            for (int b = 0; b < RA; ++b) {
                const int c = tx + 16 * b;
                if (c >= nv) continue;
                double s;
                if (ident) {
                    s = (r == c) ? 1.0 : 0.0;
                } else {
                    s = -ie * A.Kw[(long long)r * nv + c];
                    if (r == c) s += ar + ie * A.sigma[r];
                    const double vc = A.v[c];
                    if (i > 0 && vr > 0.0 && vc < 0.0) s -= ar * (double)x[a][b] * (fabs(vc) / dx);
                }
                x[a][b] = (T)s;
            }
        }
        // Gauss-Jordan inversion in place, no pivoting; column and row k are
        // published through alternating buffers, one barrier per step
        for (int k = 0; k < nv; ++k) {
            const int kq = k >> 4;   // register block of row / column k (selected by predicates)
            if (tx == (k & 15)) {
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    const int r = ty + 16 * a;
#pragma unroll
                    for (int b = 0; b < RA; ++b)
                        if (b == kq && r < nv) colk[par][r] = x[a][b];
                }
            }
            if (ty == (k & 15)) {
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    if (a != kq) continue;
#pragma unroll
                    for (int b = 0; b < RA; ++b) {
                        const int c = tx + 16 * b;
                        if (c < nv) rowk[par][c] = x[a][b];
                    }
                }
            }
            __syncthreads();
            const T p = T(1) / rowk[par][k];
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const int r = ty + 16 * a;
                if (r >= nv) continue;
                const T cr = colk[par][r] * p;
#pragma unroll
                for (int b = 0; b < RA; ++b) {
                    const int c = tx + 16 * b;
                    if (c >= nv) continue;
                    if (r != k) {
                        x[a][b] = (c != k) ? x[a][b] - cr * rowk[par][c] : -cr;
                    } else {
                        x[a][b] = (c != k) ? rowk[par][c] * p : p;
                    }
                }
            }
            par ^= 1;
        }
        T* Wi = Wm + (long long)i * n2;
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int r = ty + 16 * a;
            if (r >= nv) continue;
#pragma unroll
            for (int b = 0; b < RA; ++b) {
                const int c = tx + 16 * b;
                if (c < nv) Wi[(long long)r * nv + c] = x[a][b];
            }
        }
    }
}

__device__ __forceinline__ double kd_max_block(double x, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    __syncthreads();
    return t;
}

// Incoming datum of sample s, velocity l: entries 0..n_v/2-1 of the patch's data
// are the positive velocities at X0 (ascending), n_v/2.. the negative ones at X1.
__device__ __forceinline__ double kd_datum(const KdArgs& A, int m, int s, int l, double vl) {
    const int nv = A.n_v;
    const int t = (vl > 0.0) ? l - nv / 2 : nv / 2 + l;
    const double2 z = gaussian_pair(A.seed, (uint32_t)(t >> 1), (uint32_t)s, (uint32_t)m, kTagKinetic);
    return (t & 1) ? z.y : z.x;
}

// One CTA per (patch, 32 samples); warp w owns the velocity rows w + 8 j (j < RJ),
// lane = sample.  y (in T) shares the f layout: [node][velocity][sample]; it holds
// the residual after the residual sweep and y_i after the forward sweep.
template <class T, int RJ>
__global__ void __launch_bounds__(kKdThreads) kd_solve_kernel(KdArgs A, const T* W, T* y) {
    extern __shared__ __align__(16) unsigned char kd_dyn[];
    __shared__ double red[32];
    __shared__ double c_v[kKdMaxNv], c_a[kKdMaxNv], c_d[kKdMaxNv];
    const int nv = A.n_v, m = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const KPatchDev P = A.patches[m];
    const int nn = P.X1 - P.X0 + 1;
    const int s = blockIdx.y * kKdG + lane;
    const bool live = s < A.S;
    const long long n2 = (long long)nv * nv, S = A.S;
    const long long base = A.node_off[m];
    const T* Wm = W + base * n2;
    double* Fw = reinterpret_cast<double*>(kd_dyn);                 // 3 x nv x kKdLd (FP64 window)
    T* Z = reinterpret_cast<T*>(Fw + 3 * nv * kKdLd);               // nv x kKdLd (matvec input)
    const double dx = 1.0 / A.N, ie = 1.0 / A.eps;
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
        c_v[l] = A.v[l];
        c_a[l] = fabs(A.v[l]) / dx;
        c_d[l] = c_a[l] + ie * A.sigma[l];
    }
    __syncthreads();
    auto fidx = [&](int i, int l) { return ((base + i) * nv + l) * S + s; };
    const int nneg = nv / 2;   // velocities ascend: the first n_v/2 are negative
    int pass = 0;
    bool converged = false;
    for (;; ++pass) {
        // ---- residual sweep: r_i = b_i - (A f)_i, stored in y (rounded to T)
        double rmax = 0.0, fmx = 0.0;
        if (pass == 0) {
            // f = 0: the residual is the data at the identity rows
            for (int i = 0; i < nn; ++i) {
#pragma unroll
                for (int j = 0; j < RJ; ++j) {
                    const int l = warp + 8 * j;
                    if (l >= nv || !live) continue;
                    const double r = kd_identity(i, nn, c_v[l]) ? kd_datum(A, m, s, l, c_v[l]) : 0.0;
                    rmax = fmax(rmax, fabs(r));
                    y[fidx(i, l)] = (T)r;
                }
            }
        } else {
            // window slots: node q lives in slot q % 3
            auto load = [&](int node) {
                double* dst = Fw + (node % 3) * nv * kKdLd;
#pragma unroll
                for (int j = 0; j < RJ; ++j) {
                    const int l = warp + 8 * j;
                    if (l < nv) dst[l * kKdLd + lane] = live ? A.f[fidx(node, l)] : 0.0;
                }
            };
            load(0);
            for (int i = 0; i < nn; ++i) {
                if (i + 1 < nn) load(i + 1);
                __syncthreads();
                const double* Fi = Fw + (i % 3) * nv * kKdLd;
                const double* Fp = Fw + ((i + 2) % 3) * nv * kKdLd;   // node i-1 (unused at i = 0)
                const double* Fn = Fw + ((i + 1) % 3) * nv * kKdLd;   // node i+1 (unused at i = nn-1)
#pragma unroll
                for (int j = 0; j < RJ; ++j) {
                    const int l = warp + 8 * j;
                    if (l >= nv) continue;
                    const double vl = c_v[l], fi = Fi[l * kKdLd + lane];
                    double r, scale;
                    if (kd_identity(i, nn, vl)) {
                        r = (live ? kd_datum(A, m, s, l, vl) : 0.0) - fi;
                        scale = 1.0;
                    } else {
                        const double* kr = A.Kw + (long long)l * nv;
                        double g0 = 0.0, g1 = 0.0;
                        int k = 0;
                        for (; k + 1 < nv; k += 2) {
                            g0 = fma(__ldg(kr + k), Fi[k * kKdLd + lane], g0);
                            g1 = fma(__ldg(kr + k + 1), Fi[(k + 1) * kKdLd + lane], g1);
                        }
                        if (k < nv) g0 = fma(__ldg(kr + k), Fi[k * kKdLd + lane], g0);
                        const double nb = vl > 0.0 ? Fp[l * kKdLd + lane] : Fn[l * kKdLd + lane];
                        r = -(c_d[l] * fi - ie * (g0 + g1) - c_a[l] * nb);
                        scale = 1.0 / c_d[l];
                    }
                    if (live) {
                        rmax = fmax(rmax, fabs(r) * scale);
                        fmx = fmax(fmx, fabs(fi));
                        y[fidx(i, l)] = (T)r;
                    }
                }
                __syncthreads();   // the slot of node i-1 is reloaded with node i+2 next
            }
        }
        rmax = kd_max_block(rmax, red);
        fmx = kd_max_block(fmx, red);
        if ((pass > 0 && rmax <= A.tol * fmx) || rmax == 0.0) {   // rmax = 0: zero data, f = 0
            converged = true;
            break;
        }
        if (pass >= A.max_passes) break;
        // ---- forward sweep: y_i = W_i (r_i + a_+ y_{i-1}[+])
        T yprev[RJ];
#pragma unroll
        for (int j = 0; j < RJ; ++j) yprev[j] = T(0);
        for (int i = 0; i < nn; ++i) {
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int l = warp + 8 * j;
                if (l >= nv) continue;
                T z = live ? y[fidx(i, l)] : T(0);
                if (i > 0 && c_v[l] > 0.0) z += (T)c_a[l] * yprev[j];
                Z[l * kKdLd + lane] = z;
            }
            __syncthreads();
            const T* Wi = Wm + (long long)i * n2;
            T acc[RJ];
#pragma unroll
            for (int j = 0; j < RJ; ++j) acc[j] = T(0);
            for (int k = 0; k < nv; ++k) {
                const T zk = Z[k * kKdLd + lane];
#pragma unroll
                for (int j = 0; j < RJ; ++j) {
                    const int l = warp + 8 * j;
                    if (l < nv) acc[j] += __ldg(Wi + (long long)l * nv + k) * zk;
                }
            }
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int l = warp + 8 * j;
                if (l >= nv) continue;
                yprev[j] = acc[j];
                if (live) y[fidx(i, l)] = acc[j];
            }
            __syncthreads();   // Z is rewritten for the next node
        }
        // ---- backward sweep: x_i = y_i + W_i[:, -] (a_- x_{i+1}[-]); f += x
        T xnext[RJ];
#pragma unroll
        for (int j = 0; j < RJ; ++j) xnext[j] = T(0);
        for (int i = nn - 1; i >= 0; --i) {
            T x[RJ];
#pragma unroll
            for (int j = 0; j < RJ; ++j) x[j] = T(0);
            if (i < nn - 1) {
#pragma unroll
                for (int j = 0; j < RJ; ++j) {
                    const int l = warp + 8 * j;
                    if (l < nneg) Z[l * kKdLd + lane] = (T)c_a[l] * xnext[j];
                }
                __syncthreads();
                const T* Wi = Wm + (long long)i * n2;
                for (int k = 0; k < nneg; ++k) {
                    const T zk = Z[k * kKdLd + lane];
#pragma unroll
                    for (int j = 0; j < RJ; ++j) {
                        const int l = warp + 8 * j;
                        if (l < nv) x[j] += __ldg(Wi + (long long)l * nv + k) * zk;
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int l = warp + 8 * j;
                if (l >= nv) continue;
                if (live) {
                    const long long q = fidx(i, l);
                    x[j] += y[q];
                    A.f[q] = (pass == 0) ? (double)x[j] : A.f[q] + (double)x[j];
                }
                xnext[j] = x[j];
            }
        }
        __syncthreads();
    }
    // restriction to K_m: node-major, velocity fastest, one sample per column
    const int i0 = P.x0 - P.X0, nk_nodes = P.x1 - P.x0 + 1;
    if (live) {
        double* out = A.snaps + P.snap_offset + (long long)s * P.n_k;
        for (int i = 0; i < nk_nodes; ++i) {
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int l = warp + 8 * j;
                if (l < nv) out[(long long)i * nv + l] = A.f[fidx(i0 + i, l)];
            }
        }
        if (warp == 0) {
            A.stats[2 * ((long long)m * A.S + s) + 0] = pass;
            A.stats[2 * ((long long)m * A.S + s) + 1] = converged ? 0 : 1;
        }
    }
}

template <class T, int RA>
msp_status launch_factor(const KdArgs& A, int M, T* W, cudaStream_t s) {
    kd_factor_kernel<T, RA><<<M, kKdThreads, 0, s>>>(A, W);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

template <class T>
msp_status factor(const KdArgs& A, int M, T* W, cudaStream_t s) {
    const int nv = A.n_v;
    if (nv <= 16) return launch_factor<T, 1>(A, M, W, s);
    if (nv <= 32) return launch_factor<T, 2>(A, M, W, s);
    if (nv <= 64) return launch_factor<T, 4>(A, M, W, s);
    return launch_factor<T, 8>(A, M, W, s);
}

template <class T, int RJ>
msp_status launch_solve(const KdArgs& A, int M, const T* W, T* y, cudaStream_t s) {
    const size_t smem = sizeof(double) * 3 * A.n_v * kKdLd + sizeof(T) * A.n_v * kKdLd;
    MSP_CUDA(cudaFuncSetAttribute(kd_solve_kernel<T, RJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(M, (A.S + kKdG - 1) / kKdG);
    kd_solve_kernel<T, RJ><<<grid, kKdThreads, smem, s>>>(A, W, y);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

template <class T>
msp_status solve(const KdArgs& A, int M, const T* W, T* y, cudaStream_t s) {
    const int nv = A.n_v;
    if (nv <= 8) return launch_solve<T, 1>(A, M, W, y, s);
    if (nv <= 16) return launch_solve<T, 2>(A, M, W, y, s);
    if (nv <= 32) return launch_solve<T, 4>(A, M, W, y, s);
    if (nv <= 64) return launch_solve<T, 8>(A, M, W, y, s);
    return launch_solve<T, 16>(A, M, W, y, s);
}

}  // namespace

msp_status kinetic_direct_sample(KMedium& K, uint64_t seed, bool mixed, double tol, int max_iter, cudaStream_t s) {
    if (K.n_v > kKdMaxNv) {
        set_error("kinetic direct solver: at most 128 velocities");
        return MSP_ERR_INVALID_ARG;
    }
    KDirect& D = K.D;
    if (D.node_off.empty()) {
        long long off = 0;
        for (auto& P : K.patches) {
            D.node_off.push_back(off);
            off += P.nn;
        }
        D.n_nodes = off;
        MSP_TRY(upload(D.d_node_off, D.node_off, s));
    }
    const size_t n2 = (size_t)K.n_v * K.n_v;
    const size_t nf = (size_t)D.n_nodes * K.n_v * K.S;
    KdArgs A{};
    A.N = K.N; A.n_v = K.n_v; A.S = K.S;
    A.max_passes = std::max(1, std::min(max_iter, kKdMaxPasses));
    A.eps = K.eps; A.tol = tol; A.seed = seed;
    A.v = K.d_v.p; A.Kw = K.d_Kw.p; A.sigma = K.d_sigma.p; A.patches = K.d_patches.p;
    A.node_off = D.d_node_off.p;
    A.snaps = K.snaps.p; A.stats = K.stats.p;
    if (D.f.n < nf) MSP_TRY(D.f.alloc(nf, s));
    A.f = D.f.p;
    if (mixed) {
        if (!D.factored32) {
            MSP_TRY(D.W32.alloc((size_t)D.n_nodes * n2, s));
            MSP_TRY(factor<float>(A, K.M, D.W32.p, s));
            D.factored32 = true;
        }
        if (D.y32.n < nf) MSP_TRY(D.y32.alloc(nf, s));
        return solve<float>(A, K.M, D.W32.p, D.y32.p, s);
    }
    if (!D.factored64) {
        MSP_TRY(D.W64.alloc((size_t)D.n_nodes * n2, s));
        MSP_TRY(factor<double>(A, K.M, D.W64.p, s));
        D.factored64 = true;
    }
    if (D.y64.n < nf) MSP_TRY(D.y64.alloc(nf, s));
    return solve<double>(A, K.M, D.W64.p, D.y64.p, s);
}

}  // namespace msp
