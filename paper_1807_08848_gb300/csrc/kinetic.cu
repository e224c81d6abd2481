// Kinetic example (Sec. 4): slab radiative transfer (Eq. RTE) with the
// Henyey-Greenstein collision (Eq. HG), discrete ordinates.
//
//   v d_x f = (1/eps) L f,  (L f)_l = sum_l' w_l' k(v_l, v_l') f_l' - sigma_l f_l
//   (Gauss-Legendre v_l, w_l; at g = 0: L f = rho - f, rho = (1/2) sum_l w_l f_l)
//   implicit upwind on nodes x_i = i/N;  incoming data f(0, v>0), f(1, v<0).
//
// Offline (Eq. rte_random): per patch and sample, i.i.d. N(0,1) incoming data on the
// buffered patch, restricted to K_m.  Isotropic media default to source iteration
// -- a transport sweep of every velocity with the lagged density, then the density
// update; anisotropic ones use the direct block solver of kinetic_direct.cu.
// Extraction: the shared SVD-basis routine.  Online (Eq. rte_cond_reduced): all
// velocity components continuous at every interface plus the incoming data, least
// squares by the normal equations, which are block tridiagonal along the chain of
// patches: factorised once (FP64 block Cholesky), solved per data set with two
// corrected-semi-normal-equation refinement steps.
#include "kinetic_internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>

namespace msp {

struct KBasis {
    int N = 0, n_v = 0, M = 0;
    std::vector<double> v;
    std::vector<KPatchDev> patches;
    std::vector<int> k;
    std::vector<double> sigma;
    std::vector<long long> sigma_off, q_off;
    std::vector<int> c_off;
    int Np = 0;
    DevBuf<double> Q;
    DevBuf<KPatchDev> d_patches;
    DevBuf<int> d_k, d_c_off;
    DevBuf<long long> d_q_off;
    DevBuf<double> d_v;
    // block-tridiagonal factor of H = P^T P: L_m (k_m x k_m, lower) and C_m (k_{m+1} x k_m)
    std::vector<long long> l_off, c_blk_off;
    DevBuf<double> Lf, Cf;
    DevBuf<long long> d_l_off, d_c_blk_off;
    int max_sweeps = 0, max_tries = 0;
};

}  // namespace msp

struct msp_kmedium_s {
    msp::KMedium K;
};
struct msp_kbasis_s {
    msp::KBasis B;
};

namespace msp {

msp_status svd_bases(const double* snaps, long long snap_elems, const std::vector<long long>& snap_off,
                     const std::vector<int>& n_rows, const std::vector<int>& cols, double tau, cudaStream_t s,
                     DevBuf<double>& Q, std::vector<int>& k, std::vector<double>& sigma,
                     std::vector<long long>& sigma_off, std::vector<long long>& q_off, int& max_sweeps, int& max_tries,
                     float* mean_sweeps = nullptr, std::vector<cudaEvent_t>* marks = nullptr,
                     std::vector<int>* sweeps_out = nullptr);

namespace {

// Gauss-Legendre nodes (ascending) and weights: Newton's method on P_n from the
// Chebyshev-like initial guesses cos(pi (i - 1/4) / (n + 1/2)), with P_n and P_n'
// from the three-term recurrence.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {   // refresh the derivative at the converged root
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = wi;
        w[n - 1 - i] = wi;
    }
}

struct KSolveArgs {
    int N, n_v, S, G;
    double eps, tol;
    int max_iter;
    uint64_t seed;
    const double* v;
    const double* w;
    const KPatchDev* patches;
    double* snaps;
    int* stats;
};

template <class T>
__device__ __forceinline__ T block_max1(T x, T* buf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) buf[warp] = x;
    __syncthreads();
    T t = (lane < nw) ? buf[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    __syncthreads();
    return t;
}

// One CTA: G samples of one patch; thread (g, l) sweeps velocity l of sample g.
// Shared: f[g][node][l], rho[g][node].
__global__ void kinetic_si_kernel(KSolveArgs A) {
    extern __shared__ double ksm[];
    __shared__ double red[32];
    const int m = blockIdx.x;
    const KPatchDev P = A.patches[m];
    const int nn = P.X1 - P.X0 + 1, nv = A.n_v, G = A.G;
    double* f = ksm;                                   // G x nn x nv
    double* rho = ksm + (long long)G * nn * nv;        // G x nn
    const int g = threadIdx.x / nv, l = threadIdx.x % nv;
    const int s = blockIdx.y * G + g;
    const bool live = g < G && s < A.S;
    const double dx = 1.0 / A.N, ie = 1.0 / A.eps;
    double vl = 0.0, a2 = 0.0, b2 = 0.0, inflow = 0.0;
    if (live) {
        vl = A.v[l];
        const double a = fabs(vl) / dx, inv = 1.0 / (a + ie);
        a2 = a * inv;
        b2 = ie * inv;
        // incoming datum: entries 0..nv/2-1 are the positive velocities at X0 (ascending),
        // nv/2.. the negative ones at X1 (ascending)
        const int t = (vl > 0.0) ? l - nv / 2 : nv / 2 + l;
        const double2 z = gaussian_pair(A.seed, (uint32_t)(t >> 1), (uint32_t)s, (uint32_t)m, kTagKinetic);
        inflow = (t & 1) ? z.y : z.x;
    }
    for (int t = threadIdx.x; t < G * nn; t += blockDim.x) rho[t] = 0.0;
    __syncthreads();
    double* fg = f + (long long)(live ? g : 0) * nn * nv;
    double* rg = rho + (live ? g : 0) * nn;
    int it = 0;
    bool done = false;
    for (; it < A.max_iter && !done; ++it) {
        // transport sweep with the lagged density
        if (live) {
            if (vl > 0.0) {
                double fp = inflow;
                fg[l] = fp;
                for (int i = 1; i < nn; ++i) {
                    fp = a2 * fp + b2 * rg[i];
                    fg[(long long)i * nv + l] = fp;
                }
            } else {
                double fp = inflow;
                fg[(long long)(nn - 1) * nv + l] = fp;
                for (int i = nn - 2; i >= 0; --i) {
                    fp = a2 * fp + b2 * rg[i];
                    fg[(long long)i * nv + l] = fp;
                }
            }
        }
        __syncthreads();
        // density update and the change in it
        double dmax = 0.0, rmax = 0.0;
        for (int t = threadIdx.x; t < G * nn; t += blockDim.x) {
            const int gg = t / nn, i = t - gg * nn;
            if (blockIdx.y * G + gg >= A.S) continue;
            const double* fi = f + ((long long)gg * nn + i) * nv;
            double r = 0.0;
            for (int ll = 0; ll < nv; ++ll) r += A.w[ll] * fi[ll];
            r *= 0.5;
            dmax = fmax(dmax, fabs(r - rho[t]));
            rmax = fmax(rmax, fabs(r));
            rho[t] = r;
        }
        dmax = block_max1(dmax, red);
        rmax = block_max1(rmax, red);
        done = dmax <= A.tol * rmax;
    }
    // one more sweep so that f matches the final density exactly
    if (live) {
        if (vl > 0.0) {
            double fp = inflow;
            for (int i = 1; i < nn; ++i) {
                fp = a2 * fp + b2 * rg[i];
                fg[(long long)i * nv + l] = fp;
            }
        } else {
            double fp = inflow;
            for (int i = nn - 2; i >= 0; --i) {
                fp = a2 * fp + b2 * rg[i];
                fg[(long long)i * nv + l] = fp;
            }
        }
    }
    __syncthreads();
    // restriction to K_m: node-major, velocity fastest
    const int i0 = P.x0 - P.X0, nk_nodes = P.x1 - P.x0 + 1;
    for (int gg = 0; gg < G; ++gg) {
        const int ss = blockIdx.y * G + gg;
        if (ss >= A.S) break;
        double* out = A.snaps + P.snap_offset + (long long)ss * P.n_k;
        const double* fs = f + (long long)gg * nn * nv;
        for (int t = threadIdx.x; t < nk_nodes * nv; t += blockDim.x) out[t] = fs[(long long)i0 * nv + t];
        if (threadIdx.x == 0) {
            A.stats[2 * (m * A.S + ss) + 0] = it;
            A.stats[2 * (m * A.S + ss) + 1] = done ? 0 : 1;
        }
    }
}

// Mixed precision: source iteration on the density with FP64 residuals and FP32
// corrections.  With K the density of a transport sweep driven by the source
// b2 rho (zero inflow) and q the density of the sweep of the inflow alone, the
// converged density solves (I - K) rho = q.  Each outer step does one FP64
// sweep with the current rho (giving q + K rho and the residual
// res = q + K rho - rho), then solves (I - K) delta = res by FP32 source
// iteration to a relative 1e-6 and adds delta to rho in FP64.  Stops when
// |res| <= tol |q + K rho|; the final angular flux comes from one more FP64
// sweep with the converged density, as in the FP64 kernel.
__global__ void kinetic_si_mixed_kernel(KSolveArgs A) {
    extern __shared__ double ksm[];
    __shared__ double red[32];
    __shared__ float redf[32];
    __shared__ double w64[256];   // quadrature weights, loaded once (n_v <= 256)
    __shared__ float w32[256];
    const int m = blockIdx.x;
    const KPatchDev P = A.patches[m];
    const int nn = P.X1 - P.X0 + 1, nv = A.n_v, G = A.G;
    double* f = ksm;                                   // G x nn x nv (FP64 sweeps)
    float* f32 = reinterpret_cast<float*>(ksm);        // the same storage for the FP32 sweeps
    double* rho = ksm + (long long)G * nn * nv;        // G x nn
    double* res = rho + (long long)G * nn;             // G x nn
    float* del = reinterpret_cast<float*>(res + (long long)G * nn);   // G x nn
    float* res32 = del + (long long)G * nn;                           // G x nn: res rounded once per step
    const int g = threadIdx.x / nv, l = threadIdx.x % nv;
    const int s = blockIdx.y * G + g;
    const bool live = g < G && s < A.S;
    const double dx = 1.0 / A.N, ie = 1.0 / A.eps;
    double vl = 0.0, a2 = 0.0, b2 = 0.0, inflow = 0.0;
    if (live) {
        vl = A.v[l];
        const double a = fabs(vl) / dx, inv = 1.0 / (a + ie);
        a2 = a * inv;
        b2 = ie * inv;
        const int t = (vl > 0.0) ? l - nv / 2 : nv / 2 + l;
        const double2 z = gaussian_pair(A.seed, (uint32_t)(t >> 1), (uint32_t)s, (uint32_t)m, kTagKinetic);
        inflow = (t & 1) ? z.y : z.x;
    }
    const float a2f = (float)a2, b2f = (float)b2;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        w64[t] = A.w[t];
        w32[t] = (float)A.w[t];
    }
    for (int t = threadIdx.x; t < G * nn; t += blockDim.x) rho[t] = 0.0;
    __syncthreads();
    double* fg = f + (long long)(live ? g : 0) * nn * nv;
    float* fg32 = f32 + (long long)(live ? g : 0) * nn * nv;
    const double* rg = rho + (live ? g : 0) * nn;
    const float* dg = del + (live ? g : 0) * nn;
    auto sweep64 = [&]() {
        if (!live) return;
        if (vl > 0.0) {
            double fp = inflow;
            fg[l] = fp;
            for (int i = 1; i < nn; ++i) {
                fp = a2 * fp + b2 * rg[i];
                fg[(long long)i * nv + l] = fp;
            }
        } else {
            double fp = inflow;
            fg[(long long)(nn - 1) * nv + l] = fp;
            for (int i = nn - 2; i >= 0; --i) {
                fp = a2 * fp + b2 * rg[i];
                fg[(long long)i * nv + l] = fp;
            }
        }
    };
    int inner_total = 0, outer = 0;
    bool done = false;
    for (; outer < 64 && !done; ++outer) {
        sweep64();
        __syncthreads();
        // residual of the density and its size
        double rmax = 0.0, smax = 0.0;
        for (int t = threadIdx.x; t < G * nn; t += blockDim.x) {
            const int gg = t / nn, i = t - gg * nn;
            if (blockIdx.y * G + gg >= A.S) continue;
            const double* fi = f + ((long long)gg * nn + i) * nv;
            double r = 0.0;
            for (int ll = 0; ll < nv; ++ll) r += w64[ll] * fi[ll];
            r *= 0.5;
            res[t] = r - rho[t];
            rmax = fmax(rmax, fabs(r - rho[t]));
            smax = fmax(smax, fabs(r));
        }
        rmax = block_max1(rmax, red);
        smax = block_max1(smax, red);
        if (rmax <= A.tol * smax) {
            for (int t = threadIdx.x; t < G * nn; t += blockDim.x) rho[t] += res[t];
            done = true;
            __syncthreads();
            break;
        }
        // (I - K) delta = res by FP32 source iteration
        for (int t = threadIdx.x; t < G * nn; t += blockDim.x) del[t] = res32[t] = (float)res[t];
        __syncthreads();
        bool inner_done = false;
        for (int it = 0; it < A.max_iter && !inner_done; ++it) {
            if (live) {
                if (vl > 0.0) {
                    float fp = 0.f;
                    fg32[l] = fp;
                    for (int i = 1; i < nn; ++i) {
                        fp = a2f * fp + b2f * dg[i];
                        fg32[(long long)i * nv + l] = fp;
                    }
                } else {
                    float fp = 0.f;
                    fg32[(long long)(nn - 1) * nv + l] = fp;
                    for (int i = nn - 2; i >= 0; --i) {
                        fp = a2f * fp + b2f * dg[i];
                        fg32[(long long)i * nv + l] = fp;
                    }
                }
            }
            __syncthreads();
            float dmax = 0.f, vmax = 0.f;
            for (int t = threadIdx.x; t < G * nn; t += blockDim.x) {
                const int gg = t / nn, i = t - gg * nn;
                if (blockIdx.y * G + gg >= A.S) continue;
                const float* fi = f32 + ((long long)gg * nn + i) * nv;
                float r = 0.f;
                for (int ll = 0; ll < nv; ++ll) r = fmaf(w32[ll], fi[ll], r);
                r = 0.5f * r + res32[t];
                dmax = fmaxf(dmax, fabsf(r - del[t]));
                vmax = fmaxf(vmax, fabsf(r));
                del[t] = r;
            }
            dmax = block_max1(dmax, redf);
            vmax = block_max1(vmax, redf);
            inner_done = dmax <= 1e-6f * vmax;
            ++inner_total;
        }
        for (int t = threadIdx.x; t < G * nn; t += blockDim.x) rho[t] += (double)del[t];
        __syncthreads();
    }
    // the angular flux of the converged density
    sweep64();
    __syncthreads();
    const int i0 = P.x0 - P.X0, nk_nodes = P.x1 - P.x0 + 1;
    for (int gg = 0; gg < G; ++gg) {
        const int ss = blockIdx.y * G + gg;
        if (ss >= A.S) break;
        double* out = A.snaps + P.snap_offset + (long long)ss * P.n_k;
        const double* fs = f + (long long)gg * nn * nv;
        for (int t = threadIdx.x; t < nk_nodes * nv; t += blockDim.x) out[t] = fs[(long long)i0 * nv + t];
        if (threadIdx.x == 0) {
            A.stats[2 * (m * A.S + ss) + 0] = inner_total + outer;
            A.stats[2 * (m * A.S + ss) + 1] = done ? 0 : 1;
        }
    }
}

// ---- online: block-tridiagonal normal equations along the chain of patches
// rows of Q_m at the first (left) and last (right) node of K_m
__device__ __forceinline__ const double* qrow(const double* Q, const KPatchDev& P, int node, int l, int nv) {
    return Q + (long long)node * nv + l;   // column j at + j * n_k
}

// one CTA, sequential over patches: assemble H blocks and factorise
__global__ void kinetic_factor_kernel(int M, int nv, const double* v, const KPatchDev* patches, const int* k,
                                      const long long* q_off, const double* Q, const long long* l_off,
                                      const long long* c_off, double* Lf, double* Cf, double* work, int* fail) {
    // work: D (kmax x kmax) scratch
    __shared__ int s_ok;
    if (threadIdx.x == 0) { s_ok = 1; *fail = 0; }
    __syncthreads();
    for (int m = 0; m < M; ++m) {
        const int km = k[m];
        const KPatchDev P = patches[m];
        const double* Qm = Q + q_off[m];
        const int last = P.x1 - P.x0;
        double* D = Lf + l_off[m];
        // D = H_mm: right-interface rows (m < M-1), left-interface rows (m > 0), incoming rows
        for (int e = threadIdx.x; e < km * km; e += blockDim.x) {
            const int i = e % km, j = e / km;
            double a = 0.0;
            for (int l = 0; l < nv; ++l) {
                const bool right = (m < M - 1) || (v[l] < 0.0);
                const bool left = (m > 0) || (v[l] > 0.0);
                if (right) a += Qm[(long long)last * nv + l + (long long)i * P.n_k] * Qm[(long long)last * nv + l + (long long)j * P.n_k];
                if (left) a += Qm[l + (long long)i * P.n_k] * Qm[l + (long long)j * P.n_k];
            }
            D[e] = a;
        }
        __syncthreads();
        if (m > 0) {   // D -= C_{m-1} C_{m-1}^T
            const int kp = k[m - 1];
            const double* Cp = Cf + c_off[m - 1];
            for (int e = threadIdx.x; e < km * km; e += blockDim.x) {
                const int i = e % km, j = e / km;
                double a = 0.0;
                for (int q = 0; q < kp; ++q) a += Cp[i + (long long)q * km] * Cp[j + (long long)q * km];
                D[e] -= a;
            }
            __syncthreads();
        }
        // Cholesky D = L L^T in place (lower)
        for (int c = 0; c < km; ++c) {
            if (threadIdx.x == 0) {
                const double d = D[c + (long long)c * km];
                if (!(d > 0.0)) { s_ok = 0; D[c + (long long)c * km] = 1.0; }
                else D[c + (long long)c * km] = sqrt(d);
            }
            __syncthreads();
            const double piv = D[c + (long long)c * km];
            for (int i = c + 1 + threadIdx.x; i < km; i += blockDim.x) D[i + (long long)c * km] /= piv;
            __syncthreads();
            const int R = km - c - 1;
            for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
                const int i = c + 1 + e % R, j = c + 1 + e / R;
                if (i >= j) D[i + (long long)j * km] -= D[i + (long long)c * km] * D[j + (long long)c * km];
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < km * km; e += blockDim.x) {
            const int i = e % km, j = e / km;
            if (i < j) D[e] = 0.0;
        }
        __syncthreads();
        if (m + 1 < M) {
            // E = H_{m+1,m} = -Vl_{m+1}^T Vr_m ; C_m = E L_m^{-T}: row i of C solves L_m c = E_i^T
            const int kn = k[m + 1];
            const KPatchDev Pn = patches[m + 1];
            const double* Qn = Q + q_off[m + 1];
            double* Cm = Cf + c_off[m];
            for (int e = threadIdx.x; e < kn * km; e += blockDim.x) {
                const int i = e % kn, j = e / kn;
                double a = 0.0;
                for (int l = 0; l < nv; ++l)
                    a -= Qn[l + (long long)i * Pn.n_k] * Qm[(long long)last * nv + l + (long long)j * P.n_k];
                work[e] = a;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < kn; i += blockDim.x) {
                for (int j = 0; j < km; ++j) {   // forward substitution on row i
                    double a = work[i + (long long)j * kn];
                    for (int q = 0; q < j; ++q) a -= D[j + (long long)q * km] * Cm[i + (long long)q * kn];
                    Cm[i + (long long)j * kn] = a / D[j + (long long)j * km];
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && !s_ok) *fail = 1;
}

// Pieces of one data set's solve, one CTA per data set.
struct KOnArgs {
    int M, nv, N;
    const double* v;
    const KPatchDev* patches;
    const int* k;
    const int* c_off;
    const long long* q_off;
    const double* Q;
    const long long* l_off;
    const long long* cb_off;
    const double* Lf;
    const double* Cf;
};

// value of u_m at node `node`, velocity l for coefficients c_m
__device__ double kval(const KOnArgs& A, int m, int node, int l, const double* c) {
    const KPatchDev P = A.patches[m];
    const double* Qm = A.Q + A.q_off[m];
    double a = 0.0;
    for (int j = 0; j < A.k[m]; ++j) a += Qm[(long long)node * A.nv + l + (long long)j * P.n_k] * c[A.c_off[m] + j];
    return a;
}

// g = P^T r for the residual rows r (interfaces then incoming rows) -- rows evaluated
// from the residual vector stored per row.  Row layout: interface m (m < M-1): nv rows;
// then nv/2 left incoming rows (positive v, ascending), then nv/2 right incoming rows.
__device__ void kinetic_normal_rhs(const KOnArgs& A, const double* r, double* g) {
    const int nv = A.nv, M = A.M;
    for (int m = 0; m < M; ++m) {
        const KPatchDev P = A.patches[m];
        const double* Qm = A.Q + A.q_off[m];
        const int last = P.x1 - P.x0;
        for (int j = threadIdx.x; j < A.k[m]; j += blockDim.x) {
            double a = 0.0;
            for (int l = 0; l < nv; ++l) {
                if (m < M - 1) a += Qm[(long long)last * nv + l + (long long)j * P.n_k] * r[m * nv + l];
                if (m > 0) a -= Qm[l + (long long)j * P.n_k] * r[(m - 1) * nv + l];
            }
            if (m == 0)
                for (int t = 0; t < nv / 2; ++t) a += Qm[(nv / 2 + t) + (long long)j * P.n_k] * r[(M - 1) * nv + t];
            if (m == M - 1)
                for (int t = 0; t < nv / 2; ++t)
                    a += Qm[(long long)last * nv + t + (long long)j * P.n_k] * r[(M - 1) * nv + nv / 2 + t];
            g[A.c_off[m] + j] = a;
        }
    }
    __syncthreads();
}

// solve H x = g in place with the block factor
__device__ void kinetic_factor_solve(const KOnArgs& A, double* x) {
    const int M = A.M;
    for (int m = 0; m < M; ++m) {   // forward: L_m y_m = g_m - C_{m-1} y_{m-1}
        const int km = A.k[m];
        double* xm = x + A.c_off[m];
        if (m > 0) {
            const int kp = A.k[m - 1];
            const double* C = A.Cf + A.cb_off[m - 1];
            const double* xp = x + A.c_off[m - 1];
            for (int i = threadIdx.x; i < km; i += blockDim.x) {
                double a = 0.0;
                for (int q = 0; q < kp; ++q) a += C[i + (long long)q * km] * xp[q];
                xm[i] -= a;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double* L = A.Lf + A.l_off[m];
            for (int i = 0; i < km; ++i) {
                double a = xm[i];
                for (int q = 0; q < i; ++q) a -= L[i + (long long)q * km] * xm[q];
                xm[i] = a / L[i + (long long)i * km];
            }
        }
        __syncthreads();
    }
    for (int m = M - 1; m >= 0; --m) {   // backward: L_m^T x_m = y_m - C_m^T x_{m+1}
        const int km = A.k[m];
        double* xm = x + A.c_off[m];
        if (m + 1 < M) {
            const int kn = A.k[m + 1];
            const double* C = A.Cf + A.cb_off[m];
            const double* xn = x + A.c_off[m + 1];
            for (int j = threadIdx.x; j < km; j += blockDim.x) {
                double a = 0.0;
                for (int q = 0; q < kn; ++q) a += C[q + (long long)j * kn] * xn[q];
                xm[j] -= a;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double* L = A.Lf + A.l_off[m];
            for (int i = km - 1; i >= 0; --i) {
                double a = xm[i];
                for (int q = i + 1; q < km; ++q) a -= L[q + (long long)i * km] * xm[q];
                xm[i] = a / L[i + (long long)i * km];
            }
        }
        __syncthreads();
    }
}

// residual rows r = d - P c
__device__ void kinetic_residual(const KOnArgs& A, const double* c, const double* inl, const double* inr, double* r) {
    const int nv = A.nv, M = A.M;
    for (int t = threadIdx.x; t < (M - 1) * nv; t += blockDim.x) {
        const int m = t / nv, l = t - m * nv;
        const int last = A.patches[m].x1 - A.patches[m].x0;
        r[t] = -(kval(A, m, last, l, c) - kval(A, m + 1, 0, l, c));
    }
    for (int t = threadIdx.x; t < nv / 2; t += blockDim.x) {
        r[(M - 1) * nv + t] = inl[nv / 2 + t] - kval(A, 0, 0, nv / 2 + t, c);
        const int last = A.patches[M - 1].x1 - A.patches[M - 1].x0;
        r[(M - 1) * nv + nv / 2 + t] = inr[t] - kval(A, M - 1, last, t, c);
    }
    __syncthreads();
}

// c = argmin |P c - d| by the factorised normal equations and two refinement
// steps (corrected semi-normal equations); then the reconstruction.
__global__ void kinetic_online_kernel(KOnArgs A, const double* inflow, double* work, double* f_out, double* c_out,
                                      int Np) {
    const int b = blockIdx.x;
    const int nv = A.nv, M = A.M, N = A.N;
    const double* inl = inflow + (long long)b * 2 * nv;
    const double* inr = inl + nv;
    const int nrows = (M - 1) * nv + nv;
    double* c = work + (long long)b * (2 * Np + nrows);
    double* g = c + Np;
    double* r = g + Np;
    for (int j = threadIdx.x; j < Np; j += blockDim.x) c[j] = 0.0;
    __syncthreads();
    for (int pass = 0; pass < 3; ++pass) {
        kinetic_residual(A, c, inl, inr, r);
        kinetic_normal_rhs(A, r, g);
        kinetic_factor_solve(A, g);
        for (int j = threadIdx.x; j < Np; j += blockDim.x) c[j] += g[j];
        __syncthreads();
    }
    if (c_out)
        for (int j = threadIdx.x; j < Np; j += blockDim.x) c_out[(long long)b * Np + j] = c[j];
    // reconstruction: patch interiors, interface averages, incoming data at the ends
    double* fo = f_out + (long long)b * (N + 1) * nv;
    for (long long t = threadIdx.x; t < (long long)(N + 1) * nv; t += blockDim.x) {
        const int i = (int)(t / nv), l = (int)(t % nv);
        const int W = A.patches[0].x1 - A.patches[0].x0;
        int m = min(i / W, M - 1);
        double val;
        if (i == A.patches[m].x0 && m > 0) {
            val = 0.5 * (kval(A, m - 1, A.patches[m - 1].x1 - A.patches[m - 1].x0, l, c) + kval(A, m, 0, l, c));
        } else {
            val = kval(A, m, i - A.patches[m].x0, l, c);
        }
        if (i == 0 && A.v[l] > 0.0) val = inl[l];
        if (i == N && A.v[l] < 0.0) val = inr[l];
        fo[t] = val;
    }
}

// Per-sample iteration counts and flags to the caller's stats (optional; reading
// them synchronises the stream).
msp_status kinetic_stats(const KMedium& K, bool mixed, cudaStream_t s, msp_solve_stats* stats, const char* what) {
    if (!stats) return MSP_OK;
    std::vector<int> h(2 * (size_t)K.M * K.S);
    MSP_CUDA(cudaMemcpyAsync(h.data(), K.stats.p, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    msp_solve_stats r{};
    r.n_solves = (int64_t)K.M * K.S;
    for (size_t i = 0; i < h.size() / 2; ++i) {
        r.total_iters += h[2 * i];
        r.max_iters = std::max(r.max_iters, h[2 * i]);
        r.n_not_converged += h[2 * i + 1];
        r.unknown_iters += (long long)h[2 * i] * K.patches[i / K.S].nn * K.n_v;
    }
    r.max_refinements = (K.solver == MSP_KINETIC_DIRECT) ? r.max_iters : (mixed ? 0 : 1);
    *stats = r;
    if (r.n_not_converged) {
        set_error(what);
        return MSP_ERR_NOT_CONVERGED;
    }
    return MSP_OK;
}

}  // namespace
}  // namespace msp

using namespace msp;

extern "C" msp_status msp_kinetic_build(int n_cells, double eps, int n_v, int n_patches, int buffer, int samples,
                                        void* stream, msp_kmedium* out) {
    return msp_kinetic_build_hg(n_cells, eps, 0.0, n_v, n_patches, buffer, samples, stream, out);
}

extern "C" msp_status msp_kinetic_build_hg(int n_cells, double eps, double g, int n_v, int n_patches, int buffer,
                                           int samples, void* stream, msp_kmedium* out) {
    clear_error();
    MSP_CHECK_ARG(out, "msp_kinetic_build: NULL output");
    *out = nullptr;
    MSP_CHECK_ARG(n_cells >= 2 && n_patches >= 1 && n_cells % n_patches == 0,
                  "msp_kinetic_build: n_cells must be a positive multiple of n_patches");
    MSP_CHECK_ARG(n_v >= 2 && n_v % 2 == 0 && n_v <= 256, "msp_kinetic_build: n_v must be even, 2..256");
    MSP_CHECK_ARG(eps > 0 && buffer >= 0 && samples >= 1, "msp_kinetic_build: eps > 0, buffer >= 0, samples >= 1");
    MSP_CHECK_ARG(g > -1.0 && g < 1.0, "msp_kinetic_build: the anisotropy g must lie in (-1, 1)");
    MSP_CHECK_ARG(g == 0.0 || n_v <= 128, "msp_kinetic_build: anisotropic scattering takes at most 128 velocities");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_error("msp_kinetic_build: no usable CUDA device");
        return MSP_ERR_CUDA;
    }
    auto* h = new msp_kmedium_s();
    KMedium& K = h->K;
    K.N = n_cells; K.eps = eps; K.g = g; K.n_v = n_v; K.M = n_patches; K.buffer = buffer; K.S = samples;
    K.solver = (g == 0.0) ? MSP_KINETIC_SOURCE_ITERATION : MSP_KINETIC_DIRECT;
    gauss_legendre(n_v, K.v, K.w);
    // Eq. HG in quadrature form: k(v, v') = (1/2)(1 - g^2) / (1 + g^2 + 2 g v v'), gain
    // weights w_l' k(v_l, v_l'), loss rates sigma_l = sum_l' w_l' k(v_l', v_l)
    K.Kw.assign((size_t)n_v * n_v, 0.0);
    K.sigma.assign(n_v, 0.0);
    for (int l = 0; l < n_v; ++l)
        for (int q = 0; q < n_v; ++q) {
            const double k = 0.5 * (1.0 - g * g) / (1.0 + g * g + 2.0 * g * K.v[l] * K.v[q]);
            K.Kw[(size_t)l * n_v + q] = K.w[q] * k;
            K.sigma[q] += K.w[l] * k;
        }
    const int W = n_cells / n_patches;
    long long off = 0;
    for (int m = 0; m < n_patches; ++m) {
        KPatchDev P{};
        P.x0 = m * W; P.x1 = (m + 1) * W;
        P.X0 = std::max(0, P.x0 - buffer); P.X1 = std::min(n_cells, P.x1 + buffer);
        P.nn = P.X1 - P.X0 + 1;
        P.n_k = (W + 1) * n_v;
        P.snap_offset = off;
        off += (long long)P.n_k * samples;
        K.patches.push_back(P);
    }
    K.snap_elems = off;
    cudaStream_t s = (cudaStream_t)stream;
    msp_status st;
    if ((st = upload(K.d_v, K.v, s)) || (st = upload(K.d_w, K.w, s)) || (st = upload(K.d_patches, K.patches, s)) ||
        (st = upload(K.d_Kw, K.Kw, s)) || (st = upload(K.d_sigma, K.sigma, s)) ||
        (st = K.snaps.alloc((size_t)off, s)) || (st = K.stats.alloc((size_t)2 * n_patches * samples, s))) {
        delete h;
        return st;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        delete h;
        set_error("msp_kinetic_build: stream synchronisation failed");
        return MSP_ERR_CUDA;
    }
    *out = h;
    return MSP_OK;
}

extern "C" void msp_kinetic_destroy(msp_kmedium k) { delete k; }

extern "C" msp_status msp_kinetic_velocities(msp_kmedium k, double* v_host, double* w_host) {
    clear_error();
    MSP_CHECK_ARG(k, "msp_kinetic_velocities: NULL medium");
    for (int l = 0; l < k->K.n_v; ++l) {
        if (v_host) v_host[l] = k->K.v[l];
        if (w_host) w_host[l] = k->K.w[l];
    }
    return MSP_OK;
}

extern "C" msp_status msp_kinetic_set_solver(msp_kmedium k, int solver) {
    clear_error();
    MSP_CHECK_ARG(k, "msp_kinetic_set_solver: NULL medium");
    MSP_CHECK_ARG(solver == MSP_KINETIC_SOURCE_ITERATION || solver == MSP_KINETIC_DIRECT,
                  "msp_kinetic_set_solver: unknown solver");
    MSP_CHECK_ARG(solver == MSP_KINETIC_DIRECT || k->K.g == 0.0,
                  "msp_kinetic_set_solver: source iteration takes isotropic scattering (g = 0) only");
    MSP_CHECK_ARG(solver == MSP_KINETIC_SOURCE_ITERATION || k->K.n_v <= 128,
                  "msp_kinetic_set_solver: the direct solver takes at most 128 velocities");
    k->K.solver = solver;
    return MSP_OK;
}

extern "C" msp_status msp_kinetic_sample(msp_kmedium k, uint64_t seed, int precision, double tol, int max_iter,
                                         void* stream, msp_solve_stats* stats) {
    clear_error();
    MSP_CHECK_ARG(k, "msp_kinetic_sample: NULL medium");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_kinetic_sample: unknown precision");
    const bool mixed = precision == MSP_MIXED;
    MSP_CHECK_ARG(!mixed || k->K.n_v <= 256, "msp_kinetic_sample: the mixed path takes at most 256 velocities");
    MSP_CHECK_ARG(tol > 0 && tol < 1 && max_iter >= 1, "msp_kinetic_sample: tol in (0,1), max_iter >= 1");
    KMedium& K = k->K;
    cudaStream_t s = (cudaStream_t)stream;
    if (K.solver == MSP_KINETIC_DIRECT) {
        MSP_TRY(kinetic_direct_sample(K, seed, mixed, tol, max_iter, s));
        K.sampled = true;
        return kinetic_stats(K, mixed, s, stats, "msp_kinetic_sample: direct solve stopped at its pass limit for some samples");
    }
    int max_nn = 0;
    for (auto& P : K.patches) max_nn = std::max(max_nn, P.nn);
    const size_t per = sizeof(double) * ((size_t)max_nn * K.n_v + max_nn) +
                       (mixed ? (sizeof(double) + 2 * sizeof(float)) * (size_t)max_nn : 0);
    int G = (int)std::min<size_t>(std::max(1, 256 / K.n_v), (200 * 1024) / per);
    if (G < 1) {
        set_error("msp_kinetic_sample: buffered patch too long for on-chip sweeps");
        return MSP_ERR_INVALID_ARG;
    }
    G = std::min(G, K.S);
    KSolveArgs A{};
    A.N = K.N; A.n_v = K.n_v; A.S = K.S; A.G = G; A.eps = K.eps; A.tol = tol; A.max_iter = max_iter; A.seed = seed;
    A.v = K.d_v.p; A.w = K.d_w.p; A.patches = K.d_patches.p; A.snaps = K.snaps.p; A.stats = K.stats.p;
    const size_t smem = per * G;
    dim3 grid(K.M, (K.S + G - 1) / G);
    if (mixed) {
        MSP_CUDA(cudaFuncSetAttribute(kinetic_si_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kinetic_si_mixed_kernel<<<grid, G * K.n_v, smem, s>>>(A);
    } else {
        MSP_CUDA(cudaFuncSetAttribute(kinetic_si_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kinetic_si_kernel<<<grid, G * K.n_v, smem, s>>>(A);
    }
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    K.sampled = true;
    return kinetic_stats(K, mixed, s, stats, "msp_kinetic_sample: source iteration stopped at max_iter for some samples");
}

extern "C" msp_status msp_kinetic_get_snapshots(msp_kmedium k, int patch, double* dst, void* stream) {
    clear_error();
    MSP_CHECK_ARG(k && dst, "msp_kinetic_get_snapshots: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < k->K.M, "msp_kinetic_get_snapshots: patch out of range");
    if (!k->K.sampled) { set_error("msp_kinetic_get_snapshots: call msp_kinetic_sample first"); return MSP_ERR_STATE; }
    const KPatchDev& P = k->K.patches[patch];
    MSP_CUDA(cudaMemcpyAsync(dst, k->K.snaps.p + P.snap_offset, sizeof(double) * (size_t)P.n_k * k->K.S,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MSP_OK;
}

extern "C" msp_status msp_kinetic_extract(msp_kmedium km, double tau, void* stream, msp_kbasis* out) {
    clear_error();
    MSP_CHECK_ARG(km && out, "msp_kinetic_extract: NULL argument");
    MSP_CHECK_ARG(tau >= 0 && tau < 1, "msp_kinetic_extract: tau must lie in [0, 1)");
    *out = nullptr;
    KMedium& K = km->K;
    if (!K.sampled) { set_error("msp_kinetic_extract: call msp_kinetic_sample first"); return MSP_ERR_STATE; }
    cudaStream_t s = (cudaStream_t)stream;
    auto* h = new msp_kbasis_s();
    KBasis& B = h->B;
    B.N = K.N; B.n_v = K.n_v; B.M = K.M; B.v = K.v; B.patches = K.patches;
    std::vector<long long> soff(K.M);
    std::vector<int> rows(K.M), cols(K.M);
    for (int m = 0; m < K.M; ++m) {
        soff[m] = K.patches[m].snap_offset;
        rows[m] = K.patches[m].n_k;
        cols[m] = K.S;
    }
    msp_status st = svd_bases(K.snaps.p, K.snap_elems, soff, rows, cols, tau, s, B.Q, B.k, B.sigma, B.sigma_off, B.q_off,
                              B.max_sweeps, B.max_tries);
    if (st != MSP_OK) { delete h; return st; }
    B.c_off.assign(K.M + 1, 0);
    for (int m = 0; m < K.M; ++m) B.c_off[m + 1] = B.c_off[m] + B.k[m];
    B.Np = B.c_off[K.M];
    B.l_off.assign(K.M, 0);
    B.c_blk_off.assign(std::max(K.M - 1, 1), 0);
    long long lo = 0, co = 0;
    int kmax = 1;
    for (int m = 0; m < K.M; ++m) {
        B.l_off[m] = lo;
        lo += (long long)B.k[m] * B.k[m];
        kmax = std::max(kmax, B.k[m]);
        if (m + 1 < K.M) {
            B.c_blk_off[m] = co;
            co += (long long)B.k[m + 1] * B.k[m];
        }
    }
    DevBuf<double> work;
    DevBuf<int> fail;
    if ((st = upload(B.d_patches, B.patches, s)) || (st = upload(B.d_k, B.k, s)) || (st = upload(B.d_c_off, B.c_off, s)) ||
        (st = upload(B.d_q_off, B.q_off, s)) || (st = upload(B.d_v, B.v, s)) || (st = upload(B.d_l_off, B.l_off, s)) ||
        (st = upload(B.d_c_blk_off, B.c_blk_off, s)) || (st = B.Lf.alloc(std::max<long long>(lo, 1), s)) ||
        (st = B.Cf.alloc(std::max<long long>(co, 1), s)) || (st = work.alloc((size_t)kmax * kmax, s)) ||
        (st = fail.alloc(1, s))) {
        delete h;
        return st;
    }
    kinetic_factor_kernel<<<1, 256, 0, s>>>(K.M, K.n_v, B.d_v.p, B.d_patches.p, B.d_k.p, B.d_q_off.p, B.Q.p, B.d_l_off.p,
                                            B.d_c_blk_off.p, B.Lf.p, B.Cf.p, work.p, fail.p);
    count_launches(1);
    int hf = 0;
    if (cudaMemcpyAsync(&hf, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        delete h;
        set_error("msp_kinetic_extract: CUDA failure in the online factorisation");
        return MSP_ERR_CUDA;
    }
    if (hf) {
        delete h;
        set_error("msp_kinetic_extract: normal equations not positive definite");
        return MSP_ERR_BREAKDOWN;
    }
    *out = h;
    return MSP_OK;
}

extern "C" void msp_kinetic_basis_destroy(msp_kbasis b) { delete b; }

extern "C" msp_status msp_kinetic_basis_info(msp_kbasis b, int patch, int* k, double* sigma_host) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_kinetic_basis_info: NULL basis");
    MSP_CHECK_ARG(patch >= 0 && patch < b->B.M, "msp_kinetic_basis_info: patch out of range");
    if (k) *k = b->B.k[patch];
    if (sigma_host) {
        const long long o = b->B.sigma_off[patch];
        const long long e = (patch + 1 < b->B.M) ? b->B.sigma_off[patch + 1] : (long long)b->B.sigma.size();
        for (long long i = o; i < e; ++i) sigma_host[i - o] = b->B.sigma[i];
    }
    return MSP_OK;
}

extern "C" msp_status msp_kinetic_online_solve(msp_kbasis b, const double* inflow_dev, int batch, double* f_dev,
                                               double* c_dev, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && inflow_dev && f_dev, "msp_kinetic_online_solve: NULL argument");
    MSP_CHECK_ARG(batch >= 0, "msp_kinetic_online_solve: negative batch");
    if (batch == 0) return MSP_OK;
    KBasis& B = b->B;
    cudaStream_t s = (cudaStream_t)stream;
    const int nrows = B.M * B.n_v;
    DevBuf<double> work;
    MSP_TRY(work.alloc((size_t)batch * (2 * std::max(B.Np, 1) + nrows), s));
    KOnArgs A{};
    A.M = B.M; A.nv = B.n_v; A.N = B.N; A.v = B.d_v.p; A.patches = B.d_patches.p; A.k = B.d_k.p; A.c_off = B.d_c_off.p;
    A.q_off = B.d_q_off.p; A.Q = B.Q.p; A.l_off = B.d_l_off.p; A.cb_off = B.d_c_blk_off.p; A.Lf = B.Lf.p; A.Cf = B.Cf.p;
    kinetic_online_kernel<<<batch, 256, 0, s>>>(A, inflow_dev, work.p, f_dev, c_dev, B.Np);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    MSP_CUDA(cudaStreamSynchronize(s));   // the work buffer is released on return
    return MSP_OK;
}
