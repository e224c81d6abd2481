// Online stage by overlapping Schwarz on the reduced bases.
//
// The paper leaves the online step to a standard domain-decomposition step
// (Sec. 3, before Algorithm alg:summary); besides the least-squares glue of Eq.
// elliptic_cond_reduced, the buffered patches K~_m give the classical overlapping
// choice, restricted additive Schwarz (Cai and Sarkis, 1999): solve the local
// problem on every K~_m with the current field's values on its ring, keep the
// solution on K_m, average shared nodes with chi_m = 1/#patches.  On the reduced
// bases the local solve is projected onto span Q_m, so one step is
//     c_m <- B_m g_m(c),   B_m = Q_m^T G~_m   (k_m x n_ring, G~_m from DetLocalSolu),
// g_m(c)[r] = sum over the patches n holding ring node r of chi_n (Q_n c_n)(r), or
// phi(r) on the domain boundary.  The fixed point solves (I - T) c = F phi.
//
// Set-up (msp_ras_setup): B_m by one batched FP64 product per patch (tensor cores
// or CUDA cores, as the extraction's products), the rows chi_n Q_n[loc, :] of every
// ring entry gathered contiguously, and the two-level coarse space of Nicolaides
// (1987): one vector per patch, z_m = Q_m^T 1 / |Q_m^T 1| (the constant function
// projected on the basis), coarse matrix E = Z^T (I - T) Z (M x M, assembled from
// the ring tables) inverted by Gauss-Jordan elimination with partial pivoting.
//
// Solve (msp_online_solve_ras): restarted GMRES (restart kRasRestart) on
// (I - T) c = F phi, right-preconditioned by the deflation form A-DEF2 of Tang,
// Nabben, Vuik and Erlangga (2009), M^{-1} = I + Z E^{-1} Z^T T (one-level: M = I);
// classical Gram-Schmidt applied twice; stopped per data set when the GMRES
// residual estimate |F phi - (I - T) c| <= tol |F phi|, the true residual being
// recomputed at every restart.  Vectors are [coefficient][B]; every reduction runs
// in a fixed order that does not depend on the batch, so a data set gets the same
// bits alone or in any batch.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace msp {

namespace {

constexpr int kRasMaxBatch = 16;     // data sets per pass (registers of the dot kernel)
constexpr int kRasRestart = 30;      // GMRES restart length
constexpr int kRasChunk = 2048;      // coefficients per partial sum (fixed: batch independent)
constexpr int kRasThreads = 256;

struct RasArgs {
    int M, B;
    const int* k;
    const int* c_off;
    const long long* b_off;     // B_m blocks: k_m x n_ring_m, column-major (ld k_m)
    const double* Bm;
    const int* ring_base;       // [M + 1] first global ring index of each patch
    const int* bnd;             // per global ring node: domain ring position or -1
    const int* ent_ptr;         // per global ring node: first entry ([n_ring_tot + 1])
    const int* ent_patch;       // per entry: the owner patch n
    const long long* ent_row;   // per entry: offset of chi_n Q_n[loc, :] in rows
    const double* rows;
};

// ---------------------------------------------------------------- set-up kernels

// rows[ent_row[e] + j] = chi_e Q_n[loc_e, j], one warp per entry
__global__ void ras_rows_kernel(const double* Q, const long long* q_off, const PatchDev* patches, const int* k,
                                int n_ent, const int* ent_patch, const int* ent_loc, const double* ent_chi,
                                const long long* ent_row, double* rows) {
    const int lane = threadIdx.x & 31;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n_ent; e += (gridDim.x * blockDim.x) >> 5) {
        const int n = ent_patch[e], kn = k[n], nk = patches[n].n_k;
        const double* q = Q + q_off[n] + ent_loc[e];
        double* out = rows + ent_row[e];
        const double chi = ent_chi[e];
        for (int j = lane; j < kn; j += 32) out[j] = chi * q[(long long)j * nk];
    }
}

// z_m = Q_m^T 1 / |Q_m^T 1| (e_0 if the constant is orthogonal to the basis); one
// CTA per patch, one warp per column
__global__ void ras_z_kernel(const double* Q, const long long* q_off, const PatchDev* patches, const int* k,
                             const int* c_off, double* z) {
    __shared__ double red[64];
    const int m = blockIdx.x, km = k[m], nk = patches[m].n_k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* zm = z + c_off[m];
    for (int j = warp; j < km; j += nw) {
        const double* q = Q + q_off[m] + (long long)j * nk;
        double a = 0.0;
        for (int i = lane; i < nk; i += 32) a += q[i];
        a = warp_sum(a);
        if (lane == 0) zm[j] = a;
    }
    __syncthreads();
    double v[1] = {0.0};
    for (int j = threadIdx.x; j < km; j += blockDim.x) v[0] += zm[j] * zm[j];
    block_sum<double, 1>(v, red);
    const double nrm = sqrt(v[0]);
    __syncthreads();
    for (int j = threadIdx.x; j < km; j += blockDim.x) zm[j] = nrm > 0.0 ? zm[j] / nrm : (j == 0 ? 1.0 : 0.0);
}

// aug = [I | I] (M x 2M, row-major)
__global__ void ras_aug_init_kernel(double* aug, int M) {
    const long long n = (long long)M * 2 * M;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / (2 * M)), j = (int)(t % (2 * M));
        aug[t] = (j == i || j == i + M) ? 1.0 : 0.0;
    }
}

// Row m of E = I - Z^T T Z, into the left half of aug: beta = B_m^T z_m, then for
// every interior ring entry e (owner n) the term beta_r (rows_e . z_n), summed per
// neighbour patch in entry order by one thread per neighbour.  Dynamic shared
// memory: n_ring_m + entries_m doubles.
__global__ void ras_coarse_kernel(RasArgs A, const double* z, const int* nb_ptr, const int* nb_patch,
                                  const int* ent_nb, double* aug) {
    extern __shared__ double sh[];
    const int m = blockIdx.x, km = A.k[m], M = A.M;
    const int g0 = A.ring_base[m], g1 = A.ring_base[m + 1], nr = g1 - g0;
    const int e0 = A.ent_ptr[g0], e1 = A.ent_ptr[g1];
    double* beta = sh;
    double* ce = sh + nr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* Bm = A.Bm + A.b_off[m];
    const double* zm = z + A.c_off[m];
    for (int r = warp; r < nr; r += nw) {
        double a = 0.0;
        for (int i = lane; i < km; i += 32) a += zm[i] * Bm[i + (long long)r * km];
        a = warp_sum(a);
        if (lane == 0) beta[r] = a;
    }
    __syncthreads();
    for (int g = g0 + warp; g < g1; g += nw) {
        for (int e = A.ent_ptr[g]; e < A.ent_ptr[g + 1]; ++e) {
            const int n = A.ent_patch[e], kn = A.k[n];
            const double* row = A.rows + A.ent_row[e];
            const double* zn = z + A.c_off[n];
            double a = 0.0;
            for (int j = lane; j < kn; j += 32) a += row[j] * zn[j];
            a = warp_sum(a);
            if (lane == 0) ce[e - e0] = beta[g - g0] * a;
        }
    }
    __syncthreads();
    for (int sl = nb_ptr[m] + threadIdx.x; sl < nb_ptr[m + 1]; sl += blockDim.x) {
        double a = 0.0;
        for (int e = e0; e < e1; ++e)
            if (ent_nb[e] == sl) a += ce[e - e0];
        aug[(long long)m * 2 * M + nb_patch[sl]] -= a;
    }
}

// Gauss-Jordan step k, part 1 (one CTA): partial pivoting (largest |aug[i][k]|,
// i >= k, lowest index on ties), row swap, scaling of row k, and the column of
// multipliers for part 2 (col[k] = 0).  A zero or non-finite pivot sets *fail.
__global__ void __launch_bounds__(1024) ras_gj_pivot_kernel(double* aug, int M, int k, double* col, int* fail) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int s_p;
    __shared__ double s_inv;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long ld = 2LL * M;
    double bv = -1.0;
    int bi = M;
    for (int i = k + tid; i < M; i += blockDim.x) {
        const double v = fabs(aug[(long long)i * ld + k]);
        if (v > bv) { bv = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = bv; si[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        bv = lane < nw ? sv[lane] : -1.0;
        bi = lane < nw ? si[lane] : M;
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) s_p = bi < M ? bi : k;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
        for (long long j = tid; j < ld; j += blockDim.x) {
            const double a = aug[(long long)k * ld + j];
            aug[(long long)k * ld + j] = aug[(long long)p * ld + j];
            aug[(long long)p * ld + j] = a;
        }
    __syncthreads();
    if (tid == 0) {
        const double piv = aug[(long long)k * ld + k];
        if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
            *fail = 1;
            s_inv = 0.0;
        } else {
            s_inv = 1.0 / piv;
        }
    }
    __syncthreads();
    const double inv = s_inv;
    for (long long j = tid; j < ld; j += blockDim.x) aug[(long long)k * ld + j] *= inv;
    for (int i = tid; i < M; i += blockDim.x) col[i] = (i == k) ? 0.0 : aug[(long long)i * ld + k];
}

// Gauss-Jordan step k, part 2: aug[i][j] -= col[i] aug[k][j] for i != k, j > k
__global__ void ras_gj_elim_kernel(double* aug, int M, int k, const double* col) {
    const long long ld = 2LL * M, w = ld - k - 1;
    const long long n = (long long)M * w;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / w);
        if (i == k) continue;
        const long long j = k + 1 + t % w;
        aug[(long long)i * ld + j] -= col[i] * aug[(long long)k * ld + j];
    }
}

// ---------------------------------------------------------------- the Schwarz step

// The Schwarz step in two kernels.  mode 0: out_m = (T x)_m (ring values of the
// reconstruction of x; domain-boundary ring nodes give 0), or a_m - (T x)_m when a
// is given.  mode 1: out_m = B_m g with g = phi on the domain-boundary ring nodes and
// 0 elsewhere (the right-hand side F phi).  Both kernels stream their operands (the
// ring rows, B_m) once per call and are bound by the latency of those loads, so
// each keeps eight loads per thread in flight; every sum runs in an order fixed by
// the patch alone.
//
// Ring values gv[gr][b] of every ring node of every patch: a group of 8 lanes per
// ring node, eight loads of each operand in flight per lane (one batch covers 64
// coefficients; 8 lanes measured faster than 16), the lanes' partial sums combined
// by shuffles inside the group.
__global__ void __launch_bounds__(kRasThreads) ras_ring_kernel(RasArgs A, int n_ring_tot, const double* x,
                                                             const double* phi, int n4, double* gv, int mode) {
    const int B = A.B, sub = threadIdx.x & 7;
    const unsigned gmask = 0xFFu << ((threadIdx.x & 31) & ~7);
    for (long long gr = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 3; gr < n_ring_tot;
         gr += ((long long)gridDim.x * blockDim.x) >> 3) {
        const int bp = A.bnd[gr];
        if (mode == 1) {
            for (int b = sub; b < B; b += 8) gv[gr * B + b] = bp >= 0 ? phi[(long long)b * n4 + bp] : 0.0;
            continue;
        }
        const int e0 = A.ent_ptr[gr], e1 = bp < 0 ? A.ent_ptr[gr + 1] : e0;
        for (int b = 0; b < B; ++b) {
            double v = 0.0;
            for (int e = e0; e < e1; ++e) {
                const int n = A.ent_patch[e], kn = A.k[n];
                const double* row = A.rows + A.ent_row[e];
                const double* xn = x + (long long)A.c_off[n] * B + b;
                double t = 0.0;
                for (int j0 = sub; j0 < kn; j0 += 64) {
                    double rv[8], xv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = j0 + 8 * u;
                        rv[u] = j < kn ? row[j] : 0.0;
                        xv[u] = j < kn ? xn[(long long)j * B] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) t += rv[u] * xv[u];
                }
                t += __shfl_xor_sync(gmask, t, 1);
                t += __shfl_xor_sync(gmask, t, 2);
                t += __shfl_xor_sync(gmask, t, 4);
                v += t;
            }
            if (sub == 0) gv[gr * B + b] = v;
        }
    }
}

// out_m = B_m g_m (or a_m - B_m g_m), one CTA per patch: g_m staged in shared
// memory, then for each data set the ring nodes split into nsl contiguous slices
// (nsl fixed by k_m), thread (i, slice) sums its slice with sixteen loads in flight,
// the slices added in order.  Dynamic shared memory: n_ring_max x B + max(256,
// k_max) doubles.
__global__ void __launch_bounds__(kRasThreads) ras_bm_kernel(RasArgs A, const double* gv, const double* a,
                                                           double* out) {
    extern __shared__ double g[];
    const int m = blockIdx.x, km = A.k[m], B = A.B;
    const int g0 = A.ring_base[m], nr = A.ring_base[m + 1] - g0;
    for (int t = threadIdx.x; t < nr * B; t += blockDim.x) g[t] = gv[(long long)g0 * B + t];
    __syncthreads();
    const double* Bm = A.Bm + A.b_off[m];
    const long long base = (long long)A.c_off[m] * B;
    double* part = g + nr * B;
    const int nsl = km > 0 ? max(1, min(8, (int)blockDim.x / km)) : 1;
    const int per = (nr + nsl - 1) / nsl;
    for (int b = 0; b < B; ++b) {
        for (int w = threadIdx.x; w < km * nsl; w += blockDim.x) {
            const int i = w % km, sl = w / km;
            const int r0 = sl * per, r1 = min(nr, r0 + per);
            const double* bi = Bm + i;
            const double* gb = g + b;
            double sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = 0.0;
            int r = r0;
            // all sixteen loads of a step are issued before the first product uses one
            for (; r + 16 <= r1; r += 16) {
                double bv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) bv[u] = bi[(long long)(r + u) * km];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    sv[u] += bv[u] * gb[(r + u) * B];
                    sv[u] += bv[u + 8] * gb[(r + 8 + u) * B];
                }
            }
            for (; r < r1; ++r) sv[0] += bi[(long long)r * km] * gb[r * B];
            part[w] = ((sv[0] + sv[1]) + (sv[2] + sv[3])) + ((sv[4] + sv[5]) + (sv[6] + sv[7]));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < km; i += blockDim.x) {
            double t = 0.0;
            for (int sl = 0; sl < nsl; ++sl) t += part[sl * km + i];
            const long long o = base + (long long)i * B + b;
            out[o] = a ? a[o] - t : t;
        }
        __syncthreads();
    }
}

// p[m][b] = z_m . y_m[:, b]; one warp per patch
__global__ void ras_zt_kernel(RasArgs A, const double* z, const double* y, double* p) {
    const int lane = threadIdx.x & 31, B = A.B;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < A.M; m += (gridDim.x * blockDim.x) >> 5) {
        const int km = A.k[m], c0 = A.c_off[m];
        for (int b = 0; b < B; ++b) {
            double s = 0.0;
            for (int i = lane; i < km; i += 32) s += z[c0 + i] * y[(long long)(c0 + i) * B + b];
            s = warp_sum(s);
            if (lane == 0) p[(long long)m * B + b] = s;
        }
    }
}

// q[m][b] = sum_n E^{-1}[m][n] p[n][b]; E^{-1} is the right half of aug (ld 2M);
// one warp per row
__global__ void ras_einv_kernel(RasArgs A, const double* aug, const double* p, double* q) {
    const int lane = threadIdx.x & 31, B = A.B, M = A.M;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += (gridDim.x * blockDim.x) >> 5) {
        const double* row = aug + (long long)m * 2 * M + M;
        for (int b = 0; b < B; ++b) {
            double s = 0.0;
            for (int n = lane; n < M; n += 32) s += row[n] * p[(long long)n * B + b];
            s = warp_sum(s);
            if (lane == 0) q[(long long)m * B + b] = s;
        }
    }
}

// out[t] = base[t] + v[t] + z[i] q[patch(i)][b]  (t = i B + b; base may be null,
// q null for the one-level form)
__global__ void ras_prolong_kernel(int Np, int B, const int* coef_patch, const double* z, const double* q,
                                   const double* v, const double* base, double* out) {
    const long long n = (long long)Np * B;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / B), b = (int)(t % B);
        double s = v[t];
        if (q) s += z[i] * q[(long long)coef_patch[i] * B + b];
        out[t] = base ? base[t] + s : s;
    }
}

// r = f - x + t  (the residual f - (I - T) x with t = T x)
__global__ void ras_residual_kernel(long long n, const double* f, const double* x, const double* t, double* r) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = f[i] - x[i] + t[i];
}

// ---------------------------------------------------------------- GMRES

// Partial dot products of vectors V_i (i < nvec, each Np x B, consecutive) with w,
// one CTA per (chunk of kRasChunk coefficients, i): part[(i n_chunks + chunk) B + b].
// Every thread sums a fixed set of elements; the block sum runs in warp order.  NB
// is the batch rounded up to a power of two: each data set's sums are the same
// whatever NB is, so results do not depend on the batch.
template <int NB>
__global__ void __launch_bounds__(kRasThreads) ras_dots_kernel(const double* V, const double* w, int Np, int B,
                                                             int n_chunks, double* part) {
    __shared__ double buf[NB * 32];
    const int chunk = blockIdx.x, i = blockIdx.y;
    const double* vi = V + (long long)i * Np * B;
    double acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0;
    const int c0 = chunk * kRasChunk, c1 = min(Np, c0 + kRasChunk);
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const long long t = (long long)c * B;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < B) acc[b] += vi[t + b] * w[t + b];
    }
    block_sum<double, NB>(acc, buf);
#pragma unroll
    for (int b = 0; b < NB; ++b)   // static indices keep acc in registers
        if (b < B && threadIdx.x == b) part[((long long)i * n_chunks + chunk) * B + b] = acc[b];
}

// Sum of the partials in chunk order, one warp per (i, b).  mode 0: htmp[i][b] =
// sum and hcol[i][b] += sum (a Gram-Schmidt pass); mode 1: hcol[0][b] = sqrt(sum)
// (a norm); mode 2: st[8 b + slot] = sqrt(sum).
__global__ void ras_finalize_kernel(const double* part, int nvec, int n_chunks, int B, double* htmp, double* hcol,
                                    double* st, int mode, int slot) {
    const int lane = threadIdx.x & 31;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nvec * B; w += (gridDim.x * blockDim.x) >> 5) {
        const int i = w / B, b = w % B;
        double s = 0.0;
        for (int c = lane; c < n_chunks; c += 32) s += part[((long long)i * n_chunks + c) * B + b];
        s = warp_sum(s);
        if (lane == 0) {
            if (mode == 0) {
                htmp[(long long)i * B + b] = s;
                hcol[(long long)i * B + b] += s;
            } else if (mode == 1) {
                hcol[b] = sqrt(s);
            } else {
                st[8 * b + slot] = sqrt(s);
            }
        }
    }
}

// w[t][b] -= sum_{i < nvec} V_i[t][b] h[i][b]
__global__ void ras_orth_kernel(const double* V, int nvec, int Np, int B, const double* h, double* w) {
    const long long n = (long long)Np * B;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        double s = w[t];
        for (int i = 0; i < nvec; ++i) s -= V[(long long)i * n + t] * h[(long long)i * B + b];
        w[t] = s;
    }
}

// v[t][b] = w[t][b] / h[b hs] (0 where h is 0: the Krylov space is exhausted)
__global__ void ras_scale_kernel(long long n, int B, const double* w, const double* h, int hs, double* v) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double d = h[(t % B) * hs];
        v[t] = d > 0.0 ? w[t] / d : 0.0;
    }
}

// Per data set status st[8 b + .]: 0 |F phi|, 1 residual estimate, 2 length of
// the current cycle, 3 iterations so far, 4 converged, 5 non-finite, 6 stopped in
// this cycle, 7 beta of the cycle.  Start of a cycle (one thread per data set):
// g = beta e_1, stop at once if converged, out of iterations or non-finite.
__global__ void ras_cycle_start_kernel(double* st, double* g, int B, double tol, int max_iter) {
    const int b = threadIdx.x;
    if (b >= B) return;
    double* s = st + 8 * b;
    const double beta = s[7];
    for (int i = 0; i <= kRasRestart; ++i) g[(long long)i * B + b] = 0.0;
    g[b] = beta;
    s[1] = beta;
    s[2] = 0.0;
    s[6] = 0.0;
    if (s[4] != 0.0 || s[5] != 0.0) {
        s[6] = 1.0;
        return;
    }
    if (!isfinite(beta)) {
        s[5] = 1.0;
        s[6] = 1.0;
    } else if (beta <= tol * s[0]) {
        s[4] = 1.0;
        s[6] = 1.0;
    } else if (s[3] >= max_iter) {
        s[6] = 1.0;
    }
}

// Givens rotations of column j of the Hessenberg matrix (hh: column j at
// hh[(j (R + 1) + i) B + b]) for every data set still running in this cycle
__global__ void ras_givens_kernel(double* hh, double* cs, double* sn, double* g, double* st, int j, int B, double tol,
                                  int max_iter) {
    const int b = threadIdx.x;
    if (b >= B) return;
    double* s = st + 8 * b;
    if (s[6] != 0.0) return;
    double* h = hh + (long long)j * (kRasRestart + 1) * B;
    for (int i = 0; i < j; ++i) {
        const double c = cs[(long long)i * B + b], sv = sn[(long long)i * B + b];
        const double h0 = h[(long long)i * B + b], h1 = h[(long long)(i + 1) * B + b];
        h[(long long)i * B + b] = c * h0 + sv * h1;
        h[(long long)(i + 1) * B + b] = -sv * h0 + c * h1;
    }
    const double a = h[(long long)j * B + b], bb = h[(long long)(j + 1) * B + b];
    const double r = hypot(a, bb);
    const double c = r > 0.0 ? a / r : 1.0, sv = r > 0.0 ? bb / r : 0.0;
    cs[(long long)j * B + b] = c;
    sn[(long long)j * B + b] = sv;
    h[(long long)j * B + b] = r;
    h[(long long)(j + 1) * B + b] = 0.0;
    const double gj = g[(long long)j * B + b];
    g[(long long)j * B + b] = c * gj;
    g[(long long)(j + 1) * B + b] = -sv * gj;
    const double res = fabs(sv * gj);
    s[1] = res;
    s[2] = j + 1;
    if (!isfinite(res) || !isfinite(r)) {
        s[5] = 1.0;
        s[6] = 1.0;
    } else if (res <= tol * s[0] || j + 1 == kRasRestart || s[3] + j + 1 >= max_iter || r == 0.0) {
        s[6] = 1.0;
    }
}

// End of a cycle: y = H^{-1} g over the cycle's length (0 for data sets that did
// not iterate), iterations counted
__global__ void ras_backsolve_kernel(const double* hh, const double* g, double* st, double* y, int B) {
    const int b = threadIdx.x;
    if (b >= B) return;
    double* s = st + 8 * b;
    const int len = (s[4] != 0.0 || s[5] != 0.0) ? 0 : (int)s[2];
    for (int i = kRasRestart - 1; i >= len; --i) y[(long long)i * B + b] = 0.0;
    for (int i = len - 1; i >= 0; --i) {
        double a = g[(long long)i * B + b];
        for (int l = i + 1; l < len; ++l) a -= hh[((long long)l * (kRasRestart + 1) + i) * B + b] * y[(long long)l * B + b];
        const double d = hh[((long long)i * (kRasRestart + 1) + i) * B + b];
        y[(long long)i * B + b] = d != 0.0 ? a / d : 0.0;
    }
    s[3] += len;
}

// z[t][b] = sum_{i < R} V_i[t][b] y[i][b]
__global__ void ras_combine_kernel(const double* V, int Np, int B, const double* y, double* z) {
    const long long n = (long long)Np * B;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        double s = 0.0;
        for (int i = 0; i < kRasRestart; ++i) s += V[(long long)i * n + t] * y[(long long)i * B + b];
        z[t] = s;
    }
}

__global__ void ras_export_kernel(const double* c, double* out, int Np, int B) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)Np * B;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        out[(long long)b * Np + t / B] = c[t];
    }
}

}  // namespace

// ---------------------------------------------------------------- host side

struct RasOnline {
    int M = 0, Np = 0, max_ring = 0, max_patch_ents = 0, n_ring_tot = 0, n_ent = 0, max_k = 0;
    bool coarse = false;
    std::vector<int> ring_base_h;
    DevBuf<double> Bm, rows, z, aug;
    DevBuf<long long> b_off, ent_row;
    DevBuf<int> ring_base, bnd, ent_ptr, ent_patch, coef_patch;
    // work space for kRasMaxBatch data sets, allocated on the first solve
    bool work = false;
    int n_chunks = 0;
    DevBuf<double> V, x, f, r, t, sv, w, zc, p, q, part, hh, htmp, g, cs, sn, y, st, e, gv;
};

static RasArgs ras_args(const Basis& Bs, const RasOnline& R, int B) {
    RasArgs A{};
    A.M = R.M;
    A.B = B;
    A.k = Bs.d_k.p;
    A.c_off = Bs.d_c_off.p;
    A.b_off = R.b_off.p;
    A.Bm = R.Bm.p;
    A.ring_base = R.ring_base.p;
    A.bnd = R.bnd.p;
    A.ent_ptr = R.ent_ptr.p;
    A.ent_patch = R.ent_patch.p;
    A.ent_row = R.ent_row.p;
    A.rows = R.rows.p;
    return A;
}

// position of a domain-boundary node in the global ring (extract.cu)
int domain_ring_pos(int N, int i, int j);

static int ew_grid(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms() * 8));
}

msp_status ras_setup(Basis& Bs, const Medium& F, bool coarse, cudaStream_t s) {
    const int M = (int)Bs.patches.size(), N = Bs.N;
    MSP_CHECK_ARG(F.sampled, "msp_ras_setup: the full-basis medium has not been sampled (msp_sample_patches)");
    MSP_CHECK_ARG(F.N == N && (int)F.patches.size() == M,
                  "msp_ras_setup: the full-basis medium does not have the basis's grid and partition");
    for (int m = 0; m < M; ++m) {
        const PatchDev &a = Bs.patches[m], &b = F.patches[m];
        MSP_CHECK_ARG(a.x0 == b.x0 && a.x1 == b.x1 && a.y0 == b.y0 && a.y1 == b.y1 && a.X0 == b.X0 && a.X1 == b.X1 &&
                          a.Y0 == b.Y0 && a.Y1 == b.Y1,
                      "msp_ras_setup: the full-basis medium's patches differ from the basis's");
        MSP_CHECK_ARG(b.samples == 0 && b.cols == b.n_ring && b.n_ring == a.n_ring,
                      "msp_ras_setup: the medium is not a full-basis medium (msp_build_medium_full)");
    }
    auto R = std::make_shared<RasOnline>();
    R->M = M;
    R->Np = Bs.Np;
    R->coarse = coarse;
    // ring tables: per global ring node its domain-boundary position or its owners
    std::vector<int> ring_base(M + 1, 0), bnd, ent_ptr(1, 0), ent_patch, ent_loc, ent_nb, nb_ptr(1, 0), nb_patch;
    std::vector<double> ent_chi;
    std::vector<long long> ent_row, b_off(M + 1, 0);
    long long row_elems = 0;
    const int mx = Bs.mx, my = Bs.my;
    for (int m = 0; m < M; ++m) {
        const PatchDev& P = Bs.patches[m];
        const int e_first = (int)ent_patch.size();
        std::vector<int> nbs;
        for (int r = 0; r < P.n_ring; ++r) {
            int i, j;
            ring_node(P.X0, P.X1, P.Y0, P.Y1, r, i, j);
            if (i == 0 || j == 0 || i == N || j == N) {
                bnd.push_back(domain_ring_pos(N, i, j));
            } else {
                bnd.push_back(-1);
                // patches whose closed box holds (i, j): the break interval of i (and the
                // one before it when i sits on a break), likewise for j, in patch order
                int px[2], qy[2], npx = 0, nqy = 0;
                {
                    const int p1 = (int)(std::upper_bound(Bs.xb.begin(), Bs.xb.end(), i) - Bs.xb.begin()) - 1;
                    const int q1 = (int)(std::upper_bound(Bs.yb.begin(), Bs.yb.end(), j) - Bs.yb.begin()) - 1;
                    if (p1 > 0 && Bs.xb[p1] == i) px[npx++] = p1 - 1;
                    if (p1 >= 0 && p1 < mx) px[npx++] = p1;
                    if (q1 > 0 && Bs.yb[q1] == j) qy[nqy++] = q1 - 1;
                    if (q1 >= 0 && q1 < my) qy[nqy++] = q1;
                }
                int own[4], no = 0;
                for (int a = 0; a < nqy; ++a)
                    for (int c = 0; c < npx; ++c) own[no++] = px[c] + qy[a] * mx;
                MSP_CHECK_ARG(no > 0, "msp_ras_setup: a ring node lies in no patch");
                for (int o = 0; o < no; ++o) {
                    const PatchDev& Pn = Bs.patches[own[o]];
                    ent_patch.push_back(own[o]);
                    ent_loc.push_back((i - Pn.x0) + (j - Pn.y0) * (Pn.x1 - Pn.x0 + 1));
                    ent_chi.push_back(1.0 / no);
                    ent_row.push_back(row_elems);
                    row_elems += Bs.k[own[o]];
                    if (std::find(nbs.begin(), nbs.end(), own[o]) == nbs.end()) nbs.push_back(own[o]);
                }
            }
            ent_ptr.push_back((int)ent_patch.size());
        }
        std::sort(nbs.begin(), nbs.end());
        for (int e = e_first; e < (int)ent_patch.size(); ++e)
            ent_nb.push_back(nb_ptr.back() + (int)(std::find(nbs.begin(), nbs.end(), ent_patch[e]) - nbs.begin()));
        for (int n : nbs) nb_patch.push_back(n);
        nb_ptr.push_back((int)nb_patch.size());
        ring_base[m + 1] = ring_base[m] + P.n_ring;
        b_off[m + 1] = b_off[m] + (long long)Bs.k[m] * P.n_ring;
        R->max_ring = std::max(R->max_ring, P.n_ring);
        R->max_k = std::max(R->max_k, Bs.k[m]);
        R->max_patch_ents = std::max(R->max_patch_ents, (int)ent_patch.size() - e_first);
    }
    R->n_ring_tot = ring_base[M];
    R->n_ent = (int)ent_patch.size();
    R->ring_base_h = ring_base;
    std::vector<int> coef_patch(std::max(Bs.Np, 1), 0);
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < Bs.k[m]; ++i) coef_patch[Bs.c_off[m] + i] = m;
    b_off.pop_back();
    MSP_TRY(upload(R->ring_base, ring_base, s));
    MSP_TRY(upload(R->bnd, bnd, s));
    MSP_TRY(upload(R->ent_ptr, ent_ptr, s));
    MSP_TRY(upload(R->ent_patch, ent_patch, s));
    MSP_TRY(upload(R->ent_row, ent_row, s));
    MSP_TRY(upload(R->b_off, b_off, s));
    MSP_TRY(upload(R->coef_patch, coef_patch, s));
    DevBuf<int> d_loc, d_nb, d_nb_ptr, d_nb_patch;
    DevBuf<double> d_chi;
    MSP_TRY(upload(d_loc, ent_loc, s));
    MSP_TRY(upload(d_chi, ent_chi, s));
    MSP_TRY(upload(d_nb, ent_nb, s));
    MSP_TRY(upload(d_nb_ptr, nb_ptr, s));
    MSP_TRY(upload(d_nb_patch, nb_patch, s));
    long long b_elems = 0;
    for (int m = 0; m < M; ++m) b_elems += (long long)Bs.k[m] * Bs.patches[m].n_ring;
    MSP_TRY(R->Bm.alloc((size_t)std::max<long long>(b_elems, 1), s));
    MSP_TRY(R->rows.alloc((size_t)std::max<long long>(row_elems, 1), s));
    // B_m = Q_m^T G~_m: one product per patch with k_m > 0
    std::vector<GemmDesc> gd;
    int max_k = 1, max_r = 1;
    for (int m = 0; m < M; ++m) {
        const PatchDev& P = Bs.patches[m];
        const int km = Bs.k[m];
        if (km == 0) continue;
        gd.push_back(GemmDesc{Bs.Q.p + Bs.q_off[m], F.snaps.p + F.patches[m].snap_offset, R->Bm.p + b_off[m], km,
                              P.n_ring, P.n_k, P.n_k, P.n_k, km, 1.0, 0.0});
        max_k = std::max(max_k, km);
        max_r = std::max(max_r, P.n_ring);
    }
    if (!gd.empty()) {
        DevBuf<GemmDesc> d_gd;
        MSP_TRY(upload(d_gd, gd, s));
        if (fp64_gemm_engine() == MSP_GEMM_TENSOR_CORES && ozaki_gemm_supported(gd)) {
            OzakiWork ozw;
            MSP_TRY(ozaki_gemm_batched(gd, d_gd.p, true, false, s, ozw));
            MSP_TRY(ozaki_check(ozw, s));   // synchronises
        } else {
            gemm_batched<double>(d_gd.p, (int)gd.size(), max_k, max_r, true, false, s);
        }
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaStreamSynchronize(s));   // descriptors go out of scope
    }
    if (R->n_ent > 0) {
        ras_rows_kernel<<<ew_grid((long long)R->n_ent * 32), 256, 0, s>>>(Bs.Q.p, Bs.d_q_off.p, Bs.d_patches.p, Bs.d_k.p,
                                                                       R->n_ent, R->ent_patch.p, d_loc.p, d_chi.p,
                                                                       R->ent_row.p, R->rows.p);
        count_launches(1);
    }
    MSP_CUDA(cudaGetLastError());
    if (coarse && M > 0) {
        MSP_TRY(R->z.alloc((size_t)std::max(Bs.Np, 1), s));
        MSP_TRY(R->aug.alloc((size_t)M * 2 * M, s));
        ras_z_kernel<<<M, 256, 0, s>>>(Bs.Q.p, Bs.d_q_off.p, Bs.d_patches.p, Bs.d_k.p, Bs.d_c_off.p, R->z.p);
        ras_aug_init_kernel<<<ew_grid(2LL * M * M), 256, 0, s>>>(R->aug.p, M);
        const RasArgs A = ras_args(Bs, *R, 1);
        const size_t smem = sizeof(double) * ((size_t)R->max_ring + R->max_patch_ents);
        MSP_CUDA(cudaFuncSetAttribute(ras_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ras_coarse_kernel<<<M, 256, smem, s>>>(A, R->z.p, d_nb_ptr.p, d_nb_patch.p, d_nb.p, R->aug.p);
        count_launches(3);
        DevBuf<double> col;
        DevBuf<int> fail;
        MSP_TRY(col.alloc((size_t)M, s));
        MSP_TRY(fail.alloc(1, s));
        MSP_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), s));
        for (int k = 0; k < M; ++k) {
            ras_gj_pivot_kernel<<<1, 1024, 0, s>>>(R->aug.p, M, k, col.p, fail.p);
            ras_gj_elim_kernel<<<ew_grid((long long)M * (2LL * M - k - 1)), 256, 0, s>>>(R->aug.p, M, k, col.p);
        }
        count_launches(2LL * M);
        MSP_CUDA(cudaGetLastError());
        int hfail = 0;
        MSP_CUDA(cudaMemcpyAsync(&hfail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        if (hfail) {
            set_error("msp_ras_setup: the coarse matrix Z^T (I - T) Z is singular to working precision");
            return MSP_ERR_BREAKDOWN;
        }
    }
    MSP_CUDA(cudaStreamSynchronize(s));   // host tables and temporaries go out of scope
    Bs.ras = R;
    return MSP_OK;
}

static msp_status ras_work(const Basis& Bs, RasOnline& R, cudaStream_t s) {
    if (R.work) return MSP_OK;
    const size_t np = (size_t)std::max(Bs.Np, 1), cb = kRasMaxBatch, Rr = kRasRestart;
    R.n_chunks = std::max(1, (Bs.Np + kRasChunk - 1) / kRasChunk);
    MSP_TRY(R.V.alloc((Rr + 1) * np * cb, s));
    MSP_TRY(R.x.alloc(np * cb, s));
    MSP_TRY(R.f.alloc(np * cb, s));
    MSP_TRY(R.r.alloc(np * cb, s));
    MSP_TRY(R.t.alloc(np * cb, s));
    MSP_TRY(R.sv.alloc(np * cb, s));
    MSP_TRY(R.w.alloc(np * cb, s));
    MSP_TRY(R.zc.alloc(np * cb, s));
    MSP_TRY(R.p.alloc((size_t)std::max(R.M, 1) * cb, s));
    MSP_TRY(R.q.alloc((size_t)std::max(R.M, 1) * cb, s));
    MSP_TRY(R.part.alloc((size_t)R.n_chunks * (Rr + 1) * cb, s));
    MSP_TRY(R.hh.alloc(Rr * (Rr + 1) * cb, s));
    MSP_TRY(R.htmp.alloc((Rr + 1) * cb, s));
    MSP_TRY(R.g.alloc((Rr + 1) * cb, s));
    MSP_TRY(R.cs.alloc(Rr * cb, s));
    MSP_TRY(R.sn.alloc(Rr * cb, s));
    MSP_TRY(R.y.alloc(Rr * cb, s));
    MSP_TRY(R.st.alloc(8 * cb, s));
    MSP_TRY(R.e.alloc((size_t)std::max(Bs.n_slots, 1) * cb, s));
    MSP_TRY(R.gv.alloc((size_t)std::max(R.n_ring_tot, 1) * cb, s));
    R.work = true;
    return MSP_OK;
}

// One batch of at most kRasMaxBatch data sets.
static msp_status ras_batch(Basis& Bs, RasOnline& R, const double* phi, int B, double tol, int max_iter, double* u,
                            double* c_out, int* iters_host, cudaStream_t s, bool* not_conv, bool* nonfinite) {
    const int M = R.M, Np = Bs.Np, n4 = 4 * Bs.N, Rr = kRasRestart;
    const long long nb = (long long)Np * B;
    const RasArgs A = ras_args(Bs, R, B);
    const size_t smem = sizeof(double) * ((size_t)R.max_ring * B + (size_t)std::max(kRasThreads, R.max_k));
    MSP_CUDA(cudaFuncSetAttribute(ras_bm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ring_grid = std::max(1, std::min((R.n_ring_tot + 31) / 32, num_sms() * 16));
    auto apply = [&](const double* x, const double* a, double* out, int mode) {
        ras_ring_kernel<<<ring_grid, kRasThreads, 0, s>>>(A, R.n_ring_tot, x, phi, n4, R.gv.p, mode);
        ras_bm_kernel<<<M, kRasThreads, smem, s>>>(A, R.gv.p, a, out);
        count_launches(2);
    };
    auto dots = [&](const double* V, int nvec, const double* w) {
        const dim3 grid(R.n_chunks, nvec);
        if (B == 1) ras_dots_kernel<1><<<grid, kRasThreads, 0, s>>>(V, w, Np, B, R.n_chunks, R.part.p);
        else if (B == 2) ras_dots_kernel<2><<<grid, kRasThreads, 0, s>>>(V, w, Np, B, R.n_chunks, R.part.p);
        else if (B <= 4) ras_dots_kernel<4><<<grid, kRasThreads, 0, s>>>(V, w, Np, B, R.n_chunks, R.part.p);
        else if (B <= 8) ras_dots_kernel<8><<<grid, kRasThreads, 0, s>>>(V, w, Np, B, R.n_chunks, R.part.p);
        else ras_dots_kernel<kRasMaxBatch><<<grid, kRasThreads, 0, s>>>(V, w, Np, B, R.n_chunks, R.part.p);
        count_launches(1);
    };
    auto finalize = [&](int nvec, double* hcol, int mode, int slot) {
        ras_finalize_kernel<<<std::max(1, (nvec * B + 7) / 8), 256, 0, s>>>(R.part.p, nvec, R.n_chunks, B, R.htmp.p, hcol,
                                                                          R.st.p, mode, slot);
        count_launches(1);
    };
    // out = v + Z E^{-1} Z^T T v (the A-DEF2 preconditioner; out = v with no coarse space)
    auto precond = [&](const double* v, const double* base, double* out) {
        if (R.coarse) {
            apply(v, nullptr, R.t.p, 0);
            ras_zt_kernel<<<std::max(1, (M + 7) / 8), 256, 0, s>>>(A, R.z.p, R.t.p, R.p.p);
            ras_einv_kernel<<<std::max(1, (M + 7) / 8), 256, 0, s>>>(A, R.aug.p, R.p.p, R.q.p);
            count_launches(2);
        }
        ras_prolong_kernel<<<ew_grid(nb), 256, 0, s>>>(Np, B, R.coef_patch.p, R.z.p, R.coarse ? R.q.p : nullptr, v, base,
                                                       out);
        count_launches(1);
    };
    std::vector<double> sth(8 * (size_t)B);
    auto read_status = [&]() -> msp_status {
        MSP_CUDA(cudaMemcpyAsync(sth.data(), R.st.p, sizeof(double) * 8 * B, cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        return MSP_OK;
    };
    auto all_stopped = [&]() {
        for (int b = 0; b < B; ++b)
            if (sth[8 * b + 6] == 0.0) return false;
        return true;
    };
    MSP_CUDA(cudaMemsetAsync(R.st.p, 0, sizeof(double) * 8 * B, s));
    MSP_CUDA(cudaMemsetAsync(R.x.p, 0, sizeof(double) * nb, s));
    apply(nullptr, nullptr, R.f.p, 1);   // F phi
    dots(R.f.p, 1, R.f.p);
    finalize(1, nullptr, 2, 0);          // |F phi|
    for (int cycle = 0;; ++cycle) {
        const double* r = R.f.p;
        if (cycle > 0) {
            apply(R.x.p, nullptr, R.t.p, 0);
            ras_residual_kernel<<<ew_grid(nb), 256, 0, s>>>(nb, R.f.p, R.x.p, R.t.p, R.r.p);
            count_launches(1);
            r = R.r.p;
        }
        dots(r, 1, r);
        finalize(1, nullptr, 2, 7);      // beta
        ras_scale_kernel<<<ew_grid(nb), 256, 0, s>>>(nb, B, r, R.st.p + 7, 8, R.V.p);
        ras_cycle_start_kernel<<<1, 32, 0, s>>>(R.st.p, R.g.p, B, tol, max_iter);
        count_launches(2);
        MSP_CUDA(cudaGetLastError());
        MSP_TRY(read_status());
        if (all_stopped()) break;
        for (int j = 0; j < Rr; ++j) {
            const double* vj = R.V.p + (long long)j * nb;
            precond(vj, nullptr, R.sv.p);
            apply(R.sv.p, R.sv.p, R.w.p, 0);              // w = s - T s
            double* hcol = R.hh.p + (long long)j * (Rr + 1) * B;
            MSP_CUDA(cudaMemsetAsync(hcol, 0, sizeof(double) * (Rr + 1) * B, s));
            for (int pass = 0; pass < 2; ++pass) {        // classical Gram-Schmidt, twice
                dots(R.V.p, j + 1, R.w.p);
                finalize(j + 1, hcol, 0, 0);
                ras_orth_kernel<<<ew_grid(nb), 256, 0, s>>>(R.V.p, j + 1, Np, B, R.htmp.p, R.w.p);
                count_launches(1);
            }
            dots(R.w.p, 1, R.w.p);
            finalize(1, hcol + (long long)(j + 1) * B, 1, 0);
            ras_scale_kernel<<<ew_grid(nb), 256, 0, s>>>(nb, B, R.w.p, hcol + (long long)(j + 1) * B, 1,
                                                         R.V.p + (long long)(j + 1) * nb);
            ras_givens_kernel<<<1, 32, 0, s>>>(R.hh.p, R.cs.p, R.sn.p, R.g.p, R.st.p, j, B, tol, max_iter);
            count_launches(2);
            MSP_CUDA(cudaGetLastError());
            MSP_TRY(read_status());
            if (all_stopped()) break;
        }
        ras_backsolve_kernel<<<1, 32, 0, s>>>(R.hh.p, R.g.p, R.st.p, R.y.p, B);
        ras_combine_kernel<<<ew_grid(nb), 256, 0, s>>>(R.V.p, Np, B, R.y.p, R.zc.p);
        count_launches(2);
        precond(R.zc.p, R.x.p, R.x.p);                  // x += M^{-1} (V y)
        MSP_CUDA(cudaGetLastError());
    }
    for (int b = 0; b < B; ++b) {
        if (sth[8 * b + 5] != 0.0) *nonfinite = true;
        else if (sth[8 * b + 4] == 0.0) *not_conv = true;
        if (iters_host) iters_host[b] = (int)sth[8 * b + 3];
    }
    if (u) reconstruct_coefficients(Bs, R.x.p, B, R.e.p, phi, n4, u, s);
    if (c_out) {
        ras_export_kernel<<<ew_grid(nb), 256, 0, s>>>(R.x.p, c_out, Np, B);
        count_launches(1);
    }
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

msp_status ras_solve(Basis& Bs, const double* phi, int batch, double tol, int max_iter, double* u, double* c_out,
                     int* iters_host, cudaStream_t s) {
    if (!Bs.ras) {
        set_error("msp_online_solve_ras: msp_ras_setup has not been called on this basis");
        return MSP_ERR_INVALID_ARG;
    }
    RasOnline& R = *Bs.ras;
    MSP_TRY(ras_work(Bs, R, s));
    const int n4 = 4 * Bs.N;
    const long long nn = (long long)(Bs.N + 1) * (Bs.N + 1);
    bool not_conv = false, nonfinite = false;
    for (int b0 = 0; b0 < batch; b0 += kRasMaxBatch) {
        const int B = std::min(kRasMaxBatch, batch - b0);
        MSP_TRY(ras_batch(Bs, R, phi + (long long)b0 * n4, B, tol, max_iter, u ? u + (long long)b0 * nn : nullptr,
                          c_out ? c_out + (long long)b0 * Bs.Np : nullptr, iters_host ? iters_host + b0 : nullptr, s,
                          &not_conv, &nonfinite));
    }
    if (nonfinite) {
        set_error("msp_online_solve_ras: a data set's residual is not finite (NaN or Inf in phi)");
        return MSP_ERR_NOT_CONVERGED;
    }
    if (not_conv) {
        set_error("msp_online_solve_ras: some data sets stopped at max_iter");
        return MSP_ERR_NOT_CONVERGED;
    }
    return MSP_OK;
}

}  // namespace msp
