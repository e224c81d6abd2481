// Direct batched local solves: the local solver of Algorithm alg:summary
// (LocalPDESolver on every buffered patch, Eq. elliptic_random for the ring
// data) as a factorisation of each patch's operator that every column of the
// patch shares, in place of an iteration per column.  The paper allows any
// standard local solver; this one is a block LDL^T over the grid rows.
//
// Scaled operator A~ = S A S, S = diag(A)^(-1/2), on the interior nx x ny nodes:
// block tridiagonal over the rows j = 0..ny-1, diagonal blocks T_j (tridiagonal,
// unit diagonal, off-diagonal -a_E s s), couplings -diag(c_j) between rows j and
// j+1 with c_j[i] = a_N(i, j+1/2) s_j[i] s_{j+1}[i].
//   Factorisation (FP32):  Z_0 = T_0,  Z_j = T_j - C_{j-1} W_{j-1} C_{j-1},
//                          W_j = Z_j^{-1}  (Gauss-Jordan; Z_j is SPD).
//   Solve A~ d = g:        forward  y_0 = g_0,  w_j = W_j y_j,  y_{j+1} = g_{j+1} + c_j o w_j;
//                          backward d_{ny-1} = w_{ny-1},  d_j = w_j + W_j (c_j o d_{j+1}).
// Every step of both sweeps is a product of the nx x nx block W_j with the
// nx x 32 block of one chunk of 32 columns, so the sweeps are dense contractions
// that the CTA of a chunk runs out of shared memory.
// Accuracy comes from FP64 iterative refinement: r = b - A x in FP64 (b from
// the ring data: x holds the ring values), g = S r rounded to FP32, x += S d,
// until |r| <= tol |b| per column (a few passes: the FP32 factor reduces the
// residual by about 1e-5 per pass on the workloads' media).
//
// Storage (per patch, offsets in the Direct tables):
//   W  ny x ld x ld floats, W_j transposed (ld = nx rounded up to 4, zero padding)
//   s  ny x nx doubles; D  ny x nx floats (row j: c_j, zero on the last row)
//   X  cols x (ny+2) x (nx+2) doubles: the FP64 iterate with its ring values
//   R  chunks x ny x 32 x nx floats: the scaled residual g, column-major per row
//   K  chunks x ny x ld x 32 floats: the forward sweep's w_j
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <vector>

namespace msp {

namespace {

constexpr int kDirThreads = 256;
constexpr int kCB = 32;          // columns per chunk
constexpr int kDirMaxLd = 160;   // widest padded interior row handled (5 groups of 32 rows)
constexpr int kDirMaxPasses = 8; // refinement passes at most

struct DirArgs {
    int N;
    const double* aE;
    const double* aN;
    const PatchDev* patches;
    const int* bpos;
    uint64_t seed;
    const long long *w_off, *s_off, *x_off, *r_off, *k_off;
    const int* col_base;
    const int2* cols;
    const int4* chunks;
    const int* stat_idx;
    float* W;
    float* D;
    float* R;
    float* K;
    double* s;
    double* X;
    double* b2;
    double* r2;
    int* active;
    int* passes;
    double* snaps;
    int* stats;
    double tol;
};

struct Geo {
    int nx, ny, wd, hd, ld;
};

__host__ __device__ inline Geo geo(const PatchDev& P) {
    Geo g;
    g.nx = P.X1 - P.X0 - 1;
    g.ny = P.Y1 - P.Y0 - 1;
    g.wd = g.nx + 2;
    g.hd = g.ny + 2;
    g.ld = g.nx > 0 ? (g.nx + 3) / 4 * 4 : 0;
    return g;
}

// Position of element (k, c), c < 32, in a swizzled k x 32 block: the 16-byte
// group of c is xor-ed with k mod 8, so that 8 consecutive k of 4 consecutive c
// (the transposing stores) and 32 consecutive k of one group (the GEMM's stores)
// hit distinct banks, while each group of 4 columns stays one aligned float4.
__device__ __forceinline__ int swz(int k, int c) { return k * kCB + ((((c >> 2) ^ (k & 7))) << 2) + (c & 3); }

// ------------------------------------------------------------------ factor
// One CTA per patch: s, the couplings c_j, and W_j = Z_j^{-1} row by row.  The
// block lives in registers: thread (tr, tc) of a 16 x 16 layout holds the TS x TS
// sub-block of rows tr TS .., columns tc TS .. (TS = ceil(ld / 16), one value for the
// launch).  Z_j = T_j - C_{j-1} W_{j-1} C_{j-1} is formed elementwise from the
// registers holding W_{j-1}; Gauss-Jordan inversion in place without pivoting (Z_j
// is SPD), one barrier per pivot: after updating, the owners of row and column k+1
// publish them to double-buffered shared rows for the next pivot.  W_j^T goes to
// global memory through a padded shared copy (coalesced stores).
template <int TS>
__global__ void __launch_bounds__(kDirThreads) direct_factor_kernel(DirArgs A) {
    extern __shared__ __align__(16) float fsm[];
    const int m = blockIdx.x;
    const PatchDev P = A.patches[m];
    const Geo g = geo(P);
    if (g.nx < 1 || g.ny < 1) return;
    const int n = g.nx, ld = g.ld, N = A.N;
    constexpr int kW = 16 * TS;    // rows (and columns) the thread layout covers
    float* Zs = fsm;               // ld x (ld + 1): staging of W_j for the transposed store
    float* rb = Zs + ld * (ld + 1);   // 2 x kW: row k of the current block
    float* cb = rb + 2 * kW;          // 2 x kW: column k
    double* sv = A.s + A.s_off[m];
    float* Dv = A.D + A.s_off[m];
    float* Wout = A.W + A.w_off[m];
    const double* aE = A.aE;
    const double* aN = A.aN;
    for (int t = threadIdx.x; t < n * g.ny; t += blockDim.x) {
        const int j = t / n, i = t - j * n;
        const long long gi = P.X0 + 1 + i, gj = P.Y0 + 1 + j;
        const double d = aE[gj * N + gi - 1] + aE[gj * N + gi] + aN[(gj - 1) * (N + 1) + gi] + aN[gj * (N + 1) + gi];
        sv[t] = 1.0 / sqrt(d);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * g.ny; t += blockDim.x) {
        const int j = t / n, i = t - j * n;
        float c = 0.f;
        if (j + 1 < g.ny) {
            const long long gi = P.X0 + 1 + i, gj = P.Y0 + 1 + j;
            c = (float)(aN[gj * (N + 1) + gi] * sv[t] * sv[t + n]);
        }
        Dv[t] = c;
    }
    __syncthreads();
    const int r0 = (threadIdx.x >> 4) * TS, c0 = (threadIdx.x & 15) * TS;
    float z[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) z[a][b] = 0.f;
    for (int j = 0; j < g.ny; ++j) {
        const long long gj = P.Y0 + 1 + j;
        // Z_j from T_j and the registers holding W_{j-1}; identity on the padding
#pragma unroll
        for (int a = 0; a < TS; ++a) {
            const int r = r0 + a;
            const float dr = (j > 0 && r < n) ? Dv[(j - 1) * n + r] : 0.f;
#pragma unroll
            for (int b = 0; b < TS; ++b) {
                const int c = c0 + b;
                float v = (r == c) ? 1.f : 0.f;
                if (r < n && c < n) {
                    if (c == r + 1 || c + 1 == r) {
                        const int i = min(r, c);
                        v = -(float)(aE[gj * N + P.X0 + 1 + i] * sv[j * n + i] * sv[j * n + i + 1]);
                    }
                    if (j > 0) v -= dr * z[a][b] * Dv[(j - 1) * n + c];
                }
                z[a][b] = v;
            }
        }
        // publish row 0 and column 0
        if (r0 == 0)
#pragma unroll
            for (int b = 0; b < TS; ++b) rb[c0 + b] = z[0][b];
        if (c0 == 0)
#pragma unroll
            for (int a = 0; a < TS; ++a) cb[r0 + a] = z[a][0];
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            const int p = (k & 1) * kW, q = kW - p;
            const float inv = 1.f / cb[p + k];
            float fr[TS], rk[TS];
#pragma unroll
            for (int a = 0; a < TS; ++a) fr[a] = cb[p + r0 + a] * inv;
#pragma unroll
            for (int b = 0; b < TS; ++b) rk[b] = rb[p + c0 + b];
#pragma unroll
            for (int a = 0; a < TS; ++a) {
                const int r = r0 + a;
#pragma unroll
                for (int b = 0; b < TS; ++b) {
                    const int c = c0 + b;
                    float v = z[a][b];
                    if (r != k && c != k) v = fmaf(-fr[a], rk[b], v);
                    else if (r == k && c != k) v = rk[b] * inv;
                    else if (r != k) v = -fr[a];
                    else v = inv;
                    z[a][b] = v;
                }
            }
            // publish row k+1 and column k+1 of the updated block for the next pivot
            const int k1 = k + 1;
            if (k1 < n) {
#pragma unroll
                for (int a = 0; a < TS; ++a)
                    if (r0 + a == k1)
#pragma unroll
                        for (int b = 0; b < TS; ++b) rb[q + c0 + b] = z[a][b];
#pragma unroll
                for (int b = 0; b < TS; ++b)
                    if (c0 + b == k1)
#pragma unroll
                        for (int a = 0; a < TS; ++a) cb[q + r0 + a] = z[a][b];
            }
            __syncthreads();
        }
        // W_j^T to global (padding zero) through the padded shared copy
#pragma unroll
        for (int a = 0; a < TS; ++a)
#pragma unroll
            for (int b = 0; b < TS; ++b) {
                const int r = r0 + a, c = c0 + b;
                if (r < ld && c < ld) Zs[r * (ld + 1) + c] = (r < n && c < n) ? z[a][b] : 0.f;
            }
        __syncthreads();
        float* wj = Wout + (long long)j * ld * ld;
        for (int t = threadIdx.x; t < ld * ld; t += blockDim.x) {
            const int r = t / ld, c = t - r * ld;
            wj[t] = Zs[c * (ld + 1) + r];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ init
// One CTA per column: the FP64 iterate is the ring data with a zero interior.
__global__ void __launch_bounds__(kDirThreads) direct_init_kernel(DirArgs A) {
    const int gcol = blockIdx.x;
    const int2 mc = A.cols[gcol];
    const int m = mc.x, col = mc.y;
    const PatchDev P = A.patches[m];
    const Geo g = geo(P);
    double* x = A.X + A.x_off[m] + (long long)col * g.hd * g.wd;
    for (int t = threadIdx.x; t < g.hd * g.wd; t += blockDim.x) x[t] = 0.0;
    __syncthreads();
    if (col < P.samples) {
        const int npairs = (P.n_ring + 1) >> 1;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            const double2 z = gaussian_pair(A.seed, (uint32_t)q, (uint32_t)col, (uint32_t)m, kTagElliptic);
            int i, j;
            ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q, i, j);
            x[(j - P.Y0) * g.wd + (i - P.X0)] = z.x;
            if (2 * q + 1 < P.n_ring) {
                ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q + 1, i, j);
                x[(j - P.Y0) * g.wd + (i - P.X0)] = z.y;
            }
        }
    } else if (threadIdx.x == 0) {
        const int t0 = A.bpos[P.bpos_offset + (col - P.samples)];
        int i, j;
        ring_node(P.X0, P.X1, P.Y0, P.Y1, t0, i, j);
        x[(j - P.Y0) * g.wd + (i - P.X0)] = 1.0;
    }
    if (threadIdx.x == 0) A.passes[gcol] = 0;
}

// ------------------------------------------------------------------ residual
// One CTA per chunk: r = b - A x = -(A x) (x carries the ring data) in FP64, the
// scaled residual g = S r in FP32 for the next solve, |r|^2 per column in a fixed
// order (warp w takes columns w, w+8, w+16, w+24, lanes along the row).  first:
// |b| = |r| of the initial iterate.  A column stays active while |r| > tol |b|.
__global__ void __launch_bounds__(kDirThreads) direct_residual_kernel(DirArgs A, int first) {
    const int4 ch = A.chunks[blockIdx.x];
    const int m = ch.x, c0 = ch.y, nc = ch.z, chunk = ch.w;
    const int gbase = A.col_base[m] + c0;
    __shared__ int s_act[kCB];
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < kCB) {
        const int a = threadIdx.x < nc ? (first ? 1 : A.active[gbase + threadIdx.x]) : 0;
        s_act[threadIdx.x] = a;
        if (a) atomicOr(&s_any, 1);
    }
    __syncthreads();
    if (!s_any) return;
    const PatchDev P = A.patches[m];
    const Geo g = geo(P);
    const int n = g.nx, N = A.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* sv = A.s + A.s_off[m];
    float* Rc = A.R + A.r_off[m] + (long long)chunk * g.ny * kCB * n;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < g.ny; ++j) {
        const long long gj = P.Y0 + 1 + j;
        for (int q = 0; q < 4; ++q) {
            const int c = warp + 8 * q;
            if (c >= nc || !s_act[c]) continue;
            const double* x = A.X + A.x_off[m] + (long long)(c0 + c) * g.hd * g.wd + (j + 1) * g.wd + 1;
            float* rr = Rc + ((long long)j * kCB + c) * n;
            // first pass: the interior of the iterate is zero, so only nodes next to the
            // ring have a nonzero residual; the others are written as the zeros they are
            const bool edge_only = first && j > 0 && j + 1 < g.ny;
            for (int k = lane; k < n; k += 32) {
                if (edge_only && k > 0 && k + 1 < n) {
                    rr[k] = 0.f;
                    continue;
                }
                const long long gi = P.X0 + 1 + k;
                const double ae = A.aE[gj * N + gi], aw = A.aE[gj * N + gi - 1];
                const double an = A.aN[gj * (N + 1) + gi], as = A.aN[(gj - 1) * (N + 1) + gi];
                const double xc = x[k];
                const double r = ae * (x[k + 1] - xc) + aw * (x[k - 1] - xc) + an * (x[k + g.wd] - xc) +
                                 as * (x[k - g.wd] - xc);
                acc[q] += r * r;
                rr[k] = (float)(r * sv[j * n + k]);
            }
        }
    }
    for (int q = 0; q < 4; ++q) {
        const int c = warp + 8 * q;
        const double t = warp_sum(acc[q]);
        if (lane == 0 && c < nc && s_act[c]) {
            const int gc = gbase + c;
            double b2 = first ? t : A.b2[gc];
            if (first) A.b2[gc] = t;
            else A.passes[gc] += 1;
            A.r2[gc] = t;
            A.active[gc] = (b2 > 0.0 && t > A.tol * A.tol * b2) ? 1 : 0;
        }
    }
}

// ------------------------------------------------------------------ solve
// d = Z^{-1} g by the two sweeps for one chunk of columns, then x += S d.
// GEMM mapping: warp w owns the 4 columns 4w..4w+3, lane l the rows l + 32 q.
template <int G>
__device__ __forceinline__ void chunk_gemm(const float* Ws, const float* Ys, int n, int ld, int lane, int warp,
                                           float (&acc)[G][4]) {
#pragma unroll
    for (int q = 0; q < G; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
        const float4 y = *reinterpret_cast<const float4*>(Ys + k * kCB + ((warp ^ (k & 7)) << 2));
        const float* wk = Ws + k * ld + lane;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const float w = wk[32 * q];
            acc[q][0] = fmaf(w, y.x, acc[q][0]);
            acc[q][1] = fmaf(w, y.y, acc[q][1]);
            acc[q][2] = fmaf(w, y.z, acc[q][2]);
            acc[q][3] = fmaf(w, y.w, acc[q][3]);
        }
    }
}

__device__ __forceinline__ void stage_block(float* dst, const float* src, int count) {
    for (int t = threadIdx.x * 4; t < count; t += blockDim.x * 4)
        *reinterpret_cast<float4*>(dst + t) = __ldg(reinterpret_cast<const float4*>(src + t));
}

template <int G>
__global__ void __launch_bounds__(kDirThreads) direct_solve_kernel(DirArgs A) {
    extern __shared__ __align__(16) float ssm[];
    const int4 ch = A.chunks[blockIdx.x];
    const int m = ch.x, c0 = ch.y, nc = ch.z, chunk = ch.w;
    const int gbase = A.col_base[m] + c0;
    __shared__ int s_act[kCB];
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < kCB) {
        const int a = threadIdx.x < nc ? A.active[gbase + threadIdx.x] : 0;
        s_act[threadIdx.x] = a;
        if (a) atomicOr(&s_any, 1);
    }
    __syncthreads();
    if (!s_any) return;
    const PatchDev P = A.patches[m];
    const Geo g = geo(P);
    const int n = g.nx, ld = g.ld, ny = g.ny;
    if (n < 1 || ny < 1) return;
    float* Ws = ssm;                                    // ld x ld (+ slack for the padded rows' reads)
    float* Ys = Ws + ld * ld + 32 * G;                  // swizzled ld x 32
    float* Ps = Ys + ld * kCB;                          // swizzled ld x 32: w_{j-1} / d_{j+1}
    const float* Wg = A.W + A.w_off[m];
    const float* Dg = A.D + A.s_off[m];
    const double* sv = A.s + A.s_off[m];
    const float* Rc = A.R + A.r_off[m] + (long long)chunk * ny * kCB * n;
    float* Kc = A.K + A.k_off[m] + (long long)chunk * ny * ld * kCB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nkb = (n + 7) >> 3;
    float acc[G][4];
    // ---- forward sweep
    for (int j = 0; j < ny; ++j) {
        stage_block(Ws, Wg + (long long)j * ld * ld, ld * ld);
        // y_j = g_j + c_{j-1} o w_{j-1}: lanes take 8 rows x 4 columns
        for (int p = warp; p < nkb * 8; p += 8) {
            const int k = 8 * (p >> 3) + (lane & 7), c = 4 * (p & 7) + (lane >> 3);
            if (k < n) {
                float v = 0.f;
                if (s_act[c]) {
                    v = Rc[((long long)j * kCB + c) * n + k];
                    if (j > 0) v = fmaf(Dg[(j - 1) * n + k], Ps[swz(k, c)], v);
                }
                Ys[swz(k, c)] = v;
            }
        }
        __syncthreads();
        chunk_gemm<G>(Ws, Ys, n, ld, lane, warp, acc);
        __syncthreads();   // Ps (w_{j-1}) and Ws no longer read
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int i = lane + 32 * q;
            if (i < n) {
                const float4 v = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
                *reinterpret_cast<float4*>(Ps + i * kCB + ((warp ^ (i & 7)) << 2)) = v;
                *reinterpret_cast<float4*>(Kc + ((long long)j * ld + i) * kCB + 4 * warp) = v;
            }
        }
        __syncthreads();
    }
    // ---- backward sweep and x += S d
    for (int j = ny - 1; j >= 0; --j) {
        if (j < ny - 1) {
            stage_block(Ws, Wg + (long long)j * ld * ld, ld * ld);
            for (int p = warp; p < nkb * 8; p += 8) {
                const int k = 8 * (p >> 3) + (lane & 7), c = 4 * (p & 7) + (lane >> 3);
                if (k < n) Ys[swz(k, c)] = Dg[j * n + k] * Ps[swz(k, c)];
            }
            __syncthreads();
            chunk_gemm<G>(Ws, Ys, n, ld, lane, warp, acc);
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        }
        __syncthreads();   // Ps (d_{j+1}) and Ws no longer read
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int i = lane + 32 * q;
            if (i < n) {
                const float4 w = *reinterpret_cast<const float4*>(Kc + ((long long)j * ld + i) * kCB + 4 * warp);
                const float4 v = make_float4(acc[q][0] + w.x, acc[q][1] + w.y, acc[q][2] + w.z, acc[q][3] + w.w);
                *reinterpret_cast<float4*>(Ps + i * kCB + ((warp ^ (i & 7)) << 2)) = v;
            }
        }
        __syncthreads();
        // x_j += S d_j on the active columns: warp w takes columns w, w+8, w+16, w+24
        for (int q = 0; q < 4; ++q) {
            const int c = warp + 8 * q;
            if (c >= nc || !s_act[c]) continue;
            double* x = A.X + A.x_off[m] + (long long)(c0 + c) * g.hd * g.wd + (j + 1) * g.wd + 1;
            for (int k = lane; k < n; k += 32) x[k] += sv[j * n + k] * (double)Ps[swz(k, c)];
        }
    }
}

// ------------------------------------------------------------------ finish
// One CTA per column: restriction to K_m and the column's statistics.
__global__ void __launch_bounds__(kDirThreads) direct_finish_kernel(DirArgs A) {
    const int gcol = blockIdx.x;
    const int2 mc = A.cols[gcol];
    const int m = mc.x, col = mc.y;
    const PatchDev P = A.patches[m];
    const Geo g = geo(P);
    const double* x = A.X + A.x_off[m] + (long long)col * g.hd * g.wd;
    const int wk = P.x1 - P.x0 + 1;
    double* out = A.snaps + P.snap_offset + (long long)col * P.n_k;
    for (int t = threadIdx.x; t < P.n_k; t += blockDim.x) {
        const int jj = t / wk, ii = t - jj * wk;
        out[t] = x[(P.y0 - P.Y0 + jj) * g.wd + (P.x0 - P.X0 + ii)];
    }
    if (threadIdx.x == 0) {
        const int si = A.stat_idx[gcol];
        const int ps = A.passes[gcol];
        A.stats[3 * si + 0] = ps;
        A.stats[3 * si + 1] = ps;
        A.stats[3 * si + 2] = A.active[gcol] ? 1 : 0;
    }
}

// Tables and buffers of the direct solver (once per medium).
msp_status direct_plan(Medium& M, cudaStream_t s) {
    Medium::Direct& D = M.dir;
    if (D.planned) return MSP_OK;
    const int np = (int)M.patches.size();
    std::vector<long long> w_off(np), s_off(np), x_off(np), r_off(np), k_off(np);
    std::vector<int> col_base(np);
    std::vector<int2> cols;
    std::vector<int4> chunks;
    long long w = 0, sv = 0, x = 0, r = 0, k = 0;
    int max_ld = 0, fsm = 0, csm = 0;
    for (int m = 0; m < np; ++m) {
        const PatchDev& P = M.patches[m];
        const Geo g = geo(P);
        const int nch = (P.cols + kCB - 1) / kCB;
        w_off[m] = w; s_off[m] = sv; x_off[m] = x; r_off[m] = r; k_off[m] = k;
        col_base[m] = (int)cols.size();
        const long long nx = std::max(g.nx, 0), ny = std::max(g.ny, 0);
        w += ny * g.ld * g.ld;
        sv += ny * nx;
        x += (long long)P.cols * g.hd * g.wd;
        r += (long long)nch * ny * kCB * nx;
        k += (long long)nch * ny * g.ld * kCB;
        for (int c = 0; c < P.cols; ++c) cols.push_back(make_int2(m, c));
        for (int q = 0; q < nch; ++q) chunks.push_back(make_int4(m, q * kCB, std::min(kCB, P.cols - q * kCB), q));
        max_ld = std::max(max_ld, g.ld);
        const int G = std::max(1, (g.ld + 31) / 32);
        fsm = std::max(fsm, (int)sizeof(float) * (g.ld * (g.ld + 1) + 4 * 16 * std::max(1, (g.ld + 15) / 16)));
        csm = std::max(csm, (int)sizeof(float) * (g.ld * g.ld + 32 * G + 2 * g.ld * kCB));
    }
    // statistics slot of every column: its position in the mixed-precision item order
    std::vector<int> stat_idx(cols.size(), 0);
    const std::vector<int2>& order = M.items_prec_host[1];
    for (size_t i = 0; i < order.size(); ++i) stat_idx[col_base[order[i].x] + order[i].y] = (int)i;
    D.n_cols = (int)cols.size();
    D.n_chunks = (int)chunks.size();
    D.max_nxp = max_ld;
    D.factor_smem_max = fsm;
    D.chunk_smem_max = csm;
    D.w_elems = w; D.s_elems = sv; D.x_elems = x; D.r_elems = r; D.k_elems = k;
    MSP_TRY(upload(D.w_off, w_off, s));
    MSP_TRY(upload(D.s_off, s_off, s));
    MSP_TRY(upload(D.x_off, x_off, s));
    MSP_TRY(upload(D.r_off, r_off, s));
    MSP_TRY(upload(D.k_off, k_off, s));
    MSP_TRY(upload(D.col_base, col_base, s));
    MSP_TRY(upload(D.cols, cols, s));
    MSP_TRY(upload(D.chunks, chunks, s));
    MSP_TRY(upload(D.stat_idx, stat_idx, s));
    MSP_TRY(D.W.alloc(std::max<long long>(1, w), s));
    MSP_TRY(D.s.alloc(std::max<long long>(1, sv), s));
    MSP_TRY(D.D.alloc(std::max<long long>(1, sv), s));
    MSP_TRY(D.X.alloc(std::max<long long>(1, x), s));
    MSP_TRY(D.R.alloc(std::max<long long>(1, r), s));
    MSP_TRY(D.K.alloc(std::max<long long>(1, k), s));
    MSP_TRY(D.b2.alloc(std::max(1, D.n_cols), s));
    MSP_TRY(D.r2.alloc(std::max(1, D.n_cols), s));
    MSP_TRY(D.active.alloc(std::max(1, D.n_cols), s));
    MSP_TRY(D.passes.alloc(std::max(1, D.n_cols), s));
    MSP_CUDA(cudaStreamSynchronize(s));   // the host tables above go out of scope
    D.planned = true;
    return MSP_OK;
}

DirArgs direct_args(Medium& M, const LocalSolveCfg& cfg) {
    Medium::Direct& D = M.dir;
    DirArgs A{};
    A.N = M.N;
    A.aE = M.aE.p;
    A.aN = M.aN.p;
    A.patches = M.patches_dev.p;
    A.bpos = M.bpos_dev.p;
    A.seed = cfg.seed;
    A.w_off = D.w_off.p; A.s_off = D.s_off.p; A.x_off = D.x_off.p; A.r_off = D.r_off.p; A.k_off = D.k_off.p;
    A.col_base = D.col_base.p;
    A.cols = D.cols.p;
    A.chunks = D.chunks.p;
    A.stat_idx = D.stat_idx.p;
    A.W = D.W.p; A.D = D.D.p; A.R = D.R.p; A.K = D.K.p;
    A.s = D.s.p; A.X = D.X.p; A.b2 = D.b2.p; A.r2 = D.r2.p;
    A.active = D.active.p; A.passes = D.passes.p;
    A.snaps = M.snaps.p;
    A.stats = M.item_stats.p;
    A.tol = cfg.tol;
    return A;
}

// phases of the optional timing
enum { kPhFactor = 0, kPhInit = 1, kPhResidual = 2, kPhSolve = 3, kPhFinish = 4, kPhases = 5 };

// start (begin = true) or stop an event pair of phase ph
msp_status mark(Medium::Direct& D, int ph, bool begin, cudaStream_t s) {
    if (!D.timing) return MSP_OK;
    if (begin) {
        while ((int)D.ev.size() < D.ev_used + 2) {
            cudaEvent_t e;
            MSP_CUDA(cudaEventCreate(&e));
            D.ev.push_back(e);
            D.ev_phase.push_back(0);
        }
        D.ev_phase[D.ev_used] = ph;
        MSP_CUDA(cudaEventRecord(D.ev[D.ev_used], s));
    } else {
        MSP_CUDA(cudaEventRecord(D.ev[D.ev_used + 1], s));
        D.ev_used += 2;
    }
    return MSP_OK;
}

template <int G>
msp_status launch_solve_g(const DirArgs& A, int grid, int smem, cudaStream_t s) {
    MSP_CUDA(cudaFuncSetAttribute(direct_solve_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    direct_solve_kernel<G><<<grid, kDirThreads, smem, s>>>(A);
    count_launches(1);
    return MSP_OK;
}

}  // namespace

bool direct_fits(const Medium& M) {
    for (const PatchDev& P : M.patches) {
        const Geo g = geo(P);
        if (g.ld > kDirMaxLd) return false;
    }
    return !M.patches.empty();
}

template <int TS>
static msp_status launch_factor(const DirArgs& A, int np, int smem, cudaStream_t s) {
    MSP_CUDA(cudaFuncSetAttribute(direct_factor_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    direct_factor_kernel<TS><<<np, kDirThreads, smem, s>>>(A);
    return MSP_OK;
}

msp_status launch_local_solves_direct(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s) {
    if (!direct_fits(M)) {
        set_error("direct local solver: a buffered patch is wider than 160 interior nodes");
        return MSP_ERR_INVALID_ARG;
    }
    MSP_TRY(direct_plan(M, s));
    Medium::Direct& D = M.dir;
    DirArgs A = direct_args(M, cfg);
    const int np = (int)M.patches.size();
    D.ev_used = 0;
    if (!D.factored) {
        MSP_TRY(mark(D, kPhFactor, true, s));
        // one sub-block size for the launch, from the widest padded row
        switch (std::max(1, (D.max_nxp + 15) / 16)) {
            case 1: MSP_TRY(launch_factor<1>(A, np, D.factor_smem_max, s)); break;
            case 2: MSP_TRY(launch_factor<2>(A, np, D.factor_smem_max, s)); break;
            case 3: MSP_TRY(launch_factor<3>(A, np, D.factor_smem_max, s)); break;
            case 4: MSP_TRY(launch_factor<4>(A, np, D.factor_smem_max, s)); break;
            case 5: MSP_TRY(launch_factor<5>(A, np, D.factor_smem_max, s)); break;
            case 6: MSP_TRY(launch_factor<6>(A, np, D.factor_smem_max, s)); break;
            case 7: MSP_TRY(launch_factor<7>(A, np, D.factor_smem_max, s)); break;
            case 8: MSP_TRY(launch_factor<8>(A, np, D.factor_smem_max, s)); break;
            case 9: MSP_TRY(launch_factor<9>(A, np, D.factor_smem_max, s)); break;
            default: MSP_TRY(launch_factor<10>(A, np, D.factor_smem_max, s)); break;
        }
        count_launches(1);
        MSP_TRY(mark(D, kPhFactor, false, s));
        MSP_CUDA(cudaGetLastError());
        D.factored = true;
    }
    MSP_TRY(mark(D, kPhInit, true, s));
    direct_init_kernel<<<D.n_cols, kDirThreads, 0, s>>>(A);
    count_launches(1);
    MSP_TRY(mark(D, kPhInit, false, s));
    MSP_TRY(mark(D, kPhResidual, true, s));
    direct_residual_kernel<<<D.n_chunks, kDirThreads, 0, s>>>(A, 1);
    count_launches(1);
    MSP_TRY(mark(D, kPhResidual, false, s));
    MSP_CUDA(cudaGetLastError());
    const int G = std::max(1, (D.max_nxp + 31) / 32);
    const int passes = std::max(1, std::min(cfg.max_ref, kDirMaxPasses));
    for (int p = 0; p < passes; ++p) {
        MSP_TRY(mark(D, kPhSolve, true, s));
        switch (G) {
            case 1: MSP_TRY(launch_solve_g<1>(A, D.n_chunks, D.chunk_smem_max, s)); break;
            case 2: MSP_TRY(launch_solve_g<2>(A, D.n_chunks, D.chunk_smem_max, s)); break;
            case 3: MSP_TRY(launch_solve_g<3>(A, D.n_chunks, D.chunk_smem_max, s)); break;
            case 4: MSP_TRY(launch_solve_g<4>(A, D.n_chunks, D.chunk_smem_max, s)); break;
            default: MSP_TRY(launch_solve_g<5>(A, D.n_chunks, D.chunk_smem_max, s)); break;
        }
        MSP_TRY(mark(D, kPhSolve, false, s));
        MSP_TRY(mark(D, kPhResidual, true, s));
        direct_residual_kernel<<<D.n_chunks, kDirThreads, 0, s>>>(A, 0);
        count_launches(1);
        MSP_TRY(mark(D, kPhResidual, false, s));
        MSP_CUDA(cudaGetLastError());
    }
    MSP_TRY(mark(D, kPhFinish, true, s));
    direct_finish_kernel<<<D.n_cols, kDirThreads, 0, s>>>(A);
    count_launches(1);
    MSP_TRY(mark(D, kPhFinish, false, s));
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" msp_status msp_medium_set_timing(msp_medium m, int enable) {
    clear_error();
    MSP_CHECK_ARG(m, "msp_medium_set_timing: NULL medium");
    m->M.dir.timing = enable != 0;
    m->M.dir.ev_used = 0;
    return MSP_OK;
}

extern "C" msp_status msp_medium_direct_timing(msp_medium m, double* ms_host, int* launches_host) {
    clear_error();
    MSP_CHECK_ARG(m && ms_host, "msp_medium_direct_timing: NULL argument");
    Medium::Direct& D = m->M.dir;
    for (int p = 0; p < kPhases; ++p) {
        ms_host[p] = 0.0;
        if (launches_host) launches_host[p] = 0;
    }
    for (int i = 0; i + 1 < D.ev_used; i += 2) {
        MSP_CUDA(cudaEventSynchronize(D.ev[i + 1]));
        float t = 0.f;
        MSP_CUDA(cudaEventElapsedTime(&t, D.ev[i], D.ev[i + 1]));
        ms_host[D.ev_phase[i]] += t;
        if (launches_host) launches_host[D.ev_phase[i]] += 1;
    }
    return MSP_OK;
}

namespace msp {

}  // namespace msp
