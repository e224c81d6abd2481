// Online stage (Sec. 5.2, Eq. elliptic_cond_reduced): c = argmin |P~ c - d|_2 by
// CGLS on the normal equations, preconditioned by the block-tridiagonal Cholesky
// factor of the scaled normal matrix over rows of patches (online_factor.cu) or, on
// request, by the patch blocks alone, M = blockdiag((P~^T P~)_mm); then the
// reconstruction u = sum_m chi_m Q_m c_m with chi_m = 1/#patches sharing the node.
//
// A batch of B right-hand sides runs side by side; vectors are stored
// element-major with the batch index fastest ([element][B]).  Every quantity of
// one data set is reduced in an order that does not depend on B, so a data set
// gets bit-identical results alone or inside any batch.
#include "internal.h"
#include "device_util.cuh"
#include "dense.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <cmath>

namespace msp {

namespace {

constexpr int kRowChunk = 128;
constexpr int kMaxBatch = 64;

// scalar block per data set b (w_scal[b * 8 + .]):
//   0 gamma, 1 alpha, 2 |P^T d|, 3 |s| last, 4 done flag, 5 iterations, 6 q.q
struct OnArgs {
    int np, B, n_rows, n_chunks;
    const int* c_off;
    const int* k;
    const int* slot_off;
    const int* ne;
    const long long* e_off;
    const long long* binv_off;
    const double* E;
    const double* Binv;
    const int* row_ptr;
    const int* row_slot;
    const int* row_bnd;
    const int* tr_ptr;
    const int* tr_ent;
};

// e[slot][b] = sum_j E_m[slot][j] x_m[j][b] for every slot of patch m (one CTA per patch)
__global__ void edge_apply_kernel(OnArgs A, const double* x, double* e) {
    const int m = blockIdx.x, k = A.k[m], ns = 2 * A.ne[m], B = A.B;
    const double* Em = A.E + A.e_off[m];
    const double* xm = x + (long long)A.c_off[m] * B;
    double* em = e + (long long)A.slot_off[m] * B;
    for (int w = threadIdx.x; w < ns * B; w += blockDim.x) {
        const int s = w / B, b = w - s * B;
        const double* er = Em + (long long)s * k;
        double a = 0.0;
        for (int j = 0; j < k; ++j) a += er[j] * xm[(long long)j * B + b];
        em[w] = a;
    }
}

__device__ __forceinline__ double row_value(const OnArgs& A, const double* e, int r, int b) {
    double a = 0.0;
    for (int t = A.row_ptr[r]; t < A.row_ptr[r + 1]; ++t) {
        const unsigned v = (unsigned)A.row_slot[t];
        const double x = e[(long long)(v & 0x7fffffffu) * A.B + b];
        a += (v & 0x80000000u) ? -x : x;
    }
    return a;
}

// q = P~ x (from the edge values e), per-chunk partial sums of q.q.  If init
// is set, r = d - q instead (d from the boundary data phi, less dsub[row][b] when
// dsub is given), and partials hold nothing.  Rows of a chunk are reduced warp by
// warp, then the four warp sums in order: the order does not depend on the batch
// size.
__global__ void __launch_bounds__(kRowChunk) rows_apply_kernel(OnArgs A, const double* e, double* q, double* part,
                                                               const double* phi, int n4, double* r, int init,
                                                               const double* dsub = nullptr) {
    __shared__ double sw[kRowChunk / 32][kMaxBatch];
    const int r0 = blockIdx.x * kRowChunk, B = A.B;
    const int row = r0 + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = 0; b < B; ++b) {
        double v = 0.0;
        if (row < A.n_rows) {
            v = row_value(A, e, row, b);
            if (init) {
                const int rb = A.row_bnd[row];
                double d = rb >= 0 ? phi[(long long)b * n4 + rb] : 0.0;
                if (dsub) d -= dsub[(long long)row * B + b];
                r[(long long)row * B + b] = d - v;
                v = 0.0;
            } else {
                q[(long long)row * B + b] = v;
            }
        }
        const double w = warp_sum(v * v);
        if (lane == 0) sw[warp][b] = w;
    }
    __syncthreads();
    if (!init && threadIdx.x < B) {
        double a = 0.0;
        for (int t = 0; t < kRowChunk / 32; ++t) a += sw[t][threadIdx.x];
        part[(long long)blockIdx.x * B + threadIdx.x] = a;
    }
}

// fixed-order sum over chunks for every data set: one warp per data set
__global__ void finalize_alpha_kernel(OnArgs A, const double* part, double* scal) {
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x >> 5; b < A.B; b += blockDim.x >> 5) {
    double a = 0.0;
    for (int c = lane; c < A.n_chunks; c += 32) a += part[(long long)c * A.B + b];
    a = warp_sum(a);
    if (lane == 0) {
        double* sc = scal + 8 * b;
        sc[6] = a;
        sc[1] = (sc[4] != 0.0 || a == 0.0) ? 0.0 : sc[0] / a;
    }
    }
}

// c += alpha p, r -= alpha q
__global__ void update_cr_kernel(OnArgs A, double* c, const double* p, double* r, const double* q, const double* scal,
                                 long long nc, long long nr) {
    const int B = A.B;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc + nr; t += (long long)gridDim.x * blockDim.x) {
        if (t < nc) {
            const int b = (int)(t % B);
            c[t] += scal[8 * b + 1] * p[t];
        } else {
            const long long u = t - nc;
            const int b = (int)(u % B);
            r[u] -= scal[8 * b + 1] * q[u];
        }
    }
}

// s = P~^T r (per patch: gather the rows of every edge slot, then E_m^T), z = Binv_m s,
// partial sums (s.z, s.s) per patch.
__global__ void normal_precond_kernel(OnArgs A, const double* r, double* z, double* part) {
    extern __shared__ double sm[];
    const int m = blockIdx.x, k = A.k[m], ns = 2 * A.ne[m], B = A.B;
    double* t = sm;                       // [ns][B]
    double* sv = sm + (long long)ns * B;  // [k][B]
    const int g0 = A.slot_off[m];
    for (int w = threadIdx.x; w < ns * B; w += blockDim.x) {
        const int s = w / B, b = w - s * B;
        double a = 0.0;
        for (int u = A.tr_ptr[g0 + s]; u < A.tr_ptr[g0 + s + 1]; ++u) {
            const unsigned v = (unsigned)A.tr_ent[u];
            const double x = r[(long long)(v & 0x7fffffffu) * B + b];
            a += (v & 0x80000000u) ? -x : x;
        }
        t[w] = a;
    }
    __syncthreads();
    const double* Em = A.E + A.e_off[m];
    for (int w = threadIdx.x; w < k * B; w += blockDim.x) {
        const int j = w / B, b = w - j * B;
        double a = 0.0;
        for (int s = 0; s < ns; ++s) a += Em[(long long)s * k + j] * t[s * B + b];
        sv[w] = a;
    }
    __syncthreads();
    const double* Bi = A.Binv + A.binv_off[m];
    double* zm = z + (long long)A.c_off[m] * B;
    for (int w = threadIdx.x; w < k * B; w += blockDim.x) {
        const int i = w / B, b = w - i * B;
        double a = 0.0;
        for (int j = 0; j < k; ++j) a += Bi[i + (long long)j * k] * sv[j * B + b];
        zm[w] = a;
    }
    __syncthreads();
    // partials: thread b sums over j in order
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        double sz = 0.0, ss = 0.0;
        for (int j = 0; j < k; ++j) {
            sz += sv[j * B + b] * zm[(long long)j * B + b];
            ss += sv[j * B + b] * sv[j * B + b];
        }
        part[((long long)m * B + b) * 2 + 0] = sz;
        part[((long long)m * B + b) * 2 + 1] = ss;
    }
}

// s = P~^T r per patch (gather the rows of every edge slot, then E_m^T); [element][B]
__global__ void normal_rhs_kernel(OnArgs A, const double* r, double* sout) {
    extern __shared__ double sm[];
    const int m = blockIdx.x, k = A.k[m], ns = 2 * A.ne[m], B = A.B;
    double* t = sm;   // [ns][B]
    const int g0 = A.slot_off[m];
    for (int w = threadIdx.x; w < ns * B; w += blockDim.x) {
        const int s = w / B, b = w - s * B;
        double a = 0.0;
        for (int u = A.tr_ptr[g0 + s]; u < A.tr_ptr[g0 + s + 1]; ++u) {
            const unsigned v = (unsigned)A.tr_ent[u];
            const double x = r[(long long)(v & 0x7fffffffu) * B + b];
            a += (v & 0x80000000u) ? -x : x;
        }
        t[w] = a;
    }
    __syncthreads();
    const double* Em = A.E + A.e_off[m];
    double* so = sout + (long long)A.c_off[m] * B;
    for (int w = threadIdx.x; w < k * B; w += blockDim.x) {
        const int j = w / B, b = w - j * B;
        double a = 0.0;
        for (int s = 0; s < ns; ++s) a += Em[(long long)s * k + j] * t[s * B + b];
        so[w] = a;
    }
}

// per-patch partial sums (s.z, s.s), fixed order over the patch's unknowns
__global__ void dots_kernel(OnArgs A, const double* sv, const double* z, double* part) {
    const int m = blockIdx.x, k = A.k[m], B = A.B;
    const double* sm_ = sv + (long long)A.c_off[m] * B;
    const double* zm = z + (long long)A.c_off[m] * B;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        double sz = 0.0, ss = 0.0;
        for (int j = 0; j < k; ++j) {
            sz += sm_[(long long)j * B + b] * zm[(long long)j * B + b];
            ss += sm_[(long long)j * B + b] * sm_[(long long)j * B + b];
        }
        part[((long long)m * B + b) * 2 + 0] = sz;
        part[((long long)m * B + b) * 2 + 1] = ss;
    }
}

// gamma' = sum_m s.z, |s| = sqrt(sum_m s.s); convergence; beta.  mode 0: first
// call (sets gamma and |P^T d|), mode 1: iteration.  beta goes to scal[7].
__global__ void finalize_beta_kernel(OnArgs A, const double* part, double* scal, double tol, int max_iter, int mode) {
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x >> 5; b < A.B; b += blockDim.x >> 5) {
    double sz = 0.0, ss = 0.0;
    for (int m = lane; m < A.np; m += 32) {
        sz += part[((long long)m * A.B + b) * 2 + 0];
        ss += part[((long long)m * A.B + b) * 2 + 1];
    }
    sz = warp_sum(sz);
    ss = warp_sum(ss);
    if (lane == 0) {
        double* sc = scal + 8 * b;
        const double ns = sqrt(ss);
        // sc[4]: 0 iterating, 1 converged, 2 stopped at max_iter, 3 non-finite residual
        if (mode == 0) {
            sc[0] = sz;
            sc[2] = ns;
            sc[3] = ns;
            sc[4] = (ns == 0.0) ? 1.0 : (isfinite(ns) && isfinite(sz)) ? 0.0 : 3.0;
            sc[5] = 0.0;
            sc[7] = 0.0;
        } else if (sc[4] != 0.0) {
            sc[7] = 0.0;
        } else {
            sc[5] += 1.0;
            sc[3] = ns;
            if (!isfinite(ns) || !isfinite(sz)) {
                sc[4] = 3.0;
                sc[7] = 0.0;
            } else if (ns <= tol * sc[2] || sc[5] >= max_iter) {
                sc[4] = (ns <= tol * sc[2]) ? 1.0 : 2.0;
                sc[7] = 0.0;
            } else {
                sc[7] = sz / sc[0];
                sc[0] = sz;
            }
        }
    }
    }
}

// p = z + beta p (mode 1) or p = z (mode 0); frozen for finished data sets
__global__ void update_p_kernel(OnArgs A, double* p, const double* z, const double* scal, long long nc, int mode) {
    const int B = A.B;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        if (mode == 0) p[t] = z[t];
        else if (scal[8 * b + 4] == 0.0) p[t] = z[t] + scal[8 * b + 7] * p[t];
    }
}

// interior nodes of every K_m: u = Q_m c_m (one CTA per patch); Q in FP64, or in
// FP32 for the map-based serving path (FP32 products, FP32 accumulation)
template <class TQ, class TC>
__global__ void recon_interior_kernel(OnArgs A, const PatchDev* patches, const long long* q_off, const TQ* Q,
                                      const TC* c, double* u, int N) {
    const int m = blockIdx.x, B = A.B, k = A.k[m];
    const PatchDev P = patches[m];
    const int wi = P.x1 - P.x0 - 1, hi = P.y1 - P.y0 - 1;
    if (wi <= 0 || hi <= 0) return;
    const int wk = P.x1 - P.x0 + 1;
    const TQ* q = Q + q_off[m];
    const TC* cm = c + (long long)A.c_off[m] * B;
    const long long nn = (long long)(N + 1) * (N + 1);
    for (long long w = threadIdx.x; w < (long long)wi * hi * B; w += blockDim.x) {
        const int b = (int)(w % B);
        const long long node = w / B;
        const int ii = (int)(node % wi) + 1, jj = (int)(node / wi) + 1;
        const int loc = ii + jj * wk;
        // products and partial sums of 16 terms in TQ, the partial sums added in FP64
        double a = 0.0;
        for (int j0 = 0; j0 < k; j0 += 16) {
            TQ part = TQ(0);
            const int j1 = min(k, j0 + 16);
            for (int j = j0; j < j1; ++j) part += q[loc + (long long)j * P.n_k] * (TQ)cm[(long long)j * B + b];
            a += (double)part;
        }
        u[(long long)b * nn + (long long)(P.y0 + jj) * (N + 1) + (P.x0 + ii)] = a;
    }
}

// skeleton nodes: average of the sharing patches' values (fixed patch order);
// domain-boundary nodes take phi
__global__ void recon_skeleton_kernel(OnArgs A, int n_skel, const int* sk_ptr, const int* sk_slot,
                                      const int* sk_node, const int* sk_ring, const double* e, const double* phi,
                                      int n4, double* u, int N) {
    const int B = A.B;
    const long long nn = (long long)(N + 1) * (N + 1);
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < (long long)n_skel * B;
         w += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(w % B), x = (int)(w / B);
        double v;
        if (sk_ring[x] >= 0) {
            v = phi[(long long)b * n4 + sk_ring[x]];
        } else {
            double a = 0.0;
            const int n = sk_ptr[x + 1] - sk_ptr[x];
            for (int t = sk_ptr[x]; t < sk_ptr[x + 1]; ++t) a += e[(long long)sk_slot[t] * B + b];
            v = a / n;
        }
        u[(long long)b * nn + sk_node[x]] = v;
    }
}

__global__ void export_c_kernel(const double* c, double* out, int Np, int B) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)Np * B; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % B);
        const long long j = t / B;
        out[(long long)b * Np + j] = c[t];
    }
}


// columns j0 .. j0+B-1 of the identity on the boundary ring: phi[b][i] = (i == j0 + b)
__global__ void unit_ring_kernel(double* phi, int n4, int j0, int B) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n4 * B;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / n4), i = (int)(t % n4);
        phi[t] = (i == j0 + b) ? 1.0 : 0.0;
    }
}

__global__ void to_f32_kernel(const double* src, float* dst, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}


// c[j][b] = sum_k G[j][k] phi32[b][k] (G: Np x n4 column-major; phi32: [b][n4];
// c element-major, as the reconstruction reads it).  64 x 64 output tiles (64
// unknowns x up to 64 data sets; columns past the batch are skipped per 16-wide
// group), 16-deep K slices staged in shared memory; products and sums of 128
// consecutive terms in FP32, those partial sums accumulated in FP64 (at a
// sixty-fourth of the FP32 work, so the FP64 pipe keeps pace), so the rounding of
// the long K sum does not grow with the ring length; the total is rounded to FP32.
__global__ void __launch_bounds__(256) map_gemm_kernel(const float* G, const float* phi32, float* c, int Np, int n4,
                                                       int B) {
    constexpr int TM = 64, TN = 64, TK = 16, KF = 8;   // KF slices per FP64 accumulation
    __shared__ float Gs[TK][TM + 1];
    __shared__ float Ps[TK][TN + 1];
    const int tiles_m = (Np + TM - 1) / TM;
    const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
    const int m0 = tm * TM, n0 = tn * TN;
    if (n0 >= B) return;
    const int jmax = min(4, (B - n0 + 15) / 16);   // 16-wide column groups holding data sets (uniform per CTA)
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    float part[4][4] = {};
    int slice = 0;
    for (int k0 = 0; k0 < n4; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int mm = e % TM, kk = e / TM;
            const int gm = m0 + mm, gk = k0 + kk;
            Gs[kk][mm] = (gm < Np && gk < n4) ? G[(long long)gk * Np + gm] : 0.f;
        }
        for (int e = threadIdx.x; e < jmax * 16 * TK; e += 256) {
            const int kk = e % TK, nn = e / TK;
            const int gk = k0 + kk, gn = n0 + nn;
            Ps[kk][nn] = (gk < n4 && gn < B) ? phi32[(long long)gn * n4 + gk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Gs[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = (j < jmax) ? Ps[kk][ty + 16 * j] : 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < jmax) part[i][j] = fmaf(a[i], b[j], part[i][j]);
        }
        if (++slice == KF || k0 + TK >= n4) {
            slice = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j < jmax) acc[i][j] += (double)part[i][j];
                    part[i][j] = 0.f;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
            if (j < jmax && gm < Np && gn < B) c[(long long)gm * B + gn] = (float)acc[i][j];
        }
}
// Value slots of the edge operators for the map path: e[slot][b] for the even
// (value) slots of every patch, from FP32 operators and coefficients, partial
// sums of 16 terms in FP32 added in FP64.  Only the skeleton averages read them.
__global__ void edge_values_map_kernel(OnArgs A, const float* E32, const float* c32, double* e) {
    const int m = blockIdx.x, k = A.k[m], nt = A.ne[m], B = A.B;
    const float* Em = E32 + A.e_off[m];
    const float* xm = c32 + (long long)A.c_off[m] * B;
    double* em = e + (long long)A.slot_off[m] * B;
    for (int w = threadIdx.x; w < nt * B; w += blockDim.x) {
        const int t = w / B, b = w - t * B;
        const float* er = Em + (long long)(2 * t) * k;
        double a = 0.0;
        for (int j0 = 0; j0 < k; j0 += 16) {
            float part = 0.f;
            const int j1 = min(k, j0 + 16);
            for (int j = j0; j < j1; ++j) part = fmaf(er[j], xm[(long long)j * B + b], part);
            a += (double)part;
        }
        em[(long long)(2 * t) * B + b] = a;
    }
}

}  // namespace

static OnArgs make_args(const Basis& Bs, int B) {
    OnArgs A{};
    A.np = (int)Bs.patches.size();
    A.B = B;
    A.n_rows = Bs.n_rows;
    A.n_chunks = (Bs.n_rows + kRowChunk - 1) / kRowChunk;
    A.c_off = Bs.d_c_off.p; A.k = Bs.d_k.p; A.slot_off = Bs.d_slot_off.p; A.ne = Bs.d_ne.p;
    A.e_off = Bs.d_e_off.p; A.binv_off = Bs.d_binv_off.p; A.E = Bs.E.p; A.Binv = Bs.Binv.p;
    A.row_ptr = Bs.row_ptr.p; A.row_slot = Bs.row_slot.p; A.row_bnd = Bs.row_bnd.p;
    A.tr_ptr = Bs.tr_ptr.p; A.tr_ent = Bs.tr_ent.p;
    return A;
}

// reconstruction u = sum_m chi_m Q_m c_m (interior of the patches, then the
// skeleton from the edge values, phi on the domain boundary) for coefficients c
// in the [coefficient][B] layout; e is scratch of n_slots x B
static void reconstruct(const Basis& Bs, const OnArgs& A, const double* c, double* e, const double* phi, int n4,
                        double* u, cudaStream_t s) {
    const int np = (int)Bs.patches.size(), N = Bs.N, B = A.B;
    recon_interior_kernel<double, double><<<np, 256, 0, s>>>(A, Bs.d_patches.p, Bs.d_q_off.p, Bs.Q.p, c, u, N);
    count_launches(1);
    edge_apply_kernel<<<np, 256, 0, s>>>(A, c, e);
    count_launches(1);
    const int sk_grid = std::max(1, std::min<int>((int)(((long long)Bs.n_skel * B + 255) / 256), num_sms() * 8));
    recon_skeleton_kernel<<<sk_grid, 256, 0, s>>>(A, Bs.n_skel, Bs.sk_ptr.p, Bs.sk_slot.p, Bs.sk_node.p, Bs.sk_ring.p,
                                                  e, phi, n4, u, N);
    count_launches(1);
}

void reconstruct_coefficients(const Basis& Bs, const double* c, int B, double* e, const double* phi, int n4, double* u,
                              cudaStream_t s) {
    reconstruct(Bs, make_args(Bs, B), c, e, phi, n4, u, s);
}

// One batch of CGLS.  dsub (optional, [row][B]) is subtracted from the right-hand
// side d of the rows (the constrained variant's continuity rows carry -P c_p).
static msp_status online_batch(Basis& Bs, const double* phi, int B, double tol, int max_iter, double* u,
                               double* c_out, int* iters_host, cudaStream_t s, bool* not_conv,
                               bool* nonfinite = nullptr, const double* dsub = nullptr) {
    const int np = (int)Bs.patches.size();
    const int N = Bs.N, n4 = 4 * N;
    OnArgs A = make_args(Bs, B);
    if (Bs.cap_batch < B) {
        const int cb = kMaxBatch;
        MSP_TRY(Bs.w_c.alloc((size_t)std::max(Bs.Np, 1) * cb, s));
        MSP_TRY(Bs.w_p.alloc((size_t)std::max(Bs.Np, 1) * cb, s));
        MSP_TRY(Bs.w_z.alloc((size_t)std::max(Bs.Np, 1) * cb, s));
        MSP_TRY(Bs.w_e.alloc((size_t)std::max(Bs.n_slots, 1) * cb, s));
        MSP_TRY(Bs.w_q.alloc((size_t)std::max(Bs.n_rows, 1) * cb, s));
        MSP_TRY(Bs.w_r.alloc((size_t)std::max(Bs.n_rows, 1) * cb, s));
        MSP_TRY(Bs.w_part.alloc((size_t)std::max(A.n_chunks, 2 * np) * cb * 2, s));
        MSP_TRY(Bs.w_scal.alloc((size_t)8 * cb, s));
        Bs.cap_batch = cb;
    }
    const long long nc = (long long)Bs.Np * B, nr = (long long)Bs.n_rows * B;
    int max_ns = 0, max_k = 0;
    for (int m = 0; m < np; ++m) {
        max_ns = std::max(max_ns, 2 * Bs.n_e[m]);
        max_k = std::max(max_k, Bs.k[m]);
    }
    const size_t smem = sizeof(double) * ((size_t)max_ns * B + (size_t)max_k * B);
    if (smem > 48 * 1024) {
        MSP_CUDA(cudaFuncSetAttribute(normal_precond_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        MSP_CUDA(cudaFuncSetAttribute(normal_rhs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (Bs.w_s.n < (size_t)nc) MSP_TRY(Bs.w_s.alloc((size_t)std::max(Bs.Np, 1) * kMaxBatch, s));
    // z = M^{-1} P~^T r and the partial sums (s.z, s.s): block-row factor when built,
    // patch-block (additive Schwarz) inverses otherwise
    auto precondition = [&]() -> msp_status {
        if (Bs.bt_q > 0 && !Bs.use_block_jacobi) {
            normal_rhs_kernel<<<np, 256, smem, s>>>(A, Bs.w_r.p, Bs.w_s.p);
            count_launches(1);
            MSP_TRY(apply_online_factor(Bs, Bs.w_s.p, Bs.w_z.p, B, s));
            dots_kernel<<<np, 64, 0, s>>>(A, Bs.w_s.p, Bs.w_z.p, Bs.w_part.p);
            count_launches(1);
        } else {
            normal_precond_kernel<<<np, 256, smem, s>>>(A, Bs.w_r.p, Bs.w_z.p, Bs.w_part.p);
            count_launches(1);
        }
        return MSP_OK;
    };
    const int ew_grid = std::max(1, std::min<int>((int)((nc + nr + 255) / 256), num_sms() * 8));
    MSP_CUDA(cudaMemsetAsync(Bs.w_c.p, 0, sizeof(double) * nc, s));
    MSP_CUDA(cudaMemsetAsync(Bs.w_e.p, 0, sizeof(double) * (size_t)Bs.n_slots * B, s));
    // r = d
    rows_apply_kernel<<<A.n_chunks, kRowChunk, 0, s>>>(A, Bs.w_e.p, Bs.w_q.p, Bs.w_part.p, phi, n4, Bs.w_r.p, 1, dsub);
    count_launches(1);
    MSP_TRY(precondition());
    finalize_beta_kernel<<<1, 1024, 0, s>>>(A, Bs.w_part.p, Bs.w_scal.p, tol, max_iter, 0);
    count_launches(1);
    update_p_kernel<<<ew_grid, 256, 0, s>>>(A, Bs.w_p.p, Bs.w_z.p, Bs.w_scal.p, nc, 0);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    std::vector<double> scal(8 * (size_t)B);
    const int check_every = (Bs.bt_q > 0 && !Bs.use_block_jacobi) ? 2 : 16;
    for (int it = 0; it < max_iter; ++it) {
        edge_apply_kernel<<<np, 256, 0, s>>>(A, Bs.w_p.p, Bs.w_e.p);
        count_launches(1);
        rows_apply_kernel<<<A.n_chunks, kRowChunk, 0, s>>>(A, Bs.w_e.p, Bs.w_q.p, Bs.w_part.p, phi, n4, Bs.w_r.p, 0);
        count_launches(1);
        finalize_alpha_kernel<<<1, 1024, 0, s>>>(A, Bs.w_part.p, Bs.w_scal.p);
        count_launches(1);
        update_cr_kernel<<<ew_grid, 256, 0, s>>>(A, Bs.w_c.p, Bs.w_p.p, Bs.w_r.p, Bs.w_q.p, Bs.w_scal.p, nc, nr);
        count_launches(1);
        MSP_TRY(precondition());
        finalize_beta_kernel<<<1, 1024, 0, s>>>(A, Bs.w_part.p, Bs.w_scal.p, tol, max_iter, 1);
        count_launches(1);
        update_p_kernel<<<ew_grid, 256, 0, s>>>(A, Bs.w_p.p, Bs.w_z.p, Bs.w_scal.p, nc, 1);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        if ((it + 1) % check_every == 0 || it + 1 == max_iter) {
            MSP_CUDA(cudaMemcpyAsync(scal.data(), Bs.w_scal.p, sizeof(double) * 8 * B, cudaMemcpyDeviceToHost, s));
            unsigned int bar[4] = {0, 0, 0, 0};
            if (Bs.d_bt_bar.p)   // the factor sweeps' grid barrier raises its error word on a timeout
                MSP_CUDA(cudaMemcpyAsync(bar, Bs.d_bt_bar.p, sizeof(bar), cudaMemcpyDeviceToHost, s));
            MSP_CUDA(cudaStreamSynchronize(s));
            if (bar[2] != 0) {
                MSP_CUDA(cudaMemsetAsync(Bs.d_bt_bar.p, 0, sizeof(bar), s));
                set_error("msp_online_solve: grid barrier of the factor sweeps timed out");
                return MSP_ERR_TIMEOUT;
            }
            bool all = true;
            for (int b = 0; b < B; ++b) all &= scal[8 * b + 4] != 0.0;
            if (all) break;
        }
    }
    // the last stop test read above holds every data set's final state
    for (int b = 0; b < B; ++b) {
        if (scal[8 * b + 4] != 1.0) *not_conv = true;
        if (scal[8 * b + 4] == 3.0 && nonfinite) *nonfinite = true;
    }
    // reconstruction (skipped when only the coefficients are asked for)
    const long long nn = (long long)(N + 1) * (N + 1);
    if (u) reconstruct(Bs, A, Bs.w_c.p, Bs.w_e.p, phi, n4, u, s);
    if (c_out) {
        export_c_kernel<<<ew_grid, 256, 0, s>>>(Bs.w_c.p, c_out, Bs.Np, B);
        count_launches(1);
    }
    MSP_CUDA(cudaGetLastError());
    (void)nn;
    if (iters_host) {
        MSP_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) iters_host[b] = (int)scal[8 * b + 5];
    }
    return MSP_OK;
}

int online_batch_cap(const Basis& Bs) {
    int max_ns = 0, max_k = 0;
    for (size_t m = 0; m < Bs.patches.size(); ++m) {
        max_ns = std::max(max_ns, 2 * Bs.n_e[m]);
        max_k = std::max(max_k, Bs.k[m]);
    }
    const long long per = (long long)(max_ns + max_k) * (long long)sizeof(double);
    const long long cap = (200LL * 1024) / std::max<long long>(per, 1);
    return (int)std::max<long long>(1, std::min<long long>(kMaxBatch, cap));
}

msp_status online_solve(Basis& Bs, const double* phi, int batch, double tol, int max_iter, double* u, double* c_out,
                        int* iters_host, cudaStream_t s) {
    const int N = Bs.N;
    const long long nn = (long long)(N + 1) * (N + 1);
    bool not_conv = false, nonfinite = false;
    const int cap = online_batch_cap(Bs);
    for (int b0 = 0; b0 < batch; b0 += cap) {
        const int B = std::min(cap, batch - b0);
        MSP_TRY(online_batch(Bs, phi + (long long)b0 * 4 * N, B, tol, max_iter, u ? u + (long long)b0 * nn : nullptr,
                             c_out ? c_out + (long long)b0 * Bs.Np : nullptr, iters_host ? iters_host + b0 : nullptr, s,
                             &not_conv, &nonfinite));
    }
    if (nonfinite) {
        set_error("msp_online_solve: a data set's residual is not finite (NaN or Inf in phi); it stopped at once");
        return MSP_ERR_NOT_CONVERGED;
    }
    if (not_conv) {
        set_error("msp_online_solve: some data sets stopped at max_iter");
        return MSP_ERR_NOT_CONVERGED;
    }
    return MSP_OK;
}

// The constrained least-squares variant (online_constrained.cu): per batch, the
// particular coefficients c_p = Z phi, their continuity residual q_p = P' (E c_p)
// on the derived basis's rows, CGLS on the derived basis for min |P' z + q_p|,
// then c = c_p + N z and the reconstruction with the original bases.
msp_status online_solve_constrained(Basis& Bs, const double* phi, int batch, double tol, int max_iter, double* u,
                                    double* c_out, int* iters_host, cudaStream_t s) {
    if (!Bs.cons) MSP_TRY(build_constrained(Bs, s));
    ConstrainedOnline& C = *Bs.cons;
    Basis& R = *C.red;
    const int np = (int)Bs.patches.size(), N = Bs.N, n4 = 4 * N;
    const long long nn = (long long)(N + 1) * (N + 1);
    if (C.cap < kMaxBatch) {
        const int cb = kMaxBatch;
        MSP_TRY(C.cp.alloc((size_t)std::max(Bs.Np, 1) * cb, s));
        MSP_TRY(C.cf.alloc((size_t)std::max(Bs.Np, 1) * cb, s));
        MSP_TRY(C.ep.alloc((size_t)std::max(Bs.n_slots, 1) * cb, s));
        MSP_TRY(C.dq.alloc((size_t)std::max(R.n_rows, 1) * cb, s));
        MSP_TRY(C.part.alloc((size_t)std::max((R.n_rows + kRowChunk - 1) / kRowChunk, 1) * cb, s));
        C.cap = cb;
    }
    const int cap = std::min(online_batch_cap(Bs), online_batch_cap(R));
    bool not_conv = false, nonfinite = false;
    for (int b0 = 0; b0 < batch; b0 += cap) {
        const int B = std::min(cap, batch - b0);
        const double* ph = phi + (long long)b0 * n4;
        const OnArgs AB = make_args(Bs, B), AR = make_args(R, B);
        cons_particular(Bs, C, ph, n4, B, C.cp.p, s);
        edge_apply_kernel<<<np, 256, 0, s>>>(AB, C.cp.p, C.ep.p);
        count_launches(1);
        rows_apply_kernel<<<AR.n_chunks, kRowChunk, 0, s>>>(AR, C.ep.p, C.dq.p, C.part.p, ph, n4, nullptr, 0);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        MSP_TRY(online_batch(R, ph, B, tol, max_iter, nullptr, nullptr, iters_host ? iters_host + b0 : nullptr, s,
                             &not_conv, &nonfinite, C.dq.p));
        cons_combine(Bs, C, C.cp.p, R.w_c.p, B, C.cf.p, s);
        if (u) reconstruct(Bs, AB, C.cf.p, C.ep.p, ph, n4, u + (long long)b0 * nn, s);
        if (c_out) {
            const int ew_grid = std::max(1, std::min<int>((int)(((long long)Bs.Np * B + 255) / 256), num_sms() * 8));
            export_c_kernel<<<ew_grid, 256, 0, s>>>(C.cf.p, c_out + (long long)b0 * Bs.Np, Bs.Np, B);
            count_launches(1);
        }
        MSP_CUDA(cudaGetLastError());
    }
    if (nonfinite) {
        set_error("msp_online_solve_constrained: a data set's residual is not finite (NaN or Inf in phi)");
        return MSP_ERR_NOT_CONVERGED;
    }
    if (not_conv) {
        set_error("msp_online_solve_constrained: some data sets stopped at max_iter");
        return MSP_ERR_NOT_CONVERGED;
    }
    return MSP_OK;
}

// Boundary-to-coefficient map.  The data of Eq. elliptic_cond_reduced enter only
// through the boundary rows and linearly, so c = G phi with G = P~^+ S (S puts the
// ring values into the boundary rows).  Column j of G is the online solution for
// the j-th unit vector of the ring; the columns are computed in batches by the
// FP64 iteration above, to tolerance tol, and stored in FP32 (N_p x 4N,
// column-major), with an FP32 copy of the bases for the reconstruction.
msp_status build_online_map(Basis& Bs, double tol, int max_iter, cudaStream_t s) {
    const int N = Bs.N, n4 = 4 * N, Np = Bs.Np;
    MSP_TRY(Bs.G32.alloc(std::max<long long>((long long)Np * n4, 1), s));
    const int cap = online_batch_cap(Bs);
    DevBuf<double> phi, c64;
    MSP_TRY(phi.alloc((size_t)n4 * cap, s));
    MSP_TRY(c64.alloc((size_t)std::max(Np, 1) * cap, s));
    std::vector<int> iters(cap);
    for (int j0 = 0; j0 < n4; j0 += cap) {
        const int B = std::min(cap, n4 - j0);
        unit_ring_kernel<<<std::max(1, std::min(1024, (n4 * B + 255) / 256)), 256, 0, s>>>(phi.p, n4, j0, B);
        count_launches(1);
        bool not_conv = false;
        MSP_TRY(online_batch(Bs, phi.p, B, tol, max_iter, nullptr, c64.p, iters.data(), s, &not_conv));
        if (not_conv) {
            set_error("msp_basis_build_map: a ring unit vector stopped at max_iter");
            return MSP_ERR_NOT_CONVERGED;
        }
        const long long n = (long long)Np * B;
        to_f32_kernel<<<std::max(1, (int)std::min<long long>(2048, (n + 255) / 256)), 256, 0, s>>>(
            c64.p, Bs.G32.p + (long long)j0 * Np, n);
        count_launches(1);
    }
    long long nq = 0;
    for (size_t m = 0; m < Bs.patches.size(); ++m) nq = std::max<long long>(nq, Bs.q_off[m] + (long long)Bs.patches[m].n_k * Bs.k[m]);
    // G tiled and split for the tensor-core GEMM (element (j, k) at j + k Np)
    MSP_TRY(Bs.Gt_hi.alloc((size_t)tc_a_floats(Np, n4), s));
    MSP_TRY(Bs.Gt_lo.alloc((size_t)tc_a_floats(Np, n4), s));
    tc_tile_split(Bs.G32.p, 1, Np, Np, n4, true, Bs.Gt_hi.p, Bs.Gt_lo.p, s);
    MSP_TRY(Bs.E32.alloc(std::max<size_t>(Bs.E.n, 1), s));
    to_f32_kernel<<<std::max(1, (int)std::min<long long>(4096, ((long long)Bs.E.n + 255) / 256)), 256, 0, s>>>(
        Bs.E.p, Bs.E32.p, (long long)Bs.E.n);
    count_launches(1);
    MSP_TRY(Bs.Q32.alloc(std::max<long long>(nq, 1), s));
    to_f32_kernel<<<std::max(1, (int)std::min<long long>(4096, (nq + 255) / 256)), 256, 0, s>>>(Bs.Q.p, Bs.Q32.p, nq);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    MSP_CUDA(cudaStreamSynchronize(s));
    Bs.map_built = true;
    return MSP_OK;
}

// u = reconstruction of c = G phi for a batch (map built).  The work buffers are
// the caller's (MapWork, sized for max_batch data sets) or the call's own; with
// its own MapWork per stream, calls on different streams run at the same time.
// Each data set's result does not depend on the others in the batch.
msp_status map_work_alloc(const Basis& Bs, int max_batch, MapWork& w) {
    const int n4 = 4 * Bs.N;
    const size_t B = (size_t)std::max(1, max_batch);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.phi32, sizeof(float) * n4 * B);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.c32, sizeof(float) * std::max(Bs.Np, 1) * B);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.e, sizeof(double) * std::max(Bs.n_slots, 1) * B);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.b_hi, sizeof(float) * tc_b_floats((int)B, n4));
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.b_lo, sizeof(float) * tc_b_floats((int)B, n4));
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w.err, 0, sizeof(int));
    w.cap = (int)B;
    if (e != cudaSuccess) {
        map_work_free(w);
        set_error(std::string("map work buffers: ") + cudaGetErrorString(e));
        return MSP_ERR_OOM;
    }
    return MSP_OK;
}

void map_work_free(MapWork& w) {
    if (w.phi32) cudaFree(w.phi32);
    if (w.c32) cudaFree(w.c32);
    if (w.e) cudaFree(w.e);
    if (w.b_hi) cudaFree(w.b_hi);
    if (w.b_lo) cudaFree(w.b_lo);
    if (w.err) cudaFree(w.err);
    w = MapWork{};
}

msp_status map_work_check(MapWork& w, cudaStream_t s) {
    if (!w.err) return MSP_OK;
    int h = 0;
    MSP_CUDA(cudaMemcpyAsync(&h, w.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    if (h) {
        MSP_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
        set_error("map solve: a wait of the tensor-core GEMM timed out");
        return MSP_ERR_TIMEOUT;
    }
    return MSP_OK;
}

msp_status online_solve_map(const Basis& Bs, const double* phi, int batch, double* u, cudaStream_t s, MapWork* work) {
    if (!Bs.map_built) {
        set_error("msp_online_solve_map: the boundary-to-coefficient map has not been built");
        return MSP_ERR_INVALID_ARG;
    }
    const int N = Bs.N, n4 = 4 * N, Np = Bs.Np, np = (int)Bs.patches.size();
    const long long nn = (long long)(N + 1) * (N + 1);
    MapWork own{};
    if (!work) {
        MSP_TRY(map_work_alloc(Bs, std::min(batch, kMaxBatch), own));
        work = &own;
    }
    msp_status st = MSP_OK;
    for (int b0 = 0; b0 < batch && st == MSP_OK; b0 += work->cap) {
        const int B = std::min(work->cap, batch - b0);
        const double* ph = phi + (long long)b0 * n4;
        to_f32_kernel<<<std::max(1, std::min(1024, (n4 * B + 255) / 256)), 256, 0, s>>>(ph, work->phi32, (long long)n4 * B);
        count_launches(1);
        if (Bs.map_engine == 0 && Bs.Gt_hi.p) {
            // tensor cores: phi split and tiled, then the tcgen05 GEMM
            tc_tile_split(work->phi32, n4, 1, B, n4, false, work->b_hi, work->b_lo, s);
            TcMapArgs ta{};
            ta.a_hi = Bs.Gt_hi.p;
            ta.a_lo = Bs.Gt_lo.p;
            ta.b_hi = work->b_hi;
            ta.b_lo = work->b_lo;
            ta.M = Np;
            ta.B = B;
            ta.n_slabs = tc_slabs(n4);
            ta.c = work->c32;
            ta.err = work->err;
            MSP_TRY(tc_map_gemm(ta, s));
        } else {
            const int tiles = ((Np + 63) / 64) * ((B + 63) / 64);
            map_gemm_kernel<<<tiles, 256, 0, s>>>(Bs.G32.p, work->phi32, work->c32, Np, n4, B);
            count_launches(1);
        }
        OnArgs A = make_args(Bs, B);
        double* ub = u + (long long)b0 * nn;
        recon_interior_kernel<float, float><<<np, 256, 0, s>>>(A, Bs.d_patches.p, Bs.d_q_off.p, Bs.Q32.p, work->c32, ub, N);
        count_launches(1);
        edge_values_map_kernel<<<np, 256, 0, s>>>(A, Bs.E32.p, work->c32, work->e);
        count_launches(1);
        const int sk_grid = std::max(1, std::min<int>((int)(((long long)Bs.n_skel * B + 255) / 256), num_sms() * 8));
        recon_skeleton_kernel<<<sk_grid, 256, 0, s>>>(A, Bs.n_skel, Bs.sk_ptr.p, Bs.sk_slot.p, Bs.sk_node.p,
                                                      Bs.sk_ring.p, work->e, ph, n4, ub, N);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error(std::string("msp_online_solve_map: ") + cudaGetErrorString(e));
            st = MSP_ERR_CUDA;
        }
    }
    if (work == &own) {
        if (st == MSP_OK) st = map_work_check(own, s);
        cudaStreamSynchronize(s);
        map_work_free(own);
    }
    return st;
}

}  // namespace msp
