// The constrained least-squares variant of the online step (the remark after
// Eq. elliptic_cond_reduced): the boundary rows u_m(x) = phi(x), x on the domain
// boundary, hold exactly and only the continuity rows are solved in the least-
// squares sense.
//
// The boundary rows of patch m involve c_m alone (B = blockdiag(B_m), B_m the
// values of Q_m at the domain-boundary nodes of K_m), so the constraint is
// eliminated patch by patch by the null-space method: a Householder QR with
// column pivoting B_m^T P = Q R (k_m x nb_m, rank nb_m required) gives
//     c_m = c_p,m + N_m z_m,  c_p,m = Q_1 R_1^{-T} P^T phi_m = Z_m phi_m,  N_m = Q_2,
// with c_p,m the minimum-norm solution of B_m c_m = phi_m and N_m an orthonormal
// basis of null(B_m).  The reduced unknowns z solve the unconstrained problem
// min |P' z + P_cont c_p| whose bases are Q_m N_m on the boundary patches (Q_m
// elsewhere) and whose rows are the continuity rows only: the same online
// machinery (edge operators, block-row factor, preconditioned CGLS) on a derived
// basis, built once per basis on first use.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>
#include <memory>

namespace msp {

int domain_ring_pos(int N, int i, int j);

namespace {

constexpr int kConsMax = 1024;   // k_m and nb_m bound (shared-memory tables)

struct ConsArgs {
    const int* blist;            // boundary patches
    const int* k;                // k_m of the basis
    const int* nb;               // boundary nodes per patch
    const long long* bslot_off;  // per patch: first entry in bslot
    const int* bslot;            // ring slots t of the boundary nodes
    const long long* e_off;      // E_m offsets of the basis
    const double* E;
    const long long *a_off, *q_off, *x_off, *z_off, *n_off;   // per boundary patch
    double *A, *Q, *X, *Z, *Nm;
    int* status;
};

// One CTA (512 threads) per boundary patch, all in global memory (the blocks
// are small and touched a few times): gather B_m^T, pivoted Householder QR,
// Q formed explicitly, X = R_1^{-T}, Z_m = Q_1 X P^T, N_m = Q_2.
// status[p]: 0 on success, 1 if |R_jj| <= 1e-12 |R_00| for some j (B_m's rows are
// not independent to working accuracy).
__global__ void __launch_bounds__(512) cons_qr_kernel(ConsArgs C) {
    __shared__ double s_nrm[kConsMax];
    __shared__ double s_tau[kConsMax];
    __shared__ int s_perm[kConsMax];
    __shared__ int s_piv;
    __shared__ int s_bad;
    const int p = blockIdx.x, m = C.blist[p];
    const int k = C.k[m], nb = C.nb[m], kr = k - nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* a = C.A + C.a_off[p];   // k x nb
    double* q = C.Q + C.q_off[p];   // k x k
    double* x = C.X + C.x_off[p];   // nb x nb
    const double* Em = C.E + C.e_off[m];
    const int* sl = C.bslot + C.bslot_off[m];
    for (long long e = threadIdx.x; e < (long long)k * nb; e += blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        a[e] = Em[(long long)(2 * sl[j]) * k + i];   // value row of ring slot t_j
    }
    for (int j = threadIdx.x; j < nb; j += blockDim.x) s_perm[j] = j;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    double r00 = 0.0;
    for (int j = 0; j < nb; ++j) {
        for (int col = j + warp; col < nb; col += nw) {
            const double* ac = a + (long long)col * k;
            double t = 0.0;
            for (int i = j + lane; i < k; i += 32) t = fma(ac[i], ac[i], t);
            t = warp_sum(t);
            if (lane == 0) s_nrm[col] = t;
        }
        __syncthreads();
        if (warp == 0) {
            double best = -1.0;
            int bi = j;
            for (int col = j + lane; col < nb; col += 32)
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
        const int pv = s_piv;
        if (pv != j) {
            for (int i = threadIdx.x; i < k; i += blockDim.x) {
                const double t = a[i + (long long)j * k];
                a[i + (long long)j * k] = a[i + (long long)pv * k];
                a[i + (long long)pv * k] = t;
            }
            if (threadIdx.x == 0) {
                const int t = s_perm[j];
                s_perm[j] = s_perm[pv];
                s_perm[pv] = t;
            }
        }
        __syncthreads();
        double* aj = a + (long long)j * k;
        if (warp == 0) {
            double t = 0.0;
            for (int i = j + 1 + lane; i < k; i += 32) t = fma(aj[i], aj[i], t);
            t = warp_sum(t);
            if (lane == 0) s_nrm[j] = t;
        }
        __syncthreads();
        const double alpha = aj[j], xn2 = s_nrm[j];
        double tau = 0.0, scal = 0.0, beta = alpha;
        if (xn2 > 0.0) {
            beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
            tau = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
        }
        if (j == 0) r00 = fabs(beta);
        if (threadIdx.x == 0 && !(fabs(beta) > 1e-12 * r00)) s_bad = 1;
        __syncthreads();
        if (tau != 0.0)
            for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) aj[i] *= scal;
        if (threadIdx.x == 0) {
            aj[j] = beta;
            s_tau[j] = tau;
        }
        __syncthreads();
        if (tau != 0.0) {
            for (int col = j + 1 + warp; col < nb; col += nw) {
                double* ac = a + (long long)col * k;
                double t = (lane == 0) ? ac[j] : 0.0;
                for (int i = j + 1 + lane; i < k; i += 32) t = fma(aj[i], ac[i], t);
                t = warp_sum(t) * tau;
                if (lane == 0) ac[j] -= t;
                for (int i = j + 1 + lane; i < k; i += 32) ac[i] = fma(-t, aj[i], ac[i]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) C.status[p] = s_bad;
    if (s_bad) return;   // uniform: read after the last barrier of the loop
    // Q = H_0 ... H_{nb-1} (k x k), from the identity backwards
    for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
        const int i = (int)(e % k), j = (int)(e / k);
        q[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = nb - 1; j >= 0; --j) {
        const double tau = s_tau[j];
        if (tau != 0.0) {
            const double* aj = a + (long long)j * k;
            for (int col = j + warp; col < k; col += nw) {
                double* qc = q + (long long)col * k;
                double t = (lane == 0) ? qc[j] : 0.0;
                for (int i = j + 1 + lane; i < k; i += 32) t = fma(aj[i], qc[i], t);
                t = warp_sum(t) * tau;
                if (lane == 0) qc[j] -= t;
                for (int i = j + 1 + lane; i < k; i += 32) qc[i] = fma(-t, aj[i], qc[i]);
            }
        }
        __syncthreads();
    }
    // X = R_1^{-T} (lower triangular): column e by forward substitution on R_1^T,
    // R_1(q, l) = a[q + l k] for q <= l
    for (int e = threadIdx.x; e < nb; e += blockDim.x) {
        for (int l = 0; l < nb; ++l) {
            double acc = (l == e) ? 1.0 : 0.0;
            for (int qq = e; qq < l; ++qq) acc -= a[qq + (long long)l * k] * x[qq + (long long)e * nb];
            x[l + (long long)e * nb] = (l < e) ? 0.0 : acc / a[l + (long long)l * k];
        }
    }
    __syncthreads();
    // Z[:, perm[e]] = sum_{l >= e} Q[:, l] X[l, e];  N = Q[:, nb:]
    double* z = C.Z + C.z_off[p];
    for (long long w = threadIdx.x; w < (long long)k * nb; w += blockDim.x) {
        const int i = (int)(w % k), e = (int)(w / k);
        double acc = 0.0;
        for (int l = e; l < nb; ++l) acc = fma(q[i + (long long)l * k], x[l + (long long)e * nb], acc);
        z[i + (long long)s_perm[e] * k] = acc;
    }
    double* nm = C.Nm + C.n_off[p];
    for (long long w = threadIdx.x; w < (long long)k * kr; w += blockDim.x) {
        const int i = (int)(w % k), j = (int)(w / k);
        nm[w] = q[i + (long long)(nb + j) * k];
    }
}

// cp[c_off[m] + i][b] = sum_j Z_m[i][j] phi[b][ring_j] on the boundary patches, 0
// elsewhere (one CTA per patch)
__global__ void cons_particular_kernel(const int* k, const int* c_off, const int* nb, const long long* zp_off,
                                       const long long* bring_off, const int* bring, const double* Z,
                                       const double* phi, int n4, int B, double* cp) {
    const int m = blockIdx.x, km = k[m], nbm = nb[m];
    double* out = cp + (long long)c_off[m] * B;
    if (nbm == 0) {
        for (int w = threadIdx.x; w < km * B; w += blockDim.x) out[w] = 0.0;
        return;
    }
    const double* z = Z + zp_off[m];
    const int* rg = bring + bring_off[m];
    for (int w = threadIdx.x; w < km * B; w += blockDim.x) {
        const int i = w / B, b = w - i * B;
        double acc = 0.0;
        for (int j = 0; j < nbm; ++j) acc = fma(z[i + (long long)j * km], phi[(long long)b * n4 + rg[j]], acc);
        out[w] = acc;
    }
}

// cf = cp + N z on the boundary patches, cf = z elsewhere
__global__ void cons_combine_kernel(const int* k, const int* c_off, const int* kr, const int* cr_off, const int* nb,
                                    const long long* np_off, const double* Nm, const double* cp, const double* z,
                                    int B, double* cf) {
    const int m = blockIdx.x, km = k[m], krm = kr[m];
    double* out = cf + (long long)c_off[m] * B;
    const double* zm = z + (long long)cr_off[m] * B;
    if (nb[m] == 0) {
        for (int w = threadIdx.x; w < km * B; w += blockDim.x) out[w] = zm[w];
        return;
    }
    const double* nm = Nm + np_off[m];
    const double* cpm = cp + (long long)c_off[m] * B;
    for (int w = threadIdx.x; w < km * B; w += blockDim.x) {
        const int i = w / B, b = w - i * B;
        double acc = cpm[w];
        for (int j = 0; j < krm; ++j) acc = fma(nm[i + (long long)j * km], zm[(long long)j * B + b], acc);
        out[w] = acc;
    }
}

}  // namespace

msp_status build_constrained(Basis& B, cudaStream_t s) {
    const int np = (int)B.patches.size(), N = B.N;
    auto C = std::make_shared<ConstrainedOnline>();
    C->nb.assign(np, 0);
    std::vector<long long> bslot_off(np, 0), bring_off(np, 0);
    std::vector<int> bslot, bring, blist;
    for (int m = 0; m < np; ++m) {
        const PatchDev& P = B.patches[m];
        bslot_off[m] = bring_off[m] = (long long)bslot.size();
        for (int t = 0; t < B.n_e[m]; ++t) {
            int i, j;
            ring_node(P.x0, P.x1, P.y0, P.y1, t, i, j);
            if (i == 0 || i == N || j == 0 || j == N) {
                bslot.push_back(t);
                bring.push_back(domain_ring_pos(N, i, j));
            }
        }
        C->nb[m] = (int)(bslot.size() - bslot_off[m]);
        if (C->nb[m] > 0) {
            if (C->nb[m] > B.k[m] || B.k[m] > kConsMax) {
                set_error("constrained online solve: patch " + std::to_string(m) + " keeps " + std::to_string(B.k[m]) +
                          " basis vectors for " + std::to_string(C->nb[m]) +
                          " boundary nodes, so its boundary data cannot be imposed exactly");
                return MSP_ERR_BREAKDOWN;
            }
            blist.push_back(m);
        }
    }
    const int nbp = (int)blist.size();
    std::vector<long long> a_off(nbp), q_off(nbp), x_off(nbp), z_off(nbp), n_off(nbp);
    std::vector<long long> zp_off(np, 0), np_off(np, 0);
    long long ao = 0, qo = 0, xo = 0, zo = 0, no = 0;
    for (int p = 0; p < nbp; ++p) {
        const int m = blist[p], k = B.k[m], nb = C->nb[m];
        a_off[p] = ao; ao += (long long)k * nb;
        q_off[p] = qo; qo += (long long)k * k;
        x_off[p] = xo; xo += (long long)nb * nb;
        z_off[p] = zp_off[m] = zo; zo += (long long)k * nb;
        n_off[p] = np_off[m] = no; no += (long long)k * (k - nb);
    }
    DevBuf<int> d_blist, d_bslot, d_status;
    DevBuf<long long> d_bslot_off, d_a_off, d_q_off, d_x_off, d_z_off, d_n_off;
    DevBuf<double> A, Qs, X;
    MSP_TRY(upload(d_blist, blist, s));
    MSP_TRY(upload(d_bslot, bslot, s));
    MSP_TRY(upload(d_bslot_off, bslot_off, s));
    MSP_TRY(upload(C->d_nb, C->nb, s));
    MSP_TRY(upload(C->d_bring, bring, s));
    MSP_TRY(upload(C->d_bring_off, bring_off, s));
    MSP_TRY(upload(C->d_zp_off, zp_off, s));
    MSP_TRY(upload(C->d_np_off, np_off, s));
    MSP_TRY(upload(d_a_off, a_off, s)); MSP_TRY(upload(d_q_off, q_off, s)); MSP_TRY(upload(d_x_off, x_off, s));
    MSP_TRY(upload(d_z_off, z_off, s)); MSP_TRY(upload(d_n_off, n_off, s));
    MSP_TRY(A.alloc(std::max<long long>(ao, 1), s));
    MSP_TRY(Qs.alloc(std::max<long long>(qo, 1), s));
    MSP_TRY(X.alloc(std::max<long long>(xo, 1), s));
    MSP_TRY(C->Z.alloc(std::max<long long>(zo, 1), s));
    MSP_TRY(C->Nm.alloc(std::max<long long>(no, 1), s));
    MSP_TRY(d_status.alloc(std::max(nbp, 1), s));
    if (nbp > 0) {
        ConsArgs ca{};
        ca.blist = d_blist.p; ca.k = B.d_k.p; ca.nb = C->d_nb.p; ca.bslot_off = d_bslot_off.p; ca.bslot = d_bslot.p;
        ca.e_off = B.d_e_off.p; ca.E = B.E.p;
        ca.a_off = d_a_off.p; ca.q_off = d_q_off.p; ca.x_off = d_x_off.p; ca.z_off = d_z_off.p; ca.n_off = d_n_off.p;
        ca.A = A.p; ca.Q = Qs.p; ca.X = X.p; ca.Z = C->Z.p; ca.Nm = C->Nm.p; ca.status = d_status.p;
        cons_qr_kernel<<<nbp, 512, 0, s>>>(ca);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        std::vector<int> st(nbp);
        MSP_CUDA(cudaMemcpyAsync(st.data(), d_status.p, sizeof(int) * nbp, cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        for (int p = 0; p < nbp; ++p)
            if (st[p]) {
                set_error("constrained online solve: the boundary rows of patch " + std::to_string(blist[p]) +
                          " are not independent to working accuracy");
                return MSP_ERR_BREAKDOWN;
            }
    }
    // the derived basis: Q_m N_m on the boundary patches, Q_m elsewhere; continuity
    // rows only
    C->red = std::make_unique<Basis>();
    Basis& R = *C->red;
    R.N = B.N; R.mx = B.mx; R.my = B.my; R.xb = B.xb; R.yb = B.yb; R.patches = B.patches; R.device = B.device;
    R.no_boundary_rows = true;
    R.k.resize(np);
    R.q_off.resize(np);
    long long rq = 0;
    for (int m = 0; m < np; ++m) {
        R.k[m] = B.k[m] - C->nb[m];
        R.q_off[m] = rq;
        rq += (long long)B.patches[m].n_k * R.k[m];
    }
    R.sigma = B.sigma;
    R.sigma_off = B.sigma_off;
    MSP_TRY(R.Q.alloc(std::max<long long>(rq, 1), s));
    std::vector<GemmDesc> gd;
    for (int m = 0; m < np; ++m) {
        const long long nk = B.patches[m].n_k;
        if (R.k[m] == 0) continue;
        if (C->nb[m] == 0) {
            MSP_CUDA(cudaMemcpyAsync(R.Q.p + R.q_off[m], B.Q.p + B.q_off[m], sizeof(double) * nk * B.k[m],
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            gd.push_back(GemmDesc{B.Q.p + B.q_off[m], C->Nm.p + np_off[m], R.Q.p + R.q_off[m], (int)nk, R.k[m], B.k[m],
                                  (int)nk, B.k[m], (int)nk, 1.0, 0.0});
        }
    }
    if (!gd.empty()) {
        DevBuf<GemmDesc> d_gd;
        MSP_TRY(upload(d_gd, gd, s));
        int mm = 0, nn = 0;
        for (auto& g : gd) { mm = std::max(mm, g.M); nn = std::max(nn, g.N); }
        gemm_batched(d_gd.p, (int)gd.size(), mm, nn, false, s);
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaStreamSynchronize(s));
    }
    MSP_TRY(finish_basis(R, B.aE.p, B.aN.p, s));
    {
        std::vector<int> kr(np), cr(np);
        for (int m = 0; m < np; ++m) { kr[m] = R.k[m]; cr[m] = R.c_off[m]; }
        MSP_TRY(upload(C->d_kr, kr, s));
        MSP_TRY(upload(C->d_cr_off, cr, s));
    }
    MSP_CUDA(cudaStreamSynchronize(s));
    B.cons = C;
    return MSP_OK;
}

void cons_particular(const Basis& B, const ConstrainedOnline& C, const double* phi, int n4, int Bsz, double* cp,
                     cudaStream_t s) {
    const int np = (int)B.patches.size();
    cons_particular_kernel<<<np, 256, 0, s>>>(B.d_k.p, B.d_c_off.p, C.d_nb.p, C.d_zp_off.p, C.d_bring_off.p,
                                              C.d_bring.p, C.Z.p, phi, n4, Bsz, cp);
    count_launches(1);
}

void cons_combine(const Basis& B, const ConstrainedOnline& C, const double* cp, const double* z, int Bsz, double* cf,
                  cudaStream_t s) {
    const int np = (int)B.patches.size();
    cons_combine_kernel<<<np, 256, 0, s>>>(B.d_k.p, B.d_c_off.p, C.d_kr.p, C.d_cr_off.p, C.d_nb.p, C.d_np_off.p,
                                           C.Nm.p, cp, z, Bsz, cf);
    count_launches(1);
}

}  // namespace msp
