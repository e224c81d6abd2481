// Preconditioner of the online least-squares iteration: a block-tridiagonal
// Cholesky factorisation of the normal matrix H = P~^T P~ (Eq.
// elliptic_cond_reduced), ordered by rows of patches.
//
// H couples a patch only with its eight neighbours, so with the unknowns of one
// row of patches as a block, H is block tridiagonal: diagonal blocks D_q and
// sub-diagonal blocks E_q = H_{q+1,q}.  The factor is computed in FP32 on the
// diagonally scaled matrix Hs = S H S (S = diag(H)^(-1/2)):
//     L_q L_q^T = D_q - C_{q-1} C_{q-1}^T,   C_q = E_q L_q^{-T}
// with explicit inverses Li_q = L_q^{-1}.  Applying M^{-1} = S (L L^T)^{-1} S is
// then a forward and a backward sweep of GEMMs.  The FP64 CGLS iteration around
// it keeps the least-squares solution at FP64 accuracy; on a non-positive pivot
// the factorisation is repeated with a diagonal shift.
#include "internal.h"
#include "dense.cuh"
#include "device_util.cuh"

#include <algorithm>
#include <map>
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
    const PairBlock b = pb[blockIdx.x];
    const int ka = k[b.ma], kb = k[b.mb];
    const double* Ea = E + e_off[b.ma];
    const double* Eb = E + e_off[b.mb];
    const int ga = slot_off[b.ma], gb = slot_off[b.mb];
    for (long long w = threadIdx.x; w < (long long)ka * kb; w += blockDim.x) {
        const int i = (int)(w % ka), j = (int)(w / ka);
        double a = 0.0;
        for (int t = b.list_begin; t < b.list_end; ++t) {
            const double v = Ea[(long long)(list_sa[t] - ga) * ka + i] * Eb[(long long)(list_sb[t] - gb) * kb + j];
            a += list_sg[t] > 0 ? v : -v;
        }
        dst_base[b.dst + i + (long long)j * b.ld] = a;
    }
}

// diagonal scaling from the diagonal blocks
__global__ void diag_scale_kernel(const double* D, const long long* d_off, const int* bt_off, int nq_blocks, double* Ds,
                                  int n_total) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_total; t += gridDim.x * blockDim.x) {
        int q = 0;
        while (q + 1 < nq_blocks && bt_off[q + 1] <= t) ++q;
        const int n = bt_off[q + 1] - bt_off[q], r = t - bt_off[q];
        const double h = D[d_off[q] + r + (long long)r * n];
        Ds[t] = h > 0.0 ? 1.0 / sqrt(h) : 1.0;
    }
}

// FP32 copy of S H S for one dense block (rows from row-block qa, columns from qb),
// plus shift on the diagonal of a diagonal block
__global__ void scale_convert_kernel(const double* src, float* dst, int nr, int nc, const double* Ds, int roff,
                                     int coff, float shift, int diag) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nr * nc;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nr), j = (int)(t / nr);
        double v = src[t] * Ds[roff + i] * Ds[coff + j];
        if (diag && i == j) v += shift;
        dst[t] = (float)v;
    }
}

// Cholesky of one <= 64 x 64 diagonal tile in shared memory and the inverse of its
// factor; writes L (lower, strict upper zeroed) in place and inv(L) to `inv` (ld 64).
__global__ void potrf_tile_kernel(float* A, int lda, int nb, float* inv, int* fail) {
    __shared__ float L[kTile][kTile + 1];
    __shared__ int s_ok;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        L[i][j] = (i >= j) ? A[i + (long long)j * lda] : 0.f;
    }
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        if (threadIdx.x == 0) {
            const float d = L[k][k];
            if (!(d > 0.f) || !isfinite(d)) { s_ok = 0; L[k][k] = 1.f; }
            else L[k][k] = sqrtf(d);
        }
        __syncthreads();
        const float piv = L[k][k];
        for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) L[i][k] /= piv;
        __syncthreads();
        const int R = nb - k - 1;
        for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
            const int i = k + 1 + e % R, j = k + 1 + e / R;
            if (i >= j) L[i][j] -= L[i][k] * L[j][k];
        }
        __syncthreads();
    }
    if (!s_ok && threadIdx.x == 0) atomicExch(fail, 1);
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        A[i + (long long)j * lda] = (i >= j) ? L[i][j] : 0.f;
    }
    // inverse of the lower factor: thread j forward-substitutes column j
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        for (int i = 0; i < kTile; ++i) inv[i + j * kTile] = 0.f;
        for (int i = j; i < nb; ++i) {
            float s = (i == j) ? 1.f : 0.f;
            for (int q = j; q < i; ++q) s -= L[i][q] * inv[q + j * kTile];
            inv[i + j * kTile] = s / L[i][i];
        }
    }
}

__global__ void zero_upper_kernel(float* A, int n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % n), j = (int)(t / n);
        if (i < j) A[t] = 0.f;
    }
}

__global__ void copy_tile_kernel(const float* src, int lds, float* dst, int ldd, int nr, int nc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)nr * nc;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nr), j = (int)(e / nr);
        dst[i + (long long)j * ldd] = src[i + (long long)j * lds];
    }
}

// ---- preconditioner application helpers ([element][B] layout, B fastest)
__global__ void to_scaled_f32_kernel(const double* s, const double* Ds, float* o, long long n, int B) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * B; t += (long long)gridDim.x * blockDim.x)
        o[t] = (float)(s[t] * Ds[t / B]);
}

__global__ void from_scaled_f32_kernel(const float* x, const double* Ds, double* z, long long n, int B) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * B; t += (long long)gridDim.x * blockDim.x)
        z[t] = (double)x[t] * Ds[t / B];
}

// Y[j][b] = alpha sum_k X[k][b] M[k + j ldm] + beta Y[j][b] for b < B: one warp per
// output column j reading column j of M contiguously; per (j, b) the sum runs in
// a fixed order, independent of B.
constexpr int kSbBatch = 8;
__global__ void sb_gemm_kernel(const float* X, const float* M, int ldm, float* Y, int K, int ncols, int B, float alpha,
                               float beta) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= ncols) return;
    const float* mj = M + (long long)j * ldm;
    for (int b0 = 0; b0 < B; b0 += kSbBatch) {
        float acc[kSbBatch];
#pragma unroll
        for (int t = 0; t < kSbBatch; ++t) acc[t] = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float m = mj[k];
            const float* xk = X + (long long)k * B + b0;
#pragma unroll
            for (int t = 0; t < kSbBatch; ++t)
                if (b0 + t < B) acc[t] = fmaf(m, xk[t], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < kSbBatch; ++t) {
            const float v = warp_sum(acc[t]);
            if (lane == 0 && b0 + t < B) {
                float* y = Y + (long long)j * B + b0 + t;
                *y = (beta == 0.f) ? alpha * v : alpha * v + beta * (*y);
            }
        }
    }
}

// dst (nc x nr, col-major) = src^T (src nr x nc, col-major)
__global__ void transpose_kernel(const float* src, float* dst, int nr, int nc) {
    __shared__ float t[32][33];
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

template <class T>
msp_status upload(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    MSP_TRY(d.alloc(std::max<size_t>(1, h.size()), s));
    if (!h.empty()) MSP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
    return MSP_OK;
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

}  // namespace

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
    // next-lower patch row
    std::map<std::pair<int, int>, std::vector<std::pair<std::pair<int, int>, signed char>>> pairs;
    for (int r = 0; r + 1 < (int)row_ptr.size(); ++r) {
        for (int a = row_ptr[r]; a < row_ptr[r + 1]; ++a) {
            const unsigned va = (unsigned)row_slot[a];
            const int sa = (int)(va & 0x7fffffffu), ma = slot_patch[sa];
            for (int b = row_ptr[r]; b < row_ptr[r + 1]; ++b) {
                const unsigned vb = (unsigned)row_slot[b];
                const int sb = (int)(vb & 0x7fffffffu), mb = slot_patch[sb];
                const int qa = ma / mx, qb = mb / mx;
                if (!(qa == qb || qa == qb + 1)) continue;
                const signed char sg = (((va ^ vb) & 0x80000000u) ? -1 : 1);
                pairs[{ma, mb}].push_back({{sa, sb}, sg});
            }
        }
    }
    std::vector<PairBlock> pb;
    std::vector<int> lsa, lsb;
    std::vector<signed char> lsg;
    for (auto& kv : pairs) {
        const int ma = kv.first.first, mb = kv.first.second;
        if (B.k[ma] == 0 || B.k[mb] == 0) continue;
        const int qa = ma / mx, qb = mb / mx;
        PairBlock p{};
        p.ma = ma;
        p.mb = mb;
        p.list_begin = (int)lsa.size();
        for (auto& e : kv.second) {
            lsa.push_back(e.first.first);
            lsb.push_back(e.first.second);
            lsg.push_back(e.second);
        }
        p.list_end = (int)lsa.size();
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
    DevBuf<long long> d_doff;
    DevBuf<int> d_btoff;
    MSP_TRY(upload(d_doff, B.bt_d_off, s));
    MSP_TRY(upload(d_btoff, B.bt_off, s));
    MSP_TRY(B.bt_Ds.alloc(std::max(B.Np, 1), s));
    if (B.Np > 0) {
        diag_scale_kernel<<<grid_for(B.Np), 256, 0, s>>>(H64.p, d_doff.p, d_btoff.p, Qn, B.bt_Ds.p, B.Np);
        count_launches(1);
    }
    MSP_CUDA(cudaGetLastError());
    // FP32 factor storage: L_q (in place of D_q), Li_q, C_q (in place of E_q)
    MSP_TRY(B.bt_F.alloc(std::max<long long>(total, 1), s));
    MSP_TRY(B.bt_Li.alloc(std::max<long long>(B.bt_diag_elems, 1), s));
    int max_n = 0;
    for (int q = 0; q < Qn; ++q) max_n = std::max(max_n, B.bt_off[q + 1] - B.bt_off[q]);
    const int max_nt = (max_n + kTile - 1) / kTile;
    DevBuf<float> tinv, trow;
    DevBuf<int> fail;
    MSP_TRY(tinv.alloc((size_t)std::max(max_nt, 1) * kTile * kTile, s));
    MSP_TRY(trow.alloc((size_t)kTile * std::max(max_n, 1), s));
    MSP_TRY(fail.alloc(1, s));
    // temporary for C_q (E_q is read by every output tile of the product)
    long long max_e = 1;
    for (int q = 0; q + 1 < Qn; ++q)
        max_e = std::max<long long>(max_e, (long long)(B.bt_off[q + 2] - B.bt_off[q + 1]) * (B.bt_off[q + 1] - B.bt_off[q]));
    DevBuf<float> ctmp;
    MSP_TRY(ctmp.alloc((size_t)max_e, s));
    const float shifts[3] = {0.f, 1e-5f, 1e-3f};
    int hfail = 1;
    for (int attempt = 0; attempt < 3 && hfail; ++attempt) {
        MSP_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), s));
        MSP_CUDA(cudaMemsetAsync(B.bt_Li.p, 0, sizeof(float) * std::max<long long>(B.bt_diag_elems, 1), s));
        // scaled FP32 copies
        for (int q = 0; q < Qn; ++q) {
            const int n = B.bt_off[q + 1] - B.bt_off[q];
            if (n == 0) continue;
            scale_convert_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(H64.p + B.bt_d_off[q], B.bt_F.p + B.bt_d_off[q],
                                                                             n, n, B.bt_Ds.p, B.bt_off[q], B.bt_off[q],
                                                                             shifts[attempt], 1);
            count_launches(1);
            if (q + 1 < Qn) {
                const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
                if (n1 == 0) continue;
                scale_convert_kernel<<<grid_for((long long)n1 * n), 256, 0, s>>>(
                    H64.p + B.bt_e_off[q], B.bt_F.p + B.bt_e_off[q], n1, n, B.bt_Ds.p, B.bt_off[q + 1], B.bt_off[q], 0.f, 0);
                count_launches(1);
            }
        }
        MSP_CUDA(cudaGetLastError());
        // Collect the whole factorisation's GEMMs in order, then launch them in order
        // with their descriptors resident in one device array.
        struct Step {
            int kind;        // 0 gemm, 1 potrf tile, 2 zero upper, 3 copy tile
            GemmDescT<float> g;
            bool tA, tB;
            float* ptr;
            int ld, nb, nr, nc;
            float* inv;
            const float* src;
            int lds;
        };
        std::vector<Step> steps;
        auto add_gemm = [&](const float* A, int lda, const float* Bm, int ldb, float* C, int ldc, int M, int N, int K,
                            float alpha, float beta, bool tA, bool tB) {
            if (M <= 0 || N <= 0 || K <= 0) return;
            Step st{};
            st.kind = 0;
            st.g = GemmDescT<float>{A, Bm, C, M, N, K, lda, ldb, ldc, alpha, beta};
            st.tA = tA;
            st.tB = tB;
            steps.push_back(st);
        };
        for (int q = 0; q < Qn; ++q) {
            const int n = B.bt_off[q + 1] - B.bt_off[q];
            if (n == 0) continue;
            float* Dq = B.bt_F.p + B.bt_d_off[q];
            float* Li = B.bt_Li.p + B.bt_d_off[q];
            if (q > 0) {   // D_q -= C_{q-1} C_{q-1}^T
                const int n0 = B.bt_off[q] - B.bt_off[q - 1];
                const float* Cp = B.bt_F.p + B.bt_e_off[q - 1];
                add_gemm(Cp, n, Cp, n, Dq, n, n, n, n0, -1.f, 1.f, false, true);
            }
            const int nt = (n + kTile - 1) / kTile;
            for (int kt = 0; kt < nt; ++kt) {
                const int r0 = kt * kTile, nb = std::min(kTile, n - r0), m = n - r0 - nb;
                Step st{};
                st.kind = 1;
                st.ptr = Dq + r0 + (long long)r0 * n;
                st.ld = n;
                st.nb = nb;
                st.inv = tinv.p + (size_t)kt * kTile * kTile;
                steps.push_back(st);
                if (m > 0) {
                    float* panel = Dq + (r0 + nb) + (long long)r0 * n;
                    // panel <- panel inv(L_kk)^T (in place: one column tile)
                    add_gemm(panel, n, st.inv, kTile, panel, n, m, nb, nb, 1.f, 0.f, false, true);
                    // trailing -= panel panel^T
                    add_gemm(panel, n, panel, n, Dq + (r0 + nb) + (long long)(r0 + nb) * n, n, m, m, nb, -1.f, 1.f, false, true);
                }
            }
            Step zu{};
            zu.kind = 2;
            zu.ptr = Dq;
            zu.nb = n;
            steps.push_back(zu);
            // Li = L^{-1} by tile rows: X[it, :it] = -inv(L_ii) L[it, :it] X[:it, :it]; X[it, it] = inv(L_ii)
            for (int it = 0; it < nt; ++it) {
                const int r0 = it * kTile, nb = std::min(kTile, n - r0);
                if (it > 0) {
                    add_gemm(Dq + r0, n, Li, n, trow.p, kTile, nb, r0, r0, 1.f, 0.f, false, false);
                    add_gemm(tinv.p + (size_t)it * kTile * kTile, kTile, trow.p, kTile, Li + r0, n, nb, r0, nb, -1.f, 0.f,
                             false, false);
                }
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
            if (q + 1 < Qn) {   // C_q = E_q Li^T
                const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
                float* Eq = B.bt_F.p + B.bt_e_off[q];
                // C_q overwrites E_q: go through a temporary (E_q is read by every output tile)
                add_gemm(Eq, n1, Li, n, ctmp.p, n1, n1, n, n, 1.f, 0.f, false, true);
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
        std::vector<GemmDescT<float>> gds;
        for (auto& st : steps)
            if (st.kind == 0) gds.push_back(st.g);
        DevBuf<GemmDescT<float>> d_all;
        MSP_TRY(upload(d_all, gds, s));
        size_t gi = 0;
        for (auto& st : steps) {
            if (st.kind == 0) {
                gemm_batched<float>(d_all.p + gi, 1, st.g.M, st.g.N, st.tA, st.tB, s);
                ++gi;
            } else if (st.kind == 1) {
                potrf_tile_kernel<<<1, 256, 0, s>>>(st.ptr, st.ld, st.nb, st.inv, fail.p);
                count_launches(1);
            } else if (st.kind == 2) {
                zero_upper_kernel<<<grid_for((long long)st.nb * st.nb), 256, 0, s>>>(st.ptr, st.nb);
                count_launches(1);
            } else {
                copy_tile_kernel<<<std::max(1, std::min(1024, (st.nr * st.nc + 255) / 256)), 256, 0, s>>>(st.src, st.lds, st.ptr,
                                                                                                          st.ld, st.nr, st.nc);
                count_launches(1);
            }
        }
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaMemcpyAsync(&hfail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        B.bt_shift = shifts[attempt];
    }
    if (hfail) {
        set_error("msp_extract_basis: online preconditioner factorisation broke down after shifts");
        return MSP_ERR_BREAKDOWN;
    }
    // transposed copies for the sweeps (each product then reads contiguous columns)
    MSP_TRY(B.bt_FT.alloc(std::max<long long>(total, 1), s));
    MSP_TRY(B.bt_LiT.alloc(std::max<long long>(B.bt_diag_elems, 1), s));
    for (int q = 0; q < Qn; ++q) {
        const int n = B.bt_off[q + 1] - B.bt_off[q];
        if (n == 0) continue;
        dim3 g1((n + 31) / 32, (n + 31) / 32);
        transpose_kernel<<<g1, dim3(32, 8), 0, s>>>(B.bt_Li.p + B.bt_d_off[q], B.bt_LiT.p + B.bt_d_off[q], n, n);
        count_launches(1);
        if (q + 1 < Qn) {
            const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
            dim3 g2((n1 + 31) / 32, (n + 31) / 32);
            transpose_kernel<<<g2, dim3(32, 8), 0, s>>>(B.bt_F.p + B.bt_e_off[q], B.bt_FT.p + B.bt_e_off[q], n1, n);
            count_launches(1);
        }
    }
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

// z = S (L L^T)^{-1} S s for a batch of Bsz vectors ([element][B] layout, FP64 in and out)
msp_status apply_online_factor(Basis& B, const double* s_in, double* z_out, int Bsz, cudaStream_t s) {
    const long long n = B.Np;
    if (n == 0) return MSP_OK;
    if ((long long)B.bt_w1.n < n * Bsz) {
        MSP_TRY(B.bt_w1.alloc((size_t)n * std::max(Bsz, 1), s));
        MSP_TRY(B.bt_w2.alloc((size_t)n * std::max(Bsz, 1), s));
    }
    float* y = B.bt_w1.p;   // right-hand side, then the forward sweep's result
    float* x = B.bt_w2.p;   // backward sweep's result
    to_scaled_f32_kernel<<<grid_for(n * Bsz), 256, 0, s>>>(s_in, B.bt_Ds.p, y, n, Bsz);
    count_launches(1);
    const int Qn = B.bt_q;
    const int wpb = 8;   // warps per block of the small-batch products
    auto prod = [&](const float* X, const float* M, int ldm, float* Y, int K, int ncols, float alpha, float beta) {
        if (K <= 0 || ncols <= 0) return;
        sb_gemm_kernel<<<(ncols + wpb - 1) / wpb, 32 * wpb, 0, s>>>(X, M, ldm, Y, K, ncols, Bsz, alpha, beta);
        count_launches(1);
    };
    // forward: y_q -= x_{q-1} C_{q-1}^T;  x_q = y_q Li_q^T   (row vectors, [element][B])
    for (int q = 0; q < Qn; ++q) {
        const int nq = B.bt_off[q + 1] - B.bt_off[q];
        if (nq == 0) continue;
        float* yq = y + (long long)B.bt_off[q] * Bsz;
        float* xq = x + (long long)B.bt_off[q] * Bsz;
        if (q > 0) {
            const int n0 = B.bt_off[q] - B.bt_off[q - 1];
            prod(x + (long long)B.bt_off[q - 1] * Bsz, B.bt_FT.p + B.bt_e_off[q - 1], n0, yq, n0, nq, -1.f, 1.f);
        }
        prod(yq, B.bt_LiT.p + B.bt_d_off[q], nq, xq, nq, nq, 1.f, 0.f);
    }
    // backward: x_q -= z_{q+1} C_q;  z_q = x_q Li_q   (z written into y)
    for (int q = Qn - 1; q >= 0; --q) {
        const int nq = B.bt_off[q + 1] - B.bt_off[q];
        if (nq == 0) continue;
        float* xq = x + (long long)B.bt_off[q] * Bsz;
        float* zq = y + (long long)B.bt_off[q] * Bsz;
        if (q + 1 < Qn) {
            const int n1 = B.bt_off[q + 2] - B.bt_off[q + 1];
            prod(y + (long long)B.bt_off[q + 1] * Bsz, B.bt_F.p + B.bt_e_off[q], n1, xq, n1, nq, -1.f, 1.f);
        }
        prod(xq, B.bt_Li.p + B.bt_d_off[q], nq, zq, nq, nq, 1.f, 0.f);
    }
    from_scaled_f32_kernel<<<grid_for(n * Bsz), 256, 0, s>>>(y, B.bt_Ds.p, z_out, n, Bsz);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace msp
