// Persistence and inspection of a basis: msp_save_basis / msp_load_basis write and
// read the geometry, the bases Q_m with their singular values and the medium's face
// coefficients; the online operators (edge operators, preconditioner blocks, the
// block-row factor) are rebuilt on load by the same code as the extraction, so a
// loaded basis gives the same online results as the one saved.
// msp_get_online_system exports P~ (COO) and d of Eq. elliptic_cond_reduced.
#include "internal.h"

#include <cstdio>
#include <cstring>
#include <vector>

namespace msp {

namespace {

constexpr char kMagic[8] = {'M', 'S', 'P', 'B', 'A', 'S', 'I', 'S'};
constexpr uint32_t kVersion = 1;

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

template <class T>
bool put(FILE* f, const T* p, size_t n) {
    return n == 0 || fwrite(p, sizeof(T), n, f) == n;
}
template <class T>
bool get(FILE* f, T* p, size_t n) {
    return n == 0 || fread(p, sizeof(T), n, f) == n;
}
template <class T>
bool put_vec(FILE* f, const std::vector<T>& v) {
    const int64_t n = (int64_t)v.size();
    return put(f, &n, 1) && put(f, v.data(), v.size());
}
template <class T>
bool get_vec(FILE* f, std::vector<T>& v, int64_t max_n) {
    int64_t n = 0;
    if (!get(f, &n, 1) || n < 0 || n > max_n) return false;
    v.resize((size_t)n);
    return get(f, v.data(), v.size());
}

long long q_elems(const Basis& B) {
    long long n = 0;
    for (size_t m = 0; m < B.patches.size(); ++m) n = std::max<long long>(n, B.q_off[m] + (long long)B.patches[m].n_k * B.k[m]);
    return n;
}

}  // namespace

}  // namespace msp

using namespace msp;

extern "C" msp_status msp_save_basis(msp_basis b, const char* path) {
    clear_error();
    MSP_CHECK_ARG(b && path, "msp_save_basis: NULL argument");
    const Basis& B = b->B;
    File fh;
    fh.f = fopen(path, "wb");
    if (!fh.f) {
        set_error(std::string("msp_save_basis: cannot open ") + path + " for writing");
        return MSP_ERR_INVALID_ARG;
    }
    const long long nq = q_elems(B);
    const size_t nf = (size_t)(B.N + 1) * B.N;
    std::vector<double> Q((size_t)nq), aE(nf), aN(nf);
    MSP_CUDA(cudaMemcpy(Q.data(), B.Q.p, sizeof(double) * Q.size(), cudaMemcpyDeviceToHost));
    MSP_CUDA(cudaMemcpy(aE.data(), B.aE.p, sizeof(double) * nf, cudaMemcpyDeviceToHost));
    MSP_CUDA(cudaMemcpy(aN.data(), B.aN.p, sizeof(double) * nf, cudaMemcpyDeviceToHost));
    const int32_t hdr[4] = {(int32_t)B.N, (int32_t)B.mx, (int32_t)B.my, (int32_t)sizeof(PatchDev)};
    bool ok = put(fh.f, kMagic, 8) && put(fh.f, &kVersion, 1) && put(fh.f, hdr, 4) && put_vec(fh.f, B.xb) &&
              put_vec(fh.f, B.yb) && put_vec(fh.f, B.patches) && put_vec(fh.f, B.k) && put_vec(fh.f, B.sigma) &&
              put_vec(fh.f, B.sigma_off) && put_vec(fh.f, B.q_off) && put_vec(fh.f, Q) && put_vec(fh.f, aE) &&
              put_vec(fh.f, aN);
    if (!ok) {
        set_error(std::string("msp_save_basis: write to ") + path + " failed");
        return MSP_ERR_INVALID_ARG;
    }
    return MSP_OK;
}

extern "C" msp_status msp_load_basis(const char* path, msp_basis* out) {
    clear_error();
    MSP_CHECK_ARG(path && out, "msp_load_basis: NULL argument");
    *out = nullptr;
    File fh;
    fh.f = fopen(path, "rb");
    if (!fh.f) {
        set_error(std::string("msp_load_basis: cannot open ") + path);
        return MSP_ERR_INVALID_ARG;
    }
    char magic[8];
    uint32_t ver = 0;
    int32_t hdr[4];
    if (!get(fh.f, magic, 8) || memcmp(magic, kMagic, 8) != 0 || !get(fh.f, &ver, 1) || ver != kVersion ||
        !get(fh.f, hdr, 4) || hdr[3] != (int32_t)sizeof(PatchDev) || hdr[0] < 2 || hdr[1] < 1 || hdr[2] < 1) {
        set_error(std::string("msp_load_basis: ") + path + " is not a basis file of this library version");
        return MSP_ERR_INVALID_ARG;
    }
    auto* h = new msp_basis_s();
    Basis& B = h->B;
    B.N = hdr[0];
    B.mx = hdr[1];
    B.my = hdr[2];
    const int64_t big = (int64_t)1 << 40;
    std::vector<double> Q, aE, aN;
    const bool ok = get_vec(fh.f, B.xb, B.N + 1) && get_vec(fh.f, B.yb, B.N + 1) &&
                    get_vec(fh.f, B.patches, (int64_t)B.mx * B.my) && get_vec(fh.f, B.k, (int64_t)B.mx * B.my) &&
                    get_vec(fh.f, B.sigma, big) && get_vec(fh.f, B.sigma_off, (int64_t)B.mx * B.my) &&
                    get_vec(fh.f, B.q_off, (int64_t)B.mx * B.my) && get_vec(fh.f, Q, big) && get_vec(fh.f, aE, big) &&
                    get_vec(fh.f, aN, big);
    const size_t nf = (size_t)(B.N + 1) * B.N;
    if (!ok || B.patches.size() != (size_t)B.mx * B.my || B.k.size() != B.patches.size() ||
        B.q_off.size() != B.patches.size() || aE.size() != nf || aN.size() != nf ||
        (long long)Q.size() < q_elems(B)) {
        delete h;
        set_error(std::string("msp_load_basis: ") + path + " is truncated or inconsistent");
        return MSP_ERR_INVALID_ARG;
    }
    cudaGetDevice(&B.device);
    cudaStream_t s = nullptr;
    DevBuf<double> dE, dN;
    msp_status st = B.Q.alloc(std::max<size_t>(Q.size(), 1), s);
    if (st == MSP_OK) st = dE.alloc(nf, s);
    if (st == MSP_OK) st = dN.alloc(nf, s);
    if (st == MSP_OK && (cudaMemcpy(B.Q.p, Q.data(), sizeof(double) * Q.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(dE.p, aE.data(), sizeof(double) * nf, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(dN.p, aN.data(), sizeof(double) * nf, cudaMemcpyHostToDevice) != cudaSuccess)) {
        set_error("msp_load_basis: copy to the device failed");
        st = MSP_ERR_CUDA;
    }
    if (st == MSP_OK) st = finish_basis(B, dE.p, dN.p, s);
    if (st == MSP_OK && cudaStreamSynchronize(s) != cudaSuccess) st = MSP_ERR_CUDA;
    if (st != MSP_OK) {
        delete h;
        return st;
    }
    *out = h;
    return MSP_OK;
}

extern "C" msp_status msp_basis_patch(msp_basis b, int patch, int* n_cells, int* n_patches, msp_patch_info* out) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_basis_patch: NULL basis");
    const Basis& B = b->B;
    if (n_cells) *n_cells = B.N;
    if (n_patches) *n_patches = (int)B.patches.size();
    if (!out) return MSP_OK;
    MSP_CHECK_ARG(patch >= 0 && patch < (int)B.patches.size(), "msp_basis_patch: patch out of range");
    const PatchDev& P = B.patches[patch];
    out->x0 = P.x0; out->x1 = P.x1; out->y0 = P.y0; out->y1 = P.y1;
    out->X0 = P.X0; out->X1 = P.X1; out->Y0 = P.Y0; out->Y1 = P.Y1;
    out->n_k = P.n_k; out->n_ring = P.n_ring; out->samples = P.samples; out->n_b = P.n_b; out->cols = P.cols;
    out->snap_offset = P.snap_offset;
    return MSP_OK;
}

extern "C" msp_status msp_get_online_system(msp_basis b, const double* phi_host, int64_t capacity, int64_t* nnz,
                                            int* rows, int* cols, double* vals, double* d_host) {
    clear_error();
    MSP_CHECK_ARG(b && nnz, "msp_get_online_system: NULL argument");
    const Basis& B = b->B;
    const int np = (int)B.patches.size();
    std::vector<int> row_ptr(B.n_rows + 1), row_slot, row_bnd(B.n_rows);
    MSP_CUDA(cudaMemcpy(row_ptr.data(), B.row_ptr.p, sizeof(int) * row_ptr.size(), cudaMemcpyDeviceToHost));
    row_slot.resize(row_ptr.back());
    MSP_CUDA(cudaMemcpy(row_slot.data(), B.row_slot.p, sizeof(int) * row_slot.size(), cudaMemcpyDeviceToHost));
    MSP_CUDA(cudaMemcpy(row_bnd.data(), B.row_bnd.p, sizeof(int) * row_bnd.size(), cudaMemcpyDeviceToHost));
    // slot -> patch
    std::vector<int> slot_patch(B.n_slots);
    for (int m = 0; m < np; ++m)
        for (int g = B.slot_off[m]; g < B.slot_off[m + 1]; ++g) slot_patch[g] = m;
    int64_t count = 0;
    for (int r = 0; r < B.n_rows; ++r)
        for (int t = row_ptr[r]; t < row_ptr[r + 1]; ++t)
            count += B.k[slot_patch[(unsigned)row_slot[t] & 0x7fffffffu]];
    *nnz = count;
    if (d_host) {
        MSP_CHECK_ARG(phi_host, "msp_get_online_system: d requested without phi");
        for (int r = 0; r < B.n_rows; ++r) d_host[r] = row_bnd[r] >= 0 ? phi_host[row_bnd[r]] : 0.0;
    }
    if (!rows) return MSP_OK;
    MSP_CHECK_ARG(cols && vals && capacity >= count, "msp_get_online_system: output arrays missing or too short");
    std::vector<double> E(B.E.n);
    MSP_CUDA(cudaMemcpy(E.data(), B.E.p, sizeof(double) * E.size(), cudaMemcpyDeviceToHost));
    int64_t w = 0;
    for (int r = 0; r < B.n_rows; ++r)
        for (int t = row_ptr[r]; t < row_ptr[r + 1]; ++t) {
            const unsigned v = (unsigned)row_slot[t];
            const int g = (int)(v & 0x7fffffffu), m = slot_patch[g];
            const double sg = (v & 0x80000000u) ? -1.0 : 1.0;
            const double* er = E.data() + B.e_off[m] + (long long)(g - B.slot_off[m]) * B.k[m];
            for (int j = 0; j < B.k[m]; ++j) {
                rows[w] = r;
                cols[w] = B.c_off[m] + j;
                vals[w] = sg * er[j];
                ++w;
            }
        }
    return MSP_OK;
}
