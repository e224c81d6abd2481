// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <string>
#include <memory>
#include <vector>

#include "../../include/msp.h"
#include "dense.cuh"

namespace msp {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();
msp_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define MSP_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return ::msp::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define MSP_CHECK_ARG(cond, msg)                                                    \
    do {                                                                            \
        if (!(cond)) { ::msp::set_error(msg); return MSP_ERR_INVALID_ARG; }          \
    } while (0)

#define MSP_TRY(call)                                                               \
    do { msp_status s_ = (call); if (s_ != MSP_OK) return s_; } while (0)

// Stream-ordered device buffer owned by a handle.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    // A request beyond the device's whole memory is refused before the call (free
    // memory is no test: the stream-ordered pool may serve a request from memory it
    // holds); a stream-ordered allocation may also report its failure through the
    // last-error state instead of its return value, so that is read (and cleared)
    // right after.
    msp_status alloc(size_t count, cudaStream_t s) {
        free_now();
        if (count == 0) return MSP_OK;
        const size_t bytes = count * sizeof(T);
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e == cudaSuccess && bytes > total_b) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&p, bytes, s);
        if (e == cudaSuccess) {
            const cudaError_t late = cudaGetLastError();
            if (late != cudaSuccess) {
                if (p) cudaFreeAsync(p, s);
                e = late;
            }
        }
        if (e != cudaSuccess) {
            p = nullptr;
            set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
                      cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? MSP_ERR_OOM : MSP_ERR_CUDA;
        }
        n = count;
        return MSP_OK;
    }
    void free_now() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { free_now(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

// Stream-ordered copy of a host vector into a (re)allocated device buffer (at
// least one element, so that the pointer is valid for empty tables).
template <class T>
msp_status upload(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    MSP_TRY(d.alloc(std::max<size_t>(1, h.size()), s));
    if (!h.empty()) MSP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
    return MSP_OK;
}

// Work buffers of the tensor-core FP64 GEMM (ozaki_gemm.cu), grown on demand.
struct OzakiWork {
    DevBuf<unsigned short> slices;   // BF16 slices of both operands of every product
    DevBuf<int> scales;              // power-of-two scale exponents of the rows / columns
    DevBuf<long long> ents;          // per-product tables
    DevBuf<int> err;                 // set by a timed-out wait
};
// FP64 products on the tensor cores (error-free BF16 slicing): every descriptor
// of h (host copy of d_dev), C = alpha op(A) op(B) + beta C; the structure flags
// mark zero ranges, tiles strictly above the diagonal are skipped with `lower`.
bool ozaki_gemm_supported(const std::vector<GemmDesc>& h);
msp_status ozaki_gemm_batched(const std::vector<GemmDesc>& h, const GemmDesc* d_dev, bool transA, bool transB,
                              cudaStream_t s, OzakiWork& w);
// TIMEOUT if a product on this workspace gave up a bounded wait (synchronises).
msp_status ozaki_check(OzakiWork& w, cudaStream_t s);
// Engine of the FP64 products of the extraction and the online factorisation:
// 0 tensor cores (default), 1 CUDA cores.
int fp64_gemm_engine();
// Jacobi SVD of the extraction: FP32 sweeps first, then FP64 (msp_set_svd_mode).
bool svd_mixed();
bool svd_qr();

// ------------------------------------------------------------------ geometry

// Per-patch geometry as the kernels see it.
struct PatchDev {
    int x0, x1, y0, y1;      // K_m closed node box
    int X0, X1, Y0, Y1;      // buffered box
    int n_k, n_ring, samples, n_b, cols;
    int bpos_offset;         // first entry in the boundary-position list
    long long snap_offset;   // first element of the snapshot block
};

struct Medium {
    int N = 0;
    int mx = 0, my = 0;
    std::vector<int> xb, yb;
    std::vector<PatchDev> patches;      // host copy
    std::vector<int> bpos;              // ring positions on the domain boundary, per patch
    long long snap_elems = 0;
    int max_tile_nodes = 0;             // max (X1-X0+1)(Y1-Y0+1)
    int max_cols = 0;
    DevBuf<double> aE, aN;              // FP64 face coefficients
    DevBuf<float> aE32, aN32;           // FP32 copies (mixed path)
    DevBuf<PatchDev> patches_dev;
    DevBuf<int> bpos_dev;
    DevBuf<double> snaps;               // snapshot blocks
    DevBuf<int2> items;                 // (patch, column) work items, longest first
    std::vector<int2> items_host;
    int n_items = 0;
    int n_tile_items[2] = {0, 0};       // per precision: leading items the tile kernel takes
    DevBuf<int2> items_prec[2];         // per precision: items ordered tile-eligible first
    std::vector<int2> items_prec_host[2];
    DevBuf<int> counter;
    DevBuf<int> item_stats;             // per item: iterations, refinements, flag
    DevBuf<double> scratch;             // tile-kernel workspace (FP64 iterate per CTA)
    DevBuf<double> scratch_global;      // global-kernel workspace
    bool sampled = false;
    int device = 0;
    // launch of the local solves: mode 0 split (tile kernel + global kernel), 1 fused
    // (one persistent launch); rows instance of the tile kernel (0: the smallest that fits);
    // set by msp_medium_set_launch or by the autotuner, per precision
    int launch_mode[2] = {0, 0};
    int launch_rows[2] = {0, 0};
    bool tuned[2] = {false, false};
    // direct local solver (launch mode MSP_LAUNCH_DIRECT): per-patch FP32 inverse
    // Schur complements of the row-block LDL^T factorisation, FP64 refinement state
    struct Direct {
        bool planned = false, factored = false;
        int n_cols = 0, n_chunks = 0, max_nxp = 0;
        long long w_elems = 0, s_elems = 0, x_elems = 0, r_elems = 0, k_elems = 0;
        DevBuf<long long> w_off, s_off, x_off, r_off, k_off;   // per patch
        DevBuf<int> col_base;                                   // per patch: first global column
        DevBuf<int2> cols;                                      // global column -> (patch, column)
        DevBuf<int4> chunks;                                    // (patch, first column, columns, -)
        DevBuf<int> stat_idx;                                   // global column -> statistics slot
        DevBuf<float> W, D, R, K;
        DevBuf<double> s, X, b2, r2;
        DevBuf<int> active, passes;
        int chunk_smem_max = 0, factor_smem_max = 0;
        // optional CUDA-event timing of the phases of the last call: factor, init,
        // residual, solve, finish (start/stop event pairs, summed per phase)
        bool timing = false;
        std::vector<cudaEvent_t> ev;
        std::vector<int> ev_phase;
        int ev_used = 0;
        ~Direct() {
            for (cudaEvent_t e : ev) cudaEventDestroy(e);
        }
    } dir;
    // CUDA graph of the local-solve launches, replayed while the configuration is unchanged
    bool use_graph = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    cudaStream_t capture_stream = nullptr;
    double graph_key[2][6] = {};
    long long graph_launches[2] = {0, 0};   // kernel launches one replay of the graph makes
};

// Ring node t of node box (X0,X1,Y0,Y1): counter-clockwise from (X0,Y0).
__host__ __device__ inline void ring_node(int X0, int X1, int Y0, int Y1, int t, int& i, int& j) {
    const int wx = X1 - X0, wy = Y1 - Y0;
    if (t < wx) { i = X0 + t; j = Y0; }
    else if (t < wx + wy) { i = X1; j = Y0 + (t - wx); }
    else if (t < 2 * wx + wy) { i = X1 - (t - wx - wy); j = Y1; }
    else { i = X0; j = Y1 - (t - 2 * wx - wy); }
}

// Block-tridiagonal factor storage in one precision: L_q and C_q (F), L_q^{-1} (Li),
// their transposes, and the sweep work vectors.
template <class T>
struct BtStore {
    DevBuf<T> F, Li, FT, LiT, w1, w2;
    void free_all() {
        F.free_now(); Li.free_now(); FT.free_now(); LiT.free_now(); w1.free_now(); w2.free_now();
    }
};

// Reduced bases and the online operators of one medium.
struct Basis {
    int N = 0, mx = 0, my = 0;
    std::vector<int> xb, yb;
    std::vector<PatchDev> patches;
    std::vector<int> k;                 // kept vectors per patch
    std::vector<double> sigma;          // singular values, cols_m per patch
    std::vector<long long> sigma_off;
    std::vector<long long> q_off;       // Q_m block offsets (n_k x k_m)
    std::vector<int> c_off;             // first coefficient of patch m
    std::vector<int> n_e;               // ring nodes of K_m
    std::vector<int> slot_off;          // first edge slot of patch m (2 slots per ring node)
    std::vector<long long> e_off;       // E_m block offsets (2 n_e x k_m, row-major)
    std::vector<long long> binv_off;    // preconditioner block offsets (k_m x k_m)
    int Np = 0, n_slots = 0, n_rows = 0, n_skel = 0;
    DevBuf<double> Q, E, Binv;
    // device tables
    DevBuf<int> d_c_off, d_k, d_slot_off, d_ne;
    DevBuf<long long> d_q_off, d_e_off, d_binv_off;
    DevBuf<PatchDev> d_patches;
    DevBuf<int> row_ptr, row_slot, row_bnd;      // P~ rows: entries (global slot, sign in bit 31) and rhs ring position
    DevBuf<int> tr_ptr, tr_ent;                  // transpose: per global slot, rows (sign in bit 31)
    DevBuf<int> sk_ptr, sk_slot, sk_node, sk_ring;  // skeleton nodes: V slots, node index, ring position (-1 inside)
    // online work space (grown on demand)
    int cap_batch = 0;
    DevBuf<double> w_c, w_p, w_z, w_e, w_q, w_r, w_part, w_scal;
    DevBuf<int> w_iters;
    // block-tridiagonal FP32 factor of the scaled normal matrix (online preconditioner)
    int bt_q = 0;
    std::vector<int> bt_off;            // first unknown of each row of patches
    std::vector<long long> bt_d_off;    // diagonal block offsets
    std::vector<long long> bt_e_off;    // sub-diagonal block offsets
    long long bt_diag_elems = 0;
    float bt_shift = 0.f;
    DevBuf<double> bt_Fi;               // patch-block scaling R_m^{-1} = L_m^{-T} (H_mm = L_m L_m^T)
    int bt_prec = 0;                    // 1: FP32 factor, 2: FP64 factor
    int bt_apply_mode = 0;              // FP64 factor applied: 0 by batch size, 1 in FP64, 2 through bt32
    std::vector<int> bt_elo, bt_ehi;    // per patch: range of coupled patches in the row above
    DevBuf<int> d_bt_off;               // device copies of the block offsets (sweep kernel)
    DevBuf<int> d_bt_rowlo;             // per unknown: first nonzero column of its row of C_{q-1}
    DevBuf<long long> d_bt_d_off, d_bt_e_off;
    DevBuf<unsigned int> d_bt_bar;      // grid barrier of the sweep kernel: arrivals, generation, error
    // boundary-to-coefficient map (serving): G (N_p x 4N, FP32) and FP32 bases
    DevBuf<float> G32, Q32, E32;
    DevBuf<double> aE, aN;              // the medium's FP64 face coefficients (kept for msp_save_basis)
    DevBuf<float> Gt_hi, Gt_lo;         // G tiled for the tensor-core GEMM (TF32 high part, FP32 remainder)
    bool map_built = false;
    int map_engine = 0;                 // 0: tensor cores (tcgen05, split TF32), 1: CUDA cores (FP32 FMA)
    BtStore<float> bt32;
    BtStore<double> bt64;
    DevBuf<double> w_s;                 // normal-equation residual s = P^T r
    bool use_block_jacobi = false;      // online preconditioner: patch blocks only
    // CUDA events at the phase boundaries of the extraction that built this basis
    // (when extraction timing is on): Cholesky-QR | Jacobi SVD | truncation and
    // projection | online operators | online factor
    std::vector<cudaEvent_t> ext_ev;
    std::vector<double> jac_cols;       // per patch: snapshot columns (Jacobi work)
    std::vector<int> jac_sweeps;        // per patch: Jacobi sweeps
    ~Basis() {
        for (cudaEvent_t e : ext_ev) cudaEventDestroy(e);
    }
    int max_jacobi_sweeps = 0, max_cholqr_tries = 0;
    float mean_jacobi_sweeps = 0.f;
    int device = 0;
    // constrained least-squares variant of the online step: the derived basis and
    // tables, built on first use (online_constrained.cu); a derived basis has no
    // boundary rows
    bool no_boundary_rows = false;
    std::shared_ptr<struct ConstrainedOnline> cons;
    // overlapping Schwarz variant of the online step: B_m = Q_m^T G~_m, ring tables,
    // coarse space (online_ras.cu), built by msp_ras_setup
    std::shared_ptr<struct RasOnline> ras;
};

// Boundary data imposed exactly: per boundary patch c_m = Z_m phi_m + N_m z_m
// (null-space method), the reduced problem on the derived basis `red`.
struct ConstrainedOnline {
    std::unique_ptr<Basis> red;          // bases Q_m N_m (boundary patches) / Q_m, continuity rows only
    std::vector<int> nb;                 // domain-boundary nodes of each K_m (0 inside)
    DevBuf<int> d_nb, d_bring, d_kr, d_cr_off;
    DevBuf<long long> d_bring_off, d_zp_off, d_np_off;
    DevBuf<double> Z, Nm;                // per boundary patch: k_m x nb_m and k_m x (k_m - nb_m), column-major
    DevBuf<double> cp, cf, ep, dq, part; // work: [coefficient][B], [coefficient][B], [slot][B], [row][B], partials
    int cap = 0;
};
msp_status build_constrained(Basis& B, cudaStream_t s);
void cons_particular(const Basis& B, const ConstrainedOnline& C, const double* phi, int n4, int Bsz, double* cp,
                     cudaStream_t s);
void cons_combine(const Basis& B, const ConstrainedOnline& C, const double* cp, const double* z, int Bsz, double* cf,
                  cudaStream_t s);
msp_status online_solve_constrained(Basis& B, const double* phi, int batch, double tol, int max_iter, double* u,
                                    double* c_out, int* iters_host, cudaStream_t s);

// ------------------------------------------------------------------ launchers
namespace gpath {
struct SolveArgs;
}

struct LocalSolveCfg {
    int precision;       // MSP_FP64 / MSP_MIXED
    double tol;          // outer relative residual target
    double inner_tol;    // FP32 inner solve target (mixed)
    int max_iter;        // per inner solve
    int max_ref;         // refinement steps (mixed)
    uint64_t seed;
};

msp_status launch_medium_coefficients(Medium& M, const msp_medium_desc& d, cudaStream_t s);
// Optional subset of the items for one launch of the local solves (the autotuner's
// probe runs): the tile items, the rest, and the launch configuration to use.
struct LaunchItems {
    const int2* tile;
    int n_tile;
    const int2* rest;
    int n_rest;
    int mode, rows;
};
msp_status launch_local_solves(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s, const LaunchItems* li = nullptr);
// The direct local solver (launch mode MSP_LAUNCH_DIRECT): eligibility and launch.
bool direct_fits(const Medium& M);
msp_status launch_local_solves_direct(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s);
// The local solves of msp_sample_patches: launched directly, or through the medium's
// CUDA graph when graphs are on (captured on the first call of a configuration).
msp_status sample_launch(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s);
int tile_launch_rows(const std::vector<PatchDev>& patches, int precision);
bool tile_kernel_fits(const PatchDev& P, int precision, int R);
msp_status launch_local_solves_tile(Medium& M, const LocalSolveCfg& cfg, const int2* items, int n_items, int* counter,
                                    cudaStream_t s, const gpath::SolveArgs* fused = nullptr, int R_launch = 0);
msp_status launch_ring_samples(Medium& M, int patch, uint64_t seed, double* dst, cudaStream_t s);
msp_status build_basis(Medium& M, double tau, int precision, cudaStream_t s, Basis& B);
msp_status finish_basis(Basis& B, const double* aE_dev, const double* aN_dev, cudaStream_t s);
// boundary-to-coefficient map (serving)
struct MapWork {
    float* phi32 = nullptr;
    float* c32 = nullptr;
    double* e = nullptr;
    float* b_hi = nullptr;      // phi tiled for the tensor-core GEMM
    float* b_lo = nullptr;
    int* err = nullptr;         // timed-out waits of the tensor-core GEMM
    int cap = 0;
};
// nonzero if a map GEMM on this workspace reported a timed-out wait (synchronises the stream)
msp_status map_work_check(MapWork& w, cudaStream_t s);
msp_status map_work_alloc(const Basis& Bs, int max_batch, MapWork& w);
void map_work_free(MapWork& w);
msp_status build_online_map(Basis& Bs, double tol, int max_iter, cudaStream_t s);
msp_status online_solve_map(const Basis& Bs, const double* phi, int batch, double* u, cudaStream_t s, MapWork* work);
msp_status online_solve(Basis& B, const double* phi, int batch, double tol, int max_iter, double* u, double* c_out,
                        int* iters_host, cudaStream_t s);
msp_status build_online_factor(Basis& B, const std::vector<int>& row_ptr, const std::vector<int>& row_slot,
                               cudaStream_t s);
// u = sum_m chi_m Q_m c_m for B data sets of coefficients c ([coefficient][B]);
// e is scratch of n_slots x B doubles
void reconstruct_coefficients(const Basis& Bs, const double* c, int B, double* e, const double* phi, int n4, double* u,
                              cudaStream_t s);
// overlapping Schwarz variant of the online step (online_ras.cu)
msp_status ras_setup(Basis& Bs, const Medium& full, bool coarse, cudaStream_t s);
msp_status ras_solve(Basis& Bs, const double* phi, int batch, double tol, int max_iter, double* u, double* c_out,
                     int* iters_host, cudaStream_t s);
msp_status apply_online_factor(Basis& B, const double* s_in, double* z_out, int Bsz, cudaStream_t s);

int num_sms();
// Poll bound of the device-side grid barriers (msp_set_wait_limit).
long long wait_limit();
// Extraction phase timing on (msp_set_extract_timing); records an event on s
// into marks when it is on and marks is not null.
bool extract_timing();
msp_status phase_mark(std::vector<cudaEvent_t>* marks, cudaStream_t s);

// Count of kernel launches issued by the library (for launch accounting).
void count_launches(long long n);

}  // namespace msp

struct msp_medium_s {
    msp::Medium M;
};
struct msp_basis_s {
    msp::Basis B;
};
