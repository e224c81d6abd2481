// C ABI: errors, medium construction and the offline sampling stage.
#include "internal.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>


namespace msp {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Poll bound of the device-side grid barriers (process-wide, read at each launch).
constexpr long long kDefaultWaitLimit = 1LL << 24;
static std::atomic<long long> g_wait_limit{kDefaultWaitLimit};
long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

static std::atomic<int> g_extract_timing{0};
bool extract_timing() { return g_extract_timing.load(std::memory_order_relaxed) != 0; }
msp_status phase_mark(std::vector<cudaEvent_t>* marks, cudaStream_t s) {
    if (!marks || !extract_timing()) return MSP_OK;
    cudaEvent_t e;
    MSP_CUDA(cudaEventCreate(&e));
    marks->push_back(e);
    MSP_CUDA(cudaEventRecord(e, s));
    return MSP_OK;
}

// Engine of the FP64 products of the extraction and the online factorisation.
static std::atomic<int> g_gemm_engine{0};
int fp64_gemm_engine() { return g_gemm_engine.load(std::memory_order_relaxed); }
static std::atomic<int> g_svd_mode{MSP_SVD_QR_PRECONDITIONED};
bool svd_mixed() { return g_svd_mode.load(std::memory_order_relaxed) == MSP_SVD_FP32_PRECONDITIONED; }
bool svd_qr() { return g_svd_mode.load(std::memory_order_relaxed) == MSP_SVD_QR_PRECONDITIONED; }

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

msp_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error(std::string(what) + " failed: " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")");
    return MSP_ERR_CUDA;
}

int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
    return n;
}

static msp_status need_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        set_error(std::string("no usable CUDA device: ") + (e == cudaSuccess ? "device count is 0" : cudaGetErrorString(e)));
        return MSP_ERR_CUDA;
    }
    return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" const char* msp_last_error(void) { return g_err.c_str(); }
extern "C" const char* msp_version(void) { return "msp 0.1 (sm_103a)"; }
extern "C" int64_t msp_kernel_launches(void) { return g_launches.load(); }

extern "C" msp_status msp_set_svd_mode(int mode) {
    clear_error();
    MSP_CHECK_ARG(mode == MSP_SVD_FP64 || mode == MSP_SVD_FP32_PRECONDITIONED || mode == MSP_SVD_QR_PRECONDITIONED,
                  "msp_set_svd_mode: unknown mode");
    g_svd_mode.store(mode, std::memory_order_relaxed);
    return MSP_OK;
}

extern "C" msp_status msp_set_gemm_engine(int engine) {
    clear_error();
    MSP_CHECK_ARG(engine == MSP_GEMM_TENSOR_CORES || engine == MSP_GEMM_CUDA_CORES, "msp_set_gemm_engine: unknown engine");
    g_gemm_engine.store(engine, std::memory_order_relaxed);
    return MSP_OK;
}

extern "C" msp_status msp_set_extract_timing(int enable) {
    clear_error();
    g_extract_timing.store(enable != 0 ? 1 : 0, std::memory_order_relaxed);
    return MSP_OK;
}

extern "C" msp_status msp_set_wait_limit(int64_t polls) {
    clear_error();
    MSP_CHECK_ARG(polls >= 0, "msp_set_wait_limit: polls must be >= 0 (0 restores the default)");
    g_wait_limit.store(polls == 0 ? kDefaultWaitLimit : (long long)polls, std::memory_order_relaxed);
    return MSP_OK;
}

// det: DetLocalSolu (Algorithm alg:summary) -- every patch solves one delta
// datum per ring node of its buffered patch and no Gaussian data.
static msp_status build_medium(const msp_medium_desc* d, const msp_patch_desc* pd, void* stream, msp_medium* out,
                               bool det) {
    clear_error();
    MSP_CHECK_ARG(d && pd && out, "msp_build_medium: NULL argument");
    *out = nullptr;
    const int N = d->n_cells;
    MSP_CHECK_ARG(N >= 2 && N <= (1 << 15), "msp_build_medium: n_cells out of range [2, 32768]");
    MSP_CHECK_ARG(d->kind >= 0 && d->kind <= MSP_MEDIUM_USER, "msp_build_medium: unknown medium kind");
    if (d->kind == MSP_MEDIUM_USER)
        MSP_CHECK_ARG(d->user_aE_host && d->user_aN_host, "msp_build_medium: user medium needs aE and aN");
    if (d->kind == MSP_MEDIUM_LOGNORMAL)
        MSP_CHECK_ARG(d->n_modes >= 0 && (d->n_modes == 0 || d->modes_host), "msp_build_medium: bad mode table");
    if (d->kind == MSP_MEDIUM_CHANNELS)
        MSP_CHECK_ARG(d->n_channels >= 0 && (d->n_channels == 0 || d->channels_host), "msp_build_medium: bad channel table");
    if (d->kind == MSP_MEDIUM_PERIODIC_SIN || d->kind == MSP_MEDIUM_HOU_WU)
        MSP_CHECK_ARG(d->eps > 0, "msp_build_medium: eps must be positive");
    const int mx = pd->nx_patches, my = pd->ny_patches;
    MSP_CHECK_ARG(mx >= 1 && my >= 1 && pd->x_breaks_host && pd->y_breaks_host && pd->buffers_host &&
                      (det || pd->samples_host),
                  "msp_build_medium: bad patch description");
    MSP_TRY(need_device());

    auto* h = new msp_medium_s();
    Medium& M = h->M;
    M.N = N;
    M.mx = mx;
    M.my = my;
    M.xb.assign(pd->x_breaks_host, pd->x_breaks_host + mx + 1);
    M.yb.assign(pd->y_breaks_host, pd->y_breaks_host + my + 1);
    auto bad_breaks = [N](const std::vector<int>& b) {
        if (b.front() != 0 || b.back() != N) return true;
        for (size_t i = 1; i < b.size(); ++i)
            if (b[i] <= b[i - 1]) return true;
        return false;
    };
    if (bad_breaks(M.xb) || bad_breaks(M.yb)) {
        delete h;
        set_error("msp_build_medium: patch breaks must increase strictly from 0 to n_cells");
        return MSP_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    long long off = 0;
    for (int q = 0; q < my; ++q) {
        for (int p = 0; p < mx; ++p) {
            const int m = p + q * mx;
            const int b = pd->buffers_host[m], S = det ? 0 : pd->samples_host[m];
            if (b < 0 || (!det && S < 1)) {
                delete h;
                set_error("msp_build_medium: buffers must be >= 0 and samples >= 1");
                return MSP_ERR_INVALID_ARG;
            }
            PatchDev P{};
            P.x0 = M.xb[p]; P.x1 = M.xb[p + 1]; P.y0 = M.yb[q]; P.y1 = M.yb[q + 1];
            P.X0 = std::max(0, P.x0 - b); P.X1 = std::min(N, P.x1 + b);
            P.Y0 = std::max(0, P.y0 - b); P.Y1 = std::min(N, P.y1 + b);
            P.n_k = (P.x1 - P.x0 + 1) * (P.y1 - P.y0 + 1);
            P.n_ring = 2 * (P.X1 - P.X0) + 2 * (P.Y1 - P.Y0);
            P.samples = S;
            P.bpos_offset = (int)M.bpos.size();
            for (int t = 0; t < P.n_ring; ++t) {
                int i, j;
                ring_node(P.X0, P.X1, P.Y0, P.Y1, t, i, j);
                if (det || i == 0 || i == N || j == 0 || j == N) M.bpos.push_back(t);
            }
            P.n_b = (int)M.bpos.size() - P.bpos_offset;
            P.cols = S + P.n_b;
            P.snap_offset = off;
            off += (long long)P.n_k * P.cols;
            M.max_tile_nodes = std::max(M.max_tile_nodes, (P.X1 - P.X0 + 1) * (P.Y1 - P.Y0 + 1));
            M.max_cols = std::max(M.max_cols, P.cols);
            M.patches.push_back(P);
        }
    }
    M.snap_elems = off;
    // work items: every (patch, column), largest tiles first
    std::vector<int2> items;
    for (int m = 0; m < mx * my; ++m)
        for (int c = 0; c < M.patches[m].cols; ++c) items.push_back(make_int2(m, c));
    std::stable_sort(items.begin(), items.end(), [&](const int2& a, const int2& b) {
        const PatchDev &A = M.patches[a.x], &B = M.patches[b.x];
        return (A.X1 - A.X0) * (A.Y1 - A.Y0) > (B.X1 - B.X0) * (B.Y1 - B.Y0);
    });
    M.n_items = (int)items.size();
    M.items_host = items;
    for (int pi = 0; pi < 2; ++pi) {   // per precision: tile-eligible items first
        std::vector<int2> a, b;
        const int R = tile_launch_rows(M.patches, pi);
        for (const int2& it : items) (tile_kernel_fits(M.patches[it.x], pi, R) ? a : b).push_back(it);
        M.n_tile_items[pi] = (int)a.size();
        a.insert(a.end(), b.begin(), b.end());
        M.items_prec_host[pi] = a;
    }
    msp_status st;
#define BAIL(x)                       \
    do {                              \
        st = (x);                     \
        if (st != MSP_OK) {           \
            delete h;                 \
            return st;                \
        }                             \
    } while (0)
    cudaError_t ce;
#define BAILC(x)                                                      \
    do {                                                              \
        ce = (x);                                                     \
        if (ce != cudaSuccess) {                                      \
            delete h;                                                 \
            return cuda_fail(ce, #x, __FILE__, __LINE__);             \
        }                                                             \
    } while (0)
    BAILC(cudaGetDevice(&M.device));
    BAIL(M.patches_dev.alloc(M.patches.size(), s));
    BAIL(M.bpos_dev.alloc(std::max<size_t>(1, M.bpos.size()), s));
    BAIL(M.items.alloc(items.size(), s));
    BAIL(M.item_stats.alloc(3 * items.size(), s));
    BAIL(M.counter.alloc(1, s));
    for (int pi = 0; pi < 2; ++pi) {
        BAIL(M.items_prec[pi].alloc(items.size(), s));
        BAILC(cudaMemcpyAsync(M.items_prec[pi].p, M.items_prec_host[pi].data(), sizeof(int2) * items.size(),
                              cudaMemcpyHostToDevice, s));
    }
    BAIL(M.snaps.alloc((size_t)M.snap_elems, s));
    BAILC(cudaMemcpyAsync(M.patches_dev.p, M.patches.data(), sizeof(PatchDev) * M.patches.size(), cudaMemcpyHostToDevice, s));
    if (!M.bpos.empty())
        BAILC(cudaMemcpyAsync(M.bpos_dev.p, M.bpos.data(), sizeof(int) * M.bpos.size(), cudaMemcpyHostToDevice, s));
    BAILC(cudaMemcpyAsync(M.items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, s));
    BAIL(launch_medium_coefficients(M, *d, s));   // synchronises: host vectors above may go
#undef BAIL
#undef BAILC
    *out = h;
    return MSP_OK;
}

extern "C" msp_status msp_build_medium(const msp_medium_desc* d, const msp_patch_desc* pd, void* stream,
                                       msp_medium* out) {
    return build_medium(d, pd, stream, out, false);
}

extern "C" msp_status msp_build_medium_full(const msp_medium_desc* d, const msp_patch_desc* pd, void* stream,
                                            msp_medium* out) {
    return build_medium(d, pd, stream, out, true);
}

extern "C" void msp_medium_destroy(msp_medium m) {
    if (!m) return;
    for (auto& g : m->M.graph)
        if (g) cudaGraphExecDestroy(g);
    if (m->M.capture_stream) cudaStreamDestroy(m->M.capture_stream);
    delete m;
}

extern "C" msp_status msp_medium_counts(msp_medium m, int* n_patches, int64_t* snapshot_elems, int* n_cells) {
    clear_error();
    MSP_CHECK_ARG(m, "msp_medium_counts: NULL medium");
    if (n_patches) *n_patches = (int)m->M.patches.size();
    if (snapshot_elems) *snapshot_elems = m->M.snap_elems;
    if (n_cells) *n_cells = m->M.N;
    return MSP_OK;
}

extern "C" msp_status msp_medium_patch(msp_medium m, int patch, msp_patch_info* out) {
    clear_error();
    MSP_CHECK_ARG(m && out, "msp_medium_patch: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)m->M.patches.size(), "msp_medium_patch: patch out of range");
    const PatchDev& P = m->M.patches[patch];
    out->x0 = P.x0; out->x1 = P.x1; out->y0 = P.y0; out->y1 = P.y1;
    out->X0 = P.X0; out->X1 = P.X1; out->Y0 = P.Y0; out->Y1 = P.Y1;
    out->n_k = P.n_k; out->n_ring = P.n_ring; out->samples = P.samples; out->n_b = P.n_b; out->cols = P.cols;
    out->snap_offset = P.snap_offset;
    return MSP_OK;
}

extern "C" msp_status msp_get_coefficients(msp_medium m, double* aE_dev, double* aN_dev, void* stream) {
    clear_error();
    MSP_CHECK_ARG(m && aE_dev && aN_dev, "msp_get_coefficients: NULL argument");
    const size_t n = (size_t)(m->M.N + 1) * m->M.N;
    MSP_CUDA(cudaMemcpyAsync(aE_dev, m->M.aE.p, n * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    MSP_CUDA(cudaMemcpyAsync(aN_dev, m->M.aN.p, n * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MSP_OK;
}

extern "C" msp_status msp_sample_patches(msp_medium m, uint64_t seed, int precision, double tol, int max_iter,
                                         void* stream, msp_solve_stats* stats) {
    clear_error();
    MSP_CHECK_ARG(m, "msp_sample_patches: NULL medium");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_sample_patches: unknown precision");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_sample_patches: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_sample_patches: max_iter must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    LocalSolveCfg cfg{};
    cfg.precision = precision;
    cfg.tol = tol;
    cfg.inner_tol = 1e-4;
    cfg.max_iter = max_iter;
    cfg.max_ref = 12;
    cfg.seed = seed;
    MSP_TRY(sample_launch(m->M, cfg, s));
    m->M.sampled = true;
    if (stats) {
        std::vector<int> st(3 * (size_t)m->M.n_items);
        MSP_CUDA(cudaMemcpyAsync(st.data(), m->M.item_stats.p, st.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        MSP_CUDA(cudaStreamSynchronize(s));
        msp_solve_stats r{};
        r.n_solves = m->M.n_items;
        const std::vector<int2>& order = m->M.items_prec_host[precision == MSP_MIXED ? 1 : 0];
        for (int i = 0; i < m->M.n_items; ++i) {
            const PatchDev& P = m->M.patches[order[i].x];
            r.unknown_iters += (long long)st[3 * i] * (P.X1 - P.X0 - 1) * (P.Y1 - P.Y0 - 1);
            r.total_iters += st[3 * i];
            r.max_iters = std::max(r.max_iters, st[3 * i]);
            r.max_refinements = std::max(r.max_refinements, st[3 * i + 1]);
            r.n_not_converged += st[3 * i + 2];
        }
        *stats = r;
        if (r.n_not_converged) {
            set_error("msp_sample_patches: " + std::to_string(r.n_not_converged) + " local solves did not converge");
            return MSP_ERR_NOT_CONVERGED;
        }
    }
    return MSP_OK;
}

extern "C" msp_status msp_sample_patch_list(msp_medium m, const int* patches_host, int n_list, uint64_t seed,
                                            int precision, double tol, int max_iter, void* stream,
                                            msp_solve_stats* stats) {
    clear_error();
    MSP_CHECK_ARG(m && (patches_host || n_list == 0), "msp_sample_patch_list: NULL argument");
    MSP_CHECK_ARG(n_list >= 0, "msp_sample_patch_list: negative patch count");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_sample_patch_list: unknown precision");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_sample_patch_list: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_sample_patch_list: max_iter must be >= 1");
    Medium& M = m->M;
    const int np = (int)M.patches.size();
    std::vector<char> want(np, 0);
    for (int i = 0; i < n_list; ++i) {
        MSP_CHECK_ARG(patches_host[i] >= 0 && patches_host[i] < np, "msp_sample_patch_list: patch out of range");
        want[patches_host[i]] = 1;
    }
    const int pi = precision == MSP_MIXED ? 1 : 0;
    // the listed patches' items, in the medium's order: tile-eligible ones first
    const std::vector<int2>& all = M.items_prec_host[pi];
    std::vector<int2> sub;
    int n_tile = 0;
    for (int i = 0; i < M.n_items; ++i) {
        if (!want[all[i].x]) continue;
        sub.push_back(all[i]);
        if (i < M.n_tile_items[pi]) ++n_tile;
    }
    cudaStream_t s = (cudaStream_t)stream;
    M.sampled = true;
    if (sub.empty()) {
        if (stats) *stats = msp_solve_stats{};
        return MSP_OK;
    }
    DevBuf<int2> d_sub;
    MSP_TRY(d_sub.alloc(sub.size(), s));
    MSP_CUDA(cudaMemcpyAsync(d_sub.p, sub.data(), sizeof(int2) * sub.size(), cudaMemcpyHostToDevice, s));
    LocalSolveCfg cfg{};
    cfg.precision = precision;
    cfg.tol = tol;
    cfg.inner_tol = 1e-4;
    cfg.max_iter = max_iter;
    cfg.max_ref = 12;
    cfg.seed = seed;
    // the CG launches (a direct-solver setting of the medium applies to whole media only)
    const int mode = M.launch_mode[pi] == MSP_LAUNCH_FUSED ? MSP_LAUNCH_FUSED : MSP_LAUNCH_SPLIT;
    LaunchItems li{d_sub.p, n_tile, d_sub.p + n_tile, (int)sub.size() - n_tile, mode, M.launch_rows[pi]};
    MSP_TRY(launch_local_solves(M, cfg, s, &li));
    // statistics sit at the subset's positions; read them before d_sub goes
    std::vector<int> st(3 * sub.size());
    MSP_CUDA(cudaMemcpyAsync(st.data(), M.item_stats.p, st.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    msp_solve_stats r{};
    r.n_solves = (long long)sub.size();
    for (size_t i = 0; i < sub.size(); ++i) {
        const PatchDev& P = M.patches[sub[i].x];
        r.unknown_iters += (long long)st[3 * i] * (P.X1 - P.X0 - 1) * (P.Y1 - P.Y0 - 1);
        r.total_iters += st[3 * i];
        r.max_iters = std::max(r.max_iters, st[3 * i]);
        r.max_refinements = std::max(r.max_refinements, st[3 * i + 1]);
        r.n_not_converged += st[3 * i + 2];
    }
    if (stats) *stats = r;
    if (r.n_not_converged) {
        set_error("msp_sample_patch_list: " + std::to_string(r.n_not_converged) + " local solves did not converge");
        return MSP_ERR_NOT_CONVERGED;
    }
    return MSP_OK;
}

extern "C" msp_status msp_set_snapshots(msp_medium m, int patch, const double* src, void* stream) {
    clear_error();
    MSP_CHECK_ARG(m && src, "msp_set_snapshots: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)m->M.patches.size(), "msp_set_snapshots: patch out of range");
    const PatchDev& P = m->M.patches[patch];
    MSP_CUDA(cudaMemcpyAsync(m->M.snaps.p + P.snap_offset, src, sizeof(double) * (size_t)P.n_k * P.cols,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    m->M.sampled = true;
    return MSP_OK;
}

extern "C" msp_status msp_get_snapshots(msp_medium m, int patch, double* dst, void* stream) {
    clear_error();
    MSP_CHECK_ARG(m && dst, "msp_get_snapshots: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)m->M.patches.size(), "msp_get_snapshots: patch out of range");
    if (!m->M.sampled) { set_error("msp_get_snapshots: call msp_sample_patches first"); return MSP_ERR_STATE; }
    const PatchDev& P = m->M.patches[patch];
    MSP_CUDA(cudaMemcpyAsync(dst, m->M.snaps.p + P.snap_offset, sizeof(double) * (size_t)P.n_k * P.cols,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return MSP_OK;
}

extern "C" msp_status msp_get_samples(msp_medium m, int patch, uint64_t seed, double* dst, void* stream) {
    clear_error();
    MSP_CHECK_ARG(m && dst, "msp_get_samples: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)m->M.patches.size(), "msp_get_samples: patch out of range");
    return launch_ring_samples(m->M, patch, seed, dst, (cudaStream_t)stream);
}
