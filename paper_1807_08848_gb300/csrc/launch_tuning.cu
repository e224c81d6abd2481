// Launch configuration of the offline local solves: split or fused launch, rows
// instance of the tile kernel, the autotuner that picks them, and replay of the
// launches through a CUDA graph.
//
// Autotuner: every CG candidate (split / fused x each rows instance the eligible
// tiles fit) runs the same strided subset of the medium's items (both the tiles
// that fit on chip and the rest), once to warm up and once timed with CUDA events.
// In mixed precision the direct solver is a candidate too when the medium fits it:
// its factorisation serves every column of a patch, so it runs the whole medium,
// once untimed (which also factorises; the factor is kept) and once timed, its time
// scaled to the probe's share of the columns.  The fastest per column is kept for
// msp_sample_patches.  The CG probe runs write the snapshot columns of the subset
// with exactly the values a full run writes (every item's arithmetic is independent
// of the launch); the direct candidate writes every column with its own values, which
// the next msp_sample_patches overwrites.
#include "internal.h"

#include <algorithm>
#include <vector>

namespace msp {

namespace {

int needed_rows(const Medium& M, int precision) { return std::max(4, tile_launch_rows(M.patches, precision)); }

msp_status upload_items(DevBuf<int2>& d, const std::vector<int2>& h, cudaStream_t s) {
    MSP_TRY(d.alloc(h.size(), s));
    MSP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(int2) * h.size(), cudaMemcpyHostToDevice, s));
    MSP_CUDA(cudaStreamSynchronize(s));   // h is a local of the caller
    return MSP_OK;
}

}  // namespace

msp_status sample_launch(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s) {
    const int pi = cfg.precision == MSP_MIXED ? 1 : 0;
    if (!M.use_graph) return launch_local_solves(M, cfg, s);
    const double key[6] = {(double)cfg.precision, (double)cfg.seed, cfg.tol, (double)cfg.max_iter,
                           (double)M.launch_mode[pi], (double)M.launch_rows[pi]};
    bool same = M.graph[pi] != nullptr;
    for (int i = 0; i < 6 && same; ++i) same = M.graph_key[pi][i] == key[i];
    if (same) {
        MSP_CUDA(cudaGraphLaunch(M.graph[pi], s));
        count_launches(M.graph_launches[pi]);
        return MSP_OK;
    }
    // first call of this configuration: a direct run (it sizes and allocates the
    // scratch), then the capture of the same launches for the next calls
    MSP_TRY(launch_local_solves(M, cfg, s));
    if (M.graph[pi]) {
        cudaGraphExecDestroy(M.graph[pi]);
        M.graph[pi] = nullptr;
    }
    // captured on a private stream (the caller's may be the legacy default stream,
    // which cannot capture); nothing runs during capture, the graph runs on s
    if (!M.capture_stream) MSP_CUDA(cudaStreamCreateWithFlags(&M.capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    MSP_CUDA(cudaStreamBeginCapture(M.capture_stream, cudaStreamCaptureModeThreadLocal));
    const long long before = msp_kernel_launches();
    const msp_status st = launch_local_solves(M, cfg, M.capture_stream);
    cudaError_t e = cudaStreamEndCapture(M.capture_stream, &g);
    M.graph_launches[pi] = msp_kernel_launches() - before;
    count_launches(-M.graph_launches[pi]);   // captured, not run
    if (st != MSP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        set_error(std::string("local solves: graph capture: ") + cudaGetErrorString(e));
        return MSP_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&M.graph[pi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        M.graph[pi] = nullptr;
        set_error(std::string("local solves: graph instantiation: ") + cudaGetErrorString(e));
        return MSP_ERR_CUDA;
    }
    for (int i = 0; i < 6; ++i) M.graph_key[pi][i] = key[i];
    return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" msp_status msp_medium_set_launch(msp_medium m, int precision, int mode, int rows) {
    clear_error();
    MSP_CHECK_ARG(m, "msp_medium_set_launch: NULL medium");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_medium_set_launch: unknown precision");
    MSP_CHECK_ARG(mode == MSP_LAUNCH_SPLIT || mode == MSP_LAUNCH_FUSED || mode == MSP_LAUNCH_DIRECT,
                  "msp_medium_set_launch: unknown mode");
    if (mode == MSP_LAUNCH_DIRECT) {
        MSP_CHECK_ARG(precision == MSP_MIXED, "msp_medium_set_launch: the direct solver is a mixed-precision launch");
        MSP_CHECK_ARG(direct_fits(m->M), "msp_medium_set_launch: the direct solver takes buffered patches of at most "
                                         "160 interior nodes per row");
        m->M.launch_mode[1] = MSP_LAUNCH_DIRECT;
        m->M.launch_rows[1] = 0;
        return MSP_OK;
    }
    MSP_CHECK_ARG(rows == 0 || rows == 4 || rows == 8 || rows == 12, "msp_medium_set_launch: rows must be 0, 4, 8 or 12");
    Medium& M = m->M;
    const int pi = precision == MSP_MIXED ? 1 : 0;
    if (rows != 0 && rows < needed_rows(M, precision)) {
        set_error("msp_medium_set_launch: the eligible tiles need more rows per segment");
        return MSP_ERR_INVALID_ARG;
    }
    M.launch_mode[pi] = mode;
    M.launch_rows[pi] = rows;
    return MSP_OK;
}

extern "C" msp_status msp_medium_set_graph(msp_medium m, int enable) {
    clear_error();
    MSP_CHECK_ARG(m, "msp_medium_set_graph: NULL medium");
    m->M.use_graph = enable != 0;
    return MSP_OK;
}

extern "C" msp_status msp_medium_autotune(msp_medium m, int precision, uint64_t seed, double tol, int max_iter,
                                          int max_probe_items, void* stream, msp_tune_report* out) {
    clear_error();
    MSP_CHECK_ARG(m && out, "msp_medium_autotune: NULL argument");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_medium_autotune: unknown precision");
    MSP_CHECK_ARG(tol > 0 && tol < 1 && max_iter >= 1, "msp_medium_autotune: tol in (0, 1), max_iter >= 1");
    MSP_CHECK_ARG(max_probe_items >= 1, "msp_medium_autotune: max_probe_items must be >= 1");
    Medium& M = m->M;
    cudaStream_t s = (cudaStream_t)stream;
    const int pi = precision == MSP_MIXED ? 1 : 0;
    const std::vector<int2>& all = M.items_prec_host[pi];
    const int n_tile = M.n_tile_items[pi], n_rest = M.n_items - n_tile;
    // the probe subset: an even stride through both groups, at most max_probe_items in all
    const int stride = std::max(1, (M.n_items + max_probe_items - 1) / max_probe_items);
    std::vector<int2> sub_tile, sub_rest;
    for (int i = 0; i < n_tile; i += stride) sub_tile.push_back(all[i]);
    for (int i = 0; i < n_rest; i += stride) sub_rest.push_back(all[n_tile + i]);
    DevBuf<int2> d_tile, d_rest;
    if (!sub_tile.empty()) MSP_TRY(upload_items(d_tile, sub_tile, s));
    if (!sub_rest.empty()) MSP_TRY(upload_items(d_rest, sub_rest, s));
    LocalSolveCfg cfg{};
    cfg.precision = precision;
    cfg.tol = tol;
    cfg.inner_tol = 1e-4;
    cfg.max_iter = max_iter;
    cfg.max_ref = 12;
    cfg.seed = seed;
    msp_tune_report rep{};
    rep.probe_items = (int)(sub_tile.size() + sub_rest.size());
    cudaEvent_t e0, e1;
    MSP_CUDA(cudaEventCreate(&e0));
    MSP_CUDA(cudaEventCreate(&e1));
    float best = -1.f;
    const int r0 = needed_rows(M, precision);
    for (int mode = 0; mode < 2; ++mode) {
        for (int rows : {4, 8, 12}) {
            if (rows < r0) continue;
            if (mode == 0 && sub_tile.empty() && rows != r0) continue;
            LaunchItems li{d_tile.p, (int)sub_tile.size(), d_rest.p, (int)sub_rest.size(), mode, rows};
            float ms = -1.f;
            msp_status st = launch_local_solves(M, cfg, s, &li);   // warm-up
            if (st == MSP_OK) {
                MSP_CUDA(cudaEventRecord(e0, s));
                st = launch_local_solves(M, cfg, s, &li);
                MSP_CUDA(cudaEventRecord(e1, s));
                MSP_CUDA(cudaEventSynchronize(e1));
                if (st == MSP_OK) MSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            }
            if (st != MSP_OK && st != MSP_ERR_INVALID_ARG) {   // a rows instance that does not fit is skipped
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            if (rep.n_candidates < MSP_TUNE_MAX_CANDIDATES) {
                msp_tune_candidate& c = rep.candidates[rep.n_candidates++];
                c.mode = mode;
                c.rows = rows;
                c.ms = st == MSP_OK ? ms : -1.f;
            }
            if (st == MSP_OK && (best < 0 || ms < best)) {
                best = ms;
                rep.best_mode = mode;
                rep.best_rows = rows;
                rep.best_ms = ms;
            }
            clear_error();
        }
    }
    if (precision == MSP_MIXED && direct_fits(M) && M.n_items > 0) {
        const int saved = M.launch_mode[pi];
        M.launch_mode[pi] = MSP_LAUNCH_DIRECT;
        float ms = -1.f;
        msp_status st = launch_local_solves(M, cfg, s);   // warm-up, factorisation
        if (st == MSP_OK) {
            MSP_CUDA(cudaEventRecord(e0, s));
            st = launch_local_solves(M, cfg, s);
            MSP_CUDA(cudaEventRecord(e1, s));
            MSP_CUDA(cudaEventSynchronize(e1));
            if (st == MSP_OK) {
                MSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                ms *= (float)rep.probe_items / (float)M.n_items;
            }
        }
        M.launch_mode[pi] = saved;
        if (st != MSP_OK && st != MSP_ERR_INVALID_ARG) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        if (rep.n_candidates < MSP_TUNE_MAX_CANDIDATES) {
            msp_tune_candidate& c = rep.candidates[rep.n_candidates++];
            c.mode = MSP_LAUNCH_DIRECT;
            c.rows = 0;
            c.ms = st == MSP_OK ? ms : -1.f;
        }
        if (st == MSP_OK && (best < 0 || ms < best)) {
            best = ms;
            rep.best_mode = MSP_LAUNCH_DIRECT;
            rep.best_rows = 0;
            rep.best_ms = ms;
        }
        clear_error();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        set_error("msp_medium_autotune: no launch configuration ran");
        return MSP_ERR_CUDA;
    }
    M.launch_mode[pi] = rep.best_mode;
    M.launch_rows[pi] = rep.best_rows;
    M.tuned[pi] = true;
    *out = rep;
    return MSP_OK;
}
