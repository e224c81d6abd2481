// Offline local solves (Algorithm alg:summary, RanLocalSolu; Eq. elliptic_random):
// ring data of the buffered patch, Jacobi-preconditioned CG for the 5-point
// operator, restriction to K_m.
//
// Launch of the local solves: the tile-resident kernel (local_solve_tile.cu) for
// the tiles that fit on chip and local_solve_global<T> (any tile size; each CTA
// owns a slot of global scratch, x in FP64, the CG vectors in T; the per-item
// code is in global_path.cuh) for the rest, as two launches, or everything in one
// persistent launch of the fused tile kernel.  T = double is the plain FP64 path;
// T = float runs FP32 CG inside FP64 iterative refinement.
#include "internal.h"
#include "device_util.cuh"
#include "global_path.cuh"

#include <algorithm>
#include <cmath>

namespace msp {

namespace {

using namespace gpath;

template <class T>
__global__ void __launch_bounds__(512) local_solve_global(SolveArgs A) {
    __shared__ double red64[128];
    __shared__ T redT[128];
    char* slot = reinterpret_cast<char*>(A.scratch) + (long long)blockIdx.x * A.slot_bytes;
    for (int item = blockIdx.x; item < A.n_items; item += gridDim.x) global_item<T>(A, item, slot, red64, redT);
}

__global__ void ring_samples_kernel(SolveArgs A, int m, double* dst) {
    // one CTA per column: write the ring data in ring order
    const PatchDev P = A.patches[m];
    const int col = blockIdx.x;
    if (col >= P.cols) return;
    double* o = dst + (long long)col * P.n_ring;
    if (col < P.samples) {
        const int npairs = (P.n_ring + 1) >> 1;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            const double2 z = gaussian_pair(A.seed, (uint32_t)q, (uint32_t)col, (uint32_t)m, kTagElliptic);
            o[2 * q] = z.x;
            if (2 * q + 1 < P.n_ring) o[2 * q + 1] = z.y;
        }
    } else {
        const int t0 = A.bpos[P.bpos_offset + (col - P.samples)];
        for (int t = threadIdx.x; t < P.n_ring; t += blockDim.x) o[t] = (t == t0) ? 1.0 : 0.0;
    }
}

SolveArgs base_args(Medium& M) {
    SolveArgs A{};
    A.N = M.N;
    A.aE = M.aE.p;
    A.aN = M.aN.p;
    A.aE32 = M.aE32.p;
    A.aN32 = M.aN32.p;
    A.patches = M.patches_dev.p;
    A.bpos = M.bpos_dev.p;
    A.items = M.items.p;
    A.n_items = M.n_items;
    A.snaps = M.snaps.p;
    A.stats = M.item_stats.p;
    return A;
}

}  // namespace

msp_status launch_local_solves(Medium& M, const LocalSolveCfg& cfg, cudaStream_t s, const LaunchItems* li) {
    const bool mixed = cfg.precision == MSP_MIXED;
    const int pi = mixed ? 1 : 0;
    if (!li && M.launch_mode[pi] == MSP_LAUNCH_DIRECT) return launch_local_solves_direct(M, cfg, s);
    const int n_tile = li ? li->n_tile : M.n_tile_items[pi];
    const int2* items = li ? li->tile : M.items_prec[pi].p;
    const int n_rest = li ? li->n_rest : M.n_items - n_tile;
    const int2* rest = li ? li->rest : M.items_prec[pi].p + n_tile;
    const bool fused = (li ? li->mode : M.launch_mode[pi]) == 1;
    const int rows = li ? li->rows : M.launch_rows[pi];
    // items whose tile fits on chip: the tile-resident kernel
    if (!fused) MSP_TRY(launch_local_solves_tile(M, cfg, items, n_tile, M.counter.p, s, nullptr, rows));
    if (n_rest == 0 && !fused) return MSP_OK;
    // the rest: the global-scratch path (its own kernel, or inside the fused launch)
    SolveArgs A = base_args(M);
    A.items = rest;
    A.n_items = n_rest;
    A.stats = M.item_stats.p + 3LL * n_tile;
    A.seed = cfg.seed;
    A.tol = cfg.tol;
    A.inner_tol = cfg.inner_tol;
    A.max_iter = cfg.max_iter;
    A.max_ref = cfg.max_ref;
    const long long tsz = mixed ? 4 : 8;
    long long slot = (long long)M.max_tile_nodes * (8 + 5 * tsz);
    slot = (slot + 255) / 256 * 256;
    if (fused) {
        A.slot_bytes = slot;
        return launch_local_solves_tile(M, cfg, items, n_tile, M.counter.p, s, &A, rows);
    }
    const int threads = 512;
    const int per_sm = 2;
    const int grid = std::max(1, std::min(n_rest, num_sms() * per_sm));
    const size_t need = (size_t)slot * grid / sizeof(double) + 1;
    if (M.scratch_global.n < need) MSP_TRY(M.scratch_global.alloc(need, s));
    A.scratch = M.scratch_global.p;
    A.slot_bytes = slot;
    if (mixed)
        local_solve_global<float><<<grid, threads, 0, s>>>(A);
    else
        local_solve_global<double><<<grid, threads, 0, s>>>(A);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

msp_status launch_ring_samples(Medium& M, int patch, uint64_t seed, double* dst, cudaStream_t s) {
    SolveArgs A = base_args(M);
    A.seed = seed;
    ring_samples_kernel<<<M.patches[patch].cols, 128, 0, s>>>(A, patch, dst);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace msp
