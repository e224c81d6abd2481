// Kinetic slab medium shared by the source-iteration and direct local solvers
// (Sec. 4): patch geometry, quadrature, the Henyey-Greenstein collision in
// quadrature form (Eq. HG) and the snapshot storage.
#pragma once
#include "internal.h"

namespace msp {

struct KPatchDev {
    int x0, x1, X0, X1, nn, n_k;
    long long snap_offset;
};

// Factors and work storage of the direct block-tridiagonal local solver: per patch
// and node the inverse W_i of the Schur complement (n_v x n_v, row-major) in the
// factor's precision; f (FP64) and y (factor precision) hold every (node, velocity,
// sample) of the current iterate, sample fastest.
struct KDirect {
    std::vector<long long> node_off;    // first node of each patch in the stacked arrays
    DevBuf<long long> d_node_off;
    long long n_nodes = 0;
    DevBuf<double> W64;
    DevBuf<float> W32;
    bool factored64 = false, factored32 = false;
    DevBuf<double> f;
    DevBuf<double> y64;
    DevBuf<float> y32;
};

struct KMedium {
    int N = 0, n_v = 0, M = 0, buffer = 0, S = 0;
    double eps = 0, g = 0;
    int solver = 0;                       // MSP_KINETIC_SOURCE_ITERATION or MSP_KINETIC_DIRECT
    std::vector<double> v, w;
    std::vector<double> Kw, sigma;        // Kw[l n_v + l'] = w_l' k(v_l, v_l'), sigma_l = sum_l' w_l' k(v_l', v_l)
    std::vector<KPatchDev> patches;
    DevBuf<double> d_v, d_w, d_Kw, d_sigma;
    DevBuf<KPatchDev> d_patches;
    DevBuf<double> snaps;
    long long snap_elems = 0;
    DevBuf<int> stats;    // per (patch, sample): iterations, flag
    bool sampled = false;
    KDirect D;
};

// Direct local solves of every (patch, sample): block LU of the upwind operator
// over the nodes of the buffered patch, factor in FP64 or FP32, FP64 residual
// refinement to tol; fills snaps and stats like the source iteration.
msp_status kinetic_direct_sample(KMedium& K, uint64_t seed, bool mixed, double tol, int max_iter, cudaStream_t s);

}  // namespace msp
