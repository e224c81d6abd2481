// Tile-resident local solves: one CTA solves one (patch, column) item with the
// whole CG state on chip (Algorithm alg:summary, LocalPDESolver on the buffered
// patch; Eq. elliptic_random for the ring data).
//
// CG runs on the symmetrically Jacobi-scaled operator  A~ = S A S,
// S = diag(a_ii)^(-1/2): A~ has a unit diagonal, so the Jacobi preconditioner is
// folded into the operator and the stencil reads four scaled face coefficients
// and no diagonal.  Solving A~ d~ = S r gives the correction d = S d~.
//
// Thread mapping: the interior nx x ny unknowns are cut into strips of 32
// columns; each warp takes one strip and a segment of RPS consecutive rows, so a
// thread owns one column segment.  The search direction p lives in registers and
// is mirrored in shared memory (zero halo) for the east/west neighbours and the
// segment ends; north/south neighbours inside the segment come from registers,
// and so does the south face (the previous row's north face).  Every tile array
// uses the compile-time row pitch kPitch, so the unrolled row loop addresses each
// array as one base register plus immediate offsets.
//
//   T = float (mixed path): FP32 scaled faces in shared memory; r, A p, d and p in
//     registers.  The tile is padded with zero faces to whole strips and segments,
//     so the CG loop has no per-node branches (padded nodes stay exactly zero).
//     Outer FP64 iterative refinement: r = b - A x from the FP64 iterate x and FP64
//     coefficients, FP32 CG on S r / |S r|, x += |S r| S d~.
//   T = double (plain FP64 path): p and A p in shared memory, r in registers,
//     scaled faces and d~ in a per-CTA slot of global scratch.
//
// Items (patch, column) come from a global work counter, largest tiles first.
#include "internal.h"
#include "device_util.cuh"
#include "global_path.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace msp {

namespace {

constexpr int kTileThreads = 768;
constexpr int kNumWarps = kTileThreads / 32;
constexpr int kMaxRows = 12;  // max rows per thread segment
constexpr int kPitch = 100;   // row pitch of every tile array: padded width + 2 <= kPitch

struct TileArgs {
    int N;
    const double* aE;
    const double* aN;
    const PatchDev* patches;
    const int* bpos;
    const int2* items;
    int n_items;
    int* counter;
    double* snaps;
    uint64_t seed;
    double tol, inner_tol;
    int max_iter, max_ref;
    double* scratch;          // per CTA slot, see slot layout below
    long long slot_doubles;
    int* stats;
    int one_patch_index;      // random stream index of the patch (one-patch variant)
    PatchDev one_patch;       // the patch of the one-patch variant, passed by value
    gpath::SolveArgs g;       // fused launch: the items that do not fit on chip (global-scratch path)
};

// Thread mapping of an nx x ny interior: strips of 32 columns, segments of rps rows.
struct Mapping {
    int nstrips, nseg, rps;
};

__host__ __device__ inline bool tile_mapping(int nx, int ny, Mapping& mp) {
    mp.nstrips = (nx + 31) / 32;
    if (nx < 1 || ny < 1 || 32 * mp.nstrips + 2 > kPitch || mp.nstrips > kNumWarps) return false;
    mp.nseg = kNumWarps / mp.nstrips;
    mp.rps = (ny + mp.nseg - 1) / mp.nseg;
    return mp.rps <= kMaxRows;
}

// per-CTA global slot (doubles, rows of kPitch):
//   x  : ny+2  FP64 iterate, tile node (c, rr) at rr*kPitch + c, ring data included
//   cE : ny    cE[j][c] = east face of interior column c-1 (c = 0..nx), unscaled
//   cN : ny+1  cN[j][c] = north face of interior row j-1, unscaled
//   sv : ny    S = diag^(-1/2) of the interior nodes
//   tE : ny    scaled east faces   (FP64 path)
//   tN : ny+1  scaled north faces  (FP64 path)
//   dd : ny    correction d~       (FP64 path)
__host__ __device__ constexpr long long slot_rows(int ny) { return 7LL * ny + 4; }

// shared memory, rows of kPitch elements, PR = padded rows
//   float : ps (PR+2) | tE PR | tN PR+1
//   double: ps (ny+2) | qs ny
__host__ __device__ inline size_t smem_bytes(bool f32, int ny, int PR) {
    return f32 ? sizeof(float) * (size_t)kPitch * (3 * (size_t)PR + 3)
               : sizeof(double) * (size_t)kPitch * (2 * (size_t)ny + 2);
}

template <class T>
__device__ __forceinline__ T block_sum1(T v, T* buf) {
    T a[1] = {v};
    block_sum<T, 1>(a, buf);
    return a[0];
}

// ONE_PATCH: every item is column `item` of the single patch A.one_patch whose
// random stream index is A.one_patch_index (the variant without allocations).
// FUSED: one persistent launch for every item of the medium: the work counter
// first hands out the A.g items (tiles beyond the on-chip limit, the largest and
// slowest, solved in the CTA's slot of global scratch), then the tile items.
template <class T, int RPS, bool ONE_PATCH = false, bool FUSED = false>
__global__ void __launch_bounds__(kTileThreads, 1) local_solve_tile(TileArgs A) {
    constexpr bool kF32 = sizeof(T) == 4;
    constexpr int PI = kPitch;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[2][32];
    __shared__ double red64[2][64];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* slot = A.scratch + (long long)blockIdx.x * A.slot_doubles;
    const int N = A.N;
    __shared__ T redTg[FUSED ? 128 : 1];
    __shared__ double red64g[FUSED ? 128 : 1];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.counter, 1);
        __syncthreads();
        int item = s_item;
        if constexpr (FUSED) {
            if (item < A.g.n_items) {   // ends with a block barrier, so s_item may be rewritten next
                gpath::global_item<T>(A.g, item, reinterpret_cast<char*>(A.g.scratch) + (long long)blockIdx.x * A.g.slot_bytes,
                                      red64g, redTg);
                continue;
            }
            item -= A.g.n_items;
        }
        if (item >= A.n_items) break;
        int m, col;
        if constexpr (ONE_PATCH) {
            m = A.one_patch_index;
            col = item;
        } else {
            const int2 itm = A.items[item];
            m = itm.x;
            col = itm.y;
        }
        const PatchDev P = ONE_PATCH ? A.one_patch : A.patches[m];
        const int W = P.X1 - P.X0 + 1, H = P.Y1 - P.Y0 + 1;
        const int nx = W - 2, ny = H - 2;
        Mapping mp;
        tile_mapping(nx, ny, mp);                   // eligibility checked on the host (rps <= RPS)
        const int PR = mp.nseg * RPS;               // padded rows
        const int PC = 32 * mp.nstrips;             // padded columns
        const int strip = warp % mp.nstrips, seg = warp / mp.nstrips;
        const int i = strip * 32 + lane;            // owned interior column (may be padding)
        const int j0 = seg * RPS;                   // first owned interior row
        const bool active = seg < mp.nseg;          // warp-uniform
        const int nrow = (active && i < nx) ? max(0, min(RPS, ny - j0)) : 0;   // real rows owned

        // ---- global slot views
        double* xg = slot;
        double* cE = xg + (long long)(ny + 2) * PI;
        double* cN = cE + (long long)ny * PI;
        double* sv = cN + (long long)(ny + 1) * PI;
        double* tE = sv + (long long)ny * PI;
        double* tN = tE + (long long)ny * PI;
        double* dd = tN + (long long)(ny + 1) * PI;
        // ---- shared views
        T* ps = reinterpret_cast<T*>(smem_raw);
        float *tEs = nullptr, *tNs = nullptr;
        double* qs = nullptr;
        if constexpr (kF32) {
            tEs = reinterpret_cast<float*>(ps) + (PR + 2) * PI;
            tNs = tEs + PR * PI;
        } else {
            qs = reinterpret_cast<double*>(ps) + (ny + 2) * PI;
        }
        // ---- stage unscaled FP64 faces, zero x and p
        for (int t = threadIdx.x; t < ny * (nx + 1); t += blockDim.x) {
            const int jj = t / (nx + 1), c = t - jj * (nx + 1);
            cE[jj * PI + c] = A.aE[(long long)(P.Y0 + 1 + jj) * N + (P.X0 + c)];
        }
        for (int t = threadIdx.x; t < (ny + 1) * nx; t += blockDim.x) {
            const int jj = t / nx, c = t - jj * nx;
            cN[jj * PI + c] = A.aN[(long long)(P.Y0 + jj) * (N + 1) + (P.X0 + 1 + c)];
        }
        {
            const int prow = kF32 ? PR + 2 : H, pcol_n = kF32 ? PC + 2 : W;
            for (int t = threadIdx.x; t < prow * pcol_n; t += blockDim.x) {
                const int rr = t / pcol_n, c = t - rr * pcol_n;
                ps[rr * PI + c] = T(0);
            }
        }
        for (int t = threadIdx.x; t < H * W; t += blockDim.x) {
            const int rr = t / W, c = t - rr * W;
            xg[rr * PI + c] = 0.0;
        }
        __syncthreads();
        // ---- ring data; diagonal scaling S
        if (col < P.samples) {
            const int npairs = (P.n_ring + 1) >> 1;
            for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
                const double2 z = gaussian_pair(A.seed, (uint32_t)q, (uint32_t)col, (uint32_t)m, kTagElliptic);
                int gi, gj;
                ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q, gi, gj);
                xg[(gj - P.Y0) * PI + (gi - P.X0)] = z.x;
                if (2 * q + 1 < P.n_ring) {
                    ring_node(P.X0, P.X1, P.Y0, P.Y1, 2 * q + 1, gi, gj);
                    xg[(gj - P.Y0) * PI + (gi - P.X0)] = z.y;
                }
            }
        } else if (threadIdx.x == 0) {
            const int t0 = A.bpos[P.bpos_offset + (col - P.samples)];
            int gi, gj;
            ring_node(P.X0, P.X1, P.Y0, P.Y1, t0, gi, gj);
            xg[(gj - P.Y0) * PI + (gi - P.X0)] = 1.0;
        }
        for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
            const int jj = t / nx, c = t - jj * nx;
            sv[jj * PI + c] =
                1.0 / sqrt(cE[jj * PI + c + 1] + cE[jj * PI + c] + cN[(jj + 1) * PI + c] + cN[jj * PI + c]);
        }
        __syncthreads();
        // ---- scaled faces: a_f s_a s_b between two interior nodes, zero next to the ring or padding
        if constexpr (kF32) {
            for (int t = threadIdx.x; t < PR * (PC + 1); t += blockDim.x) {
                const int jj = t / (PC + 1), c = t - jj * (PC + 1);
                float v = 0.f;
                if (jj < ny && c >= 1 && c <= nx - 1)
                    v = (float)(cE[jj * PI + c] * sv[jj * PI + c - 1] * sv[jj * PI + c]);
                tEs[jj * PI + c] = v;
            }
            for (int t = threadIdx.x; t < (PR + 1) * PC; t += blockDim.x) {
                const int jj = t / PC, c = t - jj * PC;
                float v = 0.f;
                if (jj >= 1 && jj <= ny - 1 && c < nx)
                    v = (float)(cN[jj * PI + c] * sv[(jj - 1) * PI + c] * sv[jj * PI + c]);
                tNs[jj * PI + c] = v;
            }
        } else {
            for (int t = threadIdx.x; t < ny * (nx + 1); t += blockDim.x) {
                const int jj = t / (nx + 1), c = t - jj * (nx + 1);
                tE[jj * PI + c] = (c >= 1 && c <= nx - 1) ? cE[jj * PI + c] * sv[jj * PI + c - 1] * sv[jj * PI + c] : 0.0;
            }
            for (int t = threadIdx.x; t < (ny + 1) * nx; t += blockDim.x) {
                const int jj = t / nx, c = t - jj * nx;
                tN[jj * PI + c] =
                    (jj >= 1 && jj <= ny - 1) ? cN[jj * PI + c] * sv[(jj - 1) * PI + c] * sv[jj * PI + c] : 0.0;
            }
        }
        __syncthreads();

        // per-thread column bases (row r of the segment at offset r * PI)
        T* pcol = ps + (j0 + 1) * PI + (i + 1);          // p at node (i, j0 + r)
        double* xcol = xg + (j0 + 1) * PI + (i + 1);
        const double* e64 = cE + j0 * PI + (i + 1);       // unscaled east face; west at -1
        const double* n64 = cN + (j0 + 1) * PI + i;       // unscaled north face; south at -PI
        const double* s64 = sv + j0 * PI + i;
        const T* te;                                      // scaled east face; west at -1
        const T* tn;                                      // scaled north face; south at -PI
        if constexpr (kF32) {
            te = tEs + j0 * PI + (i + 1);
            tn = tNs + (j0 + 1) * PI + i;
        } else {
            te = tE + j0 * PI + (i + 1);
            tn = tN + (j0 + 1) * PI + i;
        }

        T rreg[RPS], p[RPS];
        int total_it = 0, refs = 0, bad = 0;
        double b2 = -1.0;
        const int passes = kF32 ? A.max_ref : 1;
        for (int pass = 0; pass < passes; ++pass) {
            // FP64 residual r = -(A x) on the owned real nodes; r~ = S r (unnormalised)
            double part[2] = {0.0, 0.0};
#pragma unroll
            for (int r = 0; r < RPS; ++r) {
                rreg[r] = 0;
                if (r < nrow) {
                    const int o = r * PI;
                    const double ae = e64[o], aw = e64[o - 1], an = n64[o], as = n64[o - PI];
                    const double v = -((ae + aw + an + as) * xcol[o] - ae * xcol[o + 1] - aw * xcol[o - 1] -
                                       an * xcol[o + PI] - as * xcol[o - PI]);
                    const double vs = v * s64[o];
                    rreg[r] = (T)vs;
                    part[0] += v * v;
                    part[1] += vs * vs;
                }
            }
            block_sum<double, 2>(part, red64[pass & 1]);
            if (b2 < 0) b2 = part[0];
            if (b2 == 0.0 || part[0] <= A.tol * A.tol * b2) break;
            const double scale = kF32 ? sqrt(part[1]) : 1.0;
            const T inv = (T)(1.0 / scale);
            int it = 0;
            if constexpr (kF32) {
                // ---- FP32 CG on the padded tile, no per-node branches
                float dreg[RPS], qreg[RPS];
                float rz = 0.f;
#pragma unroll
                for (int r = 0; r < RPS; ++r) {
                    rreg[r] *= inv;
                    p[r] = rreg[r];
                    dreg[r] = 0.f;
                    rz += rreg[r] * rreg[r];
                    if (active) pcol[r * PI] = p[r];
                }
                rz = block_sum1<float>(rz, red[0]);      // also orders the p stores above
                const float stop = (float)(A.inner_tol * A.inner_tol) * rz;
                if (rz > 0.f) {
                    for (; it < A.max_iter;) {
                        // q = A~ p = p - (sum of scaled faces x neighbours), pAp
                        float pq = 0.f;
                        if (active) {
                            float south = pcol[-PI];
                            float cs = tn[-PI];
#pragma unroll
                            for (int r = 0; r < RPS; ++r) {
                                const int o = r * PI;
                                const float north = (r + 1 < RPS) ? p[r + 1] : pcol[o + PI];
                                const float ce = te[o], cw = te[o - 1], cn = tn[o];
                                const float pc = p[r];
                                const float qq = pc - (ce * pcol[o + 1] + cw * pcol[o - 1] + cn * north + cs * south);
                                qreg[r] = qq;
                                pq += pc * qq;
                                south = pc;
                                cs = cn;
                            }
                        }
                        const float alpha = rz / block_sum1<float>(pq, red[1]);
                        float rr = 0.f;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) {
                            dreg[r] += alpha * p[r];
                            rreg[r] -= alpha * qreg[r];
                            rr += rreg[r] * rreg[r];
                        }
                        rr = block_sum1<float>(rr, red[0]);
                        ++it;
                        if (rr <= stop) break;
                        const float beta = rr / rz;
                        rz = rr;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) {
                            p[r] = rreg[r] + beta * p[r];
                            if (active) pcol[r * PI] = p[r];
                        }
                        __syncthreads();
                    }
                }
                // x += |S r| S d~ on the owned real nodes
#pragma unroll
                for (int r = 0; r < RPS; ++r)
                    if (r < nrow) xcol[r * PI] += scale * s64[r * PI] * (double)dreg[r];
            } else {
                // ---- FP64 CG, d~ accumulated in the slot
                double* dcol = dd + j0 * PI + i;
                double rz = 0.0;
#pragma unroll
                for (int r = 0; r < RPS; ++r) {
                    p[r] = 0;
                    if (r < nrow) {
                        p[r] = rreg[r];
                        rz += rreg[r] * rreg[r];
                        pcol[r * PI] = p[r];
                        dcol[r * PI] = 0.0;
                    }
                }
                rz = block_sum1<double>(rz, red[0]);
                const double stop = A.tol * A.tol * rz;
                if (rz > 0.0) {
                    for (; it < A.max_iter;) {
                        double pq = 0.0;
                        double south = (nrow > 0) ? pcol[-PI] : 0.0;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) {
                            if (r < nrow) {
                                const int o = r * PI;
                                const double north = (r + 1 < nrow) ? p[r + 1] : pcol[o + PI];
                                const double pc = p[r];
                                const double qq =
                                    pc - (te[o] * pcol[o + 1] + te[o - 1] * pcol[o - 1] + tn[o] * north + tn[o - PI] * south);
                                qs[(j0 + r) * PI + i] = qq;
                                pq += pc * qq;
                                south = pc;
                            }
                        }
                        const double alpha = rz / block_sum1<double>(pq, red[1]);
                        double rr = 0.0;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) {
                            if (r < nrow) {
                                dcol[r * PI] += alpha * p[r];
                                rreg[r] -= alpha * qs[(j0 + r) * PI + i];
                                rr += rreg[r] * rreg[r];
                            }
                        }
                        rr = block_sum1<double>(rr, red[0]);
                        ++it;
                        if (rr <= stop) break;
                        const double beta = rr / rz;
                        rz = rr;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) {
                            if (r < nrow) {
                                p[r] = rreg[r] + beta * p[r];
                                pcol[r * PI] = p[r];
                            }
                        }
                        __syncthreads();
                    }
                }
#pragma unroll
                for (int r = 0; r < RPS; ++r)
                    if (r < nrow) xcol[r * PI] += s64[r * PI] * dcol[r * PI];
            }
            if (it >= A.max_iter) bad = 1;
            total_it += it;
            ++refs;
            __syncthreads();
            if (bad) break;
        }
        if (kF32 && !bad && b2 > 0.0) {   // did the refinement reach tol?
            double part = 0.0;
#pragma unroll
            for (int r = 0; r < RPS; ++r) {
                if (r < nrow) {
                    const int o = r * PI;
                    const double ae = e64[o], aw = e64[o - 1], an = n64[o], as = n64[o - PI];
                    const double v = (ae + aw + an + as) * xcol[o] - ae * xcol[o + 1] - aw * xcol[o - 1] -
                                     an * xcol[o + PI] - as * xcol[o - PI];
                    part += v * v;
                }
            }
            const double r2 = block_sum1<double>(part, red64[0]);
            if (r2 > A.tol * A.tol * b2) bad = 1;
        }
        // ---- restriction to K_m (column `col` of the snapshot block)
        const int wk = P.x1 - P.x0 + 1;
        double* out = A.snaps + P.snap_offset + (long long)col * P.n_k;
        for (int t = threadIdx.x; t < P.n_k; t += blockDim.x) {
            const int jj = t / wk, ii = t - jj * wk;
            out[t] = xg[(P.y0 - P.Y0 + jj) * PI + (P.x0 - P.X0 + ii)];
        }
        if (threadIdx.x == 0) {
            A.stats[3 * item + 0] = total_it;
            A.stats[3 * item + 1] = refs;
            A.stats[3 * item + 2] = bad;
        }
        __syncthreads();
    }
}

// Rows per segment the tile needs, rounded up to an instantiated value.
int rows_instance(int rps) {
    for (int v : {4, 8, 12})
        if (rps <= v) return v;
    return 0;
}

template <class T, int RPS, bool FUSED = false>
msp_status launch_rps(const TileArgs& A, int grid, size_t smem, cudaStream_t s) {
    MSP_CUDA(cudaFuncSetAttribute(local_solve_tile<T, RPS, false, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    local_solve_tile<T, RPS, false, FUSED><<<grid, kTileThreads, smem, s>>>(A);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace

// Rows per segment of one tile-kernel launch: the largest instance any patch
// that fits on its own needs.
int tile_launch_rows(const std::vector<PatchDev>& patches, int precision) {
    int R = 0;
    for (const PatchDev& P : patches) {
        const int nx = P.X1 - P.X0 - 1, ny = P.Y1 - P.Y0 - 1;
        Mapping mp;
        if (!tile_mapping(nx, ny, mp)) continue;
        const int r = rows_instance(mp.rps);
        if (r && smem_bytes(precision == MSP_MIXED, ny, mp.nseg * r) <= 220 * 1024) R = std::max(R, r);
    }
    return R;
}

// Can a tile-kernel launch with R rows per segment take this patch?  Within the
// thread mapping, with the padded shared-memory footprint under the limit.
bool tile_kernel_fits(const PatchDev& P, int precision, int R) {
    const int nx = P.X1 - P.X0 - 1, ny = P.Y1 - P.Y0 - 1;
    Mapping mp;
    if (R == 0 || !tile_mapping(nx, ny, mp) || mp.rps > R) return false;
    return smem_bytes(precision == MSP_MIXED, ny, mp.nseg * R) <= 220 * 1024;
}

msp_status launch_local_solves_tile(Medium& M, const LocalSolveCfg& cfg, const int2* items, int n_items,
                                    int* counter, cudaStream_t s, const gpath::SolveArgs* fused, int R_launch) {
    if (n_items == 0 && !fused) return MSP_OK;
    TileArgs A{};
    A.N = M.N;
    A.aE = M.aE.p;
    A.aN = M.aN.p;
    A.patches = M.patches_dev.p;
    A.bpos = M.bpos_dev.p;
    A.items = items;
    A.n_items = n_items;
    A.counter = counter;
    A.snaps = M.snaps.p;
    A.seed = cfg.seed;
    A.tol = cfg.tol;
    A.inner_tol = cfg.inner_tol;
    A.max_iter = cfg.max_iter;
    A.max_ref = cfg.max_ref;
    A.stats = M.item_stats.p;
    const bool mixed = cfg.precision == MSP_MIXED;
    // one row-count instance for the launch: eligibility was decided with the
    // smallest instance every eligible tile needs; a larger one (R_launch) fits
    // those tiles as long as their shared memory stays under the limit
    const int R0 = std::max(4, tile_launch_rows(M.patches, cfg.precision));
    const int R = std::max(R0, R_launch);
    int max_ny = 0;
    size_t smem = 0;
    for (const PatchDev& P : M.patches) {
        if (!tile_kernel_fits(P, cfg.precision, R0)) continue;
        const int ny = P.Y1 - P.Y0 - 1;
        Mapping mp;
        tile_mapping(P.X1 - P.X0 - 1, ny, mp);
        smem = std::max(smem, smem_bytes(mixed, ny, mp.nseg * R));
        max_ny = std::max(max_ny, ny);
    }
    smem = (smem + 15) / 16 * 16;
    if (smem > 220 * 1024) {
        set_error("local solves: this row instance does not fit the tiles in shared memory");
        return MSP_ERR_INVALID_ARG;
    }
    const int grid = std::max(1, std::min(n_items + (fused ? fused->n_items : 0), num_sms()));
    if (fused) {
        A.g = *fused;
        const size_t gneed = (size_t)(A.g.slot_bytes / (long long)sizeof(double)) * grid + 1;
        if (M.scratch_global.n < gneed) MSP_TRY(M.scratch_global.alloc(gneed, s));
        A.g.scratch = M.scratch_global.p;
    }
    A.slot_doubles = (slot_rows(max_ny) * kPitch + 31) / 32 * 32;
    const size_t need = (size_t)A.slot_doubles * grid;
    if (M.scratch.n < need) MSP_TRY(M.scratch.alloc(need, s));
    A.scratch = M.scratch.p;
    MSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    if (fused) {
        if (mixed) {
            if (R == 4) return launch_rps<float, 4, true>(A, grid, smem, s);
            if (R == 8) return launch_rps<float, 8, true>(A, grid, smem, s);
            return launch_rps<float, 12, true>(A, grid, smem, s);
        }
        if (R == 4) return launch_rps<double, 4, true>(A, grid, smem, s);
        if (R == 8) return launch_rps<double, 8, true>(A, grid, smem, s);
        return launch_rps<double, 12, true>(A, grid, smem, s);
    }
    if (mixed) {
        if (R == 4) return launch_rps<float, 4>(A, grid, smem, s);
        if (R == 8) return launch_rps<float, 8>(A, grid, smem, s);
        return launch_rps<float, 12>(A, grid, smem, s);
    }
    if (R == 4) return launch_rps<double, 4>(A, grid, smem, s);
    if (R == 8) return launch_rps<double, 8>(A, grid, smem, s);
    return launch_rps<double, 12>(A, grid, smem, s);
}

}  // namespace msp

// ---------------------------------------------------------------------------
// Local solves of one patch without any allocation.
//
// Some callers cannot allocate device memory while they run this step: code
// that works inside a memory pool it does not own, a framework that forbids
// allocation on its hot path, or a process whose allocator is already at its
// limit.  msp_sample_patch_static takes every input and output from the caller
// and keeps its per-CTA scratch (FP64 iterate and coefficient copies, the work
// counter, the per-column statistics and the patch description) in one
// file-scope device array of kStaticScratchBytes.  That array exists once per
// device that loads the library and stays allocated until the process exits.
// ---------------------------------------------------------------------------
namespace msp {
namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;      // 32 MiB
constexpr size_t kStaticHeaderBytes = 64u << 10;       // counter, patch, statistics
constexpr int kStaticMaxColumns = 4096;                // 3 ints of statistics per column

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// device address of g_static_scratch per device, found once with the device current
std::mutex g_static_mutex;
std::vector<void*> g_static_addr;

msp_status static_scratch_address(void** out) {
    int dev = 0;
    MSP_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        MSP_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return MSP_OK;
}

}  // namespace
}  // namespace msp

extern "C" msp_status msp_sample_patch_static(const double* aE_dev, const double* aN_dev, int n_cells,
                                              const int* boxes_host, int patch_index, int samples, uint64_t seed,
                                              int precision, double tol, int max_iter, double* snap_dev, void* stream,
                                              int* n_not_converged_host) {
    using namespace msp;
    clear_error();
    MSP_CHECK_ARG(aE_dev && aN_dev && boxes_host && snap_dev, "msp_sample_patch_static: NULL argument");
    MSP_CHECK_ARG(n_cells >= 2, "msp_sample_patch_static: n_cells must be >= 2");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_sample_patch_static: unknown precision");
    MSP_CHECK_ARG(tol > 0 && tol < 1 && max_iter >= 1, "msp_sample_patch_static: tol in (0,1), max_iter >= 1");
    MSP_CHECK_ARG(samples >= 1 && samples <= kStaticMaxColumns,
                  "msp_sample_patch_static: samples must lie in [1, 4096]");
    MSP_CHECK_ARG(patch_index >= 0, "msp_sample_patch_static: patch_index must be >= 0");
    PatchDev P{};
    P.x0 = boxes_host[0]; P.x1 = boxes_host[1]; P.y0 = boxes_host[2]; P.y1 = boxes_host[3];
    P.X0 = boxes_host[4]; P.X1 = boxes_host[5]; P.Y0 = boxes_host[6]; P.Y1 = boxes_host[7];
    MSP_CHECK_ARG(0 <= P.X0 && P.X0 <= P.x0 && P.x0 < P.x1 && P.x1 <= P.X1 && P.X1 <= n_cells && 0 <= P.Y0 &&
                      P.Y0 <= P.y0 && P.y0 < P.y1 && P.y1 <= P.Y1 && P.Y1 <= n_cells,
                  "msp_sample_patch_static: boxes must satisfy 0 <= X0 <= x0 < x1 <= X1 <= N (and in y)");
    P.n_k = (P.x1 - P.x0 + 1) * (P.y1 - P.y0 + 1);
    P.n_ring = 2 * (P.X1 - P.X0) + 2 * (P.Y1 - P.Y0);
    P.samples = samples;
    P.n_b = 0;
    P.cols = samples;
    P.bpos_offset = 0;
    P.snap_offset = 0;
    const int nx = P.X1 - P.X0 - 1, ny = P.Y1 - P.Y0 - 1;
    Mapping mp;
    if (!tile_mapping(nx, ny, mp) || !rows_instance(mp.rps)) {
        set_error("msp_sample_patch_static: the buffered patch exceeds the on-chip tile (at most 98 interior columns "
                  "and 12 rows per thread segment)");
        return MSP_ERR_INVALID_ARG;
    }
    const int R = rows_instance(mp.rps);
    const bool mixed = precision == MSP_MIXED;
    size_t smem = smem_bytes(mixed, ny, mp.nseg * R);
    if (smem > 220 * 1024) {
        set_error("msp_sample_patch_static: the buffered patch exceeds shared memory");
        return MSP_ERR_INVALID_ARG;
    }
    smem = (smem + 15) / 16 * 16;
    const long long slot = (slot_rows(ny) * kPitch + 31) / 32 * 32;   // doubles
    const long long slots = (long long)((kStaticScratchBytes - kStaticHeaderBytes) / sizeof(double)) / slot;
    if (slots < 1) {
        set_error("msp_sample_patch_static: the buffered patch needs more scratch than the static array holds");
        return MSP_ERR_INVALID_ARG;
    }
    unsigned char* base = nullptr;
    MSP_TRY(static_scratch_address(reinterpret_cast<void**>(&base)));
    // header: [0, 256) work counter, [1024, ...) per-column statistics (3 ints each)
    int* counter = reinterpret_cast<int*>(base);
    int* stats = reinterpret_cast<int*>(base + 1024);
    double* scratch = reinterpret_cast<double*>(base + kStaticHeaderBytes);
    cudaStream_t s = (cudaStream_t)stream;
    MSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    TileArgs A{};
    A.N = n_cells;
    A.aE = aE_dev;
    A.aN = aN_dev;
    A.patches = nullptr;
    A.one_patch = P;
    A.bpos = nullptr;
    A.items = nullptr;
    A.n_items = samples;
    A.counter = counter;
    A.snaps = snap_dev;
    A.seed = seed;
    A.tol = tol;
    A.inner_tol = 1e-4;
    A.max_iter = max_iter;
    A.max_ref = 12;
    A.scratch = scratch;
    A.slot_doubles = slot;
    A.stats = stats;
    A.one_patch_index = patch_index;
    const int grid = (int)std::max<long long>(1, std::min<long long>({(long long)samples, slots, (long long)num_sms()}));
#define MSP_STATIC_LAUNCH(T, RR)                                                                                   \
    do {                                                                                                           \
        MSP_CUDA(cudaFuncSetAttribute(local_solve_tile<T, RR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                      (int)smem));                                                                 \
        local_solve_tile<T, RR, true><<<grid, kTileThreads, smem, s>>>(A);                                          \
    } while (0)
    if (mixed) {
        if (R == 4) MSP_STATIC_LAUNCH(float, 4);
        else if (R == 8) MSP_STATIC_LAUNCH(float, 8);
        else MSP_STATIC_LAUNCH(float, 12);
    } else {
        if (R == 4) MSP_STATIC_LAUNCH(double, 4);
        else if (R == 8) MSP_STATIC_LAUNCH(double, 8);
        else MSP_STATIC_LAUNCH(double, 12);
    }
#undef MSP_STATIC_LAUNCH
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    if (n_not_converged_host) {
        // read the not-converged flags back in chunks through a stack buffer: no
        // allocation on either side
        MSP_CUDA(cudaStreamSynchronize(s));
        int bad = 0;
        int buf[3 * 256];
        for (int c0 = 0; c0 < samples; c0 += 256) {
            const int nc = std::min(256, samples - c0);
            MSP_CUDA(cudaMemcpy(buf, stats + 3 * c0, sizeof(int) * 3 * nc, cudaMemcpyDeviceToHost));
            for (int c = 0; c < nc; ++c) bad += buf[3 * c + 2] != 0;
        }
        *n_not_converged_host = bad;
        if (bad) {
            set_error("msp_sample_patch_static: " + std::to_string(bad) + " columns stopped at max_iter");
            return MSP_ERR_NOT_CONVERGED;
        }
    }
    return MSP_OK;
}
