// Tile-resident local solves: one CTA solves one (patch, column) item with the
// whole CG state on chip (Algorithm alg:summary, LocalPDESolver on the buffered
// patch; Eq. elliptic_random for the ring data).
//
// Thread mapping: the interior nx x ny unknowns are cut into strips of 32
// columns; each warp takes one strip and a segment of consecutive rows, so a
// thread owns one column segment of up to kRows rows.  The search direction p
// lives in registers and is mirrored in shared memory (zero halo) for the
// east/west neighbours and the segment ends; north/south neighbours inside the
// segment come from registers.  Every tile array uses the compile-time row pitch
// kPitch, so the unrolled row loop addresses each array as one base register
// plus immediate offsets.
//
//   T = float (mixed path): FP32 face coefficients, Jacobi scaling and the
//     correction d in shared memory; r and A p in registers.  Outer FP64
//     iterative refinement: r = b - A x from the FP64 iterate x and FP64
//     coefficients, FP32 CG on r/|r|, x += |r| d.
//   T = double (plain FP64 path): p and A p in shared memory, r in registers,
//     coefficients and the Jacobi scaling from a per-CTA copy in global scratch;
//     the update d is applied to x directly.
//
// Items (patch, column) come from a global work counter, largest tiles first.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>

namespace msp {

namespace {

constexpr int kTileThreads = 768;
constexpr int kRows = 12;     // max rows per thread segment
constexpr int kPitch = 100;   // row pitch of every tile array: nx + 2 <= kPitch

struct TileArgs {
    int N;
    const double* aE;
    const double* aN;
    const float* aE32;
    const float* aN32;
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
};

// per-CTA global slot (doubles, pitch kPitch):
//   x   : (ny+2) rows  -- FP64 iterate with the ring data
//   cE  : ny rows      -- cE[j][c] = east face of interior column c-1 (c = 0..nx)
//   cN  : (ny+1) rows  -- cN[j][c] = north face of interior row j-1
//   dv  : ny rows      -- Jacobi scaling (FP64 path only)
__host__ __device__ constexpr long long slot_rows(int ny) { return (long long)(ny + 2) + ny + (ny + 1) + ny; }

template <class T>
struct SmemLayout;
template <>
struct SmemLayout<float> {
    // ps (ny+2) | aE ny | aN ny+1 | dv ny | ds ny   rows of kPitch floats
    static __host__ __device__ size_t bytes(int ny) { return sizeof(float) * (size_t)kPitch * (5 * (size_t)ny + 3); }
};
template <>
struct SmemLayout<double> {
    // ps (ny+2) | qs ny   rows of kPitch doubles
    static __host__ __device__ size_t bytes(int ny) { return sizeof(double) * (size_t)kPitch * (2 * (size_t)ny + 2); }
};

__host__ __device__ inline bool tile_mapping(int nx, int ny, int& nstrips, int& nseg, int& rps) {
    const int nw = kTileThreads / 32;
    nstrips = (nx + 31) / 32;
    if (nx < 1 || ny < 1 || nx + 2 > kPitch || nstrips > nw) return false;
    nseg = nw / nstrips;
    rps = (ny + nseg - 1) / nseg;
    return rps <= kRows;
}

template <class T>
__device__ __forceinline__ T block_sum1(T v, T* buf) {
    T a[1] = {v};
    block_sum<T, 1>(a, buf);
    return a[0];
}

template <class T>
__global__ void __launch_bounds__(kTileThreads, 1) local_solve_tile(TileArgs A) {
    constexpr bool kF32 = sizeof(T) == 4;
    constexpr int PI = kPitch;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red[3][64];
    __shared__ double red64[2][32];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* slot = A.scratch + (long long)blockIdx.x * A.slot_doubles;
    const int N = A.N;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(A.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= A.n_items) break;
        const int2 itm = A.items[item];
        const int m = itm.x, col = itm.y;
        const PatchDev P = A.patches[m];
        const int W = P.X1 - P.X0 + 1, H = P.Y1 - P.Y0 + 1;
        const int nx = W - 2, ny = H - 2;
        int nstrips, nseg, rps;
        tile_mapping(nx, ny, nstrips, nseg, rps);   // eligibility checked on the host
        const int strip = warp % nstrips, seg = warp / nstrips;
        const int i = strip * 32 + lane;            // owned interior column
        const int j0 = seg * rps;                   // first owned interior row
        const bool own = (seg < nseg) && (i < nx);
        const int nrow = own ? max(0, min(rps, ny - j0)) : 0;

        // ---- global slot views
        double* xg = slot;                                   // (ny+2) x PI, tile node (c, rr) at rr*PI + c
        double* cE = xg + (long long)(ny + 2) * PI;          // ny x PI
        double* cN = cE + (long long)ny * PI;                // (ny+1) x PI
        double* dv64 = cN + (long long)(ny + 1) * PI;        // ny x PI
        // ---- shared views
        T* ps = reinterpret_cast<T*>(smem_raw);              // (ny+2) x PI
        float *aEs = nullptr, *aNs = nullptr, *dvs = nullptr, *ds = nullptr;
        double* qs = nullptr;
        if constexpr (kF32) {
            aEs = reinterpret_cast<float*>(ps) + (ny + 2) * PI;
            aNs = aEs + ny * PI;
            dvs = aNs + (ny + 1) * PI;
            ds = dvs + ny * PI;
        } else {
            qs = reinterpret_cast<double*>(ps) + (ny + 2) * PI;
        }
        // ---- stage coefficients, zero x and p
        for (int t = threadIdx.x; t < ny * (nx + 1); t += blockDim.x) {
            const int jj = t / (nx + 1), c = t - jj * (nx + 1);
            const long long g = (long long)(P.Y0 + 1 + jj) * N + (P.X0 + c);
            cE[jj * PI + c] = A.aE[g];
            if constexpr (kF32) aEs[jj * PI + c] = A.aE32[g];
        }
        for (int t = threadIdx.x; t < (ny + 1) * nx; t += blockDim.x) {
            const int jj = t / nx, c = t - jj * nx;
            const long long g = (long long)(P.Y0 + jj) * (N + 1) + (P.X0 + 1 + c);
            cN[jj * PI + c] = A.aN[g];
            if constexpr (kF32) aNs[jj * PI + c] = A.aN32[g];
        }
        for (int t = threadIdx.x; t < H * W; t += blockDim.x) {
            const int rr = t / W, c = t - rr * W;
            xg[rr * PI + c] = 0.0;
            ps[rr * PI + c] = T(0);
        }
        __syncthreads();
        // ---- ring data
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
        // ---- Jacobi scaling
        for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
            const int jj = t / nx, c = t - jj * nx;
            const double dg = cE[jj * PI + c + 1] + cE[jj * PI + c] + cN[(jj + 1) * PI + c] + cN[jj * PI + c];
            if constexpr (kF32) dvs[jj * PI + c] = (float)(1.0 / dg);
            else dv64[jj * PI + c] = 1.0 / dg;
        }
        __syncthreads();

        // per-thread column bases (row r of the segment at offset r * PI)
        T* pcol = ps + (j0 + 1) * PI + (i + 1);                 // p at node (i, j0 + r)
        double* xcol = xg + (j0 + 1) * PI + (i + 1);
        const double* e64 = cE + j0 * PI + (i + 1);              // east face; west at -1
        const double* n64 = cN + (j0 + 1) * PI + i;              // north face; south at -PI
        const T* dvc;
        if constexpr (kF32) dvc = dvs + j0 * PI + i;
        else dvc = dv64 + j0 * PI + i;

        T rreg[kRows], qreg[kF32 ? kRows : 1], p[kRows];
        int total_it = 0, refs = 0, bad = 0;
        double b2 = -1.0;
        const int passes = kF32 ? A.max_ref : 1;
        for (int pass = 0; pass < passes; ++pass) {
            // FP64 residual r = -(A x) on the owned nodes (kept unscaled in T)
            double part = 0.0;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                rreg[r] = 0;
                if (r < nrow) {
                    const int o = r * PI;
                    const double ae = e64[o], aw = e64[o - 1], an = n64[o], as = n64[o - PI];
                    const double v = -((ae + aw + an + as) * xcol[o] - ae * xcol[o + 1] - aw * xcol[o - 1] -
                                       an * xcol[o + PI] - as * xcol[o - PI]);
                    rreg[r] = (T)v;
                    part += v * v;
                }
            }
            const double r2 = block_sum1<double>(part, red64[pass & 1]);
            if (b2 < 0) b2 = r2;
            if (b2 == 0.0 || r2 <= A.tol * A.tol * b2) break;
            const double scale = kF32 ? sqrt(r2) : 1.0;
            const T inv = (T)(1.0 / scale);
            // CG from d = 0: z = D^-1 r, p = z
            T rz_part = 0, rr_part = 0;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                p[r] = 0;
                if (r < nrow) {
                    const int o = r * PI;
                    const T rr_ = rreg[r] * inv;
                    rreg[r] = rr_;
                    p[r] = dvc[o] * rr_;
                    rz_part += rr_ * p[r];
                    rr_part += rr_ * rr_;
                    pcol[o] = p[r];
                    if constexpr (kF32) ds[(j0 + r) * PI + i] = 0.f;
                }
            }
            T v0[2] = {rz_part, rr_part};
            block_sum<T, 2>(v0, red[0]);     // also orders the p stores above
            T rz = v0[0];
            const T rr0 = v0[1];
            const T stop = (T)(kF32 ? A.inner_tol * A.inner_tol : A.tol * A.tol) * rr0;
            int it = 0;
            if (rr0 > T(0)) {
                float* dcol = nullptr;
                if constexpr (kF32) dcol = ds + j0 * PI + i;
                for (; it < A.max_iter;) {
                    // q = A p on the owned column segment, pAp
                    T pq = 0;
                    T south = (nrow > 0) ? pcol[-PI] : T(0);
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        if (r < nrow) {
                            const int o = r * PI;
                            const T north = (r + 1 < nrow) ? p[r + 1] : pcol[o + PI];
                            const T west = pcol[o - 1];
                            const T east = pcol[o + 1];
                            T ce, cw, cn, cs;
                            if constexpr (kF32) {
                                const float* ec = aEs + j0 * PI + (i + 1);
                                const float* nc = aNs + (j0 + 1) * PI + i;
                                ce = ec[o]; cw = ec[o - 1]; cn = nc[o]; cs = nc[o - PI];
                            } else {
                                ce = e64[o]; cw = e64[o - 1]; cn = n64[o]; cs = n64[o - PI];
                            }
                            const T pc = p[r];
                            const T qq = (ce + cw + cn + cs) * pc - ce * east - cw * west - cn * north - cs * south;
                            if constexpr (kF32) qreg[r] = qq;
                            else qs[(j0 + r) * PI + i] = qq;
                            pq += pc * qq;
                            south = pc;
                        }
                    }
                    const T pAp = block_sum1<T>(pq, red[1]);
                    const T alpha = rz / pAp;
                    T zr = 0, rr = 0;
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        if (r < nrow) {
                            const int o = r * PI;
                            T qq;
                            if constexpr (kF32) {
                                dcol[o] += alpha * p[r];
                                qq = qreg[r];
                            } else {
                                xcol[o] += alpha * p[r];
                                qq = qs[(j0 + r) * PI + i];
                            }
                            const T rr_ = rreg[r] - alpha * qq;
                            rreg[r] = rr_;
                            const T z = dvc[o] * rr_;
                            if constexpr (kF32) qreg[r] = z;
                            else qs[(j0 + r) * PI + i] = z;
                            zr += rr_ * z;
                            rr += rr_ * rr_;
                        }
                    }
                    T v2[2] = {zr, rr};
                    block_sum<T, 2>(v2, red[2]);
                    ++it;
                    if (v2[1] <= stop) break;
                    const T beta = v2[0] / rz;
                    rz = v2[0];
#pragma unroll
                    for (int r = 0; r < kRows; ++r) {
                        if (r < nrow) {
                            const int o = r * PI;
                            T z;
                            if constexpr (kF32) z = qreg[r];
                            else z = qs[(j0 + r) * PI + i];
                            p[r] = z + beta * p[r];
                            pcol[o] = p[r];
                        }
                    }
                    __syncthreads();
                }
            }
            if (it >= A.max_iter) bad = 1;
            total_it += it;
            ++refs;
            // x += |r| d on the owned nodes (FP32 path; the FP64 path updated x in place)
            if constexpr (kF32) {
#pragma unroll
                for (int r = 0; r < kRows; ++r)
                    if (r < nrow) xcol[r * PI] += scale * (double)ds[(j0 + r) * PI + i];
            }
            __syncthreads();
            if (bad) break;
        }
        if (kF32 && !bad && b2 > 0.0) {   // did the refinement reach tol?
            double part = 0.0;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
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

}  // namespace

bool tile_kernel_fits(const PatchDev& P, int precision) {
    const int nx = P.X1 - P.X0 - 1, ny = P.Y1 - P.Y0 - 1;
    int nstrips, nseg, rps;
    if (!tile_mapping(nx, ny, nstrips, nseg, rps)) return false;
    const size_t sm = precision == MSP_MIXED ? SmemLayout<float>::bytes(ny) : SmemLayout<double>::bytes(ny);
    return sm <= 220 * 1024;
}

msp_status launch_local_solves_tile(Medium& M, const LocalSolveCfg& cfg, const int2* items, int n_items,
                                    int* counter, cudaStream_t s) {
    if (n_items == 0) return MSP_OK;
    TileArgs A{};
    A.N = M.N;
    A.aE = M.aE.p; A.aN = M.aN.p; A.aE32 = M.aE32.p; A.aN32 = M.aN32.p;
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
    size_t smem = 0;
    int max_ny = 0;
    for (const PatchDev& P : M.patches) {
        if (!tile_kernel_fits(P, cfg.precision)) continue;
        const int ny = P.Y1 - P.Y0 - 1;
        smem = std::max(smem, mixed ? SmemLayout<float>::bytes(ny) : SmemLayout<double>::bytes(ny));
        max_ny = std::max(max_ny, ny);
    }
    smem = (smem + 15) / 16 * 16;
    const int grid = std::max(1, std::min(n_items, num_sms()));
    A.slot_doubles = (slot_rows(max_ny) * kPitch + 31) / 32 * 32;
    const size_t need = (size_t)A.slot_doubles * grid;
    if (M.scratch.n < need) MSP_TRY(M.scratch.alloc(need, s));
    A.scratch = M.scratch.p;
    MSP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    if (mixed) {
        MSP_CUDA(cudaFuncSetAttribute(local_solve_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        local_solve_tile<float><<<grid, kTileThreads, smem, s>>>(A);
    } else {
        MSP_CUDA(cudaFuncSetAttribute(local_solve_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        local_solve_tile<double><<<grid, kTileThreads, smem, s>>>(A);
    }
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace msp
