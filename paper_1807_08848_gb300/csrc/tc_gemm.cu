// Tensor-core (tcgen05, kind::tf32) GEMM for the boundary-to-coefficient map:
// c[j][b] = sum_k G[j][k] phi[b][k], with FP32-level accuracy from TF32 units by
// the three-term split X = X_hi + X_lo (X_hi = X rounded to TF32, X_lo the FP32
// remainder): G phi ~ G_hi phi_hi + G_hi phi_lo + G_lo phi_hi, all three products
// accumulated by the tensor core in FP32 in tensor memory.  The K sum is cut into
// chunks of kChunkSlabs x 32; each chunk's FP32 accumulator is read out of tensor
// memory and added into FP64 registers, so the rounding of the long sum does not
// grow with the ring length.
//
// Operands are stored pre-tiled in the no-swizzle K-major layout the MMA reads:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (leading
// byte offset), row-adjacent groups of 8 rows one slab row-group apart (stride
// byte offset).  Each (row tile, 32-wide K slab) block is contiguous, so one bulk
// copy (cp.async.bulk, TMA engine) moves it into shared memory.
//
// One CTA of 128 threads per 128-row tile; N = 32 data sets per launch tile.
// Thread 0 issues the bulk copies (four stages, mbarriers) and the MMAs; tcgen05
// commits release the stages and signal the chunk accumulator; the four warps read
// their 32 tensor-memory lanes each.  Every wait is bounded: on timeout the CTA
// records the failure in *err, stops issuing work, frees its tensor memory and
// leaves.
#include "internal.h"
#include "tc_gemm.cuh"

namespace msp {

namespace {

constexpr int kRows = 128;             // MMA M
constexpr int kN = 32;                 // MMA N (data sets per tile)
constexpr int kSlab = 32;              // K elements per staged slab
constexpr int kStages = 4;
constexpr int kChunkSlabs = 1;         // slabs per FP64 accumulation (32 terms)
constexpr int kAFloats = kRows * kSlab;   // one operand half of a slab
constexpr int kBFloats = kN * kSlab;
constexpr unsigned kStageBytes = (unsigned)(2 * (kAFloats + kBFloats) * sizeof(float));

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (long long spin = 0; spin < (1LL << 26); ++spin) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: start address, leading and stride byte offsets
// (all in 16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(const void* p, unsigned lbo, unsigned sbo) {
    const unsigned long long a = (smem_u32(p) >> 4) & 0x3FFFu;
    return a | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) | ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N, M.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kN >> 3) << 17) |
                            ((unsigned)(kRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(128, 1) tc_map_gemm_kernel(TcMapArgs A) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], accb;
    __shared__ unsigned s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, ntile = blockIdx.y;
    float* stage0 = reinterpret_cast<float*>(tc_smem);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const int n_slabs = A.n_slabs;
    const float* ahi = A.a_hi + (long long)tile * n_slabs * kAFloats;
    const float* alo = A.a_lo + (long long)tile * n_slabs * kAFloats;
    const float* bhi = A.b_hi + (long long)ntile * n_slabs * kBFloats;
    const float* blo = A.b_lo + (long long)ntile * n_slabs * kBFloats;
    auto stage_ptr = [&](int s) { return stage0 + (long long)s * 2 * (kAFloats + kBFloats); };
    auto issue_copy = [&](int slab) {
        const int st = slab % kStages;
        float* p = stage_ptr(st);
        mbar_expect_tx(&full[st], kStageBytes);
        bulk_g2s(p, ahi + (long long)slab * kAFloats, kAFloats * 4, &full[st]);
        bulk_g2s(p + kAFloats, alo + (long long)slab * kAFloats, kAFloats * 4, &full[st]);
        bulk_g2s(p + 2 * kAFloats, bhi + (long long)slab * kBFloats, kBFloats * 4, &full[st]);
        bulk_g2s(p + 2 * kAFloats + kBFloats, blo + (long long)slab * kBFloats, kBFloats * 4, &full[st]);
    };
    double acc[kN];
#pragma unroll
    for (int t = 0; t < kN; ++t) acc[t] = 0.0;
    if (tid == 0)
        for (int sl = 0; sl < kStages - 1 && sl < n_slabs; ++sl) issue_copy(sl);
    const int n_chunks = (n_slabs + kChunkSlabs - 1) / kChunkSlabs;
    int committed = -1;   // thread 0: last chunk whose accumulator commit was issued
    // leading byte offset: K-adjacent core matrices; stride byte offset: next 8 rows
    const unsigned lbo = 128, sbo = (kSlab / 4) * 128;
    for (int c = 0; c < n_chunks; ++c) {
        if (tid == 0 && !s_fail) {
            const int s_end = min(n_slabs, (c + 1) * kChunkSlabs);
            for (int sl = c * kChunkSlabs; sl < s_end; ++sl) {
                // refill the stage the previous slab used, once its MMAs are done
                const int nxt = sl + kStages - 1;
                if (nxt < n_slabs) {
                    if (sl >= 1 && !mbar_wait(&empty[(sl - 1) % kStages], (unsigned)(((sl - 1) / kStages) & 1))) {
                        s_fail = 1;
                        break;
                    }
                    issue_copy(nxt);
                }
                const int st = sl % kStages;
                if (!mbar_wait(&full[st], (unsigned)((sl / kStages) & 1))) {
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float* p = stage_ptr(st);
#pragma unroll
                for (int ks = 0; ks < kSlab / 8; ++ks) {   // one MMA covers K = 8 (two core matrices)
                    const unsigned off = ks * 2 * 128;
                    const unsigned long long dah = smem_desc(reinterpret_cast<const char*>(p) + off, lbo, sbo);
                    const unsigned long long dal =
                        smem_desc(reinterpret_cast<const char*>(p + kAFloats) + off, lbo, sbo);
                    const unsigned long long dbh =
                        smem_desc(reinterpret_cast<const char*>(p + 2 * kAFloats) + off, lbo, sbo);
                    const unsigned long long dbl =
                        smem_desc(reinterpret_cast<const char*>(p + 2 * kAFloats + kBFloats) + off, lbo, sbo);
                    const unsigned first = (sl == c * kChunkSlabs && ks == 0) ? 0u : 1u;
                    mma_tf32(tmem, dah, dbh, first);
                    mma_tf32(tmem, dah, dbl, 1u);
                    mma_tf32(tmem, dal, dbh, 1u);
                }
                mma_commit(&empty[st]);
            }
            mma_commit(&accb);   // the chunk's products are in tensor memory once this arrives
            committed = c;
        }
        __syncwarp();
        __syncthreads();
        if (s_fail) break;
        if (!mbar_wait(&accb, (unsigned)(c & 1))) {
            s_fail = 1;
            atomicExch(A.err, 1);
        }
        __syncthreads();
        if (s_fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned r[kN];
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < kN; ++t) acc[t] += (double)__uint_as_float(r[t]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (s_fail && tid == 0) {
        atomicExch(A.err, 1);
        // bounded wait for the MMAs already issued before the tensor memory is freed
        if (committed >= 0) mbar_wait(&accb, (unsigned)(committed & 1));
    }
    // output row j of the tile: c[j][b] for the data sets of this N tile
    const int j = tile * kRows + warp * 32 + lane;
    if (!s_fail && j < A.M) {
        const int b0 = ntile * kN;
#pragma unroll
        for (int t = 0; t < kN; ++t)
            if (b0 + t < A.B) A.c[(long long)j * A.B + b0 + t] = (float)acc[t];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
    (void)lane;
}

// Scatter of a row-major matrix X (rows x K, leading dimension ld, element (r, k) at
// r * ld_r + k * ld_k) into the tiled hi / lo layout: row tiles of R rows, K slabs of
// 32; rows and K beyond the matrix are zero.
__global__ void tc_tile_split_kernel(const float* X, long long ld_r, long long ld_k, int rows, int K, int R,
                                     int n_tiles, int n_slabs, float* hi, float* lo) {
    const long long total = (long long)n_tiles * n_slabs * R * kSlab;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // e enumerates the tiled layout: [tile][slab][row group][k group][row in group][k in group]
        const int kin = (int)(e & 3);
        const int rin = (int)((e >> 2) & 7);
        long long q = e >> 5;
        const int kg = (int)(q % (kSlab / 4));
        q /= (kSlab / 4);
        const int rg = (int)(q % (R / 8));
        q /= (R / 8);
        const int slab = (int)(q % n_slabs);
        const int t = (int)(q / n_slabs);
        const int r = t * R + rg * 8 + rin, k = slab * kSlab + kg * 4 + kin;
        float v = 0.f;
        if (r < rows && k < K) v = X[(long long)r * ld_r + (long long)k * ld_k];
        // round to TF32 (10 explicit mantissa bits), nearest, ties away from zero
        const unsigned u = __float_as_uint(v);
        const float h = __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
        hi[e] = isfinite(h) ? h : v;
        lo[e] = isfinite(h) ? v - h : 0.f;
    }
}

}  // namespace

int tc_slabs(int K) { return (K + kSlab - 1) / kSlab; }
int tc_row_tiles(int M) { return (M + kRows - 1) / kRows; }
int tc_n_tiles(int B) { return (B + kN - 1) / kN; }
long long tc_a_floats(int M, int K) { return (long long)tc_row_tiles(M) * tc_slabs(K) * kAFloats; }
long long tc_b_floats(int B, int K) { return (long long)tc_n_tiles(B) * tc_slabs(K) * kBFloats; }

void tc_tile_split(const float* X, long long ld_r, long long ld_k, int rows, int K, bool a_operand, float* hi, float* lo,
                   cudaStream_t s) {
    const int R = a_operand ? kRows : kN;
    const int nt = (rows + R - 1) / R, ns = tc_slabs(K);
    const long long total = (long long)nt * ns * R * kSlab;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 32));
    tc_tile_split_kernel<<<grid, 256, 0, s>>>(X, ld_r, ld_k, rows, K, R, nt, ns, hi, lo);
    count_launches(1);
}

msp_status tc_map_gemm(const TcMapArgs& args, cudaStream_t s) {
    const size_t smem = (size_t)kStages * kStageBytes;
    static bool attr = false;
    if (!attr) {
        MSP_CUDA(cudaFuncSetAttribute(tc_map_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    dim3 grid(tc_row_tiles(args.M), tc_n_tiles(args.B));
    tc_map_gemm_kernel<<<grid, 128, smem, s>>>(args);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    return MSP_OK;
}

}  // namespace msp
