// Tensor-core (tcgen05, kind::tf32) GEMM for the boundary-to-coefficient map:
// c[j][b] = sum_k G[j][k] phi[b][k], with FP32-level accuracy from TF32 units by
// the three-term split X = X_hi + X_lo (X_hi = X rounded to TF32, X_lo the FP32
// remainder): G phi ~ G_hi phi_hi + G_hi phi_lo + G_lo phi_hi, all three products
// accumulated by the tensor core in FP32 in tensor memory.  The K sum is cut into
// slabs of 32 terms; each slab's FP32 accumulator is read out of tensor memory and
// added into a compensated FP32 sum (two-sum per term), so the rounding of the
// long sum does not grow with the ring length.
//
// Operands are stored pre-tiled in the no-swizzle K-major layout the MMA reads:
// 8-row x 16-byte core matrices, K-adjacent core matrices 128 B apart (leading
// byte offset), row-adjacent groups of 8 rows one slab row-group apart (stride
// byte offset).  Each (row tile, 32-wide K slab) block is contiguous, so one bulk
// copy (cp.async.bulk, TMA engine) moves it into shared memory.
//
// One CTA of 128 threads per 128-row tile; N = 32 data sets per launch tile.
// Thread 0 issues the bulk copies (four stages, mbarriers) and the MMAs; tcgen05
// commits release the stages and signal the slab accumulator; the four warps read
// their 32 tensor-memory lanes each, from one of two accumulators while the MMAs
// of the next slab fill the other.  Every wait is bounded: on timeout the CTA
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

// bounded wait that also gives up as soon as another thread of the CTA has failed
__device__ __forceinline__ bool mbar_wait_or_fail(unsigned long long* bar, unsigned parity, volatile int* fail) {
    for (long long spin = 0; spin < (1LL << 26); ++spin) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((spin & 255) == 255 && *fail) return false;
    }
    return false;
}

// s + e = a + b exactly (Knuth's two-sum, six FP32 operations, no branches)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Two accumulators in tensor memory (columns 0-31 and 32-63): the MMAs of slab s
// go to accumulator s & 1 while the four warps read slab s - 1 out of the other,
// add it into a compensated FP32 sum (value + running error, two-sum per term)
// and release it (acc_free, 128 arrivals).  Thread 0 issues the copies and MMAs.
__global__ void __launch_bounds__(128, 1) tc_map_gemm_kernel(TcMapArgs A) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], accb[2], accfree[2];
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
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accb[b], 1);
            mbar_init(&accfree[b], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(64)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    volatile int* fail = &s_fail;
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
    // leading byte offset: K-adjacent core matrices; stride byte offset: next 8 rows
    const unsigned lbo = 128, sbo = (kSlab / 4) * 128;
    int last_issued[2] = {-1, -1};   // thread 0: last slab committed to each accumulator
    // thread 0: MMAs of one slab into accumulator (slab & 1); false on a timed-out wait
    auto mma_slab = [&](int sl) -> bool {
        const int nxt = sl + kStages - 1;   // refill the stage the previous slab used
        if (nxt < n_slabs) {
            if (sl >= 1 && !mbar_wait_or_fail(&empty[(sl - 1) % kStages], (unsigned)(((sl - 1) / kStages) & 1), fail))
                return false;
            issue_copy(nxt);
        }
        const int st = sl % kStages, ab = sl & 1;
        if (!mbar_wait_or_fail(&full[st], (unsigned)((sl / kStages) & 1), fail)) return false;
        if (sl >= 2 && !mbar_wait_or_fail(&accfree[ab], (unsigned)(((sl - 2) >> 1) & 1), fail)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float* p = stage_ptr(st);
        const unsigned d = tmem + (unsigned)(ab * kN);
#pragma unroll
        for (int ks = 0; ks < kSlab / 8; ++ks) {   // one MMA covers K = 8 (two core matrices)
            const unsigned off = ks * 2 * 128;
            const unsigned long long dah = smem_desc(reinterpret_cast<const char*>(p) + off, lbo, sbo);
            const unsigned long long dal = smem_desc(reinterpret_cast<const char*>(p + kAFloats) + off, lbo, sbo);
            const unsigned long long dbh = smem_desc(reinterpret_cast<const char*>(p + 2 * kAFloats) + off, lbo, sbo);
            const unsigned long long dbl =
                smem_desc(reinterpret_cast<const char*>(p + 2 * kAFloats + kBFloats) + off, lbo, sbo);
            mma_tf32(d, dah, dbh, ks == 0 ? 0u : 1u);
            mma_tf32(d, dah, dbl, 1u);
            mma_tf32(d, dal, dbh, 1u);
        }
        mma_commit(&empty[st]);
        mma_commit(&accb[ab]);
        last_issued[ab] = sl;
        return true;
    };
    float sum[kN], cmp[kN];
#pragma unroll
    for (int t = 0; t < kN; ++t) sum[t] = cmp[t] = 0.f;
    // all threads: read slab sl's accumulator, add it, release the accumulator
    // (warp-uniform result: the tensor-memory load below is a warp-collective)
    auto epilogue = [&](int sl) -> bool {
        const int ab = sl & 1;
        const bool got = mbar_wait_or_fail(&accb[ab], (unsigned)((sl >> 1) & 1), fail);
        if (!__all_sync(0xffffffffu, got)) {
            *fail = 1;
            return false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned r[kN];
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(ab * kN);
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
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accfree[ab])) : "memory");
#pragma unroll
        for (int t = 0; t < kN; ++t) {
            float s2, e2;
            two_sum(sum[t], __uint_as_float(r[t]), s2, e2);
            sum[t] = s2;
            cmp[t] += e2;
        }
        return true;
    };
    if (tid == 0)
        for (int sl = 0; sl < kStages - 1 && sl < n_slabs; ++sl) issue_copy(sl);
    bool ok = true;   // warp-uniform
    for (int sl = 0; sl < n_slabs; ++sl) {
        bool f = false;
        if (tid == 0) f = !mma_slab(sl);
        if (f) *fail = 1;
        if (__any_sync(0xffffffffu, f || *fail != 0)) {
            ok = false;
            break;
        }
        if (sl >= 1 && !epilogue(sl - 1)) {
            ok = false;
            break;
        }
    }
    if (ok && n_slabs >= 1 && !epilogue(n_slabs - 1)) ok = false;
    if (!ok) *fail = 1;
    __syncthreads();
    const bool failed = *fail != 0;
    if (failed && tid == 0) atomicExch(A.err, 1);
    // output row j of the tile: c[j][b] for the data sets of this N tile
    const int j = tile * kRows + warp * 32 + lane;
    if (!failed && j < A.M) {
        const int b0 = ntile * kN;
#pragma unroll
        for (int t = 0; t < kN; ++t)
            if (b0 + t < A.B) A.c[(long long)j * A.B + b0 + t] = sum[t] + cmp[t];
    }
    if (failed && tid == 0) {
        // bounded waits for MMAs already issued before the tensor memory is freed
        for (int b = 0; b < 2; ++b)
            if (last_issued[b] >= 0) mbar_wait(&accb[b], (unsigned)((last_issued[b] >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
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
