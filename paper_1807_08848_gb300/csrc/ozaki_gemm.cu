// FP64-accurate batched GEMM on the fifth-generation tensor cores: the snapshot
// Gram and basis-projection products of the extraction (Sec. 3.2, Eq. svd; the
// QR remark of Sec. 3.3) and the large products of the online factorisation.
//
// Error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump (2012):
// every row i of op(A) is scaled by a power of two sigma_i > max_k |a_ik| and cut
// by truncation into kSlices slices of kBeta bits,
//     a_ik = sigma_i sum_t d_ik^(t) 2^(-kBeta t),  d^(t) integers with |d| <= 127,
// and likewise every column j of op(B) with tau_j and slices e^(u).  Each slice
// is exact in BF16, each product d^(t) e^(u) exact in FP32 (|.| < 2^14), and the
// products of one diagonal t + u = g are summed by the tensor core (kind::f16,
// FP32 accumulation in tensor memory) over K chunks of 128, in which at most 8
// pairs x 128 terms x 2^14 < 2^24 keep every partial sum an exact integer.
// After each chunk the accumulators are read out of tensor memory and folded, in
// integers, into two int64 halves (exact for K up to 16256), so
//     C_ij = alpha sigma_i tau_j sum_g 2^(-kBeta g) V_g(i, j) + beta C_ij
// is formed once per element at the end from two exactly representable halves: an
// element costs a few FP64 operations (the FP64 pipe issues about two FMAs per
// clock and SM here).  Pairs with t + u > kSlices + 1
// are dropped: with 8 slices of 7 bits each dropped or truncated term is below
// about 2^-56 sigma_i tau_j, under the rounding of an FP64 product.
//
// Structure flags of the descriptors (zero ranges of op(A) or op(B)) are applied
// while slicing: those entries become zero slices whatever the memory holds.
// Layout of a sliced operand: [row tile][K slab of 16][slice][row group of 8]
// [k core of 8][row][k], BF16 -- the no-swizzle K-major layout of the MMA, 16-byte
// core matrices, K-adjacent cores 128 B apart, 8-row groups 256 B apart; the
// kSlices blocks of one (row tile, slab) are contiguous and move with one bulk copy.
//
// MMA kernel: one CTA of 256 threads per 128 x 32 output tile of one product, two
// CTAs per SM.  Thread 0 issues the bulk copies (two stages of 40 KB: 8 A slices of
// 128 x 16 and 8 B slices of 32 x 16; one slab in flight while one is multiplied)
// and the MMAs; the 8 diagonal accumulators of a chunk take 8 x 32 = 256 columns of
// tensor memory, so the two CTAs of an SM hold all 512, and the read-out of one
// CTA's chunk overlaps the other CTA's MMAs (measured faster than one CTA per SM
// with two accumulator sets and five stages).  Every wait is bounded: on timeout
// the CTA records the failure, stops issuing work, waits (bounded) for its issued
// MMAs, frees its tensor memory and leaves without writing C.
#include "internal.h"
#include "dense.cuh"

#include <algorithm>
#include <cuda_bf16.h>
#include <vector>

namespace msp {

namespace {

constexpr int kSlices = 8;
constexpr int kBeta = 7;
constexpr int kDiag = kSlices;            // diagonals g = t + u = 2 .. kSlices + 1
constexpr int kTM = 128;                  // output rows per CTA (MMA M)
constexpr int kTN = 32;                   // output columns per CTA (MMA N)
constexpr int kSlabK = 16;                // K per staged slab (one MMA)
constexpr int kCoresK = kSlabK / 8;       // 8 x 8 core matrices along K per slab
constexpr int kChunkSlabs = 128 / kSlabK; // slabs per exactness chunk (K = 128)
constexpr int kAccBufs = 1;               // accumulator sets in tensor memory per CTA
constexpr int kCtasPerSm = 3 - kAccBufs;  // one accumulator set: two CTAs share an SM
constexpr int kStages = kAccBufs == 1 ? 2 : 5;   // slabs in flight per CTA
constexpr unsigned kTmemCols = (unsigned)(kAccBufs * kDiag * kTN);   // 256 or 512
constexpr int kOzThreads = 256;
constexpr unsigned kAElems = kTM * kSlabK;                    // one A slice block
constexpr unsigned kBElems = kTN * kSlabK;
constexpr unsigned kStageBytes = (unsigned)(kSlices * (kAElems + kBElems) * 2);
constexpr int kOzMaxK = 16256;            // int32 accumulation stays exact up to here

struct OzEntry {
    long long a_sl, b_sl;                 // element offsets of the sliced operands
    long long a_sc, b_sc;                 // offsets of the row / column scales
    int rta, rtb, slabs;                  // row tiles of op(A), of op(B)^T, K slabs
    int pad;
};
static_assert(sizeof(OzEntry) % sizeof(long long) == 0, "entries travel as long long words");

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
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
        if ((spin & 255) == 255 && fail && *fail) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// shared-memory matrix descriptor: start, leading and stride byte offsets (16-byte
// units), descriptor version 1, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(const void* p, unsigned lbo, unsigned sbo) {
    const unsigned long long a = (smem_u32(p) >> 4) & 0x3FFFu;
    return a | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) | ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16 (the same type), both
// K-major, N = 32, M = 128
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kTN >> 3) << 17) |
                            ((unsigned)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// ------------------------------------------------------------------ slicing
// Operand view: R rows x K, element (r, k) at base[r * sr + k * sk]; zero where
// the structure of the product says so.
struct OpView {
    const double* base;
    long long sr, sk;
    int R, K;
    int lower_k_gt_r;    // entries with k > r are zero (op(A) lower triangular)
    int zero_k_lt_r;     // entries with k < r are zero (op(B) lower triangular, seen by column)
    int zero_k_gt_r;     // entries with k > r are zero (op(B) upper triangular, seen by column)
    const int* k_lo;     // entries with k < k_lo[r] are zero
};

__device__ __forceinline__ OpView view_a(const GemmDesc& D, bool tA) {
    OpView v;
    v.base = D.A;
    v.sr = tA ? D.lda : 1;
    v.sk = tA ? 1 : D.lda;
    v.R = D.M;
    v.K = D.K;
    v.lower_k_gt_r = D.a_lower;
    v.zero_k_lt_r = 0;
    v.zero_k_gt_r = 0;
    v.k_lo = D.a_k_lo;
    return v;
}

__device__ __forceinline__ OpView view_b(const GemmDesc& D, bool tB) {
    OpView v;   // rows = columns j of op(B); op(B)[k][j] = tB ? B[k * ldb + j] : B[j * ldb + k]
    v.base = D.B;
    v.sr = tB ? 1 : D.ldb;
    v.sk = tB ? D.ldb : 1;
    v.R = D.N;
    v.K = D.K;
    v.lower_k_gt_r = 0;
    v.zero_k_lt_r = D.b_lower;
    v.zero_k_gt_r = D.b_upper;
    v.k_lo = nullptr;
    return v;
}

__device__ __forceinline__ double op_elem(const OpView& v, int r, int k) {
    if (r >= v.R || k >= v.K) return 0.0;
    if (v.lower_k_gt_r && k > r) return 0.0;
    if (v.zero_k_lt_r && k < r) return 0.0;
    if (v.zero_k_gt_r && k > r) return 0.0;
    if (v.k_lo && k < v.k_lo[r]) return 0.0;
    return v.base[(long long)r * v.sr + (long long)k * v.sk];
}

// Per row: the scale 2^e with 2^(e-1) <= max|x| < 2^e (1 for an all-zero row),
// stored as the exponent e.  The magnitude of an FP64 value orders like its bit
// pattern with the sign cleared, so the maximum is an integer maximum (no FP64
// arithmetic: the FP64 pipe is the narrow one on this part).  One warp per row.
template <bool IS_B>
__global__ void __launch_bounds__(256) oz_scale_kernel(const GemmDesc* descs, const OzEntry* ents, bool tA, bool tB,
                                                       int* scale_exp, int max_rows) {
    const int z = blockIdx.y;
    const GemmDesc D = descs[z];
    const OpView v = IS_B ? view_b(D, tB) : view_a(D, tA);
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= v.R || r >= max_rows) return;
    unsigned long long mx = 0;
    for (int k = lane; k < v.K; k += 32) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(op_elem(v, r, k)) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if (lane == 0) {
        // mx = f 2^E with f in [1, 2) (normal) or a subnormal: scale exponent E + 1
        int e = 0;
        if (mx != 0) {
            const int be = (int)(mx >> 52);
            e = be > 0 ? be - 1023 + 1 : -1022;   // subnormals lie below 2^-1022
        }
        scale_exp[(IS_B ? ents[z].b_sc : ents[z].a_sc) + r] = e;
    }
}

// Slices of every element of the tiled layout (one thread per element, all
// slices).  With the scale 2^e and |a| = m 2^(E-52) (m the 53-bit significand),
// F = floor(|a| 2^(56-e)) = m shifted by E - e + 4 holds the 8 x 7 leading bits of
// |a| / 2^e in (0, 1); slice t is bits 55-7t .. 49-7t of F with the sign of a --
// the digits of the truncated base-128 expansion, found with integer operations.
template <bool IS_B>
__global__ void __launch_bounds__(256) oz_slice_kernel(const GemmDesc* descs, const OzEntry* ents, bool tA, bool tB,
                                                       const int* scale_exp, __nv_bfloat16* out) {
    const int z = blockIdx.y;
    const GemmDesc D = descs[z];
    const OzEntry E = ents[z];
    const OpView v = IS_B ? view_b(D, tB) : view_a(D, tA);
    const int RT = IS_B ? kTN : kTM;
    const int tiles = IS_B ? E.rtb : E.rta;
    const long long per_slice = (long long)tiles * E.slabs * RT * kSlabK;
    const long long base = IS_B ? E.b_sl : E.a_sl;
    const int* se = scale_exp + (IS_B ? E.b_sc : E.a_sc);
    // per_slice < 2^31 (checked on the host): the tiled index fits 32 bits
    const unsigned slabs_u = (unsigned)E.slabs;
    const unsigned blk = (unsigned)(RT * kSlabK);   // one (tile, slab) block of one slice
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)per_slice; e += gridDim.x * blockDim.x) {
        // e = [tile][slab][row group][k core][row][k]
        const int kk = (int)(e & 7);
        const int rr = (int)((e >> 3) & 7);
        const int kc = (int)((e >> 6) % kCoresK);
        unsigned q = e / (64u * kCoresK);
        const int rg = (int)(q % (RT / 8));
        q /= (RT / 8);
        const int slab = (int)(q % slabs_u);
        const int tile = (int)(q / slabs_u);
        const int r = tile * RT + rg * 8 + rr, k = slab * kSlabK + kc * 8 + kk;
        unsigned long long F = 0;
        bool neg = false;
        if (r < v.R && k < v.K) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(op_elem(v, r, k));
            neg = (bits >> 63) != 0;
            const int be = (int)((bits >> 52) & 0x7FF);
            const unsigned long long frac = bits & 0xFFFFFFFFFFFFFull;
            const unsigned long long m = be ? (frac | (1ull << 52)) : frac;   // significand
            const int E2 = be ? be - 1023 : -1022;                             // |a| = m 2^(E2 - 52)
            const int sh = E2 - se[r] + 4;                                     // F = m 2^sh
            if (m != 0) F = sh >= 0 ? (sh < 8 ? m << sh : 0ull) : (sh > -64 ? m >> -sh : 0ull);
        }
#pragma unroll
        for (int t = 0; t < kSlices; ++t) {
            const int d = (int)((F >> (kSlices * kBeta - kBeta * (t + 1))) & ((1u << kBeta) - 1u));
            out[base + ((long long)(e / blk) * kSlices + t) * blk + (e % blk)] = __float2bfloat16_rn((float)(neg ? -d : d));
        }
    }
}

// ------------------------------------------------------------------ MMA
struct OzArgs {
    const GemmDesc* descs;
    const OzEntry* ents;
    const __nv_bfloat16* slices;
    long long n_slices;        // elements of the slice buffer (bounds of every bulk copy)
    const int* scale_exp;      // power-of-two scale exponents of the rows / columns
    int* err;
};

__global__ void __launch_bounds__(kOzThreads, kCtasPerSm) oz_mma_kernel(OzArgs A) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], accb[kAccBufs], accfree[kAccBufs];
    __shared__ unsigned s_tmem;
    __shared__ int s_fail;
    const int z = blockIdx.z;
    const GemmDesc D = A.descs[z];
    const OzEntry E = A.ents[z];
    const int tm = blockIdx.x % E.rta, tn = blockIdx.x / E.rta;
    if (blockIdx.x >= E.rta * E.rtb) return;                       // whole CTA: uniform
    if (D.lower && tn * kTN > tm * kTM + kTM - 1) return;          // tile above the diagonal
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int h = 0; h < kAccBufs; ++h) {
            mbar_init(&accb[h], 1);
            mbar_init(&accfree[h], kOzThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    volatile int* fail = &s_fail;
    const int slabs = E.slabs;
    const int chunks = (slabs + kChunkSlabs - 1) / kChunkSlabs;
    // the kSlices blocks of one (tile, slab) lie back to back: one bulk copy each
    // for A and B per stage
    const __nv_bfloat16* a0 = A.slices + E.a_sl + (long long)tm * slabs * kSlices * kAElems;
    const __nv_bfloat16* b0 = A.slices + E.b_sl + (long long)tn * slabs * kSlices * kBElems;
    unsigned char* stage0 = oz_smem;
    auto a_stage = [&](int st, int t) { return stage0 + (size_t)st * kStageBytes + (size_t)t * kAElems * 2; };
    auto b_stage = [&](int st, int u) {
        return stage0 + (size_t)st * kStageBytes + (size_t)kSlices * kAElems * 2 + (size_t)u * kBElems * 2;
    };
    int last_copy[kStages];        // thread 0: last slab copied into each stage
    for (int st = 0; st < kStages; ++st) last_copy[st] = -1;
    auto issue_copy = [&](int slab) {
        const int st = slab % kStages;
        last_copy[st] = slab;
        mbar_expect_tx(&full[st], kStageBytes);
        bulk_g2s(a_stage(st, 0), a0 + (long long)slab * kSlices * kAElems, kSlices * kAElems * 2, &full[st]);
        bulk_g2s(b_stage(st, 0), b0 + (long long)slab * kSlices * kBElems, kSlices * kBElems * 2, &full[st]);
    };
    const unsigned lbo = 128, sbo = kCoresK * 128;   // K-adjacent cores, 8-row groups
    int last_commit[kAccBufs];       // thread 0: last chunk committed to each accumulator set
    for (int h = 0; h < kAccBufs; ++h) last_commit[h] = -1;
    // thread 0: the MMAs of one slab, then the refill of the stage the slab before
    // it used (slab sl + kStages - 1), so that the tensor pipe always holds the
    // MMAs of the slabs already staged; false on a timed-out wait.  Slab j is the
    // (j / kStages)-th use of stage j % kStages, which sets both barriers' parities.
    auto mma_slab = [&](int sl) -> bool {
        const int chunk = sl / kChunkSlabs, first = (sl % kChunkSlabs) == 0;
        const int half = chunk % kAccBufs;   // chunk c is the (c / kAccBufs)-th use of its set
        const int st = sl % kStages;
        if (!mbar_wait_or_fail(&full[st], (unsigned)((sl / kStages) & 1), fail)) return false;
        if (first && chunk >= kAccBufs &&
            !mbar_wait_or_fail(&accfree[half], (unsigned)(((chunk - kAccBufs) / kAccBufs) & 1), fail))
            return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // one thread issues every MMA, so each costs only a few instructions: the
        // descriptors of slice t / u are the stage's first ones plus a fixed start
        // offset (the 14-bit start field of an address below 256 KB does not carry)
        // and the pair loops are unrolled into 36 MMAs with fixed diagonal offsets
        const unsigned long long da0 = smem_desc(a_stage(st, 0), lbo, sbo);
        const unsigned long long db0 = smem_desc(b_stage(st, 0), lbo, sbo);
        const unsigned dh = tmem + (unsigned)(half * (kDiag * kTN));
        // the first product of diagonal g in a chunk (t = 0 in the chunk's first slab)
        // overwrites the accumulator; every later one adds to it
        const unsigned acc0 = first ? 0u : 1u;
#pragma unroll
        for (int t = 0; t < kSlices; ++t) {
#pragma unroll
            for (int u = 0; t + u <= kSlices - 1; ++u) {   // t + u (0-based) <= kSlices - 1
#pragma unroll
                for (int ks = 0; ks < kSlabK / 16; ++ks) {   // K = 16 per MMA: two core matrices
                    const unsigned long long da = da0 + (unsigned long long)((t * kAElems * 2 + ks * 256) >> 4);
                    const unsigned long long db = db0 + (unsigned long long)((u * kBElems * 2 + ks * 256) >> 4);
                    mma_bf16(dh + (unsigned)((t + u) * kTN), da, db, (t == 0 && ks == 0) ? acc0 : 1u);
                }
            }
        }
        mma_commit(&empty[st]);
        if ((sl % kChunkSlabs) == kChunkSlabs - 1 || sl == slabs - 1) {
            mma_commit(&accb[half]);
            last_commit[half] = chunk;
        }
        const int nxt = sl + kStages - 1;
        if (nxt < slabs) {
            const int prev = sl - 1;   // nxt goes into the stage of slab sl - 1 (a fresh one for sl = 0)
            if (prev >= 0 && !mbar_wait_or_fail(&empty[prev % kStages], (unsigned)((prev / kStages) & 1), fail))
                return false;
            issue_copy(nxt);
        }
        return true;
    };
    // every thread: row (warp & 3) * 32 + lane of the tile, columns (warp >> 2) * 16 + 0..15.
    // sum_g V_g 2^(-7(g+2)) = T_hi 2^-35 + T_lo 2^-63 with T_hi = sum_{g<4} V_g 2^(7(3-g)),
    // T_lo = sum_{g>=4} V_g 2^(7(7-g)): each chunk's exact integer diagonal sums go
    // straight into the two int64 halves (|T| < 2^53 for K <= 16256)
    long long th[16], tl[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) th[c] = tl[c] = 0;
    auto readout = [&](int chunk) -> bool {
        const int half = chunk % kAccBufs;
        const bool got = mbar_wait_or_fail(&accb[half], (unsigned)((chunk / kAccBufs) & 1), fail);
        if (!__all_sync(0xffffffffu, got)) {
            *fail = 1;
            return false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int g = 0; g < kDiag; ++g) {
            unsigned r[16];
            const unsigned taddr = tmem + ((unsigned)((warp & 3) * 32) << 16) +
                                   (unsigned)(half * (kDiag * kTN) + g * kTN + (warp >> 2) * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int sh = kBeta * (3 - (g & 3));
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const long long d = (long long)__float2int_rn(__uint_as_float(r[c])) << sh;
                if (g < 4) th[c] += d;
                else tl[c] += d;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accfree[half])) : "memory");
        return true;
    };
    // every copy this CTA will issue lies inside the slice buffer: checked once,
    // before the first copy (a bad table entry fails the CTA instead of copying)
    if (tid == 0) {
        const long long a_lo = E.a_sl + (long long)tm * slabs * kSlices * kAElems;
        const long long a_hi = a_lo + (long long)slabs * kSlices * kAElems;
        const long long b_lo = E.b_sl + (long long)tn * slabs * kSlices * kBElems;
        const long long b_hi = b_lo + (long long)slabs * kSlices * kBElems;
        if (a_lo < 0 || b_lo < 0 || a_hi > A.n_slices || b_hi > A.n_slices || tm >= E.rta || tn >= E.rtb) *fail = 1;
    }
    __syncthreads();
    if (tid == 0 && !*fail)
        for (int j = 0; j < kStages - 1 && j < slabs; ++j) issue_copy(j);
    bool ok = true;   // warp-uniform
    int done_chunks = 0;
    for (int sl = 0; sl < slabs; ++sl) {
        bool f = false;
        if (tid == 0) f = !mma_slab(sl);
        if (f) *fail = 1;
        if (__any_sync(0xffffffffu, f || *fail != 0)) {
            ok = false;
            break;
        }
        // once the MMAs of a chunk are issued, read out the chunk kAccBufs - 1 before
        // it (with one accumulator set: the chunk itself, before the next may start)
        if ((sl % kChunkSlabs) == kChunkSlabs - 1 || sl == slabs - 1) {
            const int chunk = sl / kChunkSlabs - (kAccBufs - 1);
            if (chunk >= 0) {
                if (!readout(chunk)) {
                    ok = false;
                    break;
                }
                done_chunks = chunk + 1;
            }
        }
    }
    for (int c = done_chunks; ok && c < chunks; ++c)
        if (!readout(c)) ok = false;
    if (!ok) *fail = 1;
    __syncthreads();
    const bool failed = *fail != 0;
    if (failed && tid == 0) atomicExch(A.err, 1);
    if (!failed) {
        const int i = tm * kTM + (warp & 3) * 32 + lane;
        if (i < D.M) {
            const int ei = A.scale_exp[E.a_sc + i];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = tn * kTN + (warp >> 2) * 16 + c;
                if (j < D.N) {
                    // T_hi (g = 0..3) and T_lo (g = 4..7), folded chunk by chunk at the read-out,
                    // are each below 2^53 in magnitude, so both convert to FP64 exactly and the
                    // element costs two conversions and two FMAs of the FP64 pipe
                    const long long thc = th[c], tlc = tl[c];
                    const int ex = ei + A.scale_exp[E.b_sc + j];
                    double v;
                    if (ex - 63 > -1022 && ex - 35 < 1023) {   // both powers of two normal: build them
                        const double ph = __longlong_as_double((long long)(ex - 35 + 1023) << 52);
                        const double pl = __longlong_as_double((long long)(ex - 63 + 1023) << 52);
                        v = fma((double)thc, ph, (double)tlc * pl);
                    } else {
                        v = ldexp((double)thc, ex - 35) + ldexp((double)tlc, ex - 63);
                    }
                    double* cp = D.C + (long long)j * D.ldc + i;
                    *cp = (D.beta == 0.0) ? D.alpha * v : fma(D.alpha, v, D.beta * (*cp));
                }
            }
        }
    }
    if (failed && tid == 0) {
        // bounded waits for the copies and MMAs already issued, before the shared
        // and tensor memory they use is given up
        for (int st = 0; st < kStages; ++st)
            if (last_copy[st] >= 0) mbar_wait_or_fail(&full[st], (unsigned)((last_copy[st] / kStages) & 1), nullptr);
        for (int h = 0; h < kAccBufs; ++h)
            if (last_commit[h] >= 0)
                mbar_wait_or_fail(&accb[h], (unsigned)((last_commit[h] / kAccBufs) & 1), nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

bool ozaki_gemm_supported(const std::vector<GemmDesc>& h) {
    for (const GemmDesc& d : h) {
        if (d.K > kOzMaxK) return false;
        // one slice of either operand, tiled, must index with 32 bits
        const long long ka = (long long)(d.K + kSlabK - 1) / kSlabK * kSlabK;
        if ((long long)(d.M + kTM - 1) / kTM * kTM * ka >= (1LL << 31)) return false;
        if ((long long)(d.N + kTN - 1) / kTN * kTN * ka >= (1LL << 31)) return false;
    }
    return true;
}

msp_status ozaki_gemm_batched(const std::vector<GemmDesc>& h, const GemmDesc* d_dev, bool transA, bool transB,
                              cudaStream_t s, OzakiWork& w) {
    const int batch = (int)h.size();
    if (batch == 0) return MSP_OK;
    std::vector<OzEntry> ents(batch);
    long long sl = 0, sc = 0;
    int max_rows_a = 0, max_rows_b = 0, max_tiles = 0;
    long long max_a_elems = 0, max_b_elems = 0;
    for (int z = 0; z < batch; ++z) {
        const GemmDesc& d = h[z];
        OzEntry& e = ents[z];
        e = OzEntry{};
        e.rta = std::max(1, (d.M + kTM - 1) / kTM);
        e.rtb = std::max(1, (d.N + kTN - 1) / kTN);
        e.slabs = std::max(1, (d.K + kSlabK - 1) / kSlabK);
        const long long a_el = (long long)kSlices * e.rta * e.slabs * kAElems;
        const long long b_el = (long long)kSlices * e.rtb * e.slabs * kBElems;
        e.a_sl = sl;
        sl += a_el;
        e.b_sl = sl;
        sl += b_el;
        e.a_sc = sc;
        sc += e.rta * kTM;
        e.b_sc = sc;
        sc += e.rtb * kTN;
        max_rows_a = std::max(max_rows_a, d.M);
        max_rows_b = std::max(max_rows_b, d.N);
        max_tiles = std::max(max_tiles, e.rta * e.rtb);
        max_a_elems = std::max(max_a_elems, a_el / kSlices);
        max_b_elems = std::max(max_b_elems, b_el / kSlices);
    }
    const size_t ent_words = sizeof(OzEntry) / sizeof(long long) * (size_t)batch;
    const bool grow = (long long)w.slices.n < sl || (long long)w.scales.n < sc || w.ents.n < ent_words;
    // products of earlier calls may still be queued on the stream and read these
    // buffers: they finish before a buffer is given up for a larger one
    if (grow) MSP_CUDA(cudaStreamSynchronize(s));
    if ((long long)w.slices.n < sl) MSP_TRY(w.slices.alloc((size_t)sl, s));
    if ((long long)w.scales.n < sc) MSP_TRY(w.scales.alloc((size_t)sc, s));
    if (w.ents.n < ent_words) MSP_TRY(w.ents.alloc(ent_words, s));
    if (!w.err.p) {
        MSP_TRY(w.err.alloc(1, s));
        MSP_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), s));
    }
    MSP_CUDA(cudaMemcpyAsync(w.ents.p, ents.data(), sizeof(OzEntry) * batch, cudaMemcpyHostToDevice, s));
    const OzEntry* d_ents = reinterpret_cast<const OzEntry*>(w.ents.p);
    __nv_bfloat16* slices = reinterpret_cast<__nv_bfloat16*>(w.slices.p);
    for (int z0 = 0; z0 < batch; z0 += 65535) {
        const int nb = std::min(65535, batch - z0);
        oz_scale_kernel<false><<<dim3((max_rows_a + 7) / 8, nb), 256, 0, s>>>(d_dev + z0, d_ents + z0, transA, transB,
                                                                              w.scales.p, max_rows_a);
        oz_scale_kernel<true><<<dim3((max_rows_b + 7) / 8, nb), 256, 0, s>>>(d_dev + z0, d_ents + z0, transA, transB,
                                                                             w.scales.p, max_rows_b);
        const int ga = (int)std::min<long long>((max_a_elems + 255) / 256, 4096);
        const int gb = (int)std::min<long long>((max_b_elems + 255) / 256, 4096);
        oz_slice_kernel<false><<<dim3(std::max(ga, 1), nb), 256, 0, s>>>(d_dev + z0, d_ents + z0, transA, transB,
                                                                         w.scales.p, slices);
        oz_slice_kernel<true><<<dim3(std::max(gb, 1), nb), 256, 0, s>>>(d_dev + z0, d_ents + z0, transA, transB,
                                                                        w.scales.p, slices);
        count_launches(4);
        OzArgs a{};
        a.descs = d_dev + z0;
        a.ents = d_ents + z0;
        a.slices = slices;
        a.n_slices = (long long)w.slices.n;
        a.scale_exp = w.scales.p;
        a.err = w.err.p;
        const int smem = kStages * (int)kStageBytes;
        MSP_CUDA(cudaFuncSetAttribute(oz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        oz_mma_kernel<<<dim3(max_tiles, 1, nb), kOzThreads, smem, s>>>(a);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
    }
    return MSP_OK;
}

msp_status ozaki_check(OzakiWork& w, cudaStream_t s) {
    if (!w.err.p) return MSP_OK;
    int h = 0;
    MSP_CUDA(cudaMemcpyAsync(&h, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    if (h) {
        MSP_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int), s));
        set_error("tensor-core FP64 GEMM: a bounded wait timed out");
        return MSP_ERR_TIMEOUT;
    }
    return MSP_OK;
}

}  // namespace msp
