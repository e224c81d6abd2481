// Device helpers: counter-based Gaussian generator and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace msp {

// Stream tags (counter word 3) of the two sample families.
constexpr uint32_t kTagElliptic = 0x4D535045u;
constexpr uint32_t kTagKinetic = 0x4D53504Bu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications with the round multipliers, a swap of the counter words and an
// xor with the key; the key advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += kWeyl0; k1 += kWeyl1; }
        const uint32_t lo0 = kMul0 * c.x, hi0 = __umulhi(kMul0, c.x);
        const uint32_t lo1 = kMul1 * c.z, hi1 = __umulhi(kMul1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Two N(0,1) values for ring-node pair q of sample s of patch m (Box-Muller on the
// two 53-bit uniforms u1 in (0,1], u2 in [0,1)).
__device__ __forceinline__ double2 gaussian_pair(uint64_t seed, uint32_t q, uint32_t s, uint32_t m,
                                                 uint32_t tag) {
    const uint4 x = philox4x32_10(make_uint4(q, s, m, tag), (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t a = ((((uint64_t)x.y) << 32) | x.x) >> 11;
    const uint64_t b = ((((uint64_t)x.w) << 32) | x.z) >> 11;
    const double u1 = ((double)a + 1.0) * 0x1.0p-53;
    const double u2 = (double)b * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sums of NV values; every thread gets the totals.  `buf` needs
// NV * 32 entries.  Deterministic: warp partials are added in warp order.  One
// __syncthreads; callers alternate buffers between consecutive reductions.
template <class T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T w = warp_sum(v[k]);
        if (lane == 0) buf[k * 32 + warp] = w;
    }
    __syncthreads();
    // every warp adds the warp partials with the same shuffle tree
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T t = (lane < nw) ? buf[k * 32 + lane] : T(0);
        v[k] = warp_sum(t);
    }
}

}  // namespace msp
