// Matrix-free 5-point operator applied to stacks of patch tiles (the operator of
// the local problems of Sec. 5 under the finite-difference reading: (A u)_ij =
// sum over the faces f of node (i, j) of a_f (u_ij - u_nbr(f)), a_f at the face
// midpoint).  This is the streaming form of the operator: every sample tile is
// read from and written to HBM once, the face coefficients of a patch are staged
// once per CTA and shared by all its samples.
//
// One CTA per (patch, chunk of samples).  The patch's faces go to shared memory
// with ordinary loads; the sample tiles arrive by one bulk asynchronous copy each
// (cp.async.bulk, the TMA engine), double-buffered and completed on an mbarrier,
// so the next tile is in flight while the current one is computed.  Every
// mbarrier wait is bounded: on timeout the CTA raises *err and leaves.
#include "internal.h"

namespace msp {

namespace {

struct StencilArgs {
    int N;
    const void* aE;
    const void* aN;
    const PatchDev* patches;
    int n_patches, S, chunk;
    int H, P;                  // tile rows, row pitch (elements, multiple of 4)
    const void* x;
    void* y;
    int* err;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
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

template <class T>
struct Vec4;
template <>
struct Vec4<float> {
    float v[4];
    __device__ __forceinline__ void load(const float* p) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ __forceinline__ void store(float* p) const {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec4<double> {
    double v[4];
    __device__ __forceinline__ void load(const double* p) {
        const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void store(double* p) const {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};

// FP32: the patch's faces and three sample tiles in shared memory (two copies in
// flight while one tile is computed).  FP64 (twice the bytes): two sample tiles,
// the faces read through L1.  Each thread computes four consecutive nodes of a
// row from vector loads of shared memory and writes them with one vector store.
template <class T>
__global__ void __launch_bounds__(512) stencil_apply_kernel(StencilArgs A) {
    constexpr bool kFacesInSmem = sizeof(T) == 4;
    constexpr int NB = kFacesInSmem ? 3 : 2;   // sample-tile buffers
    extern __shared__ __align__(128) unsigned char st_smem[];
    __shared__ __align__(8) unsigned long long bar[NB];
    __shared__ int s_fail;
    const int per = (A.S + A.chunk - 1) / A.chunk;
    const int m = blockIdx.x / A.chunk;
    const int s0 = (blockIdx.x % A.chunk) * per;
    const int s1 = min(A.S, s0 + per);
    if (m >= A.n_patches || s0 >= s1) return;
    const PatchDev Pd = A.patches[m];
    const int W = Pd.X1 - Pd.X0 + 1, Hm = Pd.Y1 - Pd.Y0 + 1;
    const int H = A.H, P = A.P, N = A.N;
    const long long tile = (long long)H * P;
    T* cE = reinterpret_cast<T*>(st_smem);   // east face of node (r, c): between c and c + 1
    T* cN = cE + tile;                       // north face of node (r, c): between r and r + 1
    T* xb = kFacesInSmem ? cN + tile : reinterpret_cast<T*>(st_smem);
    const T* aE = static_cast<const T*>(A.aE);
    const T* aN = static_cast<const T*>(A.aN);
    const T* X = static_cast<const T*>(A.x);
    T* Y = static_cast<T*>(A.y);
    const unsigned bytes = (unsigned)(tile * sizeof(T));
    const long long base = ((long long)m * A.S) * tile;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        for (int b = 0; b < NB - 1 && s0 + b < s1; ++b) {
            mbar_expect_tx(&bar[b], bytes);
            bulk_g2s(xb + b * tile, X + base + (long long)(s0 + b) * tile, bytes, &bar[b]);
        }
    }
    if constexpr (kFacesInSmem) {
        for (long long e = threadIdx.x; e < tile; e += blockDim.x) {
            const int r = (int)(e / P), c = (int)(e % P);
            const int j = Pd.Y0 + r, i = Pd.X0 + c;
            cE[e] = (r < Hm && c < W - 1) ? aE[(long long)j * N + i] : T(0);
            cN[e] = (r < Hm - 1 && c < W) ? aN[(long long)j * (N + 1) + i] : T(0);
        }
    }
    __syncthreads();
    const int quads = P / 4;
    const int nq = H * quads;
    for (int s = s0, it = 0; s < s1; ++s, ++it) {
        const int buf = it % NB;
        const unsigned parity = (unsigned)((it / NB) & 1);
        if (threadIdx.x == 0 && s + NB - 1 < s1) {   // that buffer was released by the barrier ending the last pass
            const int nb = (it + NB - 1) % NB;
            mbar_expect_tx(&bar[nb], bytes);
            bulk_g2s(xb + nb * tile, X + base + (long long)(s + NB - 1) * tile, bytes, &bar[nb]);
        }
        if (threadIdx.x == 0 && !mbar_wait(&bar[buf], parity)) {
            s_fail = 1;
            atomicExch(A.err, 1);
            // bounded waits for the copies issued into the other buffers before leaving
            for (int d = 1; d < NB && s + d < s1; ++d) mbar_wait(&bar[(it + d) % NB], (unsigned)(((it + d) / NB) & 1));
        }
        __syncthreads();
        if (s_fail) return;
        if (threadIdx.x != 0) mbar_wait(&bar[buf], parity);   // complete already: returns at once
        const T* x = xb + buf * tile;
        T* yt = Y + base + (long long)s * tile;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            const int r = q / quads, c0 = (q - r * quads) * 4;
            const int e0 = r * P + c0;
            Vec4<T> out;
            out.v[0] = out.v[1] = out.v[2] = out.v[3] = T(0);
            if (r >= 1 && r < Hm - 1 && c0 < W - 1 && c0 + 3 >= 1) {
                Vec4<T> xc, xu, xd, ce, cn, cs;
                xc.load(x + e0);
                xu.load(x + e0 + P);
                xd.load(x + e0 - P);
                const T xl = c0 > 0 ? x[e0 - 1] : T(0);
                const T xr = c0 + 4 < P ? x[e0 + 4] : T(0);
                T cw;
                if constexpr (kFacesInSmem) {
                    ce.load(cE + e0);
                    cn.load(cN + e0);
                    cs.load(cN + e0 - P);
                    cw = c0 > 0 ? cE[e0 - 1] : T(0);
                } else {
                    const T* gE = aE + (long long)(Pd.Y0 + r) * N + Pd.X0;
                    const T* gN = aN + (long long)(Pd.Y0 + r) * (N + 1) + Pd.X0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int c = c0 + t;
                        ce.v[t] = (c < W - 1) ? __ldg(gE + c) : T(0);
                        cn.v[t] = (c < W) ? __ldg(gN + c) : T(0);
                        cs.v[t] = (c < W) ? __ldg(gN - (N + 1) + c) : T(0);
                    }
                    cw = c0 > 0 ? __ldg(gE + c0 - 1) : T(0);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = c0 + t;
                    const T left = t == 0 ? xl : xc.v[t - 1];
                    const T right = t == 3 ? xr : xc.v[t + 1];
                    const T fw = t == 0 ? cw : ce.v[t - 1];
                    const T v = ce.v[t] * (xc.v[t] - right) + fw * (xc.v[t] - left) + cn.v[t] * (xc.v[t] - xu.v[t]) +
                                cs.v[t] * (xc.v[t] - xd.v[t]);
                    out.v[t] = (c >= 1 && c < W - 1) ? v : T(0);
                }
            }
            out.store(yt + e0);
        }
        __syncthreads();
    }
}

}  // namespace

msp_status apply_operator(const Medium& M, int S, int precision, const void* x, void* y, int pitch, int rows,
                          cudaStream_t s, double* ms_out) {
    int maxW = 0, maxH = 0;
    for (const PatchDev& P : M.patches) {
        maxW = std::max(maxW, P.X1 - P.X0 + 1);
        maxH = std::max(maxH, P.Y1 - P.Y0 + 1);
    }
    if (pitch < maxW || pitch % 4 != 0 || rows < maxH) {
        set_error("msp_apply_operator: pitch must be a multiple of 4 >= the widest tile and rows >= the tallest");
        return MSP_ERR_INVALID_ARG;
    }
    const bool f32 = precision == MSP_MIXED;
    if (f32 && !M.aE32.p) {
        set_error("msp_apply_operator: the medium has no FP32 coefficients");
        return MSP_ERR_INVALID_ARG;
    }
    const size_t esz = f32 ? sizeof(float) : sizeof(double);
    const size_t smem = (f32 ? 5 : 2) * (size_t)rows * pitch * esz;
    if (smem > 227 * 1024 - 256) {
        set_error("msp_apply_operator: the staged tiles of this shape exceed shared memory");
        return MSP_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(x) & 15) != 0) {
        set_error("msp_apply_operator: x must be 16-byte aligned");
        return MSP_ERR_INVALID_ARG;
    }
    DevBuf<int> err;
    MSP_TRY(err.alloc(1, s));
    MSP_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    StencilArgs A{};
    A.N = M.N;
    A.aE = f32 ? (const void*)M.aE32.p : (const void*)M.aE.p;
    A.aN = f32 ? (const void*)M.aN32.p : (const void*)M.aN.p;
    A.patches = M.patches_dev.p;
    A.n_patches = (int)M.patches.size();
    A.S = S;
    // sample chunks per patch: at least about eight waves of CTAs (one CTA per SM
    // fits in shared memory), each chunk at least 16 samples to amortise the faces
    A.chunk = std::max(1, std::min(std::max(1, S / 16), (8 * num_sms() + A.n_patches - 1) / std::max(A.n_patches, 1)));
    A.H = rows;
    A.P = pitch;
    A.x = x;
    A.y = y;
    A.err = err.p;
    const int grid = A.n_patches * A.chunk;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        MSP_CUDA(cudaEventCreate(&e0));
        MSP_CUDA(cudaEventCreate(&e1));
        MSP_CUDA(cudaEventRecord(e0, s));
    }
    if (f32) {
        MSP_CUDA(cudaFuncSetAttribute(stencil_apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        stencil_apply_kernel<float><<<grid, 512, smem, s>>>(A);
    } else {
        MSP_CUDA(cudaFuncSetAttribute(stencil_apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        stencil_apply_kernel<double><<<grid, 512, smem, s>>>(A);
    }
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    if (ms_out) {
        MSP_CUDA(cudaEventRecord(e1, s));
        MSP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MSP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        *ms_out = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int herr = 0;
    MSP_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSP_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("msp_apply_operator: a tile copy did not complete in time");
        return MSP_ERR_TIMEOUT;
    }
    return MSP_OK;
}

}  // namespace msp

using namespace msp;

extern "C" msp_status msp_operator_tile_shape(msp_medium m, int* rows, int* cols) {
    clear_error();
    MSP_CHECK_ARG(m && rows && cols, "msp_operator_tile_shape: NULL argument");
    int W = 0, H = 0;
    for (const PatchDev& P : m->M.patches) {
        W = std::max(W, P.X1 - P.X0 + 1);
        H = std::max(H, P.Y1 - P.Y0 + 1);
    }
    *rows = H;
    *cols = W;
    return MSP_OK;
}

extern "C" msp_status msp_apply_operator(msp_medium m, int samples, int precision, const void* x_dev, void* y_dev,
                                         int pitch, int rows, double* ms_out, void* stream) {
    clear_error();
    MSP_CHECK_ARG(m && x_dev && y_dev, "msp_apply_operator: NULL argument");
    MSP_CHECK_ARG(samples >= 1, "msp_apply_operator: samples must be >= 1");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_apply_operator: unknown precision");
    return apply_operator(m->M, samples, precision, x_dev, y_dev, pitch, rows, (cudaStream_t)stream, ms_out);
}
