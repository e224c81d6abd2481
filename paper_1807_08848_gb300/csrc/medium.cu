// Face coefficients of the medium on the fine grid (Sec. 5, a(x, x/eps)).
#include "internal.h"

#include <cmath>

namespace msp {

namespace {

struct MediumParams {
    int kind, N;
    double eps;
    int n_modes;
    const double* modes;   // device [n_modes][4]
    double amp, norm;
    int n_channels;
    const double* channels;  // device [n][3]
    double width, contrast;
};

__device__ double medium_at(const MediumParams& P, double x, double y) {
    const double twopi = 6.283185307179586476925286766559;
    switch (P.kind) {
        case MSP_MEDIUM_PERIODIC_SIN:
            return 2.0 + sin(twopi * x / P.eps) * sin(twopi * y / P.eps);
        case MSP_MEDIUM_HOU_WU:
            return 2.0 + sin(twopi * x) * cos(twopi * y) +
                   (2.0 + 1.8 * sin(twopi * x / P.eps)) / (2.0 + 1.8 * cos(twopi * y / P.eps)) +
                   (2.0 + sin(twopi * y / P.eps)) / (2.0 + 1.8 * cos(twopi * x / P.eps));
        case MSP_MEDIUM_LOGNORMAL: {
            double g = 0.0;
            for (int q = 0; q < P.n_modes; ++q) {
                const double* md = P.modes + 4 * q;
                double s, c;
                sincos(twopi * (md[0] * x + md[1] * y), &s, &c);
                g += md[2] * c + md[3] * s;
            }
            return exp(P.amp * P.norm * g);
        }
        case MSP_MEDIUM_CHANNELS: {
            bool inside = false;
            for (int q = 0; q < P.n_channels; ++q) {
                const double* ch = P.channels + 3 * q;
                double s, c;
                sincos(ch[2], &s, &c);
                const double dist = fabs(-(x - ch[0]) * s + (y - ch[1]) * c);
                inside |= dist <= 0.5 * P.width;
            }
            return inside ? P.contrast : 1.0;
        }
        default:
            return 0.0;
    }
}

// One thread per face.  Faces 0 .. (N+1)N-1 are aE[j][i] (x-faces), the rest aN[j][i].
__global__ void face_coefficients_kernel(MediumParams P, double* aE, double* aN, float* aE32, float* aN32) {
    const long long nE = (long long)(P.N + 1) * P.N;
    const long long total = 2 * nE;
    const double h = 1.0 / P.N;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < total;
         f += (long long)gridDim.x * blockDim.x) {
        double a;
        if (f < nE) {
            const int j = (int)(f / P.N), i = (int)(f % P.N);
            a = medium_at(P, (i + 0.5) * h, j * h);
            aE[f] = a;
            aE32[f] = (float)a;
        } else {
            const long long g = f - nE;
            const int j = (int)(g / (P.N + 1)), i = (int)(g % (P.N + 1));
            a = medium_at(P, i * h, (j + 0.5) * h);
            aN[g] = a;
            aN32[g] = (float)a;
        }
    }
}

__global__ void to_float_kernel(const double* src, float* dst, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}

}  // namespace

msp_status launch_medium_coefficients(Medium& M, const msp_medium_desc& d, cudaStream_t s) {
    const int N = M.N;
    const size_t nE = (size_t)(N + 1) * N;
    MSP_TRY(M.aE.alloc(nE, s));
    MSP_TRY(M.aN.alloc(nE, s));
    MSP_TRY(M.aE32.alloc(nE, s));
    MSP_TRY(M.aN32.alloc(nE, s));
    const int threads = 256;
    const int blocks = (int)std::min<long long>((2 * (long long)nE + threads - 1) / threads, 152LL * 32);
    if (d.kind == MSP_MEDIUM_USER) {
        MSP_CUDA(cudaMemcpyAsync(M.aE.p, d.user_aE_host, nE * sizeof(double), cudaMemcpyHostToDevice, s));
        MSP_CUDA(cudaMemcpyAsync(M.aN.p, d.user_aN_host, nE * sizeof(double), cudaMemcpyHostToDevice, s));
        to_float_kernel<<<blocks, threads, 0, s>>>(M.aE.p, M.aE32.p, (long long)nE);
        count_launches(1);
        to_float_kernel<<<blocks, threads, 0, s>>>(M.aN.p, M.aN32.p, (long long)nE);
        count_launches(1);
        MSP_CUDA(cudaGetLastError());
        MSP_CUDA(cudaStreamSynchronize(s));   // the host arrays are borrowed for this call only
        return MSP_OK;
    }
    DevBuf<double> modes, chans;
    MediumParams P{};
    P.kind = d.kind;
    P.N = N;
    P.eps = d.eps;
    P.amp = d.amp;
    P.norm = d.norm;
    P.width = d.width;
    P.contrast = d.contrast;
    if (d.kind == MSP_MEDIUM_LOGNORMAL && d.n_modes > 0) {
        MSP_TRY(modes.alloc((size_t)4 * d.n_modes, s));
        MSP_CUDA(cudaMemcpyAsync(modes.p, d.modes_host, sizeof(double) * 4 * d.n_modes, cudaMemcpyHostToDevice, s));
        P.n_modes = d.n_modes;
        P.modes = modes.p;
    }
    if (d.kind == MSP_MEDIUM_CHANNELS && d.n_channels > 0) {
        MSP_TRY(chans.alloc((size_t)3 * d.n_channels, s));
        MSP_CUDA(cudaMemcpyAsync(chans.p, d.channels_host, sizeof(double) * 3 * d.n_channels, cudaMemcpyHostToDevice, s));
        P.n_channels = d.n_channels;
        P.channels = chans.p;
    }
    face_coefficients_kernel<<<blocks, threads, 0, s>>>(P, M.aE.p, M.aN.p, M.aE32.p, M.aN32.p);
    count_launches(1);
    MSP_CUDA(cudaGetLastError());
    MSP_CUDA(cudaStreamSynchronize(s));   // temporaries below are freed on return
    return MSP_OK;
}

}  // namespace msp
