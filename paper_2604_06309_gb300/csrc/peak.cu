// dmfe_fma_rate: the FP64 or FP32 fused multiply-add rate of this GPU, measured, for the
// denominators of the arithmetic rooflines of the history-integral kernels (the FP64
// kernel is bound by the FP64 pipe; the double-float and FP32 kernels by the FP32 pipes).
//
// Every thread runs NCH independent FMA chains a = a * b + c (b, c kernel arguments, so
// nothing is folded at compile time) and writes its sum, so no chain is dead code. The
// grid is four CTAs of 256 threads per SM. One launch is timed with CUDA events on a
// private stream after a calibration launch has sized it to about 80 ms; the best of
// three is kept. Nothing about the GPU's clocks or settings is touched.
#include <cuda_runtime.h>

#include "dmfe_internal.h"

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaCtasPerSm = 4;

template <typename T, int NCH>
__global__ void __launch_bounds__(kFmaThreads) k_fma_loop(T b, T c, int iters, T* __restrict__ out) {
    T a[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < NCH; ++k) a[k] = fma(a[k], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int NCH>
int measure(double* gflops) {
    int dev = 0, nsm = 0;
    DMFE_CUDA_TRY(cudaGetDevice(&dev));
    DMFE_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * kFmaCtasPerSm;
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * kFmaThreads * sizeof(T)) != cudaSuccess) return DMFE_ERR_OOM;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DMFE_OK;
    double best = 0.0;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DMFE_ERR_CUDA;
    } else {
        const T b = (T)0.9999999, c = (T)1e-7;
        int iters = 64;
        // calibration (also the warm-up): scale the iteration count to about 80 ms
        for (int pass = 0; pass < 2 && rc == DMFE_OK; ++pass) {
            cudaEventRecord(e0, s);
            k_fma_loop<T, NCH><<<grid, kFmaThreads, 0, s>>>(b, c, iters, out);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = DMFE_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            double scale = ms > 0.f ? 80.0 / ms : 1000.0;
            scale = scale > 1000.0 ? 1000.0 : scale;
            long long nit = (long long)(iters * scale);
            iters = (int)(nit < 64 ? 64 : (nit > (1 << 26) ? (1 << 26) : nit));
        }
        for (int rep = 0; rep < 3 && rc == DMFE_OK; ++rep) {
            cudaEventRecord(e0, s);
            k_fma_loop<T, NCH><<<grid, kFmaThreads, 0, s>>>(b, c, iters, out);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = DMFE_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * 8.0 * NCH * (double)iters * grid * kFmaThreads;
            const double r = ms > 0.f ? flops / (ms * 1e-3) / 1e9 : 0.0;
            best = r > best ? r : best;
        }
        if (rc == DMFE_OK && cudaGetLastError() != cudaSuccess) rc = DMFE_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    if (rc == DMFE_OK) *gflops = best;
    return rc;
}

}  // namespace

extern "C" int dmfe_fma_rate(int bits, double* gflops) {
    if (!gflops) return DMFE_ERR_ARG;
    if (bits == 64) return measure<double, 8>(gflops);
    if (bits == 32) return measure<float, 16>(gflops);
    return DMFE_ERR_ARG;
}
