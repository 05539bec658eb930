// dmfe_sparsify_select_noalloc: the sparsification decision of dmfe_sparsify for a
// history that the caller already holds in device memory, computed without allocating
// anything.
//
// Who needs it: code that cannot call cudaMalloc -- a process in which another
// framework has reserved the device memory up front (an extra cudaMalloc would fail or
// fragment its pool), or a latency-critical loop that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree may imply. Such a caller has no dmfe_solver
// (creating one allocates), so this entry point takes the history arrays directly.
//
// The per-slice residuals need scratch memory beyond the inputs and outputs. It lives in
// one file-scope device array of fixed size, g_sp_scratch, which every GPU that loads
// this library holds until the process exits. Host code cannot use the array's name as
// a device address: every call made outside stream capture looks the address up with
// cudaGetSymbolAddress (with the device current) and caches it per device; a call inside a
// capture uses the cached address. A device reset reloads the module (the array may move),
// and the next call outside capture picks up the new address.
#include <cuda_runtime.h>

#include <mutex>

#include "dmfe_internal.h"

namespace {

static __device__ __align__(256) double g_sp_scratch[DMFE_NOALLOC_MAX_SLICES];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of g_sp_scratch on the current device: looked up again unless `stream`
// is capturing (then the address cached by an earlier call on this device is used).
int scratch_address(cudaStream_t stream, double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DMFE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DMFE_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return DMFE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sp_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DMFE_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return DMFE_OK;
}


// eps_sparse(k) for candidates k = 1 .. n-12 (Sec. 3.6), one CTA per candidate (CTA b takes
// k = b + 1); the same per-thread order, warp butterfly and warp-order sum as the solver's
// residual kernel, so the residuals are the same numbers.
constexpr int kNaResThreads = 128;

__global__ void __launch_bounds__(kNaResThreads) k_na_residual(const double* __restrict__ t,
                                                              const double* __restrict__ C,
                                                              const double* __restrict__ dC,
                                                              const double* __restrict__ R,
                                                              const double* __restrict__ dR, int n, int L,
                                                              double* __restrict__ eps) {
    const int k = blockIdx.x + 1;
    if (k > n - 12) return;
    const double h1 = t[k] - t[k - 1], h2 = t[k + 1] - t[k];
    const size_t a = (size_t)(k - 1) * L, b = (size_t)k * L, c = (size_t)(k + 1) * L;
    const SpWeights wt = sp_weights(h1, h2);
    double acc = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        acc += fabs(sp_delta(wt, C[a + i], dC[a + i], C[b + i], dC[b + i], C[c + i], dC[c + i])) +
               fabs(sp_delta(wt, R[a + i], dR[a + i], R[b + i], dR[b + i], R[c + i], dR[c + i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double wsum[kNaResThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e += wsum[w];
        eps[k] = e;
    }
}

// Greedy selection: remove k if eps(k) < tol/10 and skip k+1; if nothing qualifies,
// remove the candidate with the smallest residual. Writes removed[0..n).
__global__ void k_na_select(const double* __restrict__ eps, int n, double tol, int* __restrict__ removed) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = 0; k < n; ++k) removed[k] = 0;
    const int last = n - 12;
    if (last < 1) return;
    int count = 0;
    for (int k = 1; k <= last;) {
        if (eps[k] < tol / 10.0) {
            removed[k] = 1;
            ++count;
            k += 2;
        } else {
            ++k;
        }
    }
    if (count == 0) {
        int m = 1;
        for (int k = 2; k <= last; ++k)
            if (eps[k] < eps[m]) m = k;
        removed[m] = 1;
    }
}

}  // namespace

extern "C" int dmfe_sparsify_select_noalloc(const double* t_dev, const double* C_dev, const double* dC_dev,
                                            const double* R_dev, const double* dR_dev, int n, int L, double tol,
                                            int* removed_dev, void* stream) {
    if (!t_dev || !C_dev || !dC_dev || !R_dev || !dR_dev || !removed_dev) return DMFE_ERR_ARG;
    if (n < 1 || L < 1 || !(tol > 0.0)) return DMFE_ERR_ARG;
    if (n > DMFE_NOALLOC_MAX_SLICES) return DMFE_ERR_ARG;  // beyond the fixed scratch array
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* eps = nullptr;
    int rc = scratch_address(s, &eps);
    if (rc) return rc;
    k_na_residual<<<n > 13 ? n - 12 : 1, kNaResThreads, 0, s>>>(t_dev, C_dev, dC_dev, R_dev, dR_dev, n, L, eps);
    k_na_select<<<1, 32, 0, s>>>(eps, n, tol, removed_dev);
    if (cudaGetLastError() != cudaSuccess) return DMFE_ERR_CUDA;
    return DMFE_OK;
}
