// dc_fma_peak: the FMA throughput of this GPU's CUDA cores in FP64 or FP32,
// measured with a kernel of independent fused multiply-add chains.  It is the
// denominator of the roofline fraction of the ALU-bound kernels (the supernodal
// substitution in FP64, the multifrontal factorisation in FP32); no clock or
// power setting is touched, so it reports what the GPU gives at its current
// clocks.
#include <cuda_runtime.h>

#include <string>

#include "dc_internal.h"

namespace {

constexpr int CHAINS = 8;        // independent accumulators per thread (hides the FMA latency)
constexpr int THREADS = 256;

template <class T>
__global__ void __launch_bounds__(THREADS) k_fma_chains(T* __restrict__ out, int n_iter, T a, T b) {
    T acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < n_iter; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) acc[c] = acc[c] * a + b;
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    // a data-dependent store keeps the chains alive; the value is never read
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
dc_status measure(int n_iter, double* tflops, std::string& err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    T* out = nullptr;
    auto fail = [&](cudaError_t e) {
        err = cudaGetErrorString(e);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (out) cudaFree(out);
        cudaGetLastError();
        return DC_ERR_CUDA;
    };
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, THREADS, 0);
    if (e != cudaSuccess) return fail(e);
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    if ((e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * THREADS)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) return fail(e);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_chains<T><<<blocks, THREADS>>>(out, n_iter / 4 + 1, a, b);   // warm-up
    dc_note_launch();
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, THREADS>>>(out, n_iter, a, b);
        dc_note_launch();
        cudaEventRecord(e1);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail(e);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    const double flops = 2.0 * CHAINS * 16.0 * (double)n_iter * blocks * THREADS;
    *tflops = flops / (best * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return DC_OK;
}

std::string g_peak_err;

}  // namespace

extern "C" dc_status dc_fma_peak(int32_t precision, int32_t n_iter, double* tflops) {
    if (!tflops || (precision != 32 && precision != 64) || n_iter < 1) {
        g_peak_err = "dc_fma_peak: precision must be 32 or 64, n_iter >= 1";
        return DC_ERR_INVALID;
    }
    return precision == 64 ? measure<double>(n_iter, tflops, g_peak_err) : measure<float>(n_iter, tflops, g_peak_err);
}
