// es_probe.cu -- es_alu_peak: measured fused multiply-add throughput of the
// current device, the denominator of the arithmetic roofline of kernels that
// are bound by their FP64 or FP32 pipe rather than by HBM (instrumentation;
// the paper has no counterpart).
//
// Every thread runs kChains independent FMA recurrences a = a * m + k in
// registers for `iters` rounds (no memory traffic inside the loop), and
// writes one sum at the end so that nothing is optimised away.  The grid
// fills every SM with several resident blocks.  Timed with CUDA events on a
// private stream after one warm-up launch; flops = 2 per FMA.
#include <cuda_runtime.h>

#include "es_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T m, T k, int iters, T* out) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fma(a[c], m, k);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <class T>
int run(double* gflops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess) {
        cudaGetLastError();
        return ES_ECUDA;
    }
    const int blocks = nsm * 8;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    T* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = ES_OK;
    float ms = 0.0f;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
        rc = ES_ECUDA;
    } else {
        // (m just below one and a small k keep every chain finite)
        const T m = (T)0.9999, k = (T)1e-4;
        k_fma_chains<T><<<blocks, kThreads, 0, st>>>(m, k, iters / 8, out);
        cudaEventRecord(a, st);
        k_fma_chains<T><<<blocks, kThreads, 0, st>>>(m, k, iters, out);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.0f)
            rc = ES_ECUDA;
    }
    if (rc == ES_OK) *gflops = 2.0 * (double)blocks * kThreads * kChains * (double)iters / ((double)ms * 1e6);
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}

}  // namespace

extern "C" int es_alu_peak(int precision, double* gflops) {
    if (!gflops) return ES_EINVAL;
    if (precision == ES_FP64) return run<double>(gflops);
    if (precision == ES_MIXED32) return run<float>(gflops);
    return ES_EINVAL;
}
