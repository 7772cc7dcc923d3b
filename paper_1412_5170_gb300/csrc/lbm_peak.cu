// lbm_peak.cu -- lbm_fma_peak: the fused multiply-add throughput of this GPU
// in FP64 or FP32, measured with a kernel of independent FMA chains and
// CUDA events.  It is the roofline of the FP64 step, which is bound by
// double-precision arithmetic rather than by HBM on this GPU (the FP64 pipe
// is a small fraction of the FP32 one); the FP32 figure is given alongside.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbm.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kIters = 4096;      // iterations per launch

// Each thread runs kChains dependent chains x <- x * a + b side by side; the
// results feed a guard store that no run takes (it only keeps the compiler
// from dropping the loop).
template <typename T>
__global__ void __launch_bounds__(256) k_fma(T a, T b, T* __restrict__ sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-12345.678)) sink[blockIdx.x] = s;
}

template <typename T>
int measure(double* tflops)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LBM_E_CUDA;
    const int blocks = nsm * 8, threads = 256;
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = LBM_E_CUDA;
    if (cudaMalloc(&sink, sizeof(T) * blocks) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        // a = 1 - 2^-20, b = 2^-20: the chains stay bounded and normal
        const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
        k_fma<T><<<blocks, threads>>>(a, b, sink);   // warm-up (clocks, module load)
        float best = 3.4e38f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0);
            k_fma<T><<<blocks, threads>>>(a, b, sink);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        if (cudaGetLastError() == cudaSuccess && best < 3.4e38f) {
            const double flops = 2.0 * kChains * double(kIters) * blocks * threads;
            *tflops = flops / (best * 1e-3) / 1e12;
            status = LBM_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return status;
}

}  // namespace

extern "C" int lbm_fma_peak(int precision, double* tflops)
{
    if (!tflops || (precision != LBM_FP64 && precision != LBM_FP32_DEV)) return LBM_E_INVALID;
    return precision == LBM_FP64 ? measure<double>(tflops) : measure<float>(tflops);
}
