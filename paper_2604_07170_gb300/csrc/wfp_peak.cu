// Arithmetic peak of the current GPU, measured: a loop of independent fused multiply-adds in FP64
// or FP32, timed with CUDA events.  The FP64 path of the step is bound by FP64 issue, so its roofline
// divides by this measured rate rather than by a unit count times a clock.
#include <cuda_runtime.h>

#include <string>

#include "wfp.h"
#include "wfp_debug.h"
#include "wfp_internal.h"

namespace wfp {

// Each thread runs CHAINS independent FMA chains for `iters` rounds (2 flops per FMA).  The chains
// start from values the compiler cannot know and their sum is stored, so no FMA can be dropped.
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T a, T b, T* __restrict__ out) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 16
    for (int i = 0; i < iters; i++) {  // unrolled so that loop control takes few issue slots
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace wfp

extern "C" wfp_status wfp_debug_alu_peak(int fp64, double* tflops, double* ms) {
    if (!tflops || !ms) {
        wfp::set_error("outputs must be non-NULL");
        return WFP_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        wfp::set_error(std::string("alu peak: ") + cudaGetErrorString(e));
        return WFP_ECUDA;
    }
    constexpr int kChains = 8, kThreads = 256;
    const int blocks = sms * 8;
    const int iters = fp64 ? 2048 : 32768;
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {  // the first launch warms up
        cudaEventRecord(e0, cudaStreamPerThread);
        if (fp64)
            wfp::k_fma_loop<double, kChains><<<blocks, kThreads, 0, cudaStreamPerThread>>>(iters, 0.999999, 1e-7,
                                                                                           (double*)out);
        else
            wfp::k_fma_loop<float, kChains><<<blocks, kThreads, 0, cudaStreamPerThread>>>(iters, 0.999999f, 1e-7f,
                                                                                          (float*)out);
        cudaEventRecord(e1, cudaStreamPerThread);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float t = 0.f;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < best) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        wfp::set_error(std::string("alu peak: ") + cudaGetErrorString(e));
        return WFP_ECUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    *ms = best;
    *tflops = flops / (best * 1e-3) / 1e12;
    return WFP_OK;
}
