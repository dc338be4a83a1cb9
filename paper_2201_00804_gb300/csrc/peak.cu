// CUDA-core arithmetic peak of the device the library runs on: a kernel of
// independent fused multiply-add chains (FP32 or FP64), long enough to hide
// launch overhead, timed with CUDA events.  The pair kernels of this library
// are FP32 CUDA-core work, so their roofline is this rate, not a tensor-core
// or memory figure.
#include <cstdio>
#include <string>

#include "sibfa.h"

namespace {

constexpr int PK_CHAINS = 8;    // independent FMA chains per thread (covers the FMA latency)
constexpr int PK_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b, T *out) {
    T x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    // a store the compiler cannot drop; a and b keep every value finite
    if (s == T(-1.2345e30)) out[blockIdx.x] = s;
    if (threadIdx.x == 0 && blockIdx.x == 0) out[gridDim.x] = s;
}

template <typename T>
sibfa_status run(int iters, int blocks, double *ms, double *flops, std::string &err) {
    T *out = nullptr;
    if (cudaMalloc(&out, (blocks + 1) * sizeof(T)) != cudaSuccess) {
        err = "cudaMalloc failed";
        return SIBFA_E_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    k_fma_chains<T><<<blocks, 256>>>(iters / 8 + 1, a, b, out);   // warm-up
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, 256>>>(iters, a, b, out);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return SIBFA_E_CUDA;
    }
    *ms = t;
    *flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * 256.0 * blocks;
    return SIBFA_OK;
}

thread_local std::string g_peak_error = "no error";

}  // namespace

extern "C" sibfa_status sibfa_alu_peak(int fp64, int iters, int blocks, double *ms, double *flops) {
    if (!ms || !flops || iters < 1 || blocks < 1) {
        g_peak_error = "sibfa_alu_peak: bad argument";
        return SIBFA_E_INVALID;
    }
    return fp64 ? run<double>(iters, blocks, ms, flops, g_peak_error)
                : run<float>(iters, blocks, ms, flops, g_peak_error);
}

extern "C" const char *sibfa_alu_peak_error(void) { return g_peak_error.c_str(); }
