// Evaluation of the library's own FP32 elementary kernels beside CUDA's
// functions on caller arrays, so that tests can hold them to an error bound:
// the Newton-refined reciprocal square root and reciprocal used by the pair
// kernels, and the cancellation-free erf(alpha r)/r radial kernel (Maclaurin
// series with the downward recursion) used by the intramolecular Ewald
// exclusions.
#include "sibfa_internal.cuh"

using namespace sibfa;

namespace {

// fn 0: out[2k] = rsqrt_(x), out[2k+1] = rsqrtf(x)
// fn 1: out[2k] = rcp_(x),   out[2k+1] = 1.0f / x (IEEE division)
// fn 2: x = r;  out[5k..5k+3] = g_0..g_3 of erf(alpha r)/r, out[5k+4] = erff(alpha r) / r
__global__ void k_math(int fn, int n, const float *x, float alpha, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float v = x[k];
    if (fn == 0) {
        out[2 * k] = rsqrt_<float>(v);
        out[2 * k + 1] = rsqrtf(v);
    } else if (fn == 1) {
        out[2 * k] = rcp_<float>(v);
        out[2 * k + 1] = 1.0f / v;
    } else {
        float g[4];
        g_erf_s<float, 3>(v * v, alpha, g);
        for (int j = 0; j < 4; ++j) out[5 * k + j] = g[j];
        out[5 * k + 4] = erff(alpha * v) / v;
    }
}

}  // namespace

extern "C" sibfa_status sibfa_math_selftest(int fn, int n, const float *x, float alpha, float *out, void *stream) {
    if (fn < 0 || fn > 2 || n < 0 || (n > 0 && (!x || !out))) return SIBFA_E_INVALID;
    if (n == 0) return SIBFA_OK;
    k_math<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(fn, n, x, alpha, out);
    return cudaGetLastError() == cudaSuccess ? SIBFA_OK : SIBFA_E_CUDA;
}
