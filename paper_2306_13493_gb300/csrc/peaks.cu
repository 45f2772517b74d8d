// Machine peaks for the kernels that HBM bandwidth does not bound, measured on
// the device itself: the FP32 FMA issue rate (the bound of the row FFT pass,
// whose Philox rounds, Box-Muller and butterflies are arithmetic) and the L2
// read bandwidth (the bound of kernels whose data stay in L2: the one-block
// solvers' inputs, the coarse multigrid tail, the reductions).
//
// Both kernels only launch; the caller times them with CUDA events on the
// stream it passes.  Instrumentation of the library, not a step of the method.
#include "sce_internal.cuh"

namespace {

// Eight independent FMA chains per thread, unrolled, so every scheduler has
// an FMA ready each cycle once a few warps are resident.  The result is
// stored only if it equals a value it cannot take (keeps the chains live).
__global__ void __launch_bounds__(256) peak_fma_kernel(float *out, int iters, float a, float b) {
    float x0 = threadIdx.x * 1e-7f, x1 = x0 + 1e-7f, x2 = x0 + 2e-7f, x3 = x0 + 3e-7f;
    float x4 = x0 + 4e-7f, x5 = x0 + 5e-7f, x6 = x0 + 6e-7f, x7 = x0 + 7e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fmaf(x0, a, b);
            x1 = fmaf(x1, a, b);
            x2 = fmaf(x2, a, b);
            x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b);
            x5 = fmaf(x5, a, b);
            x6 = fmaf(x6, a, b);
            x7 = fmaf(x7, a, b);
        }
    }
    const float s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == -12345.0f) out[blockIdx.x] = s;
}

// Every thread reads float4s of the buffer with a grid stride, `reps` times,
// through L2 only (ld.global.cg); four loads in flight per thread.
__global__ void __launch_bounds__(256) peak_l2_kernel(const float4 *__restrict__ buf, long long n4,
                                                     int reps, float *out) {
    float ax = 0.f, ay = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < reps; ++r) {
        long long i = t;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const float4 v0 = __ldcg(buf + i), v1 = __ldcg(buf + i + stride);
            const float4 v2 = __ldcg(buf + i + 2 * stride), v3 = __ldcg(buf + i + 3 * stride);
            ax += (v0.x + v1.x) + (v2.x + v3.x);
            ay += (v0.w + v1.w) + (v2.w + v3.w);
        }
        for (; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            ax += v.x;
            ay += v.w;
        }
    }
    if (ax + ay == -12345.0f) out[blockIdx.x] = ax;
}

}  // namespace

extern "C" int sce_peak_fma(float *out, int blocks, int iters, void *stream) {
    if (!out || blocks <= 0 || iters <= 0) return CE_ERR_INVALID_ARG;
    peak_fma_kernel<<<blocks, 256, 0, as_stream(stream)>>>(out, iters, 0.999999f, 1e-6f);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

extern "C" int sce_peak_l2(const void *buf, size_t bytes, int reps, int blocks, float *out,
                           void *stream) {
    if (!buf || !out || bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15) || reps <= 0 ||
        blocks <= 0)
        return CE_ERR_INVALID_ARG;
    peak_l2_kernel<<<blocks, 256, 0, as_stream(stream)>>>(
        reinterpret_cast<const float4 *>(buf), (long long)(bytes / 16), reps, out);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}
