// FP32 FMA-rate probe: the measured denominator of the spectral-energy kernel's ALU roofline.
//
// Every thread runs SAL_PROBE_CHAINS independent FMA chains x <- x * a + b (a, b runtime
// values, so nothing folds), unrolled so that loop control is a few percent of the issued
// instructions.  The scalar form issues one FFMA per chain step; the packed form one
// fma.rn.f32x2 per two chains (the instruction the energy kernel uses for complex
// arithmetic).  flops per launch = 2 * SAL_PROBE_CHAINS * iters * threads.
#include "sal_internal.cuh"

namespace {

constexpr int kChains = SAL_PROBE_CHAINS;
constexpr int kThreads = 256;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kThreads) fma_probe_scalar(float *__restrict__ out, int iters, float a, float b)
{
    const int tid = blockIdx.x * kThreads + threadIdx.x;
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(tid & 1023) + (float)k;
    for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[tid] = s;
}

__global__ void __launch_bounds__(kThreads) fma_probe_packed(float *__restrict__ out, int iters, float a, float b)
{
    const int tid = blockIdx.x * kThreads + threadIdx.x;
    unsigned long long x[kChains / 2], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) {
        const float u = 1e-3f * (float)(tid & 1023) + (float)(2 * k), v = u + 1.f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(u), "f"(v));
    }
    for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains / 2; ++k)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) {
        float u, v;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(u), "=f"(v) : "l"(x[k]));
        s += u + v;
    }
    out[tid] = s;
}

}  // namespace

namespace sal {

cudaError_t launch_fma_probe(float *out, int64_t n_threads, int iters, bool packed, cudaStream_t stream)
{
    const unsigned grid = (unsigned)(n_threads / kThreads);
    // a slightly below 1 and b small keep every chain finite over any number of steps
    const float a = 0.9999999f, b = 1e-7f;
    if (packed)
        fma_probe_packed<<<grid, kThreads, 0, stream>>>(out, iters, a, b);
    else
        fma_probe_scalar<<<grid, kThreads, 0, stream>>>(out, iters, a, b);
    return cudaGetLastError();
}

}  // namespace sal
