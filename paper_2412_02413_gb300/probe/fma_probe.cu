// fma_probe.cu -- the FP32 FMA rate of this GPU, measured, for the benchmark.
// The plain path's roofline divides by the peak from unit counts (SMs x FP32
// lanes x 2 flops x clock); this probe shows what the CUDA cores sustain on a
// pure FMA stream, scalar (FFMA) or packed two-wide (FFMA2). It is bench-side
// tooling, built into its own library (libpam_probe.so), not part of libpam.
#include <cuda_runtime.h>

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent FMA chains per thread (packed: 8 pairs)

// `iters` dependent FMAs on each chain. With 0 < mul < 1 every chain converges
// to add / (1 - mul), so all values stay finite and normal. The sum is stored
// only on a condition the compiler cannot decide, so no FMA is dead code.
__global__ void __launch_bounds__(PROBE_THREADS) fma_scalar_kernel(int iters, float mul, float add, float *out)
{
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], mul, add);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == -1.0f) out[0] = s;
}

// The same with two-wide packed FMAs: each instruction does two FMAs.
__global__ void __launch_bounds__(PROBE_THREADS) fma_packed_kernel(int iters, float mul, float add, float *out)
{
    float2 a[PROBE_CHAINS];
    const float2 m = make_float2(mul, mul), c = make_float2(add, add);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = __ffma2_rn(a[k], m, c);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == -1.0f) out[0] = s;
}

}  // namespace

// FP32 flop rate in TFLOP/s of one launch of 8 independent FMA chains per
// thread on every SM (as many 256-thread blocks as fit), `iters` FMAs per
// chain, after one warm-up launch. packed = 1 uses two-wide FMAs (4 flops per
// instruction). Returns 0 on success, else the CUDA error code.
extern "C" int pam_probe_fp32_fma_rate(int iters, int packed, double *tflops)
{
    if (iters < 1 || iters > (1 << 24) || !tflops) return (int)cudaErrorInvalidValue;
    auto kern = packed ? fma_packed_kernel : fma_scalar_kernel;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PROBE_THREADS, 0);
    if (e != cudaSuccess) return (int)e;
    float *sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float))) != cudaSuccess) return (int)e;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float ms = 0.0f;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) {
        kern<<<blocks, PROBE_THREADS>>>(iters, 0.9999f, 1e-4f, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0);
    if (e == cudaSuccess) {
        kern<<<blocks, PROBE_THREADS>>>(iters, 0.9999f, 1e-4f, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(sink);
    if (e != cudaSuccess) return (int)e;
    const double flops = 2.0 * (packed ? 2 : 1) * PROBE_CHAINS * (double)iters * blocks * PROBE_THREADS;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return 0;
}
