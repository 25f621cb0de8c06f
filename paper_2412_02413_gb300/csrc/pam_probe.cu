// pam_probe.cu -- the FP32 FMA rate of this GPU, measured. The plain path's
// roofline divides by the peak from unit counts (SMs x FP32 lanes x 2 flops x
// clock); this probe shows what the CUDA cores sustain on a pure FMA stream.
#include <cuda_runtime.h>

#include <string>

#include "pam_internal.h"

namespace pam {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent FMA chains per thread

// `iters` dependent FMAs on each of PROBE_CHAINS chains. With 0 < mul < 1 every
// chain converges to add / (1 - mul), so all values stay finite and normal.
// The sum is stored only on a condition the compiler cannot decide, so no
// FMA is dead code.
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(int iters, float mul, float add, float *out)
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

pam_status pfail(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return set_error(PAM_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace
}  // namespace pam

extern "C" pam_status pam_fp32_fma_rate(int iters, double *tflops)
{
    if (iters < 1 || iters > (1 << 24) || !tflops) return pam::set_error(PAM_ERR_INVALID_ARG, "iters in [1, 2^24] and tflops");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pam::fma_probe_kernel, pam::PROBE_THREADS, 0);
    if (e != cudaSuccess) return pam::pfail(e, "device query");
    float *sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float))) != cudaSuccess) return pam::pfail(e, "allocation");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    float ms = 0.0f;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) {   // one warm-up launch, then the timed one
        pam::fma_probe_kernel<<<blocks, pam::PROBE_THREADS>>>(iters, 0.9999f, 1e-4f, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t0);
    if (e == cudaSuccess) {
        pam::fma_probe_kernel<<<blocks, pam::PROBE_THREADS>>>(iters, 0.9999f, 1e-4f, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(sink);
    if (e != cudaSuccess) return pam::pfail(e, "FMA probe");
    const double flops = 2.0 * pam::PROBE_CHAINS * (double)iters * blocks * pam::PROBE_THREADS;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return PAM_OK;
}
