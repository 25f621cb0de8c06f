// pam_metrics.cu -- image-level kernels: the AS^3 image (Eq. 20), the
// image-quality measures of the paper (Eq. 12-13: energy spread area A_0.5,
// image signal-to-noise ratio and the thresholded centroid), and the crop of
// the maps computed with 2x lateral padding (Sec. II-D).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "pam_internal.h"

namespace pam {
namespace {

constexpr int MT = 512;   // threads per frame block

// Block-wide sum of one double (every thread gets the result, summed in warp order).
__device__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < MT / 32; ++w) s += sh[w];
    return s;
}

__device__ float block_max(float v, float *sh)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = -INFINITY;
    for (int w = 0; w < MT / 32; ++w) m = fmaxf(m, sh[w]);
    return m;
}

// One block per frame. Pass 1: the maximum. Pass 2: the pixels above half of
// it (A_0.5) and their sum, the sum of the others, and the centroid sums over
// the pixels above alpha times the maximum (weights I_i, Eq. 13).
__global__ void __launch_bounds__(MT)
metrics_kernel(const float *__restrict__ img, int nz, int nx, double x0, double dx, double z0, double dz, float alpha,
               pam_image_metrics_t *__restrict__ out)
{
    __shared__ double shd[MT / 32];
    __shared__ float shf[MT / 32];
    const size_t npix = (size_t)nz * nx;
    const float *I = img + (size_t)blockIdx.x * npix;
    float m = -INFINITY;
    for (size_t x = threadIdx.x; x < npix; x += MT) m = fmaxf(m, I[x]);
    m = block_max(m, shf);
    const float half = 0.5f * m, thr = alpha * m;
    double n_in = 0.0, s_in = 0.0, s_out = 0.0, w = 0.0, wx = 0.0, wz = 0.0;
    for (size_t x = threadIdx.x; x < npix; x += MT) {
        const float v = I[x];
        if (v > half) {
            n_in += 1.0;
            s_in += v;
        } else {
            s_out += v;
        }
        if (v > thr) {
            const int j = (int)(x / nx), i = (int)(x % nx);
            w += v;
            wx += (double)v * (x0 + i * dx);
            wz += (double)v * (z0 + j * dz);
        }
    }
    n_in = block_sum(n_in, shd);
    s_in = block_sum(s_in, shd);
    s_out = block_sum(s_out, shd);
    w = block_sum(w, shd);
    wx = block_sum(wx, shd);
    wz = block_sum(wz, shd);
    if (threadIdx.x == 0) {
        pam_image_metrics_t r;
        const double n_out = (double)npix - n_in;
        r.max = m;
        r.n_inside = (int)n_in;
        r.esa_m2 = (float)(n_in * fabs(dx * dz));
        if (!(m > 0.0f) || n_in == 0.0)
            r.isnr_db = NAN;
        else if (n_out == 0.0 || s_out <= 0.0)
            r.isnr_db = INFINITY;
        else
            r.isnr_db = (float)(10.0 * log10((s_in / n_in) / (s_out / n_out)));
        r.cx_m = w > 0.0 ? (float)(wx / w) : NAN;
        r.cz_m = w > 0.0 ? (float)(wz / w) : NAN;
        out[blockIdx.x] = r;
    }
}

// Eq. 20 in place: I = (I / max I)^2 I, one block per frame.
__global__ void __launch_bounds__(MT) as3_kernel(float *__restrict__ img, size_t npix)
{
    __shared__ float shf[MT / 32];
    float *I = img + (size_t)blockIdx.x * npix;
    float m = 0.0f;
    for (size_t x = threadIdx.x; x < npix; x += MT) m = fmaxf(m, I[x]);
    m = block_max(m, shf);
    const float inv = m > 0.0f ? 1.0f / m : 0.0f;
    for (size_t x = threadIdx.x; x < npix; x += MT) {
        const float r = I[x] * inv;
        I[x] = r * r * I[x];
    }
}

// Crop of maps computed over 2 ne padded columns to the ne element columns
// (row width nx -> nxo), one block per frame. Pass 1: the maximum of rho
// over the crop. Pass 2: rho_n = rho / max and I = rho_n^2 E (Eq. 11), plus
// the optional copies of E and of the pair NCCs.
__global__ void __launch_bounds__(MT)
pad_crop_kernel(const float *__restrict__ rho_full, const float *__restrict__ e_full,
                const float *__restrict__ pairs_full, int n_pairs, int nz, int nx, int nxo, float *__restrict__ image,
                float *__restrict__ rho_n, float *__restrict__ pairs, float *__restrict__ image_as)
{
    __shared__ float shf[MT / 32];
    const size_t npix = (size_t)nz * nx, npo = (size_t)nz * nxo, f = blockIdx.x;
    const float *R = rho_full + f * npix, *E = e_full + f * npix;
    float m = 0.0f;
    for (size_t o = threadIdx.x; o < npo; o += MT) m = fmaxf(m, R[(o / nxo) * nx + o % nxo]);
    m = block_max(m, shf);
    for (size_t o = threadIdx.x; o < npo; o += MT) {
        const size_t x = (o / nxo) * nx + o % nxo;
        const float r = m > 0.0f ? R[x] / m : 0.0f, e = E[x];
        image[f * npo + o] = r * r * e;
        if (rho_n) rho_n[f * npo + o] = r;
        if (image_as) image_as[f * npo + o] = e;
        if (pairs)
            for (int k = 0; k < n_pairs; ++k) pairs[(f * n_pairs + k) * npo + o] = pairs_full[(f * n_pairs + k) * npix + x];
    }
}

pam_status mfail(pam_status s, const std::string &m) { return set_error(s, m.c_str()); }

pam_status dev_ok(const void *p, const char *name)
{
    if (!p) return mfail(PAM_ERR_INVALID_ARG, std::string(name) + " is NULL");
    if (reinterpret_cast<uintptr_t>(p) & 15u)
        return mfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return mfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return mfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return PAM_OK;
}

}  // namespace

cudaError_t launch_pad_crop(const float *rho_full, const float *e_full, const float *pairs_full, int n_pairs,
                            int n_frames, int nz, int nx, int nx_out, float *image, float *rho_n, float *pairs,
                            float *image_as, cudaStream_t st)
{
    if (n_frames == 0) return cudaSuccess;
    pad_crop_kernel<<<n_frames, MT, 0, st>>>(rho_full, e_full, pairs ? pairs_full : nullptr, n_pairs, nz, nx, nx_out,
                                             image, rho_n, pairs, image_as);
    return cudaGetLastError();
}

}  // namespace pam

extern "C" {

pam_status pam_image_metrics(const float *maps, int n_frames, int nz, int nx, double x0_m, double dx_m, double z0_m,
                             double dz_m, float alpha, pam_image_metrics_t *out, void *stream)
{
    if (n_frames < 0 || nz < 1 || nx < 1) return pam::mfail(PAM_ERR_INVALID_ARG, "sizes out of range");
    if (!(alpha > 0.0f && alpha < 1.0f)) return pam::mfail(PAM_ERR_INVALID_ARG, "alpha must be in (0, 1)");
    if (!std::isfinite(x0_m) || !std::isfinite(dx_m) || !std::isfinite(z0_m) || !std::isfinite(dz_m))
        return pam::mfail(PAM_ERR_INVALID_ARG, "pixel grid must be finite");
    if (n_frames == 0) return PAM_OK;
    pam_status s;
    if ((s = pam::dev_ok(maps, "maps")) != PAM_OK) return s;
    if ((s = pam::dev_ok(out, "out")) != PAM_OK) return s;
    pam::metrics_kernel<<<n_frames, pam::MT, 0, static_cast<cudaStream_t>(stream)>>>(maps, nz, nx, x0_m, dx_m, z0_m,
                                                                                    dz_m, alpha, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pam::mfail(PAM_ERR_CUDA, std::string("metrics launch: ") + cudaGetErrorString(e));
    return PAM_OK;
}

pam_status pam_as3(pam_plan_t p, const float *rf, int n_frames, float *image, void *stream)
{
    pam::TraceRange trace_("pam_as3");
    if (!p) return pam::mfail(PAM_ERR_INVALID_ARG, "plan is NULL");
    pam_status s = pam_as_backprop(p, rf, n_frames, -1, image, nullptr, stream);
    if (s != PAM_OK || n_frames == 0) return s;
    pam::as3_kernel<<<n_frames, pam::MT, 0, static_cast<cudaStream_t>(stream)>>>(image, (size_t)p->nz * p->nx_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pam::mfail(PAM_ERR_CUDA, std::string("AS3 launch: ") + cudaGetErrorString(e));
    p->kernels += 1;
    return PAM_OK;
}

}  // extern "C"
