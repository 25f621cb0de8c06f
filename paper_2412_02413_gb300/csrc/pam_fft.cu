// pam_fft.cu -- plan tables (FP64), the per-channel time FFT that keeps the
// selected bins (Eq. 1, F_t), and the apodized lateral DFT (Eq. 1, F_x;
// apodization patterns of Sec. II-A and II-C).
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"

namespace pam {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// A fraction of a turn in [0, 1) as a 64-bit fixed-point word (turns * 2^64),
// built from two exact 32-bit pieces so that no step rounds past 2^64.
__device__ uint64_t turns_to_word(double turns)
{
    double fr = turns - floor(turns);                  // [0, 1)
    double hi_d = floor(fr * 4294967296.0);            // exact scaling by 2^32
    double lo_d = floor((fr * 4294967296.0 - hi_d) * 4294967296.0);
    uint64_t hi = (uint64_t)hi_d, lo = (uint64_t)lo_d;
    if (hi > 0xffffffffull) hi = 0xffffffffull;
    if (lo > 0xffffffffull) lo = 0xffffffffull;
    return (hi << 32) | lo;
}

// One thread per (bin, lateral bin u). FP64 throughout (Eq. 2):
//   w = 2 pi k fs / nt, kx = 2 pi u' / (nx pitch), kz = sqrt((w/c)^2 - kx^2).
// Propagating: the phase kz*z in turns, as an exact fixed-point accumulator
// word. The anchor holds kz*z0 and the step holds kz*dz per row, so row j has
// phase anchor + j*step (mod 2^64): the 2 pi range reduction is exact integer
// wrap-around. Evanescent: amplitude exp(-kappa z) = exp2(ecoef * z).
__global__ void tables_kernel(const int *__restrict__ bins, int n_bins, int nx, int nt, double fs,
                              double c, double pitch, double z0, double dz, int evanescent_zero,
                              ulonglong2 *__restrict__ dds, float *__restrict__ ecoef,
                              float *__restrict__ live, int *__restrict__ bin_evan,
                              float2 *__restrict__ tw_t, float2 *__restrict__ tw_x)
{
    const double two_pi = 6.283185307179586476925286766559;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n_bins * nx) {
        int b = idx / nx, u = idx % nx;
        int up = (2 * u >= nx) ? u - nx : u;
        double k0 = two_pi * (double)bins[b] * fs / (double)nt / c;
        double kx = two_pi * (double)up / ((double)nx * pitch);
        double d = k0 * k0 - kx * kx;
        ulonglong2 w;
        if (d >= 0.0) {
            double kz = sqrt(d);
            w.x = turns_to_word(kz * z0 / two_pi);
            w.y = turns_to_word(kz * dz / two_pi);
            ecoef[idx] = 0.0f;
            live[idx] = 1.0f;
        } else {
            double kappa = sqrt(-d);
            w.x = 0;
            w.y = 0;
            ecoef[idx] = (float)(-kappa * 1.4426950408889634073599246810019);
            live[idx] = evanescent_zero ? 0.0f : 1.0f;
            if (!evanescent_zero) atomicOr(&bin_evan[b], 1);
        }
        dds[idx] = w;
    }
    if (idx < nt) {
        double s, co;
        sincospi(-2.0 * (double)idx / (double)nt, &s, &co);
        tw_t[idx] = make_float2((float)co, (float)s);
    }
    if (idx < nx) {
        double s, co;
        sincospi(-2.0 * (double)idx / (double)nx, &s, &co);
        tw_x[idx] = make_float2((float)co, (float)s);
    }
}

// ----------------------------------------------------------- time FFT ----
// One CTA per (pair of channels, frame). The pair is packed as z = a + i b,
// transformed by an nt-point Stockham auto-sort FFT (radix-4 stages, then one
// radix-2 stage when log2 nt is odd) in shared memory, and split back with
//   A[k] = (Z[k] + conj Z[nt-k]) / 2,  B[k] = (Z[k] - conj Z[nt-k]) / (2i).
// Only the selected bins leave the CTA: S[f][b][e].
constexpr int TFFT_THREADS = 256;

__global__ void __launch_bounds__(TFFT_THREADS)
time_fft_kernel(const float *__restrict__ rf, int ne, int nt, const float2 *__restrict__ tw,
                const int *__restrict__ bins, int n_bins, float2 *__restrict__ S,
                unsigned *__restrict__ fmax)
{
    extern __shared__ __align__(16) float2 sbuf[];
    float2 *x = sbuf, *y = sbuf + nt;
    const int f = blockIdx.y;
    const int e0 = 2 * blockIdx.x, e1 = e0 + 1;
    const bool has_b = e1 < ne;
    const float *ra = rf + ((size_t)f * ne + e0) * nt;
    const float *rb = rf + ((size_t)f * ne + (has_b ? e1 : e0)) * nt;
    if (blockIdx.x == 0 && threadIdx.x == 0) fmax[f] = 0u;

    for (int t4 = threadIdx.x; t4 < nt / 4; t4 += TFFT_THREADS) {
        float4 a = reinterpret_cast<const float4 *>(ra)[t4];
        float4 b = has_b ? reinterpret_cast<const float4 *>(rb)[t4] : make_float4(0.f, 0.f, 0.f, 0.f);
        x[4 * t4 + 0] = make_float2(a.x, b.x);
        x[4 * t4 + 1] = make_float2(a.y, b.y);
        x[4 * t4 + 2] = make_float2(a.z, b.z);
        x[4 * t4 + 3] = make_float2(a.w, b.w);
    }
    __syncthreads();

    int Ns = 1;
    const int q4 = nt / 4;
    for (; 4 * Ns <= nt; Ns *= 4) {
        const int tstride = nt / (4 * Ns);
        for (int j = threadIdx.x; j < q4; j += TFFT_THREADS) {
            const int k = j & (Ns - 1);
            float2 v0 = x[j], v1 = x[j + q4], v2 = x[j + 2 * q4], v3 = x[j + 3 * q4];
            if (Ns > 1) {
                v1 = cmul(v1, tw[k * tstride]);
                v2 = cmul(v2, tw[2 * k * tstride]);
                v3 = cmul(v3, tw[3 * k * tstride]);
            }
            // forward 4-point DFT: X_s = sum_r v_r (-i)^(r s)
            float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
            float2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
            float2 md13 = make_float2(d13.y, -d13.x);   // -i * d13
            const int base = (j - k) * 4 + k;
            y[base] = cadd(s02, s13);
            y[base + Ns] = cadd(d02, md13);
            y[base + 2 * Ns] = csub(s02, s13);
            y[base + 3 * Ns] = csub(d02, md13);
        }
        __syncthreads();
        float2 *tmp = x; x = y; y = tmp;
    }
    if (Ns < nt) {  // one radix-2 stage with Ns = nt/2
        const int h = nt / 2;
        for (int j = threadIdx.x; j < h; j += TFFT_THREADS) {
            const int k = j & (Ns - 1);
            float2 v0 = x[j], v1 = cmul(x[j + h], tw[k]);
            const int base = (j - k) * 2 + k;
            y[base] = cadd(v0, v1);
            y[base + Ns] = csub(v0, v1);
        }
        __syncthreads();
        float2 *tmp = x; x = y; y = tmp;
    }

    for (int b = threadIdx.x; b < n_bins; b += TFFT_THREADS) {
        const int k = bins[b];
        float2 zk = x[k], zm = x[nt - k];
        // A = (zk + conj zm)/2 ; B = (zk - conj zm)/(2i)
        float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        float dr = zk.x - zm.x, di = zk.y + zm.y;
        float2 B = make_float2(0.5f * di, -0.5f * dr);
        float2 *dst = S + ((size_t)f * n_bins + b) * ne;
        dst[e0] = A;
        if (has_b) dst[e1] = B;
    }
}

// -------------------------------------------------------- lateral DFT ----
// Q[f][b][q][u] = (1/nx) sum_e apod_q[e] S[f][b][e] exp(-2 pi i u e / nx)
// times the live mask (PAM_EVANESCENT_ZERO). The 1/nx of the inverse lateral
// transform is applied here. Threads (q, u); one CTA loops over BPB bins.
constexpr int LAT_BPB = 4;

__global__ void __launch_bounds__(384)
lateral_kernel(const float2 *__restrict__ S, int ne, int nx, int n_bins, int napq,
               const float *__restrict__ apod, const float2 *__restrict__ twx,
               const float *__restrict__ live, float2 *__restrict__ Q)
{
    extern __shared__ __align__(16) float2 sS[];   // [ne]
    float *sA = reinterpret_cast<float *>(sS + ne); // [napq][ne]
    float2 *sT = reinterpret_cast<float2 *>(sA + ((napq * ne + 1) & ~1)); // [nx]
    const int f = blockIdx.y;
    const int tid = threadIdx.x;
    const int q = tid / nx, u = tid % nx;
    for (int i = tid; i < napq * ne; i += blockDim.x) sA[i] = apod[i];
    for (int i = tid; i < nx; i += blockDim.x) sT[i] = twx[i];
    const float inv_nx = 1.0f / (float)nx;
    const int b_begin = blockIdx.x * LAT_BPB;
    const int b_end = min(n_bins, b_begin + LAT_BPB);
    for (int b = b_begin; b < b_end; ++b) {
        __syncthreads();
        for (int i = tid; i < ne; i += blockDim.x) sS[i] = S[((size_t)f * n_bins + b) * ne + i];
        __syncthreads();
        if (q < napq) {
            float re = 0.f, im = 0.f;
            int m = 0;  // (u * e) mod nx, advanced incrementally
            for (int e = 0; e < ne; ++e) {
                float a = sA[q * ne + e];
                float2 s = sS[e], w = sT[m];
                float xr = a * s.x, xi = a * s.y;
                re = fmaf(xr, w.x, fmaf(-xi, w.y, re));
                im = fmaf(xr, w.y, fmaf(xi, w.x, im));
                m += u;
                if (m >= nx) m -= nx;
            }
            float l = live[(size_t)b * nx + u] * inv_nx;
            Q[(((size_t)f * n_bins + b) * napq + q) * nx + u] = make_float2(re * l, im * l);
        }
    }
}

}  // namespace

cudaError_t launch_tables(const pam_plan_s &p, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p.t.bin_evan, 0, sizeof(int) * p.n_bins, st);
    if (e != cudaSuccess) return e;
    int n = p.n_bins * p.nx;
    if (p.nt > n) n = p.nt;
    int blocks = (n + 255) / 256;
    tables_kernel<<<blocks, 256, 0, st>>>(p.t.bins, p.n_bins, p.nx, p.nt, p.d.fs_hz, p.d.c_mps, p.d.pitch_m,
                                          p.d.z0_m, p.d.dz_m, (p.d.flags & PAM_EVANESCENT_ZERO) ? 1 : 0,
                                          p.t.dds, p.t.ecoef, p.t.live, p.t.bin_evan, p.t.tw_t, p.t.tw_x);
    return cudaGetLastError();
}

static size_t time_fft_smem(int nt) { return (size_t)2 * nt * sizeof(float2); }

static size_t lateral_smem(int ne, int nx, int napq)
{
    return (size_t)ne * sizeof(float2) + (size_t)((napq * ne + 1) & ~1) * sizeof(float) + (size_t)nx * sizeof(float2);
}

cudaError_t launch_time_fft(const pam_plan_s &p, const float *rf, int n_frames, cudaStream_t st)
{
    dim3 grid((p.ne + 1) / 2, n_frames);
    time_fft_kernel<<<grid, TFFT_THREADS, time_fft_smem(p.nt), st>>>(rf, p.ne, p.nt, p.t.tw_t, p.t.bins,
                                                                      p.n_bins, p.w.S, p.w.fmax);
    return cudaGetLastError();
}

cudaError_t launch_lateral(const pam_plan_s &p, int n_frames, int napq, const float *apod, cudaStream_t st)
{
    dim3 grid((p.n_bins + LAT_BPB - 1) / LAT_BPB, n_frames);
    int threads = napq * p.nx;
    threads = (threads + 31) / 32 * 32;
    lateral_kernel<<<grid, threads, lateral_smem(p.ne, p.nx, napq), st>>>(p.w.S, p.ne, p.nx, p.n_bins, napq, apod,
                                                                          p.t.tw_x, p.t.live, p.w.Q);
    return cudaGetLastError();
}

// The attribute is per kernel, not per plan: it is set to the largest
// supported nt so that plans of different sizes can coexist.
cudaError_t prepare_fft_kernels(const pam_plan_s &)
{
    return cudaFuncSetAttribute(time_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)time_fft_smem(8192));
}

}  // namespace pam
