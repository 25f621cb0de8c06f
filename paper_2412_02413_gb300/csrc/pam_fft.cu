// pam_fft.cu -- plan tables (FP64), the per-channel time FFT that keeps the
// selected bins (Eq. 1, F_t), and the apodized lateral FFT (Eq. 1, F_x;
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
// Propagating components get the phase kz*z in turns as a fixed-point
// accumulator: a 64-bit anchor holds kz*z0 and a 64-bit step holds kz*dz per
// row, so row j has phase anchor + j*step (mod 2^64). The 2 pi range
// reduction is therefore exact integer wrap-around. The kernels read the top
// 32 bits of that sum. Evanescent components get amplitude
// exp(-kappa z) = exp2(ecoef * z).
__global__ void tables_kernel(const int *__restrict__ bins, int n_bins, int nx, int nt, double fs,
                              double c, double pitch, double z0, double dz, int evanescent_zero,
                              uint4 *__restrict__ phase, float *__restrict__ live, int *__restrict__ bin_evan,
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
        uint4 w;
        if (d >= 0.0) {
            double kz = sqrt(d);
            uint64_t a = turns_to_word(kz * z0 / two_pi);
            uint64_t s = turns_to_word(kz * dz / two_pi);
            w = make_uint4((unsigned)(a >> 32), (unsigned)(s >> 32), (unsigned)(s & 0xffffffffull),
                           __float_as_uint(0.0f));
            live[idx] = 1.0f;
        } else {
            double kappa = sqrt(-d);
            w = make_uint4(0u, 0u, 0u, __float_as_uint((float)(-kappa * 1.4426950408889634073599246810019)));
            live[idx] = evanescent_zero ? 0.0f : 1.0f;
            if (!evanescent_zero) atomicOr(&bin_evan[b], 1);
        }
        phase[idx] = w;
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

// ------------------------------------------------------ Stockham FFT ----
// Forward 8-point DFT (exp(-2 pi i m r / 8)) in registers: two 4-point DFTs
// of the even and odd inputs, the odd ones turned by exp(-2 pi i r / 8).
__device__ __forceinline__ void fdft8(float2 (&v)[8])
{
    const float h = 0.70710678118654752440f;
    float2 e[4], o[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        e[r] = v[2 * r];
        o[r] = v[2 * r + 1];
    }
    auto dft4 = [](float2 (&a)[4]) {
        const float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        const float2 s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
        const float2 md13 = make_float2(d13.y, -d13.x);   // -i * d13
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, md13);
        a[3] = csub(d02, md13);
    };
    dft4(e);
    dft4(o);
    o[1] = make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));    // (1 - i) / sqrt 2
    o[2] = make_float2(o[2].y, -o[2].x);                                 // -i
    o[3] = make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));   // (-1 - i) / sqrt 2
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[r] = cadd(e[r], o[r]);
        v[r + 4] = csub(e[r], o[r]);
    }
}

// Forward FFTs (exp(-2 pi i m / n)) of `batch` contiguous n-point sequences in
// shared memory. With MAXR = 8: radix-8 stages while they fit, then radix-4;
// with MAXR = 4: radix-4 stages. Then one radix-2 stage if a factor 2 is left.
// Auto-sort ordering (a stage of radix R takes sub-transforms of length Ns to
// R Ns), so the output is in natural order. tw[m] holds exp(-2 pi i m / n)
// for m < n. x and y are ping-pong buffers; the return value is the buffer
// with the result. Every thread of the CTA must call it.
template <int MAXR>
__device__ float2 *stockham(float2 *x, float2 *y, int n, int log2n, int batch, const float2 *tw, int tid, int nth)
{
    int Ns = 1;
    if constexpr (MAXR == 8) {
        const int q8 = n >> 3;
        const int lq8 = log2n - 3;
        for (; 8 * Ns <= n; Ns <<= 3) {
            const int ts = n / (8 * Ns);
            for (int t = tid; t < batch * q8; t += nth) {
                const int bt = t >> lq8, j = t & (q8 - 1);
                const float2 *xb = x + bt * n;
                float2 *yb = y + bt * n;
                const int k = j & (Ns - 1);
                float2 v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = xb[j + r * q8];
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], tw[r * k * ts]);
                }
                fdft8(v);
                const int base = (j - k) * 8 + k;
#pragma unroll
                for (int r = 0; r < 8; ++r) yb[base + r * Ns] = v[r];
            }
            __syncthreads();
            float2 *tmp = x; x = y; y = tmp;
        }
    }
    const int q4 = n >> 2;
    const int lq4 = log2n - 2;
    for (; 4 * Ns <= n; Ns <<= 2) {
        const int ts = n / (4 * Ns);
        for (int t = tid; t < batch * q4; t += nth) {
            const int bt = t >> lq4, j = t & (q4 - 1);
            const float2 *xb = x + bt * n;
            float2 *yb = y + bt * n;
            const int k = j & (Ns - 1);
            float2 v0 = xb[j], v1 = xb[j + q4], v2 = xb[j + 2 * q4], v3 = xb[j + 3 * q4];
            if (Ns > 1) {
                v1 = cmul(v1, tw[k * ts]);
                v2 = cmul(v2, tw[2 * k * ts]);
                v3 = cmul(v3, tw[3 * k * ts]);
            }
            float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
            float2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
            float2 md13 = make_float2(d13.y, -d13.x);   // -i * d13
            const int base = (j - k) * 4 + k;
            yb[base] = cadd(s02, s13);
            yb[base + Ns] = cadd(d02, md13);
            yb[base + 2 * Ns] = csub(s02, s13);
            yb[base + 3 * Ns] = csub(d02, md13);
        }
        __syncthreads();
        float2 *tmp = x; x = y; y = tmp;
    }
    if (Ns < n) {  // radix-2 stage with Ns = n/2
        const int h = n >> 1;
        for (int t = tid; t < batch * h; t += nth) {
            const int bt = t >> (log2n - 1), j = t & (h - 1);
            const float2 *xb = x + bt * n;
            float2 *yb = y + bt * n;
            float2 v0 = xb[j], v1 = cmul(xb[j + h], tw[j]);
            yb[j] = cadd(v0, v1);
            yb[j + h] = csub(v0, v1);
        }
        __syncthreads();
        x = y;
    }
    return x;
}

// ----------------------------------------------------------- time FFT ----
// One CTA per (channel, frame). The nt real samples are packed as
// z[n] = x[2n] + i x[2n+1] and transformed by an nt/2-point FFT in shared
// memory. The two half-length spectra are then separated:
//   E[k] = (Z[k] + conj Z[M-k]) / 2,  O[k] = (Z[k] - conj Z[M-k]) / (2i),
//   X[k] = E[k] + exp(-2 pi i k / nt) O[k].
// Only the selected bins leave the CTA, as S[f][b][c] with c = cstep e
// (cstep = 2 when the channels are zero-stuffed) in rows of nev channels.
// Block (0, f) also clears the frame's rho maximum for the epilogue.
constexpr int TFFT_THREADS = 256;

template <int MAXR>
__global__ void __launch_bounds__(TFFT_THREADS)
time_fft_kernel(const float *__restrict__ rf, int ne, int nt, int log2nt, const float2 *__restrict__ tw,
                const int *__restrict__ bins, int n_bins, float2 *__restrict__ S, int nev, int cstep,
                unsigned *__restrict__ fmax)
{
    extern __shared__ __align__(16) float2 sbuf[];
    const int M = nt >> 1;
    float2 *x = sbuf, *y = sbuf + M, *tws = sbuf + 2 * M;
    const int f = blockIdx.y, e = blockIdx.x;
    const float4 *src = reinterpret_cast<const float4 *>(rf + ((size_t)f * ne + e) * nt);
    if (e == 0 && threadIdx.x == 0) fmax[f] = 0u;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    for (int i = threadIdx.x; i < nt / 4; i += TFFT_THREADS) x4[i] = src[i];  // (x0,x1),(x2,x3) pairs
    for (int m = threadIdx.x; m < M; m += TFFT_THREADS) tws[m] = tw[2 * m];    // exp(-2 pi i m / M)
    __syncthreads();
    float2 *Z = stockham<MAXR>(x, y, M, log2nt - 1, 1, tws, threadIdx.x, TFFT_THREADS);
    for (int b = threadIdx.x; b < n_bins; b += TFFT_THREADS) {
        const int k = bins[b];                                 // 0 < k < M
        const float2 zk = Z[k], zm = Z[M - k];
        const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        S[((size_t)f * n_bins + b) * nev + (size_t)e * cstep] = cadd(E, cmul(tw[k], O));
    }
}

// -------------------------------------------------------- lateral FFT ----
// V_q[u] = live[b][u] / nx * sum_e apod_q[e] S[f][b][e] exp(-2 pi i u e / nx),
// the propagator's input (Eq. 1-2); live_fs is the frame stride of the mask
// (0: one mask for all frames). One CTA per (bin, frame): the napq apodized
// rows are transformed together by the shared-memory FFT. The 1/nx of the
// inverse lateral transform is applied here.
//
// Output layout, for the fused kernel's radix-2 decimation-in-frequency split
// of the inverse lateral DFT: half g of the output pixels needs
//   x_g[u0] = W^(g u0) (P[u0] + (-1)^g P[u0 + H]),  H = nx/2, W = exp(2 pi i/nx),
// with P[u] = V[u] exp(i kz_u z). Writing u0 = L2 n1 + n2 (L2 = nx/16), the
// lane (g, n2) reads per (q, n1) one pair of complex values that it multiplies
// with its own phasor (u = g H + u0) and its partner lane's (u = (1-g) H + u0):
//   g = 0: ( V[u0],                V[u0 + H]          )
//   g = 1: ( -W^u0 V[u0 + H],      W^u0 V[u0]         )
// stored at Q[f][b][q][n1][g][n2][2] (q_per_bin = 2 napq nx complex values).
constexpr int LAT_THREADS = 128;

__global__ void __launch_bounds__(LAT_THREADS)
lateral_kernel(const float2 *__restrict__ S, int ne, int nx, int log2nx, int n_bins, int napq,
               const float *__restrict__ apod, const float2 *__restrict__ twx, const float *__restrict__ live,
               size_t live_fs, float2 *__restrict__ Q)
{
    extern __shared__ __align__(16) float2 lbuf[];
    float2 *x = lbuf, *y = lbuf + napq * nx, *tws = lbuf + 2 * napq * nx;
    const int f = blockIdx.y, b = blockIdx.x;
    const float2 *s = S + ((size_t)f * n_bins + b) * ne;
    for (int i = threadIdx.x; i < napq * nx; i += LAT_THREADS) {
        const int q = i / nx, e = i - q * nx;
        const float2 v = s[e];
        const float a = apod[q * ne + e];
        x[i] = make_float2(a * v.x, a * v.y);
    }
    for (int i = threadIdx.x; i < nx; i += LAT_THREADS) tws[i] = twx[i];
    __syncthreads();
    const float2 *X = stockham<4>(x, y, nx, log2nx, napq, tws, threadIdx.x, LAT_THREADS);
    const float inv_nx = 1.0f / (float)nx;
    float2 *dst = Q + ((size_t)f * n_bins + b) * (2 * napq * nx);
    const int H = nx / 2, L2 = nx / 16;
    for (int i = threadIdx.x; i < napq * nx; i += LAT_THREADS) {
        const int q = i / nx, u = i & (nx - 1);
        const float l = live[(size_t)f * live_fs + (size_t)b * nx + u] * inv_nx;
        const float2 v = make_float2(X[i].x * l, X[i].y * l);
        const int hi = u >= H ? 1 : 0, u0 = u - hi * H, n1 = u0 / L2, n2 = u0 - n1 * L2;
        float ws, wc;
        sincospif(2.0f * (float)u0 / (float)nx, &ws, &wc);   // W^u0, exact argument
        const float sg = hi ? -1.0f : 1.0f;
        const float2 vw = make_float2(sg * (wc * v.x - ws * v.y), sg * (wc * v.y + ws * v.x));
        const size_t base = (size_t)(q * 8 + n1) * 2;
        dst[((base + 0) * L2 + n2) * 2 + hi] = v;
        dst[((base + 1) * L2 + n2) * 2 + (1 - hi)] = vw;
    }
}

int ilog2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

size_t time_fft_smem(int nt) { return (size_t)3 * (nt / 2) * sizeof(float2); }

size_t lateral_smem(int nx, int napq) { return ((size_t)2 * napq * nx + nx) * sizeof(float2); }

}  // namespace

cudaError_t launch_tables(const pam_plan_s &p, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p.t.bin_evan, 0, sizeof(int) * p.n_bins, st);
    if (e != cudaSuccess) return e;
    int n = p.n_bins * p.nx;
    if (p.nt > n) n = p.nt;
    int blocks = (n + 255) / 256;
    tables_kernel<<<blocks, 256, 0, st>>>(p.t.bins, p.n_bins, p.nx, p.nt, p.d.fs_hz, p.d.c_mps, p.pitch_x,
                                          p.d.z0_m, p.d.dz_m, (p.d.flags & PAM_EVANESCENT_ZERO) ? 1 : 0,
                                          p.t.phase, p.t.live, p.t.bin_evan, p.t.tw_t, p.t.tw_x);
    return cudaGetLastError();
}

cudaError_t launch_time_fft(const pam_plan_s &p, const float *rf, int n_frames, cudaStream_t st)
{
    dim3 grid(p.ne, n_frames);
    auto kern = p.fft_radix == 8 ? time_fft_kernel<8> : time_fft_kernel<4>;
    kern<<<grid, TFFT_THREADS, time_fft_smem(p.nt), st>>>(rf, p.ne, p.nt, ilog2i(p.nt), p.t.tw_t, p.t.bins,
                                                          p.n_bins, p.w.S, p.nev, p.chan_step, p.w.fmax);
    return cudaGetLastError();
}

cudaError_t launch_lateral(const pam_plan_s &p, int n_frames, int napq, const float *apod, cudaStream_t st)
{
    dim3 grid(p.n_bins, n_frames);
    lateral_kernel<<<grid, LAT_THREADS, lateral_smem(p.nx, napq), st>>>(p.w.S, p.nev, p.nx, ilog2i(p.nx), p.n_bins,
                                                                        napq, apod, p.t.tw_x, p.t.live, 0, p.w.Q);
    return cudaGetLastError();
}

cudaError_t launch_lateral_frames(const pam_plan_s &p, int n_frames, int napq, const float *apod,
                                  const float *live, size_t live_fs, cudaStream_t st)
{
    dim3 grid(p.n_bins, n_frames);
    lateral_kernel<<<grid, LAT_THREADS, lateral_smem(p.nx, napq), st>>>(p.w.S, p.nev, p.nx, ilog2i(p.nx), p.n_bins,
                                                                        napq, apod, p.t.tw_x, live, live_fs, p.w.Q);
    return cudaGetLastError();
}

cudaError_t launch_tables_frame(const pam_plan_s &p, const int *bins, int n_bins, int nt, uint4 *phase, float *live,
                                int *bin_evan, float2 *tw_t, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bin_evan, 0, sizeof(int) * n_bins, st);
    if (e != cudaSuccess) return e;
    int n = n_bins * p.nx;
    if (nt > n) n = nt;
    tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(bins, n_bins, p.nx, nt, p.d.fs_hz, p.d.c_mps, p.pitch_x,
                                                    p.d.z0_m, p.d.dz_m, (p.d.flags & PAM_EVANESCENT_ZERO) ? 1 : 0,
                                                    phase, live, bin_evan, tw_t, p.t.tw_x);
    return cudaGetLastError();
}

// The attribute is per kernel, not per plan: it is set to the largest
// supported nt so that plans of different sizes can coexist.
cudaError_t prepare_fft_kernels(const pam_plan_s &)
{
    cudaError_t e = cudaFuncSetAttribute(time_fft_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)time_fft_smem(8192));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(time_fft_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)time_fft_smem(8192));
}

}  // namespace pam
