// pam_learn.cu -- the learned form of AS-TAX: a small convolutional network
// predicts the TAX NCC weight rho_TAX (Eq. 10) from band energies of the
// full-aperture AS map (Eq. 3), so that a frame needs one back-propagation
// (instead of three apodized ones) plus the network; a per-frame error gate
// runs the exact method on the depth-row tile around the predicted peak and
// sends frames that miss it through the plain AS-TAX path.
//
// Network (5 conv3x3 layers, zero padding 1): 5 -> 32 -> 32 -> 32 -> 32 -> 1,
// ReLU after the first four, head rho = eps + (1 - eps) sigmoid(z). Inputs:
// channel 0 = log10(E / max E + 1e-4) / 4 of the full-aperture energy E,
// channels 1..4 the same for the energy of each quarter of the bins.
// Operands (activations, weights, gradients) are BF16, every sum is FP32.
//
// Tensor layout of activations and gradients ("chunked, padded"): BF16
// [F][C/8][nz+2][nx+2][8], eight channels of one pixel in 16 bytes, with a
// zero border of one pixel so that every 3x3 tap reads memory.
//
// Kernels of this file run on CUDA cores; the forward of every layer also has
// a tcgen05 tensor-core version (pam_conv_tc.cu) for nx = 128.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pam_internal.h"

namespace pam {

// tcgen05 forward of layer 0..4 (pam_conv_tc.cu); nx == 128 only. Layers 0-3
// write BF16 activations after bias and ReLU, layer 4 the FP32 logit z.
cudaError_t launch_conv_tc(int layer, const uint4 *in, const uint4 *wt, const float *bias, void *out, int F, int H,
                           int *status, cudaStream_t st);
cudaError_t prepare_conv_tc();

namespace {

constexpr int NL = 5;                                   // layers
// real input channels, output channels and input chunks of 8 channels of layer l
__host__ __device__ constexpr int CIN(int l) { return l == 0 ? 5 : 32; }
__host__ __device__ constexpr int COUT(int l) { return l == NL - 1 ? 1 : 32; }
__host__ __device__ constexpr int CINC(int l) { return l == 0 ? 1 : 4; }
// tensor-core weight layout of layer l: [9][TC_KCH][TC_NCO][8] BF16
__host__ __device__ constexpr int TC_KCH(int l) { return l == 0 ? 2 : 4; }
__host__ __device__ constexpr int TC_NCO(int l) { return l == NL - 1 ? 16 : 32; }
__host__ __device__ constexpr size_t tc_count(int l) { return (size_t)9 * TC_KCH(l) * TC_NCO(l) * 8; }
__host__ __device__ constexpr size_t tc_offset(int l) { return l == 0 ? 0 : tc_offset(l - 1) + tc_count(l - 1); }
constexpr int N_BANDS = 4;
constexpr float FEATURE_FLOOR = 1e-4f;
constexpr float WEIGHT_FLOOR = 0.05f;   // loss weight w = floor + (1 - floor) min(1, E / max E)
constexpr int CT = 128;        // threads (= pixels along a row) of a CUDA-core conv block
constexpr int PR = 2;          // output rows per conv block
constexpr int WSPLIT = 131;    // padded row stride (floats) of the weight-gradient staging; odd: no bank conflicts
constexpr int RS = 16;         // rows per weight-gradient block
constexpr int EPI_THREADS = 256;

__host__ __device__ constexpr size_t w_count(int l) { return (size_t)COUT(l) * CIN(l) * 9; }
__host__ __device__ constexpr size_t p_count(int l) { return w_count(l) + COUT(l); }
__host__ __device__ constexpr size_t p_offset(int l) { return l == 0 ? 0 : p_offset(l - 1) + p_count(l - 1); }
constexpr size_t N_PARAMS = p_offset(NL);
static_assert(N_PARAMS == 29505, "parameter count of the 5-layer network");

__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ float bf_of(unsigned short h) { return __uint_as_float((unsigned)h << 16); }
__device__ __forceinline__ unsigned pack_bf2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&v);
}
__device__ __forceinline__ float round_bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ------------------------------------------------------ preparation ----
// From the FP32 master parameters: forward weights wf[l] = [CINC*8][9][COUT]
// (input channel, tap u*3+v, output channel), rounded to BF16, zero for padded
// input channels; backward-data weights wb[l] (l >= 1), the forward weights of
// the adjoint convolution, wb[o][8 - t][c] = w[o][c][t], input o padded to a
// multiple of 8; the tensor-core layout of the 32 -> 32 layers (BF16 core
// matrices [tap][chunk][out channel][8]); biases as FP32.
struct PrepPtrs {
    float *wf[NL];
    float *wb[NL];
    float *bias[NL];
    uint16_t *wtc[NL];
};

__global__ void prep_kernel(const float *__restrict__ params, PrepPtrs pp)
{
    const int l = blockIdx.y;
    const float *w = params + p_offset(l);
    const float *b = w + w_count(l);
    const int ci_pad = CINC(l) * 8, co = COUT(l), ci = CIN(l);
    const int n_f = ci_pad * 9 * co;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_f; i += gridDim.x * blockDim.x) {
        const int o = i % co, t = (i / co) % 9, c = i / (co * 9);
        pp.wf[l][i] = c < ci ? round_bf(w[((size_t)o * ci + c) * 9 + t]) : 0.0f;
    }
    if (l >= 1) {
        const int o_pad = ((co + 7) / 8) * 8;   // input channels of the adjoint
        const int n_b = o_pad * 9 * ci;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_b; i += gridDim.x * blockDim.x) {
            const int c = i % ci, t = (i / ci) % 9, o = i / (ci * 9);
            pp.wb[l][i] = o < co ? round_bf(w[((size_t)o * ci + c) * 9 + (8 - t)]) : 0.0f;
        }
    }
    {   // tensor-core layout [tap][chunk of 8 input channels][GEMM column][8], zero padded
        const int kch = TC_KCH(l), nco = TC_NCO(l);
        const int n_t = (int)tc_count(l);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_t; i += gridDim.x * blockDim.x) {
            const int k = i % 8, o = (i / 8) % nco, ch = (i / (8 * nco)) % kch, t = i / (8 * nco * kch);
            const int c = ch * 8 + k;
            const float v = (o < co && c < ci) ? w[((size_t)o * ci + c) * 9 + t] : 0.0f;
            pp.wtc[l][i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < co; i += gridDim.x * blockDim.x) pp.bias[l][i] = b[i];
}

// ----------------------------------------------------------- Adam ----
// Kingma and Ba (2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / bc1) / (sqrt(v / bc2) + eps), bc = 1 - beta^t.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float bc1, float bc2,
                            float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------- features ----
// E = sum of the band energies (fixed order) and its per-frame maximum.
__global__ void __launch_bounds__(EPI_THREADS)
energy_kernel(const float *__restrict__ bands, int npix, float *__restrict__ E, unsigned *__restrict__ emax)
{
    const int f = blockIdx.y;
    float m = 0.0f;
    for (int x = blockIdx.x * EPI_THREADS + threadIdx.x; x < npix; x += gridDim.x * EPI_THREADS) {
        const float *b = bands + (size_t)f * N_BANDS * npix + x;
        const float e = ((b[0] + b[npix]) + b[2 * (size_t)npix]) + b[3 * (size_t)npix];
        E[(size_t)f * npix + x] = e;
        m = fmaxf(m, e);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
    __shared__ float wm[EPI_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < EPI_THREADS / 32; ++w) m = fmaxf(m, wm[w]);
        atomicMax(emax + f, __float_as_uint(m));   // E >= 0: float bits order as unsigned
    }
}

// Network input, chunked and padded: ch 0 = log10(E/max + floor)/4,
// ch 1..4 = log10(E_b/max + floor)/4, ch 5..7 = 0; the border is written as zeros.
__global__ void __launch_bounds__(EPI_THREADS)
features_kernel(const float *__restrict__ bands, const float *__restrict__ E, const unsigned *__restrict__ emax,
                int H, int W, uint4 *__restrict__ feat)
{
    const int f = blockIdx.y;
    const int HP = H + 2, WP = W + 2;
    const int npix = H * W;
    const float m = __uint_as_float(emax[f]);
    const float scale = m > 0.0f ? 1.0f / m : 0.0f;
    for (int q = blockIdx.x * EPI_THREADS + threadIdx.x; q < HP * WP; q += gridDim.x * EPI_THREADS) {
        const int i = q / WP - 1, j = q % WP - 1;
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (i >= 0 && i < H && j >= 0 && j < W) {
            const size_t x = (size_t)i * W + j;
            const float *b = bands + (size_t)f * N_BANDS * npix + x;
            float v[5];
            v[0] = log10f(E[(size_t)f * npix + x] * scale + FEATURE_FLOOR) * 0.25f;
#pragma unroll
            for (int k = 0; k < N_BANDS; ++k) v[1 + k] = log10f(b[(size_t)k * npix] * scale + FEATURE_FLOOR) * 0.25f;
            o = make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], 0.0f), 0u);
        }
        feat[(size_t)f * HP * WP + q] = o;
    }
}

// ------------------------------------------------- convolution (fwd) ----
// out = epi(b + sum_{c,u,v} w[o][c][u][v] in[c][i+u-1][j+v-1]) on CUDA cores.
// One block = 128 pixels of PR output rows; thread = one pixel column, PR x COUT
// FP32 accumulators. Inputs staged channel-major in shared memory (BF16),
// weights as FP32 [CIN][9][COUT] (read as broadcast float4).
enum { EPI_RELU = 0, EPI_MASK = 1, EPI_F32 = 2 };

template <int NCI, int NCO>
constexpr size_t conv_cc_smem()
{
    return (size_t)NCI * 8 * 9 * NCO * 4 + (size_t)(PR + 2) * NCI * 8 * (CT + 2) * 2;
}

template <int NCI, int NCO, int EPI>
__global__ void __launch_bounds__(CT)
conv_cc_kernel(const uint4 *__restrict__ in, const float *__restrict__ wt, const float *__restrict__ bias,
               const uint4 *__restrict__ mask, void *__restrict__ out, int H, int W)
{
    constexpr int CI = NCI * 8, SX = CT + 2;
    extern __shared__ __align__(16) unsigned char smem[];
    float *sW = reinterpret_cast<float *>(smem);                                       // [CI][9][NCO]
    unsigned short *sIn = reinterpret_cast<unsigned short *>(smem + (size_t)CI * 9 * NCO * 4);  // [PR+2][CI][SX]
    const int tx = threadIdx.x, f = blockIdx.z;
    const int r0 = blockIdx.y * PR, x0 = blockIdx.x * CT;
    const int HP = H + 2, WP = W + 2;

    for (int i = tx; i < CI * 9 * NCO / 4; i += CT)
        reinterpret_cast<float4 *>(sW)[i] = reinterpret_cast<const float4 *>(wt)[i];
    for (int idx = tx; idx < (PR + 2) * NCI * SX; idx += CT) {
        const int k = idx / (NCI * SX), rem = idx % (NCI * SX), c = rem / SX, px = rem % SX;
        const int row = r0 + k, col = x0 + px;   // padded coordinates
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < HP && col < WP) v = in[(((size_t)f * NCI + c) * HP + row) * WP + col];
        unsigned short *d = sIn + ((size_t)k * CI + c * 8) * SX + px;
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            d[(2 * q) * SX] = (unsigned short)(wv[q] & 0xFFFFu);
            d[(2 * q + 1) * SX] = (unsigned short)(wv[q] >> 16);
        }
    }
    __syncthreads();

    float acc[PR][NCO];
#pragma unroll
    for (int pr = 0; pr < PR; ++pr)
#pragma unroll
        for (int o = 0; o < NCO; ++o) acc[pr][o] = 0.0f;

#pragma unroll 1
    for (int ci = 0; ci < CI; ++ci) {
        float xs[PR + 2][3];
#pragma unroll
        for (int k = 0; k < PR + 2; ++k)
#pragma unroll
            for (int v = 0; v < 3; ++v) xs[k][v] = bf_of(sIn[((size_t)k * CI + ci) * SX + tx + v]);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int u = t / 3, v = t % 3;
            const float *wr = sW + ((size_t)ci * 9 + t) * NCO;
            if constexpr (NCO % 4 == 0) {
#pragma unroll
                for (int o4 = 0; o4 < NCO / 4; ++o4) {
                    const float4 w4 = reinterpret_cast<const float4 *>(wr)[o4];
#pragma unroll
                    for (int pr = 0; pr < PR; ++pr) {
                        const float x = xs[pr + u][v];
                        acc[pr][4 * o4 + 0] = fmaf(x, w4.x, acc[pr][4 * o4 + 0]);
                        acc[pr][4 * o4 + 1] = fmaf(x, w4.y, acc[pr][4 * o4 + 1]);
                        acc[pr][4 * o4 + 2] = fmaf(x, w4.z, acc[pr][4 * o4 + 2]);
                        acc[pr][4 * o4 + 3] = fmaf(x, w4.w, acc[pr][4 * o4 + 3]);
                    }
                }
            } else {
#pragma unroll
                for (int o = 0; o < NCO; ++o) {
                    const float w1 = wr[o];
#pragma unroll
                    for (int pr = 0; pr < PR; ++pr) acc[pr][o] = fmaf(xs[pr + u][v], w1, acc[pr][o]);
                }
            }
        }
    }

    const int j = x0 + tx;
    if (j >= W) return;
#pragma unroll
    for (int pr = 0; pr < PR; ++pr) {
        const int i = r0 + pr;
        if (i >= H) break;
        if constexpr (EPI == EPI_F32) {
            reinterpret_cast<float *>(out)[((size_t)f * H + i) * W + j] = acc[pr][0] + bias[0];
        } else {
            constexpr int NCH = NCO / 8;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
                const size_t o = (((size_t)f * NCH + ch) * HP + (i + 1)) * WP + (j + 1);
                float y[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) y[k] = acc[pr][ch * 8 + k];
                if constexpr (EPI == EPI_RELU) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) y[k] = fmaxf(y[k] + bias[ch * 8 + k], 0.0f);
                } else {
                    // dX = conv * (act > 0); act is a BF16 ReLU output, so > 0 <=> sign clear and nonzero
                    const uint4 mk = mask[o];
                    const unsigned mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const unsigned h = (k & 1) ? (mw[k >> 1] >> 16) : (mw[k >> 1] & 0xFFFFu);
                        if (h == 0u || (h & 0x8000u)) y[k] = 0.0f;
                    }
                }
                reinterpret_cast<uint4 *>(out)[o] =
                    make_uint4(pack_bf2(y[0], y[1]), pack_bf2(y[2], y[3]), pack_bf2(y[4], y[5]), pack_bf2(y[6], y[7]));
            }
        }
    }
}

// -------------------------------------------- convolution (weight grad) ----
// dW[o][c][u][v] = sum_{n,i,j} dY[n][o][i][j] X[n][c][i+u-1][j+v-1], db[o] = sum dY.
// Block = RS rows of one frame; per row it stages three input rows (FP32,
// channel-major, stride WSPLIT) and the row of dY, and each thread accumulates
// OG output channels x one input channel x 9 taps over its range of pixels with
// a sliding window along the row. Partial sums per block go to `part`
// ([block][COUT][CI][9] then [block][COUT] for db) and are summed in block order.
// Staging (inputs + dY row) or, at the end, the split reduction buffer
// [PXS][NCOMBO][OG * 10], whichever is larger.
template <int NCI, int NCO>
constexpr size_t wgrad_smem()
{
    constexpr size_t stage = (size_t)3 * NCI * 8 * WSPLIT * 4 + (size_t)NCO * (CT + 1) * 4;
    constexpr size_t red = (size_t)256 * (NCO >= 4 ? 4 : 1) * 10 * 4;
    return stage > red ? stage : red;
}

template <int NCI, int NCO>
__global__ void __launch_bounds__(256)
wgrad_kernel(const uint4 *__restrict__ X, const uint4 *__restrict__ dY, int H, int W, float *__restrict__ part)
{
    constexpr int CI = NCI * 8, OG = NCO >= 4 ? 4 : 1, NOG = NCO / OG, NCOMBO = CI * NOG;
    constexpr int PXS = 256 / NCOMBO;
    static_assert(PXS >= 1 && NCOMBO * PXS == 256, "thread mapping of the weight gradient");
    constexpr int NCY = (NCO + 7) / 8;      // chunks of dY
    extern __shared__ __align__(16) unsigned char smem[];
    float *sX = reinterpret_cast<float *>(smem);             // [3][CI][WSPLIT]
    float *sY = sX + 3 * CI * WSPLIT;                        // [NCO][CT+1]
    const int tid = threadIdx.x;
    const int c = tid % CI, og = (tid / CI) % NOG, s = tid / NCOMBO;
    const int f = blockIdx.y, strip = blockIdx.x;
    const int HP = H + 2, WP = W + 2;
    const int p_lo = s * W / PXS, p_hi = (s + 1) * W / PXS;

    float acc[OG][9], db[OG];
#pragma unroll
    for (int k = 0; k < OG; ++k) {
        db[k] = 0.0f;
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[k][t] = 0.0f;
    }
    for (int i = strip * RS; i < min(H, strip * RS + RS); ++i) {
        __syncthreads();
        for (int idx = tid; idx < 3 * NCI * WSPLIT; idx += 256) {
            const int u = idx / (NCI * WSPLIT), rem = idx % (NCI * WSPLIT), ch = rem / WSPLIT, px = rem % WSPLIT;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (px < WP) v = X[(((size_t)f * NCI + ch) * HP + (i + u)) * WP + px];
            float *d = sX + ((size_t)u * CI + ch * 8) * WSPLIT + px;
            d[0] = bf_lo(v.x); d[WSPLIT] = bf_hi(v.x);
            d[2 * WSPLIT] = bf_lo(v.y); d[3 * WSPLIT] = bf_hi(v.y);
            d[4 * WSPLIT] = bf_lo(v.z); d[5 * WSPLIT] = bf_hi(v.z);
            d[6 * WSPLIT] = bf_lo(v.w); d[7 * WSPLIT] = bf_hi(v.w);
        }
        for (int idx = tid; idx < NCY * W; idx += 256) {
            const int ch = idx / W, px = idx % W;
            const uint4 v = dY[(((size_t)f * NCY + ch) * HP + (i + 1)) * WP + (px + 1)];
            const float y8[8] = {bf_lo(v.x), bf_hi(v.x), bf_lo(v.y), bf_hi(v.y),
                                 bf_lo(v.z), bf_hi(v.z), bf_lo(v.w), bf_hi(v.w)};
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (ch * 8 + k < NCO) sY[(ch * 8 + k) * (CT + 1) + px] = y8[k];
        }
        __syncthreads();
        if (p_lo < p_hi) {
            float xw[3][3];
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) xw[u][v + 1] = sX[((size_t)u * CI + c) * WSPLIT + p_lo + v];
            for (int px = p_lo; px < p_hi; ++px) {
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    xw[u][0] = xw[u][1];
                    xw[u][1] = xw[u][2];
                    xw[u][2] = sX[((size_t)u * CI + c) * WSPLIT + px + 2];
                }
#pragma unroll
                for (int k = 0; k < OG; ++k) {
                    const float dy = sY[(og * OG + k) * (CT + 1) + px];
                    db[k] += dy;
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc[k][t] = fmaf(dy, xw[t / 3][t % 3], acc[k][t]);
                }
            }
        }
    }
    // combine the pixel splits in order, then write this block's partial
    __syncthreads();
    float *red = sX;   // [PXS][NCOMBO][OG*10]
    {
        float *d = red + ((size_t)s * NCOMBO + (tid % NCOMBO)) * (OG * 10);
#pragma unroll
        for (int k = 0; k < OG; ++k) {
#pragma unroll
            for (int t = 0; t < 9; ++t) d[k * 10 + t] = acc[k][t];
            d[k * 10 + 9] = db[k];
        }
    }
    __syncthreads();
    if (s == 0) {
        float *dst = part + ((size_t)f * gridDim.x + strip) * ((size_t)NCO * CI * 9 + NCO);
#pragma unroll
        for (int k = 0; k < OG; ++k) {
            const int o = og * OG + k;
#pragma unroll
            for (int t = 0; t < 10; ++t) {
                float sum = 0.0f;
                for (int q = 0; q < PXS; ++q) sum += red[((size_t)q * NCOMBO + tid) * (OG * 10) + k * 10 + t];
                if (t < 9) dst[((size_t)o * CI + c) * 9 + t] = sum;
                else if (c == 0) dst[(size_t)NCO * CI * 9 + o] = sum;
            }
        }
    }
}

// Sums the weight-gradient partials of all blocks (in block order) into the
// layer's slice of the gradient vector (real input channels only).
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int n_blocks, int ci_pad, int ci, int co,
                                    float *__restrict__ grad)
{
    const int nw = co * ci * 9;
    const size_t stride = (size_t)co * ci_pad * 9 + co;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + co; i += gridDim.x * blockDim.x) {
        size_t src;
        if (i < nw) {
            const int o = i / (ci * 9), c = (i / 9) % ci, t = i % 9;
            src = ((size_t)o * ci_pad + c) * 9 + t;
        } else {
            src = (size_t)co * ci_pad * 9 + (i - nw);
        }
        float s = 0.0f;
        for (int b = 0; b < n_blocks; ++b) s += part[(size_t)b * stride + src];
        grad[i] = s;
    }
}

// ------------------------------------------------------------ head ----
// Training: rho = eps + (1-eps) sigmoid(z), the energy-weighted loss
// (1/n) sum w (rho - target)^2 with w = floor + (1 - floor) min(1, E / max E)
// and E / max E = 10^(4 x0) - 1e-4 from the input's channel 0, and dL/dz into
// channel 0 of a chunked padded tensor (channels 1..7 zero).
__global__ void __launch_bounds__(EPI_THREADS)
loss_kernel(const float *__restrict__ z, const float *__restrict__ target, const uint4 *__restrict__ feat, int H,
            int W, float eps, float inv_n, uint4 *__restrict__ dz, float *__restrict__ loss_part)
{
    const int f = blockIdx.y;
    const int npix = H * W, HP = H + 2, WP = W + 2;
    float l = 0.0f;
    for (int x = blockIdx.x * EPI_THREADS + threadIdx.x; x < npix; x += gridDim.x * EPI_THREADS) {
        const float zz = z[(size_t)f * npix + x];
        const float s = 1.0f / (1.0f + expf(-zz));
        const float d = eps + (1.0f - eps) * s - target[(size_t)f * npix + x];
        const int i = x / W, j = x % W;
        const float x0 = bf_lo(feat[((size_t)f * HP + i + 1) * WP + j + 1].x);
        const float en = fminf(fmaxf(exp10f(4.0f * x0) - FEATURE_FLOOR, 0.0f), 1.0f);
        const float wgt = WEIGHT_FLOOR + (1.0f - WEIGHT_FLOOR) * en;
        l = fmaf(wgt * d, d, l);
        const float g = 2.0f * wgt * d * inv_n * (1.0f - eps) * s * (1.0f - s);
        dz[((size_t)f * HP + i + 1) * WP + j + 1] = make_uint4(pack_bf2(g, 0.0f), 0u, 0u, 0u);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
    __shared__ float wl[EPI_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wl[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < EPI_THREADS / 32; ++w) l += wl[w];
        loss_part[(size_t)f * gridDim.x + blockIdx.x] = l;
    }
}

__global__ void loss_reduce_kernel(const float *__restrict__ part, int n, float inv_n, float *__restrict__ loss)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = (float)(s * inv_n);
}

// Inference: rho = eps + (1-eps) sigmoid(z), its per-frame maximum, and the
// brightest pixel of the predicted image rho^2 E (key: value bits, then the
// lowest linear index).
__global__ void __launch_bounds__(EPI_THREADS)
head_kernel(const float *__restrict__ z, const float *__restrict__ E, int npix, float eps, float *__restrict__ rho,
            unsigned *__restrict__ rmax, unsigned long long *__restrict__ peak)
{
    const int f = blockIdx.y;
    float m = 0.0f;
    unsigned long long key = 0ull;
    for (int x = blockIdx.x * EPI_THREADS + threadIdx.x; x < npix; x += gridDim.x * EPI_THREADS) {
        const size_t o = (size_t)f * npix + x;
        const float r = eps + (1.0f - eps) / (1.0f + expf(-z[o]));
        rho[o] = r;
        m = fmaxf(m, r);
        const float img = r * r * E[o];
        const unsigned long long k = ((unsigned long long)__float_as_uint(img) << 32) | (0xFFFFFFFFu - (unsigned)x);
        key = k > key ? k : key;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
        key = o > key ? o : key;
    }
    __shared__ float wm[EPI_THREADS / 32];
    __shared__ unsigned long long wk[EPI_THREADS / 32];
    if ((threadIdx.x & 31) == 0) {
        wm[threadIdx.x >> 5] = m;
        wk[threadIdx.x >> 5] = key;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < EPI_THREADS / 32; ++w) {
            m = fmaxf(m, wm[w]);
            key = wk[w] > key ? wk[w] : key;
        }
        atomicMax(rmax + f, __float_as_uint(m));
        atomicMax(peak + f, key);
    }
}

// --------------------------------------------------------------- gate ----
// Per frame: the row tile (of the persistent batch kernel) that holds the
// predicted peak. Thread 0 also clears the work-queue heads.
__global__ void gate_items_kernel(const unsigned long long *__restrict__ peak, int F, int W, int rows_per_tile,
                                  int2 *__restrict__ items, unsigned *__restrict__ fmax_g,
                                  unsigned *__restrict__ fmax_x, int *__restrict__ counters)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f == 0) {
        counters[0] = 0;   // gate queue head
        counters[1] = 0;   // fallback queue head
        counters[2] = 0;   // fallback item count
    }
    if (f >= F) return;
    const unsigned idx = 0xFFFFFFFFu - (unsigned)(peak[f] & 0xFFFFFFFFull);
    items[f] = make_int2(f, (int)(idx / (unsigned)W) / rows_per_tile);
    fmax_g[f] = 0u;
    fmax_x[f] = 0u;
}

// Relative L2 distance, over the gate tile, between the predicted image
// rho_pred^2 E and the exact rho^2 E (both before the max normalisation).
// A frame whose distance exceeds tol (or is not finite) is queued for the
// exact path: all of its row tiles.
__global__ void __launch_bounds__(EPI_THREADS)
gate_check_kernel(const int2 *__restrict__ items, const float *__restrict__ rho_pred, const float *__restrict__ E,
                  const float *__restrict__ rho_x, const float *__restrict__ e_x, int H, int W, int rows_per_tile,
                  float tol, float *__restrict__ gate_err, int *__restrict__ gate_pass, int2 *__restrict__ fb_items,
                  int *__restrict__ counters)
{
    const int f = blockIdx.x;
    const int npix = H * W;
    const int row0 = items[f].y * rows_per_tile, row1 = min(H, row0 + rows_per_tile);
    double num = 0.0, den = 0.0;
    for (int x = row0 * W + threadIdx.x; x < row1 * W; x += EPI_THREADS) {
        const size_t o = (size_t)f * npix + x;
        const float rp = rho_pred[o], rx = rho_x[o];
        const double ip = (double)(rp * rp) * E[o], ix = (double)(rx * rx) * e_x[o];
        num += (ip - ix) * (ip - ix);
        den += ix * ix;
    }
    __shared__ double sn[EPI_THREADS], sd[EPI_THREADS];
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int s = EPI_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sn[threadIdx.x] += sn[threadIdx.x + s];
            sd[threadIdx.x] += sd[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = sn[0], d = sd[0];
        const float err = d > 0.0 ? (float)sqrt(n / d) : (n > 0.0 ? INFINITY : 0.0f);
        const bool pass = err <= tol;   // false for NaN
        gate_err[f] = err;
        gate_pass[f] = pass ? 1 : 0;
        if (!pass) {
            const int tiles = (H + rows_per_tile - 1) / rows_per_tile;
            const int base = atomicAdd(counters + 2, tiles);
            for (int t = 0; t < tiles; ++t) fb_items[base + t] = make_int2(f, t);
        }
    }
}

// rho_n and the image: the network's rho for frames that passed the gate (with
// the full-aperture energy), the exact rho and coherent energy otherwise.
__global__ void __launch_bounds__(EPI_THREADS)
learn_finalize_kernel(const int *__restrict__ gate_pass, const float *__restrict__ rho_pred,
                      const unsigned *__restrict__ rmax_pred, const float *__restrict__ E,
                      const float *__restrict__ rho_x, const float *__restrict__ e_x,
                      const unsigned *__restrict__ rmax_x, int npix, float *__restrict__ image,
                      float *__restrict__ rho_n)
{
    const int f = blockIdx.y;
    const bool pass = gate_pass[f] != 0;
    const float m = __uint_as_float(pass ? rmax_pred[f] : rmax_x[f]);
    const float *r = (pass ? rho_pred : rho_x) + (size_t)f * npix;
    const float *e = (pass ? E : e_x) + (size_t)f * npix;
    for (int x = blockIdx.x * EPI_THREADS + threadIdx.x; x < npix; x += gridDim.x * EPI_THREADS) {
        const float rn = r[x] / m;
        image[(size_t)f * npix + x] = rn * rn * e[x];
        if (rho_n) rho_n[(size_t)f * npix + x] = rn;
    }
}

// Exact rho_TAX of a training example, copied out of the workspace.
__global__ void copy_kernel(const float *__restrict__ src, float *__restrict__ dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void reset_kernel(unsigned *__restrict__ a, unsigned *__restrict__ b, unsigned long long *__restrict__ c,
                             int F)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < F) {
        a[f] = 0u;
        b[f] = 0u;
        c[f] = 0ull;
    }
}

template <int NCI, int NCO, int EPI>
cudaError_t conv_cc(const uint4 *in, const float *wt, const float *bias, const uint4 *mask, void *out, int F, int H,
                    int W, cudaStream_t st)
{
    dim3 grid((W + CT - 1) / CT, (H + PR - 1) / PR, F);
    conv_cc_kernel<NCI, NCO, EPI><<<grid, CT, conv_cc_smem<NCI, NCO>(), st>>>(in, wt, bias, mask, out, H, W);
    return cudaGetLastError();
}

template <int NCI, int NCO>
cudaError_t wgrad(const uint4 *X, const uint4 *dY, int F, int H, int W, float *part, cudaStream_t st)
{
    dim3 grid((H + RS - 1) / RS, F);
    wgrad_kernel<NCI, NCO><<<grid, 256, wgrad_smem<NCI, NCO>(), st>>>(X, dY, H, W, part);
    return cudaGetLastError();
}

template <int NCI, int NCO, int EPI>
cudaError_t set_conv_smem()
{
    return cudaFuncSetAttribute(conv_cc_kernel<NCI, NCO, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_cc_smem<NCI, NCO>());
}
template <int NCI, int NCO>
cudaError_t set_wgrad_smem()
{
    return cudaFuncSetAttribute(wgrad_kernel<NCI, NCO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)wgrad_smem<NCI, NCO>());
}

cudaError_t prepare_learn_kernels()
{
    cudaError_t e;
    if ((e = set_conv_smem<1, 32, EPI_RELU>()) != cudaSuccess) return e;
    if ((e = set_conv_smem<4, 32, EPI_RELU>()) != cudaSuccess) return e;
    if ((e = set_conv_smem<4, 1, EPI_F32>()) != cudaSuccess) return e;
    if ((e = set_conv_smem<1, 32, EPI_MASK>()) != cudaSuccess) return e;
    if ((e = set_conv_smem<4, 32, EPI_MASK>()) != cudaSuccess) return e;
    if ((e = set_wgrad_smem<1, 32>()) != cudaSuccess) return e;
    if ((e = set_wgrad_smem<4, 32>()) != cudaSuccess) return e;
    return set_wgrad_smem<4, 1>();
}

}  // namespace
}  // namespace pam

// ------------------------------------------------------------ object ----
struct pam_learn_s {
    pam_plan_s *plan = nullptr;   // owned: geometry, tables, time/lateral workspace
    pam_plan_s *gemm = nullptr;   // owned, with tensor cores on: BF16 form for the band energies
    int F = 0, H = 0, W = 0, HP = 0, WP = 0, tiles = 0, rpt = 0, n_sms = 0;
    size_t npix = 0, ppix = 0;    // nz*nx, (nz+2)*(nx+2)
    float gate_tol = 0.05f;
    bool use_tc = false;
    long long t = 0;              // Adam steps taken
    long long kernels = 0;
    // parameters
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    pam::PrepPtrs prep{};
    float *prep_mem = nullptr;
    uint16_t *tc_mem = nullptr;
    // activations and gradients (chunked, padded BF16)
    uint4 *feat = nullptr, *dz = nullptr;
    uint4 *act[4] = {nullptr, nullptr, nullptr, nullptr};
    uint4 *g[2] = {nullptr, nullptr};
    float *z = nullptr, *bands = nullptr, *E = nullptr, *rho = nullptr, *wpart = nullptr, *loss_part = nullptr;
    int loss_blocks = 0;
    unsigned *emax = nullptr, *rmax = nullptr, *fmax_g = nullptr, *fmax_x = nullptr;
    unsigned long long *peak = nullptr;
    // gate
    pam::BatchFrame *frames = nullptr;
    int2 *items_gate = nullptr, *items_all = nullptr, *items_fb = nullptr;
    int *counters = nullptr;
    float *gate_err = nullptr;
    int *gate_pass = nullptr;
    // ordering of the host-blocking state calls: `done` is recorded on the
    // caller's stream at the end of every queued call, and the state copies run
    // on the private stream `own` behind it, so they wait for this handle's work
    // only, not for other streams of the process
    cudaStream_t own = nullptr;
    cudaEvent_t done = nullptr;
};

namespace {

using pam::CIN;
using pam::CINC;
using pam::COUT;
using pam::NL;

pam_status lfail(pam_status s, const std::string &m) { return pam::set_error(s, m.c_str()); }
pam_status lcuda(cudaError_t e, const char *where)
{
    char m[512];
    std::snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
    return pam::set_error(PAM_ERR_CUDA, m);
}

#define LTRY(x)                                                 \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) return lcuda(e_, #x);            \
    } while (0)

template <class T>
cudaError_t zalloc(T **p, size_t n)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, (n ? n : 1) * sizeof(T));
    return e;
}

void learn_free(pam_learn_s *l)
{
    if (!l) return;
    auto fr = [](void *q) { if (q) cudaFree(q); };
    fr(l->params); fr(l->grads); fr(l->adam_m); fr(l->adam_v); fr(l->prep_mem); fr(l->tc_mem);
    fr(l->feat); fr(l->dz);
    for (auto *a : l->act) fr(a);
    for (auto *a : l->g) fr(a);
    fr(l->z); fr(l->bands); fr(l->E); fr(l->rho); fr(l->wpart); fr(l->loss_part);
    fr(l->emax); fr(l->rmax); fr(l->fmax_g); fr(l->fmax_x); fr(l->peak);
    fr(l->frames); fr(l->items_gate); fr(l->items_all); fr(l->items_fb); fr(l->counters);
    fr(l->gate_err); fr(l->gate_pass);
    if (l->gemm) pam_destroy(l->gemm);
    if (l->plan) pam_destroy(l->plan);
    if (l->done) cudaEventDestroy(l->done);
    if (l->own) cudaStreamDestroy(l->own);
    delete l;
}

// End of a queued call on `st`: later state calls wait for this point.
cudaError_t mark_done(pam_learn_s *l, cudaStream_t st) { return cudaEventRecord(l->done, st); }

// The private stream, ordered after this handle's most recent queued call.
cudaError_t own_after_last_call(pam_learn_s *l) { return cudaStreamWaitEvent(l->own, l->done, 0); }

pam_status check_dev(const void *ptr, const char *name, bool required)
{
    if (!ptr) return required ? lfail(PAM_ERR_INVALID_ARG, std::string(name) + " is NULL") : PAM_OK;
    if (reinterpret_cast<uintptr_t>(ptr) & 15u)
        return lfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return lfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return lfail(PAM_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return PAM_OK;
}

cudaError_t run_prep(pam_learn_s *l, cudaStream_t st)
{
    pam::prep_kernel<<<dim3(16, NL), 256, 0, st>>>(l->params, l->prep);
    l->kernels += 1;
    return cudaGetLastError();
}

int epi_grid(size_t n) { return (int)std::min<size_t>((n + pam::EPI_THREADS - 1) / pam::EPI_THREADS, 1024); }

// Features of n frames: time FFT, full-aperture lateral FFT, band energies,
// E and its maximum, network input.
cudaError_t run_features(pam_learn_s *l, const float *rf, int n, uint4 *feat, cudaStream_t st)
{
    pam_plan_s &p = *l->plan;
    cudaError_t e;
    pam::reset_kernel<<<(n + 127) / 128, 128, 0, st>>>(l->emax, l->rmax, l->peak, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = pam::launch_time_fft(p, rf, n, st)) != cudaSuccess) return e;
    if (l->use_tc && l->gemm) {
        // tensor-core form: sum_k |p_1 + p_2 + p_3|^2 per band from the same spectra
        if ((e = pam::launch_prec_bands(*l->gemm, p.w.S, n, pam::N_BANDS, l->bands, st)) != cudaSuccess) return e;
    } else {
        if ((e = pam::launch_lateral(p, n, 1, p.t.ones, st)) != cudaSuccess) return e;
        if ((e = pam::launch_prop_bands(p, n, pam::N_BANDS, l->bands, st)) != cudaSuccess) return e;
    }
    dim3 g1(epi_grid(l->npix), n);
    pam::energy_kernel<<<g1, pam::EPI_THREADS, 0, st>>>(l->bands, (int)l->npix, l->E, l->emax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 g2(epi_grid(l->ppix), n);
    pam::features_kernel<<<g2, pam::EPI_THREADS, 0, st>>>(l->bands, l->E, l->emax, l->H, l->W, feat);
    l->kernels += (l->use_tc && l->gemm) ? 7 : 6;
    return cudaGetLastError();
}

// Network forward: z (pre-sigmoid) of n frames. `keep` stores every hidden
// activation (training); otherwise two buffers alternate.
cudaError_t run_forward(pam_learn_s *l, const uint4 *feat, int n, bool keep, cudaStream_t st)
{
    const int H = l->H, W = l->W;
    cudaError_t e;
    uint4 *a[4] = {l->act[0], l->act[1], keep ? l->act[2] : l->act[0], keep ? l->act[3] : l->act[1]};
    if (l->use_tc) {
        auto wt = [&](int k) { return reinterpret_cast<const uint4 *>(l->prep.wtc[k]); };
        int *status = l->plan->w.status;
        if ((e = pam::launch_conv_tc(0, feat, wt(0), l->prep.bias[0], a[0], n, H, status, st)) != cudaSuccess)
            return e;
        for (int k = 1; k < 4; ++k)
            if ((e = pam::launch_conv_tc(k, a[k - 1], wt(k), l->prep.bias[k], a[k], n, H, status, st)) != cudaSuccess)
                return e;
        e = pam::launch_conv_tc(4, a[3], wt(4), l->prep.bias[4], l->z, n, H, status, st);
        l->kernels += 5;
        return e;
    }
    if ((e = pam::conv_cc<1, 32, pam::EPI_RELU>(feat, l->prep.wf[0], l->prep.bias[0], nullptr, a[0], n, H, W, st)) !=
        cudaSuccess)
        return e;
    for (int k = 1; k < 4; ++k)
        if ((e = pam::conv_cc<4, 32, pam::EPI_RELU>(a[k - 1], l->prep.wf[k], l->prep.bias[k], nullptr, a[k], n, H, W,
                                                    st)) != cudaSuccess)
            return e;
    e = pam::conv_cc<4, 1, pam::EPI_F32>(a[3], l->prep.wf[4], l->prep.bias[4], nullptr, l->z, n, H, W, st);
    l->kernels += 5;
    return e;
}

// Loss and gradients of n frames into l->grads (forward included).
cudaError_t run_grads(pam_learn_s *l, const uint4 *feat, const float *target, int n, float *loss, cudaStream_t st)
{
    const int H = l->H, W = l->W;
    cudaError_t e;
    if ((e = run_forward(l, feat, n, true, st)) != cudaSuccess) return e;
    const float inv_n = (float)(1.0 / ((double)n * l->npix));
    dim3 gl(l->loss_blocks, n);
    pam::loss_kernel<<<gl, pam::EPI_THREADS, 0, st>>>(l->z, target, feat, H, W, l->plan->d.eps, inv_n, l->dz,
                                                      l->loss_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (loss) {
        pam::loss_reduce_kernel<<<1, 32, 0, st>>>(l->loss_part, l->loss_blocks * n, inv_n, loss);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        l->kernels += 1;
    }
    const int nblk = ((H + pam::RS - 1) / pam::RS) * n;
    auto reduce = [&](int layer) -> cudaError_t {
        pam::wgrad_reduce_kernel<<<64, 256, 0, st>>>(l->wpart, nblk, CINC(layer) * 8, CIN(layer), COUT(layer),
                                                     l->grads + pam::p_offset(layer));
        return cudaGetLastError();
    };
    // layer 5: dY = dz, X = a4
    if ((e = pam::wgrad<4, 1>(l->act[3], l->dz, n, H, W, l->wpart, st)) != cudaSuccess) return e;
    if ((e = reduce(4)) != cudaSuccess) return e;
    if ((e = pam::conv_cc<1, 32, pam::EPI_MASK>(l->dz, l->prep.wb[4], nullptr, l->act[3], l->g[0], n, H, W, st)) !=
        cudaSuccess)
        return e;
    // layers 4, 3, 2: dY = g, X = a_{k-1}
    int cur = 0;
    for (int k = 3; k >= 1; --k) {
        if ((e = pam::wgrad<4, 32>(l->act[k - 1], l->g[cur], n, H, W, l->wpart, st)) != cudaSuccess) return e;
        if ((e = reduce(k)) != cudaSuccess) return e;
        if ((e = pam::conv_cc<4, 32, pam::EPI_MASK>(l->g[cur], l->prep.wb[k], nullptr, l->act[k - 1], l->g[cur ^ 1],
                                                    n, H, W, st)) != cudaSuccess)
            return e;
        cur ^= 1;
    }
    // layer 1: X = features
    if ((e = pam::wgrad<1, 32>(feat, l->g[cur], n, H, W, l->wpart, st)) != cudaSuccess) return e;
    if ((e = reduce(0)) != cudaSuccess) return e;
    l->kernels += 1 + 5 * 2 + 4;
    return cudaSuccess;
}

pam_status check_frames(pam_learn_s *l, int n)
{
    if (!l) return lfail(PAM_ERR_INVALID_ARG, "learned-form handle is NULL");
    if (n < 1 || n > l->F) return lfail(PAM_ERR_INVALID_ARG, "n_frames must be in [1, max_frames]");
    return PAM_OK;
}

}  // namespace

extern "C" {

size_t pam_learn_n_params(void) { return pam::N_PARAMS; }

pam_status pam_learn_create(const pam_plan_desc *d, pam_learn_t *out)
{
    if (!out) return lfail(PAM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return lfail(PAM_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->n_apod != 3) return lfail(PAM_ERR_INVALID_ARG, "the learned form predicts the AS-TAX weight (n_apod 3)");
    if (d->flags & ~PAM_EVANESCENT_ZERO)
        return lfail(PAM_ERR_UNSUPPORTED, "the learned form runs on the plain FP32 path (flags: PAM_EVANESCENT_ZERO)");
    pam_learn_s *l = new pam_learn_s();
    pam_status s = pam_plan_create(d, &l->plan);
    if (s != PAM_OK) {
        delete l;
        return s;
    }
    pam_plan_s &p = *l->plan;
    if (p.n_bins < pam::N_BANDS) {
        learn_free(l);
        return lfail(PAM_ERR_INVALID_ARG, "the learned form needs at least 4 bins (one per band)");
    }
    l->F = p.max_frames;
    l->H = p.nz;
    l->W = p.nx;
    l->HP = l->H + 2;
    l->WP = l->W + 2;
    l->npix = (size_t)l->H * l->W;
    l->ppix = (size_t)l->HP * l->WP;
    l->rpt = pam::prop_rows_per_cta(l->W);
    l->tiles = (l->H + l->rpt - 1) / l->rpt;
    l->n_sms = p.num_sms;
    l->loss_blocks = epi_grid(l->npix);
    const size_t F = (size_t)l->F;
    auto bad = [&](cudaError_t e) -> pam_status {
        pam_status r = e == cudaErrorMemoryAllocation ? lfail(PAM_ERR_OOM, "device allocation failed")
                                                      : lcuda(e, "learned-form set-up");
        learn_free(l);
        return r;
    };
#define LALLOC(x)                                \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return bad(e_);   \
    } while (0)
    LALLOC(zalloc(&l->params, pam::N_PARAMS));
    LALLOC(zalloc(&l->grads, pam::N_PARAMS));
    LALLOC(zalloc(&l->adam_m, pam::N_PARAMS));
    LALLOC(zalloc(&l->adam_v, pam::N_PARAMS));
    size_t prep_n = 0;
    for (int k = 0; k < NL; ++k) {
        prep_n += (size_t)CINC(k) * 8 * 9 * COUT(k) + COUT(k);
        if (k >= 1) prep_n += (size_t)((COUT(k) + 7) / 8 * 8) * 9 * CIN(k);
    }
    prep_n += 4 * NL;   // float4 alignment slack
    LALLOC(zalloc(&l->prep_mem, prep_n));
    LALLOC(zalloc(&l->tc_mem, pam::tc_offset(NL)));
    {
        float *q = l->prep_mem;
        auto take = [&](size_t n) { float *r = q; q += (n + 3) / 4 * 4; return r; };
        for (int k = 0; k < NL; ++k) {
            l->prep.wf[k] = take((size_t)CINC(k) * 8 * 9 * COUT(k));
            l->prep.wb[k] = k >= 1 ? take((size_t)((COUT(k) + 7) / 8 * 8) * 9 * CIN(k)) : nullptr;
            l->prep.bias[k] = take(COUT(k));
            l->prep.wtc[k] = l->tc_mem + pam::tc_offset(k);
        }
    }
    LALLOC(zalloc(&l->feat, F * l->ppix));
    LALLOC(zalloc(&l->dz, F * l->ppix));
    for (auto &a : l->act) LALLOC(zalloc(&a, F * 4 * l->ppix));
    for (auto &a : l->g) LALLOC(zalloc(&a, F * 4 * l->ppix));
    LALLOC(zalloc(&l->z, F * l->npix));
    LALLOC(zalloc(&l->bands, F * pam::N_BANDS * l->npix));
    LALLOC(zalloc(&l->E, F * l->npix));
    LALLOC(zalloc(&l->rho, F * l->npix));
    const size_t nblk = (size_t)((l->H + pam::RS - 1) / pam::RS) * F;
    LALLOC(zalloc(&l->wpart, nblk * (32 * 32 * 9 + 32)));
    LALLOC(zalloc(&l->loss_part, (size_t)l->loss_blocks * F));
    LALLOC(zalloc(&l->emax, F));
    LALLOC(zalloc(&l->rmax, F));
    LALLOC(zalloc(&l->fmax_g, F));
    LALLOC(zalloc(&l->fmax_x, F));
    LALLOC(zalloc(&l->peak, F));
    LALLOC(zalloc(&l->frames, F));
    LALLOC(zalloc(&l->items_gate, F));
    LALLOC(zalloc(&l->items_all, F * l->tiles));
    LALLOC(zalloc(&l->items_fb, F * l->tiles));
    LALLOC(zalloc(&l->counters, 4));
    LALLOC(zalloc(&l->gate_err, F));
    LALLOC(zalloc(&l->gate_pass, F));
    {
        std::vector<pam::BatchFrame> fr(F);
        std::vector<int2> all(F * l->tiles);
        for (size_t f = 0; f < F; ++f) {
            pam::BatchFrame &b = fr[f];
            b.Q = p.w.Q + f * p.n_bins * pam::q_per_bin(3, p.nx);
            b.phase = p.t.phase;
            b.bin_evan = p.t.bin_evan;
            b.n_bins = p.n_bins;
            b.nz = p.nz;
            b.nx = p.nx;
            b.nt = p.nt;
            b.z0f = (float)p.d.z0_m;
            b.dzf = (float)p.d.dz_m;
            b.out_off = f * l->npix;
            for (int t = 0; t < l->tiles; ++t) all[f * l->tiles + t] = make_int2((int)f, t);
        }
        LALLOC(cudaMemcpy(l->frames, fr.data(), sizeof(pam::BatchFrame) * F, cudaMemcpyHostToDevice));
        LALLOC(cudaMemcpy(l->items_all, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice));
    }
    LALLOC(cudaStreamCreateWithFlags(&l->own, cudaStreamNonBlocking));
    LALLOC(cudaEventCreateWithFlags(&l->done, cudaEventDisableTiming));
    LALLOC(cudaEventRecord(l->done, l->own));
    LALLOC(pam::prepare_learn_kernels());
    if (l->W == 128) LALLOC(pam::prepare_conv_tc());
    LALLOC(run_prep(l, nullptr));
    LALLOC(cudaDeviceSynchronize());
#undef LALLOC
    *out = l;
    return PAM_OK;
}

void pam_learn_destroy(pam_learn_t l)
{
    if (!l) return;
    cudaDeviceSynchronize();
    learn_free(l);
}

pam_status pam_learn_set_params(pam_learn_t l, const float *params, size_t n)
{
    if (!l || !params) return lfail(PAM_ERR_INVALID_ARG, "NULL argument");
    if (n != pam::N_PARAMS) return lfail(PAM_ERR_INVALID_ARG, "parameter count differs from pam_learn_n_params()");
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(params[i])) return lfail(PAM_ERR_NUMERIC, "non-finite parameter");
    LTRY(own_after_last_call(l));
    LTRY(cudaMemcpyAsync(l->params, params, n * sizeof(float), cudaMemcpyHostToDevice, l->own));
    LTRY(cudaMemsetAsync(l->adam_m, 0, n * sizeof(float), l->own));
    LTRY(cudaMemsetAsync(l->adam_v, 0, n * sizeof(float), l->own));
    l->t = 0;
    LTRY(run_prep(l, l->own));
    LTRY(cudaStreamSynchronize(l->own));
    return PAM_OK;
}

pam_status pam_learn_get_params(pam_learn_t l, float *params, size_t n)
{
    if (!l || !params) return lfail(PAM_ERR_INVALID_ARG, "NULL argument");
    if (n != pam::N_PARAMS) return lfail(PAM_ERR_INVALID_ARG, "parameter count differs from pam_learn_n_params()");
    LTRY(own_after_last_call(l));
    LTRY(cudaMemcpyAsync(params, l->params, n * sizeof(float), cudaMemcpyDeviceToHost, l->own));
    LTRY(cudaStreamSynchronize(l->own));
    return PAM_OK;
}

size_t pam_learn_state_size(void) { return 3 * pam::N_PARAMS; }

pam_status pam_learn_get_state(pam_learn_t l, float *state, size_t n, long long *adam_steps)
{
    if (!l || !state) return lfail(PAM_ERR_INVALID_ARG, "NULL argument");
    if (n != 3 * pam::N_PARAMS) return lfail(PAM_ERR_INVALID_ARG, "state size differs from pam_learn_state_size()");
    const size_t np = pam::N_PARAMS;
    LTRY(own_after_last_call(l));
    LTRY(cudaMemcpyAsync(state, l->params, np * sizeof(float), cudaMemcpyDeviceToHost, l->own));
    LTRY(cudaMemcpyAsync(state + np, l->adam_m, np * sizeof(float), cudaMemcpyDeviceToHost, l->own));
    LTRY(cudaMemcpyAsync(state + 2 * np, l->adam_v, np * sizeof(float), cudaMemcpyDeviceToHost, l->own));
    LTRY(cudaStreamSynchronize(l->own));
    if (adam_steps) *adam_steps = l->t;
    return PAM_OK;
}

pam_status pam_learn_set_state(pam_learn_t l, const float *state, size_t n, long long adam_steps)
{
    if (!l || !state) return lfail(PAM_ERR_INVALID_ARG, "NULL argument");
    if (n != 3 * pam::N_PARAMS) return lfail(PAM_ERR_INVALID_ARG, "state size differs from pam_learn_state_size()");
    if (adam_steps < 0) return lfail(PAM_ERR_INVALID_ARG, "adam_steps must be >= 0");
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(state[i])) return lfail(PAM_ERR_NUMERIC, "non-finite state value");
    for (size_t i = 2 * pam::N_PARAMS; i < n; ++i)
        if (state[i] < 0.0f) return lfail(PAM_ERR_INVALID_ARG, "Adam second moments must be >= 0");
    const size_t np = pam::N_PARAMS;
    LTRY(own_after_last_call(l));
    LTRY(cudaMemcpyAsync(l->params, state, np * sizeof(float), cudaMemcpyHostToDevice, l->own));
    LTRY(cudaMemcpyAsync(l->adam_m, state + np, np * sizeof(float), cudaMemcpyHostToDevice, l->own));
    LTRY(cudaMemcpyAsync(l->adam_v, state + 2 * np, np * sizeof(float), cudaMemcpyHostToDevice, l->own));
    l->t = adam_steps;
    LTRY(run_prep(l, l->own));
    LTRY(cudaStreamSynchronize(l->own));
    return PAM_OK;
}

pam_status pam_learn_configure(pam_learn_t l, float gate_tol, int use_tensor_cores)
{
    if (!l) return lfail(PAM_ERR_INVALID_ARG, "learned-form handle is NULL");
    if (std::isnan(gate_tol)) return lfail(PAM_ERR_INVALID_ARG, "gate_tol is NaN");
    if (use_tensor_cores && l->W != 128)
        return lfail(PAM_ERR_UNSUPPORTED, "the tensor-core convolution is built for nx == 128");
    if (use_tensor_cores && !l->gemm) {
        // the band energies' tensor-core form: a BF16 plan of the same geometry
        pam_plan_desc d = l->plan->d;
        d.bins = l->plan->bins.data();
        d.n_bins = (int)l->plan->bins.size();
        d.apod = l->plan->apod.data();
        d.flags = (d.flags & PAM_EVANESCENT_ZERO) | PAM_FORM_GEMM_BF16;
        pam_status s = pam_plan_create(&d, &l->gemm);
        // apertures the form cannot pack keep the FP32 band energies
        if (s == PAM_ERR_UNSUPPORTED) l->gemm = nullptr;
        else if (s != PAM_OK) return s;
    }
    l->gate_tol = gate_tol;
    l->use_tc = use_tensor_cores != 0;
    return PAM_OK;
}

size_t pam_learn_feature_bytes(pam_learn_t l) { return l ? l->ppix * 16 : 0; }

pam_status pam_learn_example(pam_learn_t l, const float *rf, int n_frames, void *features, float *target,
                             float *energy, void *stream)
{
    pam::TraceRange trace_("pam_learn_example");
    pam_status s;
    if ((s = check_frames(l, n_frames)) != PAM_OK) return s;
    if ((s = check_dev(rf, "rf", true)) != PAM_OK) return s;
    if ((s = check_dev(features, "features", true)) != PAM_OK) return s;
    if ((s = check_dev(target, "target", false)) != PAM_OK) return s;
    if ((s = check_dev(energy, "energy", false)) != PAM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pam_plan_s &p = *l->plan;
    uint4 *feat = static_cast<uint4 *>(features);
    LTRY(run_features(l, rf, n_frames, feat, st));
    if (energy) {
        pam::copy_kernel<<<256, 256, 0, st>>>(l->E, energy, (size_t)n_frames * l->npix);
        LTRY(cudaGetLastError());
        l->kernels += 1;
    }
    if (target) {
        // exact rho_TAX (Eq. 4, 10) of every pixel: the persistent kernel over all row tiles
        LTRY(pam::launch_lateral(p, n_frames, 3, p.t.apod, st));
        pam::gate_items_kernel<<<(n_frames + 127) / 128, 128, 0, st>>>(l->peak, 0, l->W, l->rpt, l->items_gate,
                                                                       l->fmax_g, l->fmax_x, l->counters);
        LTRY(cudaGetLastError());
        pam::EpiOut out;
        out.eps = p.d.eps;
        out.rho_tmp = target;
        out.e_tmp = p.w.e_tmp;
        out.fmax = l->fmax_x;
        out.status = p.w.status;
        const int n_items = n_frames * l->tiles;
        LTRY(pam::launch_prop_batch(l->W, 3, std::min(pam::prop_ctas_per_sm() * l->n_sms, n_items), l->frames, l->items_all, n_items,
                                    l->counters + 1, out, st));
        l->kernels += 3;
    }
    LTRY(mark_done(l, st));
    return PAM_OK;
}

pam_status pam_learn_forward(pam_learn_t l, const void *features, int n_frames, float *rho, void *stream)
{
    pam_status s;
    if ((s = check_frames(l, n_frames)) != PAM_OK) return s;
    if ((s = check_dev(features, "features", true)) != PAM_OK) return s;
    if ((s = check_dev(rho, "rho", true)) != PAM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LTRY(run_forward(l, static_cast<const uint4 *>(features), n_frames, false, st));
    // rho = eps + (1 - eps) sigmoid(z); E is not needed for rho itself (the peak key uses it)
    pam::reset_kernel<<<(n_frames + 127) / 128, 128, 0, st>>>(l->emax, l->rmax, l->peak, n_frames);
    dim3 g(epi_grid(l->npix), n_frames);
    pam::head_kernel<<<g, pam::EPI_THREADS, 0, st>>>(l->z, l->E, (int)l->npix, l->plan->d.eps, rho, l->rmax, l->peak);
    LTRY(cudaGetLastError());
    l->kernels += 2;
    LTRY(mark_done(l, st));
    return PAM_OK;
}

pam_status pam_learn_grads(pam_learn_t l, const void *features, const float *target, int n_frames, float *grads,
                           float *loss, void *stream)
{
    pam_status s;
    if ((s = check_frames(l, n_frames)) != PAM_OK) return s;
    if ((s = check_dev(features, "features", true)) != PAM_OK) return s;
    if ((s = check_dev(target, "target", true)) != PAM_OK) return s;
    if ((s = check_dev(grads, "grads", false)) != PAM_OK) return s;
    if ((s = check_dev(loss, "loss", false)) != PAM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LTRY(run_grads(l, static_cast<const uint4 *>(features), target, n_frames, loss, st));
    if (grads) {
        LTRY(cudaMemcpyAsync(grads, l->grads, pam::N_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    LTRY(mark_done(l, st));
    return PAM_OK;
}

pam_status pam_learn_train_step(pam_learn_t l, const void *features, const float *target, int n_frames, float lr,
                                float *loss, void *stream)
{
    pam::TraceRange trace_("pam_learn_train_step");
    pam_status s;
    if ((s = check_frames(l, n_frames)) != PAM_OK) return s;
    if ((s = check_dev(features, "features", true)) != PAM_OK) return s;
    if ((s = check_dev(target, "target", true)) != PAM_OK) return s;
    if ((s = check_dev(loss, "loss", false)) != PAM_OK) return s;
    if (!(lr > 0.0f) || !std::isfinite(lr)) return lfail(PAM_ERR_INVALID_ARG, "lr must be a positive number");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LTRY(run_grads(l, static_cast<const uint4 *>(features), target, n_frames, loss, st));
    l->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - std::pow(b1, (double)l->t)), bc2 = (float)(1.0 - std::pow(b2, (double)l->t));
    const int n = (int)pam::N_PARAMS;
    pam::adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(l->params, l->grads, l->adam_m, l->adam_v, n, lr, (float)b1,
                                                       (float)b2, bc1, bc2, 1e-8f);
    LTRY(cudaGetLastError());
    LTRY(run_prep(l, st));
    l->kernels += 1;
    LTRY(mark_done(l, st));
    return PAM_OK;
}

pam_status pam_learn_tax(pam_learn_t l, const float *rf, int n_frames, float *image, float *rho_n, float *gate_err,
                         int *gate_pass, void *stream)
{
    pam::TraceRange trace_("pam_learn_tax");
    if (!l) return lfail(PAM_ERR_INVALID_ARG, "learned-form handle is NULL");
    if (n_frames < 0) return lfail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return PAM_OK;
    pam_status s;
    if ((s = check_dev(rf, "rf", true)) != PAM_OK) return s;
    if ((s = check_dev(image, "image", true)) != PAM_OK) return s;
    if ((s = check_dev(rho_n, "rho_n", false)) != PAM_OK) return s;
    if ((s = check_dev(gate_err, "gate_err", false)) != PAM_OK) return s;
    if ((s = check_dev(gate_pass, "gate_pass", false)) != PAM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pam_plan_s &p = *l->plan;
    const size_t fr_in = (size_t)p.ne * p.nt;
    for (int f0 = 0; f0 < n_frames; f0 += l->F) {
        const int n = std::min(l->F, n_frames - f0);
        LTRY(run_features(l, rf + (size_t)f0 * fr_in, n, l->feat, st));
        LTRY(run_forward(l, l->feat, n, false, st));
        dim3 g(epi_grid(l->npix), n);
        pam::head_kernel<<<g, pam::EPI_THREADS, 0, st>>>(l->z, l->E, (int)l->npix, p.d.eps, l->rho, l->rmax, l->peak);
        LTRY(cudaGetLastError());
        // gate: exact TAX on the row tile of the predicted peak
        pam::gate_items_kernel<<<(n + 127) / 128, 128, 0, st>>>(l->peak, n, l->W, l->rpt, l->items_gate, l->fmax_g,
                                                                l->fmax_x, l->counters);
        LTRY(cudaGetLastError());
        LTRY(pam::launch_lateral(p, n, 3, p.t.apod, st));
        pam::EpiOut out;
        out.eps = p.d.eps;
        out.rho_tmp = p.w.rho_tmp;
        out.e_tmp = p.w.e_tmp;
        out.fmax = l->fmax_g;
        out.status = p.w.status;
        LTRY(pam::launch_prop_batch(l->W, 3, std::min(pam::prop_ctas_per_sm() * l->n_sms, n), l->frames, l->items_gate, n, l->counters,
                                    out, st));
        float *gerr = gate_err ? gate_err + f0 : l->gate_err;
        int *gpass = gate_pass ? gate_pass + f0 : l->gate_pass;
        pam::gate_check_kernel<<<n, pam::EPI_THREADS, 0, st>>>(l->items_gate, l->rho, l->E, p.w.rho_tmp, p.w.e_tmp,
                                                               l->H, l->W, l->rpt, l->gate_tol, gerr, gpass,
                                                               l->items_fb, l->counters);
        LTRY(cudaGetLastError());
        // fallback: the plain method on every row tile of the frames that missed the gate
        out.fmax = l->fmax_x;
        LTRY(pam::launch_prop_batch(l->W, 3, pam::prop_ctas_per_sm() * l->n_sms, l->frames, l->items_fb, n * l->tiles, l->counters + 1, out,
                                    st, l->counters + 2));
        pam::learn_finalize_kernel<<<g, pam::EPI_THREADS, 0, st>>>(
            gpass, l->rho, l->rmax, l->E, p.w.rho_tmp, p.w.e_tmp, l->fmax_x, (int)l->npix, image + (size_t)f0 * l->npix,
            rho_n ? rho_n + (size_t)f0 * l->npix : nullptr);
        LTRY(cudaGetLastError());
        l->kernels += 7;
    }
    LTRY(mark_done(l, st));
    return PAM_OK;
}

pam_status pam_learn_sync(pam_learn_t l, void *stream)
{
    if (!l) return lfail(PAM_ERR_INVALID_ARG, "learned-form handle is NULL");
    return pam_sync(l->plan, stream);
}

pam_status pam_learn_info(pam_learn_t l, long long *kernel_launches, int *max_frames, long long *adam_steps)
{
    if (!l) return lfail(PAM_ERR_INVALID_ARG, "learned-form handle is NULL");
    if (kernel_launches) {
        long long k = 0;
        pam_profile_read(l->plan, nullptr, nullptr, &k);
        *kernel_launches = l->kernels + k;
        l->kernels = 0;
    }
    if (max_frames) *max_frames = l->F;
    if (adam_steps) *adam_steps = l->t;
    return PAM_OK;
}

}  // extern "C"
