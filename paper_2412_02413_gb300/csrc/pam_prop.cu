// pam_prop.cu -- the fused propagate-and-correlate kernel and the NCC/TAX
// epilogue.
//
// For every frequency bin w_k of Omega, depth row z_j and apodization q:
//   P_q(kx_u, z_j) = Q_q(kx_u) * exp(i kz z_j)              (Eq. 2)
//   p~_q(x_i, z_j) = sum_u P_q exp(+2 pi i u i / nx)        (inverse F_x; 1/nx is already in Q)
// followed by per-pixel sums over the bins:
//   A_qq += |p~_q|^2,  C_qr += Re conj(p~_q) p~_r           (Eq. 3, Eq. 4 + Appendix A)
// The fields p~ stay in registers and shared memory; only the per-pixel sums
// reach global memory. The epilogue forms rho_qr, the eps clamp, rho_TAX
// (Eq. 10), its per-frame maximum, rho_n and the image (Eq. 5 / 11).
//
// Work mapping of the fused kernel: 8 warps per CTA. Each depth row is owned
// by 2*(nx/16) lanes that each hold 8 pixels of that row for all apodizations.
// The nx-point inverse DFT is one radix-2 decimation-in-frequency split,
// folded into the phase words as below, followed by two (nx/2)-point halves.
// Each half is an 8-point DFT in registers, a twiddle, a transpose through
// padded shared memory and an (nx/16)-point DFT in registers. A CTA loops over
// a contiguous chunk of bins. Each bin's spectra and phase words are staged in
// shared memory with cp.async, double-buffered.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"

namespace pam {

cudaError_t prepare_fft_kernels(const pam_plan_s &p);

namespace {

constexpr int PROP_WARPS = 8;
constexpr int PROP_THREADS = 32 * PROP_WARPS;

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// sum_u v_u * exp(+2 pi i u k / N), natural order, in place.
__device__ __forceinline__ void idft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    float2 id13 = make_float2(-d13.y, d13.x);  // i * d13
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, id13);
    a3 = csub(d02, id13);
}

template <int N> struct IDft;
template <> struct IDft<1> { static __device__ __forceinline__ void run(float2 (&)[1]) {} };
template <> struct IDft<2> {
    static __device__ __forceinline__ void run(float2 (&v)[2])
    {
        float2 t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    }
};
template <> struct IDft<4> {
    static __device__ __forceinline__ void run(float2 (&v)[4]) { idft4(v[0], v[1], v[2], v[3]); }
};
template <> struct IDft<8> {
    static __device__ __forceinline__ void run(float2 (&v)[8])
    {
        const float r = 0.70710678118654752440f;
        float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        idft4(e0, e1, e2, e3);
        idft4(o0, o1, o2, o3);
        // o_k *= exp(+2 pi i k / 8)
        o1 = make_float2(r * (o1.x - o1.y), r * (o1.x + o1.y));
        o2 = make_float2(-o2.y, o2.x);
        o3 = make_float2(-r * (o3.x + o3.y), r * (o3.x - o3.y));
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};

// exp(2 pi i * w / 2^64) for a fixed-point phase word w. The top 32 bits,
// read as a signed turn count in [-1/2, 1/2), carry the angle; sincospif
// takes it in half-turns.
__device__ __forceinline__ float2 dds_phasor(uint64_t w)
{
    const int hi = (int)(uint32_t)(w >> 32);
    const float t = (float)hi * 4.6566128730773926e-10f;  // 2^-31
    float s, c;
    sincospif(t, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int NX> struct Shape {
    static constexpr int H = NX / 2;               // half length
    static constexpr int L2 = H / 8;               // lanes per half row
    static constexpr int LPR = 2 * L2;             // lanes per row
    static constexpr int RPW = 32 / LPR;           // rows per warp
    static constexpr int RPC = PROP_WARPS * RPW;   // rows per CTA
    static constexpr int KPL = 8 / L2;             // second-stage DFTs per lane
    static constexpr int TS = L2 + 1;              // padded transpose row (float2)
    static constexpr int RS = 8 * TS;              // transpose region per (aperture, row, half)
    static constexpr int LOG2NX = NX == 16 ? 4 : NX == 32 ? 5 : NX == 64 ? 6 : 7;
    static_assert(NX == 16 || NX == 32 || NX == 64 || NX == 128, "built lateral lengths");
};

template <int NAP> struct Acc { static constexpr int N = NAP == 1 ? 1 : (NAP == 2 ? 3 : 6); };

template <int NAP, int NX>
constexpr size_t prop_smem_bytes()
{
    using S = Shape<NX>;
    return (size_t)2 * NAP * NX * sizeof(float2)          // spectra, two stages
           + (size_t)2 * NX * sizeof(ulonglong2)          // phase words
           + (size_t)2 * NX * sizeof(float)               // evanescent coefficients
           + (size_t)PROP_WARPS * NAP * S::RPW * 2 * S::RS * sizeof(float2);  // transposes
}

template <int NAP, int NX, bool FIELDS>
__global__ void __launch_bounds__(PROP_THREADS, 2)
prop_corr_kernel(const float2 *__restrict__ Q, const ulonglong2 *__restrict__ dds,
                 const float *__restrict__ ecoef, const int *__restrict__ bin_evan, int n_bins, int nz,
                 float z0f, float dzf, int n_split, float *__restrict__ part, float2 *__restrict__ fields)
{
    using S = Shape<NX>;
    constexpr int H = S::H, L2 = S::L2, LPR = S::LPR, RPW = S::RPW, RPC = S::RPC, KPL = S::KPL;
    constexpr int TS = S::TS, RS = S::RS;
    constexpr int NACC = Acc<NAP>::N;
    constexpr int NOUT = KPL * L2;  // 8 pixels per lane

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sQ = reinterpret_cast<float2 *>(smem_raw);
    ulonglong2 *sD = reinterpret_cast<ulonglong2 *>(sQ + 2 * NAP * NX);
    float *sE = reinterpret_cast<float *>(sD + 2 * NX);
    float2 *sT = reinterpret_cast<float2 *>(sE + 2 * NX);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = lane / LPR, g = (lane % LPR) / L2, n2 = lane % L2;
    const int f = blockIdx.z, split = blockIdx.y;
    const int j = blockIdx.x * RPC + warp * RPW + r;
    const bool row_ok = j < nz;
    const int jj = row_ok ? j : nz - 1;
    const int b_begin = (int)(((long long)n_bins * split) / n_split);
    const int b_end = (int)(((long long)n_bins * (split + 1)) / n_split);

    float2 *myT = sT + (size_t)warp * (NAP * RPW * 2 * RS);

    // second-factor twiddles exp(+2 pi i n2 k1 / H)
    float2 tw1[8];
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        float s, c;
        sincospif(2.0f * (float)((n2 * k1) % H) / (float)H, &s, &c);
        tw1[k1] = make_float2(c, s);
    }
    // Radix-2 DIF split folded into the phase: lanes of half g take
    // x_g[n'] = exp(2 pi i g n'/nx) (P[n'] + (-1)^g P[n'+H]).
    const uint64_t g_unit = g ? (1ull << (64 - S::LOG2NX)) : 0ull;
    const uint64_t g_half = g ? (1ull << 63) : 0ull;
    const uint64_t jw = (uint64_t)jj;
    const float zj = z0f + (float)jj * dzf;

    float acc[NOUT][NACC];
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[o][a] = 0.0f;

    constexpr int NQ4 = NAP * NX / 2, ND4 = NX, NE4 = NX / 4;
    constexpr int NT4 = NQ4 + ND4 + NE4;
    auto stage_in = [&](int b, int stage) {
        const uint4 *gq = reinterpret_cast<const uint4 *>(Q + ((size_t)f * n_bins + b) * NAP * NX);
        const uint4 *gd = reinterpret_cast<const uint4 *>(dds + (size_t)b * NX);
        const uint4 *ge = reinterpret_cast<const uint4 *>(ecoef + (size_t)b * NX);
        uint4 *dq = reinterpret_cast<uint4 *>(sQ + stage * NAP * NX);
        uint4 *dd = reinterpret_cast<uint4 *>(sD + stage * NX);
        uint4 *de = reinterpret_cast<uint4 *>(sE + stage * NX);
        for (int i = tid; i < NT4; i += PROP_THREADS) {
            if (i < NQ4) cp_async16(dq + i, gq + i);
            else if (i < NQ4 + ND4) cp_async16(dd + (i - NQ4), gd + (i - NQ4));
            else cp_async16(de + (i - NQ4 - ND4), ge + (i - NQ4 - ND4));
        }
        cp_async_commit();
    };

    if (b_begin < b_end) stage_in(b_begin, 0);
    cp_async_wait_all();
    __syncthreads();

    for (int b = b_begin; b < b_end; ++b) {
        const int stage = (b - b_begin) & 1;
        if (b + 1 < b_end) stage_in(b + 1, stage ^ 1);
        const float2 *cQ = sQ + stage * NAP * NX;
        const ulonglong2 *cD = sD + stage * NX;
        const float *cE = sE + stage * NX;
        const bool evan = bin_evan[b] != 0;

        // Eq. 2 phasors of this lane's 16 lateral bins at depth z_j
        float2 ph0[8], ph1[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            const int u0 = L2 * n1 + n2;
            const ulonglong2 d0 = cD[u0], d1 = cD[u0 + H];
            const uint64_t off = g_unit * (uint64_t)u0;
            ph0[n1] = dds_phasor(d0.x + jw * d0.y + off);
            ph1[n1] = dds_phasor(d1.x + jw * d1.y + off + g_half);
            if (evan) {
                const float a0 = exp2f(cE[u0] * zj), a1 = exp2f(cE[u0 + H] * zj);
                ph0[n1] = make_float2(ph0[n1].x * a0, ph0[n1].y * a0);
                ph1[n1] = make_float2(ph1[n1].x * a1, ph1[n1].y * a1);
            }
        }

        // first factor: 8-point DFT over n1, twiddle, into the transpose region
#pragma unroll
        for (int q = 0; q < NAP; ++q) {
            float2 x[8];
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const int u0 = L2 * n1 + n2;
                x[n1] = cadd(cmul(cQ[q * NX + u0], ph0[n1]), cmul(cQ[q * NX + u0 + H], ph1[n1]));
            }
            IDft<8>::run(x);
            float2 *reg = myT + ((q * RPW + r) * 2 + g) * RS;
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) reg[k1 * TS + n2] = k1 ? cmul(x[k1], tw1[k1]) : x[k1];
        }
        __syncwarp();

        // second factor: L2-point DFTs over n2; lane owns pixels i = 2(k1 + 8 k2) + g
        float2 p[NAP][NOUT];
#pragma unroll
        for (int q = 0; q < NAP; ++q) {
            const float2 *reg = myT + ((q * RPW + r) * 2 + g) * RS;
#pragma unroll
            for (int s = 0; s < KPL; ++s) {
                const int k1 = n2 * KPL + s;
                float2 v[L2];
#pragma unroll
                for (int t = 0; t < L2; ++t) v[t] = reg[k1 * TS + t];
                IDft<L2>::run(v);
#pragma unroll
                for (int k2 = 0; k2 < L2; ++k2) p[q][s * L2 + k2] = v[k2];
            }
        }

        // per-pixel sums over the bins
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const float2 a = p[0][o];
            acc[o][0] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[o][0]));
            if constexpr (NAP >= 2) {
                const float2 bb = p[1][o];
                acc[o][1] = fmaf(bb.x, bb.x, fmaf(bb.y, bb.y, acc[o][1]));
                if constexpr (NAP == 2) {
                    acc[o][2] = fmaf(a.x, bb.x, fmaf(a.y, bb.y, acc[o][2]));
                } else {
                    const float2 cc = p[2][o];
                    acc[o][2] = fmaf(cc.x, cc.x, fmaf(cc.y, cc.y, acc[o][2]));
                    acc[o][3] = fmaf(a.x, bb.x, fmaf(a.y, bb.y, acc[o][3]));
                    acc[o][4] = fmaf(bb.x, cc.x, fmaf(bb.y, cc.y, acc[o][4]));
                    acc[o][5] = fmaf(cc.x, a.x, fmaf(cc.y, a.y, acc[o][5]));
                }
            }
        }
        if constexpr (FIELDS) {
            if (row_ok) {
                float2 *dst = fields + (((size_t)f * n_bins + b) * nz + j) * NX;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const int k1 = n2 * KPL + o / L2, k2 = o % L2;
                    dst[2 * (k1 + 8 * k2) + g] = p[0][o];
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    if (row_ok) {
        const size_t plane = (size_t)nz * NX;
        float *dst = part + (size_t)(f * n_split + split) * NACC * plane + (size_t)j * NX;
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int k1 = n2 * KPL + o / L2, k2 = o % L2;
            const int i = 2 * (k1 + 8 * k2) + g;
#pragma unroll
            for (int a = 0; a < NACC; ++a) dst[a * plane + i] = acc[o][a];
        }
    }
}

// --------------------------------------------------------- epilogue ----

__device__ __forceinline__ double ncc_pair(float c, float aq, float ar, double eps)
{
    // Eq. 4 with an FP64 denominator; zero denominator -> eps; clamp at eps.
    double den = sqrt((double)aq * (double)ar);
    double rho = den > 0.0 ? (double)c / den : eps;
    return rho < eps ? eps : rho;
}

constexpr int EPI_THREADS = 256;

template <int NAP>
__global__ void __launch_bounds__(EPI_THREADS)
epi_reduce_kernel(const float *__restrict__ part, int n_split, int npix, float eps,
                  float *__restrict__ out_main, float *__restrict__ rho_tmp, float *__restrict__ e_tmp,
                  float *__restrict__ rho_pairs, float *__restrict__ image_as, unsigned *__restrict__ fmax)
{
    constexpr int NACC = Acc<NAP>::N;
    const int f = blockIdx.y;
    const int x = blockIdx.x * EPI_THREADS + threadIdx.x;
    float rho = 0.0f;
    if (x < npix) {
        float a[NACC];
#pragma unroll
        for (int c = 0; c < NACC; ++c) a[c] = 0.0f;
        for (int s = 0; s < n_split; ++s) {
            const float *src = part + (size_t)(f * n_split + s) * NACC * npix + x;
#pragma unroll
            for (int c = 0; c < NACC; ++c) a[c] += src[(size_t)c * npix];
        }
        const size_t o = (size_t)f * npix + x;
        if constexpr (NAP == 1) {
            out_main[o] = a[0];
        } else {
            float E;
            if constexpr (NAP == 2) {
                double r12 = ncc_pair(a[2], a[0], a[1], eps);
                rho = (float)r12;
                if (rho_pairs) rho_pairs[o] = rho;
                E = a[0] + a[1] + 2.0f * a[2];
            } else {
                double r12 = ncc_pair(a[3], a[0], a[1], eps);
                double r23 = ncc_pair(a[4], a[1], a[2], eps);
                double r31 = ncc_pair(a[5], a[2], a[0], eps);
                if (rho_pairs) {
                    rho_pairs[(size_t)f * 3 * npix + x] = (float)r12;
                    rho_pairs[(size_t)f * 3 * npix + npix + x] = (float)r23;
                    rho_pairs[(size_t)f * 3 * npix + 2 * npix + x] = (float)r31;
                }
                rho = cbrtf((float)(r12 * r23 * r31));  // Eq. 10
                E = (a[0] + a[1] + a[2]) + 2.0f * (a[3] + a[4] + a[5]);
            }
            E = fmaxf(E, 0.0f);
            rho_tmp[o] = rho;
            e_tmp[o] = E;
            if (image_as) image_as[o] = E;
        }
    }
    if constexpr (NAP > 1) {
        // block max of rho (all rho > 0, so the float bits order like unsigned ints)
        __shared__ float wmax[EPI_THREADS / 32];
        float m = rho;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            m = threadIdx.x < EPI_THREADS / 32 ? wmax[threadIdx.x] : 0.0f;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
            if (threadIdx.x == 0) atomicMax(&fmax[f], __float_as_uint(m));
        }
    }
}

__global__ void __launch_bounds__(EPI_THREADS)
epi_normalize_kernel(const float *__restrict__ rho_tmp, const float *__restrict__ e_tmp,
                     const unsigned *__restrict__ fmax, int npix, float *__restrict__ image,
                     float *__restrict__ rho_n)
{
    const int f = blockIdx.y;
    const int x = blockIdx.x * EPI_THREADS + threadIdx.x;
    if (x >= npix) return;
    const size_t o = (size_t)f * npix + x;
    const float m = __uint_as_float(fmax[f]);
    const float rn = rho_tmp[o] / m;   // rho_n (Sec. II-A): maximum becomes exactly 1
    image[o] = rn * rn * e_tmp[o];     // Eq. 5 / Eq. 11
    if (rho_n) rho_n[o] = rn;
}

template <int NAP, int NX, bool FIELDS>
cudaError_t launch_prop_t(const pam_plan_s &p, int n_frames, int n_split, float *fields, cudaStream_t st)
{
    using S = Shape<NX>;
    dim3 grid((p.nz + S::RPC - 1) / S::RPC, n_split, n_frames);
    prop_corr_kernel<NAP, NX, FIELDS><<<grid, PROP_THREADS, prop_smem_bytes<NAP, NX>(), st>>>(
        p.w.Q, p.t.dds, p.t.ecoef, p.t.bin_evan, p.n_bins, p.nz, (float)p.d.z0_m, (float)p.d.dz_m, n_split,
        p.w.part, reinterpret_cast<float2 *>(fields));
    return cudaGetLastError();
}

template <int NX>
cudaError_t launch_prop_nx(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields,
                           cudaStream_t st)
{
    if (napq == 1) {
        return fields ? launch_prop_t<1, NX, true>(p, n_frames, n_split, fields, st)
                      : launch_prop_t<1, NX, false>(p, n_frames, n_split, nullptr, st);
    }
    if (napq == 2) return launch_prop_t<2, NX, false>(p, n_frames, n_split, nullptr, st);
    return launch_prop_t<3, NX, false>(p, n_frames, n_split, nullptr, st);
}

template <int NAP, int NX, bool FIELDS>
cudaError_t set_smem()
{
    return cudaFuncSetAttribute(prop_corr_kernel<NAP, NX, FIELDS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)prop_smem_bytes<NAP, NX>());
}

template <int NX>
cudaError_t prepare_nx()
{
    cudaError_t e;
    if ((e = set_smem<1, NX, false>()) != cudaSuccess) return e;
    if ((e = set_smem<1, NX, true>()) != cudaSuccess) return e;
    if ((e = set_smem<2, NX, false>()) != cudaSuccess) return e;
    return set_smem<3, NX, false>();
}

}  // namespace

int prop_rows_per_cta(int nx) { return PROP_WARPS * (32 / (nx / 8)); }

int choose_split(const pam_plan_s &p, int n_frames)
{
    const int rows = prop_rows_per_cta(p.nx);
    const long long row_tiles = (p.nz + rows - 1) / rows;
    const long long target = 2LL * p.num_sms;
    long long ns = target / (row_tiles * n_frames);
    if (ns < 1) ns = 1;
    if (ns > p.n_bins) ns = p.n_bins;
    return (int)ns;
}

cudaError_t launch_prop(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields, cudaStream_t st)
{
    switch (p.nx) {
    case 16: return launch_prop_nx<16>(p, n_frames, napq, n_split, fields, st);
    case 32: return launch_prop_nx<32>(p, n_frames, napq, n_split, fields, st);
    case 64: return launch_prop_nx<64>(p, n_frames, napq, n_split, fields, st);
    case 128: return launch_prop_nx<128>(p, n_frames, napq, n_split, fields, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epilogue(const pam_plan_s &p, int n_frames, int napq, int n_split, float *out_main,
                            float *rho_n, float *rho_pairs, float *image_as, cudaStream_t st)
{
    const int npix = p.nz * p.nx;
    dim3 grid((npix + EPI_THREADS - 1) / EPI_THREADS, n_frames);
    if (napq == 1) {
        epi_reduce_kernel<1><<<grid, EPI_THREADS, 0, st>>>(p.w.part, n_split, npix, p.d.eps, out_main, nullptr,
                                                           nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError();
    }
    if (napq == 2)
        epi_reduce_kernel<2><<<grid, EPI_THREADS, 0, st>>>(p.w.part, n_split, npix, p.d.eps, nullptr, p.w.rho_tmp,
                                                           p.w.e_tmp, rho_pairs, image_as, p.w.fmax);
    else
        epi_reduce_kernel<3><<<grid, EPI_THREADS, 0, st>>>(p.w.part, n_split, npix, p.d.eps, nullptr, p.w.rho_tmp,
                                                           p.w.e_tmp, rho_pairs, image_as, p.w.fmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    epi_normalize_kernel<<<grid, EPI_THREADS, 0, st>>>(p.w.rho_tmp, p.w.e_tmp, p.w.fmax, npix, out_main, rho_n);
    return cudaGetLastError();
}

cudaError_t prepare_kernels(const pam_plan_s &p)
{
    cudaError_t e = prepare_fft_kernels(p);
    if (e != cudaSuccess) return e;
    switch (p.nx) {
    case 16: return prepare_nx<16>();
    case 32: return prepare_nx<32>();
    case 64: return prepare_nx<64>();
    case 128: return prepare_nx<128>();
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pam
