// pam_prec.cu -- tensor-core form of the propagate-and-correlate step
// (PAM_FORM_GEMM_*).
//
// For bin w_k and depth row z_j, Eq. 1-2 map the apodized channel spectra to
// the row's fields through a circulant matrix:
//   p~_q(x_i, z_j) = sum_e c_j[(i - e) mod nx] a_q[e] S[e],
//   c_j[d] = (1/nx) sum_u exp(i kz_u z_j) exp(+2 pi i u d / nx),
// i.e. the inverse lateral DFT of the row's propagator phasors. The plan
// tabulates c_j once per (bin, row) from the exact FP64 phase words, in
// 16-bit form. A call then evaluates the sum over elements for 16 frames at a
// time as one tcgen05 GEMM per (bin, row) with M = 128 pixels,
// N = 2 x 16 (Re, Im of each frame) and K = 2 x elements:
//   A[i][k] = Re or Im c_j[(i - e_k) mod nx]   (expanded in shared memory)
//   B[k][n] = +-Re or Im of a S / sigma          (packed per call)
// so that the real GEMM yields Re and Im of the complex sum. Disjoint
// apertures are disjoint K ranges: one MMA chain per aperture accumulates
// into its own tensor-memory region. The epilogue reads the accumulators
// with tcgen05.ld and adds |p_q|^2 and Re conj(p_q) p_r into per-pixel
// registers across all bins (Eq. 3-4). The NCC/TAX epilogue kernels then
// finish exactly as in the FP32 path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"

namespace pam {
namespace {

constexpr int NXP = 128;                    // lateral length of this form
constexpr int FG = kFramesPerGroup;         // frames per CTA
constexpr int NG = 2 * FG;                  // GEMM N
constexpr int CS_A = NXP / 8 * 128;         // bytes between K chunks of A (core matrices 8 x 16 B)
constexpr int CS_B = NG / 8 * 128;          // bytes between K chunks of B
constexpr int GEMM_THREADS = 256;             // 8 warps: 2 per tensor-memory lane quarter
constexpr int TMEM_COLS = 256;              // >= 3 apertures x NG
constexpr int DS_LEN = 136;                 // entries of one shifted copy of the reversed c vector

// Offset (in 16-bit entries) of 8-entry block q of the copy of D shifted by sh,
// for half `part` (0 = Re, 1 = Im). Blocks with the same q sit next to each
// other for the 8 shifts, so the 8 lanes of a quarter warp, whose shifts are
// distinct, read 8 different 16-byte bank groups.
__device__ __forceinline__ int ds_off(int part, int sh, int q) { return ((part * (DS_LEN / 8) + q) * 8 + sh) * 8; }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---- 16-bit conversions ----
template <bool FP16>
__device__ __forceinline__ unsigned short to16(float v)
{
    if constexpr (FP16) return __half_as_ushort(__float2half_rn(v));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <bool FP16>
__device__ __forceinline__ float from16(unsigned short u)
{
    if constexpr (FP16) return __half2float(__ushort_as_half(u));
    else return __bfloat162float(__ushort_as_bfloat16(u));
}

// ---- mbarrier / bulk copy / tcgen05 (inline PTX) ----
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait (about one second of SM cycles); false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// UMMA shared-memory descriptor, canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, `lbo` bytes between core matrices along K,
// `sbo` bytes between 8-row groups, descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulators, A and B both BF16 (1)
// or FP16 (0), K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <bool FP16>
__device__ __forceinline__ unsigned umma_idesc()
{
    const unsigned fmt = FP16 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(NG >> 3) << 17) | ((unsigned)(NXP >> 4) << 24);
}

__device__ __forceinline__ void umma(unsigned tmem_d, uint64_t a, uint64_t b, unsigned idesc, unsigned accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8])
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = __uint_as_float(r[t]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// ------------------------------------------------------- plan tables ----
// c_j[d] for one (row j, bin b) per CTA, d = threadIdx.x. Phasors come from
// the exact fixed-point phase words with accurate sincospif (the table is
// built once per plan); the inverse lateral DFT is a direct FP32 sum.
template <bool FP16>
__global__ void __launch_bounds__(NXP)
prec_table_kernel(const uint4 *__restrict__ phase, const float *__restrict__ live, int nz, double z0, double dz,
                  uint32_t *__restrict__ chi, uint32_t *__restrict__ clo)
{
    __shared__ float2 ph[NXP];
    __shared__ float2 tw[NXP];
    const int j = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
    const uint4 d = phase[(size_t)b * NXP + t];
    const unsigned jw = (unsigned)j;
    const unsigned w = d.x + jw * d.y + __umulhi(jw, d.z);
    float s, c;
    sincospif((float)(int)w * 4.6566128730773926e-10f, &s, &c);  // turns * 2
    const float zj = (float)(z0 + (double)j * dz);
    const float amp = exp2f(__uint_as_float(d.w) * zj) * live[(size_t)b * NXP + t];
    ph[t] = make_float2(c * amp, s * amp);
    sincospif(2.0f * (float)t / (float)NXP, &s, &c);
    tw[t] = make_float2(c, s);
    __syncthreads();
    float re = 0.f, im = 0.f;
    for (int u = 0; u < NXP; ++u) {
        const float2 p = ph[u], e = tw[(u * t) & (NXP - 1)];
        re = fmaf(p.x, e.x, fmaf(-p.y, e.y, re));
        im = fmaf(p.x, e.y, fmaf(p.y, e.x, im));
    }
    re *= 1.0f / NXP;
    im *= 1.0f / NXP;
    const unsigned short hr = to16<FP16>(re), hi = to16<FP16>(im);
    const size_t o = ((size_t)b * nz + j) * NXP + t;
    chi[o] = (unsigned)hr | ((unsigned)hi << 16);
    if (clo) {
        const unsigned short lr = to16<FP16>(re - from16<FP16>(hr)), li = to16<FP16>(im - from16<FP16>(hi));
        clo[o] = (unsigned)lr | ((unsigned)li << 16);
    }
}

// ----------------------------------------------------- per-call prep ----
// max |Re S|, |Im S| of each frame (bits of a non-negative float).
__global__ void prec_smax_kernel(const float2 *__restrict__ S, int n_bins, int ne, unsigned *__restrict__ smax)
{
    const int b = blockIdx.x, f = blockIdx.y;
    float m = 0.f;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const float2 v = S[((size_t)f * n_bins + b) * ne + e];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&smax[f], __float_as_uint(m));
}

// Power-of-2 scale 2^E >= max of the frame, so that S / 2^E is exact and
// within [-1, 1] (FP16 range); E = 0 for an all-zero frame.
__device__ __forceinline__ int frame_exp(unsigned bits)
{
    const float m = __uint_as_float(bits);
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);   // m = f * 2^e, f in [0.5, 1)
    return e;
}

// B tile of one (bin, frame group): N = 2 x 16 rows (Re / Im output of each
// frame), K-major in the canonical no-swizzle layout. Column k of aperture q
// holds a_q S[e] (scaled) for the real half of the K range, and the values
// that pair with Im c for the imaginary half:
//   Re p = sum Re c Re s - Im c Im s,   Im p = sum Re c Im s + Im c Re s.
template <bool FP16, bool SPLIT>
__global__ void __launch_bounds__(256)
prec_bprep_kernel(const float2 *__restrict__ S, const short *__restrict__ ktab, const float *__restrict__ kwgt,
                  int K, int n_bins, int ne, int F, const unsigned *__restrict__ smax, uint8_t *__restrict__ Bhi,
                  uint8_t *__restrict__ Blo)
{
    const int b = blockIdx.x, g = blockIdx.y;
    const size_t tile = (size_t)K * NG * 2;
    uint8_t *dh = Bhi + ((size_t)g * n_bins + b) * tile;
    uint8_t *dl = SPLIT ? Blo + ((size_t)g * n_bins + b) * tile : nullptr;
    for (int idx = threadIdx.x; idx < K * NG; idx += blockDim.x) {
        const int k = idx / NG, n = idx % NG;
        const int f = g * FG + n / 2, kind = n & 1;
        float v = 0.f;
        const short kt = ktab[k];
        if (f < F && kt >= 0) {
            const int e = kt & 0x3FFF, imag = (kt >> 14) & 1;
            const float sc = kwgt[k] * ldexpf(1.0f, -frame_exp(smax[f]));
            const float2 s = S[((size_t)f * n_bins + b) * ne + e];
            const float sr = s.x * sc, si = s.y * sc;
            v = imag == 0 ? (kind == 0 ? sr : si) : (kind == 0 ? -si : sr);
        }
        const unsigned short h = to16<FP16>(v);
        const size_t off = (size_t)(k / 8) * CS_B + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
        *reinterpret_cast<unsigned short *>(dh + off) = h;
        if (SPLIT) *reinterpret_cast<unsigned short *>(dl + off) = to16<FP16>(v - from16<FP16>(h));
    }
}

// ------------------------------------------------------------- GEMM ----
// One CTA per (depth row j, group of 32 frames); 8 warps. Bins run in
// sequence: bulk-copy the bin's B tile(s) and the row's c words, expand A
// (the circulant) into shared memory, issue the MMA chains (thread 0), wait
// for their commit, and fold the accumulators into per-pixel sums. Warp w
// reads tensor-memory lane quarter w % 4 (pixels 32 (w%4) .. +31) for frames
// 16 (w/4) .. +15, so each thread keeps 16 frames x n_acc sums in registers.
template <int NAP, bool FP16, bool SPLIT>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
prec_gemm_kernel(const uint32_t *__restrict__ chi, const uint32_t *__restrict__ clo, const uint8_t *__restrict__ Bhi,
                 const uint8_t *__restrict__ Blo, const short *__restrict__ ktab, int K, int4 kq, int n_bins, int nz,
                 int F, const unsigned *__restrict__ smax, float *__restrict__ part, int *__restrict__ status,
                 bool fast)
{
    constexpr int NACC = NAP == 2 ? 3 : 6;
    constexpr int FH = FG / 2;                                // frames per epilogue thread
    extern __shared__ __align__(1024) uint8_t sm[];
    const int KC = K / 8;                                     // K chunks of 8
    uint8_t *sA = sm;                                         // KC * CS_A
    uint8_t *sB = sA + (size_t)KC * CS_A;                     // KC * CS_B
    uint8_t *sBl = sB + (size_t)KC * CS_B;                    // KC * CS_B (split)
    uint32_t *sC = reinterpret_cast<uint32_t *>(sBl + (SPLIT ? (size_t)KC * CS_B : 0));  // [2][NXP]
    short *sK = reinterpret_cast<short *>(sC + 2 * NXP);      // [K]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sK + ((K + 7) & ~7));  // [2]: data, mma
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);
    unsigned short *sDs = reinterpret_cast<unsigned short *>(bar + 4);   // [2 halves][8 shifts][DS_LEN]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = blockIdx.x, grp = blockIdx.y;
    const int quarter = warp & 3, fhalf = warp >> 2;
    const int i_epi = 32 * quarter + lane;                   // pixel of this thread's accumulator lane
    const int i_exp = tid & (NXP - 1), hpar = tid >> 7;      // expansion: pixel row, parity of its K chunks
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = tid; k < K; k += GEMM_THREADS) sK[k] = ktab[k];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const unsigned idesc = umma_idesc<FP16>();
    const int kqa[4] = {kq.x, kq.y, kq.z, kq.w};
    const unsigned bytesB = (unsigned)K * NG * 2;
    const size_t tileB = bytesB;

    float acc[FH][NACC];
#pragma unroll
    for (int f = 0; f < FH; ++f)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[f][a] = 0.f;

    unsigned ph_data = 0, ph_mma = 0;
    bool ok = true, data_pending = false, mma_pending = false;
    for (int b = 0; b < n_bins; ++b) {
        if (tid == 0) {
            mbar_expect_tx(&bar[0], (SPLIT ? 2u : 1u) * (bytesB + NXP * 4u));
            bulk_g2s(sB, Bhi + ((size_t)grp * n_bins + b) * tileB, bytesB, &bar[0]);
            bulk_g2s(sC, chi + ((size_t)b * nz + j) * NXP, NXP * 4, &bar[0]);
            if (SPLIT) {
                bulk_g2s(sBl, Blo + ((size_t)grp * n_bins + b) * tileB, bytesB, &bar[0]);
                bulk_g2s(sC + NXP, clo + ((size_t)b * nz + j) * NXP, NXP * 4, &bar[0]);
            }
        }
        ok = __syncthreads_and(mbar_wait(&bar[0], ph_data)) != 0;
        ph_data ^= 1u;
        if (!ok) {
            data_pending = true;
            break;
        }
#pragma unroll 1
        for (int pass = 0; pass < (SPLIT ? 2 : 1); ++pass) {
            // A[i][k] = (Re or Im) c[(i - e_k) mod 128]: row i of the circulant, one 16-byte
            // core-matrix row per K chunk.
            const uint32_t *cw = sC + pass * NXP;
            if (fast) {
                // Every K chunk is 8 consecutive elements e0..e0+7 of one half, so its row-i
                // segment is D[(e0 - i) mod 128 .. +8) with D[m] = c[(-m) mod 128]: one aligned
                // 16-byte load from the copy of D shifted by (e0 - i) mod 8. The copies are built
                // 8 entries at a time: D_s[8q + t] = c[-(8q + s + t)].
                for (int pq = tid; pq < 8 * (DS_LEN / 8); pq += GEMM_THREADS) {
                    const int sh = pq / (DS_LEN / 8), q = pq % (DS_LEN / 8);
                    unsigned w[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) w[t] = cw[(-(8 * q + sh + t)) & (NXP - 1)];
                    const uint4 re = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                                                __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                    const uint4 im = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                                                __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
                    *reinterpret_cast<uint4 *>(sDs + ds_off(0, sh, q)) = re;
                    *reinterpret_cast<uint4 *>(sDs + ds_off(1, sh, q)) = im;
                }
                __syncthreads();
                for (int ch = hpar; ch < KC; ch += 2) {
                    const short kt = sK[ch * 8];
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (kt >= 0) {
                        const int e0 = kt & 0x3FFF, part_im = (kt >> 14) & 1;
                        const int m0 = (e0 - i_exp) & (NXP - 1);
                        v = *reinterpret_cast<const uint4 *>(sDs + ds_off(part_im, m0 & 7, m0 >> 3));
                    }
                    *reinterpret_cast<uint4 *>(sA + (size_t)ch * CS_A + (i_exp / 8) * 128 + (i_exp % 8) * 16) = v;
                }
            } else {
                for (int ch = hpar; ch < KC; ch += 2) {
                    unsigned w4[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        unsigned h2 = 0;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const short kt = sK[ch * 8 + 2 * t + h];
                            unsigned v = 0;
                            if (kt >= 0) {
                                const int e = kt & 0x3FFF, imag = (kt >> 14) & 1;
                                v = (cw[(i_exp - e) & (NXP - 1)] >> (16 * imag)) & 0xFFFFu;
                            }
                            h2 |= v << (16 * h);
                        }
                        w4[t] = h2;
                    }
                    *reinterpret_cast<uint4 *>(sA + (size_t)ch * CS_A + (i_exp / 8) * 128 + (i_exp % 8) * 16) =
                        make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
#pragma unroll
                for (int q = 0; q < NAP; ++q) {
                    const unsigned dq = tmem + (unsigned)(q * NG);
                    for (int s = kqa[q] / 16; s < kqa[q + 1] / 16; ++s) {
                        const uint64_t da = umma_desc(smem_u32(sA) + s * 2 * CS_A, CS_A, 128);
                        const uint64_t dbh = umma_desc(smem_u32(sB) + s * 2 * CS_B, CS_B, 128);
                        const bool first = pass == 0 && s == kqa[q] / 16;
                        if (pass == 0) {
                            umma(dq, da, dbh, idesc, first ? 0u : 1u);
                            if (SPLIT) umma(dq, da, umma_desc(smem_u32(sBl) + s * 2 * CS_B, CS_B, 128), idesc, 1u);
                        } else {
                            umma(dq, da, dbh, idesc, 1u);
                        }
                    }
                }
                umma_commit(&bar[1]);
            }
            ok = __syncthreads_and(mbar_wait(&bar[1], ph_mma)) != 0;
            ph_mma ^= 1u;
            tc_fence_after();
            if (!ok) {
                mma_pending = true;
                break;
            }
        }
        if (!ok) break;
        // fold this bin's fields into the per-pixel sums (4 frames per tensor-memory read)
        const unsigned lane_base = tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)(fhalf * 2 * FH);
#pragma unroll
        for (int fc = 0; fc < FH / 4; ++fc) {
            float r[NAP][8];
#pragma unroll
            for (int q = 0; q < NAP; ++q) tmem_ld8(lane_base + (unsigned)(q * NG + fc * 8), r[q]);
            tmem_wait_ld();
#pragma unroll
            for (int ff = 0; ff < 4; ++ff) {
                const int f = fc * 4 + ff;
                const float ar = r[0][2 * ff], ai = r[0][2 * ff + 1];
                const float br = r[1][2 * ff], bi = r[1][2 * ff + 1];
                acc[f][0] = fmaf(ar, ar, fmaf(ai, ai, acc[f][0]));
                acc[f][1] = fmaf(br, br, fmaf(bi, bi, acc[f][1]));
                if constexpr (NAP == 2) {
                    acc[f][2] = fmaf(ar, br, fmaf(ai, bi, acc[f][2]));
                } else {
                    const float cr = r[2][2 * ff], ci = r[2][2 * ff + 1];
                    acc[f][2] = fmaf(cr, cr, fmaf(ci, ci, acc[f][2]));
                    acc[f][3] = fmaf(ar, br, fmaf(ai, bi, acc[f][3]));
                    acc[f][4] = fmaf(br, cr, fmaf(bi, ci, acc[f][4]));
                    acc[f][5] = fmaf(cr, ar, fmaf(ci, ai, acc[f][5]));
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) {
        atomicOr(status, 1);
        // let the copies / MMAs still in flight finish before shared and tensor memory go away
        if (data_pending) mbar_wait(&bar[0], ph_data ^ 1u);
        if (mma_pending) mbar_wait(&bar[1], ph_mma ^ 1u);
    }
    // Partial sums of the whole bin range, rescaled by sigma^2, as split 0 of the FP32 path's layout.
    const size_t npix = (size_t)nz * NXP;
#pragma unroll
    for (int f = 0; f < FH; ++f) {
        const int fr = grp * FG + fhalf * FH + f;
        if (fr < F && ok) {
            const float s2 = ldexpf(1.0f, 2 * frame_exp(smax[fr]));
#pragma unroll
            for (int a = 0; a < NACC; ++a)
                part[((size_t)fr * NACC + a) * npix + (size_t)j * NXP + i_epi] = acc[f][a] * s2;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Software-pipelined GEMM (16-bit operands, no split; K <= 256). Two sets of
// shared-memory buffers (A, B, c, shifted copies) and two tensor-memory
// accumulator sets let the CUDA cores expand A for bin b+1 and fold the sums
// of bin b while the tensor core runs the MMAs of the neighbouring bin:
//   wait data(b+1), expand(b+1) | MMA(b) running
//   wait MMA(b), load(b+2), issue MMA(b+1)
//   fold sums of bin b           | MMA(b+1) running
constexpr int TMEM_COLS_PIPE = 512;   // 2 x 3 apertures x NG

template <int NAP, bool FP16>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
prec_gemm_pipe_kernel(const uint32_t *__restrict__ chi, const uint8_t *__restrict__ Bhi, const short *__restrict__ ktab,
                      int K, int4 kq, int n_bins, int nz, int F, const unsigned *__restrict__ smax,
                      float *__restrict__ part, int *__restrict__ status, bool fast)
{
    constexpr int NACC = NAP == 2 ? 3 : 6;
    constexpr int FH = FG / 2;
    constexpr int ACC_COLS = NAP * NG;
    extern __shared__ __align__(1024) uint8_t sm[];
    const int KC = K / 8;
    const size_t szA = (size_t)KC * CS_A, szB = (size_t)KC * CS_B;
    uint8_t *sA[2] = {sm, sm + szA};
    uint8_t *sB[2] = {sm + 2 * szA, sm + 2 * szA + szB};
    uint32_t *sC0 = reinterpret_cast<uint32_t *>(sm + 2 * szA + 2 * szB);              // [2][NXP]
    unsigned short *sD0 = reinterpret_cast<unsigned short *>(sC0 + 2 * NXP);           // [2][2][8][DS_LEN]
    short *sK = reinterpret_cast<short *>(sD0 + 2 * 2 * 8 * DS_LEN);                   // [K]
    uint64_t *bar = reinterpret_cast<uint64_t *>(sK + ((K + 7) & ~7));                 // data[2], mma[2]
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = blockIdx.x, grp = blockIdx.y;
    const int quarter = warp & 3, fhalf = warp >> 2;
    const int i_epi = 32 * quarter + lane;
    const int i_exp = tid & (NXP - 1), hpar = tid >> 7;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS_PIPE)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int x = 0; x < 4; ++x) mbar_init(&bar[x], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = tid; k < K; k += GEMM_THREADS) sK[k] = ktab[k];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const unsigned idesc = umma_idesc<FP16>();
    const int kqa[4] = {kq.x, kq.y, kq.z, kq.w};
    const unsigned bytesB = (unsigned)K * NG * 2;

    float acc[FH][NACC];
#pragma unroll
    for (int f = 0; f < FH; ++f)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[f][a] = 0.f;

    int loads_issued = 0, loads_done = 0, mmas_issued = 0, mmas_done = 0;  // thread 0's bookkeeping
    auto issue_load = [&](int b) {
        if (tid == 0) {
            const int bb = b & 1;
            mbar_expect_tx(&bar[bb], bytesB + NXP * 4u);
            bulk_g2s(sB[bb], Bhi + ((size_t)grp * n_bins + b) * bytesB, bytesB, &bar[bb]);
            bulk_g2s(sC0 + bb * NXP, chi + ((size_t)b * nz + j) * NXP, NXP * 4, &bar[bb]);
            ++loads_issued;
        }
    };
    // Waits are per thread; the go / abort decision is made uniform at the one
    // CTA barrier of each bin (__syncthreads_and before the MMA issue).
    auto wait_data = [&](int b) -> bool {
        const bool r = mbar_wait(&bar[b & 1], (b >> 1) & 1);
        if (r && tid == 0) ++loads_done;
        return r;
    };
    auto expand = [&](int b) {
        const int bb = b & 1;
        const uint32_t *cw = sC0 + bb * NXP;
        unsigned short *sDs = sD0 + bb * 2 * 8 * DS_LEN;
        uint8_t *A = sA[bb];
        if (fast) {
            for (int pq = tid; pq < 8 * (DS_LEN / 8); pq += GEMM_THREADS) {
                const int sh = pq / (DS_LEN / 8), q = pq % (DS_LEN / 8);
                unsigned w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) w[t] = cw[(-(8 * q + sh + t)) & (NXP - 1)];
                *reinterpret_cast<uint4 *>(sDs + ds_off(0, sh, q)) =
                    make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                               __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                *reinterpret_cast<uint4 *>(sDs + ds_off(1, sh, q)) =
                    make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                               __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
            }
            __syncthreads();
            for (int ch = hpar; ch < KC; ch += 2) {
                const short kt = sK[ch * 8];
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (kt >= 0) {
                    const int e0 = kt & 0x3FFF, part_im = (kt >> 14) & 1;
                    const int m0 = (e0 - i_exp) & (NXP - 1);
                    v = *reinterpret_cast<const uint4 *>(sDs + ds_off(part_im, m0 & 7, m0 >> 3));
                }
                *reinterpret_cast<uint4 *>(A + (size_t)ch * CS_A + (i_exp / 8) * 128 + (i_exp % 8) * 16) = v;
            }
        } else {
            for (int ch = hpar; ch < KC; ch += 2) {
                unsigned w4[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    unsigned h2 = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const short kt = sK[ch * 8 + 2 * t + h];
                        unsigned v = 0;
                        if (kt >= 0) {
                            const int e = kt & 0x3FFF, imag = (kt >> 14) & 1;
                            v = (cw[(i_exp - e) & (NXP - 1)] >> (16 * imag)) & 0xFFFFu;
                        }
                        h2 |= v << (16 * h);
                    }
                    w4[t] = h2;
                }
                *reinterpret_cast<uint4 *>(A + (size_t)ch * CS_A + (i_exp / 8) * 128 + (i_exp % 8) * 16) =
                    make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
    };
    auto issue_mma = [&](int b) {
        if (tid == 0) {
            const int bb = b & 1;
#pragma unroll
            for (int q = 0; q < NAP; ++q) {
                const unsigned dq = tmem + (unsigned)(bb * ACC_COLS + q * NG);
                for (int s = kqa[q] / 16; s < kqa[q + 1] / 16; ++s) {
                    const uint64_t da = umma_desc(smem_u32(sA[bb]) + s * 2 * CS_A, CS_A, 128);
                    const uint64_t db = umma_desc(smem_u32(sB[bb]) + s * 2 * CS_B, CS_B, 128);
                    umma(dq, da, db, idesc, s == kqa[q] / 16 ? 0u : 1u);
                }
            }
            umma_commit(&bar[2 + bb]);
            ++mmas_issued;
        }
    };
    auto wait_mma = [&](int b) -> bool {
        const bool r = mbar_wait(&bar[2 + (b & 1)], (b >> 1) & 1);
        if (r && tid == 0) ++mmas_done;
        return r;
    };
    auto fold = [&](int b) {
        const unsigned lane_base = tmem + ((unsigned)(32 * quarter) << 16) +
                                   (unsigned)((b & 1) * ACC_COLS + fhalf * 2 * FH);
#pragma unroll
        for (int fc = 0; fc < FH / 4; ++fc) {
            float r[NAP][8];
#pragma unroll
            for (int q = 0; q < NAP; ++q) tmem_ld8(lane_base + (unsigned)(q * NG + fc * 8), r[q]);
            tmem_wait_ld();
#pragma unroll
            for (int ff = 0; ff < 4; ++ff) {
                const int f = fc * 4 + ff;
                const float ar = r[0][2 * ff], ai = r[0][2 * ff + 1];
                const float br = r[1][2 * ff], bi = r[1][2 * ff + 1];
                acc[f][0] = fmaf(ar, ar, fmaf(ai, ai, acc[f][0]));
                acc[f][1] = fmaf(br, br, fmaf(bi, bi, acc[f][1]));
                if constexpr (NAP == 2) {
                    acc[f][2] = fmaf(ar, br, fmaf(ai, bi, acc[f][2]));
                } else {
                    const float cr = r[2][2 * ff], ci = r[2][2 * ff + 1];
                    acc[f][2] = fmaf(cr, cr, fmaf(ci, ci, acc[f][2]));
                    acc[f][3] = fmaf(ar, br, fmaf(ai, bi, acc[f][3]));
                    acc[f][4] = fmaf(br, cr, fmaf(bi, ci, acc[f][4]));
                    acc[f][5] = fmaf(cr, ar, fmaf(ci, ai, acc[f][5]));
                }
            }
        }
        tc_fence_before();  // ordered before the next MMA into this set by the next bin's barrier
    };

    bool ok = true;
    if (n_bins > 0) {
        issue_load(0);
        if (n_bins > 1) issue_load(1);
        bool r = wait_data(0);
        expand(0);
        ok = __syncthreads_and(r) != 0;
        tc_fence_after();
        if (ok) issue_mma(0);
    }
    for (int b = 0; b < n_bins && ok; ++b) {
        bool r = true;
        if (b + 1 < n_bins) {
            r = wait_data(b + 1);
            expand(b + 1);                     // tensor core: MMA(b)
        }
        r = wait_mma(b) && r;
        ok = __syncthreads_and(r) != 0;        // A(b+1) complete, acc(b) ready, buffers of bin b free
        tc_fence_after();
        if (!ok) break;
        if (b + 2 < n_bins) issue_load(b + 2);
        if (b + 1 < n_bins) issue_mma(b + 1);
        fold(b);                               // tensor core: MMA(b+1)
    }
    if (!ok && tid == 0) {
        atomicOr(status, 1);
        // let the copies / MMAs still in flight finish before shared and tensor memory go away
        for (int b = loads_done; b < loads_issued; ++b) mbar_wait(&bar[b & 1], (b >> 1) & 1);
        for (int b = mmas_done; b < mmas_issued; ++b) mbar_wait(&bar[2 + (b & 1)], (b >> 1) & 1);
    }
    const size_t npix = (size_t)nz * NXP;
#pragma unroll
    for (int f = 0; f < FH; ++f) {
        const int fr = grp * FG + fhalf * FH + f;
        if (fr < F && ok) {
            const float s2 = ldexpf(1.0f, 2 * frame_exp(smax[fr]));
#pragma unroll
            for (int a = 0; a < NACC; ++a)
                part[((size_t)fr * NACC + a) * npix + (size_t)j * NXP + i_epi] = acc[f][a] * s2;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS_PIPE)
                     : "memory");
}

size_t gemm_pipe_smem(int K)
{
    const size_t kc = (size_t)K / 8;
    return 2 * kc * CS_A + 2 * kc * CS_B + 2 * NXP * 4 + 2 * 2 * 8 * DS_LEN * 2 + ((K + 7) & ~7) * 2 + 4 * 8 + 16;
}
constexpr int kMaxPipeK = 256;

size_t gemm_smem(int K, bool split)
{
    const size_t kc = (size_t)K / 8;
    return kc * CS_A + kc * CS_B * (split ? 2 : 1) + 2 * NXP * 4 + ((K + 7) & ~7) * 2 + 32 + 2 * 8 * DS_LEN * 2;
}

template <int NAP, bool FP16, bool SPLIT>
cudaError_t launch_gemm_t(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    const int groups = (n_frames + FG - 1) / FG;
    dim3 grid(p.nz, groups);
    const int4 kq = make_int4(p.kq[0], p.kq[1], p.kq[2], p.kq[3]);
    if (!SPLIT && p.K <= kMaxPipeK) {
        prec_gemm_pipe_kernel<NAP, FP16><<<grid, GEMM_THREADS, gemm_pipe_smem(p.K), st>>>(
            p.t.c_hi, reinterpret_cast<const uint8_t *>(p.w.Bhi), p.t.ktab, p.K, kq, p.n_bins, p.nz, n_frames,
            p.w.smax, p.w.part, p.w.status, p.fast_expand);
        return cudaGetLastError();
    }
    prec_gemm_kernel<NAP, FP16, SPLIT><<<grid, GEMM_THREADS, gemm_smem(p.K, SPLIT), st>>>(
        p.t.c_hi, p.t.c_lo, reinterpret_cast<const uint8_t *>(p.w.Bhi), reinterpret_cast<const uint8_t *>(p.w.Blo),
        p.t.ktab, p.K, kq, p.n_bins, p.nz, n_frames, p.w.smax, p.w.part, p.w.status, p.fast_expand);
    return cudaGetLastError();
}

template <bool FP16, bool SPLIT>
cudaError_t launch_form(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p.w.smax, 0, sizeof(unsigned) * n_frames, st);
    if (e != cudaSuccess) return e;
    prec_smax_kernel<<<dim3(p.n_bins, n_frames), 128, 0, st>>>(p.w.S, p.n_bins, p.ne, p.w.smax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int groups = (n_frames + FG - 1) / FG;
    prec_bprep_kernel<FP16, SPLIT><<<dim3(p.n_bins, groups), 256, 0, st>>>(
        p.w.S, p.t.ktab, p.t.kwgt, p.K, p.n_bins, p.ne, n_frames, p.w.smax, reinterpret_cast<uint8_t *>(p.w.Bhi),
        reinterpret_cast<uint8_t *>(p.w.Blo));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return p.n_apod == 2 ? launch_gemm_t<2, FP16, SPLIT>(p, n_frames, st) : launch_gemm_t<3, FP16, SPLIT>(p, n_frames, st);
}

template <int NAP, bool FP16, bool SPLIT>
cudaError_t set_gemm_smem()
{
    return cudaFuncSetAttribute(prec_gemm_kernel<NAP, FP16, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_smem(kMaxGemmK, SPLIT));
}

}  // namespace

cudaError_t launch_prec_tables(const pam_plan_s &p, cudaStream_t st)
{
    dim3 grid(p.nz, p.n_bins);
    if (p.form == PAM_FORM_GEMM_FP16)
        prec_table_kernel<true><<<grid, NXP, 0, st>>>(p.t.phase, p.t.live, p.nz, p.d.z0_m, p.d.dz_m, p.t.c_hi, p.t.c_lo);
    else
        prec_table_kernel<false><<<grid, NXP, 0, st>>>(p.t.phase, p.t.live, p.nz, p.d.z0_m, p.d.dz_m, p.t.c_hi, p.t.c_lo);
    return cudaGetLastError();
}

cudaError_t launch_prec(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    switch (p.form) {
    case PAM_FORM_GEMM_BF16: return launch_form<false, false>(p, n_frames, st);
    case PAM_FORM_GEMM_FP16: return launch_form<true, false>(p, n_frames, st);
    case PAM_FORM_GEMM_BF16_SPLIT: return launch_form<false, true>(p, n_frames, st);
    default: return cudaErrorInvalidValue;
    }
}

int prec_kernels() { return 3; }

cudaError_t prepare_prec_kernels()
{
    cudaError_t e;
    const int pipe = (int)gemm_pipe_smem(kMaxPipeK);
    if ((e = cudaFuncSetAttribute(prec_gemm_pipe_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe)))
        return e;
    if ((e = cudaFuncSetAttribute(prec_gemm_pipe_kernel<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe)))
        return e;
    if ((e = cudaFuncSetAttribute(prec_gemm_pipe_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe)))
        return e;
    if ((e = cudaFuncSetAttribute(prec_gemm_pipe_kernel<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe)))
        return e;
    if ((e = set_gemm_smem<2, false, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, false, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<2, true, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, true, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<2, false, true>()) != cudaSuccess) return e;
    return set_gemm_smem<3, false, true>();
}

}  // namespace pam
