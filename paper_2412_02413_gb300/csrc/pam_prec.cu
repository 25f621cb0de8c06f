// pam_prec.cu -- tensor-core form of the propagate-and-correlate step
// (PAM_FORM_GEMM_*).
//
// For bin w_k and depth row z_j, Eq. 1-2 map the apodized channel spectra to
// the row's fields through a circulant matrix:
//   p~_q(x_i, z_j) = sum_e c_j[(i - e) mod nx] a_q[e] S[e],
//   c_j[d] = (1/nx) sum_u exp(i kz_u z_j) exp(+2 pi i u d / nx),
// i.e. the inverse lateral DFT of the row's propagator phasors. The plan
// tabulates c_j once per (bin, row) from the exact FP64 phase words, in
// 16-bit form. A call then evaluates the sum over elements for FG = 32 (or 16)
// frames at a time as one tcgen05 GEMM per (bin, row) with M = 128 pixels,
// N = 2 x FG (Re, Im of each frame) and K = 16 per element block of 8:
//   A[i][k] = Re or Im c_j[(i - e_k) mod nx]   (8 x 8 Toeplitz blocks in shared memory)
//   B[k][n] = +-Re or Im of a S / sigma          (packed per call)
// so that the real GEMM yields Re and Im of the complex sum. Each aperture is
// its own K range (the element blocks it touches; elements outside it carry
// weight 0): one MMA chain per aperture accumulates into its own
// tensor-memory region. The fold reads the accumulators with tcgen05.ld and
// adds |p_q|^2 and Re conj(p_q) p_r into per-pixel registers across all bins
// (Eq. 3-4). The NCC/TAX epilogue kernels then finish exactly as in the FP32
// path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"
#include "pam_ptx.h"

namespace pam {
namespace {

using namespace ptx;

constexpr int NXP = 128;                    // lateral length of this form
// Frames per CTA (FG, 32 or 16; kFramesPerGroup sizes the workspace for the
// larger) and what follows from it: the GEMM's N = 2 FG columns (Re and Im of
// each frame) and the bytes between K chunks of the B tile.
template <int FG> struct Grp {
    static_assert(FG == 16 || FG == 32, "frames per CTA");
    static constexpr int NG = 2 * FG;
    static constexpr int CS_B = NG / 8 * 128;
    static constexpr int FW = FG / 2;        // frames per fold warp
};

__host__ __device__ __forceinline__ int K_of(int4 kq) { return kq.w; }

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
// max |Re S|, |Im S| of each frame (bits of a non-negative float). A frame's
// n_vals = n_bins x ne values are contiguous; the blocks of grid row f read
// them as float4 pairs in a grid-stride loop and fold one maximum each into
// smax[f] (the maximum does not depend on the order).
constexpr int SMAX_THREADS = 256;
__global__ void __launch_bounds__(SMAX_THREADS)
prec_smax_kernel(const float2 *__restrict__ S, int n_vals, unsigned *__restrict__ smax)
{
    __shared__ float wm[SMAX_THREADS / 32];
    const int f = blockIdx.y;
    const float4 *src = reinterpret_cast<const float4 *>(S + (size_t)f * n_vals);
    const int n4 = n_vals / 2;   // n_vals is even (ne is a multiple of 8)
    float m = 0.f;
    for (int i = blockIdx.x * SMAX_THREADS + threadIdx.x; i < n4; i += gridDim.x * SMAX_THREADS) {
        const float4 v = src[i];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < SMAX_THREADS / 32; ++w) m = fmaxf(m, wm[w]);
        atomicMax(&smax[f], __float_as_uint(m));
    }
}
// Blocks per frame of prec_smax_kernel: about 1024 float4 each, at most 32.
int smax_blocks(int n_vals)
{
    const int n = (n_vals / 2 + 4 * SMAX_THREADS - 1) / (4 * SMAX_THREADS);
    return n < 1 ? 1 : (n > 32 ? 32 : n);
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
// PAIR: the tile is stored as its two halves of N / 2 columns (the Re
// columns, then the Im columns), each in the same canonical layout, so that
// each CTA of a pair copies its half with one bulk copy.
template <bool FP16, bool SPLIT, bool PAIR, int FG>
__global__ void __launch_bounds__(256)
prec_bprep_kernel(const float2 *__restrict__ S, const short *__restrict__ ktab, const float *__restrict__ kwgt,
                  int K, int n_bins, int ne, int F, const unsigned *__restrict__ smax, uint8_t *__restrict__ Bhi,
                  uint8_t *__restrict__ Blo)
{
    constexpr int NG = Grp<FG>::NG, CS_B = Grp<FG>::CS_B;
    const int b = blockIdx.x, g = blockIdx.y;
    const size_t tile = (size_t)K * NG * 2;
    uint8_t *dh = Bhi + ((size_t)g * n_bins + b) * tile;
    uint8_t *dl = SPLIT ? Blo + ((size_t)g * n_bins + b) * tile : nullptr;
    // Thread (kc, n) writes the 8 entries k = 8 kc .. 8 kc + 7 of column n: one
    // 16-byte row of a core matrix (consecutive n, consecutive rows).
    for (int idx = threadIdx.x; idx < (K / 8) * NG; idx += blockDim.x) {
        const int kc = idx / NG, n = idx % NG;
        const int f = g * FG + n % FG, kind = n / FG;   // columns: Re of the FG frames, then Im
        const bool live = f < F;
        const float p2 = live ? ldexpf(1.0f, -frame_exp(smax[f])) : 0.f;
        const float2 *Sf = S + ((size_t)(live ? f : 0) * n_bins + b) * ne;
        unsigned h[4], l[4];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            unsigned short hh[2], ll[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int k = 8 * kc + t + u;
                float v = 0.f;
                const short kt = ktab[k];
                if (live && kt >= 0) {
                    const int e = kt & 0x3FFF, imag = (kt >> 14) & 1;
                    const float sc = kwgt[k] * p2;
                    const float2 s = Sf[e];
                    const float sr = s.x * sc, si = s.y * sc;
                    v = imag == 0 ? (kind == 0 ? sr : si) : (kind == 0 ? -si : sr);
                }
                hh[u] = to16<FP16>(v);
                ll[u] = SPLIT ? to16<FP16>(v - from16<FP16>(hh[u])) : (unsigned short)0;
            }
            h[t / 2] = (unsigned)hh[0] | ((unsigned)hh[1] << 16);
            l[t / 2] = (unsigned)ll[0] | ((unsigned)ll[1] << 16);
        }
        size_t off;
        if constexpr (PAIR) {
            const int half = n / FG, nn = n % FG;
            off = (size_t)half * K * FG * 2 + (size_t)kc * (CS_B / 2) + (nn / 8) * 128 + (nn % 8) * 16;
        } else {
            off = (size_t)kc * CS_B + (n / 8) * 128 + (n % 8) * 16;
        }
        *reinterpret_cast<uint4 *>(dh + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (SPLIT) *reinterpret_cast<uint4 *>(dl + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// ------------------------------------------------------------- GEMM ----
// The A operand (the circulant) needs no expansion. Write pixel i = 8g + r
// and element e = 8m + t with g, m < 16 blocks of 8. The entry
// c[(i - e) mod 128] = c[(8 (g - m) + r - t) mod 128] depends on the two
// blocks only through d = (g - m) mod 16, so the 128 x 128 matrix is built
// from 16 distinct 8 x 8 Toeplitz blocks T_d[r][t] = c[(8 d + r - t) mod 128].
// Each is exactly one 8-row x 16-byte core matrix of the canonical K-major
// layout. Shared memory holds T_(n mod 16) for n = 0..31 (Re parts, then Im
// parts, BLK_BYTES apart); the MMA of element block m starts at n = 16 - m, so
// that row group g (SBO = 128 bytes) reads n = 16 - m + g, i.e. T_(g - m).
// One K step of 16 is one element block: 8 columns pairing with Re c, then 8
// pairing with Im c (LBO = BLK_BYTES).
//
// One CTA per (depth row j, group of FG frames); warp-specialised, with no
// CTA-wide barrier inside the bin loop:
//   warp 0: bulk copies of each bin's B tile and c words into a ring of NST
//     stages;
//   warps 1 .. NAP: the MMA chain of aperture q = warp - 1 into one of two
//     tensor-memory accumulator sets. One issuing warp per aperture: a single
//     thread issuing every chain cannot keep up with N = 64 MMAs, which the
//     tensor core finishes in about 48 cycles each;
//   warps 4-11: build the Toeplitz blocks of bin b+1, then fold the
//     accumulators of bin b into per-pixel sums. Warp w reads tensor-memory
//     lane quarter w % 4 (pixels 32 (w%4) .. +31) for frames FG/2 ((w-4)/4) .. +FG/2-1.
// The issuing warps have the lowest warp numbers: while the build/fold warps
// issue FMAs back to back, the schedulers favour them, and MMA issue is on
// the critical path.
// mbarriers: full[s] (copy landed), sfree[s] (MMAs of the stage done; NAP
// commits), afull[t] (accumulator set t written; NAP commits), go[t] (16
// warp arrivals: the 8 build warps for bin b, once its blocks are written,
// and the 8 fold warps for bin b - 2, once set t is read out). Every wait
// is bounded; on expiry the CTA raises a shared abort flag and the device
// status word, each role drains the copies or MMAs it issued, and the CTA exits.
constexpr int BLK_BYTES = 32 * 128;       // 32 core matrices of one part (Re or Im)
constexpr int A_BYTES = 2 * BLK_BYTES;    // Re and Im
constexpr int MAX_NST = 4;
constexpr size_t GEMM_SMEM_LIMIT = 232448;  // opt-in shared memory per CTA
constexpr size_t GEMM_SMEM_EXTRA = 24 * 8 + 16;
template <int NAP>
constexpr int gemm_threads() { return 384; }   // 8 build/fold warps, 1 copy warp, NAP MMA warps (+ idle)
constexpr int REG_LAUNCH = 168, REG_CTRL = 96, REG_FOLD = 200;
static_assert(2 * 128 * REG_FOLD + 128 * REG_CTRL <= 384 * REG_LAUNCH, "register split exceeds the launch budget");

// Shared memory of one pipeline stage: NPART x (A blocks, B tile, c words);
// a CTA of a pair holds half of the B tile.
__host__ __device__ constexpr size_t gemm_stage_bytes(int K, int npart, bool pair, int fg)
{
    return (size_t)npart * (A_BYTES + (size_t)K * (pair ? fg : 2 * fg) * 2 + NXP * 4);
}
int gemm_stages(int K, bool split, bool pair, int fg)
{
    const size_t st = gemm_stage_bytes(K, split ? 2 : 1, pair, fg);
    const size_t n = (GEMM_SMEM_LIMIT - GEMM_SMEM_EXTRA) / st;
    return (int)(n < MAX_NST ? n : MAX_NST);
}
size_t gemm_smem(int K, bool split, bool pair, int fg)
{
    return gemm_stages(K, split, pair, fg) * gemm_stage_bytes(K, split ? 2 : 1, pair, fg) + GEMM_SMEM_EXTRA;
}

// steps: element block of K step st in bits 4 (st % 16) of steps[st / 16].
// BANDS: instead of the per-aperture sums, fold the full-aperture energy
// |p_1 + p_2 + p_3|^2 (Eq. 3 with apodizations that sum to one) and write it
// out per band of bins: band k = bins [n_bins k / n_bands, n_bins (k+1) / n_bands),
// to part[frame][k][nz][nx].
// PAIR: the CTAs of a 2-CTA cluster take depth rows j (even rank 0) and j + 1
// of the same frame group. Each builds its own row's A blocks and copies half
// of the B tile (rank 0 the Re columns, rank 1 the Im columns); rank 0's MMA
// warps issue cta_group::2 MMAs with M = 256 that write each CTA's own tensor
// memory. Both CTAs' build and fold warps arrive on rank 0's go barriers; the
// MMA commits arrive on the stage and accumulator barriers of both CTAs. Each
// SM thus stages and reads half of B.
template <int NAP, bool FP16, bool SPLIT, bool BANDS = false, bool PAIR = false, int FG = 32>
__global__ void __launch_bounds__(gemm_threads<NAP>(), 1)
prec_gemm_kernel(const uint32_t *__restrict__ chi, const uint32_t *__restrict__ clo, const uint8_t *__restrict__ Bhi,
                 const uint8_t *__restrict__ Blo, ulonglong2 steps, int4 kq, int n_bins, int nz, int F, int NST,
                 const unsigned *__restrict__ smax, float *__restrict__ part, int *__restrict__ status, int n_bands)
{
    static_assert(!BANDS || NAP == 3, "band energies fold three apertures");
    static_assert(!(BANDS && PAIR), "the band form runs unpaired");
    constexpr int NACC = BANDS ? 1 : (NAP == 2 ? 3 : 6);
    constexpr int NPART = SPLIT ? 2 : 1;
    constexpr int NG = Grp<FG>::NG, FW = Grp<FG>::FW;
    constexpr int ACC_COLS = NAP * NG;
    constexpr int NGC = PAIR ? NG / 2 : NG;      // B columns in this CTA's shared memory
    constexpr int CS_BC = NGC / 8 * 128;         // bytes between K chunks of this CTA's B
    constexpr unsigned TMEM_ALLOC = 2 * ACC_COLS <= 256 ? 256u : 512u;
    static_assert(2 * ACC_COLS <= 512, "two accumulator sets must fit in tensor memory");
    extern __shared__ __align__(1024) uint8_t sm[];
    const size_t bytesB = (size_t)K_of(kq) * NGC * 2;   // this CTA's part of one B tile
    const size_t stage = gemm_stage_bytes(K_of(kq), NPART, PAIR, FG);
    auto sA = [&](int s) { return sm + s * stage; };
    auto sB = [&](int s) { return sm + s * stage + NPART * A_BYTES; };
    auto sC = [&](int s) { return reinterpret_cast<uint32_t *>(sm + s * stage + NPART * (A_BYTES + bytesB)); };
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + NST * stage);    // [MAX_NST]
    uint64_t *sfree = full + MAX_NST;                                   // [MAX_NST]
    uint64_t *go = sfree + MAX_NST, *afull = go + 2;                    // [2], [2]
    uint64_t *dbar = afull + 2;                                         // [4] per-warp drain
    unsigned *tslot = reinterpret_cast<unsigned *>(dbar + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = blockIdx.x, grp = blockIdx.y;
    const unsigned rank = PAIR ? cluster_ctarank() : 0u;
    const bool row_ok = j < nz;               // a pair's second row may lie past the grid
    const int jl = row_ok ? j : nz - 1;       // row whose c words are loaded
    if (warp == 0) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                         "r"(TMEM_ALLOC)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                         "r"(TMEM_ALLOC)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
        }
    }
    if (tid == 0) {
        for (int s = 0; s < MAX_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&sfree[s], NAP);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(&go[t], PAIR ? 32 : 16);
            mbar_init(&afull[t], NAP);
        }
        for (int q = 0; q < 4; ++q) mbar_init(&dbar[q], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all();   // the peer's barriers exist before any remote arrival
    else __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    // arrival on go[t] of the pair's rank-0 CTA (or this CTA's when unpaired)
    auto go_arrive = [&](int t) {
        if constexpr (PAIR) mbar_arrive_cluster(mapa_rank(smem_u32(&go[t]), 0u));
        else mbar_arrive(&go[t]);
    };
    // Register split between the warpgroups (launch: 384 x 168 = 64512): the
    // copy / MMA warpgroup (warps 0-3) drops to REG_CTRL, the two build/fold warpgroups rise
    // to REG_FOLD (2 x 128 x REG_FOLD + 128 x REG_CTRL <= 64512). The host checks
    // that the kernel was built with 168 registers per thread before launching.
    // The band form keeps one sum per pixel and frame, and 16 frames per CTA
    // half the fold's sums: neither needs the split.
    if constexpr (!BANDS && FG == 32) {
        if (warp < 4)
            asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(REG_CTRL));
        else
            asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(REG_FOLD));
    }

    // Bounded wait that also gives up when another thread has aborted.
    auto try1 = [&](uint64_t *bar, unsigned parity) -> bool {
        if constexpr (PAIR) return mbar_try_wait_cluster(bar, parity);
        else return mbar_try_wait(bar, parity);
    };
    auto try2 = [&](uint64_t *bar, unsigned parity) -> bool {
        if constexpr (PAIR) return mbar_try_wait_cluster(bar, parity);
        else return mbar_try_wait_sleep(bar, parity);
    };
    auto wait = [&](uint64_t *bar, unsigned parity) -> bool {
        if (try1(bar, parity)) return true;
        const long long t0 = clock64();
        while (!try2(bar, parity)) {
            if (*abort_flag) return false;
            if (clock64() - t0 > (1ll << 31)) {
                *abort_flag = 1;
                atomicOr(status, 1);
                return false;
            }
        }
        return true;
    };

    if (warp >= 1 + NAP && warp < 4) {
        // spare warp of the control warpgroup (AS-DAX): nothing to do
    } else if (warp < 4) {
        // -------- warp 0: bulk-copy ring; warps 1..NAP: MMA chain of aperture q --------
        const int q = warp - 1;
        const bool producer = q < 0;
        const unsigned idesc = umma_idesc(FP16, PAIR ? 2 * NXP : NXP, NG);
        const int s0 = (q <= 0 ? kq.x : q == 1 ? kq.y : kq.z) / 16;
        const int s1 = (q <= 0 ? kq.y : q == 1 ? kq.z : kq.w) / 16;
        int issued = 0;
        auto load = [&](int b) {
            if (lane == 0) {
                const int s = b % NST;
                const size_t ob = ((size_t)grp * n_bins + b) * (PAIR ? 2 : 1) * bytesB + rank * bytesB;
                const size_t oc = ((size_t)b * nz + jl) * NXP;
                mbar_expect_tx(&full[s], (unsigned)(NPART * (bytesB + NXP * 4)));
                bulk_g2s(sB(s), Bhi + ob, (unsigned)bytesB, &full[s]);
                bulk_g2s(sC(s), chi + oc, NXP * 4, &full[s]);
                if (SPLIT) {
                    bulk_g2s(sB(s) + bytesB, Blo + ob, (unsigned)bytesB, &full[s]);
                    bulk_g2s(sC(s) + NXP, clo + oc, NXP * 4, &full[s]);
                }
            }
            __syncwarp();
            issued = b + 1;
        };
        if (producer)
            for (int b = 0; b < n_bins && b < NST; ++b) load(b);
        bool ok = true, any = false;
        if (producer) {
            for (int b = NST; b < n_bins && ok; ++b) {
                // stage of bin b - NST is free once every aperture's MMAs of that bin are done
                ok = __all_sync(0xffffffffu, wait(&sfree[b % NST], (unsigned)(b / NST - 1) & 1u));
                if (ok) load(b);
            }
        } else if (!PAIR || rank == 0) {   // a pair's MMAs are issued by its rank-0 CTA
            for (int b = 0; b < n_bins && ok; ++b) {
                const int s = b % NST, t = b & 1;
                // go[t]: the blocks of bin b are built (which the build warps did after
                // its copy landed) and accumulator set t was read out for bin b - 2
                ok = __all_sync(0xffffffffu, wait(&go[t], (unsigned)(b >> 1) & 1u));
                if (!ok) break;
                tc_fence_after();
                const uint64_t da0 = umma_desc(smem_u32(sA(s)), BLK_BYTES, 128);
                const uint64_t db0 = umma_desc(smem_u32(sB(s)), CS_BC, 128);
                const unsigned dq = tmem + (unsigned)(t * ACC_COLS + q * NG);
                auto mma = [&](uint64_t a, uint64_t bd, unsigned acc) {
                    if constexpr (PAIR) umma_elect_pair(dq, a, bd, idesc, acc);
                    else umma_elect(dq, a, bd, idesc, acc);
                };
                for (int st = s0; st < s1; ++st) {
                    const unsigned m = (unsigned)((st < 16 ? steps.x >> (4 * st) : steps.y >> (4 * (st - 16))) & 15u);
                    const uint64_t da = da0 + (uint64_t)((16u - m) * 8u);   // start address field: +128 B per block
                    const uint64_t db = db0 + (uint64_t)(st * (2 * CS_BC / 16));
                    mma(da, db, st == s0 ? 0u : 1u);
                    if (SPLIT) {
                        mma(da, db + (uint64_t)(bytesB / 16), 1u);             // hi x lo
                        mma(da + (uint64_t)(A_BYTES / 16), db, 1u);           // lo x hi
                    }
                }
                any = true;
                if constexpr (PAIR) {
                    umma_commit_pair_elect(&sfree[s], (unsigned short)3);
                    umma_commit_pair_elect(&afull[t], (unsigned short)3);
                } else {
                    umma_commit_elect(&sfree[s]);
                    umma_commit_elect(&afull[t]);
                }
            }
        }
        if constexpr (PAIR) {
            // tracks every pair MMA this warp issued (rank 0's own dbar)
            if (!ok && any && !producer) umma_commit_pair_elect(&dbar[q], (unsigned short)1);
        }
        if (!ok && lane == 0) {
            if (any) {
                if constexpr (!PAIR) umma_commit(&dbar[q]);   // tracks every MMA this thread issued
                mbar_wait(&dbar[q], 0);
            }
            // at most one copy per stage can still be in flight: the last one issued there
            for (int b = issued - NST < 0 ? 0 : issued - NST; b < issued; ++b)
                mbar_wait(&full[b % NST], (unsigned)(b / NST) & 1u);
        }
    } else {
        // ---------------- build + fold (warps 4-11) ----------------
        const int quarter = warp & 3, fh = (warp - 4) >> 2, ctid = tid - 128;
        const int i_epi = 32 * quarter + lane;
        // Sums of frame pairs (2p, 2p+1) as float2, so that one packed FMA
        // (fma.rn.f32x2) serves two frames.
        float2 acc[FW / 2][NACC];
#pragma unroll
        for (int f = 0; f < FW / 2; ++f)
#pragma unroll
            for (int a = 0; a < NACC; ++a) acc[f][a] = make_float2(0.f, 0.f);

        // Row r of block n holds the 8 entries c[(8 (n mod 16) + r - t) mod 128],
        // t = 0..7, as one 16-byte row of Re parts and one of Im parts; blocks n
        // and n + 16 are the same. With the split, thread (part, d, r) computes
        // row r of T_d of its part once and stores it in both blocks (half the
        // loads per thread of building the two parts in turn: 4% faster); with
        // one part, thread (n, r) builds row r of block n (computing once and
        // storing twice was 1.4% slower there).
        auto build = [&](int b) -> bool {
            const int s = b % NST;
            if (!wait(&full[s], (unsigned)(b / NST) & 1u)) return false;
            if constexpr (SPLIT) {
                const int pidx = ctid >> 7, d = (ctid >> 3) & 15, r = ctid & 7;
                const uint32_t *cw = sC(s) + pidx * NXP;
                const int m0 = 8 * d + r;
                unsigned w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) w[t] = cw[(m0 - t) & (NXP - 1)];
                uint8_t *A = sA(s) + pidx * A_BYTES + d * 128 + r * 16;
                const uint4 re = make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                                            __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                const uint4 im = make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                                            __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
                *reinterpret_cast<uint4 *>(A) = re;
                *reinterpret_cast<uint4 *>(A + 16 * 128) = re;
                *reinterpret_cast<uint4 *>(A + BLK_BYTES) = im;
                *reinterpret_cast<uint4 *>(A + BLK_BYTES + 16 * 128) = im;
            } else {
                const int n = ctid >> 3, r = ctid & 7;
                const uint32_t *cw = sC(s);
                const int m0 = 8 * (n & 15) + r;
                unsigned w[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) w[t] = cw[(m0 - t) & (NXP - 1)];
                uint8_t *A = sA(s) + n * 128 + r * 16;
                *reinterpret_cast<uint4 *>(A) =
                    make_uint4(__byte_perm(w[0], w[1], 0x5410), __byte_perm(w[2], w[3], 0x5410),
                               __byte_perm(w[4], w[5], 0x5410), __byte_perm(w[6], w[7], 0x5410));
                *reinterpret_cast<uint4 *>(A + BLK_BYTES) =
                    make_uint4(__byte_perm(w[0], w[1], 0x7632), __byte_perm(w[2], w[3], 0x7632),
                               __byte_perm(w[4], w[5], 0x7632), __byte_perm(w[6], w[7], 0x7632));
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) go_arrive(b & 1);
            return true;
        };
        auto fold = [&](int b) -> bool {
            const int t = b & 1;
            if (!wait(&afull[t], (unsigned)(b >> 1) & 1u)) return false;
            tc_fence_after();
            // columns of aperture q: Re of frames 0..FG-1, then Im of frames 0..FG-1
            const unsigned base = tmem + ((unsigned)(32 * quarter) << 16) + (unsigned)(t * ACC_COLS + fh * FW);
            // four frames at a time, so that the loaded values take 24 registers
#pragma unroll
            for (int h = 0; h < FW / 4; ++h) {
                float re[NAP][4], im[NAP][4];
#pragma unroll
                for (int q = 0; q < NAP; ++q) {
                    tmem_ld4(base + (unsigned)(q * NG + 4 * h), re[q]);
                    tmem_ld4(base + (unsigned)(q * NG + FG + 4 * h), im[q]);
                }
                tmem_wait_ld();
                if (h == FW / 4 - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) go_arrive(t);   // set t is free for bin b + 2
                }
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    float2 *A = acc[2 * h + pp];
                    const float2 ar = make_float2(re[0][2 * pp], re[0][2 * pp + 1]);
                    const float2 ai = make_float2(im[0][2 * pp], im[0][2 * pp + 1]);
                    const float2 br = make_float2(re[1][2 * pp], re[1][2 * pp + 1]);
                    const float2 bi = make_float2(im[1][2 * pp], im[1][2 * pp + 1]);
                    if constexpr (BANDS) {
                        const float2 cr = make_float2(re[2][2 * pp], re[2][2 * pp + 1]);
                        const float2 ci = make_float2(im[2][2 * pp], im[2][2 * pp + 1]);
                        const float2 sr = make_float2(ar.x + br.x + cr.x, ar.y + br.y + cr.y);
                        const float2 si = make_float2(ai.x + bi.x + ci.x, ai.y + bi.y + ci.y);
                        A[0] = __ffma2_rn(sr, sr, __ffma2_rn(si, si, A[0]));
                    } else {
                        A[0] = __ffma2_rn(ar, ar, __ffma2_rn(ai, ai, A[0]));
                        A[1] = __ffma2_rn(br, br, __ffma2_rn(bi, bi, A[1]));
                        if constexpr (NAP == 2) {
                            A[2] = __ffma2_rn(ar, br, __ffma2_rn(ai, bi, A[2]));
                        } else {
                            const float2 cr = make_float2(re[2][2 * pp], re[2][2 * pp + 1]);
                            const float2 ci = make_float2(im[2][2 * pp], im[2][2 * pp + 1]);
                            A[2] = __ffma2_rn(cr, cr, __ffma2_rn(ci, ci, A[2]));
                            A[3] = __ffma2_rn(ar, br, __ffma2_rn(ai, bi, A[3]));
                            A[4] = __ffma2_rn(br, cr, __ffma2_rn(bi, ci, A[4]));
                            A[5] = __ffma2_rn(cr, ar, __ffma2_rn(ci, ai, A[5]));
                        }
                    }
                }
            }
            return true;
        };

        if (lane == 0) {   // accumulator sets 0 and 1 start free (bins -2 and -1)
            go_arrive(0);
            go_arrive(1);
        }
        // Blocks are built two bins ahead, so that MMA(b+1) only waits for the
        // fold of bin b-1 to release its accumulator set. Building bin b+2 reuses
        // the stage of bin b+2-NST (NST >= 2), whose MMAs are done once fold(b)
        // has seen bin b's accumulators.
        const size_t npix = (size_t)nz * NXP;
        int band = 0;
        // write the band sums of this warp's frames and restart them
        auto flush = [&]() {
#pragma unroll
            for (int f = 0; f < FW; ++f) {
                const int fr = grp * FG + fh * FW + f;
                if (fr < F) {
                    const float s2 = ldexpf(1.0f, 2 * frame_exp(smax[fr]));
                    const float v = (f & 1) ? acc[f >> 1][0].y : acc[f >> 1][0].x;
                    part[((size_t)fr * n_bands + band) * npix + (size_t)j * NXP + i_epi] = v * s2;
                }
            }
#pragma unroll
            for (int f = 0; f < FW / 2; ++f) acc[f][0] = make_float2(0.f, 0.f);
        };
        bool ok = n_bins == 0 || build(0);
        if (ok && n_bins > 1) ok = build(1);
        for (int b = 0; b < n_bins && ok; ++b) {
            if (!fold(b)) ok = false;                            // tensor core: MMA(b+1)
            if (ok && b + 2 < n_bins && !build(b + 2)) ok = false;
            if constexpr (BANDS) {
                if (ok && b + 1 == (int)(((long long)n_bins * (band + 1)) / n_bands)) {
                    flush();
                    ++band;
                }
            }
        }
#pragma unroll
        for (int f = 0; f < (BANDS ? 0 : FW); ++f) {
            const int fr = grp * FG + fh * FW + f;
            if (fr < F && ok && row_ok) {
                const float s2 = ldexpf(1.0f, 2 * frame_exp(smax[fr]));
#pragma unroll
                for (int a = 0; a < NACC; ++a) {
                    const float v = (f & 1) ? acc[f >> 1][a].y : acc[f >> 1][a].x;
                    part[((size_t)fr * NACC + a) * npix + (size_t)j * NXP + i_epi] = v * s2;
                }
            }
        }
    }
    tc_fence_before();
    if constexpr (PAIR) cluster_sync_all();   // the peer's MMAs, copies and arrivals are done
    else __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_ALLOC)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_ALLOC)
                         : "memory");
    }
}

// The element block of every K step of 16 (4 bits per step, steps 0-15 in x and
// 16-31 in y): the MMA of a step starts its A descriptor at block 16 - m.
ulonglong2 gemm_steps(const pam_plan_s &p)
{
    ulonglong2 steps = make_ulonglong2(0ull, 0ull);
    for (int s = 0; s < p.K / 16; ++s) {
        const unsigned long long m = (unsigned long long)((p.ktab_h[(size_t)16 * s] & 0x3FFF) >> 3) & 15ull;
        if (s < 16) steps.x |= m << (4 * s);
        else steps.y |= m << (4 * (s - 16));
    }
    return steps;
}

template <int NAP, bool FP16, bool SPLIT, bool PAIR, int FG>
cudaError_t launch_gemm_t(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    const int groups = (n_frames + FG - 1) / FG;
    const int4 kq = make_int4(p.kq[0], p.kq[1], p.kq[2], p.kq[3]);
    const int nst = gemm_stages(p.K, SPLIT, PAIR, FG);
    if (nst < 2 || p.K / 16 > 32) return cudaErrorInvalidConfiguration;
    const ulonglong2 steps = gemm_steps(p);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(PAIR ? (p.nz + 1) & ~1 : p.nz, groups);   // pairs of rows: an even grid
    cfg.blockDim = dim3(gemm_threads<NAP>());
    cfg.dynamicSmemBytes = gemm_smem(p.K, SPLIT, PAIR, FG);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (PAIR) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, prec_gemm_kernel<NAP, FP16, SPLIT, false, PAIR, FG>, p.t.c_hi, p.t.c_lo,
                                       reinterpret_cast<const uint8_t *>(p.w.Bhi),
                                       reinterpret_cast<const uint8_t *>(p.w.Blo), steps, kq, p.n_bins, p.nz, n_frames,
                                       nst, p.w.smax, p.w.part, p.w.status, 0);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Per-band full-aperture energies of BF16 or FP16 form (no split): operand
// packing from the spectra S [F][n_bins][n_elem] and the BANDS GEMM.
template <bool FP16>
cudaError_t launch_bands_form(const pam_plan_s &p, const float2 *S, int n_frames, int n_bands, float *bands,
                              cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p.w.smax, 0, sizeof(unsigned) * n_frames, st);
    if (e != cudaSuccess) return e;
    prec_smax_kernel<<<dim3(smax_blocks(p.n_bins * p.ne), n_frames), SMAX_THREADS, 0, st>>>(S, p.n_bins * p.ne,
                                                                                           p.w.smax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    constexpr int FG = 32;
    const int groups = (n_frames + FG - 1) / FG;
    prec_bprep_kernel<FP16, false, false, FG><<<dim3(p.n_bins, groups), 256, 0, st>>>(
        S, p.t.ktab, p.t.kwgt, p.K, p.n_bins, p.ne, n_frames, p.w.smax, reinterpret_cast<uint8_t *>(p.w.Bhi),
        nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (gemm_stages(p.K, false, false, FG) < 2 || p.K / 16 > 32) return cudaErrorInvalidConfiguration;
    const int4 kq = make_int4(p.kq[0], p.kq[1], p.kq[2], p.kq[3]);
    const ulonglong2 steps = gemm_steps(p);
    prec_gemm_kernel<3, FP16, false, true><<<dim3(p.nz, groups), gemm_threads<3>(), gemm_smem(p.K, false, false, FG), st>>>(
        p.t.c_hi, nullptr, reinterpret_cast<const uint8_t *>(p.w.Bhi), nullptr, steps, kq, p.n_bins, p.nz, n_frames,
        gemm_stages(p.K, false, false, FG), p.w.smax, bands, p.w.status, n_bands);
    return cudaGetLastError();
}

template <bool FP16, bool SPLIT, bool PAIR, int FG>
cudaError_t launch_form_t(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    const int groups = (n_frames + FG - 1) / FG;
    prec_bprep_kernel<FP16, SPLIT, PAIR, FG><<<dim3(p.n_bins, groups), 256, 0, st>>>(
        p.w.S, p.t.ktab, p.t.kwgt, p.K, p.n_bins, p.ne, n_frames, p.w.smax, reinterpret_cast<uint8_t *>(p.w.Bhi),
        reinterpret_cast<uint8_t *>(p.w.Blo));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return p.n_apod == 2 ? launch_gemm_t<2, FP16, SPLIT, PAIR, FG>(p, n_frames, st)
                         : launch_gemm_t<3, FP16, SPLIT, PAIR, FG>(p, n_frames, st);
}

template <bool FP16, bool SPLIT>
cudaError_t launch_form(const pam_plan_s &p, int n_frames, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(p.w.smax, 0, sizeof(unsigned) * n_frames, st);
    if (e != cudaSuccess) return e;
    prec_smax_kernel<<<dim3(smax_blocks(p.n_bins * p.ne), n_frames), SMAX_THREADS, 0, st>>>(p.w.S, p.n_bins * p.ne,
                                                                                           p.w.smax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool pair = p.gemm_m == 256, f16 = p.gemm_frames == 16;
    if (pair)
        return f16 ? launch_form_t<FP16, SPLIT, true, 16>(p, n_frames, st)
                   : launch_form_t<FP16, SPLIT, true, 32>(p, n_frames, st);
    return f16 ? launch_form_t<FP16, SPLIT, false, 16>(p, n_frames, st)
               : launch_form_t<FP16, SPLIT, false, 32>(p, n_frames, st);
}

template <int NAP, bool FP16, bool SPLIT, bool BANDS = false, bool PAIR = false, int FG = 32>
cudaError_t set_gemm_smem_one()
{
    static_assert(MAX_NST >= 2, "the copy ring needs two stages");
    cudaError_t e = cudaFuncSetAttribute(prec_gemm_kernel<NAP, FP16, SPLIT, BANDS, PAIR, FG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM_LIMIT);
    if (e != cudaSuccess || BANDS || FG != 32) return e;
    // The register split (setmaxnreg) is sized for a launch of exactly REG_LAUNCH
    // registers per thread; with fewer, the increase could never be granted.
    cudaFuncAttributes a;
    if ((e = cudaFuncGetAttributes(&a, prec_gemm_kernel<NAP, FP16, SPLIT, BANDS, PAIR, FG>)) != cudaSuccess) return e;
    return a.numRegs == REG_LAUNCH ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int NAP, bool FP16, bool SPLIT, bool BANDS = false>
cudaError_t set_gemm_smem()
{
    cudaError_t e = set_gemm_smem_one<NAP, FP16, SPLIT, BANDS, false>();
    if (e != cudaSuccess || BANDS) return e;
    if ((e = set_gemm_smem_one<NAP, FP16, SPLIT, false, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem_one<NAP, FP16, SPLIT, false, false, 16>()) != cudaSuccess) return e;
    return set_gemm_smem_one<NAP, FP16, SPLIT, false, true, 16>();
}

}  // namespace

cudaError_t launch_prec_tables(const pam_plan_s &p, cudaStream_t st)
{
    dim3 grid(p.nz, p.n_bins);
    if (p.form == PAM_FORM_GEMM_FP16 || p.form == PAM_FORM_GEMM_FP16_SPLIT)
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
    case PAM_FORM_GEMM_FP16_SPLIT: return launch_form<true, true>(p, n_frames, st);
    default: return cudaErrorInvalidValue;
    }
}

int prec_kernels() { return 3; }

cudaError_t launch_prec_bands(const pam_plan_s &p, const float2 *S, int n_frames, int n_bands, float *bands,
                              cudaStream_t st)
{
    if (p.n_apod != 3 || n_bands < 1 || n_bands > p.n_bins) return cudaErrorInvalidValue;
    switch (p.form) {
    case PAM_FORM_GEMM_BF16: return launch_bands_form<false>(p, S, n_frames, n_bands, bands, st);
    case PAM_FORM_GEMM_FP16: return launch_bands_form<true>(p, S, n_frames, n_bands, bands, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_prec_kernels()
{
    cudaError_t e;
    if ((e = set_gemm_smem<2, false, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, false, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<2, true, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, true, false>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<2, false, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<2, true, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, true, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, false, false, true>()) != cudaSuccess) return e;
    if ((e = set_gemm_smem<3, true, false, true>()) != cudaSuccess) return e;
    return set_gemm_smem<3, false, true>();
}

}  // namespace pam
