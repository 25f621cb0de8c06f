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
// Work mapping of the fused kernel: one CTA per SM, 16 warps with one depth
// row per lane or 12 (8 below nx = 64) with two. Each depth row is owned by
// 2*(nx/16) lanes that each hold 8 pixels of that row for all apodizations.
// The nx-point inverse DFT is one radix-2 decimation-in-frequency split,
// folded into the staged spectra as below, followed by two (nx/2)-point
// halves. Each half is an 8-point DFT in registers, a twiddle, a transpose
// through padded shared memory and an (nx/16)-point DFT in registers. A CTA
// loops over a contiguous chunk of bins. Each bin's spectra and phase words
// are staged in shared memory by bulk copies, 3 or 4 bins in flight.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"
#include "pam_ptx.h"

namespace pam {

cudaError_t prepare_fft_kernels(const pam_plan_s &p);

namespace {

constexpr int PROP_WARPS = 16;
constexpr int PROP_THREADS = 32 * PROP_WARPS;
// Depth rows per lane (RPL) of a fused kernel: 1 with PROP_WARPS warps of up
// to 128 registers, or 2 with 12 warps of up to 168, where a lane takes two
// rows of the same pixels and every spectra and phase-word load from shared
// memory serves both. Two rows need 163 registers per thread, so 12 warps of
// them hold 1.5x the work in flight of 16 warps of one row in the same
// register file, and a CTA covers 1.5x the rows. Below nx = 64 the transposes
// of 12 such warps do not fit in shared memory, and 8 warps cover the rows of
// 16 warps of one row.
constexpr int prop_warps(int rpl, int nx) { return rpl == 1 ? PROP_WARPS : (nx >= 64 ? 12 : 8); }
// Bins in flight per CTA: 4, or 3 where 12 warps' transposes leave room for
// no more.
constexpr int prop_nstage(int rpl, int nx) { return prop_warps(rpl, nx) == 12 ? 3 : 4; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// Complex add and subtract as one packed FP32x2 instruction each (a - b as
// b * (-1) + a: the product is exact, so both round exactly like scalar FADDs).
// Measured on the fused kernel: 2% fewer cycles than scalar pairs. Storing the
// spectra pre-broadcast as (Re, Re, Im, Im) to pack the phasor products too
// was 5% slower: it doubles the spectra's shared-memory traffic.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// a + i b and a - i b: the swap of b's parts stays in scalar operands.
__device__ __forceinline__ float2 cadd_i(float2 a, float2 b) { return make_float2(a.x - b.y, a.y + b.x); }
__device__ __forceinline__ float2 csub_i(float2 a, float2 b) { return make_float2(a.x + b.y, a.y - b.x); }

// sum_u v_u * exp(+2 pi i u k / N), natural order, in place.
__device__ __forceinline__ void idft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd_i(d02, d13);   // d02 + i d13
    a3 = csub_i(d02, d13);
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
        // o_k *= exp(+2 pi i k / 8): (1 + i) o1 and (-1 + i) o3 here, the 1/sqrt(2) in the FMAs below
        o1 = make_float2(o1.x - o1.y, o1.x + o1.y);
        o3 = make_float2(-(o3.x + o3.y), o3.x - o3.y);
        const float2 rp = make_float2(r, r), rn = make_float2(-r, -r);
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = __ffma2_rn(rp, o1, e1); v[5] = __ffma2_rn(rn, o1, e1);
        v[2] = cadd_i(e2, o2); v[6] = csub_i(e2, o2);   // o2 times i
        v[3] = __ffma2_rn(rp, o3, e3); v[7] = __ffma2_rn(rn, o3, e3);
    }
};

// exp(2 pi i * w / 2^32) for a 32-bit fixed-point phase word w (the top word
// of the exact 64-bit phase accumulator). Read as a signed turn count in
// [-1/2, 1/2), the angle is already range-reduced, so the hardware sine and
// cosine approximations (absolute error about 5e-7 on [-pi, pi]) apply
// directly.
__device__ __forceinline__ float2 phase_cis(unsigned w)
{
    const float ang = (float)(int)w * 1.4629180792671596e-9f;  // 2 pi / 2^32
    float s, c;
    __sincosf(ang, &s, &c);
    return make_float2(c, s);
}

using namespace ptx;

// One CTA per SM (it takes the whole register file): with two, the warp
// scheduler favours the older CTA, which then finishes its share early and
// leaves the other running at half occupancy.
constexpr int PROP_CTAS = 1;

template <int NX, int RPL = 1> struct Shape {
    static constexpr int H = NX / 2;               // half length
    static constexpr int L2 = H / 8;               // lanes per half row
    static constexpr int LPR = 2 * L2;             // lanes per row
    static constexpr int RPW = 32 / LPR * RPL;     // rows per warp
    static constexpr int RPC = prop_warps(RPL, NX) * RPW;   // rows per CTA
    static constexpr int KPL = 8 / L2;             // second-stage DFTs per lane
    // Transpose regions per (aperture, row, half): 8 rows k1 x L2 columns, each
    // row padded by one float2 so that the stores of one k1 and the loads of
    // one column are free of bank conflicts.
    static constexpr bool V4 = NX == 128;          // second-stage reads as float4 pairs
    static constexpr int TS = V4 ? L2 + 2 : L2 + 1;   // transpose row (float2)
    static constexpr int RS = V4 ? 8 * TS + 8 : 8 * TS;   // transpose region (float2), 16 mod 32 words
    static __device__ __forceinline__ int tpos(int k1, int col) { return k1 * TS + col; }
    static_assert(NX == 16 || NX == 32 || NX == 64 || NX == 128, "built lateral lengths");
};

template <int NAP> struct Acc { static constexpr int N = NAP == 1 ? 1 : (NAP == 2 ? 3 : 6); };

// Tensor-memory columns of one CTA: the PROP_WARPS / 4 warps of each lane
// quadrant (w, w + 4, ...) hold 8 pixels x NACC sums per lane each, at columns
// [a][o] (a power of 2 of at least 32 columns is allocated); with two rows
// per lane, twice the columns per warp.
template <int NAP, int RPL = 1, int NX = 128> constexpr unsigned tmem_cols()
{
    constexpr unsigned need = (unsigned)(prop_warps(RPL, NX) / 4) * (unsigned)RPL * 8u * (unsigned)Acc<NAP>::N;
    return need <= 32u ? 32u : need <= 64u ? 64u : need <= 128u ? 128u : need <= 256u ? 256u : 512u;
}

template <int NAP, int NX, int RPL = 1>
constexpr size_t prop_smem_bytes()
{
    using S = Shape<NX, RPL>;
    constexpr int NSTAGE = prop_nstage(RPL, NX);
    return (size_t)128                                    // full / empty mbarriers
           + (size_t)NSTAGE * 2 * NAP * NX * sizeof(float2)   // paired spectra, one per stage
           + (size_t)NSTAGE * NX * sizeof(uint4)          // phase words + evanescent coefficients
           + (size_t)(NX / 2) * sizeof(float2)            // exp(+2 pi i m / (nx/2))
           + (size_t)prop_warps(RPL, NX) * NAP * S::RPW * 2 * S::RS * sizeof(float2);  // transposes
}

// Eq. 4 (with the Appendix A completion) for one pixel and one pair:
// C_qr / (sqrt(A_qq) sqrt(A_rr)). A pair with no energy gives eps, and the
// result is clamped below at eps (Sec. II-A). FP32 with correctly rounded
// sqrt and division: three roundings, below 3e-7 relative.
__device__ __forceinline__ float ncc_pair(float c, float aq, float ar, float eps)
{
    const float den = sqrtf(aq) * sqrtf(ar);
    const float rho = den > 0.0f ? c / den : eps;
    return rho < eps ? eps : rho;
}

// The per-pixel end of the method from the bin-summed accumulators a[]:
// AS (Eq. 3): the energy itself. AS-DAX / AS-TAX: the clamped pair NCCs, rho
// (rho_12, or Eq. 10's cube root of the three), and the coherent energy
// E = sum_k |sum_q p_q|^2 = sum A_qq + 2 sum C_qr. Writes the
// pre-normalisation maps and returns rho (0 for AS).
template <int NAP>
__device__ __forceinline__ float pixel_epilogue(const float (&a)[Acc<NAP>::N], const EpiOut &out, int f,
                                                size_t x)
{
    const size_t o = (size_t)f * out.npix + x;
    if constexpr (NAP == 1) {
        out.out_main[o] = a[0];
        return 0.0f;
    } else {
        float rho, E;
        if constexpr (NAP == 2) {
            rho = ncc_pair(a[2], a[0], a[1], out.eps);
            if (out.rho_pairs) out.rho_pairs[o] = rho;
            E = a[0] + a[1] + 2.0f * a[2];
        } else {
            const float r12 = ncc_pair(a[3], a[0], a[1], out.eps);
            const float r23 = ncc_pair(a[4], a[1], a[2], out.eps);
            const float r31 = ncc_pair(a[5], a[2], a[0], out.eps);
            if (out.rho_pairs) {
                float *rp = out.rho_pairs + (size_t)f * 3 * out.npix + x;
                rp[0] = r12;
                rp[out.npix] = r23;
                rp[2 * (size_t)out.npix] = r31;
            }
            rho = cbrtf(r12 * r23 * r31);  // Eq. 10
            E = (a[0] + a[1] + a[2]) + 2.0f * (a[3] + a[4] + a[5]);
        }
        E = fmaxf(E, 0.0f);
        out.rho_tmp[o] = rho;
        out.e_tmp[o] = E;
        if (out.image_as) out.image_as[o] = E;
        return rho;
    }
}

// Largest value over the CTA, folded into the frame's maximum. All rho > 0,
// so their float bits order like unsigned integers.
__device__ __forceinline__ void block_max_to(float v, unsigned *dst, float *scratch, int nthreads)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < nthreads / 32 ? scratch[threadIdx.x] : 0.0f;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (threadIdx.x == 0) atomicMax(dst, __float_as_uint(v));
    }
}

// The per-pixel sums over the bins (Eq. 3, Eq. 4 + Appendix A) live in tensor
// memory, not in registers: 48 accumulators per thread would hold the fused
// kernel to 2 CTAs per SM. A thread's 8 NACC sums are the columns
// tcol + a * 8 + o (sum a, pixel o) of its own lane; with rpl rows per lane,
// row rr's from tcol + rr * 8 * nacc.
__device__ __forceinline__ unsigned acc_tcol(unsigned tbase, int warp, int nacc, int rpl = 1)
{
    return tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)((warp >> 2) * rpl * 8 * nacc);
}

template <int NAP>
__device__ __forceinline__ void acc_zero(unsigned tcol)
{
    const float z[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (NAP == 1) {
        tmem_st8(tcol, z);
    } else if constexpr (NAP == 2) {
        tmem_st16(tcol, z);
        tmem_st8(tcol + 16, z);
    } else {
        tmem_st16(tcol, z);
        tmem_st16(tcol + 16, z);
        tmem_st16(tcol + 32, z);
    }
    tmem_wait_st();
}

// |a|^2 and Re(conj(a) b), accumulated into s
__device__ __forceinline__ float add_norm(float s, float2 a) { return fmaf(a.x, a.x, fmaf(a.y, a.y, s)); }
__device__ __forceinline__ float add_dot(float s, float2 a, float2 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, s)); }

// Adds one bin's fields p[q][o] to the sums: A_qq += |p_q|^2, C_qr += Re conj(p_q) p_r.
template <int NAP>
__device__ __forceinline__ void acc_update(unsigned tcol, const float2 (&p)[NAP][8])
{
    tmem_wait_st();   // the previous bin's stores have landed
    if constexpr (NAP == 1) {
        float v[8];
        tmem_ld8(tcol, v);
        tmem_wait_ld();
#pragma unroll
        for (int o = 0; o < 8; ++o) v[o] = add_norm(v[o], p[0][o]);
        tmem_st8(tcol, v);
    } else {
        float v[16];
        tmem_ld16(tcol, v);
        tmem_wait_ld();
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            v[o] = add_norm(v[o], p[0][o]);
            v[8 + o] = add_norm(v[8 + o], p[1][o]);
        }
        tmem_st16(tcol, v);
        if constexpr (NAP == 2) {
            float w[8];
            tmem_ld8(tcol + 16, w);
            tmem_wait_ld();
#pragma unroll
            for (int o = 0; o < 8; ++o) w[o] = add_dot(w[o], p[0][o], p[1][o]);
            tmem_st8(tcol + 16, w);
        } else {
            float w[16];
            tmem_ld16(tcol + 16, w);
            tmem_wait_ld();
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                w[o] = add_norm(w[o], p[2][o]);
                w[8 + o] = add_dot(w[8 + o], p[0][o], p[1][o]);
            }
            tmem_st16(tcol + 16, w);
            float y[16];
            tmem_ld16(tcol + 32, y);
            tmem_wait_ld();
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                y[o] = add_dot(y[o], p[1][o], p[2][o]);
                y[8 + o] = add_dot(y[8 + o], p[2][o], p[0][o]);
            }
            tmem_st16(tcol + 32, y);
        }
    }
}

// The sums of the thread's 8 pixels, acc[o][a], back in registers.
template <int NAP>
__device__ __forceinline__ void acc_read(unsigned tcol, float (&acc)[8][Acc<NAP>::N])
{
    constexpr int NACC = Acc<NAP>::N;
    tmem_wait_st();
    float v[8 * NACC];
#pragma unroll
    for (int c = 0; c < NACC; ++c) tmem_ld8(tcol + 8 * c, v + 8 * c);
    tmem_wait_ld();
#pragma unroll
    for (int o = 0; o < 8; ++o)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[o][a] = v[a * 8 + o];
}

// Shared-memory regions of the fused kernel (layout of prop_smem_bytes).
template <int NAP, int NX, int RPL = 1>
struct PropSmem {
    static constexpr int NSTAGE = prop_nstage(RPL, NX);
    uint64_t *full;   // [NSTAGE] data of a stage has landed
    uint64_t *empty;  // [NSTAGE] all warps are done with a stage
    unsigned *tslot;  // tensor-memory base address of the CTA's sums
    float4 *sQ;       // [NSTAGE][NAP][8][2][NX/16] paired spectra (lateral_kernel's layout)
    uint4 *sD;        // [NSTAGE][NX] phase words
    float2 *sW;       // [NX/2] exp(+2 pi i m / (nx/2))
    float2 *sT;       // per-warp transpose regions
    __device__ explicit PropSmem(unsigned char *raw)
    {
        full = reinterpret_cast<uint64_t *>(raw);
        empty = full + NSTAGE;
        tslot = reinterpret_cast<unsigned *>(raw + 120);
        sQ = reinterpret_cast<float4 *>(raw + 128);
        sD = reinterpret_cast<uint4 *>(sQ + NSTAGE * NAP * NX);
        sW = reinterpret_cast<float2 *>(sD + NSTAGE * NX);
        sT = sW + NX / 2;
    }
    // second-factor twiddles, the staging barriers and the tensor memory of
    // the sums (warp 0 allocates `tcols` columns); every thread calls this
    // once and gets the CTA's tensor-memory base address
    __device__ unsigned init(unsigned tcols) const
    {
        static_assert(2 * NSTAGE * sizeof(uint64_t) <= 120, "barriers overlap the tensor-memory slot");
        if (threadIdx.x < 32) tmem_alloc(tslot, tcols);
        for (int m = threadIdx.x; m < NX / 2; m += (int)blockDim.x) {
            float s, c;
            sincospif(2.0f * (float)m / (float)(NX / 2), &s, &c);
            sW[m] = make_float2(c, s);
        }
        if (threadIdx.x == 0) {
            for (int st = 0; st < NSTAGE; ++st) {
                mbar_init(&full[st], 1);
                mbar_init(&empty[st], prop_warps(RPL, NX));
            }
            mbar_fence_init();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        return *tslot;
    }
    // every thread calls this once after its last tensor-memory access
    __device__ void release(unsigned tbase, unsigned tcols) const
    {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x < 32) tmem_dealloc(tbase, tcols);
    }
};

// The bin loop of one row tile: Eq. 2 phasors, the inverse lateral DFT and
// the per-pixel sums over bins [b_begin, b_begin + nb) of one frame. Qf is the
// frame's [n_bins][NAP][8][2][NX/16] paired spectra (lateral_kernel's layout,
// 2 NAP NX complex values per bin). The lane's RPL rows rr (clamped into the
// frame) are jj[rr] at depths zj[rr]. `seq` counts the bins this CTA staged
// before this call: the staging ring's stage and phase continue from it. Row
// rr's sums accumulate in the thread's tensor-memory columns from
// tcol + rr * 8 * NACC. With FIELDS (one row per lane), lanes of valid rows
// also write bin b's fields to fields_row + b * bin_stride. Returns false if a
// bounded wait expired; the copies still in flight have landed by then.
template <int NAP, int NX, bool FIELDS, int RPL = 1>
__device__ __forceinline__ bool prop_bins(const PropSmem<NAP, NX, RPL> &sm, const float2 *__restrict__ Qf,
                                          const uint4 *__restrict__ phase, const int *__restrict__ bin_evan,
                                          int b_begin, int nb, const int (&jj)[RPL], const float (&zj)[RPL],
                                          unsigned seq, unsigned tcol, float2 *__restrict__ fields_row, bool row_ok,
                                          size_t bin_stride)
{
    using S = Shape<NX, RPL>;
    static_assert(!FIELDS || RPL == 1, "fields are written by the one-row form");
    constexpr int H = S::H, L2 = S::L2, LPR = S::LPR, RPW = S::RPW, KPL = S::KPL;
    constexpr int RS = S::RS;
    constexpr int NOUT = KPL * L2;  // 8 pixels per lane
    constexpr int NACC = Acc<NAP>::N;
    constexpr int NSTAGE = PropSmem<NAP, NX, RPL>::NSTAGE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = lane / LPR, g = (lane % LPR) / L2, n2 = lane % L2;
    float2 *myT = sm.sT + (size_t)warp * (NAP * RPW * 2 * RS);
    const float2 *sW = sm.sW;

    // Radix-2 DIF split: lanes of half g take
    // x_g[n'] = exp(2 pi i g n'/nx) (P[n'] + (-1)^g P[n'+H]); the twiddle and
    // the sign are in the paired spectra, so both halves use the same phasors.
    unsigned jw[RPL];
#pragma unroll
    for (int rr = 0; rr < RPL; ++rr) jw[rr] = (unsigned)jj[rr];

    // Staging pipeline: thread 0 keeps NSTAGE-1 bins in flight with TMA bulk
    // copies (spectra + phase words), each completing on the stage's `full`
    // barrier. Every warp arrives on the stage's `empty` barrier once it has
    // finished with the stage. Warps can therefore run up to NSTAGE-1 bins
    // apart, with no CTA-wide barrier per bin.
    constexpr unsigned BYTES_Q = NAP * NX * sizeof(float4), BYTES_D = NX * sizeof(uint4);
    int issued = 0;    // producer (thread 0): bins whose copies have been issued
    bool ok = true;    // false once a bounded wait expired
    auto issue_next = [&]() -> bool {
        const unsigned n = seq + (unsigned)issued;
        const int st = (int)(n % NSTAGE);
        if (n >= NSTAGE && !mbar_wait(&sm.empty[st], ((n / NSTAGE) - 1) & 1)) return false;
        const int b = b_begin + issued;
        mbar_expect_tx(&sm.full[st], BYTES_Q + BYTES_D);
        bulk_g2s(sm.sQ + st * NAP * NX, Qf + (size_t)b * 2 * NAP * NX, BYTES_Q, &sm.full[st]);
        bulk_g2s(sm.sD + st * NX, phase + (size_t)b * NX, BYTES_D, &sm.full[st]);
        ++issued;
        return true;
    };
    if (tid == 0)
        while (issued < nb && issued < NSTAGE - 1) issue_next();

    float2 twk[8];     // the lane's second-factor twiddles, for every bin
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) twk[k1] = sW[(n2 * k1) & (H - 1)];
    int done = 0;      // bins this warp has finished
    for (int i = 0; i < nb; ++i) {
        if (tid == 0 && issued < nb) ok = issue_next();
        const unsigned n = seq + (unsigned)i;
        const int stage = (int)(n % NSTAGE);
        if (ok) ok = mbar_wait(&sm.full[stage], (n / NSTAGE) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
            ok = false;
            break;
        }
        const int b = b_begin + i;
        const float4 *cQ = sm.sQ + stage * NAP * NX;
        const uint4 *cD = sm.sD + stage * NX;
        const bool evan = bin_evan[b] != 0;

        // Eq. 2 phasors at depth z_j: this lane computes those of the lateral
        // bins u = g H + L2 n1 + n2 (ph0) and takes the other half's from its
        // partner lane, lane ^ L2 (ph1). The row's phase word is
        // anchor + j*step_hi + hi32(j*step_lo); dropping the carry out of the
        // low word costs at most 2^-32 turn. One phase-word load serves the
        // lane's RPL rows.
        float2 ph0[RPL][8], ph1[RPL][8];
        if (evan) {
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const uint4 d = cD[g * H + L2 * n1 + n2];
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    const float2 c = phase_cis(d.x + jw[rr] * d.y + __umulhi(jw[rr], d.z));
                    const float a = exp2f(__uint_as_float(d.w) * zj[rr]);
                    ph0[rr][n1] = make_float2(c.x * a, c.y * a);
                }
            }
        } else {
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const uint4 d = cD[g * H + L2 * n1 + n2];
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) ph0[rr][n1] = phase_cis(d.x + jw[rr] * d.y + __umulhi(jw[rr], d.z));
            }
        }
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr)
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1)
                ph1[rr][n1] = make_float2(__shfl_xor_sync(0xffffffffu, ph0[rr][n1].x, L2),
                                          __shfl_xor_sync(0xffffffffu, ph0[rr][n1].y, L2));

        // first factor: 8-point DFT over n1, twiddle, into the transpose region.
        // The lane's twiddles are loaded once for all apertures (the compiler
        // reloads them per aperture otherwise; measured 2% faster). One spectra
        // load serves the lane's RPL rows.
#pragma unroll
        for (int q = 0; q < NAP; ++q) {
            float2 x[RPL][8];
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                // a ph0 + c ph1 as two chains of one multiply and three FMAs: 8 FMA-pipe
                // instructions where two complex products and a packed add take 9
                const float4 qq = cQ[((q * 8 + n1) * 2 + g) * L2 + n2];
                const float2 a = make_float2(qq.x, qq.y), c = make_float2(qq.z, qq.w);
#pragma unroll
                for (int rr = 0; rr < RPL; ++rr) {
                    const float2 p0 = ph0[rr][n1], p1 = ph1[rr][n1];
                    x[rr][n1] = make_float2(fmaf(a.x, p0.x, fmaf(-a.y, p0.y, fmaf(c.x, p1.x, -c.y * p1.y))),
                                            fmaf(a.x, p0.y, fmaf(a.y, p0.x, fmaf(c.x, p1.y, c.y * p1.x))));
                }
            }
#pragma unroll
            for (int rr = 0; rr < RPL; ++rr) {
                IDft<8>::run(x[rr]);
                float2 *reg = myT + ((q * RPW + r * RPL + rr) * 2 + g) * RS;
#pragma unroll
                for (int k1 = 0; k1 < 8; ++k1)
                    reg[S::tpos(k1, n2)] = k1 ? cmul(x[rr][k1], twk[k1]) : x[rr][k1];
            }
        }
        __syncwarp();

        // second factor: L2-point DFTs over n2; lane owns pixels i = 2(k1 + 8 k2) + g
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            const unsigned tcol_r = tcol + (unsigned)(rr * 8 * NACC);
            float2 p[NAP][NOUT];
#pragma unroll
            for (int q = 0; q < NAP; ++q) {
                const float2 *reg = myT + ((q * RPW + r * RPL + rr) * 2 + g) * RS;
#pragma unroll
                for (int s = 0; s < KPL; ++s) {
                    const int k1 = n2 * KPL + s;
                    float2 v[L2];
                    if constexpr (S::V4) {
                        const float4 *reg4 = reinterpret_cast<const float4 *>(reg + k1 * S::TS);
#pragma unroll
                        for (int t = 0; t < L2; t += 2) {
                            const float4 w4 = reg4[t / 2];
                            v[t] = make_float2(w4.x, w4.y);
                            v[t + 1] = make_float2(w4.z, w4.w);
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < L2; ++t) v[t] = reg[S::tpos(k1, t)];
                    }
                    IDft<L2>::run(v);
#pragma unroll
                    for (int k2 = 0; k2 < L2; ++k2) p[q][s * L2 + k2] = v[k2];
                }
            }

            // per-pixel sums over the bins
            acc_update<NAP>(tcol_r, p);
            if constexpr (FIELDS) {
                if (row_ok) {  // fields of bin b
                    float2 *dst = fields_row + (size_t)b * bin_stride;
#pragma unroll
                    for (int o = 0; o < NOUT; ++o) {
                        const int k1 = n2 * KPL + o / L2, k2 = o % L2;
                        dst[2 * (k1 + 8 * k2) + g] = p[0][o];
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[stage]);
        done = i + 1;
    }
    if (!ok && tid == 0) {
        // let copies still in flight land before the stages are reused or the CTA exits
        for (int k = done; k < issued; ++k) {
            const unsigned n = seq + (unsigned)k;
            mbar_wait(&sm.full[n % NSTAGE], (n / NSTAGE) & 1);
        }
    }
    return ok;
}

// CLUSTER: the n_split CTAs of a row tile form one thread-block cluster. After
// the bin loop they add their accumulators through distributed shared memory
// (in rank order, so the sum is deterministic) and finish the per-pixel
// epilogue themselves. Otherwise each CTA writes its partial sums to `part`
// for epi_reduce_kernel.
template <int NAP, int NX, bool FIELDS, bool CLUSTER>
__global__ void __launch_bounds__(PROP_THREADS, PROP_CTAS)
prop_corr_kernel(const float2 *__restrict__ Q, const uint4 *__restrict__ phase,
                 const int *__restrict__ bin_evan, int n_bins, int nz,
                 float z0f, float dzf, int n_split, float *__restrict__ part, float2 *__restrict__ fields,
                 EpiOut out)
{
    using S = Shape<NX>;
    constexpr int L2 = S::L2, LPR = S::LPR, RPW = S::RPW, RPC = S::RPC, KPL = S::KPL;
    constexpr int NACC = Acc<NAP>::N;
    constexpr int NOUT = KPL * L2;  // 8 pixels per lane

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const PropSmem<NAP, NX> sm(smem_raw);
    float2 *sT = sm.sT;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = lane / LPR, g = (lane % LPR) / L2, n2 = lane % L2;
    const int f = blockIdx.z, split = blockIdx.y;
    const int j = blockIdx.x * RPC + warp * RPW + r;
    const bool row_ok = j < nz;
    const int jj = row_ok ? j : nz - 1;
    const int b_begin = (int)(((long long)n_bins * split) / n_split);
    const int b_end = (int)(((long long)n_bins * (split + 1)) / n_split);

    const unsigned tbase = sm.init(tmem_cols<NAP>());
    const unsigned tcol = acc_tcol(tbase, warp, NACC);
    acc_zero<NAP>(tcol);
    const int jja[1] = {jj};
    const float zja[1] = {z0f + (float)jj * dzf};
    const bool ok = prop_bins<NAP, NX, FIELDS>(
        sm, Q + (size_t)f * n_bins * 2 * NAP * NX, phase, bin_evan, b_begin, b_end - b_begin, jja, zja, 0u, tcol,
        FIELDS ? fields + ((size_t)f * n_bins * nz + j) * NX : nullptr, row_ok, (size_t)nz * NX);
    if (!ok && lane == 0) atomicOr(out.status, 1);
    const bool aborted = __syncthreads_or(!ok) != 0;
    float acc[NOUT][NACC];
    acc_read<NAP>(tcol, acc);

    if constexpr (CLUSTER) {
        namespace cg = cooperative_groups;
        cg::cluster_group cluster = cg::this_cluster();
        constexpr int TILE = RPC * NX;  // pixels of the row tile (2048)
        float *sAcc = reinterpret_cast<float *>(sT);  // [NACC][TILE], reuses the transpose buffers
        __syncthreads();
        const int rowl = warp * RPW + r;
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int k1 = n2 * KPL + o / L2, k2 = o % L2;
            const int i = 2 * (k1 + 8 * k2) + g;
#pragma unroll
            for (int a = 0; a < NACC; ++a) sAcc[a * TILE + rowl * NX + i] = acc[o][a];
        }
        cluster.sync();
        // Each CTA of the cluster finishes one slice of the tile's pixels.
        const int cs = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
        const int per = (TILE + cs - 1) / cs;
        const int p_end = min(TILE, (rank + 1) * per);
        float rmax = 0.0f;
        for (int px = rank * per + tid; px < p_end; px += PROP_THREADS) {
            float a[NACC];
#pragma unroll
            for (int c = 0; c < NACC; ++c) a[c] = 0.0f;
            for (int c = 0; c < cs; ++c) {
                const float *rem = cluster.map_shared_rank(sAcc, c);
#pragma unroll
                for (int aa = 0; aa < NACC; ++aa) a[aa] += rem[aa * TILE + px];
            }
            const int row = blockIdx.x * RPC + px / NX;
            if (row < nz && !aborted) rmax = fmaxf(rmax, pixel_epilogue<NAP>(a, out, f, (size_t)row * NX + (px % NX)));
        }
        if constexpr (NAP > 1) {
            __shared__ float wmax[PROP_THREADS / 32];
            block_max_to(rmax, out.fmax + f, wmax, PROP_THREADS);
        }
        cluster.sync();  // keep this CTA's shared memory alive until every peer has read it
    } else {
        if (row_ok && !aborted) {
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
    sm.release(tbase, tmem_cols<NAP>());
}

// CTA holding tile-bin w of the linearized (frame, row tile, bin) sequence of
// W tile-bins when G CTAs take equal contiguous shares [c W / G, (c+1) W / G).
__host__ __device__ __forceinline__ int seg_cta_of(long long w, long long W, int G)
{
    return (int)(((w + 1) * (long long)G - 1) / W);
}

// Slot of CTA c's sums for tile tt when the tile is split between CTAs: a
// share has at most two partial segments, its first (slot 2c) and its last
// (slot 2c + 1).
__host__ __device__ __forceinline__ long long seg_slot(int c, long long tt, long long W, int G, int n_bins)
{
    const long long first_tt = ((long long)c * W / G) / n_bins;
    return 2LL * c + (first_tt < tt ? 1 : 0);
}

// Even division of the work: gridDim.x CTAs (one wave) each take an equal
// contiguous share of the W = frames x tiles x n_bins tile-bins, in (frame,
// tile, bin) order. A share is a run of segments, one per row tile it
// touches. A segment that covers all bins of its tile finishes the per-pixel
// epilogue itself; a partial one (only the first and the last of a share can
// be) writes its sums to slot seg_slot of part[slot][NACC][RPC][NX], and
// epi_reduce_seg_kernel adds a split tile's slots in CTA order. The staging
// ring carries over from segment to segment.
template <int NAP, int NX, int RPL>
__global__ void __launch_bounds__(32 * prop_warps(RPL, NX), PROP_CTAS)
prop_seg_kernel(const float2 *__restrict__ Q, const uint4 *__restrict__ phase, const int *__restrict__ bin_evan,
                int n_bins, int nz, int tiles, float z0f, float dzf, long long W, float *__restrict__ part,
                EpiOut out)
{
    using S = Shape<NX, RPL>;
    constexpr int L2 = S::L2, LPR = S::LPR, RPW = S::RPW, RPC = S::RPC, KPL = S::KPL;
    constexpr int NACC = Acc<NAP>::N;
    constexpr int NOUT = KPL * L2;
    constexpr int NT = 32 * prop_warps(RPL, NX);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const PropSmem<NAP, NX, RPL> sm(smem_raw);
    __shared__ float wmax[NT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = lane / LPR, g = (lane % LPR) / L2, n2 = lane % L2;
    const unsigned tbase = sm.init(tmem_cols<NAP, RPL, NX>());
    const unsigned tcol = acc_tcol(tbase, warp, NACC, RPL);
    const int G = gridDim.x, c = blockIdx.x;
    long long w = (long long)c * W / G;
    const long long w1 = (long long)(c + 1) * W / G;
    unsigned seq = 0;
    while (w < w1) {
        const long long tt = w / n_bins;
        const int b0 = (int)(w - tt * n_bins);
        const int nb = (int)min((long long)(n_bins - b0), w1 - w);
        const int f = (int)(tt / tiles), tile = (int)(tt - (long long)f * tiles);
        int jr[RPL], jj[RPL];
        float zj[RPL];
        bool rok[RPL];
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            jr[rr] = tile * RPC + warp * RPW + r * RPL + rr;
            rok[rr] = jr[rr] < nz;
            jj[rr] = rok[rr] ? jr[rr] : nz - 1;
            zj[rr] = z0f + (float)jj[rr] * dzf;
            acc_zero<NAP>(tcol + (unsigned)(rr * 8 * NACC));
        }
        const bool ok = prop_bins<NAP, NX, false, RPL>(sm, Q + (size_t)f * n_bins * 2 * NAP * NX, phase, bin_evan,
                                                       b0, nb, jj, zj, seq, tcol, nullptr, false, 0);
        seq += (unsigned)nb;
        if (!ok && lane == 0) atomicOr(out.status, 1);
        if (__syncthreads_or(!ok)) break;
        float rmax = 0.0f;
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            float acc[NOUT][NACC];
            acc_read<NAP>(tcol + (unsigned)(rr * 8 * NACC), acc);   // warp-collective
            if (nb == n_bins) {
                // the whole tile: per-pixel epilogue from the registers
                if (rok[rr]) {
#pragma unroll
                    for (int o = 0; o < NOUT; ++o) {
                        const int k1 = n2 * KPL + o / L2, k2 = o % L2;
                        const int i = 2 * (k1 + 8 * k2) + g;
                        rmax = fmaxf(rmax, pixel_epilogue<NAP>(acc[o], out, f, (size_t)jr[rr] * NX + i));
                    }
                }
            } else if (rok[rr]) {
                constexpr size_t plane = (size_t)RPC * NX;
                float *dst = part + (size_t)seg_slot(c, tt, W, G, n_bins) * NACC * plane +
                             (size_t)(jr[rr] - tile * RPC) * NX;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const int k1 = n2 * KPL + o / L2, k2 = o % L2;
                    const int i = 2 * (k1 + 8 * k2) + g;
#pragma unroll
                    for (int a = 0; a < NACC; ++a) dst[a * plane + i] = acc[o][a];
                }
            }
        }
        if constexpr (NAP > 1)
            if (nb == n_bins) block_max_to(rmax, out.fmax + f, wmax, NT);
        w += nb;
    }
    sm.release(tbase, tmem_cols<NAP, RPL, NX>());
}

// --------------------------------------------------------- epilogue ----

constexpr int EPI_THREADS = 128;

// Sums the per-split partials in split order (deterministic) and finishes
// the per-pixel epilogue. Each thread takes four pixels: one float4 of every
// accumulator plane of every split, all loads of a split issued before its
// sums.
template <int NAP>
__global__ void __launch_bounds__(EPI_THREADS)
epi_reduce_kernel(const float4 *__restrict__ part, int n_split, int npix4, EpiOut out)
{
    constexpr int NACC = Acc<NAP>::N;
    __shared__ float wmax[EPI_THREADS / 32];
    const int f = blockIdx.y;
    const int x4 = blockIdx.x * EPI_THREADS + threadIdx.x;
    float rmax = 0.0f;
    if (x4 < npix4) {
        float4 a[NACC];
#pragma unroll
        for (int c = 0; c < NACC; ++c) a[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 *src = part + (size_t)f * n_split * NACC * npix4 + x4;
        for (int s = 0; s < n_split; ++s) {
            float4 v[NACC];
#pragma unroll
            for (int c = 0; c < NACC; ++c) v[c] = src[((size_t)s * NACC + c) * npix4];
#pragma unroll
            for (int c = 0; c < NACC; ++c) {
                a[c].x += v[c].x; a[c].y += v[c].y; a[c].z += v[c].z; a[c].w += v[c].w;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float acc[NACC];
#pragma unroll
            for (int k = 0; k < NACC; ++k) acc[k] = reinterpret_cast<const float *>(&a[k])[i];
            rmax = fmaxf(rmax, pixel_epilogue<NAP>(acc, out, f, (size_t)x4 * 4 + i));
        }
    }
    if constexpr (NAP > 1) block_max_to(rmax, out.fmax + f, wmax, EPI_THREADS);
}

// The split tiles of prop_seg_kernel: for each pixel of a tile that two or
// more CTAs share, its slots added in CTA order (deterministic), then the
// per-pixel epilogue. A tile inside one CTA's share was finished by that CTA;
// its blocks return at once (a block's 128 pixels never straddle tiles).
// Layout as epi_reduce_kernel: one warp per accumulator over 32 groups of four
// pixels.
template <int NAP>
__global__ void __launch_bounds__(32 * Acc<NAP>::N)
epi_reduce_seg_kernel(const float4 *__restrict__ part, int npix4, int nx, int rpc, int n_bins, int tiles, long long W,
                      int G, EpiOut out)
{
    constexpr int NACC = Acc<NAP>::N;
    __shared__ float4 sA[NACC][32];
    __shared__ float wmax[NACC];
    const int f = blockIdx.y;
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile4 = rpc * nx / 4;                    // float4 groups per tile
    const int tile = (blockIdx.x * 32) / tile4;
    const long long tt = (long long)f * tiles + tile;
    const int cf = seg_cta_of(tt * n_bins, W, G), cl = seg_cta_of((tt + 1) * n_bins - 1, W, G);
    if (cf == cl) return;                              // block-uniform
    const int x4 = blockIdx.x * 32 + lane;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x4 < npix4) {
        // CTAs cf < cc <= cl start inside this tile (their first segment, slot
        // 2 cc); cf's segment is its last unless its share starts at this tile.
        // The slots' loads are all issued before the sums (in CTA order), in
        // batches of 16, so that their latencies overlap.
        constexpr int MAXS = 16;
        const int cf_slot = 2 * cf + ((tt > 0 && seg_cta_of(tt * n_bins - 1, W, G) == cf) ? 1 : 0);
        const size_t off = (size_t)c * tile4 + (x4 - tile * tile4);
        const int ns = cl - cf + 1;
        for (int base = 0; base < ns; base += MAXS) {
            float4 v[MAXS];
#pragma unroll
            for (int k = 0; k < MAXS; ++k) {
                const int cc = cf + base + k;
                const size_t slot = cc == cf ? (size_t)cf_slot : 2 * (size_t)cc;
                if (base + k < ns) v[k] = part[slot * NACC * tile4 + off];
            }
#pragma unroll
            for (int k = 0; k < MAXS; ++k)
                if (base + k < ns) {
                    a.x += v[k].x; a.y += v[k].y; a.z += v[k].z; a.w += v[k].w;
                }
        }
    }
    sA[c][lane] = a;
    __syncthreads();
    float rmax = 0.0f;
    if (c == 0 && x4 < npix4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float acc[NACC];
#pragma unroll
            for (int k = 0; k < NACC; ++k) acc[k] = reinterpret_cast<const float *>(&sA[k][lane])[i];
            rmax = fmaxf(rmax, pixel_epilogue<NAP>(acc, out, f, (size_t)x4 * 4 + i));
        }
    }
    if constexpr (NAP > 1) block_max_to(rmax, out.fmax + f, wmax, 32 * NACC);
}

// rho_n = rho / max (Sec. II-A: the maximum becomes exactly 1) and the image
// I = rho_n^2 E (Eq. 5 / Eq. 11). Four pixels per thread.
__global__ void __launch_bounds__(EPI_THREADS)
epi_normalize_kernel(const float4 *__restrict__ rho_tmp, const float4 *__restrict__ e_tmp,
                     const unsigned *__restrict__ fmax, int npix4, float4 *__restrict__ image,
                     float4 *__restrict__ rho_n)
{
    const int f = blockIdx.y;
    const int x = blockIdx.x * EPI_THREADS + threadIdx.x;
    if (x >= npix4) return;
    const size_t o = (size_t)f * npix4 + x;
    const float m = __uint_as_float(fmax[f]);
    const float4 r = rho_tmp[o], e = e_tmp[o];
    const float4 rn = make_float4(r.x / m, r.y / m, r.z / m, r.w / m);
    image[o] = make_float4(rn.x * rn.x * e.x, rn.y * rn.y * e.y, rn.z * rn.z * e.z, rn.w * rn.w * e.w);
    if (rho_n) rho_n[o] = rn;
}

// Persistent form for a batch of frames with their own bins and depth grids
// (uneven sample counts and depth ranges). Work items are (frame, row tile)
// pairs taken from a global counter; an item runs every bin of its frame, so
// its per-pixel epilogue follows directly from the registers. The staging
// ring's position carries over from item to item.
template <int NAP, int NX, int RPL>
__global__ void __launch_bounds__(32 * prop_warps(RPL, NX), PROP_CTAS)
prop_batch_kernel(const BatchFrame *__restrict__ frames, const int2 *__restrict__ items, int n_items,
                  const int *__restrict__ n_items_dev, int *__restrict__ counter, EpiOut out)
{
    if (n_items_dev) n_items = min(n_items, *n_items_dev);
    using S = Shape<NX, RPL>;
    constexpr int L2 = S::L2, LPR = S::LPR, RPW = S::RPW, RPC = S::RPC, KPL = S::KPL;
    constexpr int NACC = Acc<NAP>::N;
    constexpr int NOUT = KPL * L2;
    constexpr int NT = 32 * prop_warps(RPL, NX);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const PropSmem<NAP, NX, RPL> sm(smem_raw);
    __shared__ int s_item;
    __shared__ float wmax[NT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = lane / LPR, g = (lane % LPR) / L2, n2 = lane % L2;
    const unsigned tbase = sm.init(tmem_cols<NAP, RPL, NX>());
    const unsigned tcol = acc_tcol(tbase, warp, NACC, RPL);
    unsigned seq = 0;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const int2 w = items[it];
        const BatchFrame fr = frames[w.x];
        int jr[RPL], jj[RPL];
        float zj[RPL];
        bool rok[RPL];
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            jr[rr] = w.y * RPC + warp * RPW + r * RPL + rr;
            rok[rr] = jr[rr] < fr.nz;
            jj[rr] = rok[rr] ? jr[rr] : fr.nz - 1;
            zj[rr] = fr.z0f + (float)jj[rr] * fr.dzf;
            acc_zero<NAP>(tcol + (unsigned)(rr * 8 * NACC));
        }
        const bool ok = prop_bins<NAP, NX, false, RPL>(sm, fr.Q, fr.phase, fr.bin_evan, 0, fr.n_bins, jj, zj, seq,
                                                       tcol, nullptr, false, 0);
        seq += (unsigned)fr.n_bins;
        if (!ok && lane == 0) atomicOr(out.status, 1);
        if (__syncthreads_or(!ok)) break;
        float rmax = 0.0f;
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
            float acc[NOUT][NACC];
            acc_read<NAP>(tcol + (unsigned)(rr * 8 * NACC), acc);   // warp-collective
            if (rok[rr]) {
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const int k1 = n2 * KPL + o / L2, k2 = o % L2;
                    const int i = 2 * (k1 + 8 * k2) + g;
                    rmax = fmaxf(rmax, pixel_epilogue<NAP>(acc[o], out, 0, fr.out_off + (size_t)jr[rr] * NX + i));
                }
            }
        }
        block_max_to(rmax, out.fmax + w.x, wmax, NT);
    }
    sm.release(tbase, tmem_cols<NAP, RPL, NX>());
}

// Per-frame rho_n and image for a batch packed by per-frame pixel offsets.
__global__ void __launch_bounds__(EPI_THREADS)
epi_normalize_batch_kernel(const BatchFrame *__restrict__ frames, const float *__restrict__ rho_tmp,
                           const float *__restrict__ e_tmp, const unsigned *__restrict__ fmax,
                           float *__restrict__ image, float *__restrict__ rho_n)
{
    const int f = blockIdx.y;
    const BatchFrame fr = frames[f];
    const size_t npix = (size_t)fr.nz * fr.nx;
    const float m = __uint_as_float(fmax[f]);
    for (size_t x = (size_t)blockIdx.x * EPI_THREADS + threadIdx.x; x < npix; x += (size_t)gridDim.x * EPI_THREADS) {
        const size_t o = fr.out_off + x;
        const float rn = rho_tmp[o] / m;
        image[o] = rn * rn * e_tmp[o];
        if (rho_n) rho_n[o] = rn;
    }
}

template <int NAP, int NX, bool FIELDS, bool CLUSTER>
cudaError_t launch_prop_t(const pam_plan_s &p, int n_frames, int n_split, float *fields, const EpiOut &out,
                          cudaStream_t st, float *part = nullptr)
{
    using S = Shape<NX>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((p.nz + S::RPC - 1) / S::RPC, n_split, n_frames);
    cfg.blockDim = dim3(PROP_THREADS);
    cfg.dynamicSmemBytes = prop_smem_bytes<NAP, NX>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (CLUSTER) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = (unsigned)n_split;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, prop_corr_kernel<NAP, NX, FIELDS, CLUSTER>, p.w.Q, p.t.phase,
                                       p.t.bin_evan, p.n_bins, p.nz, (float)p.d.z0_m, (float)p.d.dz_m, n_split,
                                       part ? part : p.w.part, reinterpret_cast<float2 *>(fields), out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NAP, int NX, int RPL>
cudaError_t launch_seg_rt(const pam_plan_s &p, int n_frames, const EpiOut &out, cudaStream_t st)
{
    using S = Shape<NX, RPL>;
    static_assert(prop_smem_bytes<NAP, NX, RPL>() + 1024 <= 232448, "shared memory of the fused kernel");
    const int tiles = (p.nz + S::RPC - 1) / S::RPC;
    const long long W = (long long)n_frames * tiles * p.n_bins;
    const int G = prop_seg_ctas(p, n_frames);
    prop_seg_kernel<NAP, NX, RPL><<<G, 32 * prop_warps(RPL, NX), prop_smem_bytes<NAP, NX, RPL>(), st>>>(
        p.w.Q, p.t.phase, p.t.bin_evan, p.n_bins, p.nz, tiles, (float)p.d.z0_m, (float)p.d.dz_m, W, p.w.part, out);
    return cudaGetLastError();
}

template <int NAP, int NX>
cudaError_t launch_seg_t(const pam_plan_s &p, int n_frames, const EpiOut &out, cudaStream_t st)
{
    return p.lane_rows == 2 ? launch_seg_rt<NAP, NX, 2>(p, n_frames, out, st)
                            : launch_seg_rt<NAP, NX, 1>(p, n_frames, out, st);
}

template <int NX, bool CLUSTER>
cudaError_t launch_prop_nc(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields,
                           const EpiOut &out, cudaStream_t st)
{
    if (napq == 1) {
        return fields ? launch_prop_t<1, NX, true, CLUSTER>(p, n_frames, n_split, fields, out, st)
                      : launch_prop_t<1, NX, false, CLUSTER>(p, n_frames, n_split, nullptr, out, st);
    }
    if (napq == 2) return launch_prop_t<2, NX, false, CLUSTER>(p, n_frames, n_split, nullptr, out, st);
    return launch_prop_t<3, NX, false, CLUSTER>(p, n_frames, n_split, nullptr, out, st);
}

template <int NX>
cudaError_t launch_prop_nx(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields,
                           const EpiOut &out, cudaStream_t st)
{
    if (prop_seg_mode(p, n_split, fields != nullptr)) {
        if (napq == 1) return launch_seg_t<1, NX>(p, n_frames, out, st);
        if (napq == 2) return launch_seg_t<2, NX>(p, n_frames, out, st);
        return launch_seg_t<3, NX>(p, n_frames, out, st);
    }
    return prop_uses_cluster(n_split) ? launch_prop_nc<NX, true>(p, n_frames, napq, n_split, fields, out, st)
                                      : launch_prop_nc<NX, false>(p, n_frames, napq, n_split, fields, out, st);
}

// Dynamic shared memory of a fused kernel, and the largest shared-memory
// carveout, so that PROP_CTAS CTAs fit on an SM.
template <class K>
cudaError_t set_smem_of(K kernel, size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int NAP, int NX, bool FIELDS, bool CLUSTER>
cudaError_t set_smem()
{
    return set_smem_of(prop_corr_kernel<NAP, NX, FIELDS, CLUSTER>, prop_smem_bytes<NAP, NX>());
}

template <int NX, bool CLUSTER>
cudaError_t prepare_nc()
{
    cudaError_t e;
    if ((e = set_smem<1, NX, false, CLUSTER>()) != cudaSuccess) return e;
    if ((e = set_smem<1, NX, true, CLUSTER>()) != cudaSuccess) return e;
    if ((e = set_smem<2, NX, false, CLUSTER>()) != cudaSuccess) return e;
    return set_smem<3, NX, false, CLUSTER>();
}

template <int NX>
cudaError_t prepare_nx()
{
    cudaError_t e = prepare_nc<NX, true>();
    if (e == cudaSuccess) e = prepare_nc<NX, false>();
    if (e == cudaSuccess) e = set_smem_of(prop_batch_kernel<2, NX, 1>, prop_smem_bytes<2, NX, 1>());
    if (e == cudaSuccess) e = set_smem_of(prop_batch_kernel<3, NX, 1>, prop_smem_bytes<3, NX, 1>());
    if (e == cudaSuccess) e = set_smem_of(prop_batch_kernel<2, NX, 2>, prop_smem_bytes<2, NX, 2>());
    if (e == cudaSuccess) e = set_smem_of(prop_batch_kernel<3, NX, 2>, prop_smem_bytes<3, NX, 2>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<1, NX, 1>, prop_smem_bytes<1, NX, 1>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<2, NX, 1>, prop_smem_bytes<2, NX, 1>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<3, NX, 1>, prop_smem_bytes<3, NX, 1>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<1, NX, 2>, prop_smem_bytes<1, NX, 2>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<2, NX, 2>, prop_smem_bytes<2, NX, 2>());
    if (e == cudaSuccess) e = set_smem_of(prop_seg_kernel<3, NX, 2>, prop_smem_bytes<3, NX, 2>());
    return e;
}

template <int NAP, int NX, int RPL>
cudaError_t launch_batch_t(int grid, const BatchFrame *frames, const int2 *items, int n_items, const int *n_items_dev,
                           int *counter, const EpiOut &out, cudaStream_t st)
{
    static_assert(prop_smem_bytes<NAP, NX, RPL>() + 1024 <= 232448, "shared memory of the fused kernel");
    prop_batch_kernel<NAP, NX, RPL><<<grid, 32 * prop_warps(RPL, NX), prop_smem_bytes<NAP, NX, RPL>(), st>>>(
        frames, items, n_items, n_items_dev, counter, out);
    return cudaGetLastError();
}

template <int NX>
cudaError_t launch_batch_nx(int napq, int grid, const BatchFrame *frames, const int2 *items, int n_items,
                            const int *n_items_dev, int *counter, const EpiOut &out, cudaStream_t st, int rpl)
{
    if (rpl == 2)
        return napq == 2 ? launch_batch_t<2, NX, 2>(grid, frames, items, n_items, n_items_dev, counter, out, st)
                         : launch_batch_t<3, NX, 2>(grid, frames, items, n_items, n_items_dev, counter, out, st);
    return napq == 2 ? launch_batch_t<2, NX, 1>(grid, frames, items, n_items, n_items_dev, counter, out, st)
                     : launch_batch_t<3, NX, 1>(grid, frames, items, n_items, n_items_dev, counter, out, st);
}

template <int NX>
cudaError_t launch_bands_nx(const pam_plan_s &p, int n_frames, int n_bands, float *bands, cudaStream_t st)
{
    EpiOut out;
    out.status = p.w.status;
    return launch_prop_t<1, NX, false, false>(p, n_frames, n_bands, nullptr, out, st, bands);
}

// Failure-path check: one warp waits on an mbarrier that no thread or copy
// ever completes, with the bounded wait every staging pipeline uses. The wait
// gives up after about one second and the kernel reports through the status
// word, as a real stalled pipeline would, then exits normally.
__global__ void expire_wait_kernel(int *__restrict__ status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0);
    if (!ok && threadIdx.x == 0) atomicOr(status, 1);
}

}  // namespace

cudaError_t launch_expire_wait(int *status, cudaStream_t st)
{
    expire_wait_kernel<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

int prop_rows_per_cta(int nx, int rpl) { return prop_warps(rpl, nx) * rpl * (32 / (nx / 8)); }

// Rows per CTA of prop_seg_kernel for the plan's rows per lane.
static int seg_rows(const pam_plan_s &p) { return prop_rows_per_cta(p.nx, p.lane_rows); }

int prop_ctas_per_sm() { return PROP_CTAS; }

bool prop_uses_cluster(int n_split) { return n_split <= kMaxClusterSplit; }

bool prop_seg_mode(const pam_plan_s &p, int n_split, bool fields)
{
    (void)n_split;
    return p.seg_ok && p.split_override == 0 && !fields;
}

int prop_seg_ctas(const pam_plan_s &p, int n_frames)
{
    const int rows = seg_rows(p);
    const long long W = (long long)n_frames * ((p.nz + rows - 1) / rows) * p.n_bins;
    long long G = (long long)PROP_CTAS * p.num_sms;
    if (p.grid_override > 0 && p.grid_override < G) G = p.grid_override;
    return (int)(W < G ? W : G);
}

size_t prop_seg_part_floats(const pam_plan_s &p)
{
    // the larger row tile of the two rows-per-lane settings, which can change after the plan is made
    const int r1 = prop_rows_per_cta(p.nx, 1), r2 = prop_rows_per_cta(p.nx, 2);
    const int rows = r1 > r2 ? r1 : r2;
    return (size_t)2 * PROP_CTAS * p.num_sms * n_acc(p.n_apod) * rows * p.nx;
}

int choose_split(const pam_plan_s &p, int n_frames)
{
    const int rows = prop_rows_per_cta(p.nx);
    const long long row_tiles = (p.nz + rows - 1) / rows;
    long long ns;
    if (p.split_override > 0) {
        ns = p.split_override;
    } else {
        // About PROP_CTAS CTAs per SM (the register limit) over the whole grid. The
        // cluster reduction is used when this split is small enough anyway:
        // capping a larger split at the cluster size loses more to load
        // imbalance than the partial sums cost (128 x 512 frame: 9 -> 8 splits
        // measured 135 us against 108 + 11 us).
        const long long target = (long long)PROP_CTAS * p.num_sms;
        ns = target / (row_tiles * n_frames);
    }
    if (ns < 1) ns = 1;
    if (ns > p.n_bins) ns = p.n_bins;
    // the global-partials path needs n_frames * n_split units of workspace
    if (!prop_uses_cluster((int)ns) && (size_t)ns * n_frames > p.w.part_units)
        ns = (long long)(p.w.part_units / n_frames) > 1 ? (long long)(p.w.part_units / n_frames) : 1;
    return (int)ns;
}

cudaError_t launch_prop(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields, const EpiOut &out,
                        cudaStream_t st)
{
    switch (p.nx) {
    case 16: return launch_prop_nx<16>(p, n_frames, napq, n_split, fields, out, st);
    case 32: return launch_prop_nx<32>(p, n_frames, napq, n_split, fields, out, st);
    case 64: return launch_prop_nx<64>(p, n_frames, napq, n_split, fields, out, st);
    case 128: return launch_prop_nx<128>(p, n_frames, napq, n_split, fields, out, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epilogue(const pam_plan_s &p, int n_frames, int napq, int n_split, const EpiOut &out,
                            cudaStream_t st, bool from_partials, bool fields)
{
    const int npix4 = p.nz * p.nx / 4;  // nx is a multiple of 16
    dim3 grid((npix4 + EPI_THREADS - 1) / EPI_THREADS, n_frames);
    auto v4 = [](float *q) { return reinterpret_cast<float4 *>(q); };
    if (!from_partials && prop_seg_mode(p, n_split, fields)) {
        const int rows = seg_rows(p);
        const int tiles = (p.nz + rows - 1) / rows;
        const long long W = (long long)n_frames * tiles * p.n_bins;
        const int G = prop_seg_ctas(p, n_frames);
        const float4 *part = reinterpret_cast<const float4 *>(p.w.part);
        dim3 rgrid((npix4 + 31) / 32, n_frames);
        if (napq == 1)
            epi_reduce_seg_kernel<1><<<rgrid, 32 * Acc<1>::N, 0, st>>>(part, npix4, p.nx, rows, p.n_bins, tiles, W, G, out);
        else if (napq == 2)
            epi_reduce_seg_kernel<2><<<rgrid, 32 * Acc<2>::N, 0, st>>>(part, npix4, p.nx, rows, p.n_bins, tiles, W, G, out);
        else
            epi_reduce_seg_kernel<3><<<rgrid, 32 * Acc<3>::N, 0, st>>>(part, npix4, p.nx, rows, p.n_bins, tiles, W, G, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else if (from_partials || !prop_uses_cluster(n_split)) {
        const float4 *part = reinterpret_cast<const float4 *>(p.w.part);
        if (napq == 1)
            epi_reduce_kernel<1><<<grid, EPI_THREADS, 0, st>>>(part, n_split, npix4, out);
        else if (napq == 2)
            epi_reduce_kernel<2><<<grid, EPI_THREADS, 0, st>>>(part, n_split, npix4, out);
        else
            epi_reduce_kernel<3><<<grid, EPI_THREADS, 0, st>>>(part, n_split, npix4, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (napq == 1) return cudaSuccess;
    epi_normalize_kernel<<<grid, EPI_THREADS, 0, st>>>(v4(out.rho_tmp), v4(out.e_tmp), out.fmax, npix4,
                                                       v4(out.out_main), v4(out.rho_n));
    return cudaGetLastError();
}

cudaError_t launch_prop_batch(int nx, int napq, int grid, const BatchFrame *frames, const int2 *items, int n_items,
                              int *counter, const EpiOut &out, cudaStream_t st, const int *n_items_dev, int rpl)
{
    if (napq != 2 && napq != 3) return cudaErrorInvalidValue;
    if (rpl != 1 && rpl != 2) return cudaErrorInvalidValue;
    switch (nx) {
    case 16: return launch_batch_nx<16>(napq, grid, frames, items, n_items, n_items_dev, counter, out, st, rpl);
    case 32: return launch_batch_nx<32>(napq, grid, frames, items, n_items, n_items_dev, counter, out, st, rpl);
    case 64: return launch_batch_nx<64>(napq, grid, frames, items, n_items, n_items_dev, counter, out, st, rpl);
    case 128: return launch_batch_nx<128>(napq, grid, frames, items, n_items, n_items_dev, counter, out, st, rpl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prop_bands(const pam_plan_s &p, int n_frames, int n_bands, float *bands, cudaStream_t st)
{
    if (n_bands < 1 || n_bands > p.n_bins) return cudaErrorInvalidValue;
    switch (p.nx) {
    case 16: return launch_bands_nx<16>(p, n_frames, n_bands, bands, st);
    case 32: return launch_bands_nx<32>(p, n_frames, n_bands, bands, st);
    case 64: return launch_bands_nx<64>(p, n_frames, n_bands, bands, st);
    case 128: return launch_bands_nx<128>(p, n_frames, n_bands, bands, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_normalize_batch(int n_frames, int max_npix, const BatchFrame *frames, const EpiOut &out,
                                   cudaStream_t st)
{
    dim3 grid((unsigned)((max_npix + EPI_THREADS - 1) / EPI_THREADS), (unsigned)n_frames);
    epi_normalize_batch_kernel<<<grid, EPI_THREADS, 0, st>>>(frames, out.rho_tmp, out.e_tmp, out.fmax,
                                                             out.out_main, out.rho_n);
    return cudaGetLastError();
}

int epilogue_kernels(const pam_plan_s &p, int napq, int n_split, bool fields)
{
    const bool reduce = prop_seg_mode(p, n_split, fields) || !prop_uses_cluster(n_split);
    return (reduce ? 1 : 0) + (napq > 1 ? 1 : 0);
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
