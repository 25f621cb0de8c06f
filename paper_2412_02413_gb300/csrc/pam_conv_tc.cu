// pam_conv_tc.cu -- tensor-core (tcgen05) forward of the 3x3 convolutions of
// the learned NCC-weight network, for rows of nx = 128 pixels: the first layer
// (5 -> 32, bias, ReLU), the hidden layers (32 -> 32, bias, ReLU) and the last
// layer (32 -> 1, bias, FP32 output).
//
// One output row is a GEMM with M = 128 pixels, N = 32 output channels (16
// for the last layer, whose channels 1..15 carry zero weights) and K = 9 taps
// x the input channels (one chunk of 8 for the first layer, padded in shared
// memory with a zero chunk to the K step of 16):
//   y[j][o] = b[o] + sum_{u,v,c} x[i+u-1][j+v-1][c] w[o][c][u][v].
// Activations are stored chunked and padded, [C/8][nz+2][nx+2][8] BF16 per
// frame, so one padded input row of one chunk of 8 channels is 130 pixels x
// 16 bytes, contiguous. Copied as it is into shared memory, 8 consecutive
// pixels of it form one 8-row x 16-byte core matrix of the canonical K-major
// layout (no swizzle): the A operand of tap (u, v) for channel chunks (c, c+1)
// is the staged row i+u-1 starting at pixel v, i.e. a descriptor whose start
// address moves by 16 bytes per pixel, with SBO = 128 bytes (next 8 pixels)
// and LBO = 2080 bytes (next chunk of channels). No im2col is materialised.
// The B operand (weights) is resident: [tap][chunk][out channel][8] BF16.
// Each row accumulates 9 x (chunks / 2) MMAs (M = 128, K = 16) into one of two
// tensor-memory accumulator sets.
//
// One CTA per (16-row strip, frame), 6 warps:
//   warp 0: bulk copies of the strip's 18 input rows through a ring of 6 slots;
//   warp 1: the MMA chain of each output row (one elected lane issues);
//   warps 2-5: the epilogue, each reading its quarter of the 128 TMEM lanes
//     (pixels), adding the bias, and storing BF16 after ReLU (or FP32 channel 0).
// All waits are bounded; on expiry the CTA sets the status word and drains.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pam_internal.h"
#include "pam_ptx.h"

namespace pam {
namespace {

using namespace ptx;

constexpr int W = 128, WP = W + 2;
constexpr int ROWS = 16;                       // output rows per CTA
constexpr int NSLOT = 6;                       // staged input rows
constexpr int CH_BYTES = WP * 16;              // one padded row of one chunk: 2080 B
constexpr int THREADS = 192;

// Shape of one layer: NCI input chunks in global memory, KCH staged chunks
// (at least 2: one K step), NCO GEMM columns.
template <int NCI, int NCO>
struct ConvShape {
    static constexpr int KCH = NCI < 2 ? 2 : NCI;
    static constexpr int ROW_BYTES = KCH * CH_BYTES;
    static constexpr int TAP_BYTES = KCH * NCO * 16;
    static constexpr int WT_BYTES = 9 * TAP_BYTES;
    static constexpr size_t SMEM = (size_t)WT_BYTES + (size_t)NSLOT * ROW_BYTES + 256;
    // kind::f16, FP32 accumulate, A = B = BF16, both K-major, N = NCO, M = 128.
    static constexpr unsigned IDESC = ptx::umma_idesc(false, 128, NCO);
};

__device__ __forceinline__ unsigned pack2(float a, float b)
{
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %2, %1;\n" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

template <int NCI, int NCO, bool F32OUT>
__global__ void __launch_bounds__(THREADS)
conv_tc_kernel(const uint4 *__restrict__ in, const uint4 *__restrict__ wt, const float *__restrict__ bias,
               void *__restrict__ out, int H, int *__restrict__ status)
{
    using CS = ConvShape<NCI, NCO>;
    constexpr int KCH = CS::KCH, ROW_BYTES = CS::ROW_BYTES, WT_BYTES = CS::WT_BYTES;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sW = sm;                                  // [9][KCH][NCO][8] BF16
    uint8_t *sRow = sm + WT_BYTES;                     // [NSLOT][KCH][130][8] BF16
    uint64_t *full = reinterpret_cast<uint64_t *>(sRow + NSLOT * ROW_BYTES);   // [NSLOT]
    uint64_t *sfree = full + NSLOT;                    // [NSLOT]
    uint64_t *afull = sfree + NSLOT;                   // [2]
    uint64_t *aempty = afull + 2;                      // [2]
    uint64_t *wbar = aempty + 2;                       // [1]
    uint64_t *dbar = wbar + 1;                         // [1] drain
    unsigned *tslot = reinterpret_cast<unsigned *>(dbar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int strip = blockIdx.x, f = blockIdx.y;
    const int HP = H + 2;
    const int r_first = strip * ROWS;
    const int nr = min(ROWS, H - r_first);   // output rows of this CTA
    const int nin = nr + 2;                  // input rows (padded rows r_first .. r_first + nr + 1)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(64u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&sfree[s], 1);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(&afull[t], 1);
            mbar_init(&aempty[t], 4);
        }
        mbar_init(wbar, 1);
        mbar_init(dbar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if constexpr (NCI < KCH) {
        // staged chunks NCI..KCH-1 of every slot stay zero (the K padding);
        // make the generic-proxy stores visible to the tensor core
        for (int i = tid; i < NSLOT * (KCH - NCI) * CH_BYTES / 16; i += THREADS) {
            const int slot = i / ((KCH - NCI) * CH_BYTES / 16), r = i % ((KCH - NCI) * CH_BYTES / 16);
            reinterpret_cast<uint4 *>(sRow + slot * ROW_BYTES + NCI * CH_BYTES)[r] = make_uint4(0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    auto wait = [&](uint64_t *b, unsigned parity) -> bool {
        if (mbar_try_wait_sleep(b, parity)) return true;
        const long long t0 = clock64();
        while (!mbar_try_wait_sleep(b, parity)) {
            if (*abort_flag) return false;
            if (clock64() - t0 > (1ll << 31)) {
                *abort_flag = 1;
                atomicOr(status, 1);
                return false;
            }
        }
        return true;
    };

    if (warp == 0) {
        // ---------------- producer: weights, then the input rows ----------------
        int issued = 0;
        bool ok = true;
        if (lane == 0) {
            mbar_expect_tx(wbar, WT_BYTES);
            bulk_g2s(sW, wt, WT_BYTES, wbar);
            for (int k = 0; k < nin && ok; ++k) {
                const int s = k % NSLOT;
                if (k >= NSLOT) ok = wait(&sfree[s], (unsigned)(k / NSLOT - 1) & 1u);
                if (!ok) break;
                mbar_expect_tx(&full[s], NCI * CH_BYTES);
                const int prow = r_first + k;
                for (int c = 0; c < NCI; ++c)
                    bulk_g2s(sRow + s * ROW_BYTES + c * CH_BYTES, in + (((size_t)f * NCI + c) * HP + prow) * WP,
                              CH_BYTES, &full[s]);
                issued = k + 1;
            }
            if (!ok) {
                // let the copies in flight land before the CTA exits
                wait(wbar, 0);
                for (int k = issued - NSLOT < 0 ? 0 : issued - NSLOT; k < issued; ++k)
                    wait(&full[k % NSLOT], (unsigned)(k / NSLOT) & 1u);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        bool ok = __all_sync(0xffffffffu, wait(wbar, 0));
        bool any = false;
        const unsigned wbase = smem_u32(sW), rbase = smem_u32(sRow);
        for (int r = 0; r < nr && ok; ++r) {
            // input rows r, r+1, r+2 (the first two were waited for by earlier rows)
            for (int k = (r == 0 ? 0 : r + 2); k <= r + 2 && ok; ++k)
                ok = __all_sync(0xffffffffu, wait(&full[k % NSLOT], (unsigned)(k / NSLOT) & 1u));
            const int t = r & 1;
            if (ok && r >= 2) ok = __all_sync(0xffffffffu, wait(&aempty[t], (unsigned)((r >> 1) - 1) & 1u));
            if (!ok) break;
            tc_fence_after();
            const unsigned d = tmem + (unsigned)(t * 32);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int u = tap / 3, v = tap % 3;
                const unsigned arow = rbase + (unsigned)(((r + u) % NSLOT) * ROW_BYTES + v * 16);
#pragma unroll
                for (int h = 0; h < KCH / 2; ++h) {
                    const uint64_t a = umma_desc(arow + (unsigned)(2 * h * CH_BYTES), CH_BYTES, 128);
                    const uint64_t b = umma_desc(wbase + (unsigned)(tap * CS::TAP_BYTES + h * 2 * NCO * 16), NCO * 16, 128);
                    umma_elect(d, a, b, CS::IDESC, (tap | h) ? 1u : 0u);
                }
            }
            any = true;
            umma_commit_elect(&afull[t]);
            umma_commit_elect(&sfree[r % NSLOT]);
        }
        if (!ok && any && lane == 0) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(dbar))
                         : "memory");
            wait(dbar, 0);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM -> bias + ReLU -> BF16 ----------------
        const int quarter = warp & 3;
        const int j = 32 * quarter + lane;   // pixel = TMEM lane
        constexpr int NB = F32OUT ? 1 : 32;
        float b[NB];
#pragma unroll
        for (int o = 0; o < NB; ++o) b[o] = bias[o];
        for (int r = 0; r < nr; ++r) {
            const int t = r & 1;
            if (!__all_sync(0xffffffffu, wait(&afull[t], (unsigned)(r >> 1) & 1u))) break;
            tc_fence_after();
            const unsigned taddr = tmem + (unsigned)(t * 32) + ((unsigned)(32 * quarter) << 16);
            if constexpr (F32OUT) {
                unsigned a0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n" : "=r"(a0) : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&aempty[t]);
                reinterpret_cast<float *>(out)[((size_t)f * H + r_first + r) * W + j] = __uint_as_float(a0) + b[0];
            } else {
                unsigned acc[32];
                tmem_ld32(taddr, acc);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&aempty[t]);
                const int prow = r_first + r + 1;
                uint4 *dst = reinterpret_cast<uint4 *>(out) + (((size_t)f * 4) * HP + prow) * WP + (j + 1);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    float y[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) y[k] = fmaxf(__uint_as_float(acc[ch * 8 + k]) + b[ch * 8 + k], 0.0f);
                    dst[(size_t)ch * HP * WP] =
                        make_uint4(pack2(y[0], y[1]), pack2(y[2], y[3]), pack2(y[4], y[5]), pack2(y[6], y[7]));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(64u) : "memory");
}

template <int NCI, int NCO, bool F32OUT>
cudaError_t set_tc_smem()
{
    return cudaFuncSetAttribute(conv_tc_kernel<NCI, NCO, F32OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ConvShape<NCI, NCO>::SMEM);
}

template <int NCI, int NCO, bool F32OUT>
cudaError_t launch_tc(const uint4 *in, const uint4 *wt, const float *bias, void *out, int F, int H, int *status,
                      cudaStream_t st)
{
    dim3 grid((H + ROWS - 1) / ROWS, F);
    conv_tc_kernel<NCI, NCO, F32OUT><<<grid, THREADS, ConvShape<NCI, NCO>::SMEM, st>>>(in, wt, bias, out, H, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_conv_tc()
{
    cudaError_t e = set_tc_smem<1, 32, false>();
    if (e == cudaSuccess) e = set_tc_smem<4, 32, false>();
    if (e == cudaSuccess) e = set_tc_smem<4, 16, true>();
    return e;
}

cudaError_t launch_conv_tc(int layer, const uint4 *in, const uint4 *wt, const float *bias, void *out, int F, int H,
                           int *status, cudaStream_t st)
{
    if (layer == 0) return launch_tc<1, 32, false>(in, wt, bias, out, F, H, status, st);
    if (layer == 4) return launch_tc<4, 16, true>(in, wt, bias, out, F, H, status, st);
    return launch_tc<4, 32, false>(in, wt, bias, out, F, H, status, st);
}

}  // namespace pam
