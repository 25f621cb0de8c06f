// pam_batch.cu -- many frames, each with its own sample count, depth range
// and bins, in one call (pam_batch_*), replayed as a CUDA graph:
//   time_dft_kernel      the selected bins of Eq. 1 by direct summation (any nt)
//   lateral_kernel       apodized lateral FFT x napq (Eq. 1), per-frame masks
//   prop_batch_kernel    persistent propagate-and-correlate over (frame, row
//                        tile) items with the per-pixel NCC/TAX epilogue
//   epi_normalize_batch  rho_n and the image per frame (Eq. 5 / 11)
// Every frame is the plain AS-DAX / AS-TAX problem of its own geometry; only
// the packing of inputs and outputs is shared.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pam_internal.h"

namespace pam {
namespace {

struct DftFrame {
    size_t rf_off;   // floats: start of the frame's [ne][nt] block
    size_t tw_off;   // float2: start of the frame's twiddle table
    int nt;
    int n_bins;      // bins of this frame (<= the batch's n_bins; the rest of its S rows are zeroed)
};

constexpr int DFT_WARPS = 8;
constexpr int DFT_THREADS = 32 * DFT_WARPS;
constexpr int DFT_BPW = 4;                      // bins per warp
constexpr int DFT_BINS = DFT_WARPS * DFT_BPW;   // bins per CTA
constexpr int DFT_T = 64;                       // samples per staged tile
constexpr int DFT_MAX_NT = 16384;

// S[f][b][e] = sum_t rf[e][t] exp(-2 pi i k_b t / nt)   (Eq. 1, selected bins)
// by direct summation with the exact index reduction m = k t mod nt into the
// frame's twiddle table exp(-2 pi i m / nt) (built in FP64). One CTA per
// (32 bins, frame): warp w owns bins 4w..4w+3, lane l channels l + 32 c,
// c < CPL. Per 64-sample tile the CTA stages the channels' samples (rows of
// 64 + 4 floats) and the 32 bins' twiddles for those samples (rows of 64 + 4
// float2, gathered from the table, which stays in L1/L2, with the index
// stepped by k per sample), with cp.async into two buffers: tile i+1 is in
// flight while tile i is summed. Two CTAs share an SM.
// The inner loop then reads 4 samples of a channel and 4 twiddles of a bin as
// 16-byte loads (twiddle reads are warp-uniform broadcasts) and updates Re
// and Im with one packed FMA (fma.rn.f32x2). The sum of each tile is formed on
// its own and then added to the total, so the rounding error grows like
// 64 + nt/64 ulp rather than nt ulp.
constexpr int XROW = DFT_T + 4;     // floats per staged channel row
constexpr int WROW = DFT_T + 4;     // float2 per staged twiddle row

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// 4- and 8-byte asynchronous copies global -> shared (cp.async); `valid` false
// writes zeros without reading.
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int CPL>
__global__ void __launch_bounds__(DFT_THREADS, CPL >= 8 ? 1 : 2)
time_dft_kernel(const float *__restrict__ rf, const DftFrame *__restrict__ frames, const int *__restrict__ bins,
                int n_bins, int ne, const float2 *__restrict__ tw_all, float2 *__restrict__ S)
{
    extern __shared__ __align__(16) float2 dsm[];
    constexpr int WBUF = DFT_BINS * WROW;               // float2 per twiddle buffer
    constexpr int XBUF = 32 * CPL * XROW;               // floats per sample buffer
    const int f = blockIdx.y;
    const DftFrame fr = frames[f];
    const int nt = fr.nt;
    float2 *wt = dsm;                                                  // [2][DFT_BINS][WROW]
    float *xs = reinterpret_cast<float *>(wt + 2 * WBUF);             // [2][32 CPL][XROW]
    const float2 *tw = tw_all + fr.tw_off;                             // [nt]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // twiddle staging role: bin bb of the CTA, samples s + 8 j of each tile
    const int bb = tid >> 3, sg = tid & 7;
    const int bglob = blockIdx.x * DFT_BINS + bb;
    const int kb = bglob < fr.n_bins ? bins[(size_t)f * n_bins + bglob] : 0;
    const int kstep8 = (int)((8LL * kb) % nt);
    const float *x = rf + fr.rf_off;
    // Copies of tile t0 into buffer `buf` (all threads; one commit group).
    auto stage = [&](int t0, int buf) {
        const int tn = min(DFT_T, nt - t0);
        float *xb = xs + buf * XBUF;
        for (int e = warp; e < 32 * CPL; e += DFT_WARPS) {
            const bool erow = e < ne;
            const float *row = x + (size_t)(erow ? e : 0) * nt + t0;
            for (int t = lane; t < DFT_T; t += 32)
                cp_async4(xb + e * XROW + t, row + (t < tn ? t : 0), erow && t < tn);
        }
        float2 *wb = wt + buf * WBUF + bb * WROW;
        int idx = (int)(((long long)kb * (t0 + sg)) % nt);
#pragma unroll
        for (int j = 0; j < DFT_T / 8; ++j) {
            cp_async8(wb + sg + 8 * j, tw + idx);
            idx += kstep8;
            if (idx >= nt) idx -= nt;
        }
        cp_async_commit();
    };
    float2 tot[DFT_BPW][CPL];
#pragma unroll
    for (int i = 0; i < DFT_BPW; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) tot[i][c] = make_float2(0.f, 0.f);
    const int ntiles = (nt + DFT_T - 1) / DFT_T;
    stage(0, 0);
    for (int it = 0; it < ntiles; ++it) {
        const int buf = it & 1, t0 = it * DFT_T, tn = min(DFT_T, nt - t0);
        if (it + 1 < ntiles) stage(t0 + DFT_T, buf ^ 1);
        else cp_async_commit();                 // empty group keeps the wait count uniform
        cp_async_wait1();                       // this thread's copies of tile `it` have landed
        __syncthreads();                        // ... and everyone else's
        const float *xb = xs + buf * XBUF;
        const float2 *wb = wt + buf * WBUF;
        float2 part[DFT_BPW][CPL];
#pragma unroll
        for (int i = 0; i < DFT_BPW; ++i)
#pragma unroll
            for (int c = 0; c < CPL; ++c) part[i][c] = make_float2(0.f, 0.f);
        // samples past tn are zero in xs, so whole groups of 4 are summed
        for (int t = 0; t < tn; t += 4) {
            float4 xv[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) xv[c] = *reinterpret_cast<const float4 *>(xb + (lane + 32 * c) * XROW + t);
#pragma unroll
            for (int i = 0; i < DFT_BPW; ++i) {
                const float4 *wp = reinterpret_cast<const float4 *>(wb + (warp * DFT_BPW + i) * WROW + t);
                const float4 w01 = wp[0], w23 = wp[1];
                const float2 w0 = make_float2(w01.x, w01.y), w1 = make_float2(w01.z, w01.w);
                const float2 w2 = make_float2(w23.x, w23.y), w3 = make_float2(w23.z, w23.w);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    float2 a = part[i][c];
                    a = __ffma2_rn(make_float2(xv[c].x, xv[c].x), w0, a);
                    a = __ffma2_rn(make_float2(xv[c].y, xv[c].y), w1, a);
                    a = __ffma2_rn(make_float2(xv[c].z, xv[c].z), w2, a);
                    a = __ffma2_rn(make_float2(xv[c].w, xv[c].w), w3, a);
                    part[i][c] = a;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < DFT_BPW; ++i)
#pragma unroll
            for (int c = 0; c < CPL; ++c) tot[i][c] = __fadd2_rn(tot[i][c], part[i][c]);
        __syncthreads();                        // buffer `buf` is free for tile it + 2
    }
    const int b0 = blockIdx.x * DFT_BINS + warp * DFT_BPW;
#pragma unroll
    for (int i = 0; i < DFT_BPW; ++i) {
        if (b0 + i >= n_bins) continue;
        const bool used = b0 + i < fr.n_bins;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int e = lane + 32 * c;
            if (e < ne) S[((size_t)f * n_bins + b0 + i) * ne + e] = used ? tot[i][c] : make_float2(0.f, 0.f);
        }
    }
}

size_t dft_smem(int, int cpl)
{
    return 2 * ((size_t)DFT_BINS * WROW * sizeof(float2) + (size_t)32 * cpl * XROW * sizeof(float));
}

template <int CPL>
cudaError_t launch_dft_t(const float *rf, const DftFrame *frames, const int *bins, int n_bins, int ne, int F,
                         const float2 *tw, float2 *S, int max_nt, cudaStream_t st)
{
    dim3 grid((unsigned)((n_bins + DFT_BINS - 1) / DFT_BINS), (unsigned)F);
    time_dft_kernel<CPL><<<grid, DFT_THREADS, dft_smem(max_nt, CPL), st>>>(rf, frames, bins, n_bins, ne, tw, S);
    return cudaGetLastError();
}

cudaError_t launch_dft(int cpl, const float *rf, const DftFrame *frames, const int *bins, int n_bins, int ne, int F,
                       const float2 *tw, float2 *S, int max_nt, cudaStream_t st)
{
    switch (cpl) {
    case 1: return launch_dft_t<1>(rf, frames, bins, n_bins, ne, F, tw, S, max_nt, st);
    case 2: return launch_dft_t<2>(rf, frames, bins, n_bins, ne, F, tw, S, max_nt, st);
    case 4: return launch_dft_t<4>(rf, frames, bins, n_bins, ne, F, tw, S, max_nt, st);
    case 8: return launch_dft_t<8>(rf, frames, bins, n_bins, ne, F, tw, S, max_nt, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_dft()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(time_dft_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)dft_smem(DFT_MAX_NT, 1))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(time_dft_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)dft_smem(DFT_MAX_NT, 2))) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(time_dft_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)dft_smem(DFT_MAX_NT, 4))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(time_dft_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dft_smem(DFT_MAX_NT, 8));
}

pam_status fail(pam_status s, const std::string &msg) { return set_error(s, msg.c_str()); }
pam_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(PAM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device pointer argument: non-null, 16-byte aligned, device or managed memory.
pam_status check_dev(const void *ptr, const char *name, bool required)
{
    if (!ptr) return required ? fail(PAM_ERR_INVALID_ARG, std::string(name) + " is NULL") : PAM_OK;
    if (reinterpret_cast<uintptr_t>(ptr) & 15u)
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return PAM_OK;
}

size_t round4(size_t v) { return (v + 3) & ~(size_t)3; }

}  // namespace
}  // namespace pam

struct pam_batch_s {
    pam_plan_s *base = nullptr;     // geometry, apodization, workspace for F frames of n_bins bins
    int F = 0, n_bins = 0, ne = 0, nx = 0, napq = 0, max_nt = 0, max_npix = 0, cpl = 4;
    int grid = 0, grid_override = 0, n_items = 0;
    int rpl = 1;                     // depth rows per lane of the fused kernel (2 for nx >= 64)
    std::vector<int> nt, nz, nbf, bins_h;   // per frame: samples, rows, bin count; bins [F][n_bins]
    std::vector<size_t> rf_off, px_off;
    size_t rf_total = 0, px_total = 0;
    int *bins = nullptr;             // [F][n_bins]
    uint4 *phase = nullptr;          // [F][n_bins][nx]
    float *live = nullptr;           // [F][n_bins][nx]
    int *bin_evan = nullptr;         // [F][n_bins]
    float2 *tw = nullptr;            // per frame [nt_f]
    pam::DftFrame *dft = nullptr;    // [F]
    pam::BatchFrame *frames = nullptr;
    int2 *items = nullptr;           // (frame, row tile)
    int *counter = nullptr;          // work-queue head
    bool use_graph = true;
    cudaStream_t cap = nullptr;      // capture stream
    cudaGraphExec_t exec = nullptr;
    const float *g_rf = nullptr;
    float *g_img = nullptr, *g_rho = nullptr;
    int g_grid = 0;
    long long kernels = 0;
};

namespace {

void batch_free(pam_batch_s *b)
{
    auto fr = [](void *q) { if (q) cudaFree(q); };
    fr(b->bins); fr(b->phase); fr(b->live); fr(b->bin_evan); fr(b->tw); fr(b->dft); fr(b->frames);
    fr(b->items); fr(b->counter);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->base) pam_destroy(b->base);
    delete b;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
}

// Bins of one frame: explicit (n_bins of them), or n_bins of the band's K bins
// spread evenly from the first to the last (index floor(i (K-1)/(n-1) + 1/2),
// in integers). A band with fewer than n_bins bins gives all K of them: short
// frames have coarser bin spacing fs / nt.
pam_status frame_bins(const pam_plan_desc *c, const pam_frame_desc &fd, int n_bins, std::vector<int> &out)
{
    out.clear();
    const int nt = fd.n_samples;
    if (fd.bins) {
        for (int i = 0; i < n_bins; ++i) {
            const int k = fd.bins[i];
            if (k <= 0 || 2 * k >= nt) return pam::fail(PAM_ERR_INVALID_ARG, "a frame bin is outside 0 < k < nt/2");
            if (i && k <= out.back()) return pam::fail(PAM_ERR_INVALID_ARG, "frame bins must increase strictly");
            out.push_back(k);
        }
        return PAM_OK;
    }
    const double df = c->fs_hz / nt;
    int k_lo = (int)std::ceil(c->f_lo_hz / df - 1e-9), k_hi = (int)std::floor(c->f_hi_hz / df + 1e-9);
    k_lo = std::max(k_lo, 1);
    k_hi = std::min(k_hi, (nt - 1) / 2);
    const long long K = (long long)k_hi - k_lo + 1;
    if (K < 1) return pam::fail(PAM_ERR_INVALID_ARG, "a frame's band holds no DFT bin");
    const int n = (int)std::min<long long>(K, n_bins);
    for (int i = 0; i < n; ++i) {
        const long long idx = n == 1 ? 0 : (2LL * i * (K - 1) + (n - 1)) / (2LL * (n - 1));
        out.push_back(k_lo + (int)idx);
    }
    return PAM_OK;
}

pam_status enqueue(pam_batch_s *b, const float *rf, float *image, float *rho_n, cudaStream_t st)
{
    pam_plan_s &p = *b->base;
    cudaError_t e = pam::launch_dft(b->cpl, rf, b->dft, b->bins, b->n_bins, b->ne, b->F, b->tw, p.w.S, b->max_nt, st);
    if (e != cudaSuccess) return pam::cuda_fail(e, "time DFT launch");
    e = pam::launch_lateral_frames(p, b->F, b->napq, p.t.apod, b->live, (size_t)b->n_bins * b->nx, st);
    if (e != cudaSuccess) return pam::cuda_fail(e, "lateral DFT launch");
    if ((e = cudaMemsetAsync(b->counter, 0, sizeof(int), st)) != cudaSuccess) return pam::cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(p.w.fmax, 0, sizeof(unsigned) * b->F, st)) != cudaSuccess)
        return pam::cuda_fail(e, "memset");
    pam::EpiOut out;
    out.eps = p.d.eps;
    out.npix = 0;
    out.out_main = image;
    out.rho_n = rho_n;
    out.rho_tmp = p.w.rho_tmp;
    out.e_tmp = p.w.e_tmp;
    out.fmax = p.w.fmax;
    out.status = p.w.status;
    const int grid = b->grid_override > 0 ? std::min(b->grid_override, b->n_items) : b->grid;
    e = pam::launch_prop_batch(b->nx, b->napq, grid, b->frames, b->items, b->n_items, b->counter, out, st, nullptr,
                               b->rpl);
    if (e != cudaSuccess) return pam::cuda_fail(e, "propagate/correlate launch");
    e = pam::launch_normalize_batch(b->F, b->max_npix, b->frames, out, st);
    if (e != cudaSuccess) return pam::cuda_fail(e, "normalise launch");
    b->kernels += 4;
    return PAM_OK;
}

}  // namespace

extern "C" {

pam_status pam_batch_create(const pam_plan_desc *common, const pam_frame_desc *fds, int n_frames, pam_batch_t *out)
{
    if (!out) return pam::fail(PAM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!common || !fds) return pam::fail(PAM_ERR_INVALID_ARG, "descriptor is NULL");
    if (n_frames < 1 || n_frames > 65535) return pam::fail(PAM_ERR_INVALID_ARG, "n_frames must be in [1, 65535]");
    if (common->n_apod != 2 && common->n_apod != 3)
        return pam::fail(PAM_ERR_INVALID_ARG, "batches are built for AS-DAX and AS-TAX (n_apod 2 or 3)");
    if (common->bins) return pam::fail(PAM_ERR_INVALID_ARG, "bins are given per frame in a batch");
    if (common->flags & ~PAM_EVANESCENT_ZERO)
        return pam::fail(PAM_ERR_UNSUPPORTED, "batches run the plain FP32 path (flags: PAM_EVANESCENT_ZERO only)");
    if (common->n_bins < 1 || common->n_bins > 8192) return pam::fail(PAM_ERR_INVALID_ARG, "n_bins must be in [1, 8192]");
    if (!(common->fs_hz > 0.0) || !std::isfinite(common->fs_hz))
        return pam::fail(PAM_ERR_INVALID_ARG, "fs_hz must be positive");
    pam_batch_s *b = new (std::nothrow) pam_batch_s();
    if (!b) return pam::fail(PAM_ERR_OOM, "host allocation");
    b->F = n_frames;
    b->n_bins = common->n_bins;
    b->napq = common->n_apod;
    std::vector<int> fb;
    int max_nz = 0;
    for (int f = 0; f < n_frames; ++f) {
        const pam_frame_desc &fd = fds[f];
        if (fd.n_samples < 32 || fd.n_samples > pam::DFT_MAX_NT) {
            delete b;
            return pam::fail(PAM_ERR_INVALID_ARG, "frame n_samples must be in [32, 16384]");
        }
        if (fd.nz < 1 || fd.nz > 65536) {
            delete b;
            return pam::fail(PAM_ERR_INVALID_ARG, "frame nz must be in [1, 65536]");
        }
        pam_status s = frame_bins(common, fd, b->n_bins, fb);
        if (s != PAM_OK) {
            delete b;
            return s;
        }
        b->nt.push_back(fd.n_samples);
        b->nz.push_back(fd.nz);
        b->nbf.push_back((int)fb.size());
        fb.resize(b->n_bins, 0);
        b->bins_h.insert(b->bins_h.end(), fb.begin(), fb.end());
        b->max_nt = std::max(b->max_nt, fd.n_samples);
        max_nz = std::max(max_nz, fd.nz);
    }
    // Base plan: the shared geometry, apodization and workspace. Its own bins
    // (1..n_bins at a power-of-2 length) only size the workspace.
    pam_plan_desc bd = *common;
    std::vector<int> dummy(b->n_bins);
    for (int i = 0; i < b->n_bins; ++i) dummy[i] = i + 1;
    int nt0 = 64;
    while (nt0 < 2 * b->n_bins + 2) nt0 *= 2;
    bd.n_samples = nt0;
    bd.bins = dummy.data();
    bd.nz = max_nz;
    bd.max_frames = n_frames;
    pam_status s = pam_plan_create(&bd, &b->base);
    if (s != PAM_OK) {
        delete b;
        return s;
    }
    pam_plan_s &p = *b->base;
    b->ne = p.ne;
    b->nx = p.nx;
    b->cpl = b->ne <= 32 ? 1 : b->ne <= 64 ? 2 : b->ne <= 128 ? 4 : 8;
    size_t tw_total = 0;
    std::vector<size_t> tw_off(n_frames);
    for (int f = 0; f < n_frames; ++f) {
        b->rf_off.push_back(b->rf_total);
        b->rf_total += pam::round4((size_t)b->ne * b->nt[f]);
        b->px_off.push_back(b->px_total);
        b->px_total += pam::round4((size_t)b->nz[f] * b->nx);
        b->max_npix = std::max(b->max_npix, b->nz[f] * b->nx);
        tw_off[f] = tw_total;
        tw_total += (size_t)b->nt[f];
    }
    // Two rows per lane on 12 warps where they fit (nx >= 64): 1.5x the work in
    // flight per SM, and row tiles of 1.5x the rows.
    b->rpl = b->nx >= 64 ? 2 : 1;
    const int rpc = pam::prop_rows_per_cta(b->nx, b->rpl);
    std::vector<int2> items;
    for (int f = 0; f < n_frames; ++f)
        for (int t = 0; t * rpc < b->nz[f]; ++t) items.push_back(make_int2(f, t));
    b->n_items = (int)items.size();
    b->grid = std::min(b->n_items, pam::prop_ctas_per_sm() * p.num_sms);
    const size_t FB = (size_t)n_frames * b->n_bins;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&b->bins, FB);
    if (e == cudaSuccess) e = dalloc(&b->phase, FB * b->nx);
    if (e == cudaSuccess) e = dalloc(&b->live, FB * b->nx);
    if (e == cudaSuccess) e = dalloc(&b->bin_evan, FB);
    if (e == cudaSuccess) e = dalloc(&b->tw, tw_total);
    if (e == cudaSuccess) e = dalloc(&b->dft, (size_t)n_frames);
    if (e == cudaSuccess) e = dalloc(&b->frames, (size_t)n_frames);
    if (e == cudaSuccess) e = dalloc(&b->items, items.size());
    if (e == cudaSuccess) e = dalloc(&b->counter, 1);
    if (e != cudaSuccess) {
        batch_free(b);
        return e == cudaErrorMemoryAllocation ? pam::fail(PAM_ERR_OOM, "device allocation")
                                              : pam::cuda_fail(e, "device allocation");
    }
    std::vector<pam::DftFrame> dh(n_frames);
    std::vector<pam::BatchFrame> fh(n_frames);
    for (int f = 0; f < n_frames; ++f) {
        dh[f].rf_off = b->rf_off[f];
        dh[f].tw_off = tw_off[f];
        dh[f].nt = b->nt[f];
        dh[f].n_bins = b->nbf[f];
        pam::BatchFrame &x = fh[f];
        x.Q = p.w.Q + (size_t)f * b->n_bins * pam::q_per_bin(b->napq, b->nx);
        x.phase = b->phase + (size_t)f * b->n_bins * b->nx;
        x.bin_evan = b->bin_evan + (size_t)f * b->n_bins;
        x.n_bins = b->nbf[f];
        x.nz = b->nz[f];
        x.nx = b->nx;
        x.nt = b->nt[f];
        x.z0f = (float)p.d.z0_m;
        x.dzf = (float)p.d.dz_m;
        x.out_off = b->px_off[f];
    }
    e = cudaMemcpy(b->bins, b->bins_h.data(), sizeof(int) * FB, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->dft, dh.data(), sizeof(pam::DftFrame) * n_frames, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->frames, fh.data(), sizeof(pam::BatchFrame) * n_frames, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
    for (int f = 0; f < n_frames && e == cudaSuccess; ++f)
        e = pam::launch_tables_frame(p, b->bins + (size_t)f * b->n_bins, b->nbf[f], b->nt[f],
                                     b->phase + (size_t)f * b->n_bins * b->nx, b->live + (size_t)f * b->n_bins * b->nx,
                                     b->bin_evan + (size_t)f * b->n_bins, b->tw + tw_off[f], 0);
    if (e == cudaSuccess) e = pam::prepare_dft();
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_free(b);
        return pam::cuda_fail(e, "batch tables");
    }
    *out = b;
    return PAM_OK;
}

void pam_batch_destroy(pam_batch_t b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_free(b);
}

pam_status pam_batch_layout(pam_batch_t b, size_t *rf_offsets, size_t *map_offsets, size_t *rf_total,
                            size_t *map_total)
{
    if (!b) return pam::fail(PAM_ERR_INVALID_ARG, "batch is NULL");
    for (int f = 0; f < b->F; ++f) {
        if (rf_offsets) rf_offsets[f] = b->rf_off[f];
        if (map_offsets) map_offsets[f] = b->px_off[f];
    }
    if (rf_total) *rf_total = b->rf_total;
    if (map_total) *map_total = b->px_total;
    return PAM_OK;
}

int pam_batch_bins(pam_batch_t b, int frame, int *bins_out)
{
    if (!b || frame < 0 || frame >= b->F) return 0;
    if (bins_out)
        std::memcpy(bins_out, b->bins_h.data() + (size_t)frame * b->n_bins, sizeof(int) * (size_t)b->nbf[frame]);
    return b->nbf[frame];
}

pam_status pam_batch_as_tax(pam_batch_t b, const float *rf, float *image, float *rho_n, void *stream)
{
    pam::TraceRange trace_("pam_batch_as_tax");
    if (!b) return pam::fail(PAM_ERR_INVALID_ARG, "batch is NULL");
    pam_status s;
    if ((s = pam::check_dev(rf, "rf", true)) != PAM_OK) return s;
    if ((s = pam::check_dev(image, "image", true)) != PAM_OK) return s;
    if ((s = pam::check_dev(rho_n, "rho_n", false)) != PAM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!b->use_graph) return enqueue(b, rf, image, rho_n, st);
    const int grid = b->grid_override > 0 ? b->grid_override : b->grid;
    if (!b->exec || b->g_rf != rf || b->g_img != image || b->g_rho != rho_n || b->g_grid != grid) {
        // capture the call's launches on the batch's own stream, then replay on the caller's
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pam::cuda_fail(e, "graph capture");
        const long long k0 = b->kernels;
        s = enqueue(b, rf, image, rho_n, b->cap);
        b->kernels = k0;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->cap, &g);
        if (s != PAM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return pam::cuda_fail(e, "graph capture");
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return pam::cuda_fail(e, "graph instantiate");
        }
        b->g_rf = rf;
        b->g_img = image;
        b->g_rho = rho_n;
        b->g_grid = grid;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return pam::cuda_fail(e, "graph launch");
    b->kernels += 4;
    return PAM_OK;
}

pam_status pam_batch_sync(pam_batch_t b, void *stream)
{
    if (!b) return pam::fail(PAM_ERR_INVALID_ARG, "batch is NULL");
    return pam_sync(b->base, stream);
}

pam_status pam_batch_configure(pam_batch_t b, int use_graph, int persistent_ctas)
{
    if (!b) return pam::fail(PAM_ERR_INVALID_ARG, "batch is NULL");
    if (persistent_ctas < 0) return pam::fail(PAM_ERR_INVALID_ARG, "persistent_ctas must be >= 0");
    b->use_graph = use_graph != 0;
    b->grid_override = persistent_ctas;
    return PAM_OK;
}

pam_status pam_batch_info(pam_batch_t b, int *n_items, int *persistent_ctas, long long *kernel_launches)
{
    if (!b) return pam::fail(PAM_ERR_INVALID_ARG, "batch is NULL");
    if (n_items) *n_items = b->n_items;
    if (persistent_ctas) *persistent_ctas = b->grid_override > 0 ? std::min(b->grid_override, b->n_items) : b->grid;
    if (kernel_launches) *kernel_launches = b->kernels;
    return PAM_OK;
}

}  // extern "C"
