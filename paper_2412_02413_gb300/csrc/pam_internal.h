// pam_internal.h -- plan object and kernel launchers shared by the libpam
// translation units. Not part of the public ABI (that is include/pam.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pam.h"

namespace pam {

// Frames per CTA of the tensor-core form (N = 2 * frames GEMM columns).
constexpr int kFramesPerGroup = 32;
constexpr int kMaxGemmK = 384;     // GEMM depth of the tensor-core form: 16 per (aperture, 8-element block)

// Rows of the depth grid handled by one CTA of the fused propagate-and-correlate
// kernel for a lateral length nx (2*nx/16 lanes per row) and rpl depth rows per
// lane (1: 16 warps; 2: 12 warps for nx >= 64, 8 below).
int prop_ctas_per_sm();   // resident CTAs per SM of the fused kernels (their register limit)
int prop_rows_per_cta(int nx, int rpl = 1);

// Bin splits up to this size reduce inside a thread-block cluster (portable limit).
constexpr int kMaxClusterSplit = 8;

// Complex entries of the staged spectra per (frame, bin): the fused kernel's
// paired layout holds every aperture's nx values twice, once per half of its
// radix-2 split (see lateral_kernel).
inline size_t q_per_bin(int napq, int nx) { return (size_t)2 * napq * nx; }

// Destination of the per-pixel epilogue (maps of one call, [F][nz][nx]).
struct EpiOut {
    float eps = 1e-3f;
    int npix = 0;                 // nz * nx
    float *out_main = nullptr;    // AS energy (n_apod 1) or the final image (DAX / TAX)
    float *rho_n = nullptr;       // optional
    float *rho_pairs = nullptr;   // optional, [F][n_pairs][nz][nx]
    float *image_as = nullptr;    // optional
    float *rho_tmp = nullptr;     // workspace: rho before normalisation
    float *e_tmp = nullptr;       // workspace: coherent energy
    unsigned *fmax = nullptr;     // workspace: per-frame max of rho
    int *status = nullptr;        // device status word (set on an expired bounded wait)
};

// Accumulators per pixel: |p1|^2 (AS), + |p2|^2, Re p1*p2 (DAX),
// + |p3|^2, Re p2*p3, Re p3*p1 (TAX).
inline int n_acc(int n_apod) { return n_apod == 1 ? 1 : (n_apod == 2 ? 3 : 6); }

// One frame of a batch (pam_batch_*): its spectra, phase table and geometry,
// and the offset of its [nz][nx] maps in the packed outputs.
struct BatchFrame {
    const float2 *Q;        // [n_bins][napq][nx]
    const uint4 *phase;     // [n_bins][nx]
    const int *bin_evan;    // [n_bins]
    int n_bins, nz, nx, nt;
    float z0f, dzf;
    size_t out_off;         // pixel offset of the frame's maps
};

struct Workspace {
    float2 *S = nullptr;        // [max_frames][n_bins][n_elem]      selected time bins
    float2 *Q = nullptr;        // [max_frames][n_bins][napq][nx]    apodized lateral spectra / nx
    float *part = nullptr;      // [units][n_acc][nz][nx]            per-split accumulator partials
    size_t part_units = 0;
    float *rho_tmp = nullptr;   // [max_frames][nz][nx]              rho before normalisation
    float *e_tmp = nullptr;     // [max_frames][nz][nx]              sum_k |sum_q p_q|^2
    unsigned *fmax = nullptr;   // [max_frames]                      max rho bits per frame
    int *status = nullptr;      // device status word
    // tensor-core form: packed S operand tiles and the per-frame power-of-2 scale
    uint4 *Bhi = nullptr, *Blo = nullptr;   // [groups][n_bins][K * 2 * kFramesPerGroup * 2 bytes]
    unsigned *smax = nullptr;               // [max_frames] max |Re S|, |Im S| bits
    // host-buffer entry point staging (allocated on first use)
    float *rf_stage = nullptr, *img_stage = nullptr, *rho_stage = nullptr;
    // PAM_LATERAL_PAD2X: full-width maps before the crop, [max_frames][npix] each
    // (pad_pairs: [max_frames][pairs][npix]; only pad_img for n_apod == 1)
    float *pad_img = nullptr, *pad_rho = nullptr, *pad_as = nullptr, *pad_pairs = nullptr;
};

struct Tables {
    int *bins = nullptr;          // [n_bins]
    float *apod = nullptr;        // [n_apod][n_elem]
    float *ones = nullptr;        // [n_elem]
    float2 *tw_t = nullptr;       // [nt]   exp(-2 pi i m / nt)
    float2 *tw_x = nullptr;       // [nx]   exp(-2 pi i m / nx)
    // [n_bins][nx] per lateral bin u: {anchor_hi, step_hi, step_lo, ecoef bits}. The phase of row j,
    // in turns * 2^32, is anchor_hi + j*step_hi + hi32(j*step_lo) (mod 2^32): the top word of the
    // 64-bit fixed-point accumulator anchor + j*step. ecoef = -kappa*log2(e) for evanescent
    // components (amplitude exp2(ecoef*z)), 0 otherwise.
    uint4 *phase = nullptr;
    float *live = nullptr;        // [n_bins][nx] 1, or 0 for dropped evanescent components
    // tensor-core form: per (bin, depth row) the propagator point-spread c_j[d], d < nx,
    // as packed 16-bit (re, im) pairs; hi part and the rounding residual (lo)
    uint32_t *c_hi = nullptr;     // [n_bins][nz][nx]
    uint32_t *c_lo = nullptr;     // [n_bins][nz][nx] (split form only)
    short *ktab = nullptr;        // [K] element of each K column, +0x4000 for the imaginary half, -1 = pad
    float *kwgt = nullptr;        // [K] apodization weight of that element
    int *bin_evan = nullptr;      // [n_bins] 1 if any live evanescent component in the bin
};

}  // namespace pam

struct pam_plan_s {
    pam_plan_desc d{};
    int device = 0, num_sms = 0;
    int ne = 0, nt = 0, log2nt = 0, nx = 0, nz = 0, n_bins = 0, n_apod = 0, max_frames = 1;
    int nev = 0;                       // channels of S and of the lateral DFT: ne, or 2 ne (stuffed or padded)
    int chan_step = 1;                 // element e sits on channel chan_step * e of S (2 when zero-stuffed)
    int nx_out = 0;                    // image columns: nx, or ne when the lateral DFTs run padded to 2 ne
    double pitch_x = 0.0;              // channel spacing: pitch, or pitch / 2
    std::vector<int> bins;
    std::vector<float> apod;
    pam::Tables t;
    pam::Workspace w;
    // measurement hooks (pam_profile_*)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;  // pairs around propagate-and-correlate launches
    size_t prof_used = 0;              // events recorded since the last read
    long long kernels = 0;             // libpam kernel launches since the last read
    int split_override = 0;            // pam_plan_set_split (0 = automatic)
    int grid_override = 0;             // pam_plan_set_grid (0 = every SM)
    int fft_radix = 8;                 // pam_plan_set_fft_radix: largest radix of the time FFT's stages (4 or 8)
    int lane_rows = 2;                 // pam_plan_set_lane_rows: depth rows per lane of the fused kernel (1 or 2)
    int gemm_m = 128;                  // pam_plan_set_gemm_tile: M of the tensor-core form's MMA (128 or 256)
    int gemm_frames = 32;              // pam_plan_set_gemm_frames: frames per CTA of the tensor-core form (32 or 16)
    bool seg_ok = false;               // Workspace::part holds prop_seg_part_floats (even division of small batches)
    // tensor-core form (PAM_FORM_GEMM_*): 0 = plain FP32 path
    int form = 0;
    int K = 0;                         // GEMM depth: 16 per (aperture, 8-element block) pair
    int kq[4] = {0, 0, 0, 0};          // K range of aperture q: [kq[q], kq[q+1])
    std::vector<short> ktab_h;         // host copies of Tables::ktab / kwgt
    std::vector<float> kwgt_h;
};

namespace pam {

// Launchers (all asynchronous on `st`). Each returns cudaGetLastError().
cudaError_t launch_tables(const pam_plan_s &p, cudaStream_t st);
cudaError_t launch_time_fft(const pam_plan_s &p, const float *rf, int n_frames, cudaStream_t st);
cudaError_t launch_lateral(const pam_plan_s &p, int n_frames, int napq, const float *apod, cudaStream_t st);
// Per-frame masks (live + f * live_fs) and per-frame plan tables for batches.
cudaError_t launch_lateral_frames(const pam_plan_s &p, int n_frames, int napq, const float *apod,
                                  const float *live, size_t live_fs, cudaStream_t st);
cudaError_t launch_tables_frame(const pam_plan_s &p, const int *bins, int n_bins, int nt, uint4 *phase, float *live,
                                int *bin_evan, float2 *tw_t, cudaStream_t st);
// The fused propagate-and-correlate kernel. With n_split <= kMaxClusterSplit
// it runs as clusters and also writes the per-pixel epilogue into `out`.
cudaError_t launch_prop(const pam_plan_s &p, int n_frames, int napq, int n_split, float *fields,
                        const EpiOut &out, cudaStream_t st);
// The rest of the epilogue: the partial reduction (no cluster) and the rho
// normalisation (DAX / TAX).
cudaError_t launch_epilogue(const pam_plan_s &p, int n_frames, int napq, int n_split, const EpiOut &out,
                            cudaStream_t st, bool from_partials = false, bool fields = false);
int epilogue_kernels(const pam_plan_s &p, int napq, int n_split, bool fields = false);   // kernels launch_epilogue launches
// Even division (automatic split, no fields, plan memory for the segment
// sums): one wave of prop_seg_ctas CTAs over the linearized (frame, tile, bin)
// sequence; the sums of split tiles need prop_seg_part_floats floats of
// Workspace::part, whatever the number of frames. n_split is then unused.
bool prop_seg_mode(const pam_plan_s &p, int n_split, bool fields);
int prop_seg_ctas(const pam_plan_s &p, int n_frames);
size_t prop_seg_part_floats(const pam_plan_s &p);
// Batch (pam_batch.cu): the persistent propagate-and-correlate kernel over
// (frame, row tile) items and the per-frame normalisation.
// n_items_dev (optional): a device int that caps n_items when the kernel starts.
// rpl: depth rows per lane; the items' row tiles are prop_rows_per_cta(nx, rpl) rows.
cudaError_t launch_prop_batch(int nx, int napq, int grid, const BatchFrame *frames, const int2 *items, int n_items,
                              int *counter, const EpiOut &out, cudaStream_t st, const int *n_items_dev = nullptr,
                              int rpl = 1);
// Full-aperture energy split by bins: the fused kernel (one aperture, whatever
// Q holds) over n_bands contiguous chunks of Omega, chunk b = bins
// [floor(n_bins b / n_bands), floor(n_bins (b+1) / n_bands)), each chunk's
// per-pixel sum written to bands[f][b][nz][nx] (no reduction).
cudaError_t launch_prop_bands(const pam_plan_s &p, int n_frames, int n_bands, float *bands, cudaStream_t st);
cudaError_t launch_normalize_batch(int n_frames, int max_npix, const BatchFrame *frames, const EpiOut &out,
                                   cudaStream_t st);
bool prop_uses_cluster(int n_split);
// A kernel whose bounded mbarrier wait never completes (failure-path test).
cudaError_t launch_expire_wait(int *status, cudaStream_t st);

// PAM_LATERAL_PAD2X crop: columns [0, nx_out) of the full-width maps (row
// width nx) of n_frames frames. rho_n is renormalised to its maximum over the
// crop and the image rebuilt as rho_n^2 E from the full-aperture energy E.
// Outputs other than image may be NULL.
cudaError_t launch_pad_crop(const float *rho_full, const float *e_full, const float *pairs_full, int n_pairs,
                            int n_frames, int nz, int nx, int nx_out, float *image, float *rho_n, float *pairs,
                            float *image_as, cudaStream_t st);

// Host-side fault injection for tests: true when the environment variable
// PAM_FAULT names `what` ("alloc": plan allocation fails part way).
bool fault_injected(const char *what);

// NVTX range over one public call (a no-op unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
cudaError_t prepare_kernels(const pam_plan_s &p);

// Tensor-core form (pam_prec.cu): plan-time point-spread table, and the per-call
// operand packing + GEMM whose per-pixel sums feed launch_epilogue (split 1).
cudaError_t launch_prec_tables(const pam_plan_s &p, cudaStream_t st);
cudaError_t launch_prec(const pam_plan_s &p, int n_frames, cudaStream_t st);
cudaError_t prepare_prec_kernels();
int prec_kernels();   // kernels launch_prec launches
// Tensor-core form, band energies: from spectra S [F][n_bins][n_elem] (any
// plan's, same bins), the full-aperture energy sum_k |p_1 + p_2 + p_3|^2 of each
// contiguous chunk of Omega (chunks as launch_prop_bands) into bands[f][b][nz][nx].
// 3 kernels. The plan must be a BF16 or FP16 form with n_apod 3.
cudaError_t launch_prec_bands(const pam_plan_s &p, const float2 *S, int n_frames, int n_bands, float *bands,
                              cudaStream_t st);

// Records `msg` as the calling thread's pam_last_error() text and returns s.
pam_status set_error(pam_status s, const char *msg);
int choose_split(const pam_plan_s &p, int n_frames);

// Descriptor checks shared by pam_plan_create and pam_as_tax_static, writing
// only to caller-provided fixed arrays (no allocation). kMaxBins bounds every
// valid bin list: bins are strictly increasing in (0, n_samples/2) and
// n_samples <= 8192.
constexpr int kMaxBins = 4096;
// Ranges of the geometry fields common to every entry point: n_elem, pitch,
// fs, c, n_samples (a power of two in [64, 8192]), nz, z0, dz and eps.
pam_status check_desc_ranges(const pam_plan_desc *d);
// The bins of Omega (Sec. II-E band, or the explicit list) into bins[kMaxBins];
// *n_out gets their count.
pam_status desc_bins(const pam_plan_desc *d, int *bins, int *n_out);
// The n_apod apodizations (explicit, or Pattern-m of Sec. II-A/C) into
// apod[n_apod * n_elem].
pam_status desc_apod(const pam_plan_desc *d, int n_apod, float *apod);

}  // namespace pam
