/*
 * pam.h -- C ABI of libpam, GB300 (sm_103a) angular-spectrum passive acoustic
 * mapping with cross-correlated apodizations: AS, AS-DAX and AS-TAX
 * (arXiv 2412.02413).
 *
 * Every computational step runs in this library's CUDA kernels. The
 * signatures carry only plain pointers, sizes and an opaque stream handle.
 *
 * Problem statement (paper notation)
 *   rf p(x_e, z0=0, t): float32 [n_frames][n_elem][n_samples], channel-major.
 *       Element e sits at x_e = (e - (n_elem-1)/2) * pitch_m. The array face is
 *       the plane z = 0 and its centre is the origin (Fig. 1(a)).
 *   Omega: the selected DFT bins k, with w_k = 2 pi k fs / n_samples (Eq. 3).
 *   Eq. 1: P(kx, 0, w) = F_x{F_t{p}}. The forward transforms use exp(-i w t)
 *       and exp(-i kx x) and are unnormalised. kx_u = 2 pi u' / (nx * pitch)
 *       with u' = u for u < nx/2, else u - nx.
 *   Eq. 2: P(kx, z, w) = P(kx, 0, w) exp(i z sqrt(w^2/c^2 - kx^2)), principal
 *       branch. Evanescent components decay as exp(-kappa z), unless
 *       PAM_EVANESCENT_ZERO drops them.
 *   Fields: p~_q(x_i, z_j, w_k) = (1/nx) sum_u P_q exp(+2 pi i u i / nx).
 *       Pixel column i is element position x_i (nx == n_elem). Row j is at
 *       depth z_j = z0_m + j * dz_m.
 *   Eq. 3: I_AS(r) = sum_k |p~(r, w_k)|^2.
 *   Eq. 4 + Appendix A: rho_qr = Re sum_k conj(p~_q) p~_r /
 *       sqrt(sum_k |p~_q|^2 * sum_k |p~_r|^2), clamped below at eps (Sec. II-A).
 *       A zero denominator gives eps.
 *   Eq. 10: rho_TAX = cbrt(rho_12 * rho_23 * rho_31).
 *       rho_n = rho / max over the frame's pixels.
 *   Eq. 5 / Eq. 11: I = rho_n^2 * sum_k |sum_q p~_q|^2.
 *
 * Conventions of every entry point
 *   - Device buffers belong to the caller. They must be device memory that the
 *     current device can access, and 16-byte aligned; otherwise the call
 *     returns PAM_ERR_INVALID_ARG.
 *   - Output maps are float32 [n_frames][nz][nx], row-major (row = depth).
 *   - Work is queued asynchronously on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream). A returned status reports validation and launch
 *     errors. Errors raised later on the device, such as a bounded wait that
 *     timed out, are reported by pam_sync() or by the next call.
 *   - A plan is not thread-safe: calls on one plan must not overlap. No call
 *     aborts the process. pam_last_error() gives the message of the calling
 *     thread's last failure.
 *   - The public calls are NVTX ranges named after the call (visible under
 *     nsys / ncu; free when no tool is attached).
 *   - Fault injection for tests (host side), by the environment variable
 *     PAM_FAULT: "alloc" makes pam_plan_create fail with PAM_ERR_OOM part way
 *     through its allocations (it frees what it allocated); "launch" makes
 *     pam_as_backprop, pam_as_dax, pam_as_tax and the host-buffer entry points
 *     return PAM_ERR_CUDA before they queue any work.
 */
#ifndef PAM_H
#define PAM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pam_plan_s *pam_plan_t;

typedef enum {
    PAM_OK = 0,
    PAM_ERR_INVALID_ARG = 1, /* a pointer, size or descriptor field is out of range */
    PAM_ERR_UNSUPPORTED = 2, /* valid for the method, not built here (e.g. nt not a power of 2) */
    PAM_ERR_OOM = 3,         /* a device or host allocation failed */
    PAM_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    PAM_ERR_TIMEOUT = 5,     /* a kernel's bounded wait expired (device status word) */
    PAM_ERR_NUMERIC = 6      /* non-finite input detected */
} pam_status;

/* descriptor flags */
#define PAM_EVANESCENT_ZERO 0x1u /* drop components with kx^2 > (w/c)^2 instead of decaying them */
/* 2x zero-stuffing in the channel direction before apodization and the lateral
 * transform (Sec. II-D): a virtual array of 2 n_elem channels at pitch/2 whose
 * channel 2e carries element e and channel 2e+1 is zero. Virtual channel v sits
 * at x_v = (v - (2 n_elem - 1)/2) pitch/2 and is image column v, so nx = 2 n_elem
 * (built: n_elem 8..64) and the pixel pitch is pitch/2. Apodizations stay per
 * physical element (explicit or Pattern-m on the element index). Plain FP32
 * path only: not with PAM_FORM_GEMM_*, batches, the learned form or
 * pam_as_tax_static. */
#define PAM_LATERAL_UPSAMPLE2X 0x2u
/* 2x padding in the channel direction (Sec. II-D, the other reading of its
 * "2x" lateral extension): n_elem zero channels are appended after the last
 * element, the lateral transforms of Eq. 1-2 run over 2 n_elem points at the
 * element pitch (so the circular wrap-around of an n_elem-point transform is
 * gone), and every map is cropped back to the n_elem element columns: nx =
 * n_elem (built: n_elem 8..64). rho_n is normalised to its maximum over the
 * cropped image and I = rho_n^2 E_full there (Eq. 11). Plain FP32 path only,
 * like PAM_LATERAL_UPSAMPLE2X (not both), and without the `fields` output. */
#define PAM_LATERAL_PAD2X 0x4u
/* Tensor-core form of the propagation (at most one of these; default = plain FP32 FFT path).
 * For a bin w_k and depth row z_j, the element-to-pixel propagator of Eq. 1-2 is circulant:
 *   p~(x_i, z_j) = sum_e c_j[(i - e) mod nx] a_q[e] S[e],
 *   c_j[d] = (1/nx) sum_u exp(i kz_u z_j) exp(+2 pi i u d / nx).
 * The plan tabulates c_j (from the FP64 phase words) in 16-bit form. Each call runs the
 * sum over elements as a tcgen05 GEMM [pixels x elements] x [elements x frames], with FP32
 * accumulation in tensor memory. The three apodizations are disjoint K-slices of one GEMM.
 * Requirements: nx == 128, n_apod 2 or 3, apertures with disjoint element sets.
 * Typical relative L2 error of I_TAX against the FP64 oracle at 128 elements, 300 bins:
 * BF16 about 5e-4, FP16 about 6e-5, BF16 split about 2e-6, FP16 split about 1e-6 (the
 * FP16 split also keeps every NCC map within 1e-5 of the oracle, as the FP32 path does). */
#define PAM_FORM_GEMM_BF16 0x10u       /* BF16 operands */
#define PAM_FORM_GEMM_FP16 0x20u       /* FP16 operands (frames scaled by a power of 2) */
#define PAM_FORM_GEMM_BF16_SPLIT 0x40u /* BF16 hi + lo split: hi*hi + hi*lo + lo*hi */
#define PAM_FORM_GEMM_FP16_SPLIT 0x80u /* FP16 hi + lo split (frames scaled by a power of 2): 22 significant bits */

/* Acquisition and imaging geometry (Sec. II-A, Fig. 1; band selection Sec. II-D). */
typedef struct {
    int n_elem;           /* elements / channels, 8..256 */
    double pitch_m;       /* element pitch (m), > 0 */
    double fs_hz;         /* sampling rate (Hz), > 0 */
    double c_mps;         /* sound speed (m/s), > 0 */
    int n_samples;        /* samples per channel nt: a power of two, 64..8192 */
    int nx;               /* lateral pixels: 0 or n_elem (2 n_elem with PAM_LATERAL_UPSAMPLE2X).
                             The lateral DFT length is nx, or 2 n_elem with PAM_LATERAL_PAD2X.
                             Built lateral lengths: 16, 32, 64, 128 */
    int nz;               /* depth rows, 1..65535 */
    double z0_m;          /* depth of row 0 from the array face (m), >= 0 */
    double dz_m;          /* row spacing (m), > 0 */
    double f_lo_hz;       /* band used when bins == NULL: all k with f_lo <= k*fs/nt <= f_hi */
    double f_hi_hz;
    const int *bins;      /* host, explicit Omega: strictly increasing, 0 < k < nt/2; or NULL */
    int n_bins;           /* entries in bins (ignored when bins == NULL); 1..8192 */
    int n_apod;           /* 1 (AS), 2 (AS-DAX) or 3 (AS-TAX) */
    const float *apod;    /* host [n_apod][n_elem] real weights, or NULL for Pattern-m */
    int pattern_m;        /* Pattern-m (Sec. II-A): element e in aperture q iff floor(e/m) mod n_apod == q */
    float eps;            /* NCC floor (Sec. II-A, usually 0.001), 0 < eps <= 1 */
    unsigned flags;       /* PAM_EVANESCENT_ZERO, PAM_LATERAL_UPSAMPLE2X or PAM_LATERAL_PAD2X,
                             at most one PAM_FORM_GEMM_* */
    int max_frames;       /* frames per kernel batch; larger calls run in batches of this size */
} pam_plan_desc;

/* Fills `d` with defaults: nx = 0, n_apod = 3, pattern_m = 16, eps = 1e-3,
 * flags = 0, max_frames = 1, bins = apod = NULL. Geometry fields are zeroed. */
void pam_plan_desc_init(pam_plan_desc *d);

/* Builds a plan on the current CUDA device (the paper's "pre-run", Sec. II-E,
 * Table III). It validates `d` and copies it, together with the bins and the
 * apodizations. It then runs the FP64 table kernel, which computes kz
 * (Eq. 2) and the fixed-point phase words, and allocates the workspace for
 * max_frames frames. The call blocks until the tables are built. On failure
 * *out is set to NULL and nothing is left allocated. */
pam_status pam_plan_create(const pam_plan_desc *d, pam_plan_t *out);

/* Releases everything the plan owns. NULL-safe. It synchronises with the
 * plan's outstanding work first. */
void pam_destroy(pam_plan_t p);

/* Number of bins in Omega. When bins_out != NULL, also copies them there
 * (host, n_bins ints). */
int pam_plan_bins(pam_plan_t p, int *bins_out);

/* Copies the plan's apodizations to host memory [n_apod][n_elem]. Returns n_apod. */
int pam_plan_apod(pam_plan_t p, float *apod_out);

/* Pins the number of bin chunks that the fused propagate-and-correlate
 * kernel splits Omega into for one row tile: 0 = automatic (the even
 * division described at pam_plan_set_grid), n >= 1 = n chunks, capped at
 * n_bins and at what the workspace holds. Splits of up to 8 are reduced on chip inside a thread-block cluster,
 * larger ones through global partial sums. Results are deterministic for a
 * given split. Different splits round differently, by the order of the sums
 * over bins. */
pam_status pam_plan_set_split(pam_plan_t p, int n_split);

/* Number of CTAs of the fused propagate-and-correlate kernel when the split
 * is automatic (pam_plan_set_split(p, 0)): the launch is one wave of one CTA
 * per SM, each taking an equal contiguous share of the (frame, row tile, bin)
 * work. n_ctas = 0 uses every SM; 1 <= n_ctas < the SM count leaves SMs free
 * for kernels of other streams (several plans on several streams). Errors:
 * PAM_ERR_INVALID_ARG for n_ctas < 0. Larger values are capped at the SM
 * count. Different counts divide the sums over bins differently, so results
 * differ at the rounding level. */
pam_status pam_plan_set_grid(pam_plan_t p, int n_ctas);

/* Largest radix of the stages of the time FFT (Eq. 1, F_t): 8 (the default:
 * radix-8 stages while they fit, then radix 4 and 2) or 4 (radix-4 stages,
 * then radix 2). Fewer stages mean fewer passes through shared memory; the
 * two round differently. PAM_ERR_INVALID_ARG for other values. */
pam_status pam_plan_set_fft_radix(pam_plan_t p, int radix);

/* Depth rows per lane of the plain path's fused kernel when it takes the
 * whole (frame, row tile, bin) sequence in one wave (the default split): 1
 * (16 warps per CTA) or 2 (the default; each lane computing two rows of the same pixels,
 * so that each load of the staged spectra and phase words serves both; 12
 * warps for nx >= 64, which hold 1.5x the work in flight and cover 1.5x the
 * rows per CTA, and 8 warps below). The arithmetic of a row is the same
 * either way. For nx >= 64 the larger row tiles divide the bins among the
 * CTAs differently, so the sums are grouped differently and the maps agree to
 * rounding; with one CTA (pam_plan_set_grid(p, 1)) or nx < 64 they are
 * bit-identical. PAM_ERR_INVALID_ARG for other values. */
pam_status pam_plan_set_lane_rows(pam_plan_t p, int rows);

/* M tile of the tensor-core form's MMAs (PAM_FORM_GEMM_*; no effect on the
 * plain path): 128 (the default) runs one CTA per depth row; 256 runs each
 * pair of rows on a 2-CTA cluster whose MMAs (tcgen05 cta_group::2) compute
 * both rows at once, so that each SM stages and reads half of the spectra
 * operand, while the pair's even CTA issues every MMA. Results are identical
 * (the same products summed in the same order). PAM_ERR_INVALID_ARG for other
 * values. */
pam_status pam_plan_set_gemm_tile(pam_plan_t p, int m);

/* Frames per CTA of the tensor-core form (PAM_FORM_GEMM_*): 32 (the default;
 * the MMA's N = 64 columns hold Re and Im of 32 frames) or 16 (N = 32). A
 * call's frames are processed in groups of this size; with 16, a call of 16
 * frames or fewer does no MMA work for absent frames, and each MMA reads half
 * the spectra operand for the same circulant operand. Results are identical.
 * PAM_ERR_INVALID_ARG for other values. */
pam_status pam_plan_set_gemm_frames(pam_plan_t p, int frames);

/* AS back-propagation energy map, Eq. 3, for one apodization.
 *   rf          device float32 [n_frames][n_elem][n_samples]
 *   apod_index  -1 = full aperture (all ones); 0..n_apod-1 = plan aperture q
 *   energy      device float32 [n_frames][nz][nx]
 *   fields      device complex64 as interleaved float pairs
 *               [n_frames][n_bins][nz][nx][2], or NULL. This is a debug and test
 *               output: it writes every monochromatic field p~(x_i, z_j, w_k)
 *               to memory. PAM_ERR_UNSUPPORTED with PAM_LATERAL_PAD2X.
 *   stream      cudaStream_t or NULL */
pam_status pam_as_backprop(pam_plan_t p, const float *rf, int n_frames, int apod_index,
                           float *energy, float *fields, void *stream);

/* AS-TAX (Eq. 4, 10, 11). The plan must have n_apod == 3.
 *   image_tax   device [n_frames][nz][nx]  I = rho_n^2 * sum_k |p~_1 + p~_2 + p~_3|^2
 *   rho_n       device [n_frames][nz][nx] or NULL (normalised rho_TAX)
 *   rho_pairs   device [n_frames][3][nz][nx] or NULL (rho_12, rho_23, rho_31 after the clamp)
 *   image_as    device [n_frames][nz][nx] or NULL (sum_k |p~_1 + p~_2 + p~_3|^2; the AS
 *               image of Eq. 3 when the apodizations sum to one) */
pam_status pam_as_tax(pam_plan_t p, const float *rf, int n_frames, float *image_tax,
                      float *rho_n, float *rho_pairs, float *image_as, void *stream);

/* AS-DAX (Eq. 4-5). The plan must have n_apod == 2. rho_pair is
 * [n_frames][nz][nx] or NULL. */
pam_status pam_as_dax(pam_plan_t p, const float *rf, int n_frames, float *image_dax,
                      float *rho_n, float *rho_pair, float *image_as, void *stream);

/* AS-TAX (n_apod == 3) or AS-DAX (n_apod == 2) from HOST memory. rf_host
 * [n_frames][n_elem][n_samples], image_host and rho_n_host (or NULL)
 * [n_frames][nz][nx]. The copies run on `stream` through plan-owned device
 * staging buffers, which the first call allocates. The call returns after the
 * results are in host memory. Pinned host buffers make the copies faster. */
pam_status pam_as_xcorr_host(pam_plan_t p, const float *rf_host, int n_frames,
                             float *image_host, float *rho_n_host, void *stream);

/* As pam_as_xcorr_host, but returns once the upload, the kernels and the
 * downloads are queued on `stream`: the results are in host memory when the
 * stream reaches that point (cudaStreamSynchronize, an event, or pam_sync).
 * The host buffers must stay valid and unmodified until then; with pageable
 * (not pinned) buffers the copies may block. Calls on one plan share its
 * staging buffers, so they must be ordered on one stream; to overlap the
 * copies of one frame with the kernels of another, use one plan per stream. */
pam_status pam_as_xcorr_host_async(pam_plan_t p, const float *rf_host, int n_frames, float *image_host,
                                   float *rho_n_host, void *stream);

/* Size of the device array that pam_as_tax_static works in. It is part of the
 * library image on every GPU that loads the library. */
#define PAM_STATIC_SCRATCH_BYTES (16u << 20)

/* AS-TAX (as pam_as_tax) without allocating any memory, for callers that
 * cannot allocate GPU memory: code running inside a host framework that owns
 * every device allocation, real-time loops with a fixed memory footprint, or
 * plug-ins that must not bypass their process's allocator. Such callers
 * cannot create a plan, because pam_plan_create calls cudaMalloc. The paper
 * has no counterpart; this is an interface for deployment.
 *   d          geometry as for pam_plan_create; n_apod must be 3. max_frames is
 *              ignored: frames run one after another.
 *   rf         device float32 [n_frames][n_elem][n_samples]
 *   image_tax  device [n_frames][nz][nx]; rho_n device [n_frames][nz][nx] or NULL
 * The plan tables and the workspace live in one static device array of
 * PAM_STATIC_SCRATCH_BYTES. A geometry that needs more (for example a very
 * large nz * nx or n_bins) is rejected with PAM_ERR_INVALID_ARG and a message
 * that gives the size it needs. The first call on a device sets that device
 * up: it looks up the array's device address and sets kernel attributes.
 * Every call shares the one array and leaves its contents behind: calls that
 * overlap on the GPU (concurrent streams or host threads on the same device)
 * race and must be serialised by the caller. The call calls no cudaMalloc,
 * cudaFree or other allocating routine.
 * Every call uploads the bins and apodizations by cudaMemcpyAsync from
 * pageable stack memory, so the CUDA runtime may block the calling thread
 * until `stream`'s earlier work is done. Stream capture does not allow such
 * copies: on a capturing stream the call returns PAM_ERR_UNSUPPORTED before
 * queueing anything, and the capture stays valid.
 * Errors inside the kernels: there is no plan and so no pam_sync. If a
 * bounded wait in a kernel expired (a stalled staging pipeline; the call's
 * results would be partial), every element of image_tax and rho_n is NaN when
 * the stream reaches the end of the call; otherwise none is. */
pam_status pam_as_tax_static(const pam_plan_desc *d, const float *rf, int n_frames, float *image_tax,
                             float *rho_n, void *stream);

/* Failure-path check: launches on `stream` one small kernel that waits on an
 * mbarrier nothing ever completes, with the same bounded wait (about one
 * second) that the staging pipelines use. When the wait gives up, the kernel
 * sets the plan's device status word and exits, so the next pam_sync returns
 * PAM_ERR_TIMEOUT and clears it; the CUDA context stays usable. No fault, trap
 * or hang is involved. For tests of the timeout path. */
pam_status pam_debug_expire_wait(pam_plan_t p, void *stream);

/* Waits for the plan's work on `stream` and reads the device status word.
 * Returns PAM_ERR_TIMEOUT if a kernel reported an expired wait (then clears
 * it), PAM_ERR_CUDA on a runtime error, PAM_OK otherwise. */
pam_status pam_sync(pam_plan_t p, void *stream);

/* Kernel timing for measurement. While enabled, the plan records a CUDA event
 * pair on the launching stream around every launch of the fused
 * propagate-and-correlate kernel (the dominant kernel). Enabling or disabling
 * clears the counters. */
pam_status pam_profile_enable(pam_plan_t p, int on);

/* Reads and clears the counters: *prop_ms gets the summed device time of the
 * recorded propagate-and-correlate launches, *prop_launches their count, and
 * *kernel_launches the number of libpam kernels launched since the last read
 * or enable (counted whether or not timing is on). Waits for the recorded
 * events. Any output pointer may be NULL. */
pam_status pam_profile_read(pam_plan_t p, double *prop_ms, long long *prop_launches,
                            long long *kernel_launches);

/* ------------------------------------------------------------------------
 * Batches: many frames in one call, each with its own sample count, depth
 * range and bins (Eq. 1-5, 10-11 applied to each frame on its own geometry).
 * The time transform of a frame is the direct DFT of its selected bins, so
 * n_samples may be any integer (no power-of-2 requirement). One call runs a
 * fixed sequence of 4 kernels (time DFT, lateral FFT, a persistent
 * propagate-and-correlate kernel over (frame, row tile) work items, and the
 * per-frame normalisation), replayed as a CUDA graph that the batch captures
 * on its first call and again whenever the buffers change.
 * ------------------------------------------------------------------------ */
typedef struct pam_batch_s *pam_batch_t;

/* One frame of a batch. */
typedef struct {
    int n_samples;     /* nt of this frame, 32..16384, any integer */
    int nz;            /* depth rows: z_j = z0_m + j dz_m (z0_m, dz_m from the common descriptor) */
    const int *bins;   /* n_bins (common) DFT bins, 0 < k < nt/2, strictly increasing; or NULL:
                          n_bins of the band's bins spread evenly from its first to its last
                          (bin index floor(i (K-1)/(n_bins-1) + 1/2) of the K in-band bins),
                          or all K when the band holds fewer than n_bins (short frames) */
} pam_frame_desc;

/* Creates a batch. `common` is a plan descriptor whose n_elem, pitch_m, fs_hz,
 * c_mps, nx, z0_m, dz_m, f_lo_hz, f_hi_hz, n_bins (bins per frame, required),
 * n_apod (2 or 3), apod / pattern_m, eps and flags (PAM_EVANESCENT_ZERO only)
 * apply to every frame; its bins must be NULL and its n_samples, nz and
 * max_frames are ignored. The batch copies everything it needs. Inputs and
 * outputs are packed: frame f's rf [n_elem][nt_f] starts at rf_offsets[f]
 * floats, its maps [nz_f][nx] at map_offsets[f] floats (pam_batch_layout; every
 * offset is a multiple of 4). Errors: PAM_ERR_INVALID_ARG (descriptor),
 * PAM_ERR_UNSUPPORTED (a tensor-core form flag), PAM_ERR_OOM, PAM_ERR_CUDA. */
pam_status pam_batch_create(const pam_plan_desc *common, const pam_frame_desc *frames, int n_frames,
                            pam_batch_t *out);

/* Packing of a batch's buffers. rf_offsets and map_offsets (n_frames entries
 * each) and the totals (floats) may each be NULL. */
pam_status pam_batch_layout(pam_batch_t b, size_t *rf_offsets, size_t *map_offsets, size_t *rf_total,
                            size_t *map_total);

/* The bins of frame `frame` into bins_out (up to n_bins ints, may be NULL).
 * Returns the frame's bin count, or 0 for a bad handle or frame index. */
int pam_batch_bins(pam_batch_t b, int frame, int *bins_out);

/* AS-TAX (n_apod 3) or AS-DAX (n_apod 2) of every frame of the batch.
 *   rf      device float32, packed as pam_batch_layout says (16-byte aligned)
 *   image   device float32 maps, packed; rho_n the same or NULL
 * Asynchronous on `stream`. The first call, and a call whose buffers differ
 * from the previous call's, captures the launch sequence into a CUDA graph on
 * a private stream; every call then launches that graph on `stream`. Calls on
 * one batch must not overlap on the GPU (they share its workspace). */
pam_status pam_batch_as_tax(pam_batch_t b, const float *rf, float *image, float *rho_n, void *stream);

/* Waits for `stream` and reads the batch's device status word, as pam_sync. */
pam_status pam_batch_sync(pam_batch_t b, void *stream);

/* Tuning knobs. use_graph 0 launches the kernels directly (no graph);
 * persistent_ctas > 0 sets the grid of the persistent kernel (0: one per SM,
 * the most that fit; at most one per work item). */
pam_status pam_batch_configure(pam_batch_t b, int use_graph, int persistent_ctas);

/* Work items (frame, row tile), the persistent grid in use, and the libpam
 * kernels launched so far (a graph launch counts its 4 kernels). Any output
 * pointer may be NULL. */
pam_status pam_batch_info(pam_batch_t b, int *n_items, int *persistent_ctas, long long *kernel_launches);

/* Frees the batch (NULL-safe). Waits for the device first. */
void pam_batch_destroy(pam_batch_t b);

/* AS^3 (Eq. 20): I = (I_AS / max I_AS)^2 * I_AS, the full-aperture AS energy
 * (Eq. 3) weighted by its own squared normalised map instead of rho_n (the
 * paper's comparison in its appendix). image: device [n_frames][nz][nx]. The
 * maximum is taken per frame; an all-zero frame stays zero. */
pam_status pam_as3(pam_plan_t p, const float *rf, int n_frames, float *image, void *stream);

/* Image-quality measures of one map (Sec. II-D, Eq. 12-13). */
typedef struct {
    float esa_m2;   /* energy spread area A_0.5: pixels with I > max/2, times the pixel area |dx dz| */
    float isnr_db;  /* Eq. 12: 10 log10(mean I inside A_0.5 / mean I outside); +inf with nothing
                       (or only zeros) outside, NaN when max <= 0 */
    float cx_m;     /* Eq. 13 centroid sum(I_i r_i) / sum(I_i) over pixels with I_i > alpha max: */
    float cz_m;     /*   lateral and axial coordinates (m); NaN when no pixel qualifies */
    float max;      /* the map's maximum */
    int n_inside;   /* pixels in A_0.5 */
} pam_image_metrics_t;

/* Measures of n_frames maps, device float32 [n_frames][nz][nx], one CTA per
 * frame. Pixel (j, i) sits at x = x0_m + i dx_m, z = z0_m + j dz_m (for a
 * plan's grid: x0_m = -(nx-1)/2 pitch, dx_m = pitch). alpha in (0, 1): 0.7 for
 * images, 0.9 for NCC maps (Sec. II-D). out: device [n_frames]. Sums are FP64.
 * Asynchronous on `stream`. */
pam_status pam_image_metrics(const float *maps, int n_frames, int nz, int nx, double x0_m, double dx_m, double z0_m,
                             double dz_m, float alpha, pam_image_metrics_t *out, void *stream);


/* ------------------------------------------------------------------------
 * Learned form (AS-TAX with a predicted NCC weight). A 5-layer convolutional
 * network predicts rho_TAX (Eq. 10, before the max normalisation) from the
 * full-aperture AS energy (Eq. 3) and the energies of the four contiguous
 * quarters of Omega, so that a frame needs one back-propagation instead of
 * three apodized ones. Layers: conv3x3 (zero padding 1) 5 -> 32 -> 32 -> 32
 * -> 32 -> 1, ReLU after the first four, head rho = eps + (1 - eps)
 * sigmoid(z). Inputs: channel 0 = log10(E / max E + 1e-4) / 4, channels 1..4
 * the same for each quarter's energy (max over the frame's pixels of E). The
 * image is I = rho_n^2 E (Eq. 11 with the full-aperture energy, which equals
 * sum_k |p~_1 + p~_2 + p~_3|^2 when the apodizations sum to one).
 * Operands of every convolution (activations, weights, gradients) are BF16;
 * every sum is FP32. Training minimises the energy-weighted mean squared error
 * (1/n) sum w (rho - rho_TAX)^2 against the exact rho_TAX, with per-pixel
 * weight w = 0.05 + 0.95 min(1, E / max E) (E / max E = 10^(4 x0) - 1e-4 from
 * input channel 0), with Adam (Kingma and Ba 2015: beta1 0.9, beta2 0.999,
 * eps 1e-8), all on the GPU.
 *
 * Error gate: per frame, the exact method runs on the tile of 16 depth rows
 * (nx = 128; 2048 / nx rows otherwise) that holds the brightest pixel of the
 * predicted image. If the relative L2 distance there between rho_pred^2 E and
 * rho^2 E exceeds gate_tol, the frame is recomputed by the plain AS-TAX path,
 * on the GPU, within the same call.
 *
 * Parameters are a flat FP32 vector: for each layer, w[out][in][3][3] then
 * b[out] (pam_learn_n_params() = 29505 values).
 *
 * Feature tensors ("packed features") are BF16 [n_frames][nz+2][nx+2][8]:
 * the five input channels and three zeros per pixel, with a one-pixel zero
 * border (pam_learn_feature_bytes() bytes per frame).
 * ------------------------------------------------------------------------ */
typedef struct pam_learn_s *pam_learn_t;

/* Number of network parameters (29505). */
size_t pam_learn_n_params(void);

/* Creates the learned form for the geometry `d` (as pam_plan_create; n_apod
 * must be 3, no tensor-core form flag). d->max_frames is the batch size of
 * every call (pam_learn_tax runs larger calls in batches). Parameters start at
 * zero: set them with pam_learn_set_params. Errors: PAM_ERR_INVALID_ARG,
 * PAM_ERR_UNSUPPORTED, PAM_ERR_OOM, PAM_ERR_CUDA; *out is NULL on failure. */
pam_status pam_learn_create(const pam_plan_desc *d, pam_learn_t *out);

/* Frees everything (NULL-safe); waits for the device first. */
void pam_learn_destroy(pam_learn_t l);

/* Copies n = pam_learn_n_params() host floats into the network and resets the
 * Adam state. Blocks until the copy is done. PAM_ERR_NUMERIC for a non-finite
 * value.
 * This call and the three below order themselves after the most recent
 * queued call of this handle (pam_learn_example, _forward, _grads,
 * _train_step, _tax) on its stream, and wait for that work only: other streams
 * of the process keep running. Calls of one handle on different streams must
 * be ordered by the caller, as for every other call of the handle. */
pam_status pam_learn_set_params(pam_learn_t l, const float *params, size_t n);

/* Copies the current parameters to host memory. Blocks until they are there. */
pam_status pam_learn_get_params(pam_learn_t l, float *params, size_t n);

/* Training state for checkpoint and resume: parameters, Adam first and second
 * moments (3 x pam_learn_n_params() floats, in that order) and the Adam step
 * count. A training run restored with pam_learn_set_state continues exactly
 * where the saved one was: every kernel of the step reduces in a fixed order,
 * so the same batches give the same bits. Both calls block until their copies
 * are done. */
size_t pam_learn_state_size(void);
pam_status pam_learn_get_state(pam_learn_t l, float *state, size_t n, long long *adam_steps);
pam_status pam_learn_set_state(pam_learn_t l, const float *state, size_t n, long long adam_steps);

/* gate_tol: relative L2 bound of the gate (default 0.05; < 0 sends every
 * frame through the exact path, +inf accepts every frame). use_tensor_cores: 1
 * runs every layer's forward on tcgen05 and the band energies in the BF16
 * tensor-core form (PAM_FORM_GEMM_BF16, relative error about 6e-4, below the
 * BF16 rounding of the features) when that form accepts the apertures (see
 * PAM_FORM_GEMM_BF16), else on the FP32 path; nx == 128 only, else
 * PAM_ERR_UNSUPPORTED. The first call with 1 builds that form's tables (blocks).
 * 0 runs both on the FP32 path and CUDA cores (default). */
pam_status pam_learn_configure(pam_learn_t l, float gate_tol, int use_tensor_cores);

/* Bytes of one frame of packed features. */
size_t pam_learn_feature_bytes(pam_learn_t l);

/* A training example of each frame, made by the method itself:
 *   rf        device float32 [n_frames][n_elem][n_samples], n_frames <= max_frames
 *   features  device packed features (written in full, border included)
 *   target    device [n_frames][nz][nx] exact rho_TAX (Eq. 4, 10, clamped
 *             pairs, before normalisation), or NULL
 *   energy    device [n_frames][nz][nx] full-aperture energy E, or NULL */
pam_status pam_learn_example(pam_learn_t l, const float *rf, int n_frames, void *features, float *target,
                             float *energy, void *stream);

/* Network output rho (in [eps, 1)) for packed features: device [n_frames][nz][nx]. */
pam_status pam_learn_forward(pam_learn_t l, const void *features, int n_frames, float *rho, void *stream);

/* Energy-weighted mean squared error against target ([n_frames][nz][nx]) and its gradient
 * with respect to every parameter, without an update: grads device
 * [pam_learn_n_params()] or NULL, loss device [1] or NULL. */
pam_status pam_learn_grads(pam_learn_t l, const void *features, const float *target, int n_frames, float *grads,
                           float *loss, void *stream);

/* One Adam step (learning rate lr) on the batch; loss (before the step) to
 * device [1] or NULL. */
pam_status pam_learn_train_step(pam_learn_t l, const void *features, const float *target, int n_frames, float lr,
                                float *loss, void *stream);

/* Learned AS-TAX with the error gate:
 *   rf         device float32 [n_frames][n_elem][n_samples]
 *   image      device [n_frames][nz][nx]: rho_n^2 E (gate passed) or the
 *              plain AS-TAX image (gate missed)
 *   rho_n      device [n_frames][nz][nx] or NULL
 *   gate_err   device [n_frames] relative L2 distance on the gate tile, or NULL
 *   gate_pass  device int [n_frames]: 1 if the network's map was used, or NULL */
pam_status pam_learn_tax(pam_learn_t l, const float *rf, int n_frames, float *image, float *rho_n, float *gate_err,
                         int *gate_pass, void *stream);

/* As pam_sync, for the learned form's work on `stream`. */
pam_status pam_learn_sync(pam_learn_t l, void *stream);

/* Kernels launched since the last read (then cleared), the batch size and the
 * Adam steps taken. Any pointer may be NULL. */
pam_status pam_learn_info(pam_learn_t l, long long *kernel_launches, int *max_frames, long long *adam_steps);

/* Static description of a status code. */
const char *pam_status_string(pam_status s);

/* Message of the calling thread's last failed call ("" if none). */
const char *pam_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PAM_H */
