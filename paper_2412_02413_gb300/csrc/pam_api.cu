// pam_api.cu -- host side of libpam: descriptor validation, the plan
// ("pre-run", Sec. II-E), workspace, and the C entry points of include/pam.h.
// The arithmetic of every step runs in the kernels of pam_fft.cu and pam_prop.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "pam_internal.h"

namespace {

// Message of the calling thread's last failure, in a fixed buffer so that
// reporting an error never allocates.
thread_local char g_err[512];

}  // namespace

bool pam::fault_injected(const char *what)
{
    const char *v = std::getenv("PAM_FAULT");
    return v && std::strcmp(v, what) == 0;
}

pam::TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
pam::TraceRange::~TraceRange() { nvtxRangePop(); }

pam_status pam::set_error(pam_status s, const char *msg)
{
    std::snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
    return s;
}

namespace {

pam_status fail(pam_status s, const std::string &msg) { return pam::set_error(s, msg.c_str()); }

pam_status cuda_fail(cudaError_t e, const char *where)
{
    char m[512];
    std::snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
    return pam::set_error(PAM_ERR_CUDA, m);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

template <class T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

void free_plan_memory(pam_plan_s *p)
{
    auto fr = [](void *q) { if (q) cudaFree(q); };
    fr(p->t.bins); fr(p->t.apod); fr(p->t.ones); fr(p->t.tw_t); fr(p->t.tw_x);
    fr(p->t.phase); fr(p->t.live); fr(p->t.bin_evan);
    fr(p->w.S); fr(p->w.Q); fr(p->w.part); fr(p->w.rho_tmp); fr(p->w.e_tmp);
    fr(p->w.fmax); fr(p->w.status); fr(p->w.rf_stage); fr(p->w.img_stage); fr(p->w.rho_stage);
    fr(p->w.pad_img); fr(p->w.pad_rho); fr(p->w.pad_as); fr(p->w.pad_pairs);
    fr(p->t.c_hi); fr(p->t.c_lo); fr(p->t.ktab); fr(p->t.kwgt); fr(p->w.Bhi); fr(p->w.Blo); fr(p->w.smax);
    p->t = pam::Tables{};
    p->w = pam::Workspace{};
}

// A device pointer argument: non-null, 16-byte aligned, and device or managed memory.
pam_status check_dev_ptr(const void *ptr, const char *name, bool required)
{
    if (!ptr) {
        if (required) return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is NULL");
        return PAM_OK;
    }
    if (reinterpret_cast<uintptr_t>(ptr) & 15u)
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(PAM_ERR_INVALID_ARG, std::string(name) + " is not device memory");
    return PAM_OK;
}

}  // namespace

pam_status pam::check_desc_ranges(const pam_plan_desc *d)
{
    if (d->n_elem < 8 || d->n_elem > 256) return fail(PAM_ERR_INVALID_ARG, "n_elem must be in [8, 256]");
    if (!finite_pos(d->pitch_m)) return fail(PAM_ERR_INVALID_ARG, "pitch_m must be finite and > 0");
    if (!finite_pos(d->fs_hz)) return fail(PAM_ERR_INVALID_ARG, "fs_hz must be finite and > 0");
    if (!finite_pos(d->c_mps)) return fail(PAM_ERR_INVALID_ARG, "c_mps must be finite and > 0");
    if (d->n_samples < 64 || d->n_samples > 8192)
        return fail(d->n_samples > 8192 && d->n_samples > 0 ? PAM_ERR_UNSUPPORTED : PAM_ERR_INVALID_ARG,
                    "n_samples must be in [64, 8192]");
    if (!is_pow2(d->n_samples))
        return fail(PAM_ERR_UNSUPPORTED, "n_samples must be a power of two for the radix-4/2 time FFT");
    if (d->nz < 1 || d->nz > 65535) return fail(PAM_ERR_INVALID_ARG, "nz must be in [1, 65535]");
    if (!std::isfinite(d->z0_m) || d->z0_m < 0.0) return fail(PAM_ERR_INVALID_ARG, "z0_m must be finite and >= 0");
    if (!finite_pos(d->dz_m)) return fail(PAM_ERR_INVALID_ARG, "dz_m must be finite and > 0");
    if (!(d->eps > 0.0f) || !(d->eps <= 1.0f)) return fail(PAM_ERR_INVALID_ARG, "eps must be in (0, 1]");
    return PAM_OK;
}

pam_status pam::desc_bins(const pam_plan_desc *d, int *bins, int *n_out)
{
    const int nt = d->n_samples;
    int nb = 0;
    if (d->bins) {
        if (d->n_bins < 1 || d->n_bins > 8192) return fail(PAM_ERR_INVALID_ARG, "n_bins must be in [1, 8192]");
        for (int b = 0; b < d->n_bins; ++b) {
            // bins[b] >= b + 1 and 2 bins[b] < nt <= 8192, so at most kMaxBins - 1 entries are written
            const int k = d->bins[b];
            if (k <= 0 || 2 * k >= nt) return fail(PAM_ERR_INVALID_ARG, "every bin must satisfy 0 < k < n_samples/2");
            if (b > 0 && k <= d->bins[b - 1]) return fail(PAM_ERR_INVALID_ARG, "bins must be strictly increasing");
            bins[nb++] = k;
        }
    } else {
        if (!std::isfinite(d->f_lo_hz) || !std::isfinite(d->f_hi_hz) || d->f_hi_hz < d->f_lo_hz)
            return fail(PAM_ERR_INVALID_ARG, "band must satisfy f_lo_hz <= f_hi_hz (finite)");
        for (int k = 1; 2 * k < nt; ++k) {
            const double f = (double)k * d->fs_hz / (double)nt;
            if (f >= d->f_lo_hz && f <= d->f_hi_hz) bins[nb++] = k;
        }
        if (nb == 0) return fail(PAM_ERR_INVALID_ARG, "the band holds no DFT bin");
    }
    *n_out = nb;
    return PAM_OK;
}

pam_status pam::desc_apod(const pam_plan_desc *d, int n_apod, float *apod)
{
    const int ne = d->n_elem;
    if (d->apod) {
        for (int x = 0; x < n_apod * ne; ++x) {
            if (!std::isfinite(d->apod[x])) return fail(PAM_ERR_INVALID_ARG, "apodization weights must be finite");
            apod[x] = d->apod[x];
        }
    } else {
        if (d->pattern_m < 1 || d->pattern_m > ne) return fail(PAM_ERR_INVALID_ARG, "pattern_m must be in [1, n_elem]");
        for (int q = 0; q < n_apod; ++q)
            for (int e = 0; e < ne; ++e) apod[q * ne + e] = ((e / d->pattern_m) % n_apod == q) ? 1.0f : 0.0f;
    }
    return PAM_OK;
}

namespace {

pam_status validate_and_fill(const pam_plan_desc *d, pam_plan_s *p)
{
    pam_status s = pam::check_desc_ranges(d);
    if (s != PAM_OK) return s;
    const bool up2 = (d->flags & PAM_LATERAL_UPSAMPLE2X) != 0;
    const bool pad2 = (d->flags & PAM_LATERAL_PAD2X) != 0;
    if (up2 && pad2) return fail(PAM_ERR_INVALID_ARG, "PAM_LATERAL_UPSAMPLE2X and PAM_LATERAL_PAD2X exclude each other");
    const int nev = up2 || pad2 ? 2 * d->n_elem : d->n_elem;   // channels of S = lateral DFT length
    const int nx_out = up2 ? nev : d->n_elem;                    // image columns
    int nx = d->nx == 0 ? nx_out : d->nx;
    if (nx != nx_out)
        return fail(PAM_ERR_UNSUPPORTED, up2 ? "nx must be 2 n_elem with PAM_LATERAL_UPSAMPLE2X"
                                             : "nx must equal n_elem (or 2 n_elem with PAM_LATERAL_UPSAMPLE2X)");
    if (nev != 16 && nev != 32 && nev != 64 && nev != 128)
        return fail(PAM_ERR_UNSUPPORTED, "the lateral DFT length (n_elem, or 2 n_elem with PAM_LATERAL_UPSAMPLE2X "
                                         "or PAM_LATERAL_PAD2X) must be 16, 32, 64 or 128");
    if (d->n_apod < 1 || d->n_apod > 3) return fail(PAM_ERR_INVALID_ARG, "n_apod must be 1, 2 or 3");
    if (d->max_frames < 1 || d->max_frames > 65535) return fail(PAM_ERR_INVALID_ARG, "max_frames must be in [1, 65535]");
    const unsigned form_bits =
        PAM_FORM_GEMM_BF16 | PAM_FORM_GEMM_FP16 | PAM_FORM_GEMM_BF16_SPLIT | PAM_FORM_GEMM_FP16_SPLIT;
    if (d->flags & ~(PAM_EVANESCENT_ZERO | PAM_LATERAL_UPSAMPLE2X | PAM_LATERAL_PAD2X | form_bits))
        return fail(PAM_ERR_INVALID_ARG, "unknown flag bits");
    const unsigned form = d->flags & form_bits;
    if (form & (form - 1)) return fail(PAM_ERR_INVALID_ARG, "at most one PAM_FORM_GEMM_* flag");
    if (form && up2) return fail(PAM_ERR_UNSUPPORTED, "PAM_LATERAL_UPSAMPLE2X runs on the plain FP32 path only");
    if (form && pad2) return fail(PAM_ERR_UNSUPPORTED, "PAM_LATERAL_PAD2X runs on the plain FP32 path only");

    const int nt = d->n_samples;
    int nb = 0;
    p->bins.assign(pam::kMaxBins, 0);
    if ((s = pam::desc_bins(d, p->bins.data(), &nb)) != PAM_OK) return s;
    p->bins.resize(nb);

    const int ne = d->n_elem, na = d->n_apod;
    p->apod.assign((size_t)na * ne, 0.0f);
    if ((s = pam::desc_apod(d, na, p->apod.data())) != PAM_OK) return s;

    p->d = *d;
    p->d.bins = nullptr;
    p->d.apod = nullptr;
    p->d.nx = nx;
    p->d.n_bins = (int)p->bins.size();
    p->ne = ne;
    p->nev = nev;
    p->chan_step = up2 ? 2 : 1;
    p->pitch_x = up2 ? 0.5 * d->pitch_m : d->pitch_m;
    p->nt = nt;
    p->log2nt = ilog2(nt);
    p->nx = nev;
    p->nx_out = nx;
    p->nz = d->nz;
    p->n_bins = (int)p->bins.size();
    p->n_apod = na;
    p->max_frames = d->max_frames;
    p->form = (int)form;
    if (form) {
        // Tensor-core form: each aperture is a K range of one GEMM made of the aligned
        // 8-element blocks it touches (elements of the block outside the aperture get
        // weight 0). A block takes 16 K columns: 8 pairing with Re c, 8 with Im c.
        if (nx != 128) return fail(PAM_ERR_UNSUPPORTED, "the tensor-core form needs nx == 128");
        if (na < 2) return fail(PAM_ERR_INVALID_ARG, "the tensor-core form is built for AS-DAX and AS-TAX");
        p->ktab_h.clear();
        p->kwgt_h.clear();
        int k = 0;
        for (int q = 0; q < na; ++q) {
            p->kq[q] = k;
            for (int m = 0; m < nx / 8; ++m) {
                bool used = false;
                for (int t = 0; t < 8; ++t) used = used || (8 * m + t < ne && p->apod[(size_t)q * ne + 8 * m + t] != 0.0f);
                if (!used) continue;
                for (int half = 0; half < 2; ++half)
                    for (int t = 0; t < 8; ++t) {
                        const int e = 8 * m + t;
                        p->ktab_h.push_back(e < ne ? (short)(e | (half << 14)) : (short)-1);
                        p->kwgt_h.push_back(e < ne ? p->apod[(size_t)q * ne + e] : 0.0f);
                    }
                k += 16;
            }
        }
        for (int q = na; q < 4; ++q) p->kq[q] = k;
        p->K = k;
        if (k == 0) return fail(PAM_ERR_INVALID_ARG, "every aperture is empty");
        if (k > pam::kMaxGemmK)
            return fail(PAM_ERR_UNSUPPORTED,
                        "the apertures touch too many 8-element blocks for the tensor-core form "
                        "(at most 24 block-aperture pairs)");
    }
    return PAM_OK;
}

pam_status alloc_plan(pam_plan_s *p)
{
    const size_t ne = p->nev, nx = p->nx, nb = p->n_bins, F = p->max_frames;   // ne: channels of S
    const size_t npix = (size_t)p->nz * nx;
    cudaError_t e = cudaSuccess;
#define PAM_TRY(x)                                           \
    do {                                                     \
        e = (x);                                             \
        if (e != cudaSuccess) {                              \
            cudaGetLastError();                              \
            return e == cudaErrorMemoryAllocation            \
                       ? fail(PAM_ERR_OOM, #x)               \
                       : cuda_fail(e, #x);                   \
        }                                                    \
    } while (0)
    PAM_TRY(dalloc(&p->t.bins, nb));
    PAM_TRY(dalloc(&p->t.apod, (size_t)p->n_apod * ne));
    PAM_TRY(dalloc(&p->t.ones, ne));
    PAM_TRY(dalloc(&p->t.tw_t, (size_t)p->nt));
    PAM_TRY(dalloc(&p->t.tw_x, nx));
    PAM_TRY(dalloc(&p->t.phase, nb * nx));
    PAM_TRY(dalloc(&p->t.live, nb * nx));
    PAM_TRY(dalloc(&p->t.bin_evan, nb));
    PAM_TRY(dalloc(&p->w.S, F * nb * ne));
    PAM_TRY(dalloc(&p->w.Q, F * nb * pam::q_per_bin(p->n_apod, nx)));
    if (pam::fault_injected("alloc")) return fail(PAM_ERR_OOM, "injected allocation failure (PAM_FAULT=alloc)");
    int rows = pam::prop_rows_per_cta(p->nx);
    int row_tiles = (p->nz + rows - 1) / rows;
    size_t target = (size_t)pam::prop_ctas_per_sm() * p->num_sms;
    size_t split_units = (target + row_tiles - 1) / row_tiles;
    p->w.part_units = std::max(F, split_units);
    // sums of the split tiles of the even division
    const size_t part_floats = std::max(p->w.part_units * (size_t)pam::n_acc(p->n_apod) * npix,
                                        pam::prop_seg_part_floats(*p));
    PAM_TRY(dalloc(&p->w.part, part_floats));
    p->seg_ok = true;
    PAM_TRY(dalloc(&p->w.rho_tmp, F * npix));
    PAM_TRY(dalloc(&p->w.e_tmp, F * npix));
    PAM_TRY(dalloc(&p->w.fmax, F));
    PAM_TRY(dalloc(&p->w.status, 1));
    if (p->form) {
        const bool split = p->form == PAM_FORM_GEMM_BF16_SPLIT || p->form == PAM_FORM_GEMM_FP16_SPLIT;
        const size_t rows = nb * (size_t)p->nz * nx;
        const size_t groups = (F + pam::kFramesPerGroup - 1) / pam::kFramesPerGroup;
        const size_t tile16 = (size_t)p->K * 2 * pam::kFramesPerGroup * 2 / 16;   // uint4 per (group, bin) tile
        PAM_TRY(dalloc(&p->t.c_hi, rows));
        if (split) PAM_TRY(dalloc(&p->t.c_lo, rows));
        PAM_TRY(dalloc(&p->t.ktab, (size_t)p->K));
        PAM_TRY(dalloc(&p->t.kwgt, (size_t)p->K));
        PAM_TRY(dalloc(&p->w.Bhi, groups * nb * tile16));
        if (split) PAM_TRY(dalloc(&p->w.Blo, groups * nb * tile16));
        PAM_TRY(dalloc(&p->w.smax, F));
        PAM_TRY(cudaMemcpy(p->t.ktab, p->ktab_h.data(), p->K * sizeof(short), cudaMemcpyHostToDevice));
        PAM_TRY(cudaMemcpy(p->t.kwgt, p->kwgt_h.data(), p->K * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (p->nx_out != p->nx) {   // PAM_LATERAL_PAD2X: full-width maps, cropped after the epilogue
        PAM_TRY(dalloc(&p->w.pad_img, F * npix));
        if (p->n_apod >= 2) {
            PAM_TRY(dalloc(&p->w.pad_rho, F * npix));
            PAM_TRY(dalloc(&p->w.pad_as, F * npix));
            PAM_TRY(dalloc(&p->w.pad_pairs, F * (p->n_apod == 3 ? 3 : 1) * npix));
        }
    }
    PAM_TRY(cudaMemset(p->w.status, 0, sizeof(int)));
    PAM_TRY(cudaMemcpy(p->t.bins, p->bins.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
    {
        // apodization per channel of S: element e's weight at channel e (or 2e when zero-stuffed)
        const size_t step = (size_t)p->chan_step;
        std::vector<float> av((size_t)p->n_apod * ne, 0.0f);
        for (int q = 0; q < p->n_apod; ++q)
            for (int e = 0; e < p->ne; ++e) av[(size_t)q * ne + step * e] = p->apod[(size_t)q * p->ne + e];
        PAM_TRY(cudaMemcpy(p->t.apod, av.data(), av.size() * sizeof(float), cudaMemcpyHostToDevice));
        // zero-stuffed or padding channels are never written: clear them once
        if (p->nev > p->ne) PAM_TRY(cudaMemset(p->w.S, 0, F * nb * ne * sizeof(float2)));
    }
    std::vector<float> ones(ne, 1.0f);
    PAM_TRY(cudaMemcpy(p->t.ones, ones.data(), ne * sizeof(float), cudaMemcpyHostToDevice));
#undef PAM_TRY
    return PAM_OK;
}

bool oom(cudaError_t e) { return e == cudaErrorMemoryAllocation; }

void prof_release(pam_plan_s *p)
{
    for (cudaEvent_t ev : p->prof_ev) cudaEventDestroy(ev);
    p->prof_ev.clear();
    p->prof_used = 0;
}

cudaError_t prof_record(pam_plan_s *p, cudaStream_t st)
{
    if (!p->prof_on) return cudaSuccess;
    if (p->prof_used == p->prof_ev.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        p->prof_ev.push_back(ev);
    }
    return cudaEventRecord(p->prof_ev[p->prof_used++], st);
}

cudaError_t prof_begin(pam_plan_s *p, cudaStream_t st) { return prof_record(p, st); }
cudaError_t prof_end(pam_plan_s *p, cudaStream_t st) { return prof_record(p, st); }

pam::EpiOut epi_out(const pam_plan_s *p, float *main, float *rho_n, float *rho_pairs, float *image_as)
{
    pam::EpiOut o;
    o.eps = p->d.eps;
    o.npix = p->nz * p->nx;
    o.out_main = main;
    o.rho_n = rho_n;
    o.rho_pairs = rho_pairs;
    o.image_as = image_as;
    o.rho_tmp = p->w.rho_tmp;
    o.e_tmp = p->w.e_tmp;
    o.fmax = p->w.fmax;
    o.status = p->w.status;
    return o;
}

pam_status run_xcorr(pam_plan_t p, const float *rf, int n_frames, float *image, float *rho_n,
                     float *rho_pairs, float *image_as, cudaStream_t st)
{
    const size_t npix = (size_t)p->nz * p->nx_out;   // caller's maps
    const size_t fr_in = (size_t)p->ne * p->nt;
    const int npairs = p->n_apod == 3 ? 3 : 1;
    const bool crop = p->nx_out != p->nx;             // PAM_LATERAL_PAD2X
    if (pam::fault_injected("launch"))
        return fail(PAM_ERR_CUDA, "injected launch failure (PAM_FAULT=launch): nothing was queued");
    for (int f0 = 0; f0 < n_frames; f0 += p->max_frames) {
        int Fc = std::min(p->max_frames, n_frames - f0);
        float *c_img = image + (size_t)f0 * npix, *c_rho = rho_n ? rho_n + (size_t)f0 * npix : nullptr;
        float *c_pairs = rho_pairs ? rho_pairs + (size_t)f0 * npairs * npix : nullptr;
        float *c_as = image_as ? image_as + (size_t)f0 * npix : nullptr;
        cudaError_t e = pam::launch_time_fft(*p, rf + (size_t)f0 * fr_in, Fc, st);
        if (e != cudaSuccess) return cuda_fail(e, "time FFT launch");
        if (p->form) {
            // tensor-core form: pack operands, GEMM per (row, bin), epilogue from its sums
            pam::EpiOut out = epi_out(p, c_img, c_rho, c_pairs, c_as);
            if ((e = prof_begin(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
            e = pam::launch_prec(*p, Fc, st);
            if (e != cudaSuccess) return cuda_fail(e, "tensor-core form launch");
            if ((e = prof_end(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
            e = pam::launch_epilogue(*p, Fc, p->n_apod, 1, out, st, true);
            if (e != cudaSuccess) return cuda_fail(e, "epilogue launch");
            p->kernels += 1 + pam::prec_kernels() + 2;
            continue;
        }
        e = pam::launch_lateral(*p, Fc, p->n_apod, p->t.apod, st);
        if (e != cudaSuccess) return cuda_fail(e, "lateral DFT launch");
        int ns = pam::choose_split(*p, Fc);
        // with padding the epilogue writes full-width maps (rho_n and E always) for the crop
        pam::EpiOut out = crop ? epi_out(p, p->w.pad_img, p->w.pad_rho, c_pairs ? p->w.pad_pairs : nullptr, p->w.pad_as)
                               : epi_out(p, c_img, c_rho, c_pairs, c_as);
        if ((e = prof_begin(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
        e = pam::launch_prop(*p, Fc, p->n_apod, ns, nullptr, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "propagate/correlate launch");
        if ((e = prof_end(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
        e = pam::launch_epilogue(*p, Fc, p->n_apod, ns, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "epilogue launch");
        p->kernels += 3 + pam::epilogue_kernels(*p, p->n_apod, ns);
        if (crop) {
            e = pam::launch_pad_crop(p->w.pad_rho, p->w.pad_as, p->w.pad_pairs, npairs, Fc, p->nz, p->nx, p->nx_out,
                                     c_img, c_rho, c_pairs, c_as, st);
            if (e != cudaSuccess) return cuda_fail(e, "crop launch");
            p->kernels += 1;
        }
    }
    return PAM_OK;
}

}  // namespace

extern "C" {

void pam_plan_desc_init(pam_plan_desc *d)
{
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->n_apod = 3;
    d->pattern_m = 16;
    d->eps = 1e-3f;
    d->max_frames = 1;
}

pam_status pam_plan_create(const pam_plan_desc *d, pam_plan_t *out)
{
    pam::TraceRange trace_("pam_plan_create");
    if (!out) return fail(PAM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(PAM_ERR_INVALID_ARG, "descriptor is NULL");
    pam_plan_s *p = new (std::nothrow) pam_plan_s();
    if (!p) return fail(PAM_ERR_OOM, "host allocation of the plan failed");
    pam_status s = validate_and_fill(d, p);
    if (s != PAM_OK) { delete p; return s; }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "device query"); }
    s = alloc_plan(p);
    if (s != PAM_OK) {
        free_plan_memory(p);
        delete p;
        return s;
    }
    e = pam::prepare_kernels(*p);
    if (e == cudaSuccess && p->form) e = pam::prepare_prec_kernels();
    if (e == cudaSuccess) e = pam::launch_tables(*p, 0);
    if (e == cudaSuccess && p->form) e = pam::launch_prec_tables(*p, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        free_plan_memory(p);
        delete p;
        return cuda_fail(e, "plan tables");
    }
    *out = p;
    return PAM_OK;
}

void pam_destroy(pam_plan_t p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    prof_release(p);
    free_plan_memory(p);
    cudaSetDevice(cur);
    delete p;
}

int pam_plan_bins(pam_plan_t p, int *bins_out)
{
    if (!p) return 0;
    if (bins_out) std::memcpy(bins_out, p->bins.data(), p->bins.size() * sizeof(int));
    return p->n_bins;
}

int pam_plan_apod(pam_plan_t p, float *apod_out)
{
    if (!p) return 0;
    if (apod_out) std::memcpy(apod_out, p->apod.data(), p->apod.size() * sizeof(float));
    return p->n_apod;
}

pam_status pam_as_backprop(pam_plan_t p, const float *rf, int n_frames, int apod_index,
                           float *energy, float *fields, void *stream)
{
    pam::TraceRange trace_("pam_as_backprop");
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (n_frames < 0) return fail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (apod_index < -1 || apod_index >= p->n_apod) return fail(PAM_ERR_INVALID_ARG, "apod_index out of range");
    if (n_frames == 0) return PAM_OK;
    pam_status s;
    if ((s = check_dev_ptr(rf, "rf", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(energy, "energy", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(fields, "fields", false)) != PAM_OK) return s;
    const bool crop = p->nx_out != p->nx;   // PAM_LATERAL_PAD2X
    if (fields && crop) return fail(PAM_ERR_UNSUPPORTED, "the fields output is not built with PAM_LATERAL_PAD2X");
    if (pam::fault_injected("launch"))
        return fail(PAM_ERR_CUDA, "injected launch failure (PAM_FAULT=launch): nothing was queued");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float *apod = apod_index < 0 ? p->t.ones : p->t.apod + (size_t)apod_index * p->nev;
    const size_t npix = (size_t)p->nz * p->nx_out;
    const size_t fr_in = (size_t)p->ne * p->nt;
    for (int f0 = 0; f0 < n_frames; f0 += p->max_frames) {
        int Fc = std::min(p->max_frames, n_frames - f0);
        cudaError_t e = pam::launch_time_fft(*p, rf + (size_t)f0 * fr_in, Fc, st);
        if (e != cudaSuccess) return cuda_fail(e, "time FFT launch");
        e = pam::launch_lateral(*p, Fc, 1, apod, st);
        if (e != cudaSuccess) return cuda_fail(e, "lateral DFT launch");
        int ns = pam::choose_split(*p, Fc);
        float *fl = fields ? fields + (size_t)f0 * p->n_bins * npix * 2 : nullptr;
        pam::EpiOut out = epi_out(p, crop ? p->w.pad_img : energy + (size_t)f0 * npix, nullptr, nullptr, nullptr);
        if ((e = prof_begin(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
        e = pam::launch_prop(*p, Fc, 1, ns, fl, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "propagate launch");
        if ((e = prof_end(p, st)) != cudaSuccess) return cuda_fail(e, "profile event");
        e = pam::launch_epilogue(*p, Fc, 1, ns, out, st, false, fl != nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "epilogue launch");
        p->kernels += 3 + pam::epilogue_kernels(*p, 1, ns, fl != nullptr);
        if (crop) {   // element columns of the padded energy map
            const size_t w_out = (size_t)p->nx_out * sizeof(float), w_in = (size_t)p->nx * sizeof(float);
            e = cudaMemcpy2DAsync(energy + (size_t)f0 * npix, w_out, p->w.pad_img, w_in, w_out, (size_t)Fc * p->nz,
                                  cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "crop copy");
        }
    }
    return PAM_OK;
}

pam_status pam_as_tax(pam_plan_t p, const float *rf, int n_frames, float *image_tax,
                      float *rho_n, float *rho_pairs, float *image_as, void *stream)
{
    pam::TraceRange trace_("pam_as_tax");
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (p->n_apod != 3) return fail(PAM_ERR_INVALID_ARG, "pam_as_tax needs a plan with n_apod == 3");
    if (n_frames < 0) return fail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return PAM_OK;
    pam_status s;
    if ((s = check_dev_ptr(rf, "rf", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(image_tax, "image_tax", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(rho_n, "rho_n", false)) != PAM_OK) return s;
    if ((s = check_dev_ptr(rho_pairs, "rho_pairs", false)) != PAM_OK) return s;
    if ((s = check_dev_ptr(image_as, "image_as", false)) != PAM_OK) return s;
    return run_xcorr(p, rf, n_frames, image_tax, rho_n, rho_pairs, image_as, static_cast<cudaStream_t>(stream));
}

pam_status pam_as_dax(pam_plan_t p, const float *rf, int n_frames, float *image_dax,
                      float *rho_n, float *rho_pair, float *image_as, void *stream)
{
    pam::TraceRange trace_("pam_as_dax");
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (p->n_apod != 2) return fail(PAM_ERR_INVALID_ARG, "pam_as_dax needs a plan with n_apod == 2");
    if (n_frames < 0) return fail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return PAM_OK;
    pam_status s;
    if ((s = check_dev_ptr(rf, "rf", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(image_dax, "image_dax", true)) != PAM_OK) return s;
    if ((s = check_dev_ptr(rho_n, "rho_n", false)) != PAM_OK) return s;
    if ((s = check_dev_ptr(rho_pair, "rho_pair", false)) != PAM_OK) return s;
    if ((s = check_dev_ptr(image_as, "image_as", false)) != PAM_OK) return s;
    return run_xcorr(p, rf, n_frames, image_dax, rho_n, rho_pair, image_as, static_cast<cudaStream_t>(stream));
}

pam_status pam_as_xcorr_host_async(pam_plan_t p, const float *rf_host, int n_frames, float *image_host,
                                   float *rho_n_host, void *stream)
{
    pam::TraceRange trace_("pam_as_xcorr_host_async");
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (p->n_apod < 2) return fail(PAM_ERR_INVALID_ARG, "pam_as_xcorr_host needs n_apod of 2 or 3");
    if (n_frames < 0) return fail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return PAM_OK;
    if (!rf_host || !image_host) return fail(PAM_ERR_INVALID_ARG, "rf_host and image_host are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t npix = (size_t)p->nz * p->nx_out;
    const size_t fr_in = (size_t)p->ne * p->nt;
    const size_t F = p->max_frames;
    cudaError_t e;
    if (!p->w.rf_stage) {
        if ((e = dalloc(&p->w.rf_stage, F * fr_in)) != cudaSuccess ||
            (e = dalloc(&p->w.img_stage, F * npix)) != cudaSuccess ||
            (e = dalloc(&p->w.rho_stage, F * npix)) != cudaSuccess) {
            cudaGetLastError();
            return fail(oom(e) ? PAM_ERR_OOM : PAM_ERR_CUDA, "staging allocation failed");
        }
    }
    for (int f0 = 0; f0 < n_frames; f0 += p->max_frames) {
        int Fc = std::min(p->max_frames, n_frames - f0);
        e = cudaMemcpyAsync(p->w.rf_stage, rf_host + (size_t)f0 * fr_in, Fc * fr_in * sizeof(float),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "rf upload");
        pam_status s = run_xcorr(p, p->w.rf_stage, Fc, p->w.img_stage, rho_n_host ? p->w.rho_stage : nullptr,
                                 nullptr, nullptr, st);
        if (s != PAM_OK) return s;
        e = cudaMemcpyAsync(image_host + (size_t)f0 * npix, p->w.img_stage, Fc * npix * sizeof(float),
                            cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "image download");
        if (rho_n_host) {
            e = cudaMemcpyAsync(rho_n_host + (size_t)f0 * npix, p->w.rho_stage, Fc * npix * sizeof(float),
                                cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return cuda_fail(e, "rho_n download");
        }
    }
    return PAM_OK;
}

pam_status pam_as_xcorr_host(pam_plan_t p, const float *rf_host, int n_frames, float *image_host,
                             float *rho_n_host, void *stream)
{
    pam_status s = pam_as_xcorr_host_async(p, rf_host, n_frames, image_host, rho_n_host, stream);
    if (s != PAM_OK || n_frames == 0) return s;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    return PAM_OK;
}

pam_status pam_debug_expire_wait(pam_plan_t p, void *stream)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t e = pam::launch_expire_wait(p->w.status, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "expire-wait launch");
    p->kernels += 1;
    return PAM_OK;
}

pam_status pam_sync(pam_plan_t p, void *stream)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
    int status = 0;
    e = cudaMemcpy(&status, p->w.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (status != 0) {
        cudaMemset(p->w.status, 0, sizeof(int));
        return fail(PAM_ERR_TIMEOUT, "a kernel reported an expired bounded wait");
    }
    return PAM_OK;
}

pam_status pam_plan_set_grid(pam_plan_t p, int n_ctas)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (n_ctas < 0) return fail(PAM_ERR_INVALID_ARG, "n_ctas must be >= 0");
    p->grid_override = n_ctas;
    return PAM_OK;
}

pam_status pam_plan_set_fft_radix(pam_plan_t p, int radix)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (radix != 4 && radix != 8) return fail(PAM_ERR_INVALID_ARG, "radix must be 4 or 8");
    p->fft_radix = radix;
    return PAM_OK;
}

pam_status pam_plan_set_lane_rows(pam_plan_t p, int rows)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (rows != 1 && rows != 2) return fail(PAM_ERR_INVALID_ARG, "rows per lane must be 1 or 2");
    p->lane_rows = rows;
    return PAM_OK;
}

pam_status pam_plan_set_gemm_tile(pam_plan_t p, int m)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (m != 128 && m != 256) return fail(PAM_ERR_INVALID_ARG, "the GEMM tile M must be 128 or 256");
    p->gemm_m = m;
    return PAM_OK;
}

pam_status pam_plan_set_gemm_frames(pam_plan_t p, int frames)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (frames != 16 && frames != 32) return fail(PAM_ERR_INVALID_ARG, "frames per CTA must be 16 or 32");
    p->gemm_frames = frames;
    return PAM_OK;
}

pam_status pam_plan_set_split(pam_plan_t p, int n_split)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    if (n_split < 0) return fail(PAM_ERR_INVALID_ARG, "n_split must be >= 0");
    p->split_override = n_split;
    return PAM_OK;
}

pam_status pam_profile_enable(pam_plan_t p, int on)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise");
    p->prof_used = 0;
    p->kernels = 0;
    p->prof_on = on != 0;
    if (!p->prof_on) prof_release(p);
    return PAM_OK;
}

pam_status pam_profile_read(pam_plan_t p, double *prop_ms, long long *prop_launches, long long *kernel_launches)
{
    if (!p) return fail(PAM_ERR_INVALID_ARG, "plan is NULL");
    double total = 0.0;
    for (size_t i = 0; i + 1 < p->prof_used; i += 2) {
        cudaError_t e = cudaEventSynchronize(p->prof_ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event synchronise");
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, p->prof_ev[i], p->prof_ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "event elapsed time");
        total += ms;
    }
    if (prop_ms) *prop_ms = total;
    if (prop_launches) *prop_launches = (long long)(p->prof_used / 2);
    if (kernel_launches) *kernel_launches = p->kernels;
    p->prof_used = 0;
    p->kernels = 0;
    return PAM_OK;
}

const char *pam_status_string(pam_status s)
{
    switch (s) {
    case PAM_OK: return "PAM_OK";
    case PAM_ERR_INVALID_ARG: return "PAM_ERR_INVALID_ARG";
    case PAM_ERR_UNSUPPORTED: return "PAM_ERR_UNSUPPORTED";
    case PAM_ERR_OOM: return "PAM_ERR_OOM";
    case PAM_ERR_CUDA: return "PAM_ERR_CUDA";
    case PAM_ERR_TIMEOUT: return "PAM_ERR_TIMEOUT";
    case PAM_ERR_NUMERIC: return "PAM_ERR_NUMERIC";
    }
    return "PAM_ERR_UNKNOWN";
}

const char *pam_last_error(void) { return g_err; }

}  // extern "C"
