// pam_static.cu -- AS-TAX without any memory allocation.
//
// Some callers cannot allocate GPU memory at all. Examples:
//  - code inside a host framework that owns every device allocation;
//  - real-time acquisition loops certified to run with a fixed memory
//    footprint;
//  - plug-ins loaded into processes whose allocator must not be bypassed.
// They cannot create a pam_plan_t, because pam_plan_create calls cudaMalloc
// for the tables and the workspace. pam_as_tax_static serves them instead.
// It runs the same kernels as pam_as_tax, and keeps the plan tables and the
// workspace in one fixed-size array of device memory, g_scratch, that is part
// of the library image. The caller passes only the inputs and the outputs.
//
// g_scratch is PAM_STATIC_SCRATCH_BYTES (16 MiB) on every GPU that loads the
// library, until the process exits. Every call uses the same array and leaves
// its contents behind, so calls that overlap on the GPU (other streams, other
// host threads, the same device) race on it. The entry point does not check
// for that.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "pam_internal.h"

namespace {

constexpr size_t kScratchBytes = PAM_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device. In host code the name g_scratch
// stands for a host-side shadow, not a device address, so each device's
// address is looked up once with cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
void *g_scratch_dev[kMaxDevices];
std::mutex g_setup_mu;

pam_status fail(pam_status s, const char *msg) { return pam::set_error(s, msg); }

pam_status cuda_fail(cudaError_t e, const char *where)
{
    char m[256];
    std::snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
    return pam::set_error(PAM_ERR_CUDA, m);
}

// One-time set-up of the current device: the device address of g_scratch and
// the kernels' shared-memory attributes.
pam_status setup_device(int dev, unsigned char **base)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
        pam_plan_s probe;
        for (int nx = 16; nx <= 128; nx *= 2) {
            probe.nx = nx;
            e = pam::prepare_kernels(probe);
            if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
        }
        g_scratch_dev[dev] = ptr;
    }
    *base = static_cast<unsigned char *>(g_scratch_dev[dev]);
    return PAM_OK;
}

pam_status check_dev(const void *ptr, const char *what)
{
    if (!ptr) return fail(PAM_ERR_INVALID_ARG, what);
    if (reinterpret_cast<uintptr_t>(ptr) & 15u) return fail(PAM_ERR_INVALID_ARG, what);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(PAM_ERR_INVALID_ARG, what);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return fail(PAM_ERR_INVALID_ARG, what);
    return PAM_OK;
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Writes NaN to every output element when a kernel of this call reported an
// expired wait in the status word; otherwise each block only reads the word.
__global__ void static_expiry_kernel(const int *__restrict__ status, float *__restrict__ image,
                                     float *__restrict__ rho_n, size_t n)
{
    if (*status == 0) return;
    const float nan = __int_as_float(0x7fc00000);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        image[i] = nan;
        if (rho_n) rho_n[i] = nan;
    }
}

// Carves the plan tables and the one-frame workspace out of `base`. With
// base == nullptr it only counts the bytes.
size_t carve(pam_plan_s &p, int n_split, unsigned char *base)
{
    const size_t nb = p.n_bins, nx = p.nx, ne = p.ne, npix = (size_t)p.nz * p.nx;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *r = base ? base + off : nullptr;
        off += up256(bytes);
        return r;
    };
    p.t.bins = static_cast<int *>(take(nb * sizeof(int)));
    p.t.apod = static_cast<float *>(take(3 * ne * sizeof(float)));
    p.t.tw_t = static_cast<float2 *>(take((size_t)p.nt * sizeof(float2)));
    p.t.tw_x = static_cast<float2 *>(take(nx * sizeof(float2)));
    p.t.phase = static_cast<uint4 *>(take(nb * nx * sizeof(uint4)));
    p.t.live = static_cast<float *>(take(nb * nx * sizeof(float)));
    p.t.bin_evan = static_cast<int *>(take(nb * sizeof(int)));
    p.w.S = static_cast<float2 *>(take(nb * ne * sizeof(float2)));
    p.w.Q = static_cast<float2 *>(take(nb * pam::q_per_bin(3, (int)nx) * sizeof(float2)));
    // split reductions up to the cluster size stay on chip; larger ones need partials
    const size_t units = pam::prop_uses_cluster(n_split) ? 0 : (size_t)n_split;
    p.w.part = static_cast<float *>(take(units * 6 * npix * sizeof(float)));
    p.w.part_units = units;
    p.w.rho_tmp = static_cast<float *>(take(npix * sizeof(float)));
    p.w.e_tmp = static_cast<float *>(take(npix * sizeof(float)));
    p.w.fmax = static_cast<unsigned *>(take(sizeof(unsigned)));
    p.w.status = static_cast<int *>(take(sizeof(int)));
    return off;
}

}  // namespace

extern "C" pam_status pam_as_tax_static(const pam_plan_desc *d, const float *rf, int n_frames, float *image_tax,
                                        float *rho_n, void *stream)
{
    if (!d) return fail(PAM_ERR_INVALID_ARG, "descriptor is NULL");
    if (n_frames < 0) return fail(PAM_ERR_INVALID_ARG, "n_frames must be >= 0");
    // Descriptor checks: the ranges every entry point shares, then this entry
    // point's own limits; the bins and apodizations go to stack arrays.
    pam_status s = pam::check_desc_ranges(d);
    if (s != PAM_OK) return s;
    const int ne = d->n_elem, nt = d->n_samples, nz = d->nz;
    const int nx = d->nx == 0 ? ne : d->nx;
    if (nx != ne || (nx != 16 && nx != 32 && nx != 64 && nx != 128))
        return fail(PAM_ERR_UNSUPPORTED, "nx must equal n_elem and be 16, 32, 64 or 128");
    if (d->n_apod != 3) return fail(PAM_ERR_INVALID_ARG, "pam_as_tax_static needs n_apod == 3");
    if (d->flags & ~PAM_EVANESCENT_ZERO)
        return fail(PAM_ERR_INVALID_ARG, "pam_as_tax_static takes no flag but PAM_EVANESCENT_ZERO");
    int bins_h[pam::kMaxBins];
    int nb = 0;
    if ((s = pam::desc_bins(d, bins_h, &nb)) != PAM_OK) return s;
    float apod_h[3 * 256];
    if ((s = pam::desc_apod(d, 3, apod_h)) != PAM_OK) return s;

    // Geometry of a one-frame plan whose memory is g_scratch (no vectors are filled).
    pam_plan_s p;
    p.d = *d;
    p.d.bins = nullptr;
    p.d.apod = nullptr;
    p.d.nx = nx;
    p.d.n_bins = nb;
    p.ne = ne;
    p.nev = ne;
    p.pitch_x = d->pitch_m;
    p.nt = nt;
    p.nx = nx;
    p.nx_out = nx;
    p.nz = nz;
    p.n_bins = nb;
    p.n_apod = 3;
    p.max_frames = 1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(PAM_ERR_UNSUPPORTED, "device index above 63");
    e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");

    // Bin split of the automatic choice, capped at the cluster size so that the
    // split reduction needs no scratch.
    p.w.part_units = (size_t)-1;
    int ns = pam::choose_split(p, 1);
    if (ns > pam::kMaxClusterSplit) ns = pam::kMaxClusterSplit;
    const size_t need = carve(p, ns, nullptr);
    if (need > kScratchBytes) {
        char m[200];
        std::snprintf(m, sizeof(m), "this geometry needs %zu bytes of scratch; the static scratch holds %zu",
                      need, kScratchBytes);
        return fail(PAM_ERR_INVALID_ARG, m);
    }
    if (n_frames == 0) return PAM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The uploads below come from pageable stack memory, which stream capture
    // does not allow; refuse before anything is queued, so that the caller's
    // capture stays valid.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(PAM_ERR_UNSUPPORTED, "pam_as_tax_static cannot run on a capturing stream");
    if ((s = check_dev(rf, "rf must be 16-byte aligned device memory")) != PAM_OK) return s;
    if ((s = check_dev(image_tax, "image_tax must be 16-byte aligned device memory")) != PAM_OK) return s;
    if (rho_n && (s = check_dev(rho_n, "rho_n must be 16-byte aligned device memory")) != PAM_OK) return s;

    unsigned char *base = nullptr;
    if ((s = setup_device(dev, &base)) != PAM_OK) return s;
    carve(p, ns, base);

    // Pageable copies: each returns once the source has been staged, so the
    // stack arrays may go out of scope afterwards.
    if ((e = cudaMemcpyAsync(p.t.bins, bins_h, nb * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "bins upload");
    if ((e = cudaMemcpyAsync(p.t.apod, apod_h, 3 * ne * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "apodization upload");
    if ((e = cudaMemsetAsync(p.w.status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "status clear");
    if ((e = pam::launch_tables(p, st)) != cudaSuccess) return cuda_fail(e, "table kernel");

    const size_t npix = (size_t)nz * nx, fr_in = (size_t)ne * nt;
    for (int f = 0; f < n_frames; ++f) {
        if ((e = pam::launch_time_fft(p, rf + f * fr_in, 1, st)) != cudaSuccess) return cuda_fail(e, "time FFT");
        if ((e = pam::launch_lateral(p, 1, 3, p.t.apod, st)) != cudaSuccess) return cuda_fail(e, "lateral DFT");
        pam::EpiOut out;
        out.eps = d->eps;
        out.npix = (int)npix;
        out.out_main = image_tax + f * npix;
        out.rho_n = rho_n ? rho_n + f * npix : nullptr;
        out.rho_tmp = p.w.rho_tmp;
        out.e_tmp = p.w.e_tmp;
        out.fmax = p.w.fmax;
        out.status = p.w.status;
        if ((e = pam::launch_prop(p, 1, 3, ns, nullptr, out, st)) != cudaSuccess)
            return cuda_fail(e, "propagate/correlate");
        if ((e = pam::launch_epilogue(p, 1, 3, ns, out, st)) != cudaSuccess) return cuda_fail(e, "epilogue");
    }
    // Host-side injection for the tests of the expiry report: a wait that
    // nothing completes gives up after about a second and sets the status word.
    if (pam::fault_injected("static_wait") && (e = pam::launch_expire_wait(p.w.status, st)) != cudaSuccess)
        return cuda_fail(e, "injected wait");
    // No plan means no pam_sync to read the device status word, so an expired
    // bounded wait (a row tile that stopped early) shows in the outputs: every
    // element of image_tax and rho_n becomes NaN.
    static_expiry_kernel<<<2 * p.num_sms, 256, 0, st>>>(p.w.status, image_tax, rho_n, (size_t)n_frames * npix);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "expiry report");
    return PAM_OK;
}
