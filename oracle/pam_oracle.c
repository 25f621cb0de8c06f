/*
 * pam_oracle.c -- plain FP64 CPU oracle for cross-correlated angular-spectrum
 * passive acoustic mapping (arXiv 2412.02413).
 *
 * TEST INFRASTRUCTURE. It exists to check the GPU library, which never links
 * it. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * call it.
 *
 * Every function writes a definition from the paper out directly: direct DFTs
 * with exact integer angle reduction, an explicit propagator loop and explicit
 * sums. There is no blocking, fusion or reordering. Threads only split the
 * bin range of the sum over frequencies (Eq. 3-5, 11). Per-thread partial
 * sums are then added in thread order.
 *
 * Readings taken where the paper is silent or ambiguous:
 *  - Fourier sign: the forward time DFT uses exp(-i w t), so Eq. 2's
 *    exp(+i kz z) carries the array-plane spectrum into the medium
 *    (back-propagation towards the sources).
 *  - Evanescent components (kx^2 > (w/c)^2) use the principal branch of Eq. 2,
 *    kz = i*kappa, and so decay as exp(-kappa z). With evanescent_zero they
 *    are dropped instead.
 *  - The lateral DFT runs over the element index with nx = n_elem, and the
 *    inverse carries the 1/nx factor. Forward DFTs are unnormalised.
 *  - Depth z is measured from the array face (Fig. 1(a): array at z0 = 0).
 *  - NCC (Eq. 4) uses the real part of sum_w conj(p_q) p_r. Appendix A
 *    completes the negative frequencies as conjugates, which doubles every
 *    term and cancels in the ratio. A zero denominator gives rho = eps.
 *  - eps clamp (Sec. II-A): each pair coefficient is clamped before the cube
 *    root of Eq. 10.
 *  - rho_n (Sec. II-A, II-C) is rho divided by its maximum over all pixels of
 *    the frame.
 *  - Eq. 5 and Eq. 11 square rho_n together with the magnitude:
 *    I = rho_n^2 * sum_w |sum_q p_q|^2.
 */
#include "pam_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Deliberate-mistake switch for the mutation tests (0 = the correct oracle). */
static int g_mutation = 0;
void pam_oracle_set_mutation(int id) { g_mutation = id; }
#define MUT(id) (g_mutation == (id))

/* ---------------------------------------------------------------- masks -- */

/* Pattern-m apodization (Sec. II-A for n = 2, Sec. II-C for n = 3): runs of m
 * adjacent active elements, each followed by (n-1)*m inactive ones, with
 * aperture q shifted by q*m elements. */
int pam_oracle_pattern(int n_elem, int n_apod, int m, double *apod)
{
    if (n_elem <= 0 || n_apod <= 0 || m <= 0 || !apod) return -1;
    for (int q = 0; q < n_apod; ++q)
        for (int e = 0; e < n_elem; ++e) {
            int group = MUT(9) ? (e + 1) / m : e / m;
            apod[q * n_elem + e] = (group % n_apod == q) ? 1.0 : 0.0;
        }
    return 0;
}

/* Omega as a band (Sec. II-D): every bin whose frequency k*fs/nt lies in
 * [f_lo, f_hi], excluding DC and Nyquist. */
int pam_oracle_band_bins(int nt, double fs, double f_lo, double f_hi, int *bins, int cap)
{
    int n = 0;
    for (int k = 1; 2 * k < nt; ++k) {
        double f = (double)k * fs / (double)nt;
        if (f >= f_lo && f <= f_hi) {
            if (bins && n < cap) bins[n] = k;
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------ transforms -- */

/* Eq. 1, F_t: direct DFT of each channel at each selected bin. The angle index
 * (k*t) mod nt is exact integer arithmetic, so every twiddle is cos/sin of
 * 2*pi*m/nt with 0 <= m < nt. */
void pam_oracle_time_dft(const float *rf, int n_elem, int nt, const int *bins,
                         int n_bins, double *S)
{
    double sign = MUT(7) ? +1.0 : -1.0;
    for (int b = 0; b < n_bins; ++b) {
        long long k = bins[b];
        for (int e = 0; e < n_elem; ++e) {
            double re = 0.0, im = 0.0;
            for (int t = 0; t < nt; ++t) {
                long long m = (k * (long long)t) % nt;
                double ang = 2.0 * M_PI * (double)m / (double)nt;
                double x = (double)rf[(size_t)e * nt + t];
                re += x * cos(ang);
                im += sign * x * sin(ang);
            }
            S[((size_t)b * n_elem + e) * 2 + 0] = re;
            S[((size_t)b * n_elem + e) * 2 + 1] = im;
        }
    }
}

/* Eq. 1, F_x: apodize along the elements, then a direct DFT over the element
 * index. */
void pam_oracle_lateral_dft(const double *S_row, const double *apod, int n_elem,
                            int nx, double *Q)
{
    for (int u = 0; u < nx; ++u) {
        double re = 0.0, im = 0.0;
        for (int e = 0; e < n_elem; ++e) {
            double a = apod ? apod[e] : 1.0;
            long long m = ((long long)u * e) % nx;
            double ang = -2.0 * M_PI * (double)m / (double)nx;
            double c = cos(ang), s = sin(ang);
            double xr = a * S_row[2 * e], xi = a * S_row[2 * e + 1];
            re += xr * c - xi * s;
            im += xr * s + xi * c;
        }
        Q[2 * u] = re;
        Q[2 * u + 1] = im;
    }
}

/* Eq. 2 wavenumbers. Lateral bin u holds the spatial frequency u' = u for
 * u < nx/2 and u - nx otherwise (FFT order, Nyquist negative):
 * kx = 2*pi*u'/(nx*pitch). kz = sqrt((w/c)^2 - kx^2), principal branch. */
void pam_oracle_kz(double f_hz, double c, double pitch, int nx, int u,
                   double *kx, double *kz_re, double *kz_im)
{
    int up = u;
    if (!MUT(3) && 2 * u >= nx) up = u - nx;
    double kxv = 2.0 * M_PI * (double)up / ((double)nx * pitch);
    double k = 2.0 * M_PI * f_hz / c;
    double d = k * k - kxv * kxv;
    if (kx) *kx = kxv;
    if (d >= 0.0) { *kz_re = sqrt(d); *kz_im = 0.0; }
    else          { *kz_re = 0.0;     *kz_im = sqrt(-d); }
}

/* Eq. 2: P = Q * exp(i kz dz) with complex kz = kr + i ki, which is
 * exp(-ki dz) * (cos(kr dz) + i sin(kr dz)). */
void pam_oracle_propagate(const double *Q, const double *kz, int nx, double dz,
                          int evanescent_zero, double *P)
{
    double sgn = MUT(1) ? -1.0 : 1.0;
    for (int u = 0; u < nx; ++u) {
        double kr = kz[2 * u], ki = kz[2 * u + 1];
        double amp, ph;
        int drop = evanescent_zero && (MUT(13) ? ki == 0.0 : ki > 0.0);
        if (MUT(14)) drop = 0;
        if (drop) { amp = 0.0; ph = 0.0; }
        else { amp = exp(-ki * dz); ph = sgn * kr * dz; }
        double c = amp * cos(ph), s = amp * sin(ph);
        double qr = Q[2 * u], qi = Q[2 * u + 1];
        P[2 * u] = qr * c - qi * s;
        P[2 * u + 1] = qr * s + qi * c;
    }
}

/* Inverse lateral DFT back to the element grid, with the 1/nx factor. */
void pam_oracle_lateral_idft(const double *P, int nx, double *p)
{
    double scale = MUT(2) ? 1.0 : 1.0 / (double)nx;
    for (int i = 0; i < nx; ++i) {
        double re = 0.0, im = 0.0;
        for (int u = 0; u < nx; ++u) {
            long long m = ((long long)u * i) % nx;
            double ang = 2.0 * M_PI * (double)m / (double)nx;
            double c = cos(ang), s = sin(ang);
            re += P[2 * u] * c - P[2 * u + 1] * s;
            im += P[2 * u] * s + P[2 * u + 1] * c;
        }
        p[2 * i] = re * scale;
        p[2 * i + 1] = im * scale;
    }
}

static int geom_ok(const pam_oracle_geom *g)
{
    if (!g || g->n_elem <= 0 || g->nt <= 1 || g->nz <= 0 || g->n_bins <= 0 || !g->bins)
        return 0;
    if (g->nx != g->n_elem) return 0;
    if (!(g->pitch > 0) || !(g->fs > 0) || !(g->c > 0) || !(g->z0 >= 0) || !(g->dz > 0)) return 0;
    for (int b = 0; b < g->n_bins; ++b)
        if (g->bins[b] <= 0 || 2 * g->bins[b] >= g->nt) return 0;
    return 1;
}

/* kz for every lateral bin u of one frequency bin. */
static void kz_row(const pam_oracle_geom *g, int k, double *kz)
{
    double f = (double)k * g->fs / (double)g->nt;
    for (int u = 0; u < g->nx; ++u)
        pam_oracle_kz(f, g->c, g->pitch, g->nx, u, NULL, &kz[2 * u], &kz[2 * u + 1]);
}

/* ---------------------------------------------------------------- fields -- */

/* p~(x_i, z_j, w_b) for one apodization: F_t, apodize, F_x, Eq. 2 from the
 * array face to z_j, inverse F_x. */
int pam_oracle_fields(const pam_oracle_geom *g, const float *rf, const double *apod,
                      double *fields)
{
    if (!geom_ok(g) || !rf || !fields) return -1;
    int ne = g->n_elem, nx = g->nx;
    double *S = malloc(sizeof(double) * 2 * ne * g->n_bins);
    double *Q = malloc(sizeof(double) * 2 * nx);
    double *P = malloc(sizeof(double) * 2 * nx);
    double *kz = malloc(sizeof(double) * 2 * nx);
    if (!S || !Q || !P || !kz) { free(S); free(Q); free(P); free(kz); return -2; }
    pam_oracle_time_dft(rf, ne, g->nt, g->bins, g->n_bins, S);
    for (int b = 0; b < g->n_bins; ++b) {
        pam_oracle_lateral_dft(S + (size_t)b * ne * 2, apod, ne, nx, Q);
        kz_row(g, g->bins[b], kz);
        for (int j = 0; j < g->nz; ++j) {
            double z = g->z0 + (double)j * g->dz;
            pam_oracle_propagate(Q, kz, nx, z, g->evanescent_zero, P);
            pam_oracle_lateral_idft(P, nx, fields + (((size_t)b * g->nz + j) * nx) * 2);
        }
    }
    free(S); free(Q); free(P); free(kz);
    return 0;
}

/* ------------------------------------------------------- threaded sums -- */

/* One worker sums the per-pixel quantities over its share of the bins:
 *   A_qq = sum |p_q|^2,  C_qr = Re sum conj(p_q) p_r,  E = sum |sum_q p_q|^2. */
typedef struct {
    const pam_oracle_geom *g;
    const double *S;      /* [n_bins][n_elem][2] */
    const double *apod;   /* [n_apod][n_elem] or NULL (one all-ones aperture) */
    int n_apod;
    int b_begin, b_end;
    double *acc;          /* [7][nz][nx] */
    int status;
} worker_t;

static void *worker_run(void *arg)
{
    worker_t *w = (worker_t *)arg;
    const pam_oracle_geom *g = w->g;
    int ne = g->n_elem, nx = g->nx, nz = g->nz, na = w->n_apod;
    size_t npix = (size_t)nz * nx;
    double *Q = malloc(sizeof(double) * 2 * nx * na);
    double *P = malloc(sizeof(double) * 2 * nx);
    double *p = malloc(sizeof(double) * 2 * nx * na);
    double *kz = malloc(sizeof(double) * 2 * nx);
    if (!Q || !P || !p || !kz) { w->status = -2; free(Q); free(P); free(p); free(kz); return NULL; }
    for (int b = w->b_begin; b < w->b_end; ++b) {
        for (int q = 0; q < na; ++q)
            pam_oracle_lateral_dft(w->S + (size_t)b * ne * 2,
                                   w->apod ? w->apod + (size_t)q * ne : NULL, ne, nx,
                                   Q + (size_t)q * nx * 2);
        kz_row(g, g->bins[b], kz);
        for (int j = 0; j < nz; ++j) {
            double z = g->z0 + (double)j * g->dz;
            for (int q = 0; q < na; ++q) {
                pam_oracle_propagate(Q + (size_t)q * nx * 2, kz, nx, z, g->evanescent_zero, P);
                pam_oracle_lateral_idft(P, nx, p + (size_t)q * nx * 2);
            }
            for (int i = 0; i < nx; ++i) {
                size_t px = (size_t)j * nx + i;
                double sr = 0.0, si = 0.0;
                for (int q = 0; q < na; ++q) {
                    double re = p[((size_t)q * nx + i) * 2], im = p[((size_t)q * nx + i) * 2 + 1];
                    w->acc[q * npix + px] += re * re + im * im;
                    sr += re;
                    si += im;
                }
                /* pairs (1,2), (2,3), (3,1) in slots 3, 4, 5 */
                for (int s = 0; s < 3 && na >= 2; ++s) {
                    int q = s, r = (s + 1) % na;
                    if (na == 2 && s > 0) break;
                    double qr = p[((size_t)q * nx + i) * 2], qi = p[((size_t)q * nx + i) * 2 + 1];
                    double rr = p[((size_t)r * nx + i) * 2], ri = p[((size_t)r * nx + i) * 2 + 1];
                    w->acc[(3 + s) * npix + px] += qr * rr + qi * ri;
                }
                if (MUT(5)) {
                    double e = 0.0;
                    for (int q = 0; q < na; ++q) {
                        double re = p[((size_t)q * nx + i) * 2], im = p[((size_t)q * nx + i) * 2 + 1];
                        e += re * re + im * im;
                    }
                    w->acc[6 * npix + px] += e;
                } else {
                    w->acc[6 * npix + px] += sr * sr + si * si;
                }
            }
        }
    }
    free(Q); free(P); free(p); free(kz);
    w->status = 0;
    return NULL;
}

/* Runs the workers over contiguous bin ranges and adds their partial sums in
 * worker order into acc [7][nz][nx]. */
static int sum_over_bins(const pam_oracle_geom *g, const float *rf, const double *apod,
                         int n_apod, double *acc, int n_threads)
{
    int ne = g->n_elem;
    size_t npix = (size_t)g->nz * g->nx;
    if (n_threads <= 0) n_threads = 1;
    if (n_threads > g->n_bins) n_threads = g->n_bins;
    double *S = malloc(sizeof(double) * 2 * ne * g->n_bins);
    worker_t *w = calloc((size_t)n_threads, sizeof(worker_t));
    pthread_t *th = calloc((size_t)n_threads, sizeof(pthread_t));
    double *part = calloc((size_t)n_threads * 7 * npix, sizeof(double));
    if (!S || !w || !th || !part) { free(S); free(w); free(th); free(part); return -2; }
    pam_oracle_time_dft(rf, ne, g->nt, g->bins, g->n_bins, S);
    for (int t = 0; t < n_threads; ++t) {
        w[t].g = g; w[t].S = S; w[t].apod = apod; w[t].n_apod = n_apod;
        w[t].b_begin = (int)((long long)g->n_bins * t / n_threads);
        w[t].b_end = (int)((long long)g->n_bins * (t + 1) / n_threads);
        w[t].acc = part + (size_t)t * 7 * npix;
        w[t].status = -1;
    }
    int rc = 0;
    if (n_threads == 1) {
        worker_run(&w[0]);
    } else {
        int started = 0;
        for (int t = 0; t < n_threads; ++t) {
            if (pthread_create(&th[t], NULL, worker_run, &w[t]) != 0) { rc = -3; break; }
            ++started;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < n_threads && rc == 0; ++t)
        if (w[t].status != 0) rc = w[t].status;
    memset(acc, 0, sizeof(double) * 7 * npix);
    for (int t = 0; t < n_threads && rc == 0; ++t)
        for (size_t x = 0; x < 7 * npix; ++x) acc[x] += part[(size_t)t * 7 * npix + x];
    free(S); free(w); free(th); free(part);
    return rc;
}

/* ------------------------------------------------------------- images -- */

/* Eq. 3: I(r) = sum over w in Omega of |p~(r, w)|^2. */
int pam_oracle_as_backprop(const pam_oracle_geom *g, const float *rf, const double *apod,
                           double *energy, int n_threads)
{
    if (!geom_ok(g) || !rf || !energy) return -1;
    size_t npix = (size_t)g->nz * g->nx;
    double *acc = malloc(sizeof(double) * 7 * npix);
    if (!acc) return -2;
    int rc = sum_over_bins(g, rf, apod, 1, acc, n_threads);
    if (rc == 0) memcpy(energy, acc, sizeof(double) * npix);
    free(acc);
    return rc;
}

/* Eq. 4 with the Appendix A completion: real NCC of apertures q and r, clamped
 * at eps (Sec. II-A). A zero denominator gives eps. */
static double ncc(double Cqr, double Aqq, double Arr, double eps)
{
    double den = MUT(4) ? Aqq * Arr : sqrt(Aqq * Arr);
    double rho = (den > 0.0) ? Cqr / den : eps;
    return rho < eps ? eps : rho;
}

/* AS-DAX (Eq. 4-5) and AS-TAX (Eq. 4, 10, 11). */
int pam_oracle_as_xcorr(const pam_oracle_geom *g, const float *rf, int n_apod,
                        const double *apod, double eps, double *image, double *rho_n,
                        double *rho_pairs, double *image_as, double *acc_out, int n_threads)
{
    if (!geom_ok(g) || !rf || !apod || !image || (n_apod != 2 && n_apod != 3)) return -1;
    if (!(eps > 0.0)) return -1;
    size_t npix = (size_t)g->nz * g->nx;
    double *acc = malloc(sizeof(double) * 7 * npix);
    double *rho = malloc(sizeof(double) * npix);
    if (!acc || !rho) { free(acc); free(rho); return -2; }
    int rc = sum_over_bins(g, rf, apod, n_apod, acc, n_threads);
    if (rc != 0) { free(acc); free(rho); return rc; }
    const double *A11 = acc, *A22 = acc + npix, *A33 = acc + 2 * npix;
    const double *C12 = acc + 3 * npix, *C23 = acc + 4 * npix, *C31 = acc + 5 * npix;
    const double *E = acc + 6 * npix;
    double rmax = 0.0;
    for (size_t x = 0; x < npix; ++x) {
        double r;
        if (n_apod == 2) {
            r = ncc(C12[x], A11[x], A22[x], eps);
            if (rho_pairs) rho_pairs[x] = r;
        } else {
            double r12, r23, r31;
            if (MUT(8)) {
                double d12 = sqrt(A11[x] * A22[x]), d23 = sqrt(A22[x] * A33[x]), d31 = sqrt(A33[x] * A11[x]);
                r12 = d12 > 0 ? C12[x] / d12 : eps;
                r23 = d23 > 0 ? C23[x] / d23 : eps;
                r31 = d31 > 0 ? C31[x] / d31 : eps;
            } else {
                r12 = ncc(C12[x], A11[x], A22[x], eps);
                r23 = ncc(C23[x], A22[x], A33[x], eps);
                r31 = ncc(C31[x], A33[x], A11[x], eps);
            }
            if (rho_pairs) {
                rho_pairs[x] = r12;
                rho_pairs[npix + x] = r23;
                rho_pairs[2 * npix + x] = r31;
            }
            /* Eq. 10: cube root of the product of the three pair NCCs. */
            r = MUT(6) ? sqrt(r12 * r23) : cbrt(r12 * r23 * r31);
            if (MUT(8) && r < eps) r = eps;
        }
        rho[x] = r;
        if (r > rmax) rmax = r;
    }
    double mean = 0.0;
    for (size_t x = 0; x < npix; ++x) mean += rho[x];
    mean /= (double)npix;
    for (size_t x = 0; x < npix; ++x) {
        /* rho_n: divide by the maximum of the frame (Sec. II-A). */
        double rn = rho[x] / (MUT(10) ? mean : rmax);
        if (rho_n) rho_n[x] = rn;
        /* Eq. 5 / Eq. 11 */
        image[x] = rn * rn * E[x];
        if (image_as) image_as[x] = E[x];
    }
    if (acc_out) {
        memcpy(acc_out, acc, sizeof(double) * 7 * npix);
        if (n_apod == 2) memset(acc_out + 2 * npix, 0, sizeof(double) * npix);
        if (n_apod == 2) memset(acc_out + 4 * npix, 0, sizeof(double) * 2 * npix);
    }
    free(acc); free(rho);
    return 0;
}
