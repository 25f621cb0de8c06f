/*
 * pam_oracle.h -- plain FP64 CPU oracle for cross-correlated angular-spectrum
 * passive acoustic mapping (AS, AS-DAX, AS-TAX; arXiv 2412.02413).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may call this library. The GPU library neither links nor
 * includes it; the two share no header, helper or table.
 *
 * Conventions (the paper's Eq. 1-4, 10, 11 and the readings listed with each
 * function in pam_oracle.c):
 *   rf        float32 [n_elem][nt], channel-major, one frame.
 *   complex   interleaved doubles (re, im).
 *   element e sits at x_e = (e - (n_elem-1)/2) * pitch; the lateral DFT runs
 *             over the element index with length nx == n_elem; pixel column i
 *             is element position x_i.
 *   depth     row j is at z_j = z0 + j*dz, measured from the array face.
 */
#ifndef PAM_ORACLE_H
#define PAM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_elem;          /* channels */
    int nt;              /* samples per channel */
    int nx;              /* lateral DFT length (== n_elem) */
    int nz;              /* depth rows */
    int n_bins;          /* number of selected DFT bins */
    const int *bins;     /* selected bins k, 0 < k < nt/2 */
    double pitch;        /* element pitch, m */
    double fs;           /* sampling rate, Hz */
    double c;            /* sound speed, m/s */
    double z0;           /* first depth, m (>= 0) */
    double dz;           /* depth step, m */
    int evanescent_zero; /* 1: drop kx^2 > (w/c)^2 components; 0: decay them */
} pam_oracle_geom;

/* Pattern-m complementary apodization: element e is active in aperture q
 * (0-based) iff floor(e/m) mod n_apod == q. apod is [n_apod][n_elem]. */
int pam_oracle_pattern(int n_elem, int n_apod, int m, double *apod);

/* Every bin k with f_lo <= k*fs/nt <= f_hi and 0 < k < nt/2, ascending.
 * Returns the count (bins written up to cap). */
int pam_oracle_band_bins(int nt, double fs, double f_lo, double f_hi, int *bins, int cap);

/* Direct time DFT (Eq. 1, F_t): S[b][e] = sum_t rf[e][t] exp(-2 pi i k_b t / nt). */
void pam_oracle_time_dft(const float *rf, int n_elem, int nt, const int *bins,
                         int n_bins, double *S /* [n_bins][n_elem][2] */);

/* Apodized lateral DFT (Eq. 1, F_x): Q[u] = sum_e apod[e] S[e] exp(-2 pi i u e / nx). */
void pam_oracle_lateral_dft(const double *S_row /* [n_elem][2] */, const double *apod,
                            int n_elem, int nx, double *Q /* [nx][2] */);

/* kx of lateral bin u and kz = sqrt((w/c)^2 - kx^2) on the principal branch
 * (kz = i*kappa for evanescent components). */
void pam_oracle_kz(double f_hz, double c, double pitch, int nx, int u,
                   double *kx, double *kz_re, double *kz_im);

/* Spectral propagator (Eq. 2): P[u] = Q[u] exp(i kz[u] dz). */
void pam_oracle_propagate(const double *Q, const double *kz /* [nx][2] */, int nx,
                          double dz, int evanescent_zero, double *P);

/* Inverse lateral DFT: p[i] = (1/nx) sum_u P[u] exp(+2 pi i u i / nx). */
void pam_oracle_lateral_idft(const double *P, int nx, double *p);

/* Monochromatic fields of one apodization (apod NULL = all ones):
 * fields[b][j][i] = p~(x_i, z_j, w_b), complex. */
int pam_oracle_fields(const pam_oracle_geom *g, const float *rf, const double *apod,
                      double *fields /* [n_bins][nz][nx][2] */);

/* AS energy map (Eq. 3) of one apodization (apod NULL = all ones). */
int pam_oracle_as_backprop(const pam_oracle_geom *g, const float *rf, const double *apod,
                           double *energy /* [nz][nx] */, int n_threads);

/* AS-DAX (n_apod = 2, Eq. 5) or AS-TAX (n_apod = 3, Eq. 10-11).
 * image [nz][nx]; rho_n [nz][nx] or NULL; rho_pairs [n_pairs][nz][nx] or NULL
 * (pairs (1,2) for DAX; (1,2),(2,3),(3,1) for TAX); image_as [nz][nx] or NULL
 * (sum over bins of |sum_q p_q|^2); acc [7][nz][nx] or NULL (A11, A22, A33,
 * C12, C23, C31, E_full; unused slots zero). */
int pam_oracle_as_xcorr(const pam_oracle_geom *g, const float *rf, int n_apod,
                        const double *apod /* [n_apod][n_elem] */, double eps,
                        double *image, double *rho_n, double *rho_pairs,
                        double *image_as, double *acc, int n_threads);

/* Test hook: selects a deliberate mistake (0 = none) so that the test suite can
 * show that its pins catch it. Never set outside those tests. */
void pam_oracle_set_mutation(int id);

#ifdef __cplusplus
}
#endif
#endif
