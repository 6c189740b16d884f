/*
 * pa_oracle.h -- plain FP64 CPU oracle for higher-order DMAS photoacoustic
 * beamforming (Mulani, Paul, Singh, "Higher-order correlation based
 * real-time beamforming in photoacoustic imaging", arXiv 2203.14906).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The CUDA product path
 * neither includes this header nor links this code; the two share no code,
 * tables or constants.
 *
 * Every function is a direct, unblocked statement of the operation it
 * names, in double precision, with the passage of the paper it follows.
 * Conventions the paper leaves open are stated beside each function.
 */
#ifndef PA_ORACLE_H
#define PA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_elem;      /* N: array elements                                  */
  double pitch_m;      /* element pitch; element i at x=(i-(N-1)/2)*pitch    */
  double c_m_s;        /* speed of sound                                     */
  double fs_hz;        /* RF sampling rate                                   */
  double t0_s;         /* time of the first RF sample after the laser shot  */
  int32_t n_samples;   /* Ns: samples per channel                            */
  int32_t nx, nz;      /* image grid (lateral x depth), pixel centres        */
  double x0_m, x1_m;   /* lateral extent                                     */
  double z0_m, z1_m;   /* depth extent                                       */
  int32_t order_k;     /* correlation order of the HO-DMAS output (1..8)     */
  double f_number;     /* 0: full aperture; >0: dynamic aperture + Hann      */
  double f0_hz;        /* pulse centre frequency (post-filter band)          */
  double band_lo_hz;   /* <=0 (with band_hi>=0): parity-dependent default    */
  double band_hi_hz;   /* <0: band-pass off (analytic mask only)            */
  double dyn_range_db; /* log-compression dynamic range                      */
  int32_t nearest;     /* 1: integer delays as Eq. 1 writes them (no interp.) */
} or_desc;

/* ---- geometry and delay (Eq. 1 and Section 2.1) ---- */
double or_elem_x(const or_desc* d, int i);
double or_pix_x(const or_desc* d, int j);
double or_pix_z(const or_desc* d, int l);
/* One-way time of flight from pixel (j,l) to element i, in samples. */
double or_delay(const or_desc* d, int i, int j, int l);
/* Linear interpolation of row[] at fractional index tau; 0 when either tap
 * lies outside [0, ns-1] (such a channel contributes nothing). */
double or_lerp(const double* row, int ns, double tau);
/* Nearest sample of row[] at fractional index tau: the integer delay of
 * Eq. 1, n = floor(tau + 1/2) (halves round up); 0 unless 0 <= n <= ns-1. */
double or_nearest(const double* row, int ns, double tau);
/* The delayed sample of one channel: or_nearest when d->nearest, else
 * or_lerp. */
double or_sample(const or_desc* d, const double* row, double tau);
/* Dynamic-aperture Hann weight (1 when f_number <= 0). */
double or_apod(const or_desc* d, int i, int j, int l);

/* ---- roots, power sums, elementary symmetric sums (Eqs. 2-9) ---- */
/* Signed real k-th root sgn(s)|s|^(1/k) (Eqs. 2, 5; real odd root Eqs. 4, 6). */
double or_root(double s, int k);
/* p[m] = sum_i x_i^m for m = 0..k (p[0] = n). */
void or_power_sums(const double* x, int n, int k, double* p);
/* Newton's identities: e[0..k] from p[1..k]. */
void or_newton(const double* p, int k, double* e);
/* The paper's explicit O(N) forms in the raw signals s_i:
 * k=1 Eq. 1, k=2 Eq. 3, k=3 Eq. 7, k=4 Eq. 8, k=5 Eq. 9; NaN otherwise. */
double or_paper_form(const double* s, int n, int k);
/* Definition: sum over all k-subsets of the signed k-th root of the product
 * (Eq. 2 for k=2, Eqs. 4-6 for k=3..5).  O(N^k): tiny apertures only. */
double or_bruteforce(const double* s, int n, int k);
/* DMAS-k of one pixel's delayed signals via root -> power sums -> Newton. */
double or_dmas_k(const double* s, int n, int k);

/* ---- full beamformer on one frame rf[N][Ns] ---- */
/* Writes [nx][nz] images (z fastest).  Any output pointer may be NULL. */
void or_beamform(const or_desc* d, const double* rf, double* das,
                 double* dmas, double* ho);
/* Same, but only for the pixels listed (j[q], l[q]); outputs are [q]. */
void or_beamform_pixels(const or_desc* d, const double* rf, int nq,
                        const int32_t* j, const int32_t* l, double* das,
                        double* dmas, double* ho);
/* HO output by the k-subset definition (or_bruteforce); tiny N only. */
void or_beamform_bruteforce(const or_desc* d, const double* rf, double* ho);

/* ---- post-processing (Section 3: band-pass, Hilbert envelope, log) ---- */
int or_fft_size(int nz); /* M = 2^ceil(log2 nz) */
/* In-place radix-2 FFT; inverse includes the 1/M factor.  Returns 0 on
 * success, -1 if M is not a power of two. */
int or_fft(double* re, double* im, int m, int inverse);
/* Direct O(M^2) DFT (self-check of or_fft). */
void or_dft(const double* re, const double* im, int m, int inverse,
            double* out_re, double* out_im);
/* Equivalent temporal frequency of depth bin b (one-way, z = c t). */
double or_bin_hz(const or_desc* d, int m, int b);
/* H[b] = band-pass(f_b) * analytic mask, b in [0, M).  even_order selects
 * the band around 2 f0 (even orders rectify the signal).  Returns 1 if the
 * band lies wholly above the axial Nyquist rate (DC removal only). */
int or_post_mask(const or_desc* d, int even_order, int m, double* h);
/* env[z] = |IFFT(H . FFT(col zero-padded to M))|[z], z < nz. */
void or_envelope(const double* col, int nz, int m, const double* h,
                 double* env);
/* Envelope of every column of a [nx][nz] image. */
void or_envelope_image(const or_desc* d, int even_order, const double* raw,
                       double* env);
/* out = clip(20 log10(env / max env), -dr, 0); all -dr if max is 0. */
void or_log_image(const double* env, int64_t n, double dr_db, double* out);

/* ---- threading (OpenMP over image columns; 1 if built without it) ---- */
void or_set_threads(int n);
int or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif /* PA_ORACLE_H */
