/*
 * pa_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Straight-line statements of the paper's definitions in double precision.
 * Parallelism is only across independent image columns (OpenMP), which
 * changes no arithmetic.  Nothing here is shared with the CUDA path.
 */
#include "pa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Geometry and delay (Section 2.1, Eq. 1: s_i[k + Delta_i]).           */
/* ------------------------------------------------------------------ */

double or_elem_x(const or_desc* d, int i) {
  /* Linear array centred on x = 0 (convention; the paper gives none). */
  return ((double)i - 0.5 * (double)(d->n_elem - 1)) * d->pitch_m;
}

double or_pix_x(const or_desc* d, int j) {
  return d->x0_m + ((double)j + 0.5) * (d->x1_m - d->x0_m) / (double)d->nx;
}

double or_pix_z(const or_desc* d, int l) {
  return d->z0_m + ((double)l + 0.5) * (d->z1_m - d->z0_m) / (double)d->nz;
}

double or_delay(const or_desc* d, int i, int j, int l) {
  /* Photoacoustic reception is one-way: the wave leaves the pixel at the
   * laser shot and reaches element i after r / c. */
  double dx = or_pix_x(d, j) - or_elem_x(d, i);
  double z = or_pix_z(d, l);
  double r = sqrt(dx * dx + z * z);
  return d->fs_hz * (r / d->c_m_s - d->t0_s);
}

double or_lerp(const double* row, int ns, double tau) {
  double fl = floor(tau);
  if (fl < 0.0 || fl + 1.0 > (double)(ns - 1)) return 0.0;
  int n0 = (int)fl;
  double a = tau - fl;
  return row[n0] + a * (row[n0 + 1] - row[n0]);
}

double or_nearest(const double* row, int ns, double tau) {
  double n = floor(tau + 0.5);
  if (n < 0.0 || n > (double)(ns - 1)) return 0.0;
  return row[(int)n];
}

double or_sample(const or_desc* d, const double* row, double tau) {
  return d->nearest ? or_nearest(row, d->n_samples, tau)
                    : or_lerp(row, d->n_samples, tau);
}

double or_apod(const or_desc* d, int i, int j, int l) {
  if (d->f_number <= 0.0) return 1.0;
  double z = or_pix_z(d, l);
  double half = z / (2.0 * d->f_number); /* active half-aperture */
  if (!(half > 0.0)) return 0.0;
  double dx = or_elem_x(d, i) - or_pix_x(d, j);
  if (fabs(dx) > half) return 0.0;
  double cw = cos(M_PI * dx / (2.0 * half)); /* Hann over the aperture */
  return cw * cw;
}

/* ------------------------------------------------------------------ */
/* Roots, power sums and elementary symmetric sums (Eqs. 2-9).         */
/* ------------------------------------------------------------------ */

double or_root(double s, int k) {
  if (s == 0.0) return 0.0;
  if (k == 1) return s;
  /* Signed root: Eq. 2 and Eq. 5 write sign(.)|.|^(1/k) explicitly; for odd
   * k (Eqs. 4, 6) the real root of a negative number has the same value. */
  return copysign(pow(fabs(s), 1.0 / (double)k), s);
}

void or_power_sums(const double* x, int n, int k, double* p) {
  p[0] = (double)n;
  for (int m = 1; m <= k; ++m) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += pow(x[i], (double)m);
    p[m] = acc;
  }
}

void or_newton(const double* p, int k, double* e) {
  /* m e_m = sum_{i=1}^{m} (-1)^(i-1) e_{m-i} p_i  (Newton's identities). */
  e[0] = 1.0;
  for (int m = 1; m <= k; ++m) {
    double acc = 0.0;
    for (int i = 1; i <= m; ++i) {
      double term = e[m - i] * p[i];
      acc += (i % 2 == 1) ? term : -term;
    }
    e[m] = acc / (double)m;
  }
}

double or_paper_form(const double* s, int n, int k) {
  if (k == 1) { /* Eq. 1 */
    double das = 0.0;
    for (int i = 0; i < n; ++i) das += s[i];
    return das;
  }
  if (k == 2) { /* Eq. 3 */
    double a = 0.0, b = 0.0;
    for (int i = 0; i < n; ++i) {
      a += copysign(sqrt(fabs(s[i])), s[i]);
      b += fabs(s[i]);
    }
    return (a * a - b) / 2.0;
  }
  if (k == 3) { /* Eq. 7 with c_i = cbrt(s_i) */
    double sc = 0.0, sc2 = 0.0, ss = 0.0;
    for (int i = 0; i < n; ++i) {
      double c = cbrt(s[i]);
      sc += c;
      sc2 += c * c;
      ss += s[i];
    }
    return (sc * sc * sc + 2.0 * ss - 3.0 * sc * sc2) / 6.0;
  }
  if (k == 4) { /* Eq. 8 with q_i = sign(s_i)|s_i|^(1/4) */
    double sq = 0.0, sq3 = 0.0, sr = 0.0, sa = 0.0;
    for (int i = 0; i < n; ++i) {
      double a = fabs(s[i]);
      double q = copysign(pow(a, 0.25), s[i]);
      sq += q;
      sq3 += copysign(pow(pow(a, 0.25), 3.0), s[i]);
      sr += sqrt(a);
      sa += a;
    }
    return (pow(sq, 4.0) - 6.0 * sa + 3.0 * sr * sr - 6.0 * sr * sq * sq +
            8.0 * sq3 * sq) / 24.0;
  }
  if (k == 5) { /* Eq. 9 with f_i = s_i^(1/5) (real root) */
    double f1 = 0.0, f2 = 0.0, f3 = 0.0, f4 = 0.0, ss = 0.0;
    for (int i = 0; i < n; ++i) {
      double f = copysign(pow(fabs(s[i]), 0.2), s[i]);
      f1 += f;
      f2 += f * f;
      f3 += f * f * f;
      f4 += f * f * f * f;
      ss += s[i];
    }
    return (pow(f1, 5.0) + 24.0 * ss - 30.0 * f1 * f4 + 20.0 * f3 * f1 * f1 -
            20.0 * f3 * f2 + 15.0 * f2 * f2 * f1 - 10.0 * f2 * f1 * f1 * f1) /
           120.0;
  }
  return NAN;
}

double or_bruteforce(const double* s, int n, int k) {
  if (k < 1 || k > n) return 0.0;
  int idx[16];
  if (k > 16) return NAN;
  for (int t = 0; t < k; ++t) idx[t] = t;
  double acc = 0.0;
  for (;;) {
    double prod = 1.0;
    for (int t = 0; t < k; ++t) prod *= s[idx[t]];
    acc += or_root(prod, k); /* root of the product, as Eqs. 2, 4-6 write */
    int t = k - 1;
    while (t >= 0 && idx[t] == n - k + t) --t;
    if (t < 0) break;
    ++idx[t];
    for (int u = t + 1; u < k; ++u) idx[u] = idx[u - 1] + 1;
  }
  return acc;
}

double or_dmas_k(const double* s, int n, int k) {
  double x_stack[512];
  double* x = (n <= 512) ? x_stack : (double*)malloc(sizeof(double) * n);
  double p[17], e[17];
  if (k > 16) return NAN;
  for (int i = 0; i < n; ++i) x[i] = or_root(s[i], k);
  or_power_sums(x, n, k, p);
  or_newton(p, k, e);
  if (x != x_stack) free(x);
  return e[k];
}

/* ------------------------------------------------------------------ */
/* Beamformer: delay -> interpolate -> apodise -> DAS / DMAS / DMAS-k. */
/* ------------------------------------------------------------------ */

static void pixel(const or_desc* d, const double* rf, int j, int l,
                  double* s_buf, double* das, double* dmas, double* ho) {
  int n = d->n_elem, ns = d->n_samples;
  for (int i = 0; i < n; ++i) {
    double tau = or_delay(d, i, j, l);
    double s = or_sample(d, rf + (int64_t)i * ns, tau);
    s_buf[i] = or_apod(d, i, j, l) * s;
  }
  if (das) *das = or_paper_form(s_buf, n, 1);
  if (dmas) *dmas = or_paper_form(s_buf, n, 2);
  if (ho) *ho = or_dmas_k(s_buf, n, d->order_k);
}

void or_beamform(const or_desc* d, const double* rf, double* das,
                 double* dmas, double* ho) {
  int nx = d->nx, nz = d->nz;
#pragma omp parallel
  {
    double* s_buf = (double*)malloc(sizeof(double) * (size_t)d->n_elem);
#pragma omp for schedule(dynamic)
    for (int j = 0; j < nx; ++j) {
      for (int l = 0; l < nz; ++l) {
        int64_t q = (int64_t)j * nz + l;
        pixel(d, rf, j, l, s_buf, das ? das + q : NULL, dmas ? dmas + q : NULL,
              ho ? ho + q : NULL);
      }
    }
    free(s_buf);
  }
}

void or_beamform_pixels(const or_desc* d, const double* rf, int nq,
                        const int32_t* j, const int32_t* l, double* das,
                        double* dmas, double* ho) {
#pragma omp parallel
  {
    double* s_buf = (double*)malloc(sizeof(double) * (size_t)d->n_elem);
#pragma omp for schedule(dynamic)
    for (int q = 0; q < nq; ++q) {
      pixel(d, rf, j[q], l[q], s_buf, das ? das + q : NULL,
            dmas ? dmas + q : NULL, ho ? ho + q : NULL);
    }
    free(s_buf);
  }
}

void or_beamform_bruteforce(const or_desc* d, const double* rf, double* ho) {
  int n = d->n_elem, ns = d->n_samples;
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  for (int j = 0; j < d->nx; ++j) {
    for (int l = 0; l < d->nz; ++l) {
      for (int i = 0; i < n; ++i) {
        double tau = or_delay(d, i, j, l);
        s[i] = or_apod(d, i, j, l) * or_sample(d, rf + (int64_t)i * ns, tau);
      }
      ho[(int64_t)j * d->nz + l] = or_bruteforce(s, n, d->order_k);
    }
  }
  free(s);
}

/* ------------------------------------------------------------------ */
/* Post-processing (Section 3): band-pass, Hilbert envelope, log.      */
/* ------------------------------------------------------------------ */

int or_fft_size(int nz) {
  int m = 1;
  while (m < nz) m <<= 1;
  return m;
}

int or_fft(double* re, double* im, int m, int inverse) {
  if (m < 1 || (m & (m - 1)) != 0) return -1;
  /* bit-reversal permutation */
  for (int i = 1, j = 0; i < m; ++i) {
    int bit = m >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
  /* iterative Cooley-Tukey butterflies; e^{-2 pi i/len} forward */
  for (int len = 2; len <= m; len <<= 1) {
    double ang = (inverse ? 2.0 : -2.0) * M_PI / (double)len;
    for (int i = 0; i < m; i += len) {
      for (int k = 0; k < len / 2; ++k) {
        double wr = cos(ang * k), wi = sin(ang * k);
        int a = i + k, b = i + k + len / 2;
        double tr = re[b] * wr - im[b] * wi;
        double ti = re[b] * wi + im[b] * wr;
        re[b] = re[a] - tr;
        im[b] = im[a] - ti;
        re[a] += tr;
        im[a] += ti;
      }
    }
  }
  if (inverse) {
    for (int i = 0; i < m; ++i) {
      re[i] /= (double)m;
      im[i] /= (double)m;
    }
  }
  return 0;
}

void or_dft(const double* re, const double* im, int m, int inverse,
            double* out_re, double* out_im) {
  double sgn = inverse ? 1.0 : -1.0;
  for (int b = 0; b < m; ++b) {
    double ar = 0.0, ai = 0.0;
    for (int n = 0; n < m; ++n) {
      double ang = sgn * 2.0 * M_PI * (double)(((int64_t)b * n) % m) / (double)m;
      double c = cos(ang), s = sin(ang);
      ar += re[n] * c - im[n] * s;
      ai += re[n] * s + im[n] * c;
    }
    out_re[b] = inverse ? ar / m : ar;
    out_im[b] = inverse ? ai / m : ai;
  }
}

double or_bin_hz(const or_desc* d, int m, int b) {
  double dz = (d->z1_m - d->z0_m) / (double)d->nz;
  return d->c_m_s * (double)b / ((double)m * dz);
}

static double raised_cos_band(double f, double lo, double hi, double roll) {
  if (f >= lo && f <= hi) return 1.0;
  if (f < lo) {
    double u = lo - f;
    return (u < roll) ? 0.5 * (1.0 + cos(M_PI * u / roll)) : 0.0;
  }
  double u = f - hi;
  return (u < roll) ? 0.5 * (1.0 + cos(M_PI * u / roll)) : 0.0;
}

int or_post_mask(const or_desc* d, int even_order, int m, double* h) {
  /* Band-pass (reading: Section 3 names a band-pass filter but gives no
   * band): a raised-cosine band around f0 for DAS and odd orders, around
   * 2 f0 for even orders, roll-off 0.25 f0 each side, clipped at the axial
   * Nyquist rate c / (2 dz).  Times the analytic-signal mask of the Hilbert
   * transform: 1 at DC and M/2, 2 on positive bins, 0 on negative bins. */
  double dz = (d->z1_m - d->z0_m) / (double)d->nz;
  double f_nyq = d->c_m_s / (2.0 * dz);
  double f0 = d->f0_hz;
  double roll = 0.25 * f0;
  int off = d->band_hi_hz < 0.0;
  double lo, hi;
  if (d->band_lo_hz > 0.0 && d->band_hi_hz > 0.0) {
    lo = d->band_lo_hz;
    hi = d->band_hi_hz;
  } else if (even_order) {
    lo = 1.5 * f0;
    hi = 2.5 * f0;
  } else {
    lo = 0.5 * f0;
    hi = 1.5 * f0;
  }
  int dc_only = (!off) && (lo >= f_nyq);
  if (hi > f_nyq) hi = f_nyq;
  for (int b = 0; b < m; ++b) {
    double analytic = (b == 0 || 2 * b == m) ? 1.0 : (2 * b < m ? 2.0 : 0.0);
    double bp;
    if (analytic == 0.0) {
      bp = 0.0;
    } else if (off) {
      bp = 1.0;
    } else if (dc_only) {
      bp = (b == 0) ? 0.0 : 1.0;
    } else {
      bp = raised_cos_band(or_bin_hz(d, m, b), lo, hi, roll);
    }
    h[b] = bp * analytic;
  }
  return dc_only;
}

void or_envelope(const double* col, int nz, int m, const double* h,
                 double* env) {
  double* re = (double*)calloc((size_t)m, sizeof(double));
  double* im = (double*)calloc((size_t)m, sizeof(double));
  for (int z = 0; z < nz; ++z) re[z] = col[z];
  or_fft(re, im, m, 0);
  for (int b = 0; b < m; ++b) {
    re[b] *= h[b];
    im[b] *= h[b];
  }
  or_fft(re, im, m, 1);
  for (int z = 0; z < nz; ++z) env[z] = sqrt(re[z] * re[z] + im[z] * im[z]);
  free(re);
  free(im);
}

void or_envelope_image(const or_desc* d, int even_order, const double* raw,
                       double* env) {
  int m = or_fft_size(d->nz);
  double* h = (double*)malloc(sizeof(double) * (size_t)m);
  or_post_mask(d, even_order, m, h);
#pragma omp parallel for schedule(dynamic)
  for (int j = 0; j < d->nx; ++j) {
    int64_t q = (int64_t)j * d->nz;
    or_envelope(raw + q, d->nz, m, h, env + q);
  }
  free(h);
}

void or_log_image(const double* env, int64_t n, double dr_db, double* out) {
  double mx = 0.0;
  for (int64_t q = 0; q < n; ++q)
    if (env[q] > mx) mx = env[q];
  for (int64_t q = 0; q < n; ++q) {
    double v = -dr_db;
    if (mx > 0.0 && env[q] > 0.0) {
      v = 20.0 * log10(env[q] / mx);
      if (v < -dr_db) v = -dr_db;
      if (v > 0.0) v = 0.0;
    }
    out[q] = v;
  }
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
