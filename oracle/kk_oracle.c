/*
 * oracle/kk_oracle.c -- FP64 reference image formation for KK and DAS.
 *
 * TEST INFRASTRUCTURE.  This file is part of the slow, plain CPU oracle.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load it.  It shares no code with the CUDA library.
 *
 * Every sum is written out as the paper defines it; the only parallelism is an
 * OpenMP split over output pixels (which does not change any result: each
 * pixel's sum runs in pair order on one thread).
 *
 * Complex arrays are interleaved (re, im) doubles, row-major.
 */
#include <math.h>
#include <stdint.h>

/* Linear interpolation of a complex record y[0..T-1] at fractional sample s:
 * k = floor(s), f = s - k; value (1-f) y[k] + f y[k+1] when 0 <= k and
 * k+1 <= T-1, otherwise 0 (the reading used for the paper's unspecified
 * interpolation, Section II-B). */
static void lerp(const double *y, int T, double s, double *re, double *im) {
  double kf = floor(s);
  if (!(kf >= 0.0) || kf + 1.0 > (double)(T - 1)) {
    *re = 0.0;
    *im = 0.0;
    return;
  }
  long k = (long)kf;
  double f = s - kf;
  *re = (1.0 - f) * y[2 * k] + f * y[2 * (k + 1)];
  *im = (1.0 - f) * y[2 * k + 1] + f * y[2 * (k + 1) + 1];
}

/*
 * KK image formation, Eq. (KK) of Section II-B:
 *   B_j(r) = sum over pairs p=(i,o) in group j of
 *            RF_theta_p( tau_in(r, theta_i) + tau_out(r, theta_o) )
 *   tau_in  = (x sin theta_i + z cos theta_i) / c
 *   tau_out = ((x - xref_o) sin theta_o + z cos theta_o) / c
 * The record y_p[t] holds RF_theta at time t / fs, so the sample position is
 * s = fs * (tau_in + tau_out).  xref_o is the reference lateral position of
 * the shear used for receive angle theta_o (the array end that keeps every
 * shear a non-negative advance, Eq. (compression)); it appears here because
 * the sheared record's time origin sits at that element.
 *
 * y       [P][T] complex
 * sin_i, cos_i, sin_o, cos_o, xref_o : [P] per pair
 * group   [P] in [0, J)
 * pix_x, pix_z : [n_pix] pixel coordinates (m)
 * B       [J][n_pix] complex (overwritten)
 */
int orc_kk_beamform(int P, int T, const double *y, const double *sin_i,
                    const double *cos_i, const double *sin_o,
                    const double *cos_o, const double *xref_o,
                    const int32_t *group, int J, int n_pix,
                    const double *pix_x, const double *pix_z, double fs,
                    double c, const double *w, double *B) {
  if (P < 0 || T < 2 || J < 1 || n_pix < 0) return 1;
  for (int p = 0; p < P; ++p)
    if (group[p] < 0 || group[p] >= J) return 2;
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n_pix; ++q) {
    const double x = pix_x[q], z = pix_z[q];
    for (int j = 0; j < J; ++j) {
      B[2 * ((long)j * n_pix + q)] = 0.0;
      B[2 * ((long)j * n_pix + q) + 1] = 0.0;
    }
    for (int p = 0; p < P; ++p) {
      const double tau_in = (x * sin_i[p] + z * cos_i[p]) / c;
      const double tau_out = ((x - xref_o[p]) * sin_o[p] + z * cos_o[p]) / c;
      double re, im;
      lerp(y + 2L * p * T, T, fs * (tau_in + tau_out), &re, &im);
      const double wp = w ? w[p] : 1.0;
      B[2 * ((long)group[p] * n_pix + q)] += wp * re;
      B[2 * ((long)group[p] * n_pix + q) + 1] += wp * im;
    }
  }
  return 0;
}

/*
 * Receive aperture weight of element offset d = |x - u_l| at depth z for an
 * F-number F (Table 1 lists the F-numbers of the acquisitions; Eq. (DAS) is
 * stated without apodization): half-width h = z / (2 F); boxcar 1 for
 * d <= h, Hann (1 + cos(pi d / h)) / 2 for d <= h, 0 beyond; F <= 0 means the
 * full aperture (weight 1).
 */
static double aperture(double d, double z, double F, int window) {
  if (F <= 0.0) return 1.0;
  const double h = z / (2.0 * F);
  if (!(d <= h)) return 0.0;
  if (window == 0) return 1.0;
  return 0.5 * (1.0 + cos(M_PI * d / h));
}

/*
 * CPWC delay-and-sum, Eq. (DAS) of Section II-B:
 *   B(r) = sum_{i,l} a_l(r) y_il( tau_in(r, theta_i) + |r - (u_l, 0)| / c )
 * with the receive aperture weight a_l(r) above (1 for the full aperture).
 * y   [N][L][T] complex analytic channel data
 * B   [n_pix] complex (overwritten)
 */
int orc_das_beamform(int N, int L, int T, const double *y, const double *sin_i,
                     const double *cos_i, const double *elem_x, int n_pix,
                     const double *pix_x, const double *pix_z, double fs,
                     double c, double f_number, int window, double *B) {
  if (N < 0 || L < 0 || T < 2 || n_pix < 0) return 1;
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n_pix; ++q) {
    const double x = pix_x[q], z = pix_z[q];
    double accr = 0.0, acci = 0.0;
    for (int i = 0; i < N; ++i) {
      const double tau_in = (x * sin_i[i] + z * cos_i[i]) / c;
      for (int l = 0; l < L; ++l) {
        const double dx = x - elem_x[l];
        const double tau_out = sqrt(dx * dx + z * z) / c;
        const double a = aperture(fabs(dx), z, f_number, window);
        double re, im;
        lerp(y + 2L * ((long)i * L + l) * T, T, fs * (tau_in + tau_out), &re, &im);
        accr += a * re;
        acci += a * im;
      }
    }
    B[2 * q] = accr;
    B[2 * q + 1] = acci;
  }
  return 0;
}

/*
 * Volumetric KK image formation with a 2D array: Eq. (KK) with plane waves
 * in three dimensions (the extension to 2D arrays and volumes the paper
 * names in Section IV):
 *   tau_in  = (x sx_i + y sy_i + z sz_i) / c
 *   tau_out = ((x - xref_o) sx_o + (y - yref_o) sy_o + z sz_o) / c
 * (sx, sy, sz) is the unit propagation direction of each plane wave; xref_o,
 * yref_o the corner of the array that keeps the receive shear a
 * non-negative advance in each direction.
 * y [P][T] complex; direction cosines and references [P]; group [P];
 * pix_x, pix_y, pix_z [n_pix]; B [J][n_pix] complex (overwritten).
 */
int orc_kk_beamform_vol(int P, int T, const double *y, const double *sx_i, const double *sy_i,
                        const double *sz_i, const double *sx_o, const double *sy_o,
                        const double *sz_o, const double *xref_o, const double *yref_o,
                        const int32_t *group, int J, int n_pix, const double *pix_x,
                        const double *pix_y, const double *pix_z, double fs, double c,
                        double *B) {
  if (P < 0 || T < 2 || J < 1 || n_pix < 0) return 1;
  for (int p = 0; p < P; ++p)
    if (group[p] < 0 || group[p] >= J) return 2;
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n_pix; ++q) {
    const double x = pix_x[q], yy = pix_y[q], z = pix_z[q];
    for (int j = 0; j < J; ++j) {
      B[2 * ((long)j * n_pix + q)] = 0.0;
      B[2 * ((long)j * n_pix + q) + 1] = 0.0;
    }
    for (int p = 0; p < P; ++p) {
      const double tau_in = (x * sx_i[p] + yy * sy_i[p] + z * sz_i[p]) / c;
      const double tau_out =
          ((x - xref_o[p]) * sx_o[p] + (yy - yref_o[p]) * sy_o[p] + z * sz_o[p]) / c;
      double re, im;
      lerp(y + 2L * p * T, T, fs * (tau_in + tau_out), &re, &im);
      B[2 * ((long)group[p] * n_pix + q)] += re;
      B[2 * ((long)group[p] * n_pix + q) + 1] += im;
    }
  }
  return 0;
}

/*
 * Volumetric CPWC delay-and-sum, Eq. (DAS) with a 2D array:
 *   B(r) = sum_{i,l} y_il( tau_in(r, i) + |r - (u_l, v_l, 0)| / c )
 * y [N][L][T] complex analytic channel data; sx_i, sy_i, sz_i [N];
 * elem_x, elem_y [L]; B [n_pix] complex (overwritten).
 */
int orc_das_beamform_vol(int N, int L, int T, const double *y, const double *sx_i,
                         const double *sy_i, const double *sz_i, const double *elem_x,
                         const double *elem_y, int n_pix, const double *pix_x,
                         const double *pix_y, const double *pix_z, double fs, double c,
                         double *B) {
  if (N < 0 || L < 0 || T < 2 || n_pix < 0) return 1;
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n_pix; ++q) {
    const double x = pix_x[q], yy = pix_y[q], z = pix_z[q];
    double accr = 0.0, acci = 0.0;
    for (int i = 0; i < N; ++i) {
      const double tau_in = (x * sx_i[i] + yy * sy_i[i] + z * sz_i[i]) / c;
      for (int l = 0; l < L; ++l) {
        const double dx = x - elem_x[l], dy = yy - elem_y[l];
        const double tau_out = sqrt(dx * dx + dy * dy + z * z) / c;
        double re, im;
        lerp(y + 2L * ((long)i * L + l) * T, T, fs * (tau_in + tau_out), &re, &im);
        accr += re;
        acci += im;
      }
    }
    B[2 * q] = accr;
    B[2 * q + 1] = acci;
  }
  return 0;
}
