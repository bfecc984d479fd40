/*
 * kksynth/sim.c -- seeded synthetic RF for plane-wave compounding.
 *
 * Input generation only: this file holds the forward model that turns a
 * phantom (point scatterers) into channel data.  It contains none of the
 * beamforming method's arithmetic (no decomposition, no image formation) and
 * is shared by the oracle side and the CUDA side, which both read the bytes it
 * produces.
 *
 * Forward model (linear superposition of two-way far-field delays):
 *   rf[i][l][n] = sum_s a_s * p(n/fs - tau_in(i,s) - tau_out(l,s))
 *   tau_in  = (x_s sin(theta_i) + z_s cos(theta_i)) / c   (plane-wave transmit
 *             passing the origin at t = 0)
 *   tau_out = sqrt((x_s - u_l)^2 + z_s^2) / c             (spherical receive)
 *   p(t)    = exp(-alpha t^2) cos(2 pi f0 t), truncated to |t| <= half_window.
 * No directivity, spreading or attenuation.
 *
 * The pulse is evaluated with exact recurrences per (channel, scatterer):
 * the Gaussian by g[k+1] = g[k] q[k], q[k+1] = q[k] qq, and the carrier by a
 * complex rotation.  Everything is FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int kks_simulate(int n_tx, const double *tx_angles, int n_elem,
                 const double *elem_x, int T, double fs, double c, double f0,
                 double alpha, double half_window, int n_scat,
                 const double *sx, const double *sz, const double *amp,
                 double *rf /* [n_tx][n_elem][T], overwritten */) {
  if (n_tx <= 0 || n_elem <= 0 || T <= 0 || n_scat < 0) return 1;
  const double h = 1.0 / fs;
  const double qq = exp(-2.0 * alpha * h * h);
  const double rot_c = cos(2.0 * M_PI * f0 * h);
  const double rot_s = sin(2.0 * M_PI * f0 * h);

  /* receive path lengths, shared by all transmit angles */
  double *tout = (double *)malloc(sizeof(double) * (size_t)n_elem * (size_t)(n_scat > 0 ? n_scat : 1));
  if (!tout) return 2;
#pragma omp parallel for schedule(static)
  for (int l = 0; l < n_elem; ++l)
    for (int s = 0; s < n_scat; ++s) {
      double dx = sx[s] - elem_x[l];
      tout[(size_t)l * n_scat + s] = sqrt(dx * dx + sz[s] * sz[s]) / c;
    }

#pragma omp parallel for schedule(dynamic, 4)
  for (int ch = 0; ch < n_tx * n_elem; ++ch) {
    const int i = ch / n_elem, l = ch % n_elem;
    const double si = sin(tx_angles[i]), ci = cos(tx_angles[i]);
    double *out = rf + (size_t)ch * T;
    for (int n = 0; n < T; ++n) out[n] = 0.0;
    const double *to = tout + (size_t)l * n_scat;
    for (int s = 0; s < n_scat; ++s) {
      const double tau = (sx[s] * si + sz[s] * ci) / c + to[s];
      long n0 = (long)ceil((tau - half_window) * fs);
      long n1 = (long)floor((tau + half_window) * fs);
      if (n0 < 0) n0 = 0;
      if (n1 > T - 1) n1 = T - 1;
      if (n0 > n1) continue;
      const double dt0 = (double)n0 * h - tau;
      double g = amp[s] * exp(-alpha * dt0 * dt0);
      double q = exp(-alpha * (2.0 * dt0 * h + h * h));
      double er = cos(2.0 * M_PI * f0 * dt0), ei = sin(2.0 * M_PI * f0 * dt0);
      for (long n = n0; n <= n1; ++n) {
        out[n] += g * er;
        g *= q;
        q *= qq;
        const double nr = er * rot_c - ei * rot_s;
        ei = er * rot_s + ei * rot_c;
        er = nr;
      }
    }
  }
  free(tout);
  return 0;
}

/*
 * Volumetric forward model for a 2D array (elements at (u_l, v_l, 0)):
 *   tau_in  = (x_s sx_i + y_s sy_i + z_s sz_i) / c,
 *             (sx, sy, sz) = (sin ax_i, sin ay_i, sqrt(1 - sin^2 ax_i - sin^2 ay_i))
 *   tau_out = |r_s - (u_l, v_l, 0)| / c
 * with the same pulse and recurrences as kks_simulate.
 */
int kks_simulate3(int n_tx, const double *tx_ax, const double *tx_ay, int n_elem,
                  const double *elem_x, const double *elem_y, int T, double fs, double c,
                  double f0, double alpha, double half_window, int n_scat, const double *px,
                  const double *py, const double *pz, const double *amp,
                  double *rf /* [n_tx][n_elem][T], overwritten */) {
  if (n_tx <= 0 || n_elem <= 0 || T <= 0 || n_scat < 0) return 1;
  for (int i = 0; i < n_tx; ++i) {
    const double a = sin(tx_ax[i]), b = sin(tx_ay[i]);
    if (a * a + b * b >= 1.0) return 3;
  }
  const double h = 1.0 / fs;
  const double qq = exp(-2.0 * alpha * h * h);
  const double rot_c = cos(2.0 * M_PI * f0 * h);
  const double rot_s = sin(2.0 * M_PI * f0 * h);
  double *tout = (double *)malloc(sizeof(double) * (size_t)n_elem * (size_t)(n_scat > 0 ? n_scat : 1));
  if (!tout) return 2;
#pragma omp parallel for schedule(static)
  for (int l = 0; l < n_elem; ++l)
    for (int s = 0; s < n_scat; ++s) {
      const double dx = px[s] - elem_x[l], dy = py[s] - elem_y[l];
      tout[(size_t)l * n_scat + s] = sqrt(dx * dx + dy * dy + pz[s] * pz[s]) / c;
    }
#pragma omp parallel for schedule(dynamic, 4)
  for (int ch = 0; ch < n_tx * n_elem; ++ch) {
    const int i = ch / n_elem, l = ch % n_elem;
    const double sx = sin(tx_ax[i]), sy = sin(tx_ay[i]);
    const double sz = sqrt(1.0 - sx * sx - sy * sy);
    double *out = rf + (size_t)ch * T;
    for (int n = 0; n < T; ++n) out[n] = 0.0;
    const double *to = tout + (size_t)l * n_scat;
    for (int s = 0; s < n_scat; ++s) {
      const double tau = (px[s] * sx + py[s] * sy + pz[s] * sz) / c + to[s];
      long n0 = (long)ceil((tau - half_window) * fs);
      long n1 = (long)floor((tau + half_window) * fs);
      if (n0 < 0) n0 = 0;
      if (n1 > T - 1) n1 = T - 1;
      if (n0 > n1) continue;
      const double dt0 = (double)n0 * h - tau;
      double g = amp[s] * exp(-alpha * dt0 * dt0);
      double q = exp(-alpha * (2.0 * dt0 * h + h * h));
      double er = cos(2.0 * M_PI * f0 * dt0), ei = sin(2.0 * M_PI * f0 * dt0);
      for (long n = n0; n <= n1; ++n) {
        out[n] += g * er;
        g *= q;
        q *= qq;
        const double nr = er * rot_c - ei * rot_s;
        ei = er * rot_s + ei * rot_c;
        er = nr;
      }
    }
  }
  free(tout);
  return 0;
}
