/*
 * aera_oracle.c -- plain FP64 CPU oracle for AERA antenna-response unfolding.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library. It shares no code, header, table or
 * constant generator with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes, per (station, candidate direction) pair, following the radio
 * reconstruction of arXiv 1507.07733, Sec. 2 (voltage traces of the two channels ->
 * antenna pattern evaluated for the direction -> E-field reconstructed -> maximum of
 * the envelope of the E-field used as timing -> timing yields the direction):
 *
 *   1. V_c[k] = sum_n v_c[n] exp(-2 pi i k n / N)          naive O(N^2) DFT per channel
 *   2. in-band bins: 30 MHz <= k fs / N <= 80 MHz            (Sec. 1: 30-80 MHz antennas)
 *   3. H[c][p](zen, az, f_k): trilinear interpolation of real and imaginary parts over
 *      the tabulated (zenith, azimuth, frequency) nodes      (Sec. 3: VEL known at
 *      discrete frequencies and angles, interpolated in between)
 *   4. per in-band bin: solve V = H E for E = (E_theta, E_phi) in closed form
 *   5. analytic signal z_p[n] = (1/N) sum_{k in band} 2 E_p[k] exp(+2 pi i k n / N);
 *      E-field e_p = Re z_p; envelope env = sqrt(|z_theta|^2 + |z_phi|^2)
 *      (Sec. 4: envelope = sqrt(x^2 + H(x)^2), H the Hilbert transform)
 *   6. peak = argmax env (lowest index on ties); peak time = t_start + peak * 1e9/fs ns
 *   7. per direction: plane-wave delays tau_s = -n.x_s / c, t0 = mean(t_s - tau_s),
 *      residual r_s = t_s - tau_s - t0, chi2 = sum r_s^2 (two-pass mean)
 *
 * Readings where the paper is silent or garbled (the printed envelope formula puts the
 * square inside the Hilbert transform; the sign of the Hilbert phase; the treatment of
 * out-of-band bins; near-singular 2x2 systems; tie-breaks) are the ones documented in
 * the project's design notes and repeated at each function below.
 *
 * Built with -ffp-contract=off so that no multiply-add is fused on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_BAND_LO_HZ 30e6
#define ORC_BAND_HI_HZ 80e6
#define ORC_C_M_PER_NS 0.299792458
#define ORC_SINGULAR_REL 1e-6

#define ORC_ST_SINGULAR 1u     /* at least one in-band bin had a near-singular H */
#define ORC_ST_ZEN_CLAMP 2u    /* zenith outside the table, clamped to its edge */
#define ORC_ST_BAD_DIR 4u      /* direction without a cell (see orc_dir_ok): all outputs zero */

typedef struct {
  int32_t n_zen;  double zen0_rad, dzen_rad;
  int32_t n_az;   double az0_rad, daz_rad;
  int32_t n_freq; double f0_hz, df_hz;
} orc_pattern;

/* ---- 2. band mask -------------------------------------------------------------- */

/* 1 if bin k of an N-point transform at sample rate fs lies in [30, 80] MHz. */
int orc_in_band(int n, double fs_hz, int k) {
  double f = (double)k * fs_hz / (double)n;
  return f >= ORC_BAND_LO_HZ && f <= ORC_BAND_HI_HZ;
}

/* ---- 1. and 5. naive DFT ----------------------------------------------------------- */

/* out[k] = sum_n in[n] exp(sign * 2 pi i k n / N); complex data interleaved [N][2].
 * No normalisation. The twiddle for (k, n) is taken from a table indexed k*n mod N. */
void orc_dft(int n, int sign, const double *in, double *out) {
  double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  for (int t = 0; t < n; ++t) {
    double a = 2.0 * ORC_PI * (double)t / (double)n;
    tw[2 * t] = cos(a);
    tw[2 * t + 1] = sign * sin(a);
  }
  for (int k = 0; k < n; ++k) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < n; ++j) {
      int t = (int)(((int64_t)k * j) % n);
      double wr = tw[2 * t], wi = tw[2 * t + 1];
      sr += in[2 * j] * wr - in[2 * j + 1] * wi;
      si += in[2 * j] * wi + in[2 * j + 1] * wr;
    }
    out[2 * k] = sr;
    out[2 * k + 1] = si;
  }
  free(tw);
}

/* Spectra of both channels of one station: spec[c][k][2] for c = 0, 1 (full N bins).
 * Each real channel is transformed on its own (no two-for-one packing). */
void orc_station_spectrum(int n, const float *trace /* [2][N] */, double *spec /* [2][N][2] */) {
  double *buf = (double *)malloc(sizeof(double) * 2 * (size_t)n);
  for (int c = 0; c < 2; ++c) {
    for (int j = 0; j < n; ++j) {
      buf[2 * j] = (double)trace[(size_t)c * n + j];
      buf[2 * j + 1] = 0.0;
    }
    orc_dft(n, -1, buf, spec + (size_t)c * 2 * n);
  }
  free(buf);
}

/* ---- 3. trilinear VEL interpolation ----------------------------------------------- */

/* Cell index and fraction along a clamped axis: u clamped to [0, n-1], cell capped at n-2. */
static void clamped_cell(double u, int n, int *i, double *t, int *clamped) {
  if (u < 0.0) { u = 0.0; *clamped = 1; }
  if (u > (double)(n - 1)) { u = (double)(n - 1); *clamped = 1; }
  int c = (int)floor(u);
  if (c > n - 2) c = n - 2;
  *i = c;
  *t = u - (double)c;
}

/* H[c][p][re,im] at (zen, az, f). Zenith and frequency clamp to the table edges; azimuth
 * is periodic (node n_az is node 0). The real and imaginary parts are interpolated
 * independently and linearly along each axis: the weight of a corner is the product of
 * its three 1-D weights. */
void orc_vel(const orc_pattern *pt, const float *table, double zen, double az, double f_hz,
             double *H /* [2][2][2] */, uint32_t *status) {
  int iz, ifr, cl = 0, dummy = 0;
  double tz, tf;
  clamped_cell((zen - pt->zen0_rad) / pt->dzen_rad, pt->n_zen, &iz, &tz, &cl);
  clamped_cell((f_hz - pt->f0_hz) / pt->df_hz, pt->n_freq, &ifr, &tf, &dummy);
  if (cl && status) *status |= ORC_ST_ZEN_CLAMP;
  double ua = (az - pt->az0_rad) / pt->daz_rad;
  ua = ua - (double)pt->n_az * floor(ua / (double)pt->n_az);
  int ia = (int)floor(ua);
  double ta = ua - (double)ia;
  if (ia >= pt->n_az) ia -= pt->n_az;
  int ia1 = ia + 1 == pt->n_az ? 0 : ia + 1;
  for (int q = 0; q < 8; ++q) H[q] = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int da = 0; da < 2; ++da)
      for (int df = 0; df < 2; ++df) {
        double w = (dz ? tz : 1.0 - tz) * (da ? ta : 1.0 - ta) * (df ? tf : 1.0 - tf);
        size_t node = ((size_t)(iz + dz) * pt->n_az + (size_t)(da ? ia1 : ia)) * pt->n_freq +
                      (size_t)(ifr + df);
        const float *v = table + node * 8;   /* [c][p][re,im] */
        for (int q = 0; q < 8; ++q) H[q] += w * (double)v[q];
      }
}

/* ---- 4. closed-form 2x2 complex solve ---------------------------------------------- */

/* Solve V_c = sum_p H[c][p] E_p for E. H = [[H0t, H0p], [H1t, H1p]] (rows: channels).
 *   det = H0t H1p - H0p H1t
 *   E_t = (H1p V0 - H0p V1) / det,   E_p = (H0t V1 - H1t V0) / det
 * Near-singular reading: if |det| <= 1e-6 (|H0t||H1p| + |H0p||H1t|) the bin gets E = 0
 * and the function returns 1. *margin receives |det| / (|H0t||H1p| + |H0p||H1t|). */
int orc_solve(const double *H, const double *V /* [2][re,im] */, double *E /* [2][re,im] */,
              double *margin) {
  double a_r = H[0], a_i = H[1];   /* H0t */
  double b_r = H[2], b_i = H[3];   /* H0p */
  double c_r = H[4], c_i = H[5];   /* H1t */
  double d_r = H[6], d_i = H[7];   /* H1p */
  double det_r = (a_r * d_r - a_i * d_i) - (b_r * c_r - b_i * c_i);
  double det_i = (a_r * d_i + a_i * d_r) - (b_r * c_i + b_i * c_r);
  double scale = hypot(a_r, a_i) * hypot(d_r, d_i) + hypot(b_r, b_i) * hypot(c_r, c_i);
  double adet = hypot(det_r, det_i);
  if (margin) *margin = scale > 0.0 ? adet / scale : 0.0;
  if (!(adet > ORC_SINGULAR_REL * scale)) {
    E[0] = E[1] = E[2] = E[3] = 0.0;
    return 1;
  }
  double v0r = V[0], v0i = V[1], v1r = V[2], v1i = V[3];
  double nt_r = (d_r * v0r - d_i * v0i) - (b_r * v1r - b_i * v1i);
  double nt_i = (d_r * v0i + d_i * v0r) - (b_r * v1i + b_i * v1r);
  double np_r = (a_r * v1r - a_i * v1i) - (c_r * v0r - c_i * v0i);
  double np_i = (a_r * v1i + a_i * v1r) - (c_r * v0i + c_i * v0r);
  double den = det_r * det_r + det_i * det_i;
  E[0] = (nt_r * det_r + nt_i * det_i) / den;
  E[1] = (nt_i * det_r - nt_r * det_i) / den;
  E[2] = (np_r * det_r + np_i * det_i) / den;
  E[3] = (np_i * det_r - np_r * det_i) / den;
  return 0;
}

/* ---- 4.-6. one (station, direction) pair from the station's spectra ------------------ */

/* A direction the pattern can be evaluated at: finite, with an azimuth less than 2^52
 * azimuth steps from az0 (beyond, one FP64 unit is a whole step and the position inside the
 * period is lost). Any other direction has no cell and is treated like a non-finite one. */
static int orc_dir_ok(const orc_pattern *pt, double zen, double az) {
  if (!isfinite(zen) || !isfinite(az)) return 0;
  return fabs((az - pt->az0_rad) / pt->daz_rad) < 0x1p52;
}

/* Unfold one pair. spec = orc_station_spectrum output. Writes efield [2][N] (may be NULL),
 * env [N] (may be NULL), the peak index/amplitude and the status bits. min_margin gets the
 * smallest |det|/scale over in-band bins (used by tests to skip bins near the threshold). */
void orc_unfold_pair(const orc_pattern *pt, const float *table, int n, double fs_hz,
                     const double *spec, double zen, double az,
                     double *efield, double *env, int32_t *peak_idx, double *peak_amp,
                     uint32_t *status, double *min_margin) {
  uint32_t st = 0;
  double mm = INFINITY;
  double *Z = (double *)calloc((size_t)4 * n, sizeof(double));   /* [2 pol][N][2] */
  double *z = (double *)malloc(sizeof(double) * 4 * (size_t)n);
  double *e = (double *)malloc(sizeof(double) * 3 * (size_t)n);  /* e_t, e_p, env */
  if (!orc_dir_ok(pt, zen, az)) {
    st |= ORC_ST_BAD_DIR;
    memset(e, 0, sizeof(double) * 3 * (size_t)n);
  } else {
    for (int k = 0; k < n; ++k) {
      if (!orc_in_band(n, fs_hz, k)) continue;          /* out of band: E = 0 */
      double H[8], V[4], E[4], mg;
      orc_vel(pt, table, zen, az, (double)k * fs_hz / (double)n, H, &st);
      V[0] = spec[2 * k];             V[1] = spec[2 * k + 1];
      V[2] = spec[2 * (n + k)];       V[3] = spec[2 * (n + k) + 1];
      if (orc_solve(H, V, E, &mg)) st |= ORC_ST_SINGULAR;
      if (mg < mm) mm = mg;
      for (int p = 0; p < 2; ++p) {                      /* one-sided spectrum, doubled */
        Z[(size_t)p * 2 * n + 2 * k] = 2.0 * E[2 * p];
        Z[(size_t)p * 2 * n + 2 * k + 1] = 2.0 * E[2 * p + 1];
      }
    }
    for (int p = 0; p < 2; ++p) orc_dft(n, +1, Z + (size_t)p * 2 * n, z + (size_t)p * 2 * n);
    for (int j = 0; j < n; ++j) {
      double tr = z[2 * j] / n, ti = z[2 * j + 1] / n;
      double pr = z[2 * (n + j)] / n, pi = z[2 * (n + j) + 1] / n;
      e[j] = tr;
      e[n + j] = pr;
      e[2 * n + j] = sqrt(tr * tr + ti * ti + pr * pr + pi * pi);
    }
  }
  int best = 0;
  for (int j = 1; j < n; ++j)
    if (e[2 * n + j] > e[2 * n + best]) best = j;     /* strict: lowest index wins ties */
  if (efield) memcpy(efield, e, sizeof(double) * 2 * (size_t)n);
  if (env) memcpy(env, e + 2 * (size_t)n, sizeof(double) * (size_t)n);
  *peak_idx = best;
  *peak_amp = e[2 * (size_t)n + best];
  *status = st;
  if (min_margin) *min_margin = mm;
  free(Z); free(z); free(e);
}

/* ---- 7. plane-wave timing residual ------------------------------------------------- */

/* n = (sin zen cos az, sin zen sin az, cos zen) points to the source; azimuth counts
 * counter-clockwise from east (+x). tau_s = -n.x_s * n_refr / c. Two-pass mean. */
void orc_residual(int n_st, const double *pos /* [S][3] */, const double *peak_time,
                  double zen, double az, double n_refr,
                  double *res /* [S] */, double *t0, double *chi2) {
  if (n_st <= 0) { *t0 = 0.0; *chi2 = 0.0; return; }
  double nx = sin(zen) * cos(az), ny = sin(zen) * sin(az), nz = cos(zen);
  double sum = 0.0;
  for (int s = 0; s < n_st; ++s) {
    double tau = -(nx * pos[3 * s] + ny * pos[3 * s + 1] + nz * pos[3 * s + 2]) * n_refr /
                 ORC_C_M_PER_NS;
    res[s] = peak_time[s] - tau;
    sum += res[s];
  }
  double mean = sum / n_st, ss = 0.0;
  for (int s = 0; s < n_st; ++s) {
    res[s] = res[s] - mean;
    ss += res[s] * res[s];
  }
  *t0 = mean;
  *chi2 = ss;
}

/* ---- sub-sample peak (a variant: the paper times stations by the envelope maximum and
 * says nothing finer) --------------------------------------------------------------------
 * The parabola through (k-1, env[k-1]), (k, env[k]), (k+1, env[k+1]) has its vertex at
 * k + delta with delta = (env[k-1] - env[k+1]) / (2 (env[k-1] - 2 env[k] + env[k+1])).
 * Readings: delta = 0 at the two ends of the trace and where the second difference is not
 * negative (no strict maximum); a vertex further than half a sample from k is clamped to
 * +-1/2 (k is the sample maximum, so the true vertex of a concave fit lies within). */
double orc_peak_offset(int n, const double *env, int k) {
  if (k <= 0 || k >= n - 1) return 0.0;
  double a = env[k - 1], b = env[k], c = env[k + 1];
  double second = a - 2.0 * b + c;
  if (!(second < 0.0)) return 0.0;
  double delta = 0.5 * (a - c) / second;
  if (delta > 0.5) delta = 0.5;
  if (delta < -0.5) delta = -0.5;
  return delta;
}

/* ---- signal-to-noise ratio and SNR-weighted residual (a variant: the paper defines no
 * noise estimate and no timing weights) ---------------------------------------------------
 * SNR of a pair: (env[k] / noise)^2 at the envelope maximum k, noise^2 being the mean of
 * env[n]^2 over the samples with |n - k| > N/16 (the pulse is taken to lie within N/16
 * samples of its maximum). 0 when no sample lies outside that window or their mean is 0. */
double orc_snr(int n, const double *env, int k) {
  int w = n / 16, count = 0;
  double ss = 0.0;
  for (int i = 0; i < n; ++i) {
    int d = i > k ? i - k : k - i;
    if (d > w) {
      ss += env[i] * env[i];
      count += 1;
    }
  }
  if (count == 0 || !(ss > 0.0)) return 0.0;
  double noise2 = ss / count;
  return env[k] * env[k] / noise2;
}

/* Plane-wave residual with a weight w_s >= 0 per station (w = SNR: a station's timing
 * variance taken inversely proportional to its SNR):
 *   d_s = t_s - tau_s,  t0 = sum w d / sum w,  r_s = d_s - t0,  chi2 = sum w r^2.
 * With sum w == 0 this is the unweighted fit (orc_residual). */
void orc_residual_weighted(int n_st, const double *pos, const double *peak_time, const double *w,
                           double zen, double az, double n_refr, double *res, double *t0, double *chi2) {
  double sw = 0.0;
  for (int s = 0; s < n_st; ++s) sw += w[s];
  if (!(sw > 0.0)) {
    orc_residual(n_st, pos, peak_time, zen, az, n_refr, res, t0, chi2);
    return;
  }
  double nx = sin(zen) * cos(az), ny = sin(zen) * sin(az), nz = cos(zen);
  double swd = 0.0;
  for (int s = 0; s < n_st; ++s) {
    double tau = -(nx * pos[3 * s] + ny * pos[3 * s + 1] + nz * pos[3 * s + 2]) * n_refr /
                 ORC_C_M_PER_NS;
    res[s] = peak_time[s] - tau;
    swd += w[s] * res[s];
  }
  double mean = swd / sw, ss = 0.0;
  for (int s = 0; s < n_st; ++s) {
    res[s] = res[s] - mean;
    ss += w[s] * res[s] * res[s];
  }
  *t0 = mean;
  *chi2 = ss;
}

/* ---- whole event -------------------------------------------------------------------- */

/* All pairs of one event. Output layouts: efield [D][S][2][N], env [D][S][N],
 * peak_idx/peak_amp/peak_time/residual/status/min_margin [D][S], t0/chi2 [D].
 * efield and env may be NULL (peaks only). Pairs run in parallel when OpenMP is on;
 * each pair's arithmetic is independent of the thread that runs it. */
void orc_unfold_event(const orc_pattern *pt, const float *table, int n_st, int n, double fs_hz,
                      double n_refr, const float *traces, const double *pos,
                      const double *t_start_ns, int n_dir, const double *dirs,
                      double *efield, double *env, int32_t *peak_idx, double *peak_amp,
                      double *peak_time, double *residual, double *t0, double *chi2,
                      uint32_t *status, double *min_margin) {
  double *spec = (double *)malloc(sizeof(double) * 4 * (size_t)n * n_st);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < n_st; ++s)
    orc_station_spectrum(n, traces + (size_t)s * 2 * n, spec + (size_t)s * 4 * n);
  double dt_ns = 1e9 / fs_hz;
#pragma omp parallel for schedule(dynamic)
  for (int q = 0; q < n_dir * n_st; ++q) {
    int d = q / n_st, s = q % n_st;
    double amp, mm;
    orc_unfold_pair(pt, table, n, fs_hz, spec + (size_t)s * 4 * n, dirs[2 * d], dirs[2 * d + 1],
                    efield ? efield + (size_t)q * 2 * n : NULL,
                    env ? env + (size_t)q * n : NULL, &peak_idx[q], &amp, &status[q], &mm);
    peak_amp[q] = amp;
    if (min_margin) min_margin[q] = mm;
    peak_time[q] = t_start_ns[s] + (double)peak_idx[q] * dt_ns;
  }
  for (int d = 0; d < n_dir; ++d)
    orc_residual(n_st, pos, peak_time + (size_t)d * n_st, dirs[2 * d], dirs[2 * d + 1], n_refr,
                 residual + (size_t)d * n_st, &t0[d], &chi2[d]);
  free(spec);
}

/* A sample of pairs of one event, given as (station, direction) index lists. Used where
 * the whole event is too large for this oracle: each listed pair gets its spectrum, its
 * unfolding and its peak. Outputs are [n_pairs]-major with the per-pair layouts above. */
void orc_unfold_sample(const orc_pattern *pt, const float *table, int n, double fs_hz,
                       const float *traces, const double *t_start_ns, const double *dirs,
                       int n_pairs, const int32_t *st_idx, const int32_t *dir_idx,
                       double *efield, double *env, int32_t *peak_idx, double *peak_amp,
                       double *peak_time, uint32_t *status, double *min_margin) {
  double dt_ns = 1e9 / fs_hz;
#pragma omp parallel for schedule(dynamic)
  for (int q = 0; q < n_pairs; ++q) {
    int s = st_idx[q], d = dir_idx[q];
    double *spec = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    double amp, mm;
    orc_station_spectrum(n, traces + (size_t)s * 2 * n, spec);
    orc_unfold_pair(pt, table, n, fs_hz, spec, dirs[2 * d], dirs[2 * d + 1],
                    efield ? efield + (size_t)q * 2 * n : NULL,
                    env ? env + (size_t)q * n : NULL, &peak_idx[q], &amp, &status[q], &mm);
    peak_amp[q] = amp;
    if (min_margin) min_margin[q] = mm;
    peak_time[q] = t_start_ns[s] + (double)peak_idx[q] * dt_ns;
    free(spec);
  }
}

/* ---- iterative reconstruction (Sec. 2) ------------------------------------------------
 * 1. initial timing: per station the sample where the voltage trace is largest,
 *    argmax_n v0[n]^2 + v1[n]^2 (lowest index on ties), t_s = t_start + n 1e9/fs;
 * 2. triangulation: the plane wave t_s = t0 - n.x_s * n_refr / c fitted by least squares;
 * 3. the antenna pattern evaluated for that direction and every station's E-field unfolded;
 * 4. the envelope maxima become the new timing; repeat until the direction stops changing.
 * Readings (the paper gives none of these details): unweighted least squares; the fit is
 * linear in (t0, nx, ny) for a fixed nz = sqrt(1 - nx^2 - ny^2), solved by Cramer's rule and
 * repeated ORC_FIT_PASSES times with nz updated from the previous solution (nz = 1 first);
 * nx^2 + ny^2 > 1 is scaled back to the horizon; convergence when the angle between successive
 * directions is below tol_rad or the station times repeat. */

#define ORC_FIT_PASSES 4

void orc_voltage_peaks(int n_st, int n, double fs_hz, const float *traces, const double *t_start_ns,
                       int32_t *idx, double *t_ns) {
  for (int s = 0; s < n_st; ++s) {
    const float *v0 = traces + (size_t)s * 2 * n, *v1 = v0 + n;
    int best = 0;
    double bv = -1.0;
    for (int j = 0; j < n; ++j) {
      double p = (double)v0[j] * v0[j] + (double)v1[j] * v1[j];
      if (p > bv) { bv = p; best = j; }
    }
    idx[s] = best;
    t_ns[s] = t_start_ns[s] + (double)best * (1e9 / fs_hz);
  }
}

/* Least-squares plane-wave direction from station times. Returns 0, or 1 if the stations
 * do not determine a direction (fewer than 3 or collinear). */
int orc_plane_fit(int n_st, const double *pos, const double *t_ns, double n_refr, double *zen, double *az,
                  double *t0) {
  if (n_st < 3) return 1;
  double k = n_refr / ORC_C_M_PER_NS;   /* ns per metre */
  double nx = 0.0, ny = 0.0, nz = 1.0, c0 = 0.0;
  for (int pass = 0; pass < ORC_FIT_PASSES; ++pass) {
    /* model y_s = t_s + k nz z_s = c0 - k nx x_s - k ny y_s: unknowns (c0, a, b) with a = -k nx,
     * b = -k ny; normal equations of the regressors (1, x_s, y_s) */
    double m[3][3] = {{0}}, r[3] = {0};
    for (int s = 0; s < n_st; ++s) {
      double f[3] = {1.0, pos[3 * s], pos[3 * s + 1]};
      double y = t_ns[s] + k * nz * pos[3 * s + 2];
      for (int i = 0; i < 3; ++i) {
        r[i] += f[i] * y;
        for (int j = 0; j < 3; ++j) m[i][j] += f[i] * f[j];
      }
    }
    double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                 m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                 m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    double scale = m[0][0] * m[1][1] * m[2][2];
    if (!(fabs(det) > 1e-12 * scale)) return 1;
    double sol[3];
    for (int c = 0; c < 3; ++c) {   /* Cramer: replace column c by r */
      double a[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a[i][j] = j == c ? r[i] : m[i][j];
      double dc = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                  a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                  a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
      sol[c] = dc / det;
    }
    c0 = sol[0];
    nx = -sol[1] / k;
    ny = -sol[2] / k;
    double h2 = nx * nx + ny * ny;
    if (h2 > 1.0) {
      double h = sqrt(h2);
      nx /= h;
      ny /= h;
      h2 = 1.0;
    }
    nz = sqrt(1.0 - h2);
  }
  *zen = atan2(sqrt(nx * nx + ny * ny), nz);
  double a = atan2(ny, nx);
  *az = a < 0.0 ? a + 2.0 * ORC_PI : a;
  *t0 = c0;
  return 0;
}

/* The whole loop for one event. history gets (zenith, azimuth) after every fit (up to
 * max_iter + 1 entries); peak_idx_hist the station peak indices used by every fit
 * [(max_iter + 1)][S]. Outputs of the final unfold: efield [S][2][N], env [S][N] (may be
 * NULL), peak_idx/peak_amp/peak_time/status [S]. Returns the number of unfold iterations, or
 * -1 if the first fit failed. */
int orc_reconstruct(const orc_pattern *pt, const float *table, int n_st, int n, double fs_hz, double n_refr,
                    const float *traces, const double *pos, const double *t_start_ns, int max_iter, double tol_rad,
                    double *history, int32_t *peak_idx_hist, double *zen_out, double *az_out, double *t0_out,
                    double *chi2_out, double *efield, double *env, int32_t *peak_idx, double *peak_amp,
                    double *peak_time, uint32_t *status) {
  double *spec = (double *)malloc(sizeof(double) * 4 * (size_t)n * n_st);
  double *t_ns = (double *)malloc(sizeof(double) * n_st);
  double *res = (double *)malloc(sizeof(double) * n_st);
  int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * n_st);
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < n_st; ++s)
    orc_station_spectrum(n, traces + (size_t)s * 2 * n, spec + (size_t)s * 4 * n);
  orc_voltage_peaks(n_st, n, fs_hz, traces, t_start_ns, idx, t_ns);
  double zen = NAN, az = NAN, t0 = NAN;
  int iters = 0;
  memcpy(peak_idx_hist, idx, sizeof(int32_t) * n_st);
  if (orc_plane_fit(n_st, pos, t_ns, n_refr, &zen, &az, &t0)) {
    iters = -1;
  } else {
    history[0] = zen;
    history[1] = az;
    double dt_ns = 1e9 / fs_hz;
    for (int it = 1; it <= max_iter; ++it) {
#pragma omp parallel for schedule(dynamic)
      for (int s = 0; s < n_st; ++s) {
        double amp, mm;
        orc_unfold_pair(pt, table, n, fs_hz, spec + (size_t)s * 4 * n, zen, az,
                        efield ? efield + (size_t)s * 2 * n : NULL, env ? env + (size_t)s * n : NULL,
                        &peak_idx[s], &amp, &status[s], &mm);
        peak_amp[s] = amp;
        peak_time[s] = t_start_ns[s] + (double)peak_idx[s] * dt_ns;
      }
      iters = it;
      int same = memcmp(peak_idx, peak_idx_hist + (size_t)(it - 1) * n_st, sizeof(int32_t) * n_st) == 0;
      memcpy(peak_idx_hist + (size_t)it * n_st, peak_idx, sizeof(int32_t) * n_st);
      double nzen, naz, nt0;
      if (orc_plane_fit(n_st, pos, peak_time, n_refr, &nzen, &naz, &nt0)) break;
      double ax = sin(zen) * cos(az), ay = sin(zen) * sin(az), az_ = cos(zen);
      double bx = sin(nzen) * cos(naz), by = sin(nzen) * sin(naz), bz = cos(nzen);
      double dot = ax * bx + ay * by + az_ * bz;
      double ang = acos(dot > 1.0 ? 1.0 : (dot < -1.0 ? -1.0 : dot));
      history[2 * it] = nzen;
      history[2 * it + 1] = naz;
      int done = same || ang < tol_rad;
      zen = nzen;
      az = naz;
      t0 = nt0;
      if (done) break;
    }
  }
  if (iters >= 0) {
    /* chi2 of the final fit with the final station times */
    double t0r, chi2;
    const double *tt = iters == 0 ? t_ns : peak_time;
    orc_residual(n_st, pos, tt, zen, az, n_refr, res, &t0r, &chi2);
    *chi2_out = chi2;
  }
  *zen_out = zen;
  *az_out = az;
  *t0_out = t0;
  free(spec); free(t_ns); free(res); free(idx);
  return iters;
}
