/*
 * Seeded synthetic depth-sequence generator.
 *
 * This is the input source shared by the CUDA path and the CPU oracle.  It
 * renders noisy z-depth maps of analytic scenes by ray casting in FP64 and
 * holds none of the fusion method's arithmetic: no TSDF, no band, no
 * observation model, no solver.  The camera model is the OpenCV pinhole
 * (+z forward, x right, y down); the depth stored for a pixel is the z
 * coordinate of the first surface hit along the ray through the pixel centre.
 *
 * Noise: D = D_true + sigma(D_true) * n, with sigma(z) = a + b z^2 and n a
 * standard normal drawn by Box-Muller from a counter-based SplitMix64 hash
 * keyed by (seed, frame, pixel).  Dropout: a pixel is set to 0 (invalid)
 * when an independent uniform from the same hash falls below the dropout
 * probability.  Rays that hit nothing give 0 (invalid).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SC_SPHERE 0 /* params: cx cy cz r                                     */
#define SC_UNION 1  /* box c(3) half(3), sphere c(3) r, torus c(3) R r (axis z) */
#define SC_BLOB 2   /* c(3) r0 amp norm lip coef[48] (real SH, degrees 1..6)  */
#define SC_PLANE 3  /* n(3) c: surface {x : n.x = c}                           */

static uint64_t sm_mix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform in (0, 1) from a 64-bit key */
static double unit_open(uint64_t key) {
  return ((double)(sm_mix(key) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ---------------- ray / primitive intersections (FP64) ------------------ */

/* smallest s > eps with |o + s u - c| = r, u unit; returns INFINITY if none */
static double hit_sphere(const double o[3], const double u[3], const double c[3], double r) {
  double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
  double b = oc[0] * u[0] + oc[1] * u[1] + oc[2] * u[2];
  double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - r * r;
  double disc = b * b - cc;
  if (disc < 0) return INFINITY;
  double sq = sqrt(disc);
  double s0 = -b - sq, s1 = -b + sq;
  if (s0 > 1e-9) return s0;
  if (s1 > 1e-9) return s1;
  return INFINITY;
}

static double hit_box(const double o[3], const double u[3], const double c[3], const double hs[3]) {
  double tmin = -INFINITY, tmax = INFINITY;
  for (int a = 0; a < 3; ++a) {
    double lo = c[a] - hs[a] - o[a], hi = c[a] + hs[a] - o[a];
    if (u[a] == 0.0) {
      if (lo > 0 || hi < 0) return INFINITY;
      continue;
    }
    double t0 = lo / u[a], t1 = hi / u[a];
    if (t0 > t1) { double tt = t0; t0 = t1; t1 = tt; }
    if (t0 > tmin) tmin = t0;
    if (t1 < tmax) tmax = t1;
  }
  if (tmax < tmin) return INFINITY;
  if (tmin > 1e-9) return tmin;
  if (tmax > 1e-9) return tmax;
  return INFINITY;
}

static double torus_sdf(const double p[3], const double c[3], double R, double r) {
  double x = p[0] - c[0], y = p[1] - c[1], z = p[2] - c[2];
  double q = sqrt(x * x + y * y) - R;
  return sqrt(q * q + z * z) - r;
}

/* sphere tracing of an exact SDF (Lipschitz 1) inside its bounding sphere */
static double hit_torus(const double o[3], const double u[3], const double c[3], double R, double r) {
  double s_in = hit_sphere(o, u, c, R + r + 1e-6);
  double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
  int inside = (oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2]) < (R + r) * (R + r);
  if (!inside && !isfinite(s_in)) return INFINITY;
  double s = inside ? 0.0 : s_in;
  double s_far = s + 2.0 * (R + r) + 1e-3;
  for (int it = 0; it < 20000 && s < s_far; ++it) {
    double p[3] = {o[0] + s * u[0], o[1] + s * u[1], o[2] + s * u[2]};
    double f = torus_sdf(p, c, R, r);
    if (f < 1e-10) return s;
    s += f;
  }
  return INFINITY;
}

/* real orthonormal spherical harmonics, degrees 1..6 (48 terms), at unit w */
static double sh_series(const double* coef, const double w[3]) {
  double x = w[2];
  double st = sqrt(fmax(0.0, 1.0 - x * x));
  double phi = atan2(w[1], w[0]);
  double P[7][7];
  memset(P, 0, sizeof(P));
  P[0][0] = 1.0;
  for (int m = 1; m <= 6; ++m) P[m][m] = -(2.0 * m - 1.0) * st * P[m - 1][m - 1];
  for (int m = 0; m <= 5; ++m) P[m + 1][m] = x * (2.0 * m + 1.0) * P[m][m];
  for (int m = 0; m <= 6; ++m)
    for (int l = m + 2; l <= 6; ++l)
      P[l][m] = ((2.0 * l - 1.0) * x * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
  double g = 0.0;
  int k = 0;
  for (int l = 1; l <= 6; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double f = 1.0;
      for (int q = l - am + 1; q <= l + am; ++q) f *= q; /* (l+|m|)!/(l-|m|)! */
      double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) / f);
      double y;
      if (m == 0) y = K * P[l][0];
      else if (m > 0) y = sqrt(2.0) * K * cos(m * phi) * P[l][am];
      else y = sqrt(2.0) * K * sin(am * phi) * P[l][am];
      g += coef[k++] * y;
    }
  }
  return g;
}

static double blob_radius(const double* prm, const double w[3]) {
  return prm[3] * (1.0 + prm[4] * sh_series(prm + 8, w) / prm[5]);
}

static double blob_f(const double* prm, const double p[3]) {
  double d[3] = {p[0] - prm[0], p[1] - prm[1], p[2] - prm[2]};
  double rho = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (rho < 1e-12) return -prm[3];
  double w[3] = {d[0] / rho, d[1] / rho, d[2] / rho};
  return rho - blob_radius(prm, w);
}

/* star-shaped surface: conservative sphere tracing with step f / L */
static double hit_blob(const double o[3], const double u[3], const double* prm) {
  double rmax = prm[3] * (1.0 + prm[4]) * 1.001;
  double s_in = hit_sphere(o, u, prm, rmax);
  if (!isfinite(s_in)) return INFINITY;
  double s = s_in, s_far = s_in + 2.0 * rmax + 1e-3, L = prm[6];
  for (int it = 0; it < 100000 && s < s_far; ++it) {
    double p[3] = {o[0] + s * u[0], o[1] + s * u[1], o[2] + s * u[2]};
    double f = blob_f(prm, p);
    if (f < 1e-10) return s;
    s += f / L;
  }
  return INFINITY;
}

static double hit_plane(const double o[3], const double u[3], const double* prm) {
  double dn = prm[0] * u[0] + prm[1] * u[1] + prm[2] * u[2];
  if (dn == 0.0) return INFINITY;
  double s = (prm[3] - (prm[0] * o[0] + prm[1] * o[1] + prm[2] * o[2])) / dn;
  return s > 1e-9 ? s : INFINITY;
}

static double scene_hit(int type, const double* prm, const double o[3], const double u[3]) {
  switch (type) {
    case SC_SPHERE: return hit_sphere(o, u, prm, prm[3]);
    case SC_UNION: {
      double a = hit_box(o, u, prm, prm + 3);
      double b = hit_sphere(o, u, prm + 6, prm[9]);
      double c = hit_torus(o, u, prm + 10, prm[13], prm[14]);
      double m = a < b ? a : b;
      return m < c ? m : c;
    }
    case SC_BLOB: return hit_blob(o, u, prm);
    case SC_PLANE: return hit_plane(o, u, prm);
  }
  return INFINITY;
}

/* Exact (or, for the blob, radial) signed distance of the scene at p. */
double synth_scene_sdf(int type, const double* prm, const double p[3]) {
  switch (type) {
    case SC_SPHERE: {
      double d[3] = {p[0] - prm[0], p[1] - prm[1], p[2] - prm[2]};
      return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - prm[3];
    }
    case SC_UNION: {
      double q[3], out = 0, in = -INFINITY;
      for (int a = 0; a < 3; ++a) {
        q[a] = fabs(p[a] - prm[a]) - prm[3 + a];
        double qa = q[a] > 0 ? q[a] : 0;
        out += qa * qa;
        if (q[a] > in) in = q[a];
      }
      double box = sqrt(out) + (in < 0 ? in : 0);
      double d[3] = {p[0] - prm[6], p[1] - prm[7], p[2] - prm[8]};
      double sph = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - prm[9];
      double tor = torus_sdf(p, prm + 10, prm[13], prm[14]);
      double m = box < sph ? box : sph;
      return m < tor ? m : tor;
    }
    case SC_BLOB: return blob_f(prm, p);
    case SC_PLANE: return prm[3] - (prm[0] * p[0] + prm[1] * p[1] + prm[2] * p[2]);
  }
  return INFINITY;
}

void synth_scene_sdf_many(int type, const double* prm, int64_t n, const double* pts, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = synth_scene_sdf(type, prm, pts + 3 * i);
}

/* max |g| and max angular gradient |grad_S g| over n Fibonacci directions */
void synth_blob_stats(const double* coef, int n, double* gmax, double* gradmax) {
  double gm = 0, dm = 0, ga = M_PI * (3.0 - sqrt(5.0)), e = 1e-5;
  for (int i = 0; i < n; ++i) {
    double z = 1.0 - (2.0 * i + 1.0) / n, r = sqrt(fmax(0.0, 1.0 - z * z)), ph = i * ga;
    double w[3] = {r * cos(ph), r * sin(ph), z};
    double g = sh_series(coef, w);
    if (fabs(g) > gm) gm = fabs(g);
    /* two tangent directions */
    double a[3] = {fabs(w[2]) < 0.9 ? 0 : 1, 0, fabs(w[2]) < 0.9 ? 1 : 0};
    double t1[3] = {w[1] * a[2] - w[2] * a[1], w[2] * a[0] - w[0] * a[2], w[0] * a[1] - w[1] * a[0]};
    double n1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int k = 0; k < 3; ++k) t1[k] /= n1;
    double t2[3] = {w[1] * t1[2] - w[2] * t1[1], w[2] * t1[0] - w[0] * t1[2], w[0] * t1[1] - w[1] * t1[0]};
    double gg = 0;
    for (int dsel = 0; dsel < 2; ++dsel) {
      const double* t = dsel ? t2 : t1;
      double wp[3], wn[3];
      for (int k = 0; k < 3; ++k) { wp[k] = w[k] + e * t[k]; wn[k] = w[k] - e * t[k]; }
      double np = sqrt(wp[0] * wp[0] + wp[1] * wp[1] + wp[2] * wp[2]);
      double nn = sqrt(wn[0] * wn[0] + wn[1] * wn[1] + wn[2] * wn[2]);
      for (int k = 0; k < 3; ++k) { wp[k] /= np; wn[k] /= nn; }
      double dg = (sh_series(coef, wp) - sh_series(coef, wn)) / (2 * e);
      gg += dg * dg;
    }
    if (sqrt(gg) > dm) dm = sqrt(gg);
  }
  *gmax = gm;
  *gradmax = dm;
}

/*
 * Render T depth maps.  poses: [T][3][4] world<-camera (R | C), FP64.
 * depth: [T][H][W] float32 output.
 */
void synth_render(int type, const double* prm, int T, int H, int W, const double* poses,
                  double fx, double fy, double cx, double cy, double sig_a, double sig_b,
                  double dropout, uint64_t seed, int nthreads, float* depth) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (int64_t row = 0; row < (int64_t)T * H; ++row) {
    int t = (int)(row / H), py = (int)(row % H);
    const double* P = poses + 12 * t;
    for (int px = 0; px < W; ++px) {
      double dc[3] = {(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0};
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = P[4 * a] * dc[0] + P[4 * a + 1] * dc[1] + P[4 * a + 2] * dc[2];
      double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double u[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
      double o[3] = {P[3], P[7], P[11]};
      double s = scene_hit(type, prm, o, u);
      int64_t pix = ((int64_t)t * H + py) * W + px;
      float out = 0.0f;
      if (isfinite(s)) {
        double z = s / nd; /* z-depth: d has unit z in camera frame */
        double v = z;
        if (sig_a != 0.0 || sig_b != 0.0) {
          uint64_t key = sm_mix(seed) ^ ((uint64_t)pix * 4 + 0);
          double u1 = unit_open(key), u2 = unit_open(key ^ 0x5851F42D4C957F2DULL);
          double g = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
          v = z + (sig_a + sig_b * z * z) * g;
        }
        if (dropout > 0.0) {
          uint64_t key = sm_mix(seed ^ 0xD1342543DE82EF95ULL) ^ ((uint64_t)pix * 4 + 1);
          if (unit_open(key) < dropout) v = 0.0;
        }
        out = (float)v;
        if (!(out > 0.0f)) out = 0.0f;
      }
      depth[pix] = out;
    }
  }
}
