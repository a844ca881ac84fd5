/*
 * BayesFusion-SDF CPU oracle: a plain, slow, obviously-correct restatement of
 * the method (Sec. 3 of the paper, Algorithm 1) used ONLY as test
 * infrastructure: by the tests, by the smoke check and by the benchmark's
 * CPU-baseline arm.  The product path never links, loads or calls it, and it
 * shares no source with the CUDA library.
 *
 * Precision.  Every real-valued quantity (samples, weights, the system Q and
 * h, PCG vectors and inner products, probe sums, vertex positions, NBV
 * utilities) is FP64.  Discrete decisions -- which pixel a voxel projects to,
 * which TSDF samples count, band membership, candidate bricks, the voxels a
 * ray's DDA visits, the ray-cast depth used by view scoring -- follow a fixed
 * IEEE FP32 specification: every operation rounded separately, no fused
 * multiply-add (this file is compiled with -ffp-contract=off), in the order
 * written below.  That makes the integer outputs well defined and comparable
 * bit for bit with any other implementation of the same specification.
 *
 * Readings of the paper fixed here (the paper leaves these open):
 *  - grid: unknowns at voxel centres of a cubic n^3 lattice; centre(i) =
 *    origin + (i + 1/2) h; linear index i + n (j + n k); bricks of 8^3,
 *    brick linear index bi + nb (bj + nb bk), local index lx + 8 ly + 64 lz.
 *  - camera: pinhole, world<-camera pose [R | C], z-depth maps, pixel centre
 *    (px + 1/2, py + 1/2).
 *  - coarse TSDF (Sec. 3.3): unit weight per frame, sample = min(D - z_c,
 *    tau_c), frames whose sample is below -tau_c skipped, tsdf = sum / count.
 *  - band (Sec. 3.3, band equation with alpha = 1): B = {count > 0 and
 *    |tsdf| <= b h}; boundary dB = band voxels with fewer than 6 band
 *    6-neighbours (the grid edge counts as outside).
 *  - candidate bricks: bricks within Chebyshev distance r_B (in bricks) of a
 *    brick holding a back-projected valid pixel, r_B = floor((1.25 tau_c/h
 *    + 2)/8) + 1; only their voxels get a TSDF.
 *  - observations (Sec. 3.5, projective SDF and linear row): one row per
 *    (pixel, voxel visited by the pixel ray's DDA over [s_p - tau, s_p +
 *    tau]), a_i = e_j, n = -ray direction, so y = clamp(r.(p - x_j), -tau,
 *    tau)/h in voxel units, with precision w = h^2 / sigma^2, sigma^2 =
 *    sigma_d(D)^2 + sigma_pose^2 + sigma_model^2 and sigma_d(D) = a + b D^2
 *    at the measured z-depth D (noise equation of Sec. 3.5).
 *  - prior (Sec. 3.6, Q0): w_ij = 1 on 6-neighbour band pairs; the anchor
 *    term expands to lambda_b on the diagonal of boundary voxels and
 *    lambda_b tsdf_i/h in h.
 *  - PCG (Sec. 3.6): Jacobi preconditioner, x0 = 0 unless given, stop when
 *    ||r||_2 <= tol ||h||_2, then recompute the true residual and restart
 *    (at most 3 times) if it misses the tolerance.
 *  - probes (Sec. 3.7, diag equation): Rademacher entries from a
 *    counter-based SplitMix64 hash of (seed, probe index, linear voxel index).
 *  - marching cubes (Sec. 3.8): cubes of 8 band voxels, inside = mu < 0,
 *    polygons traced face by face with ambiguous faces separating the inside
 *    corners, fan triangulation from the lowest-numbered edge of each loop.
 *  - view utility (Sec. 3.8, NBV equation): s'_i = 1/(1/s_i + dd_i) from the
 *    candidate view's predicted observations; s_i floored at 1/Q_ii.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ band */

typedef struct {
  int n, nb;
  float h;
  float org[3];
  int64_t N;        /* band voxels */
  int32_t NB;       /* active bricks */
  int64_t n_cand;   /* candidate bricks */
  int32_t* dir;     /* [nb^3] brick rank or -1 */
  int32_t* bcoord;  /* [NB][3] */
  uint64_t* mask;   /* [NB][8] 512-bit band mask */
  int64_t* off;     /* [NB+1] first compact index of each brick */
  int64_t* lin;     /* [N] linear voxel index */
  float* tsdf;      /* [N] metres */
  int32_t* wcount;  /* [N] TSDF sample count */
  uint8_t* bdry;    /* [N] 1 if in dB */
  uint8_t* deg;     /* [N] band 6-neighbour count */
  int32_t* nbr;     /* [NB][6] rank of -x,+x,-y,+y,-z,+z brick or -1 */
} bfo_band;

typedef struct {
  float R[9]; /* row-major world<-camera rotation */
  float C[3]; /* camera centre */
} fpose;

static fpose load_pose(const float* P) {
  fpose p;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) p.R[3 * a + b] = P[4 * a + b];
    p.C[a] = P[4 * a + 3];
  }
  return p;
}

static int depth_valid(float D) { return D > 0.0f && D < INFINITY; }

/* FP32 spec: centre coordinate of voxel index i along one axis */
static float vox_centre(float org, float h, int i) { return org + ((float)i + 0.5f) * h; }

/* FP32 spec: project a world point; returns 1 and the pixel if visible */
static int project(const fpose* P, const float x[3], float fx, float fy, float cx, float cy, int W,
                   int H, int* px, int* py, float* zc) {
  float dx = x[0] - P->C[0], dy = x[1] - P->C[1], dz = x[2] - P->C[2];
  float xc = (P->R[0] * dx + P->R[3] * dy) + P->R[6] * dz;
  float yc = (P->R[1] * dx + P->R[4] * dy) + P->R[7] * dz;
  float z = (P->R[2] * dx + P->R[5] * dy) + P->R[8] * dz;
  if (!(z > 0.0f)) return 0;
  float u = (fx * xc) / z + cx;
  float v = (fy * yc) / z + cy;
  if (!(u >= 0.0f && u < (float)W && v >= 0.0f && v < (float)H)) return 0;
  *px = (int)u;
  *py = (int)v;
  *zc = z;
  return 1;
}

/* FP32 spec: pixel ray.  dw = R K^-1 u~ (unnormalised), nrm = |K^-1 u~| */
typedef struct {
  float dw[3], r[3], nrm;
} fray;

static fray pixel_ray(const fpose* P, int px, int py, float fx, float fy, float cx, float cy) {
  fray q;
  float a = ((float)px + 0.5f - cx) / fx;
  float b = ((float)py + 0.5f - cy) / fy;
  q.nrm = sqrtf((a * a + b * b) + 1.0f);
  for (int k = 0; k < 3; ++k) {
    q.dw[k] = (P->R[3 * k + 0] * a + P->R[3 * k + 1] * b) + P->R[3 * k + 2];
    q.r[k] = q.dw[k] / q.nrm;
  }
  return q;
}

static int brick_radius(double trunc_vox) { return (int)floor((1.25 * trunc_vox + 2.0) / 8.0) + 1; }

static int64_t band_index(const bfo_band* B, int i, int j, int k) {
  int n = B->n;
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return -1;
  int nb = B->nb;
  int32_t r = B->dir[(i >> 3) + nb * ((j >> 3) + nb * (k >> 3))];
  if (r < 0) return -1;
  int l = (i & 7) + 8 * (j & 7) + 64 * (k & 7);
  const uint64_t* m = B->mask + 8 * (int64_t)r;
  if (!((m[l >> 6] >> (l & 63)) & 1ULL)) return -1;
  int64_t c = 0;
  for (int w = 0; w < (l >> 6); ++w) c += __builtin_popcountll(m[w]);
  if (l & 63) c += __builtin_popcountll(m[l >> 6] & ((1ULL << (l & 63)) - 1ULL));
  return B->off[r] + c;
}

int64_t bfo_band_index(const bfo_band* B, int i, int j, int k) { return band_index(B, i, j, k); }

void bfo_band_free(bfo_band* B) {
  if (!B) return;
  free(B->dir); free(B->bcoord); free(B->mask); free(B->off); free(B->lin);
  free(B->tsdf); free(B->wcount); free(B->bdry); free(B->deg); free(B->nbr);
  free(B);
}

/*
 * Band builder (Sec. 3.3 TSDF bootstrap and band; Sec. 3.4 sparse bricks).
 * depth [T][H][W] (0 / non-finite = invalid), poses [T][3][4] world<-camera.
 */
bfo_band* bfo_build_band(const float* depth, int T, int H, int W, const float* poses, float fx, float fy,
                         float cx, float cy, int n, float h, const float* org, double band_vox,
                         double trunc_vox, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  bfo_band* B = (bfo_band*)calloc(1, sizeof(bfo_band));
  B->n = n;
  B->nb = n / 8;
  B->h = h;
  for (int a = 0; a < 3; ++a) B->org[a] = org[a];
  int nb = B->nb;
  int64_t nb3 = (int64_t)nb * nb * nb;
  int rB = brick_radius(trunc_vox);
  float h8 = 8.0f * h;
  float tauc = (float)trunc_vox * h;
  float beta = (float)band_vox * h;

  /* 1. bricks holding a back-projected valid pixel */
  uint8_t* hit = (uint8_t*)calloc(nb3, 1);
  for (int t = 0; t < T; ++t) {
    fpose P = load_pose(poses + 12 * t);
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        float D = depth[((int64_t)t * H + py) * W + px];
        if (!depth_valid(D)) continue;
        fray q = pixel_ray(&P, px, py, fx, fy, cx, cy);
        int bc[3], ok = 1;
        for (int k = 0; k < 3; ++k) {
          float p = P.C[k] + D * q.dw[k];
          float g = (p - org[k]) / h8;
          if (g < -(float)rB || g >= (float)(nb + rB)) { ok = 0; break; }
          int b = (int)floorf(g);
          bc[k] = b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
        }
        if (ok) hit[bc[0] + (int64_t)nb * (bc[1] + (int64_t)nb * bc[2])] = 1;
      }
  }
  /* 2. candidate bricks: Chebyshev dilation by rB */
  uint8_t* cand = (uint8_t*)calloc(nb3, 1);
  int64_t ncand = 0;
  for (int bk = 0; bk < nb; ++bk)
    for (int bj = 0; bj < nb; ++bj)
      for (int bi = 0; bi < nb; ++bi) {
        int found = 0;
        for (int dk = -rB; dk <= rB && !found; ++dk)
          for (int dj = -rB; dj <= rB && !found; ++dj)
            for (int di = -rB; di <= rB && !found; ++di) {
              int x = bi + di, y = bj + dj, z = bk + dk;
              if (x < 0 || y < 0 || z < 0 || x >= nb || y >= nb || z >= nb) continue;
              if (hit[x + (int64_t)nb * (y + (int64_t)nb * z)]) found = 1;
            }
        if (found) { cand[bi + (int64_t)nb * (bj + (int64_t)nb * bk)] = 1; ++ncand; }
      }
  free(hit);
  B->n_cand = ncand;
  int64_t* clist = (int64_t*)malloc(sizeof(int64_t) * (ncand ? ncand : 1));
  {
    int64_t c = 0;
    for (int64_t b = 0; b < nb3; ++b) if (cand[b]) clist[c++] = b;
  }
  free(cand);

  /* 3. TSDF of every candidate voxel, frames in order */
  float* ts = (float*)malloc(sizeof(float) * 512 * (ncand ? ncand : 1));
  int32_t* wc = (int32_t*)malloc(sizeof(int32_t) * 512 * (ncand ? ncand : 1));
  fpose* PP = (fpose*)malloc(sizeof(fpose) * (T ? T : 1));
  for (int t = 0; t < T; ++t) PP[t] = load_pose(poses + 12 * t);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t c = 0; c < ncand; ++c) {
    int64_t b = clist[c];
    int bi = (int)(b % nb), bj = (int)((b / nb) % nb), bk = (int)(b / ((int64_t)nb * nb));
    for (int l = 0; l < 512; ++l) {
      int i = 8 * bi + (l & 7), j = 8 * bj + ((l >> 3) & 7), k = 8 * bk + (l >> 6);
      float x[3] = {vox_centre(org[0], h, i), vox_centre(org[1], h, j), vox_centre(org[2], h, k)};
      float S = 0.0f;
      int32_t cnt = 0;
      for (int t = 0; t < T; ++t) {
        int px, py;
        float zc;
        if (!project(&PP[t], x, fx, fy, cx, cy, W, H, &px, &py, &zc)) continue;
        float D = depth[((int64_t)t * H + py) * W + px];
        if (!depth_valid(D)) continue;
        float sdf = D - zc;
        if (sdf < -tauc) continue;
        float smp = sdf < tauc ? sdf : tauc;
        S = S + smp;
        cnt += 1;
      }
      ts[512 * c + l] = cnt > 0 ? S / (float)cnt : 0.0f;
      wc[512 * c + l] = cnt;
    }
  }
  free(PP);

  /* 4. band mask, active bricks in ascending linear brick index */
  B->dir = (int32_t*)malloc(sizeof(int32_t) * nb3);
  for (int64_t b = 0; b < nb3; ++b) B->dir[b] = -1;
  int32_t NB = 0;
  int64_t N = 0;
  uint64_t* cmask = (uint64_t*)calloc(8 * (ncand ? ncand : 1), sizeof(uint64_t));
  for (int64_t c = 0; c < ncand; ++c) {
    int any = 0;
    for (int l = 0; l < 512; ++l) {
      int in = wc[512 * c + l] > 0 && fabsf(ts[512 * c + l]) <= beta;
      if (in) { cmask[8 * c + (l >> 6)] |= 1ULL << (l & 63); any = 1; ++N; }
    }
    if (any) B->dir[clist[c]] = NB++;
  }
  B->NB = NB;
  B->N = N;
  B->bcoord = (int32_t*)malloc(sizeof(int32_t) * 3 * (NB ? NB : 1));
  B->mask = (uint64_t*)malloc(sizeof(uint64_t) * 8 * (NB ? NB : 1));
  B->off = (int64_t*)malloc(sizeof(int64_t) * (NB + 1));
  B->lin = (int64_t*)malloc(sizeof(int64_t) * (N ? N : 1));
  B->tsdf = (float*)malloc(sizeof(float) * (N ? N : 1));
  B->wcount = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
  B->bdry = (uint8_t*)malloc(N ? N : 1);
  B->deg = (uint8_t*)malloc(N ? N : 1);
  B->nbr = (int32_t*)malloc(sizeof(int32_t) * 6 * (NB ? NB : 1));
  int64_t pos = 0;
  for (int64_t c = 0; c < ncand; ++c) {
    int64_t b = clist[c];
    int32_t r = B->dir[b];
    if (r < 0) continue;
    int bi = (int)(b % nb), bj = (int)((b / nb) % nb), bk = (int)(b / ((int64_t)nb * nb));
    B->bcoord[3 * r] = bi; B->bcoord[3 * r + 1] = bj; B->bcoord[3 * r + 2] = bk;
    memcpy(B->mask + 8 * (int64_t)r, cmask + 8 * c, 64);
    B->off[r] = pos;
    for (int l = 0; l < 512; ++l) {
      if (!((cmask[8 * c + (l >> 6)] >> (l & 63)) & 1ULL)) continue;
      int i = 8 * bi + (l & 7), j = 8 * bj + ((l >> 3) & 7), k = 8 * bk + (l >> 6);
      B->lin[pos] = i + (int64_t)n * (j + (int64_t)n * k);
      B->tsdf[pos] = ts[512 * c + l];
      B->wcount[pos] = wc[512 * c + l];
      ++pos;
    }
  }
  B->off[NB] = pos;
  free(ts); free(wc); free(cmask); free(clist);

  /* 5. neighbour bricks, degree and boundary */
  for (int32_t r = 0; r < NB; ++r) {
    int bc[3] = {B->bcoord[3 * r], B->bcoord[3 * r + 1], B->bcoord[3 * r + 2]};
    for (int f = 0; f < 6; ++f) {
      int q[3] = {bc[0], bc[1], bc[2]};
      q[f >> 1] += (f & 1) ? 1 : -1;
      int32_t v = -1;
      if (q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && q[0] < nb && q[1] < nb && q[2] < nb)
        v = B->dir[q[0] + (int64_t)nb * (q[1] + (int64_t)nb * q[2])];
      B->nbr[6 * r + f] = v;
    }
  }
  for (int64_t v = 0; v < N; ++v) {
    int64_t L = B->lin[v];
    int i = (int)(L % n), j = (int)((L / n) % n), k = (int)(L / ((int64_t)n * n));
    int d = (band_index(B, i - 1, j, k) >= 0) + (band_index(B, i + 1, j, k) >= 0) +
            (band_index(B, i, j - 1, k) >= 0) + (band_index(B, i, j + 1, k) >= 0) +
            (band_index(B, i, j, k - 1) >= 0) + (band_index(B, i, j, k + 1) >= 0);
    B->deg[v] = (uint8_t)d;
    B->bdry[v] = d < 6;
  }
  return B;
}

/* --------------------------------------------------- observations (DDA) */

/* Observation precision in voxel units (noise equation of Sec. 3.5):
 * sigma_d(D) = a + b D^2 evaluated at the measured z-depth. */
static double obs_weight(double h, double D, double sa, double sb, double sp, double sm) {
  double sd = sa + sb * D * D;
  double s2 = sd * sd + sp * sp + sm * sm;
  return h * h / s2;
}

static int dda_max_steps(double band_vox) { return 3 * (int)ceil(2.0 * band_vox) + 12; }

/*
 * FP32-spec Amanatides-Woo traversal of s in [s_p - tau, s_p + tau] along the
 * pixel ray; calls visit(i,j,k) for each voxel entered (ties broken x<y<z).
 */
typedef void (*visit_fn)(void* ctx, int i, int j, int k);

static void dda(const float C[3], const float r[3], float sp, float tau, float h, const float org[3],
                int max_steps, visit_fn visit, void* ctx) {
  float s0 = sp - tau;
  if (s0 < 0.0f) s0 = 0.0f;
  float s1 = sp + tau;
  float P0[3];
  int idx[3], step[3];
  float tmax[3], tdel[3];
  for (int k = 0; k < 3; ++k) {
    P0[k] = C[k] + s0 * r[k];
    float g = (P0[k] - org[k]) / h;
    if (!(fabsf(g) < 1.0e6f)) return;
    idx[k] = (int)floorf(g);
  }
  for (int k = 0; k < 3; ++k) {
    if (r[k] > 0.0f) {
      step[k] = 1;
      tdel[k] = h / r[k];
      float bnd = org[k] + (float)(idx[k] + 1) * h;
      tmax[k] = s0 + (bnd - P0[k]) / r[k];
    } else if (r[k] < 0.0f) {
      step[k] = -1;
      tdel[k] = h / (-r[k]);
      float bnd = org[k] + (float)idx[k] * h;
      tmax[k] = s0 + (bnd - P0[k]) / r[k];
    } else {
      step[k] = 0;
      tdel[k] = INFINITY;
      tmax[k] = INFINITY;
    }
  }
  for (int it = 0; it < max_steps; ++it) {
    visit(ctx, idx[0], idx[1], idx[2]);
    int a = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
    if (tmax[a] > s1) break;
    idx[a] += step[a];
    tmax[a] = tmax[a] + tdel[a];
  }
}

typedef struct {
  const bfo_band* B;
  double r[3], p[3], w, tau, h;
  double* d;
  double* hd;
  int64_t visits, hits;
  int64_t* trace;   /* optional: record visited linear indices */
  int64_t ntrace, cap;
} integ_ctx;

static void integ_visit(void* vctx, int i, int j, int k) {
  integ_ctx* c = (integ_ctx*)vctx;
  c->visits++;
  if (c->trace && c->ntrace < c->cap) {
    int n = c->B->n;
    c->trace[c->ntrace++] = (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n)
                                ? -1 : i + (int64_t)n * (j + (int64_t)n * k);
  }
  int64_t v = band_index(c->B, i, j, k);
  if (v < 0) return;
  c->hits++;
  if (!c->d) return;
  const float* o = c->B->org;
  double xj[3] = {(double)o[0] + (i + 0.5) * c->h, (double)o[1] + (j + 0.5) * c->h,
                  (double)o[2] + (k + 0.5) * c->h};
  double y = c->r[0] * (c->p[0] - xj[0]) + c->r[1] * (c->p[1] - xj[1]) + c->r[2] * (c->p[2] - xj[2]);
  if (y > c->tau) y = c->tau;
  if (y < -c->tau) y = -c->tau;
  y /= c->h;
  c->d[v] += c->w;
  c->hd[v] += c->w * y;
}

/*
 * Depth integration (Sec. 3.5 back-projection, projective SDF, linear row,
 * noise model): d_j = sum w, hdata_j = sum w y over all observations of
 * band voxel j, in voxel units.  d, hd: [N] zeroed by the caller.
 */
void bfo_integrate(const bfo_band* B, const float* depth, int T, int H, int W, const float* poses,
                   float fx, float fy, float cx, float cy, double band_vox, double sa, double sb,
                   double sp, double sm, double* d, double* hd, int64_t* stats) {
  float tau = (float)band_vox * B->h;
  int ms = dda_max_steps(band_vox);
  integ_ctx c;
  memset(&c, 0, sizeof(c));
  c.B = B;
  c.d = d;
  c.hd = hd;
  c.h = B->h;
  c.tau = (double)band_vox * (double)B->h;
  for (int t = 0; t < T; ++t) {
    fpose P = load_pose(poses + 12 * t);
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        float D = depth[((int64_t)t * H + py) * W + px];
        if (!depth_valid(D)) continue;
        fray q = pixel_ray(&P, px, py, fx, fy, cx, cy);
        float spf = D * q.nrm;
        /* FP64 geometry of the sample */
        double a = ((double)px + 0.5 - cx) / fx, b = ((double)py + 0.5 - cy) / fy;
        double nr = sqrt(a * a + b * b + 1.0);
        for (int k = 0; k < 3; ++k) {
          double dwk = (double)P.R[3 * k] * a + (double)P.R[3 * k + 1] * b + (double)P.R[3 * k + 2];
          c.r[k] = dwk / nr;
          c.p[k] = (double)P.C[k] + (double)D * dwk;
        }
        c.w = obs_weight(B->h, D, sa, sb, sp, sm);
        dda(P.C, q.r, spf, tau, B->h, B->org, ms, integ_visit, &c);
      }
  }
  if (stats) { stats[0] = c.visits; stats[1] = c.hits; }
}

/* Voxels visited by one pixel ray's DDA (for traversal tests). */
int64_t bfo_dda_trace(const bfo_band* B, const float* pose, float fx, float fy, float cx, float cy, int px,
                      int py, float D, double band_vox, int64_t* out, int64_t cap) {
  fpose P = load_pose(pose);
  fray q = pixel_ray(&P, px, py, fx, fy, cx, cy);
  integ_ctx c;
  memset(&c, 0, sizeof(c));
  c.B = B;
  c.trace = out;
  c.cap = cap;
  dda(P.C, q.r, D * q.nrm, (float)band_vox * B->h, B->h, B->org, dda_max_steps(band_vox), integ_visit, &c);
  return c.ntrace;
}

/* ----------------------------------------------------- system assembly */

/*
 * Posterior precision and information vector (Sec. 3.6, Q0 and precision
 * equations): Q = lambda L_B + lambda_b I_dB + diag(d);
 * h = hdata + lambda_b [dB] tsdf/h.  Off-diagonals are -lambda.
 */
void bfo_assemble(const bfo_band* B, const double* d, const double* hd, double lam, double lamb,
                  double* qdiag, double* rhs) {
  for (int64_t v = 0; v < B->N; ++v) {
    qdiag[v] = lam * B->deg[v] + lamb * B->bdry[v] + d[v];
    rhs[v] = hd[v] + lamb * B->bdry[v] * ((double)B->tsdf[v] / (double)B->h);
  }
}

typedef struct {
  int64_t N;
  int64_t* rp;
  int64_t* ci;
  double* val;
} csr;

static csr build_csr(const bfo_band* B, double lam, const double* qdiag) {
  csr A;
  A.N = B->N;
  A.rp = (int64_t*)malloc(sizeof(int64_t) * (B->N + 1));
  A.ci = (int64_t*)malloc(sizeof(int64_t) * 7 * (B->N ? B->N : 1));
  A.val = (double*)malloc(sizeof(double) * 7 * (B->N ? B->N : 1));
  int n = B->n;
  int64_t e = 0;
  for (int64_t v = 0; v < B->N; ++v) {
    A.rp[v] = e;
    int64_t L = B->lin[v];
    int i = (int)(L % n), j = (int)((L / n) % n), k = (int)(L / ((int64_t)n * n));
    A.ci[e] = v; A.val[e] = qdiag[v]; ++e;
    int nbh[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    for (int f = 0; f < 6; ++f) {
      int64_t u = band_index(B, nbh[f][0], nbh[f][1], nbh[f][2]);
      if (u >= 0 && lam != 0.0) { A.ci[e] = u; A.val[e] = -lam; ++e; }
    }
  }
  A.rp[B->N] = e;
  return A;
}

static void free_csr(csr* A) { free(A->rp); free(A->ci); free(A->val); }

static void csr_mv(const csr* A, const double* x, double* y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t v = 0; v < A->N; ++v) {
    double s = 0.0;
    for (int64_t e = A->rp[v]; e < A->rp[v + 1]; ++e) s += A->val[e] * x[A->ci[e]];
    y[v] = s;
  }
}

static double dot(int64_t N, const double* a, const double* b) {
  double s = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : s) schedule(static)
#endif
  for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
  return s;
}

/* y = Q x (Sec. 3.6 precision equation) */
void bfo_spmv(const bfo_band* B, double lam, const double* qdiag, const double* x, double* y) {
  csr A = build_csr(B, lam, qdiag);
  csr_mv(&A, x, y);
  free_csr(&A);
}

/* Q in CSR for dense checks: rp [N+1], ci/val [nnz]; returns nnz (arrays may be NULL to query) */
int64_t bfo_csr(const bfo_band* B, double lam, const double* qdiag, int64_t* rp, int64_t* ci, double* val) {
  csr A = build_csr(B, lam, qdiag);
  int64_t nnz = A.rp[A.N];
  if (rp) memcpy(rp, A.rp, sizeof(int64_t) * (A.N + 1));
  if (ci) memcpy(ci, A.ci, sizeof(int64_t) * nnz);
  if (val) memcpy(val, A.val, sizeof(double) * nnz);
  free_csr(&A);
  return nnz;
}

/* PCG with Jacobi preconditioner (Sec. 3.6 MAP solve).  status: 0 converged,
 * 1 iteration limit, 2 breakdown (p.Qp <= 0). */
static int pcg_csr(const csr* A, const double* diag, const double* b, const double* x0, double tol,
                   int max_iter, double* x, int* iters, double* relres) {
  int64_t N = A->N;
  double* r = (double*)malloc(sizeof(double) * (N ? N : 1));
  double* z = (double*)malloc(sizeof(double) * (N ? N : 1));
  double* p = (double*)malloc(sizeof(double) * (N ? N : 1));
  double* q = (double*)malloc(sizeof(double) * (N ? N : 1));
  int status = 1, it = 0, restarts = 0;
  double bn = sqrt(dot(N, b, b));
#ifdef _OPENMP
  #pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < N; ++i) x[i] = x0 ? x0[i] : 0.0;
  if (bn == 0.0) {
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    *iters = 0;
    *relres = 0.0;
    free(r); free(z); free(p); free(q);
    return 0;
  }
  for (;;) {
    csr_mv(A, x, q);
#ifdef _OPENMP
    #pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - q[i];
    double rn = sqrt(dot(N, r, r));
    if (rn <= tol * bn) { status = 0; break; }
#ifdef _OPENMP
    #pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < N; ++i) { z[i] = r[i] / diag[i]; p[i] = z[i]; }
    double rho = dot(N, r, z);
    int conv = 0;
    while (it < max_iter) {
      csr_mv(A, p, q);
      double pq = dot(N, p, q);
      ++it;
      if (!(pq > 0.0)) { status = 2; break; }
      double alpha = rho / pq;
#ifdef _OPENMP
      #pragma omp parallel for schedule(static)
#endif
      for (int64_t i = 0; i < N; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
      rn = sqrt(dot(N, r, r));
      if (rn <= tol * bn) { conv = 1; break; }
#ifdef _OPENMP
      #pragma omp parallel for schedule(static)
#endif
      for (int64_t i = 0; i < N; ++i) z[i] = r[i] / diag[i];
      double rho2 = dot(N, r, z);
      double beta = rho2 / rho;
      rho = rho2;
#ifdef _OPENMP
      #pragma omp parallel for schedule(static)
#endif
      for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (status == 2 || !conv) break;
    /* true residual check; restart from x if it misses */
    if (++restarts > 3) break;
  }
  csr_mv(A, x, q);
#ifdef _OPENMP
  #pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < N; ++i) r[i] = b[i] - q[i];
  double rt = sqrt(dot(N, r, r)) / bn;
  if (status != 2) status = (rt <= tol) ? 0 : 1;
  *iters = it;
  *relres = rt;
  free(r); free(z); free(p); free(q);
  return status;
}

int bfo_pcg(const bfo_band* B, double lam, const double* qdiag, const double* rhs, const double* x0,
            double tol, int max_iter, double* x, int* iters, double* relres) {
  csr A = build_csr(B, lam, qdiag);
  int st = pcg_csr(&A, qdiag, rhs, x0, tol, max_iter, x, iters, relres);
  free_csr(&A);
  return st;
}

/* ------------------------------------------------------------- probes */

static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t bfo_splitmix64(uint64_t x) { return splitmix64(x); }

/* Rademacher entry of probe k at linear voxel index lin: +1 if the top bit of
 * the hash is 0, else -1. */
static double rademacher(uint64_t seed, uint64_t k, uint64_t lin) {
  uint64_t v = splitmix64(splitmix64(seed) ^ (k * 0xD1B54A32D192ED03ULL) ^ lin);
  return (v >> 63) ? -1.0 : 1.0;
}

void bfo_probe(uint64_t seed, uint64_t k, int64_t n, const int64_t* lin, double* z) {
#ifdef _OPENMP
  #pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) z[i] = rademacher(seed, k, (uint64_t)lin[i]);
}

/*
 * Randomized diagonal estimator (Sec. 3.7 diag equation):
 * s = (1/K) sum_k z_k (.) Q^-1 z_k.  Also returns the per-probe products
 * z_k (.) u_k summed in u_sum (= K s) and, if per_probe is non-NULL, the
 * first n_keep probe solutions u_k ([n_keep][N]).
 */
int bfo_hutchinson(const bfo_band* B, double lam, const double* qdiag, int K, uint64_t seed, double tol,
                   int max_iter, int k0, double* s, int* total_iters, double* per_probe, int n_keep) {
  int64_t N = B->N;
  csr A = build_csr(B, lam, qdiag);
  double* z = (double*)malloc(sizeof(double) * (N ? N : 1));
  double* u = (double*)malloc(sizeof(double) * (N ? N : 1));
  for (int64_t i = 0; i < N; ++i) s[i] = 0.0;
  int tot = 0, worst = 0;
  for (int k = 0; k < K; ++k) {
    bfo_probe(seed, (uint64_t)(k0 + k), N, B->lin, z);
    int it;
    double rr;
    int st = pcg_csr(&A, qdiag, z, NULL, tol, max_iter, u, &it, &rr);
    if (st > worst) worst = st;
    tot += it;
#ifdef _OPENMP
    #pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < N; ++i) s[i] += z[i] * u[i];
    if (per_probe && k < n_keep) memcpy(per_probe + (int64_t)k * N, u, sizeof(double) * N);
  }
#ifdef _OPENMP
  #pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < N; ++i) s[i] /= K;
  *total_iters = tot;
  free(z); free(u);
  free_csr(&A);
  return worst;
}

/* ------------------------------------------------------ marching cubes */

/* Cube corner c = dx + 2 dy + 4 dz.  Edge e = 4 a + u + 2 v where a is the
 * edge axis and (u, v) the cube coordinates of the other two axes in
 * increasing axis order. */
static int edge_of(int c1, int c2) {
  int diff = c1 ^ c2, a = diff == 1 ? 0 : (diff == 2 ? 1 : 2);
  int lo = c1 & c2, bits[3] = {lo & 1, (lo >> 1) & 1, (lo >> 2) & 1};
  int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
  return 4 * a + bits[o1] + 2 * bits[o2];
}

/* Polygonise one cube: for each face, walked counter-clockwise as seen from
 * outside the cube, every run of inside corners gives a directed segment
 * from the crossing where the walk enters the run to the one where it
 * leaves it.  Chaining segments gives closed loops (each crossed edge has
 * one incoming and one outgoing segment); loops are started from their
 * lowest-numbered edge, in increasing order, and fan-triangulated.
 * Returns the number of triangles, written as edge triples to tri. */
static int polygonise(int cs, int tri[][3]) {
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s) {
      int b = (a + 1) % 3, c = (a + 2) % 3;
      int q[4];
      /* (b, c) coordinates in CCW order seen from outside */
      int ob[4] = {0, 1, 1, 0}, oc[4] = {0, 0, 1, 1};
      for (int m = 0; m < 4; ++m) {
        int bb = s ? ob[m] : oc[m], cc = s ? oc[m] : ob[m];
        q[m] = (s << a) | (bb << b) | (cc << c);
      }
      for (int m = 0; m < 4; ++m) {
        int in0 = (cs >> q[m]) & 1, in1 = (cs >> q[(m + 1) & 3]) & 1;
        if (in0 || !in1) continue; /* entry: outside -> inside */
        int ent = edge_of(q[m], q[(m + 1) & 3]);
        for (int j = 1; j < 4; ++j) {
          int c0 = q[(m + j) & 3], c1 = q[(m + j + 1) & 3];
          if (((cs >> c0) & 1) && !((cs >> c1) & 1)) { next[ent] = edge_of(c0, c1); break; }
        }
      }
    }
  int used[12] = {0}, nt = 0;
  for (int e = 0; e < 12; ++e) {
    if (next[e] < 0 || used[e]) continue;
    int loop[12], m = 0, cur = e;
    do { loop[m++] = cur; used[cur] = 1; cur = next[cur]; } while (cur != e && m < 12);
    for (int i = 1; i + 1 < m; ++i) { tri[nt][0] = loop[0]; tri[nt][1] = loop[i]; tri[nt][2] = loop[i + 1]; ++nt; }
  }
  return nt;
}

int bfo_mc_case(int cs, int32_t* tri) { return polygonise(cs, (int(*)[3])tri); }

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Marching cubes (Sec. 3.8) over cubes whose 8 corner voxels are all in the
 * band.  mu: [N] float (any unit; inside = mu < 0).  Vertices are the
 * crossed grid edges used by a triangle, in ascending (compact index of the
 * edge's lower voxel, axis); a vertex sits at t = mu_a / (mu_a - mu_b) from
 * the lower voxel a, in metres.  Triangles in ascending compact index of the
 * cube's base voxel, then loop order.  Outputs are malloc'd (bfo_free).
 */
void bfo_mc(const bfo_band* B, const float* mu, int64_t* nv, double** verts, int64_t* nt, int32_t** tris) {
  int64_t N = B->N, cap = 1024, ntri = 0;
  int n = B->n;
  int64_t* tk = (int64_t*)malloc(sizeof(int64_t) * 3 * cap);
  for (int64_t v = 0; v < N; ++v) {
    int64_t L = B->lin[v];
    int i = (int)(L % n), j = (int)((L / n) % n), k = (int)(L / ((int64_t)n * n));
    int64_t ci[8];
    int ok = 1, cs = 0;
    for (int c = 0; c < 8 && ok; ++c) {
      ci[c] = band_index(B, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1));
      if (ci[c] < 0) ok = 0;
      else if (mu[ci[c]] < 0.0f) cs |= 1 << c;
    }
    if (!ok || cs == 0 || cs == 255) continue;
    int tri[16][3];
    int m = polygonise(cs, tri);
    for (int t = 0; t < m; ++t) {
      if (ntri == cap) { cap *= 2; tk = (int64_t*)realloc(tk, sizeof(int64_t) * 3 * cap); }
      for (int q = 0; q < 3; ++q) {
        int e = tri[t][q], a = e >> 2, u = e & 1, w = (e >> 1) & 1;
        int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
        int lo[3] = {0, 0, 0};
        lo[o1] = u;
        lo[o2] = w;
        int c = lo[0] | (lo[1] << 1) | (lo[2] << 2);
        tk[3 * ntri + q] = ci[c] * 3 + a; /* edge key: (lower voxel, axis) */
      }
      ++ntri;
    }
  }
  int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * 3 * (ntri ? ntri : 1));
  memcpy(keys, tk, sizeof(int64_t) * 3 * ntri);
  qsort(keys, 3 * ntri, sizeof(int64_t), cmp_i64);
  int64_t nu = 0;
  for (int64_t q = 0; q < 3 * ntri; ++q)
    if (q == 0 || keys[q] != keys[q - 1]) keys[nu++] = keys[q];
  double* V = (double*)malloc(sizeof(double) * 3 * (nu ? nu : 1));
  for (int64_t q = 0; q < nu; ++q) {
    int64_t va = keys[q] / 3;
    int a = (int)(keys[q] % 3);
    int64_t L = B->lin[va];
    int ijk[3] = {(int)(L % n), (int)((L / n) % n), (int)(L / ((int64_t)n * n))};
    int ijk2[3] = {ijk[0], ijk[1], ijk[2]};
    ijk2[a] += 1;
    int64_t vb = band_index(B, ijk2[0], ijk2[1], ijk2[2]);
    double ma = mu[va], mb = mu[vb];
    double t = ma / (ma - mb);
    for (int d = 0; d < 3; ++d) V[3 * q + d] = (double)B->org[d] + (ijk[d] + 0.5) * (double)B->h;
    V[3 * q + a] += t * (double)B->h;
  }
  int32_t* TR = (int32_t*)malloc(sizeof(int32_t) * 3 * (ntri ? ntri : 1));
  for (int64_t q = 0; q < 3 * ntri; ++q) {
    int64_t lo = 0, hi = nu - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (keys[mid] < tk[q]) lo = mid + 1; else hi = mid;
    }
    TR[q] = (int32_t)lo;
  }
  free(tk);
  free(keys);
  *nv = nu;
  *verts = V;
  *nt = ntri;
  *tris = TR;
}

void bfo_free(void* p) { free(p); }

/* ------------------------------------------------------ view scoring */

/* FP32 spec trilinear interpolation of mu at world point x; 0 if any of the
 * 8 surrounding voxel centres is outside the band. */
static int interp_mu(const bfo_band* B, const float* mu, const float x[3], float* out) {
  int id[3];
  float fr[3];
  for (int k = 0; k < 3; ++k) {
    float g = (x[k] - B->org[k]) / B->h - 0.5f;
    if (!(fabsf(g) < 1.0e6f)) return 0;
    float fl = floorf(g);
    id[k] = (int)fl;
    fr[k] = g - fl;
  }
  float v[8];
  for (int c = 0; c < 8; ++c) {
    int64_t q = band_index(B, id[0] + (c & 1), id[1] + ((c >> 1) & 1), id[2] + ((c >> 2) & 1));
    if (q < 0) return 0;
    v[c] = mu[q];
  }
  float c00 = v[0] + (v[1] - v[0]) * fr[0], c10 = v[2] + (v[3] - v[2]) * fr[0];
  float c01 = v[4] + (v[5] - v[4]) * fr[0], c11 = v[6] + (v[7] - v[6]) * fr[0];
  float c0 = c00 + (c10 - c00) * fr[1], c1 = c01 + (c11 - c01) * fr[1];
  *out = c0 + (c1 - c0) * fr[2];
  return 1;
}

/* FP32 spec ray cast of the zero crossing (outside -> inside) of the mu
 * interpolant: march at h/2 from the grid entry, then 10 bisection steps.
 * Returns the predicted z-depth, or 0 if the ray finds no crossing. */
static float raycast_depth(const bfo_band* B, const float* mu, const float C[3], const fray* q) {
  float lo_b[3], hi_b[3], sn = 0.0f, sx = INFINITY;
  float ext = (float)B->n * B->h;
  for (int k = 0; k < 3; ++k) {
    lo_b[k] = B->org[k];
    hi_b[k] = B->org[k] + ext;
    if (q->r[k] != 0.0f) {
      float t0 = (lo_b[k] - C[k]) / q->r[k], t1 = (hi_b[k] - C[k]) / q->r[k];
      if (t0 > t1) { float tt = t0; t0 = t1; t1 = tt; }
      if (t0 > sn) sn = t0;
      if (t1 < sx) sx = t1;
    } else if (C[k] < lo_b[k] || C[k] > hi_b[k]) {
      return 0.0f;
    }
  }
  if (!(sn < sx)) return 0.0f;
  float hs = 0.5f * B->h;
  int have_prev = 0;
  float prev_v = 0.0f, prev_s = 0.0f;
  for (int k = 0;; ++k) {
    float s = sn + (float)k * hs;
    if (s > sx) break;
    float x[3] = {C[0] + s * q->r[0], C[1] + s * q->r[1], C[2] + s * q->r[2]};
    float v;
    if (!interp_mu(B, mu, x, &v)) { have_prev = 0; continue; }
    if (have_prev && prev_v > 0.0f && v <= 0.0f) {
      float lo = prev_s, hi = s;
      for (int it = 0; it < 10; ++it) {
        float mid = 0.5f * (lo + hi);
        float xm[3] = {C[0] + mid * q->r[0], C[1] + mid * q->r[1], C[2] + mid * q->r[2]};
        float vm;
        if (interp_mu(B, mu, xm, &vm) && vm > 0.0f) lo = mid; else hi = mid;
      }
      return (0.5f * (lo + hi)) / q->nrm;
    }
    have_prev = 1;
    prev_v = v;
    prev_s = s;
  }
  return 0.0f;
}

typedef struct {
  const bfo_band* B;
  double w;
  double* dd;
} dd_ctx;

static void dd_visit(void* vctx, int i, int j, int k) {
  dd_ctx* c = (dd_ctx*)vctx;
  int64_t v = band_index(c->B, i, j, k);
  if (v >= 0) c->dd[v] += c->w;
}

/* Predicted depth map of a candidate view (for tests): depth [H][W]. */
void bfo_predict_depth(const bfo_band* B, const float* mu, const float* pose, float fx, float fy, float cx,
                       float cy, int W, int H, float* depth) {
  fpose P = load_pose(pose);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      fray q = pixel_ray(&P, px, py, fx, fy, cx, cy);
      depth[(int64_t)py * W + px] = raycast_depth(B, mu, P.C, &q);
    }
}

/*
 * Next-best-view utility (Sec. 3.8 NBV equation).  For each candidate view:
 * predicted depth by ray casting mu, predicted precision increments dd from
 * the same observation model as integration, and
 * U = sum_{|mu_i| <= eps} (s_i - 1/(1/s_i + dd_i)), with s_i floored at
 * 1/Q_ii.  mu in voxel units (float), s in voxel^2.  U: [V]; returns argmax
 * (lowest index on ties).
 */
int bfo_score_views(const bfo_band* B, const float* mu, const double* s, const double* qdiag,
                    const float* cand, int V, float fx, float fy, float cx, float cy, int W, int H,
                    double band_vox, double sa, double sb, double sp, double sm, double eps, double* U) {
  int64_t N = B->N;
  double* dd = (double*)malloc(sizeof(double) * (N ? N : 1));
  float tau = (float)band_vox * B->h;
  int ms = dda_max_steps(band_vox), best = 0;
  for (int v = 0; v < V; ++v) {
    memset(dd, 0, sizeof(double) * N);
    fpose P = load_pose(cand + 12 * v);
    dd_ctx c = {B, 0.0, dd};
    for (int py = 0; py < H; ++py)
      for (int px = 0; px < W; ++px) {
        fray q = pixel_ray(&P, px, py, fx, fy, cx, cy);
        float D = raycast_depth(B, mu, P.C, &q);
        if (!depth_valid(D)) continue;
        c.w = obs_weight(B->h, D, sa, sb, sp, sm);
        dda(P.C, q.r, D * q.nrm, tau, B->h, B->org, ms, dd_visit, &c);
      }
    double u = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      if (!(fabs((double)mu[i]) <= eps)) continue;
      double si = s[i], fl = 1.0 / qdiag[i];
      if (!(si >= fl)) si = fl;
      /* s - 1/(1/s + dd), written without cancellation */
      u += si * si * dd[i] / (1.0 + si * dd[i]);
    }
    U[v] = u;
    if (u > U[best]) best = v;
  }
  free(dd);
  return best;
}

/* ------------------------------------------- learned-part input tiles */

/* Network inputs of every active brick: a 10^3 tile (brick + 1-voxel halo,
 * tile index tx + 10 ty + 100 tz), channel 0 = tsdf/h, channel 1 =
 * log(1 + d) at band voxels, 0 elsewhere.  feat: [NB][1000][2]. */
void bfo_net_features(const bfo_band* B, const double* d, double* feat) {
  for (int32_t r = 0; r < B->NB; ++r) {
    const int* bc = B->bcoord + 3 * (int64_t)r;
    for (int tz = 0; tz < 10; ++tz)
      for (int ty = 0; ty < 10; ++ty)
        for (int tx = 0; tx < 10; ++tx) {
          int64_t v = band_index(B, 8 * bc[0] + tx - 1, 8 * bc[1] + ty - 1, 8 * bc[2] + tz - 1);
          double* f = feat + ((int64_t)r * 1000 + tx + 10 * ty + 100 * tz) * 2;
          f[0] = v >= 0 ? (double)B->tsdf[v] / (double)B->h : 0.0;
          f[1] = v >= 0 ? log1p(d[v]) : 0.0;
        }
  }
}
