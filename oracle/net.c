/*
 * Oracle of the learned warm start / variance surrogate -- TEST
 * INFRASTRUCTURE (tests, smoke check, CPU baseline only).
 *
 * The network is not part of the paper (its Sec. 6 names prior learning as
 * future work); it is defined here, in plain FP64 loops, as the reference for
 * the CUDA kernels:
 *   input   per active brick a 10^3 tile (the 8^3 brick and a 1-voxel halo),
 *           2 channels: tsdf/h and log(1 + d) at band voxels, 0 elsewhere;
 *   layers  four 3x3x3 convolutions 2 -> 32 -> 32 -> 32 -> 2 with bias,
 *           zero padding at the tile boundary ("same" size 10^3), ReLU after
 *           the first three;
 *   output  at the 8^3 centre: mu_hat = tsdf/h + o0 (voxels) and
 *           log s_hat = o1 - log Q_ii (both outputs are residuals on a
 *           closed-form baseline: the TSDF, and the Jacobi value 1/Q_ii that
 *           bounds (Q^-1)_ii from below for SPD Q);
 *   loss    L = (1/M) sum over band voxels of (mu_hat - mu)^2 + (log s_hat - log s)^2.
 * Weights W_l[tap][ci][co], tap = (dz+1) 9 + (dy+1) 3 + (dx+1), then b_l[co];
 * the flat parameter vector is W1 b1 W2 b2 W3 b3 W4 b4.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TV 1000
static const int CIN[4] = {2, 32, 32, 32};
static const int COUT[4] = {32, 32, 32, 2};

int64_t bfo_net_nparams(void) {
  int64_t n = 0;
  for (int l = 0; l < 4; ++l) n += 27 * CIN[l] * COUT[l] + COUT[l];
  return n;
}

static int shift(int v, int tap) {
  int tx = v % 10, ty = (v / 10) % 10, tz = v / 100;
  int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
  tx += dx;
  ty += dy;
  tz += dz;
  if (tx < 0 || ty < 0 || tz < 0 || tx > 9 || ty > 9 || tz > 9) return -1;
  return tx + 10 * ty + 100 * tz;
}

static void conv_fwd(const double* W, const double* b, int ci_n, int co_n, const double* x, double* y, int relu) {
  for (int v = 0; v < TV; ++v)
    for (int co = 0; co < co_n; ++co) {
      double s = b[co];
      for (int tap = 0; tap < 27; ++tap) {
        int u = shift(v, tap);
        if (u < 0) continue;
        for (int ci = 0; ci < ci_n; ++ci) s += W[(tap * ci_n + ci) * co_n + co] * x[u * ci_n + ci];
      }
      y[v * co_n + co] = relu ? (s > 0 ? s : 0) : s;
    }
}

/*
 * Loss, gradient and predictions over NB brick tiles.
 *   feat [NB][1000][2] inputs; lq [NB][512] log Q_ii at the centre voxels
 *   (local index lx + 8 ly + 64 lz); tgt [NB][512][2] targets (mu, log s);
 *   mask [NB][512] 1 = band.  grad [P] (may be NULL); pred [NB][512][2]
 *   (may be NULL).
 */
double bfo_net_loss(const double* params, int NB, const double* feat, const double* lq, const double* tgt,
                    const uint8_t* mask, double* grad, double* pred) {
  const double* W[4];
  const double* B[4];
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    W[l] = params + off;
    off += 27 * CIN[l] * COUT[l];
    B[l] = params + off;
    off += COUT[l];
  }
  if (grad) memset(grad, 0, sizeof(double) * off);
  double* gW[4];
  double* gB[4];
  if (grad) {
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
      gW[l] = grad + o;
      o += 27 * CIN[l] * COUT[l];
      gB[l] = grad + o;
      o += COUT[l];
    }
  }
  int64_t M = 0;
  for (int64_t q = 0; q < (int64_t)NB * 512; ++q) M += mask[q] != 0;
  if (M == 0) return 0.0;
  double* act[5];
  act[0] = NULL;
  for (int l = 0; l < 4; ++l) act[l + 1] = (double*)malloc(sizeof(double) * TV * COUT[l]);
  double* g[5];
  for (int l = 0; l < 5; ++l) g[l] = (double*)malloc(sizeof(double) * TV * 32);
  double loss = 0.0;
  for (int b = 0; b < NB; ++b) {
    const double* x0 = feat + (int64_t)b * TV * 2;
    act[0] = (double*)x0;
    for (int l = 0; l < 4; ++l) conv_fwd(W[l], B[l], CIN[l], COUT[l], act[l], act[l + 1], l < 3);
    /* loss and its gradient at the output */
    memset(g[4], 0, sizeof(double) * TV * 2);
    for (int lz = 0; lz < 8; ++lz)
      for (int ly = 0; ly < 8; ++ly)
        for (int lx = 0; lx < 8; ++lx) {
          int loc = lx + 8 * ly + 64 * lz, v = (lx + 1) + 10 * (ly + 1) + 100 * (lz + 1);
          double mh = x0[v * 2] + act[4][v * 2], lh = act[4][v * 2 + 1] - lq[(int64_t)b * 512 + loc];
          if (pred) {
            pred[((int64_t)b * 512 + loc) * 2] = mh;
            pred[((int64_t)b * 512 + loc) * 2 + 1] = lh;
          }
          if (!mask[(int64_t)b * 512 + loc]) continue;
          double e0 = mh - tgt[((int64_t)b * 512 + loc) * 2], e1 = lh - tgt[((int64_t)b * 512 + loc) * 2 + 1];
          loss += (e0 * e0 + e1 * e1) / M;
          g[4][v * 2] = 2 * e0 / M;
          g[4][v * 2 + 1] = 2 * e1 / M;
        }
    if (!grad) continue;
    /* backward through the four layers */
    for (int l = 3; l >= 0; --l) {
      const int ci_n = CIN[l], co_n = COUT[l];
      double* gy = g[l + 1];
      if (l < 3)
        for (int q = 0; q < TV * co_n; ++q)
          if (!(act[l + 1][q] > 0)) gy[q] = 0; /* ReLU */
      const double* x = act[l];
      for (int v = 0; v < TV; ++v)
        for (int co = 0; co < co_n; ++co) {
          double d = gy[v * co_n + co];
          if (d == 0) continue;
          gB[l][co] += d;
          for (int tap = 0; tap < 27; ++tap) {
            int u = shift(v, tap);
            if (u < 0) continue;
            for (int ci = 0; ci < ci_n; ++ci) gW[l][(tap * ci_n + ci) * co_n + co] += x[u * ci_n + ci] * d;
          }
        }
      if (l == 0) break;
      double* gx = g[l];
      memset(gx, 0, sizeof(double) * TV * ci_n);
      for (int v = 0; v < TV; ++v)
        for (int co = 0; co < co_n; ++co) {
          double d = gy[v * co_n + co];
          if (d == 0) continue;
          for (int tap = 0; tap < 27; ++tap) {
            int u = shift(v, tap);
            if (u < 0) continue;
            for (int ci = 0; ci < ci_n; ++ci) gx[u * ci_n + ci] += W[l][(tap * ci_n + ci) * co_n + co] * d;
          }
        }
    }
  }
  for (int l = 1; l < 5; ++l) free(act[l]);
  for (int l = 0; l < 5; ++l) free(g[l]);
  return loss;
}
