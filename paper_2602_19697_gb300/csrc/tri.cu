// Trilinear observation rows and the 27-point posterior precision they give.
//
// Sec. 3.5 writes each depth observation as a linear row a_i over the voxel
// values holding the trilinear interpolation weights of the sample point,
// one for each of the 8 voxel centres of the cell around it.  Then A^T W A
// (Sec. 3.6 precision equation) couples every voxel with its 26 neighbours
// and Q = lambda L + lambda_b I_dB + A^T W A is a 27-point stencil with
// per-voxel coefficients; h = A^T W y + b0 as before.
//
// Samples: on every valid pixel's ray at s_p + k h, |k| <= floor(band_vox)
// (2b + 1 per ray), observed value y = -k voxels (the projective SDF with
// n = -r), precision w = h^2 / sigma^2 as for the voxel-binned rows.  The
// cell, the weights and which corners count follow an FP32 specification
// (separately rounded operations in a fixed order, tri_row), so the rows are
// reproducible bit for bit; a row is used when every corner with a non-zero
// weight is a band voxel.
//
// Integration (k_tri_integrate): one thread per pixel; for each used sample
// d += w wt_c, hdata += w wt_c y at the corners and, for each pair of corners
// c <= c', w wt_c wt_c' onto the coupling of the pair, stored once at the
// corner from which the other lies at an offset o >= 13 of the 27-point
// neighbourhood (o = (dx + 1) + 3 (dy + 1) + 9 (dz + 1)); FP32 L2 atomics.
// Assembly (k_tri_assemble) fills all 27 coefficients of each voxel (the
// other half by symmetry from the neighbour's entry) and adds the prior.
//
// SpMV (k_spmv27): one 128-thread CTA per brick at a time; the brick and a
// one-voxel halo from its 26 neighbour bricks are staged in a 10^3 tile (0
// off the band), then y_j = sum_o Q[o][j] x(j + off(o)) in the fixed order
// o = 0 .. 26.  The coefficients ([27][N], coalesced per offset) are the
// stream: 108 bytes per band voxel plus x and y.
//
// Solvers: Jacobi PCG per column (two reductions per iteration, FP32
// vectors, FP64 inner products) for C = 1 (the mean) or C = TRI_R probe
// columns ([N][C] layout), inside FP64 iterative refinement: the true
// residual b - Q x of the FP64 master iterate (FP64 SpMV) decides
// convergence and is the next correction solve's right-hand side.  The host
// drives the iterations.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace {

constexpr int TB = 128;        // threads per brick CTA
constexpr int NRED = 152 * 4;  // CTAs of the reduction kernels
constexpr int MAXC = TRI_R;

__device__ __forceinline__ int tri_off(int o, int a) { return (a == 0 ? o % 3 : (a == 1 ? (o / 3) % 3 : o / 9)) - 1; }

struct TriRow {
  int idx[8];
  float wt[8];
  bool used;
};

// The FP32-specification row of the sample at s = s_p + k h on the pixel ray.
__device__ __forceinline__ TriRow tri_row(const BandView& B, const Pose& P, const Ray& ray, float sp, float kh) {
  TriRow row;
  const float org[3] = {B.o0, B.o1, B.o2};
  const float s = f_add(sp, kh);
  float f[3];
  int i0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = f_add(P.C[a], f_mul(s, ray.r[a]));
    const float g = f_sub(f_div(f_sub(q, org[a]), B.h), 0.5f);
    const float fl = floorf(g);
    i0[a] = fabsf(fl) < 1.0e8f ? (int)fl : (fl > 0.0f ? (1 << 30) : -(1 << 30));
    f[a] = f_sub(g, fl);
  }
  row.used = true;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const float wx = cx ? f[0] : f_sub(1.0f, f[0]);
    const float wy = cy ? f[1] : f_sub(1.0f, f[1]);
    const float wz = cz ? f[2] : f_sub(1.0f, f[2]);
    const float w = f_mul(f_mul(wx, wy), wz);
    const int j = band_lookup(B, i0[0] + cx, i0[1] + cy, i0[2] + cz);
    if (j < 0 && w != 0.0f) row.used = false;
    row.idx[c] = j < 0 ? 0 : j;
    row.wt[c] = w;
  }
  if (!row.used) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      row.idx[c] = 0;
      row.wt[c] = 0.0f;
    }
  }
  return row;
}

__device__ __forceinline__ void pixel_of(int64_t q, const Intr& K, int* t, int* px, int* py) {
  *t = (int)(q / ((int64_t)K.H * K.W));
  const int rem = (int)(q - (int64_t)(*t) * K.H * K.W);
  *py = rem / K.W;
  *px = rem - *py * K.W;
}

__global__ void __launch_bounds__(256) k_tri_integrate(BandView B, const float* __restrict__ depth, int T, Intr K,
                                                       const float* __restrict__ poses, int nk, float sa, float sb,
                                                       float s2_extra, float* __restrict__ d, float* __restrict__ hd,
                                                       float* __restrict__ c27) {
  const int64_t npix = (int64_t)T * K.H * K.W;
  const float h = B.h;
  const size_t N = (size_t)B.N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
    const float D = __ldg(depth + q);
    if (!depth_ok(D)) continue;
    int t, px, py;
    pixel_of(q, K, &t, &px, &py);
    const Pose P = load_pose(poses + 12 * t);
    const Ray ray = pixel_ray(P, px, py, K);
    const float sp = f_mul(D, ray.nrm);
    const float sd = sa + sb * D * D;
    const float w = (h * h) / (sd * sd + s2_extra);
    for (int kk = -nk; kk <= nk; ++kk) {
      const TriRow row = tri_row(B, P, ray, sp, f_mul((float)kk, h));
      if (!row.used) continue;
      const float y = (float)(-kk);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float wc = row.wt[c];
        if (wc == 0.0f) continue;
        const float a = w * wc;
        atomicAdd(d + row.idx[c], a);
        atomicAdd(hd + row.idx[c], a * y);
#pragma unroll
        for (int c2 = c; c2 < 8; ++c2) {
          const float wc2 = row.wt[c2];
          if (wc2 == 0.0f) continue;
          // offset of corner c2 from corner c, each component in {-1, 0, 1}
          const int o = ((c2 & 1) - (c & 1) + 1) + 3 * (((c2 >> 1) & 1) - ((c >> 1) & 1) + 1) +
                        9 * (((c2 >> 2) & 1) - ((c >> 2) & 1) + 1);
          const float v = a * wc2;
          if (o >= 13) atomicAdd(c27 + (size_t)(o - 13) * N + row.idx[c], v);
          else atomicAdd(c27 + (size_t)(13 - o) * N + row.idx[c2], v);  // 26 - o >= 13, seen from corner c2
        }
      }
    }
  }
}

// Rows of every sample (frames, pixels row by row, k = -b .. b) for the export: invalid pixels give unused rows.
__global__ void __launch_bounds__(256) k_tri_rows(BandView B, const float* __restrict__ depth, int T, Intr K,
                                                  const float* __restrict__ poses, int nk, int32_t* __restrict__ idx,
                                                  float* __restrict__ wts, uint8_t* __restrict__ used) {
  const int64_t npix = (int64_t)T * K.H * K.W;
  const int ns = 2 * nk + 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
    const float D = __ldg(depth + q);
    const bool ok = depth_ok(D);
    int t, px, py;
    pixel_of(q, K, &t, &px, &py);
    const Pose P = load_pose(poses + 12 * t);
    const Ray ray = pixel_ray(P, px, py, K);
    const float sp = f_mul(ok ? D : 0.0f, ray.nrm);
    for (int kk = -nk; kk <= nk; ++kk) {
      const int64_t m = q * ns + (kk + nk);
      TriRow row;
      if (ok) {
        row = tri_row(B, P, ray, sp, f_mul((float)kk, B.h));
      } else {
        row.used = false;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          row.idx[c] = 0;
          row.wt[c] = 0.0f;
        }
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        idx[8 * m + c] = row.idx[c];
        wts[8 * m + c] = row.wt[c];
      }
      used[m] = row.used;
    }
  }
}

// Q[o][j] for all 27 offsets, qd = Q[13], rhs = hdata + lambda_b [dB] tsdf / h.
__global__ void k_tri_assemble(BandView B, const uint8_t* __restrict__ info, const float* __restrict__ tsdf,
                               const float* __restrict__ hd, const float* __restrict__ c27, float lam, float lamb,
                               float inv_h, float* __restrict__ q27, float* __restrict__ qd, float* __restrict__ rhs) {
  const size_t N = (size_t)B.N;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    const int L = __ldg(B.lin + v);
    const int i = L % B.n, j = (L / B.n) % B.n, k = L / (B.n * B.n);
    const int inf = info[v];
    const float deg = (float)(inf & 7), bd = (float)(inf >> 3);
    for (int o = 0; o < 27; ++o) {
      const int dx = tri_off(o, 0), dy = tri_off(o, 1), dz = tri_off(o, 2);
      float val = 0.0f;
      if (o == 13) {
        val = c27[v] + (lam * deg + lamb * bd);
      } else {
        const int u = band_lookup(B, i + dx, j + dy, k + dz);
        if (u >= 0) {
          val = o > 13 ? c27[(size_t)(o - 13) * N + v] : c27[(size_t)(13 - o) * N + u];
          if (abs(dx) + abs(dy) + abs(dz) == 1) val -= lam;
        }
      }
      q27[(size_t)o * N + v] = val;
    }
    qd[v] = q27[(size_t)13 * N + v];
    rhs[v] = hd[v] + lamb * bd * tsdf[v] * inv_h;
  }
}

// Y = Q X for C columns ([N][C]); TI: type of X, TO: type of Y and of the sums.
template <int C, class TI, class TO>
__global__ void __launch_bounds__(TB) k_spmv27(BandView B, const float* __restrict__ q27, const TI* __restrict__ X,
                                               TO* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char tri_smem[];
  TI* tile = reinterpret_cast<TI*>(tri_smem);  // [1000][C]
  __shared__ int nrank[27];                      // ranks of the brick and its 26 neighbours (-1: none)
  const size_t N = (size_t)B.N;
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    if (threadIdx.x < 27) {
      const int o = threadIdx.x;
      const int ci = __ldg(B.bcoord + 4 * b) + o % 3 - 1, cj = __ldg(B.bcoord + 4 * b + 1) + (o / 3) % 3 - 1,
                ck = __ldg(B.bcoord + 4 * b + 2) + o / 9 - 1;
      const bool in = (unsigned)ci < (unsigned)B.nb && (unsigned)cj < (unsigned)B.nb && (unsigned)ck < (unsigned)B.nb;
      nrank[o] = in ? __ldg(B.dir + (ci + B.nb * (cj + B.nb * ck))) : -1;
    }
    __syncthreads();
    // all of the thread's slots at once, so that their lookup and load chains overlap
#pragma unroll
    for (int k = 0; k < (1000 + TB - 1) / TB; ++k) {
      const int sl = threadIdx.x + k * TB;
      if (sl < 1000) {
        const int gx = sl % 10 - 1, gy = (sl / 10) % 10 - 1, gz = sl / 100 - 1;  // in [-1, 8] per axis
        const int dx = (gx > 7) - (gx < 0), dy = (gy > 7) - (gy < 0), dz = (gz > 7) - (gz < 0);
        const int r = nrank[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
        const int l = (gx - 8 * dx) + 8 * (gy - 8 * dy) + 64 * (gz - 8 * dz);
        int u = -1;
        if (r >= 0) {
          const MetaWord m = B.meta[16 * r + (l >> 5)];
          const uint32_t bit = 1u << (l & 31);
          if (m.bits & bit) u = m.base + __popc(m.bits & (bit - 1u));
        }
#pragma unroll
        for (int c = 0; c < C; ++c) tile[sl * C + c] = u >= 0 ? X[(size_t)u * C + c] : TI(0);
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int e = threadIdx.x; e < 512 * C; e += TB) {
      const int l = e / C, c = e - l * C;
      const MetaWord m = B.meta[16 * b + (l >> 5)];
      const uint32_t bit = 1u << (l & 31);
      if (!(m.bits & bit)) continue;
      const int v = m.base + __popc(m.bits & (bit - 1u));
      const int p = ((l & 7) + 1) + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1);
      TO acc = TO(0);
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        const int to = (o % 3 - 1) + 10 * ((o / 3) % 3 - 1) + 100 * (o / 9 - 1);
        acc += (TO)__ldg(q27 + (size_t)o * N + v) * (TO)tile[(p + to) * C + c];
      }
      Y[(size_t)v * C + c] = acc;
    }
    __syncthreads();
  }
}

// ---- PCG over C columns -----------------------------------------------------

struct TriState {
  double rho[MAXC], alpha[MAXC], beta[MAXC], rr[MAXC], rs[MAXC], eta2[MAXC];
  double rt2[MAXC], bb[MAXC], tol2;
  int done[MAXC], conv[MAXC], iters[MAXC];
  int status, all_done, all_conv, live;
};

// per-CTA FP64 partials part[q][c][NRED] of NQ quantities
template <int C, int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ][C], double* part) {
  __shared__ double sh[NQ][C][8];
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double x = v[q][c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[q][c][wrp] = x;
    }
  __syncthreads();
  if (threadIdx.x < NQ * C) {
    const int q = threadIdx.x / C, c = threadIdx.x % C;
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[q][c][w];
    part[((size_t)q * C + c) * NRED + blockIdx.x] = s;
  }
}

// true residual of the master iterate: rt = B - QX (FP64), rf = rt as float; partials |rt|^2, |B|^2
template <int C>
__global__ void __launch_bounds__(256) k_tri_resid(int N, const float* __restrict__ Bv, const double* __restrict__ qx,
                                                   float* __restrict__ rf, double* part) {
  double v[2][C];
#pragma unroll
  for (int c = 0; c < C; ++c) v[0][c] = v[1][c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t e = (size_t)i * C + c;
      const double b = Bv[e], r = b - qx[e];
      rf[e] = (float)r;
      v[0][c] += r * r;
      v[1][c] += b * b;
    }
  }
  block_partials<C, 2>(v, part);
}

// start of a correction solve: x = 0, z = r / qd, p = z; partials r.z, r.r
template <int C>
__global__ void __launch_bounds__(256) k_tri_start(int N, const float* __restrict__ qd, const float* __restrict__ r,
                                                   float* __restrict__ x, float* __restrict__ z, float* __restrict__ p,
                                                   double* part) {
  double v[2][C];
#pragma unroll
  for (int c = 0; c < C; ++c) v[0][c] = v[1][c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const float iq = 1.0f / qd[i];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t e = (size_t)i * C + c;
      const float rv = r[e], zv = rv * iq;
      x[e] = 0.0f;
      z[e] = zv;
      p[e] = zv;
      v[0][c] += (double)rv * zv;
      v[1][c] += (double)rv * rv;
    }
  }
  block_partials<C, 2>(v, part);
}

// partial p.q
template <int C>
__global__ void __launch_bounds__(256) k_tri_pq(int N, const float* __restrict__ p, const float* __restrict__ q,
                                                double* part) {
  double v[1][C];
#pragma unroll
  for (int c = 0; c < C; ++c) v[0][c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t e = (size_t)i * C + c;
      v[0][c] += (double)p[e] * q[e];
    }
  block_partials<C, 1>(v, part);
}

// x += alpha p, r -= alpha q, z = r / qd; partials r.z, r.r
template <int C>
__global__ void __launch_bounds__(256) k_tri_upd(int N, const TriState* __restrict__ st, const float* __restrict__ qd,
                                                 const float* __restrict__ p, const float* __restrict__ q,
                                                 float* __restrict__ x, float* __restrict__ r, float* __restrict__ z,
                                                 double* part) {
  float al[C];
#pragma unroll
  for (int c = 0; c < C; ++c) al[c] = (float)st->alpha[c];
  double v[2][C];
#pragma unroll
  for (int c = 0; c < C; ++c) v[0][c] = v[1][c] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const float iq = 1.0f / qd[i];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t e = (size_t)i * C + c;
      x[e] += al[c] * p[e];
      const float rv = r[e] - al[c] * q[e], zv = rv * iq;
      r[e] = rv;
      z[e] = zv;
      v[0][c] += (double)rv * zv;
      v[1][c] += (double)rv * rv;
    }
  }
  block_partials<C, 2>(v, part);
}

// p = z + beta p
template <int C>
__global__ void __launch_bounds__(256) k_tri_dir(int N, const TriState* __restrict__ st, const float* __restrict__ z,
                                                 float* __restrict__ p) {
  float be[C];
#pragma unroll
  for (int c = 0; c < C; ++c) be[c] = (float)st->beta[c];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const size_t e = (size_t)i * C + c;
      p[e] = z[e] + be[c] * p[e];
    }
}

// xm += x (FP64 master iterate)
template <int C>
__global__ void k_tri_acc(int N, const float* __restrict__ x, double* __restrict__ xm) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)N * C; e += (size_t)gridDim.x * blockDim.x)
    xm[e] += (double)x[e];
}

// Fixed-order sums of the partials and the scalar updates of one step (one CTA).
constexpr int RED_RES = 0, RED_START = 1, RED_PQ = 2, RED_UPD = 3;
template <int C>
__global__ void k_tri_reduce(TriState* st, const double* __restrict__ part, int mode, int ncols, int max_iter) {
  __shared__ double tot[2][C];
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  const int nq = mode == RED_PQ ? 1 : 2;
  for (int qc = wrp; qc < nq * C; qc += blockDim.x >> 5) {
    const double* pp = part + (size_t)qc * NRED;
    double s = 0.0;
    for (int i = lane; i < NRED; i += 32) s += pp[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tot[qc / C][qc % C] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int live = 0, all_conv = 1;
  for (int c = 0; c < C; ++c) {
    if (c >= ncols) {
      st->done[c] = 1;
      st->conv[c] = 1;
      st->alpha[c] = st->beta[c] = 0.0;
      continue;
    }
    if (mode == RED_RES) {
      st->rt2[c] = tot[0][c];
      st->bb[c] = tot[1][c];
      st->conv[c] = tot[0][c] <= st->tol2 * tot[1][c] || tot[1][c] == 0.0;
      double eta = st->conv[c] ? 0.5 : 0.5 * sqrt(st->tol2 * tot[1][c] / tot[0][c]);
      eta = fmin(fmax(eta, 1e-7), 0.5);
      st->eta2[c] = eta * eta;
    } else if (mode == RED_START) {
      st->rho[c] = tot[0][c];
      st->rs[c] = tot[1][c];
      st->done[c] = st->conv[c] || tot[1][c] == 0.0;
      st->alpha[c] = st->beta[c] = 0.0;
    } else if (mode == RED_PQ) {
      if (!st->done[c]) {
        const double pq = tot[0][c];
        if (!(pq > 0.0) || !isfinite(pq)) {
          st->done[c] = 1;
          st->status = 2;
          st->alpha[c] = 0.0;
        } else {
          st->alpha[c] = st->rho[c] / pq;
        }
      } else {
        st->alpha[c] = 0.0;
      }
    } else {  // RED_UPD
      if (!st->done[c]) {
        st->iters[c] += 1;
        const double rz = tot[0][c], rr = tot[1][c];
        st->rr[c] = rr;
        if (!isfinite(rr) || !isfinite(rz)) {
          st->done[c] = 1;
          st->status = 2;
        } else if (rr <= st->eta2[c] * st->rs[c] || st->iters[c] >= max_iter) {
          st->done[c] = 1;
        } else {
          st->beta[c] = rz / st->rho[c];
          st->rho[c] = rz;
        }
      }
      if (st->done[c]) st->alpha[c] = st->beta[c] = 0.0;
    }
    live |= !st->done[c];
    all_conv &= st->conv[c];
  }
  st->live = live;
  st->all_conv = all_conv;
}

__global__ void k_tri_state_init(TriState* st, double tol) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    memset(st, 0, sizeof(TriState));
    st->tol2 = tol * tol;
  }
}

// probe right-hand sides: B[i][c] = z_{k0 + c}(lin_i) for c < ncols, else 0
template <int C>
__global__ void k_tri_probes(int N, const int32_t* __restrict__ lin, uint64_t mseed, int k0, int ncols,
                             float* __restrict__ Bv) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)N * C; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / C;
    const int c = (int)(e - i * C);
    float z = 0.0f;
    if (c < ncols) {
      const uint64_t v = splitmix64(mseed ^ ((uint64_t)(k0 + c) * 0xD1B54A32D192ED03ULL) ^ (uint64_t)(uint32_t)lin[i]);
      z = (v >> 63) ? -1.0f : 1.0f;
    }
    Bv[e] = z;
  }
}

// s += sum_c z_c xm_c (probe sums, FP64 per voxel)
template <int C>
__global__ void k_tri_hsum(int N, const float* __restrict__ Bv, const double* __restrict__ xm, double* __restrict__ acc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) s += (double)Bv[(size_t)i * C + c] * xm[(size_t)i * C + c];
    acc[i] += s;
  }
}

__global__ void k_tri_scale(int N, const double* __restrict__ acc, double scale, float* __restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) s[i] = (float)(acc[i] * scale);
}

__global__ void k_d2f(size_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

unsigned grid_n(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int C, class TI, class TO>
bf_status spmv27_launch(bf_ctx* ctx, const bf_band* b, const TI* X, TO* Y) {
  const size_t smem = (size_t)1000 * C * sizeof(TI);
  static bool attr = false;
  if (!attr) {
    BF_CK(cudaFuncSetAttribute(k_spmv27<C, TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const int grid = b->NB < 152 * 16 ? b->NB : 152 * 16;
  k_spmv27<C, TI, TO><<<grid, TB, smem, ctx->stream>>>(band_view(b), b->q27, X, Y);
  count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// Workspace of one solve over C columns (freed when the solve returns).
template <int C>
struct TriWork {
  float *Bv = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr;
  double *xm = nullptr, *qx = nullptr, *part = nullptr;
  TriState* st = nullptr;
  TriState* h_st = nullptr;
  cudaStream_t s = nullptr;
  ~TriWork() {
    void* ptrs[] = {Bv, r, z, p, q, x, xm, qx, part, st};
    for (void* v : ptrs)
      if (v) cudaFreeAsync(v, s);
    if (h_st) cudaFreeHost(h_st);
  }
};

template <int C>
bf_status tri_work_alloc(bf_ctx* ctx, const bf_band* b, TriWork<C>& w) {
  const size_t n = (size_t)b->N * C;
  w.s = ctx->stream;
  BF_TRY(dev_alloc_t(ctx, &w.Bv, n));
  BF_TRY(dev_alloc_t(ctx, &w.r, n));
  BF_TRY(dev_alloc_t(ctx, &w.z, n));
  BF_TRY(dev_alloc_t(ctx, &w.p, n));
  BF_TRY(dev_alloc_t(ctx, &w.q, n));
  BF_TRY(dev_alloc_t(ctx, &w.x, n));
  BF_TRY(dev_alloc_t(ctx, &w.xm, n));
  BF_TRY(dev_alloc_t(ctx, &w.qx, n));
  BF_TRY(dev_alloc_t(ctx, &w.part, (size_t)2 * C * NRED));
  BF_TRY(dev_alloc_t(ctx, &w.st, 1));
  BF_CK(cudaMallocHost(&w.h_st, sizeof(TriState)));
  return BF_OK;
}

// Solve Q X = Bv (in w.Bv) for ncols columns into the FP64 master iterate w.xm: FP32 PCG correction solves inside
// FP64 refinement until every column's true residual is <= tol |b|.  *iters: PCG iterations summed over columns.
template <int C>
bf_status tri_solve(bf_ctx* ctx, const bf_band* b, TriWork<C>& w, int ncols, double tol, int max_iter, int* iters,
                    double* relres) {
  cudaStream_t s = ctx->stream;
  const int N = (int)b->N;
  const unsigned g = NRED;  // every partial-sum kernel runs exactly NRED CTAs (the reduction sums NRED partials)
  auto red = [&](int mode) -> bf_status {
    k_tri_reduce<C><<<1, 256, 0, s>>>(w.st, w.part, mode, ncols, max_iter);
    count_launch();
    return BF_OK;
  };
  auto read = [&]() -> bf_status {
    BF_CK(cudaMemcpyAsync(w.h_st, w.st, sizeof(TriState), cudaMemcpyDeviceToHost, s));
    BF_CK(cudaStreamSynchronize(s));
    return BF_OK;
  };
  k_tri_state_init<<<1, 32, 0, s>>>(w.st, tol);
  count_launch();
  BF_CK(cudaMemsetAsync(w.xm, 0, (size_t)N * C * sizeof(double), s));
  bool conv = false;
  for (int outer = 0; outer < REFINE_MAX_PASSES; ++outer) {
    BF_TRY((spmv27_launch<C, double, double>(ctx, b, w.xm, w.qx)));
    k_tri_resid<C><<<g, 256, 0, s>>>(N, w.Bv, w.qx, w.r, w.part);
    count_launch();
    BF_TRY(red(RED_RES));
    BF_TRY(read());
    if (w.h_st->all_conv) {
      conv = true;
      break;
    }
    bool budget_left = false;
    for (int c = 0; c < ncols; ++c) budget_left |= w.h_st->iters[c] < max_iter;
    if (!budget_left || w.h_st->status == 2) break;
    k_tri_start<C><<<g, 256, 0, s>>>(N, b->qd, w.r, w.x, w.z, w.p, w.part);
    count_launch();
    BF_TRY(red(RED_START));
    for (int it = 0; it < max_iter; ++it) {
      BF_TRY((spmv27_launch<C, float, float>(ctx, b, w.p, w.q)));
      k_tri_pq<C><<<g, 256, 0, s>>>(N, w.p, w.q, w.part);
      count_launch();
      BF_TRY(red(RED_PQ));
      k_tri_upd<C><<<g, 256, 0, s>>>(N, w.st, b->qd, w.p, w.q, w.x, w.r, w.z, w.part);
      count_launch();
      BF_TRY(red(RED_UPD));
      k_tri_dir<C><<<g, 256, 0, s>>>(N, w.st, w.z, w.p);
      count_launch();
      BF_CK(cudaGetLastError());
      BF_TRY(read());
      if (!w.h_st->live) break;
    }
    k_tri_acc<C><<<grid_n((int64_t)N * C, 256, 152 * 16), 256, 0, s>>>(N, w.x, w.xm);
    count_launch();
  }
  BF_CK(cudaGetLastError());
  BF_TRY(read());
  int tot = 0;
  double worst = 0.0;
  for (int c = 0; c < ncols; ++c) {
    tot += w.h_st->iters[c];
    const double rel = w.h_st->bb[c] > 0 ? sqrt(w.h_st->rt2[c] / w.h_st->bb[c]) : 0.0;
    worst = rel > worst ? rel : worst;
  }
  if (iters) *iters = tot;
  if (relres) *relres = worst;
  if (w.h_st->status == 2) return bf_fail(ctx, BF_BREAKDOWN, "trilinear PCG breakdown");
  if (!conv) return bf_fail(ctx, BF_NOT_CONVERGED, "trilinear PCG iteration limit reached");
  return BF_OK;
}

}  // namespace

bf_status tri_integrate(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses, const Intr& K) {
  cudaStream_t s = ctx->stream;
  bf_status st;
  if (b->obs_mode != 0 && b->obs_mode != 3)
    return bf_fail(ctx, BF_ESTATE, "bf_integrate_depth: the band accumulates voxel-binned rows since its last "
                                   "bf_reset_observations");
  const size_t N = (size_t)(b->N ? b->N : 1);
  if (!b->d) {
    if ((st = dev_alloc_t(ctx, &b->d, N))) return st;
    if ((st = dev_alloc_t(ctx, &b->hd, N))) return st;
    if ((st = dev_alloc_t(ctx, &b->qd, N))) return st;
    if ((st = dev_alloc_t(ctx, &b->rhs, N))) return st;
    BF_CK(cudaMemsetAsync(b->d, 0, N * sizeof(float), s));
    BF_CK(cudaMemsetAsync(b->hd, 0, N * sizeof(float), s));
  }
  if (!b->c27) {
    if ((st = dev_alloc_t(ctx, &b->c27, 14 * N))) return st;
    if ((st = dev_alloc_t(ctx, &b->q27, 27 * N))) return st;
    BF_CK(cudaMemsetAsync(b->c27, 0, 14 * N * sizeof(float), s));
  }
  const bf_params& p = b->prm;
  if (b->N > 0 && T > 0) {
    const int nk = (int)floor(p.band_vox + 1e-9);
    const float s2x = (float)(p.sig_pose * p.sig_pose + p.sig_model * p.sig_model);
    const int64_t npix = (int64_t)T * K.H * K.W;
    k_tri_integrate<<<grid_n(npix, 256, 152 * 64), 256, 0, s>>>(band_view(b), depth, T, K, poses, nk, (float)p.sig_a,
                                                                (float)p.sig_b, s2x, b->d, b->hd, b->c27);
    count_launch();
    BF_CK(cudaGetLastError());
  }
  b->obs_mode = 3;
  if (b->N > 0) {
    k_tri_assemble<<<grid_n(b->N, 256, 152 * 16), 256, 0, s>>>(band_view(b), b->info, b->tsdf, b->hd, b->c27,
                                                               (float)p.lambda, (float)p.lambda_b,
                                                               1.0f / b->grid.voxel, b->q27, b->qd, b->rhs);
    count_launch();
    BF_CK(cudaGetLastError());
  }
  b->integrated = true;
  return BF_OK;
}

bf_status tri_rows(bf_ctx* ctx, const bf_band* b, const float* depth, int T, const float* poses, const Intr& K,
                   int32_t* idx, float* wts, uint8_t* used) {
  const int nk = (int)floor(b->prm.band_vox + 1e-9);
  const int64_t npix = (int64_t)T * K.H * K.W;
  if (npix > 0) {
    k_tri_rows<<<grid_n(npix, 256, 152 * 64), 256, 0, ctx->stream>>>(band_view(b), depth, T, K, poses, nk, idx, wts,
                                                                       used);
    count_launch();
    BF_CK(cudaGetLastError());
  }
  return BF_OK;
}

bf_status tri_spmv(bf_ctx* ctx, const bf_band* b, const float* x, float* y) {
  if (b->N == 0) return BF_OK;
  return spmv27_launch<1, float, float>(ctx, b, x, y);
}

bf_status tri_solve_mean(bf_ctx* ctx, bf_band* b, double tol, int max_iter, float* mu, int* iters, double* relres) {
  if (b->N == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return BF_OK;
  }
  TriWork<1> w;
  BF_TRY(tri_work_alloc<1>(ctx, b, w));
  BF_CK(cudaMemcpyAsync(w.Bv, b->rhs, (size_t)b->N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  const bf_status st = tri_solve<1>(ctx, b, w, 1, tol, max_iter, iters, relres);
  k_d2f<<<grid_n(b->N, 256, 152 * 16), 256, 0, ctx->stream>>>((size_t)b->N, w.xm, mu);
  count_launch();
  BF_CK(cudaGetLastError());
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return st;
}

bf_status tri_variance(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                       int max_iter, float* s_out, int* total_iters) {
  cudaStream_t s = ctx->stream;
  const int N = (int)b->N;
  if (N == 0) {
    if (total_iters) *total_iters = 0;
    return BF_OK;
  }
  TriWork<TRI_R> w;
  BF_TRY(tri_work_alloc<TRI_R>(ctx, b, w));
  double* acc = nullptr;
  BF_TRY(dev_alloc_t(ctx, &acc, (size_t)N));
  BF_CK(cudaMemsetAsync(acc, 0, (size_t)N * sizeof(double), s));
  const uint64_t mseed = splitmix64(seed);
  int tot = 0;
  bf_status result = BF_OK;
  for (int k0 = kb; k0 < ke; k0 += TRI_R) {
    const int ncols = ke - k0 < TRI_R ? ke - k0 : TRI_R;
    k_tri_probes<TRI_R><<<grid_n((int64_t)N * TRI_R, 256, 152 * 16), 256, 0, s>>>(N, b->lin, mseed, k0, ncols, w.Bv);
    count_launch();
    int it = 0;
    const bf_status st = tri_solve<TRI_R>(ctx, b, w, ncols, tol, max_iter, &it, nullptr);
    tot += it;
    k_tri_hsum<TRI_R><<<grid_n(N, 256, 152 * 16), 256, 0, s>>>(N, w.Bv, w.xm, acc);
    count_launch();
    if (st != BF_OK) {
      result = st;
      break;
    }
  }
  k_tri_scale<<<grid_n(N, 256, 152 * 16), 256, 0, s>>>(N, acc, scale, s_out);
  count_launch();
  BF_CK(cudaGetLastError());
  BF_CK(cudaStreamSynchronize(s));
  dev_free(s, acc);
  if (total_iters) *total_iters = tot;
  return result;
}
