// Next-best-view utilities (Sec. 3.8 NBV equation; Algorithm 1 step 8).
//
// k_nbv_obs: one thread per (candidate, pixel).  The pixel ray is cast
// through the trilinear interpolant of mu (defined where all 8 surrounding
// voxel centres are in the band): march at h/2 from the grid entry to the
// first outside -> inside crossing, then 10 bisection steps -- all in the
// FP32 specification arithmetic, so the predicted depth is reproducible bit
// for bit.  The predicted pixel then adds w(D) = h^2/sigma(D)^2 to dd[v][j]
// of every band voxel j its DDA segment enters (the integration model).
// k_nbv_util: U[v] = sum_{|mu_j| <= eps} s_j^2 dd_j / (1 + s_j dd_j), s_j
// floored at 1/Q_jj, per-CTA FP64 partials summed in a fixed order.
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

// trilinear interpolant of mu at grid coordinates g = (x - origin)/h - 1/2 (false where a corner is
// outside the band)
__device__ __forceinline__ bool interp_mu_g(const BandView& B, const float* __restrict__ mu, const float g[3],
                                            float* out) {
  int id[3];
  float fr[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!(fabsf(g[k]) < 1.0e6f)) return false;
    float fl = floorf(g[k]);
    id[k] = (int)fl;
    fr[k] = f_sub(g[k], fl);
  }
  float v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int q = band_lookup(B, id[0] + (c & 1), id[1] + ((c >> 1) & 1), id[2] + ((c >> 2) & 1));
    if (q < 0) return false;
    v[c] = __ldg(mu + q);
  }
  float c00 = f_add(v[0], f_mul(f_sub(v[1], v[0]), fr[0]));
  float c10 = f_add(v[2], f_mul(f_sub(v[3], v[2]), fr[0]));
  float c01 = f_add(v[4], f_mul(f_sub(v[5], v[4]), fr[0]));
  float c11 = f_add(v[6], f_mul(f_sub(v[7], v[6]), fr[0]));
  float c0 = f_add(c00, f_mul(f_sub(c10, c00), fr[1]));
  float c1 = f_add(c01, f_mul(f_sub(c11, c01), fr[1]));
  *out = f_add(c0, f_mul(f_sub(c1, c0), fr[2]));
  return true;
}

// the interpolant at a world point x
__device__ __forceinline__ bool interp_mu(const BandView& B, const float* __restrict__ mu, const float x[3],
                                          float* out) {
  const float org[3] = {B.o0, B.o1, B.o2};
  float g[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = f_sub(f_div(f_sub(x[k], org[k]), B.h), 0.5f);
  return interp_mu_g(B, mu, g, out);
}

__device__ __forceinline__ float raycast_depth(const BandView& B, const float* __restrict__ mu, const float C[3],
                                               const Ray& q) {
  const float org[3] = {B.o0, B.o1, B.o2};
  const float ext = f_mul((float)B.n, B.h);
  float sn = 0.0f, sx = __int_as_float(0x7f800000);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float lo = org[k], hi = f_add(org[k], ext);
    if (q.r[k] != 0.0f) {
      float t0 = f_div(f_sub(lo, C[k]), q.r[k]), t1 = f_div(f_sub(hi, C[k]), q.r[k]);
      if (t0 > t1) { float tt = t0; t0 = t1; t1 = tt; }
      if (t0 > sn) sn = t0;
      if (t1 < sx) sx = t1;
    } else if (C[k] < lo || C[k] > hi) {
      return 0.0f;
    }
  }
  if (!(sn < sx)) return 0.0f;
  const float hs = f_mul(0.5f, B.h);
  bool have_prev = false;
  float prev_v = 0.0f, prev_s = 0.0f;
  const int kmax = 4 * B.n + 8;  // the grid diagonal is < 3.47 n half-steps
  for (int k = 0; k < kmax; ++k) {
    float s = f_add(sn, f_mul((float)k, hs));
    if (s > sx) break;
    float x[3] = {f_add(C[0], f_mul(s, q.r[0])), f_add(C[1], f_mul(s, q.r[1])), f_add(C[2], f_mul(s, q.r[2]))};
    // empty-space skip: while the lowest of the 8 interpolation corners lies in a brick outside the band,
    // every step fails; jump to the last step that is surely still in that brick (steps are computed from
    // k, not accumulated, so the steps taken are the same as without the skip).  The exit bound is plain
    // FP32 with a margin of 0.02 h + 1e-6 s, far above its rounding error.
    float g[3];
    bool inside = true;
    int bc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      g[a] = f_sub(f_div(f_sub(x[a], org[a]), B.h), 0.5f);
      const int id = (int)floorf(g[a]);
      inside = inside && fabsf(g[a]) < 1.0e6f && id >= 0 && id < B.n;
      bc[a] = id >> 3;
    }
    if (inside && __ldg(B.dir + (bc[0] + B.nb * (bc[1] + B.nb * bc[2]))) < 0) {
      float se = 3.0e38f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float r = q.r[a];
        if (r > 0.0f) se = fminf(se, (org[a] + B.h * (8.0f * bc[a] + 8.5f) - C[a]) / r);
        else if (r < 0.0f) se = fminf(se, (org[a] + B.h * (8.0f * bc[a] + 0.5f) - C[a]) / r);
      }
      const float kl = floorf((se - 0.02f * B.h - 1e-6f * fabsf(se) - sn) / hs);
      if (kl > (float)k) k = kl < (float)kmax ? (int)kl : kmax;
      have_prev = false;
      continue;
    }
    float v;
    if (!interp_mu_g(B, mu, g, &v)) {
      have_prev = false;
      continue;
    }
    if (have_prev && prev_v > 0.0f && v <= 0.0f) {
      float lo = prev_s, hi = s;
      for (int it = 0; it < 10; ++it) {
        float mid = f_mul(0.5f, f_add(lo, hi));
        float xm[3] = {f_add(C[0], f_mul(mid, q.r[0])), f_add(C[1], f_mul(mid, q.r[1])),
                       f_add(C[2], f_mul(mid, q.r[2]))};
        float vm;
        if (interp_mu(B, mu, xm, &vm) && vm > 0.0f) lo = mid;
        else hi = mid;
      }
      return f_div(f_mul(0.5f, f_add(lo, hi)), q.nrm);
    }
    have_prev = true;
    prev_v = v;
    prev_s = s;
  }
  return 0.0f;
}

__global__ void __launch_bounds__(256) k_nbv_obs(BandView B, const float* __restrict__ mu,
                                                 const float* __restrict__ cand, int V, Intr K, float tau,
                                                 int max_steps, float sa, float sb, float s2x, float* __restrict__ dd,
                                                 float* __restrict__ pred) {
  const int64_t npix = (int64_t)K.W * K.H;
  const int64_t n = npix * V;
  const float org[3] = {B.o0, B.o1, B.o2};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    int v = (int)(q / npix);
    int rem = (int)(q - (int64_t)v * npix);
    int py = rem / K.W, px = rem - py * K.W;
    Pose P = load_pose(cand + 12 * v);
    Ray ray = pixel_ray(P, px, py, K);
    float D = raycast_depth(B, mu, P.C, ray);
    if (pred) pred[q] = D;
    if (!depth_ok(D)) continue;
    float sd = sa + sb * D * D;
    float w = (B.h * B.h) / (sd * sd + s2x);
    float* ddv = dd + (int64_t)v * B.N;
    dda_walk(P.C, ray.r, f_mul(D, ray.nrm), tau, B.h, org, max_steps, [&](int i, int j, int k) {
      int idx = band_lookup(B, i, j, k);
      if (idx >= 0) atomicAdd(ddv + idx, w);
    });
  }
}

constexpr int RT = 256;

__global__ void __launch_bounds__(RT) k_nbv_util(int N, const float* __restrict__ mu, const float* __restrict__ s,
                                                 const float* __restrict__ qd, const float* __restrict__ dd, float eps,
                                                 double* __restrict__ part) {
  const int v = blockIdx.y;
  const float* ddv = dd + (int64_t)v * N;
  double acc = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < N; i += gridDim.x * RT) {
    float m = __ldg(mu + i);
    if (!(fabsf(m) <= eps)) continue;
    double d = (double)ddv[i];
    if (d == 0.0) continue;
    double si = (double)__ldg(s + i), fl = 1.0 / (double)__ldg(qd + i);
    if (!(si >= fl)) si = fl;
    acc += si * si * d / (1.0 + si * d);
  }
  __shared__ double sh[RT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < RT / 32; ++w) t += sh[w];
    part[(int64_t)v * gridDim.x + blockIdx.x] = t;
  }
}

// Q_jj + dd_j: the diagonal after the candidate's predicted observations
__global__ void k_qd_plus(int N, const float* __restrict__ qd, const float* __restrict__ dd, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) out[i] = qd[i] + dd[i];
}

// per-CTA FP64 partials of sum_{|mu_j| <= eps} (s_j - s'_j) for candidate v -> part[v][CTA]
__global__ void __launch_bounds__(RT) k_nbv_exact(int N, const float* __restrict__ mu, const float* __restrict__ s,
                                                  const float* __restrict__ s2, float eps, int v,
                                                  double* __restrict__ part) {
  double acc = 0.0;
  for (int i = blockIdx.x * RT + threadIdx.x; i < N; i += gridDim.x * RT) {
    if (!(fabsf(__ldg(mu + i)) <= eps)) continue;
    acc += (double)__ldg(s + i) - (double)__ldg(s2 + i);
  }
  __shared__ double sh[RT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < RT / 32; ++w) t += sh[w];
    part[(int64_t)v * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void k_nbv_sum(const double* __restrict__ part, int nblk, int V, double* __restrict__ U) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  double t = 0;
  for (int b = 0; b < nblk; ++b) t += part[(int64_t)v * nblk + b];
  U[v] = t;
}

}  // namespace

// the candidates' predicted observations dd [V][N] (zeroed first)
static bf_status nbv_observations(bf_ctx* ctx, const bf_band* b, const float* mu, const float* cand, int V,
                                  const Intr& K, float* dd) {
  cudaStream_t st_ = ctx->stream;
  const int64_t N = b->N;
  BF_CK(cudaMemsetAsync(dd, 0, (size_t)V * N * 4, st_));
  const bf_params& p = b->prm;
  float tau = (float)p.band_vox * b->grid.voxel;
  float s2x = (float)(p.sig_pose * p.sig_pose + p.sig_model * p.sig_model);
  int64_t n = (int64_t)V * K.W * K.H;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  k_nbv_obs<<<(unsigned)g, 256, 0, st_>>>(band_view(b), mu, cand, V, K, tau, dda_max_steps(p.band_vox),
                                         (float)p.sig_a, (float)p.sig_b, s2x, dd, nullptr);
  count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// U [V] from the device copy dU: argmax and the copy to the caller's buffer
static bf_status nbv_finish(bf_ctx* ctx, const double* dU, int V, double* U, int* best) {
  cudaStream_t st_ = ctx->stream;
  std::vector<double> hU(V);
  BF_CK(cudaMemcpyAsync(hU.data(), dU, (size_t)V * 8, cudaMemcpyDeviceToHost, st_));
  BF_CK(cudaStreamSynchronize(st_));
  int bi = 0;
  for (int v = 1; v < V; ++v)
    if (hU[v] > hU[bi]) bi = v;
  if (best) *best = bi;
  if (is_device_ptr(U)) BF_CK(cudaMemcpyAsync(U, dU, (size_t)V * 8, cudaMemcpyDeviceToDevice, st_));
  else memcpy(U, hU.data(), (size_t)V * 8);
  return BF_OK;
}

bf_status nbv_exact_impl(bf_ctx* ctx, bf_band* b, const float* mu, const float* cand, int V, const Intr& K,
                         double eps, int Kp, uint64_t seed, double tol, int max_iter, int R, double* U, int* best,
                         int* total_iters) {
  cudaStream_t st_ = ctx->stream;
  const int64_t N = b->N;
  bf_status st;
  const int nblk = 152 * 2;
  float* dd = (float*)ws_get(ctx, WS_TMP0, (size_t)V * (N ? N : 1) * 4, &st);
  if (st) return st;
  double* part = (double*)ws_get(ctx, WS_TMP1, (size_t)V * nblk * 8 + (size_t)V * 8, &st);
  if (st) return st;
  float* qd2 = (float*)ws_get(ctx, WS_TMP2, (size_t)(N ? N : 1) * 4, &st);
  if (st) return st;
  float* s0 = (float*)ws_get(ctx, WS_TMP3, (size_t)(N ? N : 1) * 4, &st);
  if (st) return st;
  float* s2 = (float*)ws_get(ctx, WS_TMP4, (size_t)(N ? N : 1) * 4, &st);
  if (st) return st;
  double* dU = part + (size_t)V * nblk;
  int tot = 0;
  if (N > 0) {
    BF_TRY(nbv_observations(ctx, b, mu, cand, V, K, dd));
    int it = 0;
    BF_TRY(variance_impl(ctx, b, 0, Kp, 1.0 / Kp, seed, tol, max_iter, R, 0u, s0, &it));
    tot += it;
    float* const qd0 = b->qd;
    for (int v = 0; v < V; ++v) {
      k_qd_plus<<<(unsigned)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16), 256, 0, st_>>>(
          (int)N, qd0, dd + (size_t)v * N, qd2);
      count_launch();
      b->qd = qd2;  // the band's diagonal with the candidate's precision, for this estimate only
      st = variance_impl(ctx, b, 0, Kp, 1.0 / Kp, seed, tol, max_iter, R, 0u, s2, &it);
      b->qd = qd0;
      if (st) return st;
      tot += it;
      k_nbv_exact<<<nblk, RT, 0, st_>>>((int)N, mu, s0, s2, (float)eps, v, part);
      count_launch();
    }
    k_nbv_sum<<<(V + 127) / 128, 128, 0, st_>>>(part, nblk, V, dU);
    count_launch();
    BF_CK(cudaGetLastError());
  } else {
    BF_CK(cudaMemsetAsync(dU, 0, (size_t)V * 8, st_));
  }
  if (total_iters) *total_iters = tot;
  return nbv_finish(ctx, dU, V, U, best);
}

bf_status nbv_impl(bf_ctx* ctx, const bf_band* b, const float* mu, const float* s, const float* cand, int V,
                   const Intr& K, double eps, double* U, int* best) {
  cudaStream_t st_ = ctx->stream;
  const int64_t N = b->N;
  bf_status st;
  float* dd = (float*)ws_get(ctx, WS_TMP0, (size_t)V * (N ? N : 1) * 4, &st);
  if (st) return st;
  const int nblk = 152 * 2;
  double* part = (double*)ws_get(ctx, WS_TMP1, (size_t)V * nblk * 8 + (size_t)V * 8, &st);
  if (st) return st;
  double* dU = part + (size_t)V * nblk;
  if (N > 0) {
    BF_CK(cudaMemsetAsync(dd, 0, (size_t)V * N * 4, st_));
    const bf_params& p = b->prm;
    float tau = (float)p.band_vox * b->grid.voxel;
    float s2x = (float)(p.sig_pose * p.sig_pose + p.sig_model * p.sig_model);
    int64_t n = (int64_t)V * K.W * K.H;
    int64_t g = (n + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    k_nbv_obs<<<(unsigned)g, 256, 0, st_>>>(band_view(b), mu, cand, V, K, tau, dda_max_steps(p.band_vox),
                                           (float)p.sig_a, (float)p.sig_b, s2x, dd, nullptr); count_launch();
    dim3 gr(nblk, V);
    k_nbv_util<<<gr, RT, 0, st_>>>((int)N, mu, s, b->qd, dd, (float)eps, part); count_launch();
    k_nbv_sum<<<(V + 127) / 128, 128, 0, st_>>>(part, nblk, V, dU); count_launch();
    BF_CK(cudaGetLastError());
  } else {
    BF_CK(cudaMemsetAsync(dU, 0, (size_t)V * 8, st_));
  }
  std::vector<double> hU(V);
  BF_CK(cudaMemcpyAsync(hU.data(), dU, (size_t)V * 8, cudaMemcpyDeviceToHost, st_));
  BF_CK(cudaStreamSynchronize(st_));
  int bi = 0;
  for (int v = 1; v < V; ++v)
    if (hU[v] > hU[bi]) bi = v;
  if (best) *best = bi;
  if (is_device_ptr(U)) BF_CK(cudaMemcpyAsync(U, dU, (size_t)V * 8, cudaMemcpyDeviceToDevice, st_));
  else memcpy(U, hU.data(), (size_t)V * 8);
  return BF_OK;
}
