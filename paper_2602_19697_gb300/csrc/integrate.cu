// Depth-to-SDF observations and posterior assembly (Sec. 3.5 back-projection,
// projective SDF, linear-row and noise equations; Sec. 3.6 Q0, precision and
// mean equations; Algorithm 1 steps 3-4).
//
// k_integrate: one thread per pixel (consecutive threads = consecutive pixels
// of a row, so depth loads coalesce).  The pixel ray's segment [s_p - tau,
// s_p + tau] is walked by the FP32-spec DDA; each band voxel entered gets
// d += w, hdata += w y through L2 atomics (fire-and-forget reductions).  The
// FP32 sums depend on the order the atomics land in; with FIX the FP32
// samples w and w y are added instead as int64 in units of 2^-32 (rounded to
// the nearest unit, exact from there on, so the sums do not depend on the
// order) and k_fix_out converts the totals to FP32.
// k_assemble: Q_jj = lambda deg + lambda_b [dB] + d, h = hdata + lambda_b
// [dB] tsdf / h.
#include "internal.cuh"

namespace {

template <bool FIX>
__global__ void __launch_bounds__(256) k_integrate(BandView B, const float* __restrict__ depth, int T, Intr K,
                                                   const float* __restrict__ poses, float tau, int max_steps,
                                                   float sa, float sb, float s2_extra, float* __restrict__ d,
                                                   float* __restrict__ hd, int64_t* __restrict__ dfx,
                                                   int64_t* __restrict__ hfx) {
  int64_t npix = (int64_t)T * K.H * K.W;
  const float org[3] = {B.o0, B.o1, B.o2};
  const float h = B.h, inv_h = 1.0f / B.h;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
    float D = __ldg(depth + q);
    if (!depth_ok(D)) continue;
    int t = (int)(q / ((int64_t)K.H * K.W));
    int rem = (int)(q - (int64_t)t * K.H * K.W);
    int py = rem / K.W, px = rem - py * K.W;
    Pose P = load_pose(poses + 12 * t);
    Ray ray = pixel_ray(P, px, py, K);
    float sp = f_mul(D, ray.nrm);
    // sample geometry (real-valued, ordinary FP32)
    float p0 = P.C[0] + D * ray.dw[0], p1 = P.C[1] + D * ray.dw[1], p2 = P.C[2] + D * ray.dw[2];
    float sd = sa + sb * D * D;
    float w = (h * h) / (sd * sd + s2_extra);
    dda_walk(P.C, ray.r, sp, tau, h, org, max_steps, [&](int i, int j, int k) {
      int v = band_lookup(B, i, j, k);
      if (v < 0) return;
      float x0 = B.o0 + ((float)i + 0.5f) * h, x1 = B.o1 + ((float)j + 0.5f) * h, x2 = B.o2 + ((float)k + 0.5f) * h;
      float y = ray.r[0] * (p0 - x0) + ray.r[1] * (p1 - x1) + ray.r[2] * (p2 - x2);
      y = fminf(fmaxf(y, -tau), tau) * inv_h;
      if (FIX) {
        const float scale = (float)(1ull << OBS_FIX_BITS);
        atomicAdd(reinterpret_cast<unsigned long long*>(dfx + v), (unsigned long long)__float2ll_rn(w * scale));
        atomicAdd(reinterpret_cast<unsigned long long*>(hfx + v), (unsigned long long)__float2ll_rn((w * y) * scale));
      } else {
        atomicAdd(d + v, w);
        atomicAdd(hd + v, w * y);
      }
    });
  }
}

// d, hd = the fixed-point totals in FP32
__global__ void k_fix_out(int N, const int64_t* __restrict__ dfx, const int64_t* __restrict__ hfx, float* __restrict__ d,
                          float* __restrict__ hd) {
  const double unit = 1.0 / (double)(1ull << OBS_FIX_BITS);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    d[v] = (float)((double)dfx[v] * unit);
    hd[v] = (float)((double)hfx[v] * unit);
  }
}

// FP64 copies of the observation sums: the fixed-point totals exactly (to 53 bits), else the FP32 sums
__global__ void k_obs_f64(int N, const int64_t* __restrict__ dfx, const int64_t* __restrict__ hfx,
                          const float* __restrict__ d, const float* __restrict__ hd, double* __restrict__ d64,
                          double* __restrict__ h64) {
  const double unit = 1.0 / (double)(1ull << OBS_FIX_BITS);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    if (d64) d64[v] = dfx ? (double)dfx[v] * unit : (double)d[v];
    if (h64) h64[v] = hfx ? (double)hfx[v] * unit : (double)hd[v];
  }
}

__global__ void k_assemble(int N, const uint8_t* __restrict__ info, const float* __restrict__ tsdf,
                           const float* __restrict__ d, const float* __restrict__ hd, float lam, float lamb,
                           float inv_h, float* __restrict__ qd, float* __restrict__ rhs) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
    int inf = info[v];
    float deg = (float)(inf & 7), bd = (float)(inf >> 3);
    qd[v] = lam * deg + lamb * bd + d[v];
    rhs[v] = hd[v] + lamb * bd * tsdf[v] * inv_h;
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

bf_status band_integrate(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses, const Intr& K,
                         bool fixed_point) {
  cudaStream_t s = ctx->stream;
  bf_status st;
  const int mode = fixed_point ? 2 : 1;
  if (b->obs_mode != 0 && b->obs_mode != mode)
    return bf_fail(ctx, BF_ESTATE, "bf_integrate_depth: the band accumulates in the other mode since its last "
                                   "bf_reset_observations");
  if (fixed_point && !b->dfx) {
    if ((st = dev_alloc_t(ctx, &b->dfx, b->N ? b->N : 1))) return st;
    if ((st = dev_alloc_t(ctx, &b->hfx, b->N ? b->N : 1))) return st;
    BF_CK(cudaMemsetAsync(b->dfx, 0, (b->N ? b->N : 1) * sizeof(int64_t), s));
    BF_CK(cudaMemsetAsync(b->hfx, 0, (b->N ? b->N : 1) * sizeof(int64_t), s));
  }
  if (!b->d) {
    if ((st = dev_alloc_t(ctx, &b->d, b->N ? b->N : 1))) return st;
    if ((st = dev_alloc_t(ctx, &b->hd, b->N ? b->N : 1))) return st;
    if ((st = dev_alloc_t(ctx, &b->qd, b->N ? b->N : 1))) return st;
    if ((st = dev_alloc_t(ctx, &b->rhs, b->N ? b->N : 1))) return st;
    BF_CK(cudaMemsetAsync(b->d, 0, b->N * sizeof(float), s));
    BF_CK(cudaMemsetAsync(b->hd, 0, b->N * sizeof(float), s));
  }
  if (b->N > 0 && T > 0) {
    const bf_params& p = b->prm;
    float tau = (float)p.band_vox * b->grid.voxel;
    float s2x = (float)(p.sig_pose * p.sig_pose + p.sig_model * p.sig_model);
    int64_t npix = (int64_t)T * K.H * K.W;
    if (fixed_point) {
      k_integrate<true><<<grid_for(npix, 256), 256, 0, s>>>(band_view(b), depth, T, K, poses, tau,
                                                            dda_max_steps(p.band_vox), (float)p.sig_a, (float)p.sig_b,
                                                            s2x, b->d, b->hd, b->dfx, b->hfx);
      count_launch();
      k_fix_out<<<grid_for(b->N, 256), 256, 0, s>>>((int)b->N, b->dfx, b->hfx, b->d, b->hd);
      count_launch();
    } else {
      k_integrate<false><<<grid_for(npix, 256), 256, 0, s>>>(band_view(b), depth, T, K, poses, tau,
                                                             dda_max_steps(p.band_vox), (float)p.sig_a,
                                                             (float)p.sig_b, s2x, b->d, b->hd, nullptr, nullptr);
      count_launch();
    }
    BF_CK(cudaGetLastError());
    b->obs_mode = mode;
  }
  return band_assemble(ctx, b);
}

bf_status band_observations_f64(bf_ctx* ctx, const bf_band* b, double* d64, double* h64) {
  if (b->N > 0) {
    const bool fix = b->obs_mode == 2;
    k_obs_f64<<<grid_for(b->N, 256), 256, 0, ctx->stream>>>((int)b->N, fix ? b->dfx : nullptr, fix ? b->hfx : nullptr,
                                                            b->d, b->hd, d64, h64);
    count_launch();
    BF_CK(cudaGetLastError());
  }
  return BF_OK;
}

bf_status band_assemble(bf_ctx* ctx, bf_band* b) {
  if (b->N > 0) {
    k_assemble<<<grid_for(b->N, 256), 256, 0, ctx->stream>>>((int)b->N, b->info, b->tsdf, b->d, b->hd,
                                                             (float)b->prm.lambda, (float)b->prm.lambda_b,
                                                             1.0f / b->grid.voxel, b->qd, b->rhs); count_launch();
    BF_CK(cudaGetLastError());
  }
  b->integrated = true;
  return BF_OK;
}
