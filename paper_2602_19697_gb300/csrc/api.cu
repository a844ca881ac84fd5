// C ABI of the posterior-solver library: argument checks, host/device
// staging, context and workspace management.  The computation lives in the
// other translation units.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.cuh"

static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

bf_status bf_fail(bf_ctx* ctx, bf_status st, const char* what, const char* detail) {
  if (ctx) {
    ctx->err = what ? what : "";
    if (detail) {
      ctx->err += ": ";
      ctx->err += detail;
    }
  }
  return st;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bf_status dev_alloc(bf_ctx* ctx, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return bf_fail(ctx, BF_ENOMEM, "device allocation failed", cudaGetErrorString(e));
  }
  return BF_OK;
}

void dev_free(cudaStream_t s, void* p) {
  if (p) cudaFreeAsync(p, s);
}

void* ws_get(bf_ctx* ctx, int slot, size_t bytes, bf_status* st) {
  Workspace& w = ctx->ws[slot];
  if (bytes == 0) bytes = 16;
  if (w.cap < bytes) {
    if (w.p) cudaFreeAsync(w.p, ctx->stream);
    w.p = nullptr;
    w.cap = 0;
    size_t cap = bytes + bytes / 8;
    if (cudaMallocAsync(&w.p, cap, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      *st = bf_fail(ctx, BF_ENOMEM, "workspace allocation failed");
      return nullptr;
    }
    w.cap = cap;
  }
  *st = BF_OK;
  return w.p;
}

namespace {

__global__ void k_i32_to_i64(const int32_t* in, int64_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

__global__ void k_bdry(const uint8_t* info, uint8_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = info[i] >> 3;
}

__global__ void k_mask64(const MetaWord* meta, uint64_t* out, int64_t nwords64) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords64; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint64_t)meta[2 * i].bits | ((uint64_t)meta[2 * i + 1].bits << 32);
}

unsigned gsize(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

bool valid_intr(const bf_intrinsics* K) {
  return K && K->W > 0 && K->H > 0 && K->W <= 16384 && K->H <= 16384 && K->fx > 0 && K->fy > 0 &&
         std::isfinite(K->cx) && std::isfinite(K->cy);
}

Intr to_intr(const bf_intrinsics* K) {
  Intr k;
  k.fx = K->fx;
  k.fy = K->fy;
  k.cx = K->cx;
  k.cy = K->cy;
  k.W = K->W;
  k.H = K->H;
  return k;
}

}  // namespace

extern "C" {

bf_status bf_create(int device, void* stream, bf_ctx** out) {
  if (!out) return BF_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return BF_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return BF_ECUDA;
  bf_ctx* ctx = new (std::nothrow) bf_ctx();
  if (!ctx) return BF_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaMallocHost(&ctx->h_pinned, 64) != cudaSuccess) {
    delete ctx;
    return BF_ENOMEM;
  }
  // the device error word of the kernels with bounded waits (allocated here, so that no later call allocates it)
  if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaFreeHost(ctx->h_pinned);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return BF_ENOMEM;
  }
  *out = ctx;
  return BF_OK;
}

void bf_destroy(bf_ctx* ctx) {
  if (!ctx) return;
  enter_device(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& w : ctx->ws)
    if (w.p) cudaFree(w.p);
  if (ctx->mesh_v) cudaFree(ctx->mesh_v);
  if (ctx->mesh_t) cudaFree(ctx->mesh_t);
  if (ctx->mc_table) cudaFree(ctx->mc_table);
  if (ctx->mc_ntri) cudaFree(ctx->mc_ntri);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (BlockGraph* g : ctx->blk) block_graph_free(g);
  for (SolveGraph* g : ctx->sgl) solve_graph_free(g);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  delete ctx;
}

const char* bf_last_error(const bf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

bf_status bf_set_stream(bf_ctx* ctx, void* stream) {
  if (!ctx) return BF_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return BF_OK;
}

bf_status bf_build_band(bf_ctx* ctx, const float* depth, int T, const float* poses, const bf_intrinsics* K,
                        const bf_grid* grid, const bf_params* prm, bf_band** out) {
  BF_ENTER(ctx);
  if (!ctx || !out) return BF_EINVAL;
  *out = nullptr;
  if (!depth || !poses || !grid || !prm || T < 1 || !valid_intr(K))
    return bf_fail(ctx, BF_EINVAL, "bf_build_band: null pointer, T < 1 or bad intrinsics");
  if (grid->n < 8 || grid->n > 2048 || grid->n % 8 != 0 || !(grid->voxel > 0.0f))
    return bf_fail(ctx, BF_EINVAL, "bf_build_band: n must be a multiple of 8 in [8, 2048], voxel > 0");
  if (!(prm->band_vox > 0.0) || !(prm->trunc_vox > prm->band_vox) || prm->trunc_vox > 256.0 ||
      !(prm->lambda >= 0.0) || !(prm->lambda_b >= 0.0))
    return bf_fail(ctx, BF_EINVAL, "bf_build_band: need 0 < band_vox < trunc_vox <= 256, lambda, lambda_b >= 0");
  const float *d_depth, *d_poses;
  size_t npix = (size_t)T * K->H * K->W;
  BF_TRY(stage_in(ctx, depth, npix, WS_STAGE0, &d_depth));
  BF_TRY(stage_in(ctx, poses, (size_t)T * 12, WS_STAGE1, &d_poses));
  return band_build(ctx, d_depth, T, d_poses, to_intr(K), *grid, *prm, out);
}

void bf_band_free(bf_band* b) {
  if (!b) return;
  enter_device(b->device);
  cudaStreamSynchronize(b->stream);
  void* ptrs[] = {b->dir, b->bcoord, b->meta, b->off, b->nbr, b->lin, b->tsdf, b->wcount, b->info,
                  b->d, b->hd, b->qd, b->rhs, b->nb6, b->sp_ext, b->sp_ne, b->sp_slot, b->dfx, b->hfx,
                  b->c27, b->q27};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

bf_status bf_band_info(const bf_band* b, int64_t* n_vox, int32_t* n_bricks, int64_t* n_cand) {
  if (!b) return BF_EINVAL;
  if (n_vox) *n_vox = b->N;
  if (n_bricks) *n_bricks = b->NB;
  if (n_cand) *n_cand = b->ncand;
  return BF_OK;
}

bf_status bf_export_band(bf_ctx* ctx, const bf_band* b, int64_t* lin, float* tsdf, int32_t* wcount, uint8_t* bdry,
                         int32_t* brick_dir, uint64_t* mask) {
  BF_ENTER(ctx);
  if (!ctx || !b) return BF_EINVAL;
  cudaStream_t s = ctx->stream;
  const int64_t N = b->N;
  bool host;
  if (lin && N) {
    int64_t* d;
    BF_TRY(stage_out(ctx, lin, N, WS_OUT0, &d, &host));
    k_i32_to_i64<<<gsize(N), 256, 0, s>>>(b->lin, d, N); count_launch();
    BF_TRY(copy_out(ctx, lin, d, N, host));
  }
  if (tsdf && N) {
    if (is_device_ptr(tsdf)) BF_CK(cudaMemcpyAsync(tsdf, b->tsdf, N * 4, cudaMemcpyDeviceToDevice, s));
    else BF_CK(cudaMemcpy(tsdf, b->tsdf, N * 4, cudaMemcpyDeviceToHost));
  }
  if (wcount && N) {
    if (is_device_ptr(wcount)) BF_CK(cudaMemcpyAsync(wcount, b->wcount, N * 4, cudaMemcpyDeviceToDevice, s));
    else BF_CK(cudaMemcpy(wcount, b->wcount, N * 4, cudaMemcpyDeviceToHost));
  }
  if (bdry && N) {
    uint8_t* d;
    BF_TRY(stage_out(ctx, bdry, N, WS_OUT0, &d, &host));
    k_bdry<<<gsize(N), 256, 0, s>>>(b->info, d, N); count_launch();
    BF_TRY(copy_out(ctx, bdry, d, N, host));
  }
  if (brick_dir) {
    size_t nb3 = (size_t)b->nb * b->nb * b->nb;
    if (is_device_ptr(brick_dir)) BF_CK(cudaMemcpyAsync(brick_dir, b->dir, nb3 * 4, cudaMemcpyDeviceToDevice, s));
    else BF_CK(cudaMemcpy(brick_dir, b->dir, nb3 * 4, cudaMemcpyDeviceToHost));
  }
  if (mask && b->NB) {
    uint64_t* d;
    int64_t nw = (int64_t)b->NB * 8;
    BF_TRY(stage_out(ctx, mask, nw, WS_OUT1, &d, &host));
    k_mask64<<<gsize(nw), 256, 0, s>>>(b->meta, d, nw); count_launch();
    BF_TRY(copy_out(ctx, mask, d, nw, host));
  }
  BF_CK(cudaGetLastError());
  return BF_OK;
}

bf_status bf_integrate_depth_ex(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses,
                                const bf_intrinsics* K, unsigned flags) {
  BF_ENTER(ctx);
  if (!ctx || !b) return BF_EINVAL;
  if (!depth || !poses || T < 1 || !valid_intr(K))
    return bf_fail(ctx, BF_EINVAL, "bf_integrate_depth: null pointer, T < 1 or bad intrinsics");
  if (flags & ~(BF_INTEGRATE_DETERMINISTIC | BF_INTEGRATE_TRILINEAR))
    return bf_fail(ctx, BF_EINVAL, "bf_integrate_depth_ex: unknown flags");
  if ((flags & BF_INTEGRATE_DETERMINISTIC) && (flags & BF_INTEGRATE_TRILINEAR))
    return bf_fail(ctx, BF_EINVAL, "bf_integrate_depth_ex: trilinear rows have no deterministic mode");
  const float *d_depth, *d_poses;
  BF_TRY(stage_in(ctx, depth, (size_t)T * K->H * K->W, WS_STAGE0, &d_depth));
  BF_TRY(stage_in(ctx, poses, (size_t)T * 12, WS_STAGE1, &d_poses));
  if (flags & BF_INTEGRATE_TRILINEAR) return tri_integrate(ctx, b, d_depth, T, d_poses, to_intr(K));
  if (b->obs_mode == 3)
    return bf_fail(ctx, BF_ESTATE, "bf_integrate_depth: the band accumulates trilinear rows since its last "
                                   "bf_reset_observations");
  return band_integrate(ctx, b, d_depth, T, d_poses, to_intr(K), (flags & BF_INTEGRATE_DETERMINISTIC) != 0);
}

bf_status bf_integrate_depth(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses,
                             const bf_intrinsics* K) {
  return bf_integrate_depth_ex(ctx, b, depth, T, poses, K, 0u);
}

bf_status bf_reset_observations(bf_ctx* ctx, bf_band* b) {
  BF_ENTER(ctx);
  if (!ctx || !b) return BF_EINVAL;
  b->obs_mode = 0;
  if (b->dfx) {
    BF_CK(cudaMemsetAsync(b->dfx, 0, (b->N ? b->N : 1) * sizeof(int64_t), ctx->stream));
    BF_CK(cudaMemsetAsync(b->hfx, 0, (b->N ? b->N : 1) * sizeof(int64_t), ctx->stream));
  }
  if (b->c27) BF_CK(cudaMemsetAsync(b->c27, 0, (size_t)14 * (b->N ? b->N : 1) * sizeof(float), ctx->stream));
  if (b->d) {
    BF_CK(cudaMemsetAsync(b->d, 0, b->N * 4, ctx->stream));
    BF_CK(cudaMemsetAsync(b->hd, 0, b->N * 4, ctx->stream));
    return band_assemble(ctx, b);
  }
  return BF_OK;
}

bf_status bf_export_system(bf_ctx* ctx, const bf_band* b, float* d, float* hdata, float* qdiag, float* rhs) {
  BF_ENTER(ctx);
  if (!ctx || !b) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_export_system: call bf_integrate_depth first");
  const float* src[4] = {b->d, b->hd, b->qd, b->rhs};
  float* dst[4] = {d, hdata, qdiag, rhs};
  for (int k = 0; k < 4; ++k) {
    if (!dst[k] || !b->N) continue;
    if (is_device_ptr(dst[k])) BF_CK(cudaMemcpyAsync(dst[k], src[k], b->N * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    else {
      BF_CK(cudaStreamSynchronize(ctx->stream));
      BF_CK(cudaMemcpy(dst[k], src[k], b->N * 4, cudaMemcpyDeviceToHost));
    }
  }
  return BF_OK;
}

bf_status bf_export_observations_f64(bf_ctx* ctx, const bf_band* b, double* d, double* hdata) {
  BF_ENTER(ctx);
  if (!ctx || !b) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_export_observations_f64: call bf_integrate_depth first");
  if (!b->N || (!d && !hdata)) return BF_OK;
  double *dd = nullptr, *dh = nullptr;
  bool host_d = false, host_h = false;
  if (d) BF_TRY(stage_out(ctx, d, b->N, WS_OUT0, &dd, &host_d));
  if (hdata) BF_TRY(stage_out(ctx, hdata, b->N, WS_OUT1, &dh, &host_h));
  BF_TRY(band_observations_f64(ctx, b, dd, dh));
  if (d) BF_TRY(copy_out(ctx, d, (const double*)dd, b->N, host_d));
  if (hdata) BF_TRY(copy_out(ctx, hdata, (const double*)dh, b->N, host_h));
  return BF_OK;
}

bf_status bf_spmv(bf_ctx* ctx, const bf_band* b, const float* x, float* y) {
  BF_ENTER(ctx);
  if (!ctx || !b || !x || !y) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_spmv: call bf_integrate_depth first");
  const float* dx;
  float* dy;
  bool host;
  BF_TRY(stage_in(ctx, x, b->N, WS_STAGE2, &dx));
  BF_TRY(stage_out(ctx, y, b->N, WS_OUT0, &dy, &host));
  BF_TRY(spmv_launch(ctx, b, dx, dy));
  BF_TRY(copy_out(ctx, y, (const float*)dy, b->N, host));
  return host ? device_wait_status(ctx, "bf_spmv") : BF_OK;  // host output: the call is synchronous anyway
}

bf_status bf_spmm(bf_ctx* ctx, bf_band* b, const float* X, int R, float* Y) {
  BF_ENTER(ctx);
  if (!ctx || !b || !X || !Y) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_spmm: call bf_integrate_depth first");
  if (R != 8 && R != 16 && R != 32) return bf_fail(ctx, BF_EINVAL, "bf_spmm: R must be 8, 16 or 32");
  if (b->obs_mode == 3) return bf_fail(ctx, BF_ESTATE, "bf_spmm: the band holds trilinear rows (27-point Q)");
  const float* dX;
  float* dY;
  bool host;
  const size_t n = (size_t)b->N * R;
  BF_TRY(stage_in(ctx, X, n, WS_STAGE2, &dX));
  BF_TRY(stage_out(ctx, Y, n, WS_OUT0, &dY, &host));
  BF_TRY(spmm_launch(ctx, b, dX, R, dY));
  return copy_out(ctx, Y, (const float*)dY, n, host);
}

bf_status bf_solve_mean(bf_ctx* ctx, bf_band* b, double rel_tol, int max_iter, unsigned flags, float* mu,
                        int* iters, double* rel_res) {
  BF_ENTER(ctx);
  if (!ctx || !b || !mu) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_solve_mean: call bf_integrate_depth first");
  if (!(rel_tol > 0.0) || !(rel_tol < 1.0) || max_iter < 1 || max_iter > 10000000)
    return bf_fail(ctx, BF_EINVAL, "bf_solve_mean: need 0 < rel_tol < 1 and 1 <= max_iter <= 1e7");
  if (b->obs_mode == 3 && (flags & BF_SOLVE_WARM))
    return bf_fail(ctx, BF_EINVAL, "bf_solve_mean: no warm start with trilinear rows");
  float* dmu;
  bool host;
  BF_TRY(stage_out(ctx, mu, b->N, WS_OUT0, &dmu, &host));
  if ((flags & BF_SOLVE_WARM) && host && b->N)
    BF_CK(cudaMemcpyAsync(dmu, mu, b->N * 4, cudaMemcpyHostToDevice, ctx->stream));
  bf_status st = b->obs_mode == 3 ? tri_solve_mean(ctx, b, rel_tol, max_iter, dmu, iters, rel_res)
                                  : solve_mean_impl(ctx, b, rel_tol, max_iter, flags, dmu, iters, rel_res);
  if (st == BF_OK || st == BF_NOT_CONVERGED || st == BF_BREAKDOWN) {
    bf_status c = copy_out(ctx, mu, (const float*)dmu, b->N, host);
    if (c != BF_OK) return c;
  }
  return st;
}

bf_status bf_estimate_variance(bf_ctx* ctx, bf_band* b, int K, uint64_t seed, double rel_tol, int max_iter,
                               int rhs_block, unsigned flags, float* s, int* total_iters) {
  BF_ENTER(ctx);
  if (!ctx || !b || !s) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_estimate_variance: call bf_integrate_depth first");
  if (K < 1 || !(rel_tol > 0.0) || !(rel_tol < 1.0) || max_iter < 1 || max_iter > 10000000)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance: need K >= 1, 0 < rel_tol < 1, 1 <= max_iter <= 1e7");
  if (rhs_block != 0 && rhs_block != 1 && rhs_block != 8 && rhs_block != 16 && rhs_block != 32)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance: rhs_block must be 0, 1, 8, 16 or 32");
  if (b->obs_mode == 3 && rhs_block != 0 && rhs_block != TRI_R)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance: trilinear rows take rhs_block 0 or 8");
  float* ds;
  bool host;
  BF_TRY(stage_out(ctx, s, b->N, WS_OUT1, &ds, &host));
  bf_status st = b->obs_mode == 3
                     ? tri_variance(ctx, b, 0, K, 1.0 / K, seed, rel_tol, max_iter, ds, total_iters)
                     : variance_impl(ctx, b, 0, K, 1.0 / K, seed, rel_tol, max_iter, rhs_block, flags, ds, total_iters);
  if (st == BF_OK || st == BF_NOT_CONVERGED || st == BF_BREAKDOWN) {
    bf_status c = copy_out(ctx, s, (const float*)ds, b->N, host);
    if (c != BF_OK) return c;
  }
  return st;
}

bf_status bf_estimate_variance_range(bf_ctx* ctx, bf_band* b, int k_begin, int k_end, double scale, uint64_t seed,
                                     double rel_tol, int max_iter, int rhs_block, unsigned flags, float* s_sum,
                                     int* total_iters) {
  BF_ENTER(ctx);
  if (!ctx || !b || !s_sum) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_estimate_variance_range: call bf_integrate_depth first");
  if (k_begin < 0 || k_end <= k_begin || !(rel_tol > 0.0) || !(rel_tol < 1.0) || max_iter < 1 || max_iter > 10000000)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance_range: need 0 <= k_begin < k_end, 0 < rel_tol < 1");
  if (!(scale > 0.0) || !std::isfinite(scale))
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance_range: scale must be finite and > 0");
  if (rhs_block != 0 && rhs_block != 1 && rhs_block != 8 && rhs_block != 16 && rhs_block != 32)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance_range: rhs_block must be 0, 1, 8, 16 or 32");
  if (b->obs_mode == 3 && rhs_block != 0 && rhs_block != TRI_R)
    return bf_fail(ctx, BF_EINVAL, "bf_estimate_variance_range: trilinear rows take rhs_block 0 or 8");
  float* ds;
  bool host;
  BF_TRY(stage_out(ctx, s_sum, b->N, WS_OUT1, &ds, &host));
  bf_status st = b->obs_mode == 3
                     ? tri_variance(ctx, b, k_begin, k_end, scale, seed, rel_tol, max_iter, ds, total_iters)
                     : variance_impl(ctx, b, k_begin, k_end, scale, seed, rel_tol, max_iter, rhs_block, flags, ds,
                                     total_iters);
  if (st == BF_OK || st == BF_NOT_CONVERGED || st == BF_BREAKDOWN) {
    bf_status c = copy_out(ctx, s_sum, (const float*)ds, b->N, host);
    if (c != BF_OK) return c;
  }
  return st;
}

bf_status bf_extract_surface(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt) {
  BF_ENTER(ctx);
  if (!ctx || !b || !mu || !nv || !nt) return BF_EINVAL;
  const float* dmu;
  BF_TRY(stage_in(ctx, mu, b->N, WS_STAGE2, &dmu));
  return mc_impl(ctx, b, dmu, nv, nt);
}

bf_status bf_extract_surface_dc(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt) {
  BF_ENTER(ctx);
  if (!b || !mu || !nv || !nt) return BF_EINVAL;
  const float* dmu;
  BF_TRY(stage_in(ctx, mu, b->N, WS_STAGE2, &dmu));
  return dc_impl(ctx, b, dmu, nv, nt);
}

bf_status bf_get_surface(bf_ctx* ctx, float* verts, int32_t* tris) {
  BF_ENTER(ctx);
  if (!ctx) return BF_EINVAL;
  if (verts && ctx->mesh_nv) {
    cudaMemcpyKind k = is_device_ptr(verts) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    BF_CK(cudaMemcpyAsync(verts, ctx->mesh_v, ctx->mesh_nv * 12, k, ctx->stream));
  }
  if (tris && ctx->mesh_nt) {
    cudaMemcpyKind k = is_device_ptr(tris) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    BF_CK(cudaMemcpyAsync(tris, ctx->mesh_t, ctx->mesh_nt * 12, k, ctx->stream));
  }
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return BF_OK;
}

bf_status bf_score_views(bf_ctx* ctx, const bf_band* b, const float* mu, const float* s, const float* cand, int V,
                         const bf_intrinsics* K, double eps, double* U, int* best) {
  BF_ENTER(ctx);
  if (!ctx || !b || !mu || !s || !cand || !U || V < 1 || !valid_intr(K) || !(eps >= 0.0))
    return bf_fail(ctx, BF_EINVAL, "bf_score_views: null pointer, V < 1, eps < 0 or bad intrinsics");
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_score_views: call bf_integrate_depth first");
  const float *dmu, *ds, *dc;
  BF_TRY(stage_in(ctx, mu, b->N, WS_STAGE2, &dmu));
  BF_TRY(stage_in(ctx, s, b->N, WS_STAGE3, &ds));
  BF_TRY(stage_in(ctx, cand, (size_t)V * 12, WS_STAGE1, &dc));
  return nbv_impl(ctx, b, dmu, ds, dc, V, to_intr(K), eps, U, best);
}

bf_status bf_score_views_exact(bf_ctx* ctx, bf_band* b, const float* mu, const float* cand, int V,
                               const bf_intrinsics* K, double eps, int K_probes, uint64_t seed, double rel_tol,
                               int max_iter, int rhs_block, double* U, int* best, int* total_iters) {
  BF_ENTER(ctx);
  if (!ctx || !b || !mu || !cand || !U || V < 1 || !valid_intr(K) || !(eps >= 0.0) || K_probes < 1 ||
      !(rel_tol > 0.0) || max_iter < 1)
    return bf_fail(ctx, BF_EINVAL, "bf_score_views_exact: null pointer, V < 1, K < 1, eps < 0, rel_tol <= 0, "
                                   "max_iter < 1 or bad intrinsics");
  if (rhs_block != 0 && rhs_block != 1 && rhs_block != 8 && rhs_block != 16 && rhs_block != 32)
    return bf_fail(ctx, BF_EINVAL, "bf_score_views_exact: rhs_block must be 0, 1, 8, 16 or 32");
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_score_views_exact: call bf_integrate_depth first");
  if (b->obs_mode == 3) return bf_fail(ctx, BF_ESTATE, "bf_score_views_exact: the band holds trilinear rows");
  const float *dmu, *dc;
  BF_TRY(stage_in(ctx, mu, b->N, WS_STAGE2, &dmu));
  BF_TRY(stage_in(ctx, cand, (size_t)V * 12, WS_STAGE1, &dc));
  return nbv_exact_impl(ctx, b, dmu, dc, V, to_intr(K), eps, K_probes, seed, rel_tol, max_iter, rhs_block, U, best,
                        total_iters);
}

bf_status bf_export_trilinear_rows(bf_ctx* ctx, const bf_band* b, const float* depth, int T, const float* poses,
                                   const bf_intrinsics* K, int32_t* idx, float* wts, uint8_t* used, int64_t* M) {
  BF_ENTER(ctx);
  if (!b || !M || !depth || !poses || T < 1 || !valid_intr(K))
    return bf_fail(ctx, BF_EINVAL, "bf_export_trilinear_rows: null pointer, T < 1 or bad intrinsics");
  const int64_t ns = 2 * (int64_t)floor(b->prm.band_vox + 1e-9) + 1;
  const int64_t m = (int64_t)T * K->H * K->W * ns;
  *M = m;
  if (!idx && !wts && !used) return BF_OK;
  if (!idx || !wts || !used) return bf_fail(ctx, BF_EINVAL, "bf_export_trilinear_rows: give all three arrays or none");
  const float *d_depth, *d_poses;
  BF_TRY(stage_in(ctx, depth, (size_t)T * K->H * K->W, WS_STAGE0, &d_depth));
  BF_TRY(stage_in(ctx, poses, (size_t)T * 12, WS_STAGE1, &d_poses));
  int32_t* di;
  float* dw;
  uint8_t* du;
  bool hi, hw, hu;
  BF_TRY(stage_out(ctx, idx, (size_t)m * 8, WS_OUT0, &di, &hi));
  BF_TRY(stage_out(ctx, wts, (size_t)m * 8, WS_OUT1, &dw, &hw));
  BF_TRY(stage_out(ctx, used, (size_t)m, WS_TMP2, &du, &hu));
  BF_TRY(tri_rows(ctx, b, d_depth, T, d_poses, to_intr(K), di, dw, du));
  BF_TRY(copy_out(ctx, idx, (const int32_t*)di, (size_t)m * 8, hi));
  BF_TRY(copy_out(ctx, wts, (const float*)dw, (size_t)m * 8, hw));
  BF_TRY(copy_out(ctx, used, (const uint8_t*)du, (size_t)m, hu));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return BF_OK;
}

bf_status bf_export_precision27(bf_ctx* ctx, const bf_band* b, float* coef) {
  BF_ENTER(ctx);
  if (!b || !coef) return BF_EINVAL;
  if (b->obs_mode != 3 || !b->q27)
    return bf_fail(ctx, BF_ESTATE, "bf_export_precision27: the band holds no trilinear rows");
  const size_t n = (size_t)27 * b->N;
  if (!n) return BF_OK;
  if (is_device_ptr(coef)) BF_CK(cudaMemcpyAsync(coef, b->q27, n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  else {
    BF_CK(cudaStreamSynchronize(ctx->stream));
    BF_CK(cudaMemcpy(coef, b->q27, n * 4, cudaMemcpyDeviceToHost));
  }
  return BF_OK;
}

bf_status bf_bench_kernel(bf_ctx* ctx, bf_band* b, int which, int R, int reps, double* ms_per_launch) {
  BF_ENTER(ctx);
  if (!ctx || !b || !ms_per_launch || reps < 1 || reps > 100000) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_bench_kernel: call bf_integrate_depth first");
  if (b->N == 0) return bf_fail(ctx, BF_EINVAL, "bf_bench_kernel: empty band");
  cudaStream_t s = ctx->stream;
  if (b->obs_mode == 3 && which != BF_KERNEL_SPMV)
    return bf_fail(ctx, BF_ESTATE, "bf_bench_kernel: the band holds trilinear rows (27-point Q): SpMV only");
  if (which == BF_KERNEL_SPMV || which == BF_KERNEL_SPMM) {
    if (which == BF_KERNEL_SPMM && R != 8 && R != 16 && R != 32)
      return bf_fail(ctx, BF_EINVAL, "bf_bench_kernel: R must be 8, 16 or 32");
    const int cols = which == BF_KERNEL_SPMM ? R : 1;
    const size_t bytes = (size_t)b->N * cols * 4;
    bf_status st;
    float* x = (float*)ws_get(ctx, WS_TMP0, bytes, &st);
    if (st) return st;
    float* y = (float*)ws_get(ctx, WS_TMP1, bytes, &st);
    if (st) return st;
    BF_CK(cudaMemsetAsync(x, 0, bytes, s));
    if (which == BF_KERNEL_SPMM) BF_TRY(spmm_launch(ctx, b, x, R, y));  // builds the gather plan outside the timing
    cudaEvent_t e0, e1;
    BF_CK(cudaEventCreate(&e0));
    BF_CK(cudaEventCreate(&e1));
    BF_CK(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) {
      float* in = (i & 1) ? y : x;
      float* out = (i & 1) ? x : y;
      BF_TRY(which == BF_KERNEL_SPMM ? spmm_launch(ctx, b, in, R, out) : spmv_launch(ctx, b, in, out));
    }
    BF_CK(cudaEventRecord(e1, s));
    BF_CK(cudaEventSynchronize(e1));
    float t = 0;
    BF_CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = t / reps;
    return device_wait_status(ctx, "bf_bench_kernel");
  }
  if (which == BF_KERNEL_BLOCK_ITER) return bench_block_iter(ctx, b, R, reps, ms_per_launch);
  return bf_fail(ctx, BF_EINVAL, "bf_bench_kernel: unknown kernel");
}

bf_status bf_launch_count(int64_t* n) {
  if (!n) return BF_EINVAL;
  *n = launch_total();
  return BF_OK;
}

}  // extern "C"
