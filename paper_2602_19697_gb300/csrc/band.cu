// Band builder: coarse TSDF bootstrap, narrow-band activation and sparse
// brick compaction (Sec. 3.3 band equation, Sec. 3.4; Algorithm 1 steps 1-2).
//
// Pipeline (all on the context stream):
//   k_mark_hit     one thread per pixel: brick holding the back-projected point
//   k_dilate       three separable passes: Chebyshev dilation by r_B bricks
//   scan           candidate bricks in ascending linear brick index
//   k_tsdf         one CTA per candidate brick, one thread per voxel, frames in
//                  order; band bits by warp ballot
//   scan           active bricks -> ranks; voxel counts -> offsets
//   k_fill/k_meta  directory, coordinates, per-word lookup table
//   k_compact      compact tsdf / linear index / sample count
//   k_nbr, k_info  face-neighbour bricks, degree and boundary flag
// Every decision uses the FP32 specification arithmetic of internal.cuh.
#include "internal.cuh"

namespace {

__global__ void k_mark_hit(const float* __restrict__ depth, int T, Intr K, const float* __restrict__ poses,
                           float o0, float o1, float o2, float h8, int nb, int rB, uint8_t* hit) {
  int64_t npix = (int64_t)T * K.H * K.W;
  float org[3] = {o0, o1, o2};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npix; q += (int64_t)gridDim.x * blockDim.x) {
    float D = __ldg(depth + q);
    if (!depth_ok(D)) continue;
    int t = (int)(q / ((int64_t)K.H * K.W));
    int rem = (int)(q - (int64_t)t * K.H * K.W);
    int py = rem / K.W, px = rem - py * K.W;
    Pose P = load_pose(poses + 12 * t);
    Ray r = pixel_ray(P, px, py, K);
    int bc[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float p = f_add(P.C[k], f_mul(D, r.dw[k]));
      float g = f_div(f_sub(p, org[k]), h8);
      if (g < -(float)rB || g >= (float)(nb + rB)) ok = false;
      int b = ok ? (int)floorf(g) : 0;
      bc[k] = b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
    }
    if (ok) hit[bc[0] + (int64_t)nb * (bc[1] + (int64_t)nb * bc[2])] = 1;
  }
}

__global__ void k_dilate(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int nb, int rB, int axis) {
  int64_t nb3 = (int64_t)nb * nb * nb;
  int64_t stride = axis == 0 ? 1 : (axis == 1 ? nb : (int64_t)nb * nb);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb3; b += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)((b / stride) % nb);
    uint8_t v = 0;
    for (int d = -rB; d <= rB && !v; ++d) {
      int cc = c + d;
      if (cc >= 0 && cc < nb) v = in[b + d * stride];
    }
    out[b] = v;
  }
}

__global__ void k_u8_to_i32(const uint8_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] ? 1 : 0;
}

__global__ void k_list(const uint8_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t n,
                       int32_t* __restrict__ list) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) list[pos[i]] = (int32_t)i;
}

constexpr int POSE_CHUNK = 128;

// One CTA per candidate brick, 512 threads (one per local voxel).
__global__ void __launch_bounds__(512) k_tsdf(const int32_t* __restrict__ clist, const float* __restrict__ depth,
                                              int T, Intr K, const float* __restrict__ poses, float o0, float o1,
                                              float o2, float h, int nb, float tauc, float beta,
                                              float* __restrict__ ts, int32_t* __restrict__ wc,
                                              uint32_t* __restrict__ cmask, int32_t* __restrict__ ccount) {
  __shared__ float sp[POSE_CHUNK * 12];
  __shared__ int32_t scount;
  int c = blockIdx.x;
  int b = clist[c];
  int bi = b % nb, bj = (b / nb) % nb, bk = b / (nb * nb);
  int l = threadIdx.x;
  int i = 8 * bi + (l & 7), j = 8 * bj + ((l >> 3) & 7), k = 8 * bk + (l >> 6);
  float x0 = vox_c(o0, h, i), x1 = vox_c(o1, h, j), x2 = vox_c(o2, h, k);
  if (l == 0) scount = 0;
  float S = 0.0f;
  int cnt = 0;
  const int64_t fsz = (int64_t)K.H * K.W;
  for (int t0 = 0; t0 < T; t0 += POSE_CHUNK) {
    int nt = min(POSE_CHUNK, T - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < nt * 12; q += blockDim.x) sp[q] = poses[12 * t0 + q];
    __syncthreads();
    for (int tt = 0; tt < nt; ++tt) {
      const float* P = sp + 12 * tt;
      float dx = f_sub(x0, P[3]), dy = f_sub(x1, P[7]), dz = f_sub(x2, P[11]);
      float xc = f_add(f_add(f_mul(P[0], dx), f_mul(P[4], dy)), f_mul(P[8], dz));
      float yc = f_add(f_add(f_mul(P[1], dx), f_mul(P[5], dy)), f_mul(P[9], dz));
      float zc = f_add(f_add(f_mul(P[2], dx), f_mul(P[6], dy)), f_mul(P[10], dz));
      if (!(zc > 0.0f)) continue;
      float u = f_add(f_div(f_mul(K.fx, xc), zc), K.cx);
      float v = f_add(f_div(f_mul(K.fy, yc), zc), K.cy);
      if (!(u >= 0.0f && u < (float)K.W && v >= 0.0f && v < (float)K.H)) continue;
      int px = (int)u, py = (int)v;
      float D = __ldg(depth + (int64_t)(t0 + tt) * fsz + (int64_t)py * K.W + px);
      if (!depth_ok(D)) continue;
      float sdf = f_sub(D, zc);
      if (sdf < -tauc) continue;
      float smp = sdf < tauc ? sdf : tauc;
      S = f_add(S, smp);
      cnt += 1;
    }
  }
  float tsdf = cnt > 0 ? f_div(S, (float)cnt) : 0.0f;
  bool in = cnt > 0 && fabsf(tsdf) <= beta;
  ts[(int64_t)c * 512 + l] = tsdf;
  wc[(int64_t)c * 512 + l] = cnt;
  uint32_t bits = __ballot_sync(0xffffffffu, in);
  if ((l & 31) == 0) {
    cmask[(int64_t)c * 16 + (l >> 5)] = bits;
    atomicAdd(&scount, __popc(bits));
  }
  __syncthreads();
  if (l == 0) ccount[c] = scount;
}

__global__ void k_active_flag(const int32_t* __restrict__ ccount, int32_t* __restrict__ flag, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = ccount[i] > 0 ? 1 : 0;
}

__global__ void k_fill(const int32_t* __restrict__ clist, const int32_t* __restrict__ ccount,
                       const int32_t* __restrict__ rank, int64_t ncand, int nb, int32_t* __restrict__ dir,
                       int32_t* __restrict__ bcoord, int32_t* __restrict__ counts, int32_t* __restrict__ cand_of) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncand; c += (int64_t)gridDim.x * blockDim.x) {
    if (ccount[c] <= 0) continue;
    int r = rank[c];
    int b = clist[c];
    dir[b] = r;
    bcoord[4 * r] = b % nb;
    bcoord[4 * r + 1] = (b / nb) % nb;
    bcoord[4 * r + 2] = b / (nb * nb);
    bcoord[4 * r + 3] = 0;
    counts[r] = ccount[c];
    cand_of[r] = (int32_t)c;
  }
}

// per-word lookup: bits and compact index of the word's first band voxel
__global__ void k_meta(const int32_t* __restrict__ cand_of, const uint32_t* __restrict__ cmask,
                       const int32_t* __restrict__ off, int NB, MetaWord* __restrict__ meta) {
  int r = blockIdx.x * (blockDim.x / 16) + threadIdx.x / 16;
  int w = threadIdx.x & 15;
  bool live = r < NB;  // all lanes stay for the segmented shuffle
  uint32_t bits = live ? cmask[(int64_t)cand_of[r] * 16 + w] : 0u;
  int pc = __popc(bits);
  // exclusive prefix over the 16 words of this brick (16-lane segment)
  int x = pc;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o, 16);
    if (w >= o) x += y;
  }
  if (!live) return;
  MetaWord m;
  m.bits = bits;
  m.base = off[r] + x - pc;
  meta[16 * r + w] = m;
}

__global__ void __launch_bounds__(512) k_compact(const int32_t* __restrict__ cand_of, const MetaWord* __restrict__ meta,
                                                 const float* __restrict__ ts, const int32_t* __restrict__ wc,
                                                 const int32_t* __restrict__ bcoord, int n, float* __restrict__ tsdf,
                                                 int32_t* __restrict__ wcount, int32_t* __restrict__ lin) {
  int r = blockIdx.x;
  int l = threadIdx.x;
  MetaWord m = meta[16 * r + (l >> 5)];
  uint32_t bit = 1u << (l & 31);
  if (!(m.bits & bit)) return;
  int idx = m.base + __popc(m.bits & (bit - 1u));
  int64_t c = cand_of[r];
  tsdf[idx] = ts[c * 512 + l];
  wcount[idx] = wc[c * 512 + l];
  int i = 8 * bcoord[4 * r] + (l & 7), j = 8 * bcoord[4 * r + 1] + ((l >> 3) & 7), k = 8 * bcoord[4 * r + 2] + (l >> 6);
  lin[idx] = i + n * (j + n * k);
}

__global__ void k_nbr(const int32_t* __restrict__ bcoord, const int32_t* __restrict__ dir, int NB, int nb,
                      int32_t* __restrict__ nbr) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NB * 6) return;
  int r = q / 6, f = q - 6 * r;
  int c[3] = {bcoord[4 * r], bcoord[4 * r + 1], bcoord[4 * r + 2]};
  c[f >> 1] += (f & 1) ? 1 : -1;
  int v = -1;
  if (c[0] >= 0 && c[1] >= 0 && c[2] >= 0 && c[0] < nb && c[1] < nb && c[2] < nb)
    v = dir[c[0] + nb * (c[1] + nb * c[2])];
  nbr[q] = v;
}

__global__ void k_info(BandView B, uint8_t* __restrict__ info) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int L = B.lin[v];
    int i = L % B.n, j = (L / B.n) % B.n, k = L / (B.n * B.n);
    int d = (band_lookup(B, i - 1, j, k) >= 0) + (band_lookup(B, i + 1, j, k) >= 0) +
            (band_lookup(B, i, j - 1, k) >= 0) + (band_lookup(B, i, j + 1, k) >= 0) +
            (band_lookup(B, i, j, k - 1) >= 0) + (band_lookup(B, i, j, k + 1) >= 0);
    info[v] = (uint8_t)(d | ((d < 6) << 3));
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

BandView band_view(const bf_band* b) {
  BandView v;
  v.n = b->grid.n;
  v.nb = b->nb;
  v.NB = b->NB;
  v.N = (int)b->N;
  v.h = b->grid.voxel;
  v.o0 = b->grid.origin[0];
  v.o1 = b->grid.origin[1];
  v.o2 = b->grid.origin[2];
  v.dir = b->dir;
  v.meta = b->meta;
  v.off = b->off;
  v.nbr = b->nbr;
  v.bcoord = b->bcoord;
  v.lin = b->lin;
  return v;
}

static bf_status read_i32(bf_ctx* ctx, const int32_t* dptr, int32_t* host) {
  BF_CK(cudaMemcpyAsync(ctx->h_pinned, dptr, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  *host = ctx->h_pinned[0];
  return BF_OK;
}

bf_status band_build(bf_ctx* ctx, const float* depth, int T, const float* poses, const Intr& K, const bf_grid& g,
                     const bf_params& p, bf_band** out) {
  cudaStream_t s = ctx->stream;
  const int n = g.n, nb = n / 8;
  const int64_t nb3 = (int64_t)nb * nb * nb;
  const int rB = brick_radius(p.trunc_vox);
  const float h = g.voxel;
  const float h8 = 8.0f * h;
  const float tauc = (float)p.trunc_vox * h;
  const float beta = (float)p.band_vox * h;
  bf_status st = BF_OK;

  // candidate bricks
  uint8_t* hitA = (uint8_t*)ws_get(ctx, WS_TMP0, nb3, &st);
  if (st) return st;
  uint8_t* hitB = (uint8_t*)ws_get(ctx, WS_TMP1, nb3, &st);
  if (st) return st;
  int32_t* pos = (int32_t*)ws_get(ctx, WS_TMP2, (nb3 + 1) * sizeof(int32_t), &st);
  if (st) return st;
  BF_CK(cudaMemsetAsync(hitA, 0, nb3, s));
  int64_t npix = (int64_t)T * K.H * K.W;
  k_mark_hit<<<grid_for(npix, 256), 256, 0, s>>>(depth, T, K, poses, g.origin[0], g.origin[1], g.origin[2], h8, nb,
                                                rB, hitA); count_launch();
  BF_CK(cudaGetLastError());
  k_dilate<<<grid_for(nb3, 256), 256, 0, s>>>(hitA, hitB, nb, rB, 0); count_launch();
  k_dilate<<<grid_for(nb3, 256), 256, 0, s>>>(hitB, hitA, nb, rB, 1); count_launch();
  k_dilate<<<grid_for(nb3, 256), 256, 0, s>>>(hitA, hitB, nb, rB, 2); count_launch();
  BF_CK(cudaGetLastError());
  k_u8_to_i32<<<grid_for(nb3, 256), 256, 0, s>>>(hitB, pos, nb3); count_launch();
  BF_TRY(scan_i32(ctx, pos, pos, nb3, pos + nb3));
  int32_t ncand = 0;
  BF_TRY(read_i32(ctx, pos + nb3, &ncand));

  bf_band* b = new bf_band();
  b->grid = g;
  b->prm = p;
  b->nb = nb;
  b->ncand = ncand;
  b->stream = s;
  b->device = ctx->device;
  auto fail = [&](bf_status e) {
    bf_band_free(b);
    return e;
  };
  if ((st = dev_alloc_t(ctx, &b->dir, nb3))) return fail(st);
  if (cudaMemsetAsync(b->dir, 0xff, nb3 * sizeof(int32_t), s) != cudaSuccess)
    return fail(bf_fail(ctx, BF_ECUDA, "memset dir"));
  if (ncand == 0) {
    b->NB = 0;
    b->N = 0;
    if ((st = dev_alloc_t(ctx, &b->off, 1))) return fail(st);
    cudaMemsetAsync(b->off, 0, sizeof(int32_t), s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(bf_fail(ctx, BF_ECUDA, "sync"));
    *out = b;
    return BF_OK;
  }
  int32_t* clist = (int32_t*)ws_get(ctx, WS_TMP3, (size_t)ncand * sizeof(int32_t), &st);
  if (st) return fail(st);
  k_list<<<grid_for(nb3, 256), 256, 0, s>>>(hitB, pos, nb3, clist); count_launch();

  // TSDF of candidate voxels
  float* ts = (float*)ws_get(ctx, WS_TMP4, (size_t)ncand * 512 * sizeof(float), &st);
  if (st) return fail(st);
  int32_t* wc = (int32_t*)ws_get(ctx, WS_TMP5, (size_t)ncand * 512 * sizeof(int32_t), &st);
  if (st) return fail(st);
  uint32_t* cmask = (uint32_t*)ws_get(ctx, WS_TMP0, (size_t)ncand * 16 * sizeof(uint32_t), &st);
  if (st) return fail(st);
  int32_t* ccount = (int32_t*)ws_get(ctx, WS_TMP1, (size_t)ncand * 3 * sizeof(int32_t) + 16, &st);
  if (st) return fail(st);
  int32_t* rank = ccount + ncand;
  int32_t* rank_tot = rank + ncand;
  k_tsdf<<<(unsigned)ncand, 512, 0, s>>>(clist, depth, T, K, poses, g.origin[0], g.origin[1], g.origin[2], h, nb,
                                        tauc, beta, ts, wc, cmask, ccount); count_launch();
  if (cudaGetLastError() != cudaSuccess) return fail(bf_fail(ctx, BF_ECUDA, "k_tsdf launch"));
  k_active_flag<<<grid_for(ncand, 256), 256, 0, s>>>(ccount, rank, ncand); count_launch();
  if ((st = scan_i32(ctx, rank, rank, ncand, rank_tot))) return fail(st);
  int32_t NB = 0;
  if ((st = read_i32(ctx, rank_tot, &NB))) return fail(st);
  b->NB = NB;
  if ((st = dev_alloc_t(ctx, &b->bcoord, (size_t)4 * (NB ? NB : 1)))) return fail(st);
  if ((st = dev_alloc_t(ctx, &b->off, (size_t)NB + 1))) return fail(st);
  if ((st = dev_alloc_t(ctx, &b->meta, (size_t)16 * (NB ? NB : 1)))) return fail(st);
  if ((st = dev_alloc_t(ctx, &b->nbr, (size_t)6 * (NB ? NB : 1)))) return fail(st);
  int32_t* cand_of = pos;  // reuse: NB <= nb3
  k_fill<<<grid_for(ncand, 256), 256, 0, s>>>(clist, ccount, rank, ncand, nb, b->dir, b->bcoord, b->off, cand_of); count_launch();
  if ((st = scan_i32(ctx, b->off, b->off, NB, b->off + NB))) return fail(st);
  int32_t N = 0;
  if ((st = read_i32(ctx, b->off + NB, &N))) return fail(st);
  b->N = N;
  if (NB > 0) {
    k_meta<<<(NB + 7) / 8, 128, 0, s>>>(cand_of, cmask, b->off, NB, b->meta); count_launch();
    if ((st = dev_alloc_t(ctx, &b->lin, N))) return fail(st);
    if ((st = dev_alloc_t(ctx, &b->tsdf, N))) return fail(st);
    if ((st = dev_alloc_t(ctx, &b->wcount, N))) return fail(st);
    if ((st = dev_alloc_t(ctx, &b->info, N))) return fail(st);
    k_compact<<<NB, 512, 0, s>>>(cand_of, b->meta, ts, wc, b->bcoord, n, b->tsdf, b->wcount, b->lin); count_launch();
    k_nbr<<<(NB * 6 + 255) / 256, 256, 0, s>>>(b->bcoord, b->dir, NB, nb, b->nbr); count_launch();
    k_info<<<grid_for(N, 256), 256, 0, s>>>(band_view(b), b->info); count_launch();
    if (cudaGetLastError() != cudaSuccess) return fail(bf_fail(ctx, BF_ECUDA, "band kernels launch"));
  }
  *out = b;
  return BF_OK;
}
