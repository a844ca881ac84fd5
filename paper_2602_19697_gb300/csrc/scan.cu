// Exclusive prefix sums of int32 arrays (three-phase: tile scan, scan of tile
// totals, add-back), used for brick and mesh compaction.
#include "internal.cuh"

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_V = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* total) {
  __shared__ int32_t warp_tot[SCAN_T / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t t = lane < SCAN_T / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < SCAN_T / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  int32_t before = wid > 0 ? warp_tot[wid - 1] : 0;
  *total = warp_tot[SCAN_T / 32 - 1];
  return before + x - v;
}

__global__ void k_scan_tile(const int32_t* in, int32_t* out, int64_t n, int32_t* tile_sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
  int32_t v[SCAN_V];
  int32_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_V; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    s += v[q];
  }
  int32_t tot;
  int32_t pre = block_excl_scan(s, &tot);
#pragma unroll
  for (int q = 0; q < SCAN_V; ++q) {
    if (base + q < n) out[base + q] = pre;
    pre += v[q];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int32_t* out, int64_t n, const int32_t* tile_pre) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int32_t add = tile_pre[blockIdx.x];
  for (int q = threadIdx.x; q < SCAN_TILE; q += SCAN_T)
    if (base + q < n) out[base + q] += add;
}

__global__ void k_copy_total(const int32_t* tile_sums, int32_t* total) { *total = tile_sums[0]; }

}  // namespace

static bf_status scan_level(bf_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                            int32_t* scratch, int64_t scratch_left) {
  if (n <= 0) {
    if (total) BF_CK(cudaMemsetAsync(total, 0, sizeof(int32_t), ctx->stream));
    return BF_OK;
  }
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt > scratch_left) return bf_fail(ctx, BF_EINVAL, "scan: scratch too small");
  int32_t* sums = scratch;
  k_scan_tile<<<(unsigned)nt, SCAN_T, 0, ctx->stream>>>(in, out, n, sums); count_launch();
  BF_CK(cudaGetLastError());
  if (nt == 1) {
    if (total) {
      k_copy_total<<<1, 1, 0, ctx->stream>>>(sums, total);
      count_launch();
    }
    return BF_OK;
  }
  BF_TRY(scan_level(ctx, sums, sums, nt, total, scratch + nt, scratch_left - nt));
  k_scan_add<<<(unsigned)nt, SCAN_T, 0, ctx->stream>>>(out, n, sums); count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}

bf_status scan_i32(bf_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, int32_t* total) {
  int64_t need = 0, m = n;
  while (m > 1) {
    m = (m + SCAN_TILE - 1) / SCAN_TILE;
    need += m;
  }
  need += 2;
  bf_status st = BF_OK;
  int32_t* scratch = (int32_t*)ws_get(ctx, WS_SCAN, (size_t)need * sizeof(int32_t), &st);
  if (st != BF_OK) return st;
  return scan_level(ctx, in, out, n, total, scratch, need);
}
