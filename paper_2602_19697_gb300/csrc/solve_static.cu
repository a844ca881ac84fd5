// Allocation-free variant of the mean solve (bf_solve_mean_static).
//
// For callers that cannot allocate device memory while they run -- a
// real-time loop with a fixed memory budget, or a host that owns the device
// allocator and forbids cudaMalloc from libraries -- this entry point solves
// Q mu = h with every scratch vector in one file-scope __device__ array of
// fixed size (STATIC_MAX_VOX band voxels).  The array exists on every GPU
// that loads the library, from load until process exit.
//
// Method: Jacobi-PCG in its two-kernel form with FP32 vectors and FP64 inner
// products, inside iterative refinement on an FP64 master iterate (true
// residual h - Q x64 in FP64), the same stopping rule as bf_solve_mean.  No
// graph is used (instantiating one allocates); the host launches the
// iterations and reads the stop flag every 16 iterations.
//
// The array is shared by every call: a call clears what must start at zero
// (state, counters, correction vector), and calls whose GPU work overlaps
// (two streams, two threads) race on it.
#include <cstring>

#include "internal.cuh"

namespace {

constexpr int SBT = 128;              // threads per brick CTA
constexpr int SNCTA = 152 * 4;        // brick CTAs (strided over the bricks)
constexpr int64_t STATIC_MAX_VOX = 262144;

struct SState {
  int done, status, iter, inner_done;  // first 32 bytes are read back by the host
  double rr0, bb0;
  double alpha, beta, rho, rr, bb, tol2, tol0;
  int max_iter;
  unsigned int cnt;
};

// byte layout of the scratch array
constexpr size_t S_X64 = 0;                                  // double [max]
constexpr size_t S_R = S_X64 + 8 * STATIC_MAX_VOX;           // float  [max]
constexpr size_t S_P0 = S_R + 4 * STATIC_MAX_VOX;            // float  [max]
constexpr size_t S_P1 = S_P0 + 4 * STATIC_MAX_VOX;           // float  [max]
constexpr size_t S_Q = S_P1 + 4 * STATIC_MAX_VOX;            // float  [max]
constexpr size_t S_X = S_Q + 4 * STATIC_MAX_VOX;             // float  [max]
constexpr size_t S_PART = S_X + 4 * STATIC_MAX_VOX;          // double [3][SNCTA]
constexpr size_t S_STATE = S_PART + 8 * 3 * SNCTA;           // SState
constexpr size_t S_BYTES = S_STATE + 256;

static __device__ __align__(256) unsigned char g_solve_scratch[S_BYTES];

struct Ptrs {
  double* x64;
  float *r, *p[2], *q, *x;
  double* part;
  SState* st;
};

__device__ __forceinline__ Ptrs carve(unsigned char* base) {
  Ptrs P;
  P.x64 = (double*)(base + S_X64);
  P.r = (float*)(base + S_R);
  P.p[0] = (float*)(base + S_P0);
  P.p[1] = (float*)(base + S_P1);
  P.q = (float*)(base + S_Q);
  P.x = (float*)(base + S_X);
  P.part = (double*)(base + S_PART);
  P.st = (SState*)(base + S_STATE);
  return P;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA sums -> part[k][blockIdx]; true in the last CTA to arrive, which then
// holds the fixed-order totals in tot[]
template <int NV>
__device__ bool reduce_all(double (&v)[NV], double* part, unsigned int* cnt, double (&tot)[NV]) {
  __shared__ double sh[NV][SBT / 32];
  __shared__ double fin[NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = wsum(v[k]);
    if (lane == 0) sh[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < SBT / 32; ++q) s += sh[k][q];
      part[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  for (int k = w; k < NV; k += SBT / 32) {
    // the lane's partials in index order, eight loads in flight at a time
    const double* p = part + (size_t)k * gridDim.x;
    const int n = (int)gridDim.x;
    double s = 0;
    for (int i0 = lane; i0 < n; i0 += 8 * 32) {
      double v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = i0 + 32 * j < n ? __ldcg(p + i0 + 32 * j) : 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j) s += v[j];
    }
    s = wsum(s);
    if (lane == 0) fin[k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = fin[k];
  return true;
}

__device__ __forceinline__ void meta7(const BandView& B, int b, MetaWord (*sm)[16]) {
  if (threadIdx.x < 112) {
    int which = threadIdx.x >> 4, w = threadIdx.x & 15;
    int r = which == 0 ? b : __ldg(B.nbr + 6 * b + which - 1);
    MetaWord m;
    m.bits = 0;
    m.base = 0;
    if (r >= 0) m = B.meta[16 * r + w];
    sm[which][w] = m;
  }
}

__device__ __forceinline__ int slot(const MetaWord (*sm)[16], int which, int l) {
  MetaWord m = sm[which][l >> 5];
  uint32_t bit = 1u << (l & 31);
  return (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
}

__device__ __forceinline__ int tile_of(int l) { return (l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1); }

__device__ __forceinline__ void halo(const MetaWord (*sm)[16], int q, int* idx, int* tp) {
  int f = q >> 6, u = q & 7, v = (q >> 3) & 7, a = f >> 1, side = f & 1;
  int lc[3], tc[3];
  int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
  lc[a] = side ? 0 : 7;
  tc[a] = side ? 9 : 0;
  lc[o1] = u;
  lc[o2] = v;
  tc[o1] = u + 1;
  tc[o2] = v + 1;
  *idx = slot(sm, 1 + f, lc[0] + 8 * lc[1] + 64 * lc[2]);
  *tp = tc[0] + 10 * tc[1] + 100 * tc[2];
}

template <class T>
__device__ __forceinline__ T six(const T* t, int c) {
  return ((t[c - 1] + t[c + 1]) + (t[c - 10] + t[c + 10])) + (t[c - 100] + t[c + 100]);
}

__global__ void k_s_init(unsigned char* base, int N, const float* __restrict__ mu0, int warm, double tol, int max_iter) {
  Ptrs P = carve(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    P.x64[i] = warm ? (double)mu0[i] : 0.0;
    P.x[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SState* st = P.st;
    st->done = st->status = st->iter = st->inner_done = 0;
    st->tol0 = tol;
    st->max_iter = max_iter;
    st->alpha = st->beta = 0.0;
    st->cnt = 0;
  }
}

// true residual r = h - Q x64 (FP64), r.r, h.h, r.(r/qd); sets up the
// correction solve (stop test, eta, rho, beta = 0)
__global__ void __launch_bounds__(SBT) k_s_res(unsigned char* base, BandView B, float lam,
                                               const float* __restrict__ qd, const float* __restrict__ rhs) {
  Ptrs P = carve(base);
  __shared__ double tile[1000];
  __shared__ MetaWord sm[7][16];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
    meta7(B, b, sm);
    __syncthreads();
    int idx[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = threadIdx.x + SBT * s;
      idx[s] = slot(sm, 0, l);
      tile[tile_of(l)] = idx[s] >= 0 ? P.x64[idx[s]] : 0.0;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int j, tp;
      halo(sm, threadIdx.x + SBT * s, &j, &tp);
      tile[tp] = j >= 0 ? P.x64[j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (idx[s] < 0) continue;
      const int c = tile_of(threadIdx.x + SBT * s);
      const double q = (double)__ldg(qd + idx[s]), h = (double)__ldg(rhs + idx[s]);
      const double r = h - (q * tile[c] - (double)lam * six(tile, c));
      P.r[idx[s]] = (float)r;
      acc[0] += r * r;
      acc[1] += h * h;
      acc[2] += r * r / q;
    }
  }
  double tot[3];
  if (!reduce_all<3>(acc, P.part, &P.st->cnt, tot)) return;
  if (threadIdx.x == 0) {
    SState* st = P.st;
    st->rr0 = tot[0];
    st->bb0 = tot[1];
    const int conv = tot[0] <= st->tol0 * st->tol0 * tot[1] || tot[1] == 0.0;
    if (conv) st->status = 0;
    else if (st->iter >= st->max_iter) st->status = 1;
    st->done = conv || st->iter >= st->max_iter || st->status == 2;
    double eta = conv ? 0.5 : 0.5 * st->tol0 * sqrt(tot[1] / tot[0]);
    eta = fmin(fmax(eta, 1e-7), 0.5);
    st->tol2 = eta * eta;
    st->bb = tot[0];
    st->rho = tot[2];
    st->beta = 0.0;
    st->inner_done = st->done;
    st->cnt = 0;
  }
}

// p_out = r/qd + beta p_in (own voxels and halo), q = Q p_out, alpha = rho / p.q
__global__ void __launch_bounds__(SBT) k_s_a(unsigned char* base, BandView B, float lam, const float* __restrict__ qd,
                                             int in) {
  Ptrs P = carve(base);
  SState* st = P.st;
  if (st->inner_done) return;
  __shared__ float tile[1000];
  __shared__ MetaWord sm[7][16];
  const float bt = (float)st->beta;
  const float* __restrict__ pin = P.p[in];
  float* __restrict__ pout = P.p[in ^ 1];
  double acc[1] = {0.0};
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
    meta7(B, b, sm);
    __syncthreads();
    int idx[4];
    float pv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = threadIdx.x + SBT * s;
      idx[s] = slot(sm, 0, l);
      float v = 0.0f;
      if (idx[s] >= 0) {
        const int i = idx[s];
        v = P.r[i] / __ldg(qd + i) + (bt != 0.0f ? bt * pin[i] : 0.0f);
      }
      pv[s] = v;
      tile[tile_of(l)] = v;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int j, tp;
      halo(sm, threadIdx.x + SBT * s, &j, &tp);
      float v = 0.0f;
      if (j >= 0) v = P.r[j] / __ldg(qd + j) + (bt != 0.0f ? bt * pin[j] : 0.0f);
      tile[tp] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (idx[s] < 0) continue;
      const int c = tile_of(threadIdx.x + SBT * s);
      const float y = __ldg(qd + idx[s]) * tile[c] - lam * six(tile, c);
      P.q[idx[s]] = y;
      pout[idx[s]] = pv[s];
      acc[0] += (double)pv[s] * (double)y;
    }
  }
  double tot[1];
  if (!reduce_all<1>(acc, P.part, &st->cnt, tot)) return;
  if (threadIdx.x == 0) {
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      st->status = 2;
      st->done = st->inner_done = 1;
      st->alpha = 0.0;
    } else {
      st->alpha = st->rho / tot[0];
    }
    st->cnt = 0;
  }
}

// x += alpha p, r -= alpha q, rho' = r.(r/qd), r.r; beta and the stop test
__global__ void __launch_bounds__(SBT) k_s_b(unsigned char* base, int N, const float* __restrict__ qd, int cur) {
  Ptrs P = carve(base);
  SState* st = P.st;
  if (st->inner_done) return;
  const float a = (float)st->alpha;
  const float* __restrict__ p = P.p[cur];
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * SBT + threadIdx.x; i < N; i += gridDim.x * SBT) {
    P.x[i] += a * p[i];
    const float r = P.r[i] - a * P.q[i];
    P.r[i] = r;
    acc[0] += (double)r * (double)r / (double)__ldg(qd + i);
    acc[1] += (double)r * (double)r;
  }
  double tot[2];
  if (!reduce_all<2>(acc, P.part, &st->cnt, tot)) return;
  if (threadIdx.x == 0) {
    st->iter += 1;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      st->status = 2;
      st->done = st->inner_done = 1;
    } else if (tot[1] <= st->tol2 * st->bb || st->iter >= st->max_iter) {
      st->inner_done = 1;
    }
    st->beta = tot[0] / st->rho;
    st->rho = tot[0];
    st->cnt = 0;
  }
}

__global__ void k_s_axpy(unsigned char* base, int N) {
  Ptrs P = carve(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    P.x64[i] += (double)P.x[i];
    P.x[i] = 0.0f;
  }
}

__global__ void k_s_out(unsigned char* base, int N, float* __restrict__ mu) {
  Ptrs P = carve(base);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) mu[i] = (float)P.x64[i];
}

// device address of the scratch array, looked up once per device
unsigned char* g_scratch_addr[64] = {nullptr};

}  // namespace

extern "C" bf_status bf_solve_mean_static(bf_ctx* ctx, bf_band* b, double rel_tol, int max_iter, float* mu,
                                          int* iters, double* rel_res) {
  BF_ENTER(ctx);
  if (!ctx || !b || !mu) return BF_EINVAL;
  if (!b->integrated || b->obs_mode == 3) return BF_ESTATE;  // the 7-point system only
  if (!(rel_tol > 0.0) || !(rel_tol < 1.0) || max_iter < 1 || max_iter > 10000000) return BF_EINVAL;
  if (b->N > STATIC_MAX_VOX) return BF_EINVAL;  // larger bands need bf_solve_mean
  if (!is_device_ptr(mu)) return BF_EINVAL;     // no staging buffer to copy through
  if (ctx->device < 0 || ctx->device >= 64) return BF_EINVAL;
  if (b->N == 0) {
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    return BF_OK;
  }
  unsigned char*& base = g_scratch_addr[ctx->device];
  if (!base) {
    // once per device, with that device current (ctx calls run on it)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_solve_scratch) != cudaSuccess) {
      cudaGetLastError();
      return BF_ECUDA;
    }
    base = (unsigned char*)p;
  }
  cudaStream_t s = ctx->stream;
  const int N = (int)b->N;
  const BandView bv = band_view(b);
  const float lam = (float)b->prm.lambda;
  // every kernel that writes partial sums runs at most SNCTA CTAs (the
  // partial-sum area holds 3 x SNCTA doubles)
  const unsigned gN = (unsigned)((N + SBT - 1) / SBT < SNCTA ? (N + SBT - 1) / SBT : SNCTA);
  const unsigned gB = (unsigned)(b->NB < SNCTA ? b->NB : SNCTA);
  k_s_init<<<gN, SBT, 0, s>>>(base, N, mu, 0, rel_tol, max_iter);
  count_launch();
  SState* hs = (SState*)ctx->h_pinned;  // 64 pinned bytes owned by the context; the first 32 are read
  bool done = false;
  for (int outer = 0; outer < REFINE_MAX_PASSES && !done; ++outer) {
    k_s_res<<<gB, SBT, 0, s>>>(base, bv, lam, b->qd, b->rhs);
    count_launch();
    if (cudaMemcpyAsync(hs, base + S_STATE, 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return BF_ECUDA;
    if (hs->done) {
      done = true;
      break;
    }
    for (int chunk = 0; chunk < (max_iter + 15) / 16 + 1; ++chunk) {
      for (int k = 0; k < 8; ++k) {
        k_s_a<<<gB, SBT, 0, s>>>(base, bv, lam, b->qd, 0);
        k_s_b<<<gN, SBT, 0, s>>>(base, N, b->qd, 1);
        k_s_a<<<gB, SBT, 0, s>>>(base, bv, lam, b->qd, 1);
        k_s_b<<<gN, SBT, 0, s>>>(base, N, b->qd, 0);
        count_launch(4);
      }
      if (cudaMemcpyAsync(hs, base + S_STATE, 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return BF_ECUDA;
      if (hs->inner_done) break;
    }
    k_s_axpy<<<gN, SBT, 0, s>>>(base, N);
    count_launch();
  }
  if (!done) {  // final true residual after the last correction
    k_s_res<<<gB, SBT, 0, s>>>(base, bv, lam, b->qd, b->rhs);
    count_launch();
  }
  k_s_out<<<gN, SBT, 0, s>>>(base, N, mu);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return BF_ECUDA;
  if (cudaMemcpyAsync(hs, base + S_STATE, 32, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BF_ECUDA;
  if (iters) *iters = hs->iter;
  if (rel_res) *rel_res = hs->bb0 > 0 ? sqrt(hs->rr0 / hs->bb0) : 0.0;
  if (hs->status == 2) return BF_BREAKDOWN;
  if (!hs->done || hs->status == 1) return BF_NOT_CONVERGED;
  return BF_OK;
}
