// Matrix-free 7-point SpMV and Jacobi-PCG for the MAP mean (Sec. 3.6 MAP
// equation, solved by PCG; Algorithm 1 step 5).
//
// Layout.  Band vectors are compact ([N], brick-ordered).  k_brick runs one
// 128-thread CTA per active 8^3 brick: it stages the brick's voxels and the
// facing layers of its six neighbour bricks into a 10^3 shared-memory tile
// (non-band slots hold 0, so the stencil needs no masks), then applies
// (Qx)_j = Q_jj x_j - lambda * sum of the six tile neighbours.
//
// PCG (Jacobi M = diag Q), two kernels per iteration:
//   A  k_brick<MODE_PCG>: p <- r/qd + beta p (own voxels and halo, recomputed
//      identically by every CTA that needs them), q = Q p, partial p.q;
//      the last CTA to finish reduces the partials in a fixed order
//      (deterministic) and sets alpha = rho / p.q.
//   B  k_update: x += alpha p, r -= alpha q, partial r.(r/qd) and r.r; the
//      last CTA sets beta, rho, the iteration count and the stop flag.
// p ping-pongs between two buffers, so one graph body holds two iterations.
// The loop is a CUDA-graph WHILE node: B clears the condition when the
// recursive residual meets the tolerance, the iteration limit is reached or
// a scalar breaks down; A and B return at once once the stop flag is set.
// After the loop, k_brick<MODE_RESID> recomputes the true residual
// b - Q x with FP64 accumulation and restarts the loop if it misses.
#include <cstdio>

#include "internal.cuh"

namespace {

constexpr int MODE_PLAIN = 0;  // y = Q x
constexpr int MODE_PCG = 1;    // fused p update, q = Q p, p.q
constexpr int MODE_RESID = 2;  // r = b - Q x (FP64), p = 0, r.r, r.z, b.b (FP64 solver restart)
constexpr int MODE_OUTER = 3;  // as RESID from the FP64 master iterate; sets up the FP32 correction solve
constexpr int BT = 128;        // threads per brick CTA

struct PcgState {
  double rho, pq, alpha, beta, rr, bb, tol2;  // inner (current) PCG
  double rr0, bb0, tol0;                      // true residual, |h|^2, requested tolerance
  int iter, max_iter, done, status;
  unsigned int cntA, cntB, cntR;
  unsigned int guard;  // body executions, a hard stop independent of the reductions
  unsigned int nexec;  // graph-body kernels executed (for launch accounting)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of NV doubles (blockDim.x = 32 * NW); result valid in thread 0
template <int NV, int NW>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][NW];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
#pragma unroll
      for (int q = 0; q < NW; ++q) s += sh[k][q];
      v[k] = s;
    }
  }
  __syncthreads();
}

// Publish this CTA's partial sums; returns true in every thread of the last
// CTA to arrive, which then sees all partials.
template <int NV>
__device__ __forceinline__ bool publish_partials(const double (&v)[NV], double* part, unsigned int* counter) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[(size_t)k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// fixed-order reduction of the partials by the last CTA (NW warps)
template <int NV, int NW>
__device__ __forceinline__ void reduce_partials(const double* part, double (&out)[NV]) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(part + (size_t)k * gridDim.x + i);
    v[k] = s;
  }
  block_sum<NV, NW>(v);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = v[k];
}

template <class T, int mode, class TO = T>
__global__ void __launch_bounds__(BT) k_brick(BandView B, float lam, const float* __restrict__ qd,
                                              const T* __restrict__ xin, const T* __restrict__ rin,
                                              TO* __restrict__ pout, TO* __restrict__ yout,
                                              const float* __restrict__ rhs, double* part, PcgState* st,
                                              cudaGraphConditionalHandle handle) {
  if (mode == MODE_PCG) {
    // Inside the WHILE body: block 0 ends the loop once the stop flag is set
    // or the body has run more than 2 max_iter + 64 times.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->nexec += 2;  // this kernel and the update that follows it
      unsigned g = atomicAdd(&st->guard, 1u);
      if (st->done || g > 2u * (unsigned)st->max_iter + 64u) {
        if (!st->done) { st->status = 1; st->done = 1; }
        cudaGraphSetConditional(handle, 0);
      }
    }
    if (st->done) return;
  }
  __shared__ T tile[1000];
  __shared__ MetaWord sm[7][16];
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  const double beta = (mode == MODE_PCG) ? st->beta : 0.0;
  const T betaT = (T)beta;
  if (tid < 7 * 16) {
    int which = tid >> 4, w = tid & 15;
    int r = which == 0 ? b : __ldg(B.nbr + 6 * b + which - 1);
    MetaWord m;
    m.bits = 0;
    m.base = 0;
    if (r >= 0) m = B.meta[16 * r + w];
    sm[which][w] = m;
  }
  __syncthreads();
  // own voxels: 4 slots per thread, slot l = tid + 128 s
  int idx[4];
  float qv[4];
  T val[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int l = tid + BT * s;
    MetaWord m = sm[0][l >> 5];
    uint32_t bit = 1u << (l & 31);
    idx[s] = (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    T v = 0;
    float q = 0.0f;
    if (idx[s] >= 0) {
      q = __ldg(qd + idx[s]);
      if (mode == MODE_PCG) v = (T)__ldg(rin + idx[s]) / (T)q + betaT * __ldg(xin + idx[s]);
      else v = __ldg(xin + idx[s]);
    }
    val[s] = v;
    qv[s] = q;
    int l = tid + BT * s;
    tile[(l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1)] = v;
  }
  // halo: 6 faces x 64 slots, 3 per thread
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    int q = tid + BT * s;
    int f = q >> 6, u = q & 7, v = (q >> 3) & 7;
    int a = f >> 1, side = f & 1;
    int lc[3], tc[3];
    int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
    lc[a] = side ? 0 : 7;
    tc[a] = side ? 9 : 0;
    lc[o1] = u;
    lc[o2] = v;
    tc[o1] = u + 1;
    tc[o2] = v + 1;
    int l = lc[0] + 8 * lc[1] + 64 * lc[2];
    MetaWord m = sm[1 + f][l >> 5];
    uint32_t bit = 1u << (l & 31);
    T hv = 0;
    if (m.bits & bit) {
      int j = m.base + __popc(m.bits & (bit - 1u));
      if (mode == MODE_PCG) hv = (T)__ldg(rin + j) / (T)__ldg(qd + j) + betaT * __ldg(xin + j);
      else hv = __ldg(xin + j);
    }
    tile[tc[0] + 10 * tc[1] + 100 * tc[2]] = hv;
  }
  __syncthreads();
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (idx[s] < 0) continue;
    int l = tid + BT * s;
    int c = (l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1);
    T nsum = ((tile[c - 1] + tile[c + 1]) + (tile[c - 10] + tile[c + 10])) + (tile[c - 100] + tile[c + 100]);
    if (mode == MODE_RESID || mode == MODE_OUTER) {
      double ns = (((double)tile[c - 1] + (double)tile[c + 1]) + ((double)tile[c - 10] + (double)tile[c + 10])) +
                  ((double)tile[c - 100] + (double)tile[c + 100]);
      double qx = (double)qv[s] * (double)tile[c] - (double)lam * ns;
      double r = (double)__ldg(rhs + idx[s]) - qx;
      yout[idx[s]] = (TO)r;
      pout[idx[s]] = (TO)0;
      acc[0] += r * r;
      acc[1] += r * r / (double)qv[s];
      double bb = (double)__ldg(rhs + idx[s]);
      acc[2] += bb * bb;
    } else {
      T y = (T)qv[s] * tile[c] - (T)lam * nsum;
      yout[idx[s]] = y;
      if (mode == MODE_PCG) {
        pout[idx[s]] = val[s];
        acc[0] += (double)val[s] * (double)y;
      }
    }
  }
  if (mode == MODE_PLAIN) return;
  if (mode == MODE_PCG) {
    double v1[1] = {acc[0]};
    block_sum<1, BT / 32>(v1);
    if (!publish_partials<1>(v1, part, &st->cntA)) return;
    double tot[1];
    reduce_partials<1, BT / 32>(part, tot);
    if (tid == 0) {
      double pq = tot[0];
      st->pq = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = 2;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = st->rho / pq;
      }
      st->cntA = 0;
    }
  } else {
    double v3[3] = {acc[0], acc[1], acc[2]};
    block_sum<3, BT / 32>(v3);
    if (!publish_partials<3>(v3, part, &st->cntR)) return;
    double tot[3];
    reduce_partials<3, BT / 32>(part, tot);
    if (tid == 0) {
      const double rr = tot[0], bb = tot[2];
      st->rr0 = rr;
      st->bb0 = bb;
      st->rr = rr;
      st->rho = tot[1];
      st->beta = 0.0;
      int conv = rr <= st->tol0 * st->tol0 * bb || bb == 0.0;
      if (mode == MODE_OUTER) {
        // correction solve Q d = r to a relative reduction eta that lands
        // the next true residual near half the requested tolerance
        st->bb = rr;
        double eta = conv ? 0.5 : 0.5 * st->tol0 * sqrt(bb / rr);
        eta = fmin(fmax(eta, 1e-5), 0.5);
        st->tol2 = eta * eta;
      } else {
        st->bb = bb;
        st->tol2 = st->tol0 * st->tol0;
      }
      if (conv) st->status = 0;
      else if (st->iter >= st->max_iter) st->status = 1;
      st->done = conv || st->iter >= st->max_iter || st->status == 2;
      st->cntR = 0;
      st->guard = 0;
    }
  }
}

constexpr int UT = 256;

template <class T>
__global__ void __launch_bounds__(UT) k_update(int N, const float* __restrict__ qd, T* __restrict__ x,
                                               const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ r,
                                               double* part, PcgState* st, cudaGraphConditionalHandle handle) {
  if (st->done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    return;
  }
  const T alpha = (T)st->alpha;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * UT + threadIdx.x; i < N; i += gridDim.x * UT) {
    T pi = p[i], qi = q[i];
    x[i] += alpha * pi;
    T ri = r[i] - alpha * qi;
    r[i] = ri;
    double rd = (double)ri;
    rr += rd * rd;
    rz += rd * rd / (double)__ldg(qd + i);
  }
  double v[2] = {rz, rr};
  block_sum<2, UT / 32>(v);
  if (!publish_partials<2>(v, part, &st->cntB)) return;
  double tot[2];
  reduce_partials<2, UT / 32>(part, tot);
  if (threadIdx.x == 0) {
    double rho_new = tot[0];
    st->iter += 1;
    st->rr = tot[1];
    if (!isfinite(rho_new) || !isfinite(tot[1])) {
      st->status = 2;
      st->done = 1;
    } else if (tot[1] <= st->tol2 * st->bb) {
      st->status = 0;
      st->done = 1;
    } else if (st->iter >= st->max_iter) {
      st->status = 1;
      st->done = 1;
    }
    st->beta = rho_new / st->rho;
    st->rho = rho_new;
    st->cntB = 0;
    if (st->done) cudaGraphSetConditional(handle, 0);
  }
}

template <class T>
__global__ void k_cast_out(int N, const T* __restrict__ x, float* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = (float)x[i];
}

template <class T>
__global__ void k_cast_in(int N, const float* __restrict__ x, T* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = (T)x[i];
}

__global__ void k_axpy64(int N, const float* __restrict__ d, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) x[i] += (double)d[i];
}

__global__ void k_state_init(PcgState* st, double tol, int max_iter) {
  st->tol0 = tol;
  st->tol2 = tol * tol;
  st->max_iter = max_iter;
  st->iter = 0;
  st->status = 0;
  st->done = 0;
  st->beta = 0.0;
  st->cntA = st->cntB = st->cntR = 0;
  st->guard = 0;
  st->nexec = 0;
}

}  // namespace

struct SolveGraph {
  bool fp64 = false;
  int64_t N = 0;
  void *x = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
  double* x64 = nullptr;  // FP64 master iterate (FP32 mode)
  double* part = nullptr;
  PcgState* st = nullptr;
  PcgState* h_st = nullptr;
  int nblkB = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

void solve_graph_free(SolveGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  cudaFree(g->x);
  cudaFree(g->x64);
  cudaFree(g->r);
  cudaFree(g->p0);
  cudaFree(g->p1);
  cudaFree(g->q);
  cudaFree(g->part);
  cudaFree(g->st);
  if (g->h_st) cudaFreeHost(g->h_st);
  delete g;
}

template <class T>
static void launch_A(const BandView& bv, const bf_band* b, SolveGraph* g, const T* pin, T* pout, cudaStream_t s,
                     cudaGraphConditionalHandle h) {
  k_brick<T, MODE_PCG, T><<<b->NB, BT, 0, s>>>(bv, (float)b->prm.lambda, b->qd, pin, (const T*)g->r, pout, (T*)g->q,
                                            nullptr, g->part, g->st, h);
}

template <class T>
static void launch_B(const bf_band* b, SolveGraph* g, const T* p, cudaStream_t s, cudaGraphConditionalHandle h) {
  k_update<T><<<g->nblkB, UT, 0, s>>>((int)b->N, b->qd, (T*)g->x, p, (const T*)g->q, (T*)g->r, g->part, g->st, h);
}

template <class T>
static void launch_R(const BandView& bv, const bf_band* b, SolveGraph* g, cudaStream_t s) {
  // FP64 solver: r = b - Q x (written to g->r), p0 = 0
  k_brick<T, MODE_RESID, T><<<b->NB, BT, 0, s>>>(bv, (float)b->prm.lambda, b->qd, (const T*)g->x, nullptr, (T*)g->p0,
                                              (T*)g->r, b->rhs, g->part, g->st, cudaGraphConditionalHandle()); count_launch();
}

static void launch_outer(const BandView& bv, const bf_band* b, SolveGraph* g, cudaStream_t s) {
  // FP32 solver: r = b - Q x64 in FP64, stored as the FP32 correction rhs
  k_brick<double, MODE_OUTER, float><<<b->NB, BT, 0, s>>>(bv, (float)b->prm.lambda, b->qd, g->x64, nullptr,
                                                           (float*)g->p0, (float*)g->r, b->rhs, g->part, g->st,
                                                           cudaGraphConditionalHandle()); count_launch();
}

template <class T>
static bf_status build_graph(bf_ctx* ctx, bf_band* b, SolveGraph* g) {
  BandView bv = band_view(b);
  BF_CK(cudaGraphCreate(&g->graph, 0));
  cudaGraphConditionalHandle h;
  BF_CK(cudaGraphConditionalHandleCreate(&h, g->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BF_CK(cudaGraphAddNode(&node, g->graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  BF_CK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  BF_CK(cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  launch_A<T>(bv, b, g, (const T*)g->p0, (T*)g->p1, g->cap, h);
  launch_B<T>(b, g, (const T*)g->p1, g->cap, h);
  launch_A<T>(bv, b, g, (const T*)g->p1, (T*)g->p0, g->cap, h);
  launch_B<T>(b, g, (const T*)g->p0, g->cap, h);
  cudaGraph_t out_body;
  cudaError_t e = cudaStreamEndCapture(g->cap, &out_body);
  if (e != cudaSuccess) return bf_fail(ctx, BF_ECUDA, "capture PCG body", cudaGetErrorString(e));
  BF_CK(cudaGraphInstantiate(&g->exec, g->graph, 0));
  return BF_OK;
}

template <class T>
static bf_status get_graph(bf_ctx* ctx, bf_band* b, SolveGraph** out) {
  bool fp64 = sizeof(T) == 8;
  SolveGraph* g = b->sg;
  if (g && (g->fp64 != fp64 || g->N != b->N)) {
    cudaStreamSynchronize(ctx->stream);
    solve_graph_free(g);
    g = b->sg = nullptr;
  }
  if (!g) {
    g = new SolveGraph();
    b->sg = g;
    g->fp64 = fp64;
    g->N = b->N;
    size_t nb = (size_t)(b->N ? b->N : 1) * sizeof(T);
    BF_CK(cudaMalloc(&g->x, nb));
    BF_CK(cudaMalloc(&g->r, nb));
    BF_CK(cudaMalloc(&g->p0, nb));
    BF_CK(cudaMalloc(&g->p1, nb));
    BF_CK(cudaMalloc(&g->q, nb));
    if (!fp64) BF_CK(cudaMalloc(&g->x64, (size_t)(b->N ? b->N : 1) * sizeof(double)));
    int64_t nblk = (b->N + UT * 4 - 1) / (UT * 4);
    if (nblk > 152 * 8) nblk = 152 * 8;
    if (nblk < 1) nblk = 1;
    g->nblkB = (int)nblk;
    size_t np = (size_t)3 * (b->NB > nblk ? b->NB : nblk);
    BF_CK(cudaMalloc(&g->part, np * sizeof(double)));
    BF_CK(cudaMalloc(&g->st, sizeof(PcgState)));
    BF_CK(cudaMallocHost(&g->h_st, sizeof(PcgState)));
    BF_TRY(build_graph<T>(ctx, b, g));
  }
  *out = g;
  return BF_OK;
}

// FP64 mode: FP64 PCG with true-residual restarts.  FP32 mode: iterative
// refinement -- FP64 master iterate x64, FP64 true residual r = h - Q x64,
// FP32 PCG on Q d = r to a relative reduction eta, x64 += d, until the true
// residual meets the tolerance or the iteration budget is spent.
template <class T>
static bf_status solve_t(bf_ctx* ctx, bf_band* b, double tol, int max_iter, unsigned flags, float* mu, int* iters,
                         double* relres) {
  cudaStream_t s = ctx->stream;
  SolveGraph* g = nullptr;
  BF_TRY(get_graph<T>(ctx, b, &g));
  const bool fp64 = sizeof(T) == 8;
  BandView bv = band_view(b);
  const int N = (int)b->N;
  unsigned gx = (unsigned)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
  if (gx < 1) gx = 1;
  double* xm = fp64 ? (double*)g->x : g->x64;
  if (flags & BF_SOLVE_WARM) {
    k_cast_in<double><<<gx, 256, 0, s>>>(N, mu, xm);
    count_launch();
  } else BF_CK(cudaMemsetAsync(xm, 0, (size_t)N * sizeof(double), s));
  k_state_init<<<1, 1, 0, s>>>(g->st, tol, max_iter); count_launch();
  if (fp64) launch_R<T>(bv, b, g, s);
  else launch_outer(bv, b, g, s);
  BF_CK(cudaGetLastError());
  bool done = false;
  for (int outer = 0; outer < 64; ++outer) {
    BF_CK(cudaMemcpyAsync(g->h_st, g->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    BF_CK(cudaStreamSynchronize(s));
    if (g->h_st->done) {
      done = true;
      break;
    }
    if (!fp64) BF_CK(cudaMemsetAsync(g->x, 0, (size_t)N * sizeof(float), s));
    BF_CK(cudaGraphLaunch(g->exec, s));
    if (fp64) {
      launch_R<T>(bv, b, g, s);
    } else {
      k_axpy64<<<gx, 256, 0, s>>>(N, (const float*)g->x, g->x64); count_launch();
      launch_outer(bv, b, g, s);
    }
    BF_CK(cudaGetLastError());
  }
  k_cast_out<double><<<gx, 256, 0, s>>>(N, xm, mu); count_launch();
  BF_CK(cudaGetLastError());
  const PcgState& h = *g->h_st;
  count_launch(h.nexec);
  if (iters) *iters = h.iter;
  if (relres) *relres = h.bb0 > 0 ? sqrt(h.rr0 / h.bb0) : 0.0;
  if (h.status == 2) return bf_fail(ctx, BF_BREAKDOWN, "PCG breakdown (p.Qp <= 0 or non-finite)");
  if (!done || h.status == 1) return bf_fail(ctx, BF_NOT_CONVERGED, "PCG iteration limit reached");
  return BF_OK;
}

bf_status solve_mean_impl(bf_ctx* ctx, bf_band* b, double tol, int max_iter, unsigned flags, float* mu, int* iters,
                          double* relres) {
  if (b->N == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return BF_OK;
  }
  if (flags & BF_SOLVE_FP64) return solve_t<double>(ctx, b, tol, max_iter, flags, mu, iters, relres);
  return solve_t<float>(ctx, b, tol, max_iter, flags, mu, iters, relres);
}

bf_status spmv_launch(bf_ctx* ctx, const bf_band* b, const float* x, float* y) {
  if (b->N == 0) return BF_OK;
  k_brick<float, MODE_PLAIN, float><<<b->NB, BT, 0, ctx->stream>>>(band_view(b), (float)b->prm.lambda, b->qd, x, nullptr,
                                                           nullptr, y, nullptr, nullptr, nullptr,
                                                           cudaGraphConditionalHandle()); count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}
