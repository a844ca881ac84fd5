// Probe estimate of diag(Q^-1) (Sec. 3.7 diag equation; Algorithm 1 step 6)
// with the K probe solves batched as block PCG over R right-hand sides.
//
// Layout: block vectors are [N][R] float (row = one band voxel, R columns
// contiguous), the probes Z are [N][R] bf16 (+-1 is exact in bf16).  Each
// column is an independent Jacobi-PCG with its own alpha, beta and stop
// flag; converged columns are frozen (alpha = 0).  Per iteration:
//   A  k_blk_spmv: per brick (CTA-strided), per 4-column chunk: p <- r/qd +
//      beta p staged with the halo in a 10^3 float4 shared tile, q = Q p,
//      partial p.q per column; the last CTA sets alpha per column.
//   B  k_blk_update: x += alpha p, r -= alpha q, partial r.(r/qd), r.r per
//      column; the last CTA sets beta, stop flags and the iteration count.
// The loop runs as a CUDA-graph WHILE node as in the single-RHS solver.
// After convergence the true residual (FP64 accumulation) is recomputed per
// column and the columns that miss restart; then s += z (.) x.
#include "internal.cuh"

#include <cuda_bf16.h>

namespace {

constexpr int MAXR = 32;
constexpr int BT = 128;
constexpr int UT = 256;

struct BlkState {
  double rho[MAXR], pq[MAXR], alpha[MAXR], beta[MAXR], rr[MAXR], bb[MAXR], tol2[MAXR];  // inner PCG per column
  double rr0[MAXR], bb0[MAXR];  // true residual and |z|^2 per column
  int done[MAXR], iters[MAXR];
  double tol0;
  int iter, max_iter, all_done, status, ncols;
  unsigned int cntA, cntB, cntR, guard;
  unsigned int nexec;  // graph-body kernels executed (for launch accounting)
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 operator+(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 operator-(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 operator*(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }

// sum over the threads of a CTA that share (threadIdx.x % G), per component;
// result in out[g][k] (shared), valid after the call
template <int NV, int NW>
__device__ __forceinline__ void group_sum(double (&v)[NV], int G, double (*out)[NV]) {
  __shared__ double sh[NW][8][NV];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o >= G; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  if (lane < G) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[w][lane][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < G) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0;
      for (int q = 0; q < NW; ++q) s += sh[q][threadIdx.x][k];
      out[threadIdx.x][k] = s;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// fixed-order sum of part[k][c][0..nblk) for all c < R, k < NV, into tot[k][c]:
// one warp per (k, c), lanes strided over the partials, xor-shuffle tree
template <int NV>
__device__ __forceinline__ void sum_partials(const double* part, int R, int nblk, double (*tot)[MAXR]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int kc = w; kc < NV * R; kc += nw) {
    const double* p = part + (size_t)kc * nblk;
    double s = 0;
    for (int i = lane; i < nblk; i += 32) s += __ldcg(p + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) tot[kc / R][kc % R] = s;
  }
  __syncthreads();
}

// halo slot q in [0, 384): face q/64, (u, v) = (q & 7, (q >> 3) & 7) over the
// face's other two axes; returns the neighbour's compact index (or -1) and
// the position in the 10^3 tile
__device__ __forceinline__ void halo_slot(const MetaWord (*sm)[16], int q, int* hidx, int* htile) {
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
  *hidx = (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
  *htile = tc[0] + 10 * tc[1] + 100 * tc[2];
}

// One CTA per brick (CTA-strided), 4 columns per pass through a float4 tile:
// p <- r/qd + beta p (own voxels and halo), q = Q p, partial p.q per column.
template <int R>
__global__ void __launch_bounds__(BT) k_blk_spmv(BandView B, float lam, const float* __restrict__ qd,
                                                 const float* __restrict__ pin, const float* __restrict__ rin,
                                                 float* __restrict__ pout, float* __restrict__ yout, double* part,
                                                 BlkState* st, cudaGraphConditionalHandle handle) {
  constexpr int NCH = R / 4;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->nexec += 2;  // this kernel and the update that follows it
    unsigned g = atomicAdd(&st->guard, 1u);
    if (st->all_done || g > 2u * (unsigned)st->max_iter + 64u) {
      if (!st->all_done) { st->status = 1; st->all_done = 1; }
      cudaGraphSetConditional(handle, 0);
    }
  }
  if (st->all_done) return;
  __shared__ float4 tile[1000];
  __shared__ MetaWord sm[7][16];
  __shared__ float hq[384];
  __shared__ float sbeta[R];
  __shared__ double red[4][4];
  const int tid = threadIdx.x;
  if (tid < R) sbeta[tid] = (float)st->beta[tid];
  double acc[NCH][4];
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[ch][k] = 0.0;

  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
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
    int idx[4], hidx[3], htile[3];
    float qv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = tid + BT * s;
      MetaWord m = sm[0][l >> 5];
      uint32_t bit = 1u << (l & 31);
      idx[s] = (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
      qv[s] = idx[s] >= 0 ? __ldg(qd + idx[s]) : 1.0f;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int q = tid + BT * s;
      halo_slot(sm, q, &hidx[s], &htile[s]);
      hq[q] = hidx[s] >= 0 ? __ldg(qd + hidx[s]) : 1.0f;
    }
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      const float4 bet = make_float4(sbeta[4 * ch], sbeta[4 * ch + 1], sbeta[4 * ch + 2], sbeta[4 * ch + 3]);
      float4 val[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        float4 v = f4(0.0f);
        if (idx[s] >= 0) {
          const size_t o = (size_t)idx[s] * R + 4 * ch;
          float4 rr = __ldg((const float4*)(rin + o));
          float4 pp = __ldg((const float4*)(pin + o));
          v = rr * f4(1.0f / qv[s]) + bet * pp;
        }
        val[s] = v;
        int l = tid + BT * s;
        tile[(l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1)] = v;
      }
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        float4 v = f4(0.0f);
        if (hidx[s] >= 0) {
          const size_t o = (size_t)hidx[s] * R + 4 * ch;
          float4 rr = __ldg((const float4*)(rin + o));
          float4 pp = __ldg((const float4*)(pin + o));
          v = rr * f4(1.0f / hq[tid + BT * s]) + bet * pp;
        }
        tile[htile[s]] = v;
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (idx[s] < 0) continue;
        int l = tid + BT * s;
        int c = (l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1);
        const size_t o = (size_t)idx[s] * R + 4 * ch;
        float4 ns = ((tile[c - 1] + tile[c + 1]) + (tile[c - 10] + tile[c + 10])) + (tile[c - 100] + tile[c + 100]);
        float4 y = f4(qv[s]) * tile[c] - f4(lam) * ns;
        *(float4*)(yout + o) = y;
        *(float4*)(pout + o) = val[s];
        acc[ch][0] += (double)val[s].x * y.x;
        acc[ch][1] += (double)val[s].y * y.y;
        acc[ch][2] += (double)val[s].z * y.z;
        acc[ch][3] += (double)val[s].w * y.w;
      }
      __syncthreads();
    }
  }
  const int nblk = gridDim.x;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = acc[ch][k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((tid & 31) == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[tid >> 5][k] = v[k];
    }
    __syncthreads();
    if (tid < 4) part[(size_t)(4 * ch + tid) * nblk + blockIdx.x] = red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
    __syncthreads();
  }
  if (!arrive_last(&st->cntA)) return;
  __shared__ double tot[3][MAXR];
  sum_partials<1>(part, R, nblk, tot);
  if (tid < R) {
    int c = tid;
    double pq = tot[0][c];
    st->pq[c] = pq;
    if (st->done[c]) {
      st->alpha[c] = 0.0;
    } else if (!(pq > 0.0) || !isfinite(pq)) {
      st->alpha[c] = 0.0;
      st->done[c] = 1;
      st->status = 2;
    } else {
      st->alpha[c] = st->rho[c] / pq;
    }
  }
  __syncthreads();
  if (tid == 0) st->cntA = 0;
}

struct D4 {
  double v[4];
};

// True residual of the FP64 master iterate, per column: r = z - Q x64
// (FP64), stored as the FP32 right-hand side of the next correction solve;
// p = 0; per-column r.r, r.(r/qd), z.z.  The last CTA sets up the inner
// solve: rhs norm, rho, per-column relative target eta, stop flags.
template <int R>
__global__ void __launch_bounds__(BT) k_blk_outer(BandView B, float lam, const float* __restrict__ qd,
                                                  const double* __restrict__ x64, float* __restrict__ rout,
                                                  float* __restrict__ pout, const __nv_bfloat16* __restrict__ Z,
                                                  double* part, BlkState* st) {
  constexpr int NCH = R / 4;
  __shared__ D4 tile[1000];
  __shared__ MetaWord sm[7][16];
  __shared__ double red[4][12];
  const int tid = threadIdx.x;
  double acc[3][NCH][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[a][ch][k] = 0.0;
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
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
    int idx[4], hidx[3], htile[3];
    float qv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = tid + BT * s;
      MetaWord m = sm[0][l >> 5];
      uint32_t bit = 1u << (l & 31);
      idx[s] = (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
      qv[s] = idx[s] >= 0 ? __ldg(qd + idx[s]) : 1.0f;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) halo_slot(sm, tid + BT * s, &hidx[s], &htile[s]);
    for (int ch = 0; ch < NCH; ++ch) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        D4 v = {{0.0, 0.0, 0.0, 0.0}};
        if (idx[s] >= 0) {
          const double* src = x64 + (size_t)idx[s] * R + 4 * ch;
#pragma unroll
          for (int k = 0; k < 4; ++k) v.v[k] = src[k];
        }
        int l = tid + BT * s;
        tile[(l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1)] = v;
      }
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        D4 v = {{0.0, 0.0, 0.0, 0.0}};
        if (hidx[s] >= 0) {
          const double* src = x64 + (size_t)hidx[s] * R + 4 * ch;
#pragma unroll
          for (int k = 0; k < 4; ++k) v.v[k] = src[k];
        }
        tile[htile[s]] = v;
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (idx[s] < 0) continue;
        int l = tid + BT * s;
        int c = (l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1);
        const size_t o = (size_t)idx[s] * R + 4 * ch;
        float rc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          double ns = ((tile[c - 1].v[k] + tile[c + 1].v[k]) + (tile[c - 10].v[k] + tile[c + 10].v[k])) +
                      (tile[c - 100].v[k] + tile[c + 100].v[k]);
          double zb = (double)__bfloat162float(Z[o + k]);
          double r = zb - ((double)qv[s] * tile[c].v[k] - (double)lam * ns);
          rc[k] = (float)r;
          acc[0][ch][k] += r * r;
          acc[1][ch][k] += r * r / (double)qv[s];
          acc[2][ch][k] += zb * zb;
        }
        *(float4*)(rout + o) = make_float4(rc[0], rc[1], rc[2], rc[3]);
        *(float4*)(pout + o) = f4(0.0f);
      }
      __syncthreads();
    }
  }
  const int nblk = gridDim.x;
  for (int ch = 0; ch < NCH; ++ch) {
    double v[12];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double x = acc[a][ch][k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        v[4 * a + k] = x;
      }
    if ((tid & 31) == 0) {
#pragma unroll
      for (int q = 0; q < 12; ++q) red[tid >> 5][q] = v[q];
    }
    __syncthreads();
    if (tid < 12) {
      int a = tid >> 2, k = tid & 3;
      part[((size_t)a * R + 4 * ch + k) * nblk + blockIdx.x] = red[0][tid] + red[1][tid] + red[2][tid] + red[3][tid];
    }
    __syncthreads();
  }
  if (!arrive_last(&st->cntR)) return;
  __shared__ double tot[3][MAXR];
  sum_partials<3>(part, R, nblk, tot);
  if (tid < R) {
    int c = tid;
    const double rr = tot[0][c], bb = tot[2][c];
    st->rr0[c] = rr;
    st->bb0[c] = bb;
    st->rr[c] = rr;
    st->bb[c] = rr;
    st->rho[c] = tot[1][c];
    st->beta[c] = 0.0;
    st->alpha[c] = 0.0;
    const int conv = (c >= st->ncols) || rr <= st->tol0 * st->tol0 * bb || bb == 0.0;
    double eta = conv ? 0.5 : 0.5 * st->tol0 * sqrt(bb / rr);
    eta = fmin(fmax(eta, 1e-5), 0.5);
    st->tol2[c] = eta * eta;
    st->done[c] = conv;
  }
  __syncthreads();
  if (tid == 0) {
    int all = 1;
    for (int c = 0; c < R; ++c) all &= st->done[c];
    if (all && st->status != 2) st->status = 0;
    if (!all && st->iter >= st->max_iter) st->status = 1;
    st->all_done = all || st->iter >= st->max_iter || st->status == 2;
    st->cntR = 0;
    st->guard = 0;
  }
}

template <int R>
__global__ void __launch_bounds__(UT) k_blk_update(int N, const float* __restrict__ qd, float* __restrict__ x,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   float* __restrict__ r, double* part, BlkState* st,
                                                   cudaGraphConditionalHandle handle) {
  constexpr int G = R / 4;
  if (st->all_done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    return;
  }
  const int g = threadIdx.x % G;
  const float4 al = make_float4((float)st->alpha[4 * g], (float)st->alpha[4 * g + 1], (float)st->alpha[4 * g + 2],
                                (float)st->alpha[4 * g + 3]);
  double rz[4] = {0, 0, 0, 0}, rr[4] = {0, 0, 0, 0};
  const int64_t n4 = (int64_t)N * G;
  for (int64_t e = (int64_t)blockIdx.x * UT + threadIdx.x; e < n4; e += (int64_t)gridDim.x * UT) {
    int64_t i = e / G;
    float4 pi = ((const float4*)p)[e], qi = ((const float4*)q)[e];
    float4 xi = ((float4*)x)[e], ri = ((float4*)r)[e];
    xi = xi + al * pi;
    ri = ri - al * qi;
    ((float4*)x)[e] = xi;
    ((float4*)r)[e] = ri;
    double iq = 1.0 / (double)__ldg(qd + i);
    double a0 = ri.x, a1 = ri.y, a2 = ri.z, a3 = ri.w;
    rr[0] += a0 * a0; rr[1] += a1 * a1; rr[2] += a2 * a2; rr[3] += a3 * a3;
    rz[0] += a0 * a0 * iq; rz[1] += a1 * a1 * iq; rz[2] += a2 * a2 * iq; rz[3] += a3 * a3 * iq;
  }
  __shared__ double gs[8][8];
  double v[8] = {rz[0], rz[1], rz[2], rz[3], rr[0], rr[1], rr[2], rr[3]};
  group_sum<8, UT / 32>(v, G, gs);
  const int nblk = gridDim.x;
  if (threadIdx.x < G) {
    for (int k = 0; k < 4; ++k) {
      part[((size_t)0 * R + 4 * threadIdx.x + k) * nblk + blockIdx.x] = gs[threadIdx.x][k];
      part[((size_t)1 * R + 4 * threadIdx.x + k) * nblk + blockIdx.x] = gs[threadIdx.x][4 + k];
    }
  }
  if (!arrive_last(&st->cntB)) return;
  __shared__ double tot[3][MAXR];
  sum_partials<2>(part, R, nblk, tot);
  __shared__ int any_live;
  if (threadIdx.x == 0) {
    any_live = 0;
    st->iter += 1;
  }
  __syncthreads();
  if (threadIdx.x < R) {
    int c = threadIdx.x;
    if (!st->done[c]) {
      double rho_new = tot[0][c];
      st->rr[c] = tot[1][c];
      st->iters[c] += 1;
      if (!isfinite(rho_new) || !isfinite(tot[1][c])) {
        st->done[c] = 1;
        st->status = 2;
      } else if (tot[1][c] <= st->tol2[c] * st->bb[c]) {
        st->done[c] = 1;
      } else {
        st->beta[c] = rho_new / st->rho[c];
        st->rho[c] = rho_new;
        atomicOr(&any_live, 1);
      }
    }
    if (st->done[c]) st->beta[c] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!any_live || st->iter >= st->max_iter) {
      st->all_done = 1;
      cudaGraphSetConditional(handle, 0);
    }
    st->cntB = 0;
  }
}

// Z[i][c] = Rademacher(seed, k0 + c, lin_i) for c < ncols, 0 beyond; x = 0
template <int R>
__global__ void k_probes(int N, const int32_t* __restrict__ lin, uint64_t mseed, int k0, int ncols,
                         __nv_bfloat16* __restrict__ Z, double* __restrict__ x) {
  const int64_t n = (int64_t)N * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / R;
    int c = (int)(e - i * R);
    float z = 0.0f;
    if (c < ncols) {
      uint64_t v = mix64(mseed ^ ((uint64_t)(k0 + c) * 0xD1B54A32D192ED03ULL) ^ (uint64_t)(uint32_t)lin[i]);
      z = (v >> 63) ? -1.0f : 1.0f;
    }
    Z[e] = __float2bfloat16(z);
    x[e] = 0.0;
  }
}

// s_acc[i] += sum_c z[i][c] x[i][c]
template <int R>
__global__ void k_hutch(int N, const __nv_bfloat16* __restrict__ Z, const double* __restrict__ x,
                        double* __restrict__ sacc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < R; ++c) s += (double)__bfloat162float(Z[(size_t)i * R + c]) * x[(size_t)i * R + c];
    sacc[i] += s;
  }
}

__global__ void k_finish(int N, const double* __restrict__ sacc, double invK, float* __restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) s[i] = (float)(sacc[i] * invK);
}

__global__ void k_axpy64(int64_t n, const float* __restrict__ d, double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

__global__ void k_blk_init(BlkState* st, double tol, int max_iter, int ncols) {
  int c = threadIdx.x;
  if (c < MAXR) {
    st->done[c] = 0;
    st->iters[c] = 0;
    st->beta[c] = 0.0;
    st->alpha[c] = 0.0;
  }
  if (c == 0) {
    st->tol0 = tol;
    st->max_iter = max_iter;
    st->iter = 0;
    st->all_done = 0;
    st->status = 0;
    st->ncols = ncols;
    st->cntA = st->cntB = st->cntR = 0;
    st->guard = 0;
    st->nexec = 0;
  }
}

unsigned grid_for(int64_t n, int threads, int64_t cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

struct BlockGraph {
  int R = 0;
  int64_t N = 0;
  float *x = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;  // FP32 correction solve
  double* x64 = nullptr;                                                        // FP64 master iterates
  __nv_bfloat16* Z = nullptr;
  double* sacc = nullptr;
  double* part = nullptr;
  BlkState* st = nullptr;
  BlkState* h_st = nullptr;
  int nblkA = 0, nblkB = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

void block_graph_free(BlockGraph* g) {
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
  cudaFree(g->Z);
  cudaFree(g->sacc);
  cudaFree(g->part);
  cudaFree(g->st);
  if (g->h_st) cudaFreeHost(g->h_st);
  delete g;
}

template <int R>
static void blk_A(const BandView& bv, const bf_band* b, BlockGraph* g, const float* pin, float* pout, cudaStream_t s,
                  cudaGraphConditionalHandle h) {
  k_blk_spmv<R><<<g->nblkA, BT, 0, s>>>(bv, (float)b->prm.lambda, b->qd, pin, g->r, pout, g->q, g->part, g->st, h);
}

template <int R>
static void blk_B(const bf_band* b, BlockGraph* g, const float* p, cudaStream_t s, cudaGraphConditionalHandle h) {
  k_blk_update<R><<<g->nblkB, UT, 0, s>>>((int)b->N, b->qd, g->x, p, g->q, g->r, g->part, g->st, h);
}

template <int R>
static void blk_outer(const BandView& bv, const bf_band* b, BlockGraph* g, cudaStream_t s) {
  k_blk_outer<R><<<g->nblkA, BT, 0, s>>>(bv, (float)b->prm.lambda, b->qd, g->x64, g->r, g->p0, g->Z, g->part, g->st); count_launch();
}

template <int R>
static bf_status get_block_graph(bf_ctx* ctx, bf_band* b, BlockGraph** out) {
  BlockGraph* g = b->bg;
  if (g && (g->R != R || g->N != b->N)) {
    cudaStreamSynchronize(ctx->stream);
    block_graph_free(g);
    g = b->bg = nullptr;
  }
  if (!g) {
    g = new BlockGraph();
    b->bg = g;
    g->R = R;
    g->N = b->N;
    size_t nv = (size_t)(b->N ? b->N : 1) * R;
    BF_CK(cudaMalloc(&g->x, nv * 4));
    BF_CK(cudaMalloc(&g->x64, nv * 8));
    BF_CK(cudaMalloc(&g->r, nv * 4));
    BF_CK(cudaMalloc(&g->p0, nv * 4));
    BF_CK(cudaMalloc(&g->p1, nv * 4));
    BF_CK(cudaMalloc(&g->q, nv * 4));
    BF_CK(cudaMalloc(&g->Z, nv * 2));
    BF_CK(cudaMalloc(&g->sacc, (size_t)(b->N ? b->N : 1) * 8));
    g->nblkA = (int)(b->NB < 152 * 8 ? b->NB : 152 * 8);
    if (g->nblkA < 1) g->nblkA = 1;
    g->nblkB = (int)grid_for((int64_t)b->N * (R / 4), UT * 4, 152 * 8);
    int np = g->nblkA > g->nblkB ? g->nblkA : g->nblkB;
    BF_CK(cudaMalloc(&g->part, (size_t)3 * R * np * sizeof(double)));
    BF_CK(cudaMalloc(&g->st, sizeof(BlkState)));
    BF_CK(cudaMallocHost(&g->h_st, sizeof(BlkState)));
    BandView bv = band_view(b);
    BF_CK(cudaGraphCreate(&g->graph, 0));
    cudaGraphConditionalHandle h;
    BF_CK(cudaGraphConditionalHandleCreate(&h, g->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np2 = {};
    np2.type = cudaGraphNodeTypeConditional;
    np2.conditional.handle = h;
    np2.conditional.type = cudaGraphCondTypeWhile;
    np2.conditional.size = 1;
    cudaGraphNode_t node;
    BF_CK(cudaGraphAddNode(&node, g->graph, nullptr, nullptr, 0, &np2));
    cudaGraph_t body = np2.conditional.phGraph_out[0];
    BF_CK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
    BF_CK(cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    blk_A<R>(bv, b, g, g->p0, g->p1, g->cap, h);
    blk_B<R>(b, g, g->p1, g->cap, h);
    blk_A<R>(bv, b, g, g->p1, g->p0, g->cap, h);
    blk_B<R>(b, g, g->p0, g->cap, h);
    cudaGraph_t ob;
    cudaError_t e = cudaStreamEndCapture(g->cap, &ob);
    if (e != cudaSuccess) return bf_fail(ctx, BF_ECUDA, "capture block PCG body", cudaGetErrorString(e));
    BF_CK(cudaGraphInstantiate(&g->exec, g->graph, 0));
  }
  *out = g;
  return BF_OK;
}

template <int R>
static bf_status variance_t(bf_ctx* ctx, bf_band* b, int K, uint64_t seed, double tol, int max_iter, float* s_out,
                            int* total_iters) {
  cudaStream_t s = ctx->stream;
  BlockGraph* g = nullptr;
  BF_TRY(get_block_graph<R>(ctx, b, &g));
  BandView bv = band_view(b);
  const int N = (int)b->N;
  BF_CK(cudaMemsetAsync(g->sacc, 0, (size_t)N * 8, s));
  uint64_t mseed = 0;
  {  // host copy of the probe seed mix (same function as the device)
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    mseed = z ^ (z >> 31);
  }
  int tot_it = 0;
  bf_status result = BF_OK;
  const int64_t NR = (int64_t)N * R;
  const unsigned gNR = grid_for(NR, 256, 152 * 32);
  for (int k0 = 0; k0 < K; k0 += R) {
    // one block of R probes: FP64 master iterates, FP32 correction solves
    int ncols = K - k0 < R ? K - k0 : R;
    k_probes<R><<<gNR, 256, 0, s>>>(N, b->lin, mseed, k0, ncols, g->Z, g->x64); count_launch();
    k_blk_init<<<1, MAXR, 0, s>>>(g->st, tol, max_iter, ncols); count_launch();
    blk_outer<R>(bv, b, g, s);
    BF_CK(cudaGetLastError());
    bool done = false;
    for (int outer = 0; outer < 64; ++outer) {
      BF_CK(cudaMemcpyAsync(g->h_st, g->st, sizeof(BlkState), cudaMemcpyDeviceToHost, s));
      BF_CK(cudaStreamSynchronize(s));
      if (g->h_st->all_done) {
        done = true;
        break;
      }
      BF_CK(cudaMemsetAsync(g->x, 0, (size_t)NR * 4, s));
      BF_CK(cudaGraphLaunch(g->exec, s));
      k_axpy64<<<gNR, 256, 0, s>>>(NR, g->x, g->x64); count_launch();
      blk_outer<R>(bv, b, g, s);
      BF_CK(cudaGetLastError());
    }
    const BlkState& h = *g->h_st;
    count_launch(h.nexec);
    for (int c = 0; c < ncols; ++c) tot_it += h.iters[c];
    k_hutch<R><<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, g->Z, g->x64, g->sacc); count_launch();
    BF_CK(cudaGetLastError());
    if (h.status == 2) { result = BF_BREAKDOWN; break; }
    if (!done || h.status == 1) { result = BF_NOT_CONVERGED; break; }
  }
  k_finish<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, g->sacc, 1.0 / K, s_out); count_launch();
  BF_CK(cudaGetLastError());
  if (total_iters) *total_iters = tot_it;
  if (result == BF_BREAKDOWN) return bf_fail(ctx, BF_BREAKDOWN, "block PCG breakdown");
  if (result == BF_NOT_CONVERGED) return bf_fail(ctx, BF_NOT_CONVERGED, "block PCG iteration limit reached");
  return BF_OK;
}

namespace {
__global__ void k_bench_state(BlkState* st) {
  int c = threadIdx.x;
  if (c < MAXR) {
    st->done[c] = 0;
    st->beta[c] = 0.5;
    st->rho[c] = 1.0;
  }
  if (c == 0) {
    st->all_done = 0;
    st->max_iter = 1 << 28;
    st->guard = 0;
    st->cntA = 0;
  }
}

template <int R>
bf_status bench_blk_t(bf_ctx* ctx, bf_band* b, int reps, double* ms) {
  BlockGraph* g = nullptr;
  BF_TRY(get_block_graph<R>(ctx, b, &g));
  cudaStream_t s = ctx->stream;
  BandView bv = band_view(b);
  k_bench_state<<<1, MAXR, 0, s>>>(g->st); count_launch();
  cudaEvent_t e0, e1;
  BF_CK(cudaEventCreate(&e0));
  BF_CK(cudaEventCreate(&e1));
  BF_CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) {
    blk_A<R>(bv, b, g, (i & 1) ? g->p1 : g->p0, (i & 1) ? g->p0 : g->p1, s, cudaGraphConditionalHandle());
    count_launch();
  }
  BF_CK(cudaEventRecord(e1, s));
  BF_CK(cudaEventSynchronize(e1));
  float t = 0;
  BF_CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return BF_OK;
}
}  // namespace

bf_status bench_block_spmv(bf_ctx* ctx, bf_band* b, int R, int reps, double* ms) {
  switch (R) {
    case 8: return bench_blk_t<8>(ctx, b, reps, ms);
    case 16: return bench_blk_t<16>(ctx, b, reps, ms);
    case 32: return bench_blk_t<32>(ctx, b, reps, ms);
  }
  return bf_fail(ctx, BF_EINVAL, "R must be 8, 16 or 32");
}

bf_status variance_impl(bf_ctx* ctx, bf_band* b, int K, uint64_t seed, double tol, int max_iter, int R,
                        unsigned flags, float* s, int* total_iters) {
  (void)flags;
  if (b->N == 0) {
    if (total_iters) *total_iters = 0;
    return BF_OK;
  }
  if (R == 0) R = K >= 32 ? 32 : (K >= 16 ? 16 : 8);
  switch (R) {
    case 8: return variance_t<8>(ctx, b, K, seed, tol, max_iter, s, total_iters);
    case 16: return variance_t<16>(ctx, b, K, seed, tol, max_iter, s, total_iters);
    case 32: return variance_t<32>(ctx, b, K, seed, tol, max_iter, s, total_iters);
  }
  return bf_fail(ctx, BF_EINVAL, "rhs_block must be 0, 8, 16 or 32");
}
