// Probe estimate of diag(Q^-1) (Sec. 3.7 diag equation; Algorithm 1 step 6)
// with the K probe solves batched as block PCG over R right-hand sides.
//
// Layout: block vectors are [N][R] float (one row per band voxel, the R
// probe columns contiguous, so a warp reads a row as one 128-byte line);
// probes Z are [N][R] bf16 (+-1 is exact in bf16).  Every column is an
// independent Jacobi-PCG with its own scalars and stop flag; converged
// columns are frozen (alpha = beta = 0).
//
// Iteration: the single-reduction form of PCG (Chronopoulos & Gear, 1989):
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//   u = r / qd,      w = Q u,        gamma = r.u,   delta = w.u,  r.r
// with s = Q p carried by recurrence, so Q is applied once per iteration, to
// u, and u = r / qd is never stored.  One pass per iteration (k_blk_it) over
// tiles of consecutive rows: the own rows' vectors are updated (streaming,
// float4 over 4 columns), u' of the own rows and of the rows outside the tile
// that its face neighbours reference (a per-band gather plan) goes to shared
// memory, and w' = Q u' is formed from there.  r, w, s are double-buffered,
// since other CTAs recompute u' of a row from its old r, w, s.
// Partial sums are FP32 products summed per thread, accumulated in FP64 from
// the CTA reduction on, reduced per CTA and then by the last CTA in a fixed
// order (deterministic), which updates per column
//   beta' = gamma'/gamma,  alpha' = gamma' / (delta' - beta' gamma'/alpha)
// and the stop flags.  The iteration loop is a CUDA-graph WHILE node.
//
// Refinement: master iterates xm per column in float-float arithmetic (an
// unevaluated sum hi + lo of two floats, about 48 significant bits: Dekker's
// exact product by FMA and Knuth's exact sum); k_blk_res adds the FP32
// correction x to xm and computes the true residual z - Q xm in that
// arithmetic, the FP32 solve reduces it by a factor eta, until every column
// meets the tolerance.  (FP64 would serve
// too, but its throughput on this GPU is a small fraction of FP32's.)
//
// The solver (workspaces, state, graph) belongs to the context, one per
// block width R: kernels read band pointers and sizes from a device-resident
// argument block, so the captured graph serves every band.
#include <climits>
#include <cstring>

#include "internal.cuh"

#include <cuda_bf16.h>

namespace {

constexpr int MAXR = 32;
constexpr int CT = 512;   // threads per CTA of the row kernels
// smallest relative residual reduction asked of one FP32 correction solve
// (the FP32 recursive residual keeps falling below the true one's floor)
constexpr double ETA_MIN = 1e-7;
// Resident CTAs per SM of the row kernels for R columns: one for R = 32
// (512 threads with up to 128 registers each keep all four own-row items of
// a thread in flight; measured 1.79 against 2.11 ms per iteration on the
// 7.2 M-voxel object band), two otherwise (R = 16: 1.01 against 1.07 ms).
template <int R>
__host__ __device__ constexpr int blk_occ() { return R >= 32 ? 1 : 2; }
template <int R>
__host__ __device__ constexpr int blk_ncta() { return 152 * blk_occ<R>(); }
// own-row items of the probe iteration in flight per thread
template <int R>
__host__ __device__ constexpr int blk_p1_unroll() { return R >= 32 ? 4 : 1; }
// a correction solve reduces its right-hand side to BLK_ETA tol |z| (measured on the object band:
// 0.5 takes 2408 iterations for 128 probes, 0.25 2554 and 0.1 2697, with no fewer residual passes)
constexpr double BLK_ETA = 0.5;
// resident CTAs per SM of the residual pass: two for every R (its float-float columns go in passes of 16; for
// R = 32 two CTAs took the 128-probe estimate on the object band from 154.6 to 149.3 ms against one)
template <int R>
__host__ __device__ constexpr int res_occ() { return 2; }
// float-float columns per pass of the residual pass (all 32 columns in one pass at one CTA per SM measured
// slower: 157.4 against 149.5 ms for the 128-probe estimate)
template <int R>
__host__ __device__ constexpr int res_cc() { return R < 16 ? R : 16; }
// CTA sums are reduced in two levels: NGRP groups of gridDim.x / NGRP CTAs (8 or 16), then the group sums
constexpr int NCTA_MAX = 152 * 2, NGRP = 19;
static_assert(NCTA_MAX % NGRP == 0 && 152 % NGRP == 0 && NCTA_MAX / NGRP <= 16, "reduction groups");
// SpMM pass: tiles of SP_TR rows plus at most SP_EMAX external rows staged in
// shared memory (SP_ROWS rows); SP_GLOBAL marks a neighbour read from global
// memory (a tile whose external rows overflow the list)
constexpr int SP_TR = 256, SP_EMAX = 384, SP_ROWS = SP_TR + SP_EMAX;
constexpr int16_t SP_GLOBAL = 32767;


struct BlkState {
  double alpha[MAXR], beta[MAXR], gamma[MAXR], rr[MAXR], bb[MAXR], tol2[MAXR];
  double rr0[MAXR], bb0[MAXR];  // true residual and |z|^2 per column
  int done[MAXR], iters[MAXR];
  double tol0;
  int iter, max_iter, all_done, status, ncols;
  int first;  // the next finalize starts a correction solve
  int par;    // which of the double-buffered r, w, s is current
  // The correction x is written every second iteration: x += alpha_{k-1} p_{k-1} + alpha_k p_k, with
  // p_{k-1} the direction the iteration reads anyway.  xvalid: x holds a value (else it is zero);
  // xpend: the last iteration's alpha p is not yet in x (aprev holds that alpha per column).
  alignas(16) float aprev[MAXR];
  int xvalid, xpend;
  int want_sq;  // the residual pass also forms the probe values' second moments (hsq)
  int xmpar;    // which of the double-buffered master iterates is current
  unsigned int cnt, guard;
  unsigned int gcnt[NGRP];  // CTAs of each reduction group that have written their partials
  unsigned int nexec;  // graph-body kernels executed (for launch accounting)
};

// Everything a kernel needs about the band and the workspaces.
struct BlkArgs {
  int N;
  float lam;
  const int32_t* nb6;  // [N][6] face-neighbour indices, -1 outside the band
  const int32_t* sp_ext;   // [tiles][SP_EMAX] sorted external rows of each SpMM tile
  const int32_t* sp_ne;    // [tiles] their count
  const int16_t* sp_slot;  // [N][8] staged slot of each face neighbour (6 used)
  const float* qd;     // [N] Q_jj
  float* iq;           // [N] 1 / Q_jj
  float* r[2];         // residual, double-buffered ([BlkState::par] is current)
  float* w[2];         // Q u
  float* s[2];         // Q p (by recurrence)
  float* p;
  float* x;            // FP32 correction
  float2* xm[2];       // float-float master iterates (hi, lo), double-buffered ([BlkState::xmpar] is current)
  const __nv_bfloat16* Z;
  double* part;        // [3][R][CTAs of the launch]
  double* part1;       // [3][R][CTAs of the launch] the iteration's partials (r'.u', r'.r', w'.u')
  double* gpart;       // [3][R][NGRP] group sums of the partials
  double* hsum;        // [N] sum over the block's columns of z (.) xm, from the last residual pass
  double* hsq;         // [N] the same for (z (.) xm)^2 (formed when BlkState::want_sq)
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) { return splitmix64(x); }

// float-float arithmetic: (hi, lo) with |lo| <= ulp(hi)/2
__device__ __forceinline__ float2 two_sum(float a, float b) {  // a + b = s + e exactly (Knuth)
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
  const float2 t = two_sum(x.x, y.x);
  return quick_two_sum(t.x, __fadd_rn(t.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 ff_add_f(float2 x, float b) {
  const float2 t = two_sum(x.x, b);
  return quick_two_sum(t.x, __fadd_rn(t.y, x.y));
}
__device__ __forceinline__ float2 ff_mul_f(float2 x, float b) {  // exact product of hi by FMA (Dekker)
  const float p = __fmul_rn(x.x, b);
  const float e = __fmaf_rn(x.y, b, __fmaf_rn(x.x, b, -p));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_neg(float2 x) { return make_float2(-x.x, -x.y); }

// Fixed-order two-level sum of the CTA partials part[k][c][0..gridDim.x) for all
// c < R, k < NV.  Called by every thread of every CTA after its partials are
// written.  The last CTA of each group of GSZ sums the group (a half-warp per
// (k, c), shuffle tree) into gpart[k][c][group]; the last group's finisher sums
// the NGRP group values (a warp per (k, c)) into tot[k][c] and returns true in
// all its threads; every other CTA returns false.  The counters are left at 0
// for the next launch except st->cnt, which the caller resets.
template <int NV>
__device__ __forceinline__ bool reduce_partials(const double* part, double* gpart, BlkState* st, int R,
                                                double (*tot)[MAXR]) {
  __shared__ bool s_last;
  const int GSZ = gridDim.x / NGRP, ncta = gridDim.x;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5, grp = blockIdx.x / GSZ;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&st->gcnt[grp], 1u) == GSZ - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  // group level: half-warp h takes (k, c) = kb + (h & 1) for kb = 2 * warp, 2 * warp + CT / 16, ...
  for (int kb = 2 * wrp; kb < NV * R; kb += CT / 16) {
    const int kc = kb + ((threadIdx.x >> 4) & 1);
    const bool on = kc < NV * R;
    double v = (on && (lane & 15) < GSZ) ? __ldcg(part + (size_t)kc * ncta + grp * GSZ + (lane & 15)) : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (on && (lane & 15) == 0) gpart[(size_t)kc * NGRP + grp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->gcnt[grp] = 0;
    __threadfence();
    s_last = atomicAdd(&st->cnt, 1u) == NGRP - 1;
  }
  __syncthreads();
  if (!s_last) return false;
  // last level: warp per (k, c), lanes over the group sums
  for (int kc = wrp; kc < NV * R; kc += CT / 32) {
    double v = lane < NGRP ? __ldcg(gpart + (size_t)kc * NGRP + lane) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) tot[kc / R][kc % R] = v;
  }
  __syncthreads();
  return true;
}


// One residual pass of the refinement, per tile of SP_TR rows in NP passes of
// CC columns: the new master iterates xm' = xm + d (d the FP32 correction x,
// plus the alpha p the last iteration left pending; xm' = d for the block's
// first correction) of the tile's own rows and of its external face
// neighbours (the band's gather plan) are formed into shared memory, the own
// rows' written to the other xm buffer (other CTAs still read the old one);
// then the true residual r = z - Q xm' in float-float arithmetic, stored as the
// FP32 right-hand side (r[par]) of the next correction solve, per-column r.r
// and z.z (FP32 products summed per thread, FP64 from the CTA sums on), and
// the row's probe sums sum_c z xm', sum_c (z xm')^2 (float-float over the
// columns, FP64 per row).  The last CTA sets, per column, the stop flag (true
// residual within tolerance) and the correction target
// eta = 0.5 tol |z| / |r| clamped to [ETA_MIN, 0.5], and flips xmpar.
template <int R>
__global__ void __launch_bounds__(CT, res_occ<R>()) k_blk_res(const BlkArgs* __restrict__ A, BlkState* st, int first) {
  constexpr int CC = res_cc<R>();      // columns per pass
  constexpr int NP = R / CC;           // passes
  constexpr int F4 = CC / 2;           // float4 (two float2 columns) per row and pass
  constexpr int RPS = 32 / F4;         // rows per warp step of the stencil phase
  constexpr int OWN = (SP_TR * F4 + CT - 1) / CT;
  constexpr int XN = (SP_EMAX * F4 + CT - 1) / CT;
  static_assert(SP_TR == 16 * (CT / 32) && 16 % RPS == 0 && CT % F4 == 0, "tile / CTA shape");
  const int N = A->N;
  const float lam = A->lam;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5, k2 = threadIdx.x % F4;
  const int xp = st->xmpar;
  const bool wsq = st->want_sq;
  const float4* __restrict__ xin = reinterpret_cast<const float4*>(A->xm[xp]);
  float4* __restrict__ xout = reinterpret_cast<float4*>(A->xm[xp ^ 1]);
  const float2* __restrict__ x2 = reinterpret_cast<const float2*>(A->x);
  const float2* __restrict__ p2 = reinterpret_cast<const float2*>(A->p);
  float2* __restrict__ r2 = reinterpret_cast<float2*>(A->r[st->par]);
  const int xv = st->xvalid, xpd = st->xpend;
  float ap[NP][2];
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) {
    ap[pp][0] = xpd ? st->aprev[pp * CC + 2 * k2] : 0.f;
    ap[pp][1] = xpd ? st->aprev[pp * CC + 2 * k2 + 1] : 0.f;
  }
  // xm' of this thread's two columns of pass pp in row `row` (the same arithmetic in every CTA)
  auto upd = [&](int row, int pp) -> float4 {
    const size_t e = (size_t)row * (R / 2) + pp * F4 + k2;
    float2 d = xv ? x2[e] : make_float2(0.f, 0.f);
    if (xpd) {
      const float2 pv = p2[e];
      d.x = fmaf(ap[pp][0], pv.x, d.x);
      d.y = fmaf(ap[pp][1], pv.y, d.y);
    }
    if (first) return make_float4(d.x, 0.f, d.y, 0.f);
    const float4 o = xin[e];
    const float2 a = ff_add_f(make_float2(o.x, o.y), d.x), b = ff_add_f(make_float2(o.z, o.w), d.y);
    return make_float4(a.x, a.y, b.x, b.y);
  };
  extern __shared__ __align__(16) float4 sx4[];  // [SP_ROWS][F4] staged xm'
  __shared__ float4 hrow[SP_TR];                 // per own row: probe sums over the passes so far (ff, ff)
  float fr[NP][2], fz[NP][2];
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) fr[pp][0] = fr[pp][1] = fz[pp][0] = fz[pp][1] = 0.0f;
  const int ntiles = (N + SP_TR - 1) / SP_TR;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int t0 = tile * SP_TR, t1 = min(N, t0 + SP_TR);
    const int ne = __ldg(A->sp_ne + tile);
    const int32_t* __restrict__ ext = A->sp_ext + (size_t)tile * SP_EMAX;
    uint4 slv = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    float qv = 0.0f;
    {
      const int myrow = t0 + 16 * wrp + (lane & 15);
      if (lane < 16 && myrow < t1) {
        slv = __ldg(reinterpret_cast<const uint4*>(A->sp_slot) + myrow);
        qv = __ldg(A->qd + myrow);
      }
    }
    int ji[XN];
#pragma unroll
    for (int i = 0; i < XN; ++i) {
      const int q = threadIdx.x + i * CT;
      ji[i] = q < SP_EMAX * F4 ? __ldg(ext + q / F4) : 0;
    }
    const int nown = (t1 - t0) * F4, next = ne * F4;
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      // the probe values of this thread's rows in the stencil phase, loaded with the master iterates
      __nv_bfloat162 zst[16 / RPS];
#pragma unroll
      for (int jstep = 0; jstep < 16 / RPS; ++jstep) {
        const int row = t0 + 16 * wrp + jstep * RPS + lane / F4;
        zst[jstep] = row < t1 ? *reinterpret_cast<const __nv_bfloat162*>(A->Z + (size_t)row * R + pp * CC + 2 * k2)
                              : __floats2bfloat162_rn(0.f, 0.f);
      }
      __syncthreads();  // the previous readers of sx4 are done
#pragma unroll
      for (int i = 0; i < OWN; ++i) {
        const int q = threadIdx.x + i * CT;
        if (q < nown) {
          const int row = t0 + q / F4;
          const float4 v = upd(row, pp);
          sx4[q] = v;
          xout[(size_t)row * (R / 2) + pp * F4 + k2] = v;
        }
      }
#pragma unroll
      for (int i = 0; i < XN; ++i) {
        const int q = threadIdx.x + i * CT;
        if (q < next) sx4[SP_TR * F4 + q] = upd(ji[i], pp);
      }
      __syncthreads();
#pragma unroll
      for (int jstep = 0; jstep < 16 / RPS; ++jstep) {
        const int src = jstep * RPS + lane / F4;  // row of the warp's 16, and the lane holding its slots
        const int rr = 16 * wrp + src, row = t0 + rr;
        const uint32_t sx = __shfl_sync(0xffffffffu, slv.x, src), sy = __shfl_sync(0xffffffffu, slv.y, src),
                       sz = __shfl_sync(0xffffffffu, slv.z, src);
        const float q = __shfl_sync(0xffffffffu, qv, src);
        const bool ok = row < t1;
        float2 t = make_float2(0.f, 0.f), qq = make_float2(0.f, 0.f);
        if (ok) {
          const int sv[6] = {(int16_t)(sx & 0xffffu), (int16_t)(sx >> 16), (int16_t)(sy & 0xffffu),
                             (int16_t)(sy >> 16),     (int16_t)(sz & 0xffffu), (int16_t)(sz >> 16)};
          const float4 xo = sx4[rr * F4 + k2];
          float2 n0 = make_float2(0.f, 0.f), n1 = n0;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const int sk = sv[k];
            if (sk < 0) continue;
            const float4 v = sk == SP_GLOBAL ? upd(__ldg(A->nb6 + 6 * (size_t)row + k), pp) : sx4[sk * F4 + k2];
            n0 = ff_add(n0, make_float2(v.x, v.y));
            n1 = ff_add(n1, make_float2(v.z, v.w));
          }
          const int c0 = pp * CC + 2 * k2;
          const __nv_bfloat162 zz = zst[jstep];
          const float z0 = __low2float(zz), z1 = __high2float(zz);
          const float2 xo0 = make_float2(xo.x, xo.y), xo1 = make_float2(xo.z, xo.w);
          const float2 qx0 = ff_add(ff_mul_f(xo0, q), ff_neg(ff_mul_f(n0, lam)));
          const float2 qx1 = ff_add(ff_mul_f(xo1, q), ff_neg(ff_mul_f(n1, lam)));
          const float2 rf0 = ff_add_f(ff_neg(qx0), z0), rf1 = ff_add_f(ff_neg(qx1), z1);
          const float ra = __fadd_rn(rf0.x, rf0.y), rb = __fadd_rn(rf1.x, rf1.y);
          r2[((size_t)row * R + c0) / 2] = make_float2(ra, rb);
          fr[pp][0] += ra * ra;
          fr[pp][1] += rb * rb;
          fz[pp][0] += z0 * z0;
          fz[pp][1] += z1 * z1;
          const float2 t0v = make_float2(z0 * xo0.x, z0 * xo0.y), t1v = make_float2(z1 * xo1.x, z1 * xo1.y);  // exact
          t = ff_add(t0v, t1v);
          if (wsq) {
            const float pa = __fmul_rn(t0v.x, t0v.x), pb = __fmul_rn(t1v.x, t1v.x);
            qq = ff_add(quick_two_sum(pa, __fmaf_rn(2.0f * t0v.x, t0v.y, __fmaf_rn(t0v.x, t0v.x, -pa))),
                        quick_two_sum(pb, __fmaf_rn(2.0f * t1v.x, t1v.y, __fmaf_rn(t1v.x, t1v.x, -pb))));
          }
        }
        // the row's probe sums over its column pairs (lanes of the row), then over the passes
#pragma unroll
        for (int o = F4 / 2; o > 0; o >>= 1) {
          t = ff_add(t, make_float2(__shfl_xor_sync(0xffffffffu, t.x, o), __shfl_xor_sync(0xffffffffu, t.y, o)));
          if (wsq)
            qq = ff_add(qq, make_float2(__shfl_xor_sync(0xffffffffu, qq.x, o), __shfl_xor_sync(0xffffffffu, qq.y, o)));
        }
        if (ok && k2 == 0) {
          if (pp > 0) {
            const float4 h = hrow[rr];
            t = ff_add(make_float2(h.x, h.y), t);
            qq = ff_add(make_float2(h.z, h.w), qq);
          }
          if (pp + 1 < NP) {
            hrow[rr] = make_float4(t.x, t.y, qq.x, qq.y);
          } else {
            A->hsum[row] = (double)t.x + (double)t.y;
            if (wsq) A->hsq[row] = (double)qq.x + (double)qq.y;
          }
        }
      }
    }
  }
  // per-column CTA sums (lanes sharing threadIdx % F4, then warps) -> part[q][c][CTA], q: 0 = r.r, 1 = z.z
  {
    constexpr int NA = 2 * NP * 2;
    __shared__ double shr[CT / 32][F4][NA];
    double acc[NA];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        acc[(0 * NP + pp) * 2 + j] = (double)fr[pp][j];
        acc[(1 * NP + pp) * 2 + j] = (double)fz[pp][j];
      }
#pragma unroll
    for (int k = 0; k < NA; ++k)
      for (int o = 16; o >= F4; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane < F4) {
#pragma unroll
      for (int k = 0; k < NA; ++k) shr[wrp][lane][k] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < 2 * R) {
      const int qk = threadIdx.x / R, cc = threadIdx.x % R;
      const int pp = cc / CC, kk = (cc % CC) / 2, j = cc & 1;
      double tsum = 0.0;
      for (int ww = 0; ww < CT / 32; ++ww) tsum += shr[ww][kk][(qk * NP + pp) * 2 + j];
      A->part[((size_t)qk * R + cc) * gridDim.x + blockIdx.x] = tsum;
    }
  }
  __shared__ double tot[3][MAXR];
  if (!reduce_partials<2>(A->part, A->gpart, st, R, tot)) return;
  if (threadIdx.x < R) {
    const int cc = threadIdx.x;
    const double rr = tot[0][cc], bb = tot[1][cc];
    st->rr0[cc] = rr;
    st->bb0[cc] = bb;
    st->bb[cc] = rr;  // the correction solve's right-hand side norm
    const int conv = (cc >= st->ncols) || rr <= st->tol0 * st->tol0 * bb || bb == 0.0;
    double eta = conv ? 0.5 : BLK_ETA * st->tol0 * sqrt(bb / rr);
    eta = fmin(fmax(eta, ETA_MIN), 0.5);
    st->tol2[cc] = eta * eta;
    st->done[cc] = conv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int q = 0; q < R; ++q) all &= st->done[q];
    if (all && st->status != 2) st->status = 0;
    if (!all && st->iter >= st->max_iter) st->status = 1;
    st->all_done = all || st->iter >= st->max_iter || st->status == 2;
    st->first = 1;
    st->xmpar ^= 1;
    st->cnt = 0;
    st->guard = 0;
  }
}

// Element update of one row, float4 over 4 columns (separately rounded, so
// that a row's u comes out bit-identical in the CTA that owns the row and in
// every CTA that stages it as an external neighbour):
//   s' = w + beta s,  r' = r - alpha s',  u' = r' / Q_jj
// (beta == 0 starts a new direction: the old s is not read).
__device__ __forceinline__ void pf_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ float bmul(float b, float v) { return b != 0.f ? __fmul_rn(b, v) : 0.f; }
__device__ __forceinline__ float4 next_s(float4 w, float4 s, float4 be) {
  return make_float4(__fadd_rn(w.x, bmul(be.x, s.x)), __fadd_rn(w.y, bmul(be.y, s.y)), __fadd_rn(w.z, bmul(be.z, s.z)),
                     __fadd_rn(w.w, bmul(be.w, s.w)));
}
__device__ __forceinline__ float4 next_r(float4 r, float4 sn, float4 al) {
  return make_float4(__fsub_rn(r.x, __fmul_rn(al.x, sn.x)), __fsub_rn(r.y, __fmul_rn(al.y, sn.y)),
                     __fsub_rn(r.z, __fmul_rn(al.z, sn.z)), __fsub_rn(r.w, __fmul_rn(al.w, sn.w)));
}
__device__ __forceinline__ float4 scale4(float4 a, float q) {
  return make_float4(__fmul_rn(a.x, q), __fmul_rn(a.y, q), __fmul_rn(a.z, q), __fmul_rn(a.w, q));
}

// One block-PCG iteration in one pass over the band (mode as below):
//   phase 1, the tile's own rows (float4 over 4 columns, streaming):
//     u = r/Q_jj, p' = u + beta p, s' = w + beta s, r' = r - alpha s',
//     u' = r'/Q_jj; every second iteration x += alpha_prev p + alpha p'
//     (the other one leaves alpha p' pending); partial sums r'.u', r'.r'
//   phase 2, the external rows its face neighbours reference: u' from their
//     (old) r, w, s by the same arithmetic
//   phase 3, w' = Q u' for the own rows from the staged u'; partial w'.u'.
// Streaming traffic that no other tile of the launch reads again (the own
// rows' p and x, and every row written) goes through evict-first loads and
// stores, leaving L2 to the r, w, s lines that other tiles gather as external
// rows.
// INIT (start of a correction solve from r): u = r/Q_jj, w = Q u, written to
// w[par]; r stays, x is zero, and p and s are not read by the next iteration
// (beta = 0 there).  Otherwise r, w, s are double-buffered (read [par],
// written [par ^ 1]; other CTAs read the old values of rows this CTA
// updates) and p, x are updated in place.  The last CTA reduces the partial
// sums in a fixed order and updates the per-column scalars (first pass of a
// correction solve: alpha = gamma/delta, beta = 0; afterwards the
// single-reduction recurrence and the stop test on r.r), then flips par
// (not after INIT).
// mode: IT_GRAPH inside the solver graph (may end the WHILE loop), IT_START
// host-launched start of a correction solve, IT_BENCH / IT_BENCH_HOLD timing
// of an iteration that writes / holds x (scalars, par and data are left as
// they are: alpha = beta = 0 keeps the data fixed).
constexpr int IT_GRAPH = 0, IT_BENCH = 1, IT_START = 2, IT_BENCH_HOLD = 3;

template <int R, bool INIT>
__global__ void __launch_bounds__(CT, blk_occ<R>()) k_blk_it(const BlkArgs* __restrict__ A, BlkState* st,
                                                  cudaGraphConditionalHandle handle, int mode) {
  const bool bench = mode == IT_BENCH || mode == IT_BENCH_HOLD;
  if (mode == IT_GRAPH && blockIdx.x == 0 && threadIdx.x == 0) {
    st->nexec += 1;
    unsigned gd = atomicAdd(&st->guard, 1u);
    if (st->all_done || gd > 2u * (unsigned)st->max_iter + 64u) {
      if (!st->all_done) {
        st->status = 1;
        st->all_done = 1;
      }
      cudaGraphSetConditional(handle, 0);
    }
  }
  if (!bench && st->all_done) return;  // also a start pass after the true residual met the tolerance
  constexpr int Q4 = R / 4;                          // float4 per row
  constexpr int OWN = SP_TR * Q4 / CT;               // own-row float4 per thread
  constexpr int XN = (SP_EMAX * Q4 + CT - 1) / CT;  // external float4 per thread (at most)
  static_assert(SP_TR * Q4 % CT == 0 && SP_TR == 16 * (CT / 32), "tile / CTA shape");
  const int N = A->N;
  const float lam = A->lam;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  const int par = bench ? 0 : st->par;
  const float4* __restrict__ rA = reinterpret_cast<const float4*>(A->r[par]);
  const float4* __restrict__ wA = reinterpret_cast<const float4*>(A->w[par]);
  const float4* __restrict__ sA = reinterpret_cast<const float4*>(A->s[par]);
  float4* __restrict__ rB = reinterpret_cast<float4*>(A->r[par ^ 1]);
  float4* __restrict__ sB = reinterpret_cast<float4*>(A->s[par ^ 1]);
  float* __restrict__ wB = A->w[INIT ? par : par ^ 1];
  float4* __restrict__ p4 = reinterpret_cast<float4*>(A->p);
  float4* __restrict__ x4 = reinterpret_cast<float4*>(A->x);
  const float* __restrict__ iq = A->iq;
  // this thread's 4 columns in phases 1 and 2 (the float4 index stride CT is a multiple of Q4)
  const int g = threadIdx.x % Q4;
  float4 al = make_float4(0.f, 0.f, 0.f, 0.f), be = al, ap = al;
  // x: xhold leaves this iteration's alpha p' pending; otherwise x (read only when xread) is written
  bool xhold = mode == IT_BENCH_HOLD, xread = true;
  if (!INIT && !bench) {
    al = make_float4((float)st->alpha[4 * g], (float)st->alpha[4 * g + 1], (float)st->alpha[4 * g + 2],
                     (float)st->alpha[4 * g + 3]);
    be = make_float4((float)st->beta[4 * g], (float)st->beta[4 * g + 1], (float)st->beta[4 * g + 2],
                     (float)st->beta[4 * g + 3]);
    xhold = !st->xpend;
    xread = st->xvalid;
    if (!xhold) ap = *reinterpret_cast<const float4*>(st->aprev + 4 * g);
  }
  extern __shared__ __align__(16) float us[];  // [SP_ROWS][R] u' of the own and external rows
  float4* us4 = reinterpret_cast<float4*>(us);
  // per-thread FP32 partial sums over the CTA's tiles (at most 4 products per
  // tile and thread), FP64 from the CTA reduction on
  float fa[8], ft[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 8; ++k) fa[k] = 0.0f;
  const int ntiles = (N + SP_TR - 1) / SP_TR;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int t0 = tile * SP_TR, t1 = min(N, t0 + SP_TR);
    const int ne = __ldg(A->sp_ne + tile);
    const int32_t* __restrict__ ext = A->sp_ext + (size_t)tile * SP_EMAX;
    uint4 slv = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    float qv = 0.0f;
    {
      const int myrow = t0 + 16 * wrp + (lane & 15);
      if (lane < 16 && myrow < t1) {
        slv = __ldg(reinterpret_cast<const uint4*>(A->sp_slot) + myrow);
        qv = __ldg(A->qd + myrow);
      }
    }
    int ji[XN];
#pragma unroll
    for (int i = 0; i < XN; ++i) {
      const int q = threadIdx.x + i * CT;
      ji[i] = q < SP_EMAX * Q4 ? __ldg(ext + q / Q4) : 0;
    }
    __syncthreads();  // the previous tile's readers of us are done
    // phase 1: own rows
    const int nown = (t1 - t0) * Q4;
#pragma unroll blk_p1_unroll<R>()
    for (int i = 0; i < OWN; ++i) {
      const int q = threadIdx.x + i * CT;
      if (q >= nown) break;
      const size_t gq = (size_t)t0 * Q4 + q;
      if (!INIT && OWN > blk_p1_unroll<R>() && q + CT < nown) {  // the thread's next item into L2 (one at a time)
        pf_l2(rA + gq + CT); pf_l2(wA + gq + CT); pf_l2(sA + gq + CT); pf_l2(p4 + gq + CT);
        if (!xhold && xread) pf_l2(x4 + gq + CT);
      }
      const float qi = __ldg(iq + t0 + q / Q4);
      const float4 ri = rA[gq];
      float4 rn, un;
      if (INIT) {
        rn = ri;
        un = scale4(ri, qi);
      } else {
        const float4 wi = wA[gq], si = sA[gq], pi = __ldcs(p4 + gq);
        const float4 u0 = scale4(ri, qi);
        const float4 pn = make_float4(__fadd_rn(u0.x, bmul(be.x, pi.x)), __fadd_rn(u0.y, bmul(be.y, pi.y)),
                                      __fadd_rn(u0.z, bmul(be.z, pi.z)), __fadd_rn(u0.w, bmul(be.w, pi.w)));
        const float4 sn = next_s(wi, si, be);
        rn = next_r(ri, sn, al);
        un = scale4(rn, qi);
        __stcs(p4 + gq, pn);
        if (!xhold) {
          const float4 xi = xread ? __ldcs(x4 + gq) : make_float4(0.f, 0.f, 0.f, 0.f);
          __stcs(x4 + gq, make_float4(fmaf(al.x, pn.x, fmaf(ap.x, pi.x, xi.x)), fmaf(al.y, pn.y, fmaf(ap.y, pi.y, xi.y)),
                               fmaf(al.z, pn.z, fmaf(ap.z, pi.z, xi.z)), fmaf(al.w, pn.w, fmaf(ap.w, pi.w, xi.w))));
        }
        __stcs(sB + gq, sn);
        __stcs(rB + gq, rn);
      }
      us4[q] = un;
      fa[0] += rn.x * un.x; fa[1] += rn.y * un.y; fa[2] += rn.z * un.z; fa[3] += rn.w * un.w;
      fa[4] += rn.x * rn.x; fa[5] += rn.y * rn.y; fa[6] += rn.z * rn.z; fa[7] += rn.w * rn.w;
    }
    // phase 2: external rows
    const int next = ne * Q4;
#pragma unroll  // every external-row item of the thread in flight (measured 1.75 against 1.80 ms per R = 32 iteration)
    for (int i = 0; i < XN; ++i) {
      const int q = threadIdx.x + i * CT;
      if (q >= next) break;
      const size_t gj = (size_t)ji[i] * Q4 + (q % Q4);
      const float qj = __ldg(iq + ji[i]);
      const float4 rj = rA[gj];
      float4 un;
      if (INIT) {
        un = scale4(rj, qj);
      } else {
        const float4 sn = next_s(wA[gj], sA[gj], be);
        un = scale4(next_r(rj, sn, al), qj);
      }
      us4[SP_TR * Q4 + q] = un;
    }
    __syncthreads();
    {  // the next tile's own rows of r, w, s, p (and x; the start pass: r only) into L2, one bulk prefetch per vector
      const int tn = tile + gridDim.x;
      if (tn < ntiles && threadIdx.x < (INIT ? 1 : 5) && (threadIdx.x < 4 || (!xhold && xread))) {
        const size_t n0 = (size_t)tn * SP_TR * Q4, n1 = min((size_t)N * Q4, n0 + (size_t)SP_TR * Q4);
        const float4* v = threadIdx.x == 0 ? rA : threadIdx.x == 1 ? wA : threadIdx.x == 2 ? sA : threadIdx.x == 3 ? p4 : x4;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(v + n0), "r"((uint32_t)((n1 - n0) * 16))
                     : "memory");
      }
    }
    // phase 3: w' = Q u' for the own rows, four columns (one float4 of u') per lane
    constexpr int RPS = 32 / Q4;  // rows per warp step
#pragma unroll 1
    for (int jstep = 0; jstep < 16 / RPS; ++jstep) {
      const int src = jstep * RPS + lane / Q4;  // row of the warp's 16, and the lane holding its slots
      const int rr = 16 * wrp + src, row = t0 + rr;
      const uint32_t sx = __shfl_sync(0xffffffffu, slv.x, src), sy = __shfl_sync(0xffffffffu, slv.y, src),
                     sz = __shfl_sync(0xffffffffu, slv.z, src);
      const float q = __shfl_sync(0xffffffffu, qv, src);
      if (row >= t1) continue;
      const int sv[6] = {(int16_t)(sx & 0xffffu), (int16_t)(sx >> 16), (int16_t)(sy & 0xffffu),
                         (int16_t)(sy >> 16),     (int16_t)(sz & 0xffffu), (int16_t)(sz >> 16)};
      const float4 uo = us4[rr * Q4 + g];
      // u' of face neighbour k: staged row, or formed from global memory beyond the staged list
      auto nbu = [&](int k) -> float4 {
        const int sk = sv[k];
        if (sk >= 0 && sk != SP_GLOBAL) return us4[sk * Q4 + g];
        if (sk < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
        const int j = __ldg(A->nb6 + 6 * (size_t)row + k);
        const size_t gj = (size_t)j * Q4 + g;
        const float qj = __ldg(iq + j);
        if (INIT) return scale4(rA[gj], qj);
        return scale4(next_r(rA[gj], next_s(wA[gj], sA[gj], be), al), qj);
      };
      auto add4 = [](float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); };
      const float4 s01 = add4(nbu(0), nbu(1)), s23 = add4(nbu(2), nbu(3)), s45 = add4(nbu(4), nbu(5));
      const float4 ns = add4(add4(s01, s23), s45);
      float4 wn;
      wn.x = q * uo.x - lam * ns.x;
      wn.y = q * uo.y - lam * ns.y;
      wn.z = q * uo.z - lam * ns.z;
      wn.w = q * uo.w - lam * ns.w;
      __stcs(reinterpret_cast<float4*>(wB) + (size_t)row * Q4 + g, wn);
      ft[0] += wn.x * uo.x; ft[1] += wn.y * uo.y; ft[2] += wn.z * uo.z; ft[3] += wn.w * uo.w;
    }
  }
  // per-column CTA sums (lanes sharing threadIdx % Q4, then warps): r'.u', r'.r', w'.u' -> part1
  {
    __shared__ double sh1[CT / 32][8][12];
    double acc1[12];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc1[k] = (double)fa[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc1[8 + k] = (double)ft[k];
#pragma unroll
    for (int k = 0; k < 12; ++k)
      for (int o = 16; o >= Q4; o >>= 1) acc1[k] += __shfl_xor_sync(0xffffffffu, acc1[k], o);
    if (lane < Q4) {
#pragma unroll
      for (int k = 0; k < 12; ++k) sh1[wrp][lane][k] = acc1[k];
    }
    __syncthreads();
    if (threadIdx.x < 3 * R) {
      const int qk = threadIdx.x / R, cc = threadIdx.x % R;  // qk: 0 = r.u, 1 = r.r, 2 = w.u
      double t = 0.0;
      for (int ww = 0; ww < CT / 32; ++ww) t += sh1[ww][cc / 4][4 * qk + (cc & 3)];
      A->part1[((size_t)qk * R + cc) * gridDim.x + blockIdx.x] = t;
    }
  }
  __shared__ double tot1[3][MAXR];
  if (!reduce_partials<3>(A->part1, A->gpart, st, R, tot1)) return;
  if (bench) {
    if (threadIdx.x == 0) st->cnt = 0;
    return;
  }
  __shared__ int any_live;
  const bool first = st->first;
  if (threadIdx.x == 0) {
    any_live = 0;
    if (!first) st->iter += 1;
  }
  __syncthreads();
  if (threadIdx.x < R) {
    const int cc = threadIdx.x;
    const double gm = tot1[0][cc], rr = tot1[1][cc], d = tot1[2][cc];
    if (!INIT) st->aprev[cc] = xhold ? (float)st->alpha[cc] : 0.0f;  // the alpha this iteration used
    if (!st->done[cc]) {
      if (first) {
        st->gamma[cc] = gm;
        st->beta[cc] = 0.0;
        if (!(d > 0.0) || !isfinite(d) || !isfinite(gm)) {
          st->done[cc] = 1;
          st->status = 2;
        } else {
          st->alpha[cc] = gm / d;
          atomicOr(&any_live, 1);
        }
      } else {
        st->rr[cc] = rr;
        st->iters[cc] += 1;
        if (!isfinite(gm) || !isfinite(d) || !isfinite(rr)) {
          st->done[cc] = 1;
          st->status = 2;
        } else if (rr <= st->tol2[cc] * st->bb[cc]) {
          st->done[cc] = 1;
        } else {
          const double beta = gm / st->gamma[cc];
          const double den = d - beta * gm / st->alpha[cc];
          if (!(den > 0.0) || !isfinite(den)) {
            st->done[cc] = 1;
            st->status = 2;
          } else {
            st->beta[cc] = beta;
            st->alpha[cc] = gm / den;
            st->gamma[cc] = gm;
            atomicOr(&any_live, 1);
          }
        }
      }
    }
    if (st->done[cc]) {
      st->alpha[cc] = 0.0;
      st->beta[cc] = 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->first = 0;
    if (INIT) {
      st->xvalid = 0;
      st->xpend = 0;
    } else {
      st->par ^= 1;
      st->xvalid |= !xhold;
      st->xpend = xhold;
    }
    if (!any_live || st->iter >= st->max_iter) {
      st->all_done = 1;
      if (mode == IT_GRAPH) cudaGraphSetConditional(handle, 0);
    }
    st->cnt = 0;
  }
}

// Z[i][c] = Rademacher(seed, k0 + c, lin_i) for c < ncols, 0 beyond, and the
// first correction right-hand side r = z - Q 0 = z (xm = 0 is implied: the
// first correction is copied into xm rather than added)
template <int R>
__global__ void k_probes(int N, const int32_t* __restrict__ lin, uint64_t mseed, int k0, int ncols,
                         __nv_bfloat16* __restrict__ Z, float* __restrict__ r0) {
  // a thread forms 8 consecutive columns of one row: one 16-byte store of Z, two of r
  constexpr int G = R / 8;  // column groups per row
  const int64_t n = (int64_t)N * G;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / G;
    const int c0 = (int)(e - i * G) * 8;
    const uint64_t li = (uint64_t)(uint32_t)__ldg(lin + i);
    float z[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      z[k] = 0.0f;
      if (c0 + k < ncols) {
        const uint64_t v = mix64(mseed ^ ((uint64_t)(k0 + c0 + k) * 0xD1B54A32D192ED03ULL) ^ li);
        z[k] = (v >> 63) ? -1.0f : 1.0f;
      }
    }
    uint4 zb;
    __nv_bfloat162* zh = reinterpret_cast<__nv_bfloat162*>(&zb);
#pragma unroll
    for (int k = 0; k < 4; ++k) zh[k] = __floats2bfloat162_rn(z[2 * k], z[2 * k + 1]);
    reinterpret_cast<uint4*>(Z)[e] = zb;
    reinterpret_cast<float4*>(r0)[2 * e] = make_float4(z[0], z[1], z[2], z[3]);
    reinterpret_cast<float4*>(r0)[2 * e + 1] = make_float4(z[4], z[5], z[6], z[7]);
  }
}

// Y = Q X for R right-hand sides (X, Y [N][R], the columns of a row
// contiguous): the matrix-free 7-point stencil of the precision (Sec. 3.6),
// applied per tile of SP_TR rows with the tile's own rows and its external
// face-neighbour rows (the band's gather plan) staged in shared memory, then
// four columns of a row per lane; the neighbour sum keeps the order
// ((x-1 + x+1) + (y-1 + y+1)) + (z-1 + z+1) of the single-RHS SpMV.
template <int R>
__global__ void __launch_bounds__(CT, blk_occ<R>()) k_spmm(int N, float lam, const float* __restrict__ qd,
                                                const int32_t* __restrict__ nb6, const int32_t* __restrict__ sp_ext,
                                                const int32_t* __restrict__ sp_ne, const int16_t* __restrict__ sp_slot,
                                                const float* __restrict__ X, float* __restrict__ Y) {
  constexpr int Q4 = R / 4;
  constexpr int OWN = SP_TR * Q4 / CT;
  constexpr int XN = (SP_EMAX * Q4 + CT - 1) / CT;
  static_assert(SP_TR * Q4 % CT == 0 && SP_TR == 16 * (CT / 32), "tile / CTA shape");
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5, g = threadIdx.x % Q4;
  const float4* __restrict__ X4 = reinterpret_cast<const float4*>(X);
  float4* __restrict__ Y4 = reinterpret_cast<float4*>(Y);
  extern __shared__ __align__(16) float us[];  // [SP_ROWS][R]
  float4* us4 = reinterpret_cast<float4*>(us);
  const int ntiles = (N + SP_TR - 1) / SP_TR;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int t0 = tile * SP_TR, t1 = min(N, t0 + SP_TR);
    const int ne = __ldg(sp_ne + tile);
    const int32_t* __restrict__ ext = sp_ext + (size_t)tile * SP_EMAX;
    uint4 slv = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    float qv = 0.0f;
    {
      const int myrow = t0 + 16 * wrp + (lane & 15);
      if (lane < 16 && myrow < t1) {
        slv = __ldg(reinterpret_cast<const uint4*>(sp_slot) + myrow);
        qv = __ldg(qd + myrow);
      }
    }
    int ji[XN];
#pragma unroll
    for (int i = 0; i < XN; ++i) {
      const int q = threadIdx.x + i * CT;
      ji[i] = q < SP_EMAX * Q4 ? __ldg(ext + q / Q4) : 0;
    }
    __syncthreads();  // the previous tile's readers of us are done
    const int nown = (t1 - t0) * Q4;
#pragma unroll
    for (int i = 0; i < OWN; ++i) {
      const int q = threadIdx.x + i * CT;
      if (q < nown) us4[q] = __ldg(X4 + (size_t)t0 * Q4 + q);
    }
    const int next = ne * Q4;
#pragma unroll
    for (int i = 0; i < XN; ++i) {
      const int q = threadIdx.x + i * CT;
      if (q < next) us4[SP_TR * Q4 + q] = __ldg(X4 + (size_t)ji[i] * Q4 + (q % Q4));
    }
    __syncthreads();
    constexpr int RPS = 32 / Q4;  // rows per warp step
#pragma unroll 1
    for (int jstep = 0; jstep < 16 / RPS; ++jstep) {
      const int src = jstep * RPS + lane / Q4;  // row of the warp's 16, and the lane holding its slots
      const int rr = 16 * wrp + src, row = t0 + rr;
      const uint32_t sx = __shfl_sync(0xffffffffu, slv.x, src), sy = __shfl_sync(0xffffffffu, slv.y, src),
                     sz = __shfl_sync(0xffffffffu, slv.z, src);
      const float q = __shfl_sync(0xffffffffu, qv, src);
      if (row >= t1) continue;
      const int sv[6] = {(int16_t)(sx & 0xffffu), (int16_t)(sx >> 16), (int16_t)(sy & 0xffffu),
                         (int16_t)(sy >> 16),     (int16_t)(sz & 0xffffu), (int16_t)(sz >> 16)};
      const float4 xo = us4[rr * Q4 + g];
      auto nbx = [&](int k) -> float4 {  // staged row, or read from global memory beyond the staged list
        const int sk = sv[k];
        if (sk >= 0 && sk != SP_GLOBAL) return us4[sk * Q4 + g];
        if (sk < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
        return __ldg(X4 + (size_t)__ldg(nb6 + 6 * (size_t)row + k) * Q4 + g);
      };
      auto add4 = [](float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); };
      const float4 s01 = add4(nbx(0), nbx(1)), s23 = add4(nbx(2), nbx(3)), s45 = add4(nbx(4), nbx(5));
      const float4 ns = add4(add4(s01, s23), s45);
      Y4[(size_t)row * Q4 + g] = make_float4(q * xo.x - lam * ns.x, q * xo.y - lam * ns.y, q * xo.z - lam * ns.z,
                                             q * xo.w - lam * ns.w);
    }
  }
}

__global__ void k_finish(int N, const double* __restrict__ sacc, double invK, float* __restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) s[i] = (float)(sacc[i] * invK);
}

// s_acc += hsum, sq += hsq (the block's probe sums from its last residual pass)
__global__ void k_hadd(int N, const double* __restrict__ hsum, const double* __restrict__ hsq, double* __restrict__ sacc,
                       double* __restrict__ sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    sacc[i] += hsum[i];
    if (sq) sq[i] += hsq[i];
  }
}

// per-voxel indices of the six face neighbours (-x, +x, -y, +y, -z, +z), -1 outside the band
__global__ void k_nb6(BandView B, int32_t* __restrict__ nb6) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int L = B.lin[v];
    int i = L % B.n, j = (L / B.n) % B.n, k = L / (B.n * B.n);
    nb6[6 * (size_t)v + 0] = band_lookup(B, i - 1, j, k);
    nb6[6 * (size_t)v + 1] = band_lookup(B, i + 1, j, k);
    nb6[6 * (size_t)v + 2] = band_lookup(B, i, j - 1, k);
    nb6[6 * (size_t)v + 3] = band_lookup(B, i, j + 1, k);
    nb6[6 * (size_t)v + 4] = band_lookup(B, i, j, k - 1);
    nb6[6 * (size_t)v + 5] = band_lookup(B, i, j, k + 1);
  }
}

// SpMM plan of one tile (one CTA of 256 threads per tile): the sorted unique
// rows outside [t0, t1) referenced by the tile's face neighbours (the first
// SP_EMAX are staged), and per row the slot of each neighbour: own row
// j - t0, external row SP_TR + e, -1 none, SP_GLOBAL beyond the list.
__global__ void __launch_bounds__(256) k_sp_plan(int N, const int32_t* __restrict__ nb6, int32_t* __restrict__ ext,
                                                 int32_t* __restrict__ ne_out, int16_t* __restrict__ slot) {
  constexpr int C = 2048;  // >= 6 SP_TR candidates, a power of two
  __shared__ int cand[C];
  __shared__ int uniq[C];
  __shared__ int cnt[256];
  __shared__ int nc;
  const int t0 = blockIdx.x * SP_TR, t1 = min(N, t0 + SP_TR);
  if (threadIdx.x == 0) nc = 0;
  for (int q = threadIdx.x; q < C; q += blockDim.x) cand[q] = INT_MAX;
  __syncthreads();
  for (int q = threadIdx.x; q < (t1 - t0) * 6; q += blockDim.x) {
    const int j = nb6[6 * (size_t)t0 + q];
    if (j >= 0 && (j < t0 || j >= t1)) cand[atomicAdd(&nc, 1)] = j;
  }
  __syncthreads();
  // bitonic sort, ascending (INT_MAX padding last)
  for (int k = 2; k <= C; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int l = threadIdx.x; l < C; l += blockDim.x) {
        const int p = l ^ jj;
        if (p > l) {
          const int a = cand[l], b = cand[p];
          if ((a > b) == ((l & k) == 0)) {
            cand[l] = b;
            cand[p] = a;
          }
        }
      }
      __syncthreads();
    }
  // unique: thread t keeps the first occurrences in cand[8t, 8t + 8)
  const int base = 8 * threadIdx.x;
  int mine = 0;
  for (int l = base; l < base + 8; ++l)
    mine += cand[l] != INT_MAX && (l == 0 || cand[l] != cand[l - 1]);
  cnt[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int c = cnt[t];
      cnt[t] = run;
      run += c;
    }
    nc = run;
  }
  __syncthreads();
  int pos = cnt[threadIdx.x];
  for (int l = base; l < base + 8; ++l)
    if (cand[l] != INT_MAX && (l == 0 || cand[l] != cand[l - 1])) uniq[pos++] = cand[l];
  __syncthreads();
  const int ne = nc, nkeep = min(ne, SP_EMAX);
  for (int e = threadIdx.x; e < nkeep; e += blockDim.x) ext[(size_t)blockIdx.x * SP_EMAX + e] = uniq[e];
  if (threadIdx.x == 0) ne_out[blockIdx.x] = nkeep;
  for (int row = t0 + threadIdx.x; row < t1; row += blockDim.x) {
    int16_t sv[8];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int j = nb6[6 * (size_t)row + k];
      int16_t v = -1;
      if (j >= t0 && j < t1) {
        v = (int16_t)(j - t0);
      } else if (j >= 0) {
        int lo = 0, hi = ne;  // first index with uniq[idx] >= j
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (uniq[mid] < j) lo = mid + 1;
          else hi = mid;
        }
        v = lo < SP_EMAX ? (int16_t)(SP_TR + lo) : SP_GLOBAL;
      }
      sv[k] = v;
    }
    sv[6] = sv[7] = -1;
    uint4 o;
    o.x = (uint16_t)sv[0] | ((uint32_t)(uint16_t)sv[1] << 16);
    o.y = (uint16_t)sv[2] | ((uint32_t)(uint16_t)sv[3] << 16);
    o.z = (uint16_t)sv[4] | ((uint32_t)(uint16_t)sv[5] << 16);
    o.w = (uint16_t)sv[6] | ((uint32_t)(uint16_t)sv[7] << 16);
    reinterpret_cast<uint4*>(slot)[row] = o;
  }
}

__global__ void k_inv(int N, const float* __restrict__ qd, float* __restrict__ iq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) iq[i] = 1.0f / qd[i];
}

// State for a new block of probes.  With xm = 0 the true residual is z
// itself, so |r|^2 = |z|^2 = N for every live column and no residual pass is
// needed before the first correction solve.
__global__ void k_blk_init(BlkState* st, double tol, int max_iter, int ncols, int N, double eta_min, int want_sq) {
  int c = threadIdx.x;
  if (c < MAXR) {
    const int live = c < ncols;
    st->done[c] = !live;
    st->iters[c] = 0;
    st->beta[c] = 0.0;
    st->alpha[c] = 0.0;
    st->rr0[c] = st->bb0[c] = st->bb[c] = live ? (double)N : 0.0;
    const double eta = fmin(fmax(BLK_ETA * tol, eta_min), 0.5);
    st->tol2[c] = eta * eta;
  }
  if (c == 0) {
    st->tol0 = tol;
    st->max_iter = max_iter;
    st->iter = 0;
    st->all_done = 0;
    st->status = 0;
    st->ncols = ncols;
    st->want_sq = want_sq;
    st->xmpar = 0;
    st->first = 1;
    st->par = 0;  // k_probes wrote the first right-hand side into r[0]
    st->cnt = 0;
    for (int q = 0; q < NGRP; ++q) st->gcnt[q] = 0;
    st->guard = 0;
    st->nexec = 0;
  }
}

__global__ void k_bench_state(BlkState* st) {
  int c = threadIdx.x;
  if (c < MAXR) {
    st->beta[c] = 0.0;  // bounded values over repeated launches
    st->alpha[c] = 0.0;
  }
  if (c == 0) {
    st->cnt = 0;
    for (int q = 0; q < NGRP; ++q) st->gcnt[q] = 0;
    st->all_done = 0;
  }
}

constexpr size_t sp_smem(int R) { return (size_t)SP_ROWS * R * sizeof(float); }

unsigned grid_for(int64_t n, int threads, int64_t cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

struct BlockGraph {
  int R = 0;
  int64_t cap_rows = 0;
  BlkArgs h;                    // host copy of the argument block
  BlkArgs* h_pin = nullptr;     // pinned staging for the upload
  BlkArgs* d_args = nullptr;
  __nv_bfloat16* Z = nullptr;
  double* sacc = nullptr;
  BlkState* st = nullptr;
  BlkState* h_st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

static void free_arrays(BlockGraph* g) {
  void* ptrs[] = {g->h.r[0], g->h.w[0], g->h.s[0], g->h.r[1], g->h.w[1], g->h.s[1], g->h.p, g->h.x,
                  g->h.xm[0], g->h.xm[1], g->h.iq,       g->h.part, g->h.part1, g->Z, g->sacc, g->h.hsum, g->h.hsq, g->h.gpart};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  g->cap_rows = 0;
}

void block_graph_free(BlockGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  free_arrays(g);
  if (g->d_args) cudaFree(g->d_args);
  if (g->st) cudaFree(g->st);
  if (g->h_st) cudaFreeHost(g->h_st);
  if (g->h_pin) cudaFreeHost(g->h_pin);
  delete g;
}

template <int R>
static void blk_iter(BlockGraph* g, cudaStream_t s, cudaGraphConditionalHandle h) {
  k_blk_it<R, false><<<blk_ncta<R>(), CT, sp_smem(R), s>>>(g->d_args, g->st, h, IT_GRAPH);
}

// start of a correction solve from r: u = r/Q_jj, w = Q u, x = 0, alpha
template <int R>
static void blk_start(BlockGraph* g, cudaStream_t s) {
  k_blk_it<R, true><<<blk_ncta<R>(), CT, sp_smem(R), s>>>(g->d_args, g->st, cudaGraphConditionalHandle(), IT_START);
  count_launch();
}

// shared memory of the residual pass: the staged master iterates of a tile (16 columns at a time)
template <int R>
constexpr size_t res_smem() { return (size_t)SP_ROWS * res_cc<R>() / 2 * sizeof(float4); }

// xm += correction, true residual, stop test; then the start of the next correction solve
template <int R>
static void blk_outer(BlockGraph* g, cudaStream_t s, bool first) {
  k_blk_res<R><<<152 * res_occ<R>(), CT, res_smem<R>(), s>>>(g->d_args, g->st, first ? 1 : 0);
  count_launch();
  blk_start<R>(g, s);
}

static int ridx(int R) { return R == 8 ? 0 : (R == 16 ? 1 : 2); }

// The band's face-neighbour table and SpMM gather plan (built once per band).
static bf_status ensure_sp_plan(bf_ctx* ctx, bf_band* b) {
  cudaStream_t s = ctx->stream;
  if (!b->nb6) {
    BF_TRY(dev_alloc_t(ctx, &b->nb6, (size_t)6 * (b->N ? b->N : 1)));
    k_nb6<<<grid_for(b->N, 256, 152 * 16), 256, 0, s>>>(band_view(b), b->nb6);
    count_launch();
  }
  if (!b->sp_slot) {
    const int nt = (int)((b->N + SP_TR - 1) / SP_TR);
    BF_TRY(dev_alloc_t(ctx, &b->sp_ext, (size_t)SP_EMAX * (nt ? nt : 1)));
    BF_TRY(dev_alloc_t(ctx, &b->sp_ne, (size_t)(nt ? nt : 1)));
    BF_TRY(dev_alloc_t(ctx, &b->sp_slot, (size_t)8 * (b->N ? b->N : 1)));
    if (nt) {
      k_sp_plan<<<nt, 256, 0, s>>>((int)b->N, b->nb6, b->sp_ext, b->sp_ne, b->sp_slot);
      count_launch();
    }
  }
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// The context's block solver for width R, with workspaces for >= N rows and
// the argument block pointing at band b.
template <int R>
static bf_status get_block_solver(bf_ctx* ctx, bf_band* b, BlockGraph** out) {
  BlockGraph*& g = ctx->blk[ridx(R)];
  cudaStream_t s = ctx->stream;
  if (!g) {
    g = new BlockGraph();
    g->R = R;
    BF_CK(cudaFuncSetAttribute(k_blk_it<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp_smem(R)));
    BF_CK(cudaFuncSetAttribute(k_blk_it<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp_smem(R)));
    BF_CK(cudaFuncSetAttribute(k_blk_res<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem<R>()));
    memset(&g->h, 0, sizeof(g->h));
    BF_CK(cudaMalloc(&g->d_args, sizeof(BlkArgs)));
    BF_CK(cudaMallocHost(&g->h_pin, sizeof(BlkArgs)));
    BF_CK(cudaMalloc(&g->st, sizeof(BlkState)));
    BF_CK(cudaMallocHost(&g->h_st, sizeof(BlkState)));
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
    // two iterations per evaluation of the WHILE condition (the launch gap between plain kernel nodes is
    // shorter); the second one returns at once when the first finished the solve
    blk_iter<R>(g, g->cap, h);
    blk_iter<R>(g, g->cap, h);
    cudaGraph_t ob;
    cudaError_t e = cudaStreamEndCapture(g->cap, &ob);
    if (e != cudaSuccess) return bf_fail(ctx, BF_ECUDA, "capture block PCG body", cudaGetErrorString(e));
    BF_CK(cudaGraphInstantiate(&g->exec, g->graph, 0));
  }
  if (b->N > g->cap_rows) {
    BF_CK(cudaStreamSynchronize(s));
    free_arrays(g);
    const int64_t rows = b->N + b->N / 8 + 1024;
    const size_t nv = (size_t)rows * R;
    for (int k = 0; k < 2; ++k) {
      BF_CK(cudaMalloc(&g->h.r[k], nv * 4));
      BF_CK(cudaMalloc(&g->h.w[k], nv * 4));
      BF_CK(cudaMalloc(&g->h.s[k], nv * 4));
    }
    BF_CK(cudaMalloc(&g->h.p, nv * 4));
    BF_CK(cudaMalloc(&g->h.x, nv * 4));
    BF_CK(cudaMalloc(&g->h.xm[0], nv * sizeof(float2)));
    BF_CK(cudaMalloc(&g->h.xm[1], nv * sizeof(float2)));
    BF_CK(cudaMalloc(&g->h.hsum, (size_t)rows * sizeof(double)));
    BF_CK(cudaMalloc(&g->h.hsq, (size_t)rows * sizeof(double)));
    BF_CK(cudaMalloc(&g->Z, nv * 2));
    BF_CK(cudaMalloc(&g->h.iq, (size_t)rows * 4));
    BF_CK(cudaMalloc(&g->sacc, (size_t)rows * 8));
    BF_CK(cudaMalloc(&g->h.part, (size_t)3 * R * NCTA_MAX * sizeof(double)));
    BF_CK(cudaMalloc(&g->h.part1, (size_t)3 * R * NCTA_MAX * sizeof(double)));
    BF_CK(cudaMalloc(&g->h.gpart, (size_t)3 * R * NGRP * sizeof(double)));
    g->cap_rows = rows;
  }
  BF_TRY(ensure_sp_plan(ctx, b));
  g->h.N = (int)b->N;
  g->h.lam = (float)b->prm.lambda;
  g->h.nb6 = b->nb6;
  g->h.sp_ext = b->sp_ext;
  g->h.sp_ne = b->sp_ne;
  g->h.sp_slot = b->sp_slot;
  g->h.qd = b->qd;
  g->h.Z = g->Z;
  // the previous upload from h_pin has completed: every solve ends with a sync
  *g->h_pin = g->h;
  BF_CK(cudaMemcpyAsync(g->d_args, g->h_pin, sizeof(BlkArgs), cudaMemcpyHostToDevice, s));
  *out = g;
  return BF_OK;
}

template <int R>
static bf_status variance_t(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                            int max_iter, float* s_out, int* total_iters, double* sq, double* s1) {
  cudaStream_t s = ctx->stream;
  BlockGraph* g = nullptr;
  BF_TRY(get_block_solver<R>(ctx, b, &g));
  const int N = (int)b->N;
  BF_CK(cudaMemsetAsync(g->sacc, 0, (size_t)N * 8, s));
  k_inv<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, b->qd, g->h.iq);
  count_launch();
  uint64_t mseed = 0;
  {  // host copy of the probe seed mix (same function as the device)
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    mseed = z ^ (z >> 31);
  }
  int tot_it = 0;
  bf_status result = BF_OK;
  for (int k0 = kb; k0 < ke; k0 += R) {
    // one block of R probes: float-float master iterates, FP32 correction solves
    int ncols = ke - k0 < R ? ke - k0 : R;
    k_probes<R><<<grid_for((int64_t)N * (R / 8), 256, 152 * 16), 256, 0, s>>>(N, b->lin, mseed, k0, ncols, g->Z,
                                                                         g->h.r[0]);
    count_launch();
    k_blk_init<<<1, MAXR, 0, s>>>(g->st, tol, max_iter, ncols, N, ETA_MIN, sq != nullptr);
    count_launch();
    blk_start<R>(g, s);
    BF_CK(cudaGetLastError());
    bool done = false;
    int nouter = 0;  // residual passes run (the last one leaves the block's probe sums in hsum, hsq)
    for (int outer = 0; outer < REFINE_MAX_PASSES; ++outer) {
      // correction solve (its first kernel ends the loop at once if the state is already final), then the
      // residual pass and the next start; the host looks at the state only after each residual pass
      BF_CK(cudaGraphLaunch(g->exec, s));
      blk_outer<R>(g, s, nouter == 0);
      ++nouter;
      BF_CK(cudaGetLastError());
      BF_CK(cudaMemcpyAsync(g->h_st, g->st, sizeof(BlkState), cudaMemcpyDeviceToHost, s));
      BF_CK(cudaStreamSynchronize(s));
      if (g->h_st->all_done) {
        done = true;
        break;
      }
    }
    const BlkState& h = *g->h_st;
    count_launch(h.nexec);
    for (int c = 0; c < ncols; ++c) tot_it += h.iters[c];
    k_hadd<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, g->h.hsum, g->h.hsq, g->sacc, sq);
    count_launch();
    BF_CK(cudaGetLastError());
    if (h.status == 2) { result = BF_BREAKDOWN; break; }
    if (!done || h.status == 1) { result = BF_NOT_CONVERGED; break; }
  }
  k_finish<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, g->sacc, scale, s_out);
  if (s1) BF_CK(cudaMemcpyAsync(s1, g->sacc, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  count_launch();
  BF_CK(cudaGetLastError());
  BF_CK(cudaStreamSynchronize(s));
  if (total_iters) *total_iters = tot_it;
  if (result == BF_BREAKDOWN) return bf_fail(ctx, BF_BREAKDOWN, "block PCG breakdown");
  if (result == BF_NOT_CONVERGED) return bf_fail(ctx, BF_NOT_CONVERGED, "block PCG iteration limit reached");
  return BF_OK;
}

// time one block-PCG iteration (k_blk_it in timing mode)
template <int R>
static bf_status bench_blk_t(bf_ctx* ctx, bf_band* b, int reps, double* ms) {
  BlockGraph* g = nullptr;
  BF_TRY(get_block_solver<R>(ctx, b, &g));
  cudaStream_t s = ctx->stream;
  k_inv<<<grid_for(b->N, 256, 152 * 16), 256, 0, s>>>((int)b->N, b->qd, g->h.iq);
  count_launch();
  k_bench_state<<<1, MAXR, 0, s>>>(g->st);
  count_launch();
  cudaEvent_t e0, e1;
  BF_CK(cudaEventCreate(&e0));
  BF_CK(cudaEventCreate(&e1));
  BF_CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) {  // alternately an iteration that writes x and one that holds it
    k_blk_it<R, false><<<blk_ncta<R>(), CT, sp_smem(R), s>>>(g->d_args, g->st, cudaGraphConditionalHandle(),
                                                    (i & 1) ? IT_BENCH_HOLD : IT_BENCH);
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

bf_status bench_block_iter(bf_ctx* ctx, bf_band* b, int R, int reps, double* ms) {
  switch (R) {
    case 8: return bench_blk_t<8>(ctx, b, reps, ms);
    case 16: return bench_blk_t<16>(ctx, b, reps, ms);
    case 32: return bench_blk_t<32>(ctx, b, reps, ms);
  }
  return bf_fail(ctx, BF_EINVAL, "R must be 8, 16 or 32");
}

// One probe vector z_k (the same counter-based Rademacher values as k_probes)
__global__ void k_probe1(int N, const int32_t* __restrict__ lin, uint64_t mseed, int k, float* __restrict__ z) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const uint64_t v = mix64(mseed ^ ((uint64_t)k * 0xD1B54A32D192ED03ULL) ^ (uint64_t)(uint32_t)lin[i]);
    z[i] = (v >> 63) ? -1.0f : 1.0f;
  }
}

// s_acc += z (.) x, sq += (z (.) x)^2 if sq
__global__ void k_hutch1(int N, const float* __restrict__ z, const float* __restrict__ x, double* __restrict__ sacc,
                         double* __restrict__ sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double t = (double)z[i] * (double)x[i];
    sacc[i] += t;
    if (sq) sq[i] += t * t;
  }
}

// The probes one at a time as single right-hand-side solves (the unbatched
// form of the estimator, for comparison with the block solver).
static bf_status variance_single(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                                 int max_iter, float* s_out, int* total_iters, double* sq, double* s1) {
  cudaStream_t s = ctx->stream;
  const int N = (int)b->N;
  float *z = nullptr, *x = nullptr;
  double* sacc = nullptr;
  bf_status r = BF_OK;
  if ((r = dev_alloc_t(ctx, &z, N)) || (r = dev_alloc_t(ctx, &x, N)) || (r = dev_alloc_t(ctx, &sacc, N))) {
    dev_free(s, z);
    dev_free(s, x);
    return r;
  }
  uint64_t mseed = 0;
  {  // host copy of the probe seed mix (same function as the device)
    uint64_t zz = seed + 0x9E3779B97F4A7C15ULL;
    zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ULL;
    zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBULL;
    mseed = zz ^ (zz >> 31);
  }
  int tot = 0;
  if (cudaMemsetAsync(sacc, 0, (size_t)N * 8, s) != cudaSuccess) r = bf_fail(ctx, BF_ECUDA, "memset");
  for (int k = kb; k < ke && r == BF_OK; ++k) {
    k_probe1<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, b->lin, mseed, k, z);
    count_launch();
    int it = 0;
    r = solve_rhs_impl(ctx, b, z, tol, max_iter, x, &it, nullptr);
    tot += it;
    if (r == BF_OK) {
      k_hutch1<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, z, x, sacc, sq);
      count_launch();
    }
  }
  if (r == BF_OK) {
    k_finish<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(N, sacc, scale, s_out);
    count_launch();
    if (s1 && cudaMemcpyAsync(s1, sacc, (size_t)N * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      r = bf_fail(ctx, BF_ECUDA, "copy probe sums");
    if (cudaStreamSynchronize(s) != cudaSuccess) r = bf_fail(ctx, BF_ECUDA, "variance_single");
  }
  dev_free(s, z);
  dev_free(s, x);
  dev_free(s, sacc);
  if (total_iters) *total_iters = tot;
  return r;
}

// probes k in [kb, ke); s = scale * sum_k z_k (.) Q^-1 z_k; sq (device, may be
// null) += sum_k (z_k (.) Q^-1 z_k)^2; s1 (device, may be null) = the FP64 sum
bf_status variance_impl(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                        int max_iter, int R, unsigned flags, float* s, int* total_iters, double* sq, double* s1) {
  (void)flags;
  if (b->N == 0) {
    if (total_iters) *total_iters = 0;
    return BF_OK;
  }
  const int K = ke - kb;
  if (R == 0) BF_TRY(autotune_rhs_block(ctx, b, K, false, &R, nullptr));  // library choice: measured
  if (R == 1) return variance_single(ctx, b, kb, ke, scale, seed, tol, max_iter, s, total_iters, sq, s1);
  switch (R) {
    case 8: return variance_t<8>(ctx, b, kb, ke, scale, seed, tol, max_iter, s, total_iters, sq, s1);
    case 16: return variance_t<16>(ctx, b, kb, ke, scale, seed, tol, max_iter, s, total_iters, sq, s1);
    case 32: return variance_t<32>(ctx, b, kb, ke, scale, seed, tol, max_iter, s, total_iters, sq, s1);
  }
  return bf_fail(ctx, BF_EINVAL, "rhs_block must be 0, 1, 8, 16 or 32");
}

template <int R>
static bf_status spmm_t(bf_ctx* ctx, bf_band* b, const float* X, float* Y) {
  BF_CK(cudaFuncSetAttribute(k_spmm<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp_smem(R)));
  BF_TRY(ensure_sp_plan(ctx, b));
  k_spmm<R><<<blk_ncta<R>(), CT, sp_smem(R), ctx->stream>>>((int)b->N, (float)b->prm.lambda, b->qd, b->nb6, b->sp_ext,
                                                   b->sp_ne, b->sp_slot, X, Y);
  count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}

bf_status spmm_launch(bf_ctx* ctx, bf_band* b, const float* X, int R, float* Y) {
  if (b->N == 0) return BF_OK;
  switch (R) {
    case 8: return spmm_t<8>(ctx, b, X, Y);
    case 16: return spmm_t<16>(ctx, b, X, Y);
    case 32: return spmm_t<32>(ctx, b, X, Y);
    default: return bf_fail(ctx, BF_EINVAL, "bf_spmm: R must be 8, 16 or 32");
  }
}
