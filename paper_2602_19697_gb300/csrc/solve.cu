// Matrix-free 7-point SpMV and Jacobi-PCG for the MAP mean (Sec. 3.6 MAP
// equation, solved by PCG; Algorithm 1 step 5).
//
// Brick tiles.  Band vectors are compact ([N], brick-ordered).  A 128-thread
// CTA handles one active 8^3 brick at a time (CTAs stride over the bricks):
// it stages the brick's voxels and the facing layers of its six neighbour
// bricks into a 10^3 shared-memory tile (non-band slots hold 0, so the
// stencil needs no masks) and applies
//   (Qx)_j = Q_jj x_j - lambda * (sum of the six tile neighbours).
//
// PCG.  The single-reduction form (Chronopoulos & Gear, 1989), one fused
// kernel per iteration:
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,
//   u = r / Q_jj,    w = Q u,         gamma = r.u,   delta = w.u,   r.r
// (s = Q p is carried by recurrence, so Q is applied once, to u).  The tile
// holds u, recomputed for halo voxels from their r, w, s; r, w, s ping-pong
// between two buffers because the halo needs their old values.  Each CTA
// writes FP64 partial sums; the last CTA to finish reduces them in a fixed
// order (deterministic) and sets
//   beta' = gamma'/gamma,  alpha' = gamma' / (delta' - beta' gamma'/alpha)
// and the stop flag.  The iteration loop is a CUDA-graph WHILE node (two
// iterations per body) that the kernels end from the device.
//
// Refinement.  FP64 master iterate x64: k_outer computes the true residual
// h - Q x64 with FP64 arithmetic; the correction solve (FP32 vectors, or FP64
// with BF_SOLVE_FP64) reduces it by eta = 0.5 tol |h| / |r| (clamped); x64 +=
// x; repeat until the true residual meets the tolerance.
//
// The solver belongs to the context (one per precision): kernels read the
// band and workspace pointers from a device-resident argument block, so the
// captured graph serves every band.
#include <cstring>

#include "internal.cuh"

namespace {

constexpr int BT = 128;             // threads per brick CTA
constexpr int NCTA = 152 * 8;       // brick CTAs (strided over the bricks)

struct PcgState {
  double alpha, beta, gamma, rr, bb, tol2;  // correction solve
  double rr0, bb0, tol0, eta_min;           // true residual, |h|^2, requested tolerance
  int iter, max_iter, done, status;
  unsigned int cnt, guard;
  unsigned int nexec;  // graph-body kernels executed (for launch accounting)
};

template <class T>
struct SolveArgs {
  BandView B;
  float lam;
  const float* qd;
  const float* rhs;
  T* r[2];
  T* w[2];
  T* s[2];
  T* p;
  T* x;
  double* x64;
  double* part;  // [3][NCTA]
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sums of NV doubles -> part[k][blockIdx.x]; returns true in the
// last CTA to arrive, after which every partial is visible
template <int NV>
__device__ __forceinline__ bool publish(double (&v)[NV], double* part, unsigned int* counter) {
  __shared__ double sh[NV][BT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
      for (int q = 0; q < BT / 32; ++q) s += sh[k][q];
      part[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// fixed-order sums of the partials (one warp per quantity), valid in all threads
template <int NV>
__device__ __forceinline__ void gather(const double* part, double (&tot)[NV]) {
  __shared__ double sh[NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < NV; k += BT / 32) {
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
    s = warp_sum(s);
    if (lane == 0) sh[k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = sh[k];
}

// brick metadata of brick b and its six face neighbours
__device__ __forceinline__ void load_meta(const BandView& B, int b, MetaWord (*sm)[16]) {
  const int tid = threadIdx.x;
  if (tid < 7 * 16) {
    int which = tid >> 4, w = tid & 15;
    int r = which == 0 ? b : __ldg(B.nbr + 6 * b + which - 1);
    MetaWord m;
    m.bits = 0;
    m.base = 0;
    if (r >= 0) m = B.meta[16 * r + w];
    sm[which][w] = m;
  }
}

__device__ __forceinline__ int own_tile(int l) { return (l & 7) + 1 + 10 * (((l >> 3) & 7) + 1) + 100 * ((l >> 6) + 1); }

__device__ __forceinline__ int slot_index(const MetaWord (*sm)[16], int which, int l) {
  MetaWord m = sm[which][l >> 5];
  uint32_t bit = 1u << (l & 31);
  return (m.bits & bit) ? m.base + __popc(m.bits & (bit - 1u)) : -1;
}

// halo slot q in [0, 384): compact index of the neighbour voxel (or -1) and
// its position in the tile
__device__ __forceinline__ void halo_slot(const MetaWord (*sm)[16], int q, int* idx, int* tpos) {
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
  *idx = slot_index(sm, 1 + f, lc[0] + 8 * lc[1] + 64 * lc[2]);
  *tpos = tc[0] + 10 * tc[1] + 100 * tc[2];
}

template <class T>
__device__ __forceinline__ T nsum(const T* t, int c) {
  return ((t[c - 1] + t[c + 1]) + (t[c - 10] + t[c + 10])) + (t[c - 100] + t[c + 100]);
}

// y = Q x (plain SpMV, FP32) for x not on a 16-byte boundary (k_spmv_t below
// takes aligned arrays).  A CTA walks bricks b, b + grid, ...; the x
// and Q_jj loads of the next brick are issued while the current brick is
// formed, its lookup words (own and six neighbours) one brick earlier and the
// neighbour ranks one brick earlier still, so no round trip to memory is
// waited for in the steady state.
constexpr int SPMV_OCC = 8;  // resident CTAs per SM (64 registers x 128 threads)
constexpr int CG_OCC = 8, CG_NCTA = 152 * CG_OCC;  // k_cg: resident CTAs per SM, grid

// rank of brick b (thread's slot 0) or of its face neighbour (slots 1-6); -1 if none
__device__ __forceinline__ int meta_rank(const BandView& B, int b) {
  const int which = threadIdx.x >> 4;
  if (b >= B.NB || threadIdx.x >= 7 * 16) return -1;
  return which == 0 ? b : __ldg(B.nbr + 6 * b + which - 1);
}
__device__ __forceinline__ MetaWord meta_word(const BandView& B, int r) {
  MetaWord m;
  m.bits = 0;
  m.base = 0;
  if (r >= 0) m = B.meta[16 * r + (threadIdx.x & 15)];
  return m;
}

// The SpMV tile: pitch 24 in x (own lx at x = lx + 4, so a thread's four
// voxels are one aligned float4 and eight lanes' float4 fall in distinct
// banks), 10 rows in y (own ly at ly + 1) and 10 planes of pitch 248 in z (own
// lz at lz + 1; 248 = 24 mod 32, so that a warp's stores of a y face hit 32
// distinct banks).  The -x and +x halo faces, whose tile positions would all
// be congruent mod 8, sit in a separate array hx[side][z][y] of side pitch 80
// instead.  Halo face f at face coordinates (u, v): local index in the
// neighbour brick [0] + u [1] + v [2], position [3] + u [4] + v [5] in hx
// (faces -x, +x) or in the tile (faces -y, +y, -z, +z); (u, v) are the two
// other axes in increasing order.
constexpr int SP_PY = 24, SP_PZ = 248, SP_TILE = 10 * SP_PZ, SP_HX = 80;
__constant__ int c_halo24[6][6] = {
    {7, 8, 64, 0, 1, 8},        {0, 8, 64, SP_HX, 1, 8},    {56, 1, 64, 4 + SP_PZ, 1, SP_PZ},
    {0, 1, 64, 4 + 9 * SP_PY + SP_PZ, 1, SP_PZ},          {448, 1, 8, 4 + SP_PY, 1, SP_PY},
    {0, 1, 8, 4 + SP_PY + 9 * SP_PZ, 1, SP_PY},
};

// Loads of one brick, issued one brick ahead of their use.  Thread t owns
// local indices 4t .. 4t+3 (one lookup word, one x-row).
struct SpmvLoads {
  int i0;       // compact index of the first present voxel of the four
  uint32_t m4;  // presence bits of the four voxels
  float4 xv, q;
  float hv[3];
  int tp[3];
};

__device__ __forceinline__ void spmv_issue(const MetaWord (*sm)[16], const float* __restrict__ x,
                                           const float* __restrict__ qd, SpmvLoads& L) {
  const int l0 = 4 * threadIdx.x;
  const MetaWord m = sm[0][l0 >> 5];
  L.m4 = (m.bits >> (l0 & 31)) & 0xFu;
  L.i0 = m.base + __popc(m.bits & ((1u << (l0 & 31)) - 1u));
  float xs[4], qs[4];
  int i = L.i0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const bool on = (L.m4 >> s) & 1u;
    xs[s] = on ? __ldg(x + i) : 0.0f;
    qs[s] = on ? __ldg(qd + i) : 0.0f;
    i += on;
  }
  L.xv = make_float4(xs[0], xs[1], xs[2], xs[3]);
  L.q = make_float4(qs[0], qs[1], qs[2], qs[3]);
#pragma unroll
  for (int s = 0; s < 3; ++s) {  // halo: slot h = face f (warp-uniform), face coordinates (u, v)
    const int h = threadIdx.x + BT * s, f = h >> 6, u = h & 7, v = (h >> 3) & 7;
    const int j = slot_index(sm, 1 + f, c_halo24[f][0] + u * c_halo24[f][1] + v * c_halo24[f][2]);
    L.tp[s] = c_halo24[f][3] + u * c_halo24[f][4] + v * c_halo24[f][5];
    L.hv[s] = j >= 0 ? __ldg(x + j) : 0.0f;
  }
}


// Software pipeline over the CTA's bricks b0, b1 = b0 + grid, ...: in the
// iteration of brick b_i the tile receives b_i's values (loaded during the
// previous iteration), the loads of b_{i+1} are issued (its lookup words
// fetched one iteration earlier still), and y of b_i is formed, four voxels
// per thread from float4 reads of the tile; the neighbour sum keeps the
// order ((x-1 + x+1) + (y-1 + y+1)) + (z-1 + z+1).
__global__ void __launch_bounds__(BT, SPMV_OCC) k_spmv(BandView B, float lam, const float* __restrict__ qd,
                                                       const float* __restrict__ x, float* __restrict__ y) {
  __shared__ __align__(16) float tile[SP_TILE];
  __shared__ float hx[2 * SP_HX];
  __shared__ MetaWord sm[2][7][16];
  const int g = gridDim.x;
  if (threadIdx.x < 7 * 16) sm[0][threadIdx.x >> 4][threadIdx.x & 15] = meta_word(B, meta_rank(B, blockIdx.x));
  MetaWord nm = meta_word(B, meta_rank(B, blockIdx.x + g));  // lookup words of b_1
  int nr = meta_rank(B, blockIdx.x + 2 * g);                   // ranks for b_2
  __syncthreads();
  SpmvLoads cur, nxt;
  if ((int)blockIdx.x < B.NB) spmv_issue(sm[0], x, qd, cur);
  // x and Q_jj of the brick two ahead are prefetched into L2 as whole lines (its range one iteration earlier)
  int2 pr = make_int2(0, 0);
  if (threadIdx.x == 0 && (int)blockIdx.x + 2 * g < B.NB)
    pr = make_int2(__ldg(B.off + blockIdx.x + 2 * g), __ldg(B.off + blockIdx.x + 2 * g + 1));
  const int l0 = 4 * threadIdx.x;
  const int t0 = ((l0 & 7) + 4) + SP_PY * (((l0 >> 3) & 7) + 1) + SP_PZ * ((l0 >> 6) + 1);
  // -x (lx = 0 threads) or +x (lx = 4 threads) halo value of the thread's row
  const int xside = (l0 >> 2) & 1, hxi = xside * SP_HX + 8 * (l0 >> 6) + ((l0 >> 3) & 7);
  int it = 0;
  for (int b = blockIdx.x; b < B.NB; b += g, ++it) {
    if (threadIdx.x == 0) {
      if (pr.y > pr.x) {
        prefetch_range(x, pr.x, pr.y);
        prefetch_range(qd, pr.x, pr.y);
      }
      const int bn = b + 3 * g;
      pr = bn < B.NB ? make_int2(__ldg(B.off + bn), __ldg(B.off + bn + 1)) : make_int2(0, 0);
    }
    const int pn = (it + 1) & 1;
    // tile <- b's values; lookup words of the next brick into the other buffer
    *reinterpret_cast<float4*>(tile + t0) = cur.xv;
    hx[cur.tp[0]] = cur.hv[0];  // slots 0 .. BT-1 are the two x faces
#pragma unroll
    for (int s = 1; s < 3; ++s) tile[cur.tp[s]] = cur.hv[s];
    if (threadIdx.x < 7 * 16) sm[pn][threadIdx.x >> 4][threadIdx.x & 15] = nm;
    __syncthreads();
    if (b + g < B.NB) spmv_issue(sm[pn], x, qd, nxt);
    nm = meta_word(B, nr);
    nr = meta_rank(B, b + 3 * g);
    // own values as this thread stored them; the in-row x neighbours come from the lane holding the
    // other half of the row (lane ^ 1)
    const float4 c = cur.xv;
    const float xo = __shfl_xor_sync(0xffffffffu, xside ? c.x : c.w, 1);
    if (cur.m4) {
      const float xh = hx[hxi];
      const float xl = xside ? xo : xh, xr = xside ? xh : xo;
      const float4 ym = *reinterpret_cast<const float4*>(tile + t0 - SP_PY);
      const float4 yp = *reinterpret_cast<const float4*>(tile + t0 + SP_PY);
      const float4 zm = *reinterpret_cast<const float4*>(tile + t0 - SP_PZ);
      const float4 zp = *reinterpret_cast<const float4*>(tile + t0 + SP_PZ);
      const float xm[4] = {xl, c.x, c.y, c.z}, xp[4] = {c.y, c.z, c.w, xr};
      const float cc[4] = {c.x, c.y, c.z, c.w}, qq[4] = {cur.q.x, cur.q.y, cur.q.z, cur.q.w};
      const float ym4[4] = {ym.x, ym.y, ym.z, ym.w}, yp4[4] = {yp.x, yp.y, yp.z, yp.w};
      const float zm4[4] = {zm.x, zm.y, zm.z, zm.w}, zp4[4] = {zp.x, zp.y, zp.z, zp.w};
      int i = cur.i0;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if ((cur.m4 >> s) & 1u) {
          const float ns = ((xm[s] + xp[s]) + (ym4[s] + yp4[s])) + (zm4[s] + zp4[s]);
          y[i] = qq[s] * cc[s] - lam * ns;
          ++i;
        }
      }
    }
    __syncthreads();  // tile and this iteration's lookup buffer are free again
    cur = nxt;
  }
}

// y = Q x (plain SpMV, FP32), one warp per brick, the brick's runs staged by
// bulk copies.  Lane (lx, q) = lx + 8 q holds the brick's 16 voxels (lx, q +
// 4 h, lz), slot s = 2 lz + h, i.e. local index lane + 32 s: slot s is exactly
// lookup word s, so the lane's rank in the brick's compact run is (word base
// - run start) + popc(bits below the lane), and the present lanes of a slot
// read consecutive words of the staged run (no bank conflicts) and store a
// contiguous run of y.  The z neighbours are the lane's own slots s -+ 2; the
// x and y neighbours come by shuffles in the warp, the lane at the end of a
// row or column handing out the neighbour brick's face value in place of its
// own; the faces are gathered packed (64 values of a face pair per load) from
// global memory and handed to the end lanes by one more shuffle.
//
// Each warp walks bricks b, b + W, ... (W warps in the grid): while brick b_i
// is formed, lane 0 arms the other buffer's mbarrier and lanes 0-8 issue the
// bulk copies of b_{i+1}: its x and Q_jj runs (from the 16-byte granule at or
// below the run start up to the granule end at or above the run end, clipped
// to the last whole granule of the arrays; the clipped tail is read directly)
// and the 128-byte lookup blocks of the brick and of its six face neighbours
// (zeros for a missing one); the neighbour ranks and run bounds of b_{i+2} are
// loaded into registers.  A wait that runs out sets *err and ends the warp
// after its copies in flight have landed (or a second wait has run out).
constexpr int SPT = 4;        // warps per CTA
constexpr int SPT_OCC = 4;    // resident CTAs per SM (124 registers)
constexpr int SPT_RUN = 528;  // staged run capacity (floats): 512 + two granule slacks, 16-byte multiple

struct __align__(16) SptBuf {
  float xr[2][SPT_RUN];
  float qr[2][SPT_RUN];
  MetaWord m[2][7][16];  // the brick (0) and its face neighbours -x, +x, -y, +y, -z, +z (1-6)
  uint64_t bar[2];
};

// lanes 0-5: face neighbour ranks of brick b; lanes 6, 7: its run bounds off[b], off[b + 1]
__device__ __forceinline__ int spw_ranks(const BandView& B, int b, int lane) {
  if (b >= B.NB || lane >= 8) return -1;
  return lane < 6 ? __ldg(B.nbr + 6 * b + lane) : __ldg(B.off + b + lane - 6);
}

__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          (uint32_t)__cvta_generic_to_shared(sdst)),
      "l"(gsrc), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
      : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// stage brick b (ranks and run bounds in lanes 0-7 of rk) into buffer k
__device__ __forceinline__ void spt_stage(const BandView& B, int b, int rk, SptBuf& S, int k,
                                          const float* __restrict__ x, const float* __restrict__ qd, int nfl,
                                          int lane) {
  const int o0 = __shfl_sync(0xffffffffu, rk, 6), o1 = __shfl_sync(0xffffffffu, rk, 7);
  const int a0 = o0 & ~3, a1 = min((o1 + 3) & ~3, nfl);
  const uint32_t bytes = a1 > a0 ? 4u * (uint32_t)(a1 - a0) : 0u;
  // lanes 2-8: lookup block j = lane - 2 (the brick, then its neighbours from lanes 0-5 of rk)
  const int j = lane - 2;
  const int rj = __shfl_sync(0xffffffffu, rk, (j - 1) & 31);
  const int r = j == 0 ? b : rj;
  const bool meta_copy = lane >= 2 && lane < 9 && r >= 0;
  const uint32_t nmeta = __popc(__ballot_sync(0xffffffffu, meta_copy));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the buffer before the copies
  if (lane == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&S.bar[k])),
                 "r"(2u * bytes + 128u * nmeta)
                 : "memory");
  if (lane < 2 && bytes) bulk_g2s(lane ? S.qr[k] : S.xr[k], (lane ? qd : x) + a0, bytes, &S.bar[k]);
  if (meta_copy) bulk_g2s(S.m[k][j], B.meta + 16 * (size_t)r, 128u, &S.bar[k]);
  if (lane >= 2 && lane < 9 && r < 0) {
    int4* d = reinterpret_cast<int4*>(S.m[k][j]);
#pragma unroll
    for (int c = 0; c < 8; ++c) d[c] = make_int4(0, 0, 0, 0);
  }
}

// value of x at local index 32 w + bit of the staged brick m16 (0 outside the band)
__device__ __forceinline__ float face_x(const MetaWord* m16, const float* __restrict__ x, int w, int bit) {
  const MetaWord m = m16[w];
  return (m.bits >> bit) & 1u ? __ldg(x + m.base + __popc(m.bits & ((1u << bit) - 1u))) : 0.0f;
}

// One brick of k_spmv_t from its staged runs xr, qr (xr[0] = the run's first
// voxel) and lookup words M[7][16]; o0 = the run start.  FULLB: all 512
// voxels in the band, so slot s of the lane is run element lane + 32 s (no
// rank arithmetic, no presence tests); otherwise the lane's rank in the run is
// found from the slot's word, and a slot whose word is empty is skipped.
template <bool FULLB>
__device__ __forceinline__ void spt_brick(const MetaWord (*M)[16], const float* xr, const float* qr, int o0,
                                          const float* __restrict__ x, float* __restrict__ y, float lam) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, lx = lane & 7, q = lane >> 3;
  const uint32_t below = (1u << lane) - 1u;
  const int pside = lane >> 4, pc = lane & 7, pz = (lane >> 3) & 1;
  const int sxm = (lane & 24) | ((lane - 1) & 7), sxp = (lane & 24) | ((lane + 1) & 7);
  const int sym = (lane - 8) & 31, syp = (lane + 8) & 31;
  const int sxf = (lx == 0 ? 16 : 0) + q, syf = (q == 0 ? 16 : 0) + lx;
  int ix[16];  // rank of the lane's voxel in the run, or -1
  float v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    if (FULLB) {
      ix[s] = lane + 32 * s;
      v[s] = xr[ix[s]];
    } else {
      const MetaWord m = M[0][s];
      ix[s] = (m.bits >> lane) & 1u ? m.base - o0 + __popc(m.bits & below) : -1;
      v[s] = ix[s] >= 0 ? xr[ix[s]] : 0.0f;
    }
  }
  // -z neighbour's plane lz = 7 (words 14, 15) and +z neighbour's plane 0 (words 0, 1), the lane's own (lx, ly)
  float zf[4];
  zf[0] = face_x(M[5], x, 14, lane);
  zf[1] = face_x(M[5], x, 15, lane);
  zf[2] = face_x(M[6], x, 0, lane);
  zf[3] = face_x(M[6], x, 1, lane);
  float XF[4], YF[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int lz = 2 * k + pz;
    // x faces: local (7 or 0) + 8 ly + 64 lz with ly = pc: word 2 lz + (ly >> 2), bit (7 or 0) + 8 (ly & 3)
    XF[k] = face_x(M[1 + pside], x, 2 * lz + (pc >> 2), (pside ? 0 : 7) + 8 * (pc & 3));
    // y faces: local lx + 8 (7 or 0) + 64 lz with lx = pc: word 2 lz + (1 or 0), bit lx + (24 or 0)
    YF[k] = face_x(M[3 + pside], x, 2 * lz + (pside ? 0 : 1), pc + (pside ? 0 : 24));
  }
#pragma unroll
  for (int lz = 0; lz < 8; ++lz) {
    // lanes q = 3 receive the -y face value (lx, lz), lanes q = 0 the +y one
    const float yfv = __shfl_sync(FULL, YF[lz >> 1], syf + 8 * (lz & 1));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = 2 * lz + h;
      if (!FULLB && M[0][s].bits == 0u) continue;  // no band voxel in this slot (warp-uniform)
      const float c = v[s];
      // lanes lx = 7 receive the -x face value (ly = q + 4h, lz), lanes lx = 0 the +x one
      const float xfv = __shfl_sync(FULL, XF[lz >> 1], sxf + 8 * (lz & 1) + 4 * h);
      const float xm = __shfl_sync(FULL, lx == 7 ? xfv : c, sxm);
      const float xp = __shfl_sync(FULL, lx == 0 ? xfv : c, sxp);
      // ly - 1 of lane q = 0 is lane q = 3 of the other half (h = 1) or the -y face (h = 0)
      const float ym = __shfl_sync(FULL, q == 3 ? (h == 0 ? yfv : v[s - h]) : c, sym);
      // ly + 1 of lane q = 3 is lane q = 0 of the other half (h = 0) or the +y face (h = 1)
      const float yp = __shfl_sync(FULL, q == 0 ? (h == 0 ? v[s + 1 - h] : yfv) : c, syp);
      const float zm = lz > 0 ? v[s - 2 * (lz > 0)] : zf[h];
      const float zp = lz < 7 ? v[s + 2 * (lz < 7)] : zf[2 + h];
      const float ns = ((xm + xp) + (ym + yp)) + (zm + zp);
      if (FULLB || ix[s] >= 0) y[o0 + ix[s]] = qr[ix[s]] * c - lam * ns;
    }
  }
}

__global__ void __launch_bounds__(32 * SPT, SPT_OCC) k_spmv_t(BandView B, float lam, const float* __restrict__ qd,
                                                               const float* __restrict__ x, float* __restrict__ y,
                                                               int nfl, int* __restrict__ err) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ SptBuf sbuf[SPT];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int nw = gridDim.x * SPT;
  SptBuf& S = sbuf[wi];
  int b = blockIdx.x * SPT + wi;
  if (b >= B.NB) return;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&S.bar[k]))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  int rk = spw_ranks(B, b, lane);
  spt_stage(B, b, rk, S, 0, x, qd, nfl, lane);
  int o0 = __shfl_sync(FULL, rk, 6), o1 = __shfl_sync(FULL, rk, 7);  // run of the brick being formed
  rk = spw_ranks(B, b + nw, lane);
  for (int it = 0; b < B.NB; b += nw, ++it) {
    const int cur = it & 1, bn = b + nw;
    const int n0 = __shfl_sync(FULL, rk, 6), n1 = __shfl_sync(FULL, rk, 7);
    if (bn < B.NB) spt_stage(B, bn, rk, S, cur ^ 1, x, qd, nfl, lane);
    rk = spw_ranks(B, bn + nw, lane);
    if (!bar_wait(&S.bar[cur], (uint32_t)(it >> 1) & 1u)) {
      if (lane == 0) atomicOr(err, 1);
      bar_wait(&S.bar[cur], (uint32_t)(it >> 1) & 1u);
      if (bn < B.NB) bar_wait(&S.bar[cur ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
      return;
    }
    const int a0 = o0 & ~3, a1 = min((o1 + 3) & ~3, nfl);
    if (o1 > a1) {  // the run reaches past the last whole granule: its tail read directly
      const int t = max(a1, o0) + lane;
      if (t < o1) {
        S.xr[cur][t - a0] = __ldg(x + t);
        S.qr[cur][t - a0] = __ldg(qd + t);
      }
      __syncwarp();
    }
    if (o1 - o0 == 512)
      spt_brick<true>(S.m[cur], S.xr[cur] + (o0 - a0), S.qr[cur] + (o0 - a0), o0, x, y, lam);
    else
      spt_brick<false>(S.m[cur], S.xr[cur] + (o0 - a0), S.qr[cur] + (o0 - a0), o0, x, y, lam);
    o0 = n0;
    o1 = n1;
    __syncwarp();  // the buffer of b_i is free for b_{i+2}
  }
}

// True residual of the FP64 master iterate: r[0] = h - Q x64 (FP64), r.r and
// h.h; the last CTA sets the stop flag and the correction target eta.  ZERO:
// x64 is zero (a cold start), so r = h, read row by row without the SpMV.
template <class T, bool ZERO = false>
__global__ void __launch_bounds__(BT) k_outer(const SolveArgs<T>* __restrict__ A, PcgState* st) {
  __shared__ double tile[1000];
  __shared__ MetaWord sm[7][16];
  const BandView& B = A->B;
  const double* __restrict__ x64 = A->x64;
  double acc[2] = {0.0, 0.0};
  if (ZERO) {
    for (int i = blockIdx.x * BT + threadIdx.x; i < B.N; i += gridDim.x * BT) {
      const double h = (double)__ldg(A->rhs + i);
      A->r[0][i] = (T)h;
      acc[0] += h * h;
      acc[1] += h * h;
    }
  }
  for (int b = ZERO ? B.NB : blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
    load_meta(B, b, sm);
    __syncthreads();
    int idx[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = threadIdx.x + BT * s;
      idx[s] = slot_index(sm, 0, l);
      tile[own_tile(l)] = idx[s] >= 0 ? x64[idx[s]] : 0.0;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int j, tp;
      halo_slot(sm, threadIdx.x + BT * s, &j, &tp);
      tile[tp] = j >= 0 ? x64[j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (idx[s] < 0) continue;
      int c = own_tile(threadIdx.x + BT * s);
      const double h = (double)__ldg(A->rhs + idx[s]);
      const double r = h - ((double)__ldg(A->qd + idx[s]) * tile[c] - (double)A->lam * nsum(tile, c));
      A->r[0][idx[s]] = (T)r;
      acc[0] += r * r;
      acc[1] += h * h;
    }
  }
  if (!publish<2>(acc, A->part, &st->cnt)) return;
  double tot[2];
  gather<2>(A->part, tot);
  if (threadIdx.x == 0) {
    const double rr = tot[0], bb = tot[1];
    st->rr0 = rr;
    st->bb0 = bb;
    st->bb = rr;
    const int conv = rr <= st->tol0 * st->tol0 * bb || bb == 0.0;
    double eta = conv ? 0.5 : 0.5 * st->tol0 * sqrt(bb / rr);
    eta = fmin(fmax(eta, st->eta_min), 0.5);
    st->tol2 = eta * eta;
    if (conv) st->status = 0;
    else if (st->iter >= st->max_iter) st->status = 1;
    st->done = conv || st->iter >= st->max_iter || st->status == 2;
    st->cnt = 0;
    st->guard = 0;
  }
}

// Correction-solve start: u = r/qd, w = Q u, p = s = x = 0, gamma = r.u,
// delta = w.u; alpha = gamma/delta.
template <class T>
__global__ void __launch_bounds__(BT) k_cg_init(const SolveArgs<T>* __restrict__ A, PcgState* st) {
  if (st->done) return;  // the true residual already met the tolerance: no correction solve follows
  __shared__ T tile[1000];
  __shared__ MetaWord sm[7][16];
  const BandView& B = A->B;
  const T* __restrict__ r = A->r[0];
  double acc[2] = {0.0, 0.0};
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
    load_meta(B, b, sm);
    __syncthreads();
    int idx[4];
    T uo[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = threadIdx.x + BT * s;
      idx[s] = slot_index(sm, 0, l);
      uo[s] = idx[s] >= 0 ? r[idx[s]] / (T)__ldg(A->qd + idx[s]) : (T)0;
      tile[own_tile(l)] = uo[s];
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int j, tp;
      halo_slot(sm, threadIdx.x + BT * s, &j, &tp);
      tile[tp] = j >= 0 ? r[j] / (T)__ldg(A->qd + j) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (idx[s] < 0) continue;
      int c = own_tile(threadIdx.x + BT * s);
      const T wi = (T)__ldg(A->qd + idx[s]) * uo[s] - (T)A->lam * nsum(tile, c);
      A->w[0][idx[s]] = wi;
      A->s[0][idx[s]] = (T)0;
      A->p[idx[s]] = (T)0;
      A->x[idx[s]] = (T)0;
      acc[0] += (double)r[idx[s]] * (double)uo[s];
      acc[1] += (double)wi * (double)uo[s];
    }
  }
  if (!publish<2>(acc, A->part, &st->cnt)) return;
  double tot[2];
  gather<2>(A->part, tot);
  if (threadIdx.x == 0) {
    const double g = tot[0], d = tot[1];
    st->gamma = g;
    st->beta = 0.0;
    if (!st->done && (!(d > 0.0) || !isfinite(d) || !isfinite(g))) {
      st->status = 2;
      st->done = 1;
    }
    st->alpha = st->done ? 0.0 : g / d;
    st->cnt = 0;
    st->guard = 0;
  }
}

// One single-reduction PCG iteration (see the file comment); (r, w, s) read
// from buffer `in`, written to buffer 1 - in; p, x in place.
template <class T>
__global__ void __launch_bounds__(BT, CG_OCC) k_cg(const SolveArgs<T>* __restrict__ A, int in, PcgState* st,
                                                  cudaGraphConditionalHandle handle) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->nexec += 1;
    unsigned g = atomicAdd(&st->guard, 1u);
    if (st->done || g > 2u * (unsigned)st->max_iter + 64u) {
      if (!st->done) {
        st->status = 1;
        st->done = 1;
      }
      cudaGraphSetConditional(handle, 0);
    }
  }
  if (st->done) return;
  __shared__ T tile[1000];
  __shared__ MetaWord sm[7][16];
  const BandView& B = A->B;
  const T a = (T)st->alpha, bt = (T)st->beta;
  const T* __restrict__ r_in = A->r[in];
  const T* __restrict__ w_in = A->w[in];
  const T* __restrict__ s_in = A->s[in];
  T* __restrict__ r_out = A->r[in ^ 1];
  T* __restrict__ w_out = A->w[in ^ 1];
  T* __restrict__ s_out = A->s[in ^ 1];
  T* __restrict__ p = A->p;
  T* __restrict__ x = A->x;
  const float* __restrict__ qd = A->qd;
  // inner products: per-brick partial sums in T, accumulated in FP64
  double acc[3] = {0.0, 0.0, 0.0};
  // lookup words of the next brick fetched during the current one (as in k_spmv)
  MetaWord nm = meta_word(B, meta_rank(B, blockIdx.x));
  int nr = meta_rank(B, blockIdx.x + gridDim.x);
  // threads 0-5: the run bounds of the next brick, whose runs of r, w, s, p, x and Q_jj they prefetch into L2
  // while this brick is formed (the bounds of the brick after it loaded meanwhile)
  int2 pr = make_int2(0, 0);
  if (threadIdx.x < 6 && (int)(blockIdx.x + gridDim.x) < B.NB)
    pr = make_int2(__ldg(B.off + blockIdx.x + gridDim.x), __ldg(B.off + blockIdx.x + gridDim.x + 1));
  for (int b = blockIdx.x; b < B.NB; b += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < 7 * 16) sm[threadIdx.x >> 4][threadIdx.x & 15] = nm;
    __syncthreads();
    nm = meta_word(B, nr);
    nr = meta_rank(B, b + 2 * gridDim.x);
    if (threadIdx.x < 6) {
      if (pr.y > pr.x) {
        const int t = threadIdx.x;
        if (t < 5)
          prefetch_range(t == 0 ? r_in : t == 1 ? w_in : t == 2 ? s_in : t == 3 ? (const T*)p : (const T*)x, pr.x, pr.y);
        else
          prefetch_range(qd, pr.x, pr.y);
      }
      const int bn2 = b + 2 * gridDim.x;
      pr = bn2 < B.NB ? make_int2(__ldg(B.off + bn2), __ldg(B.off + bn2 + 1)) : make_int2(0, 0);
    }
    int idx[4];
    T rn[4], un[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int l = threadIdx.x + BT * s;
      idx[s] = slot_index(sm, 0, l);
      rn[s] = un[s] = (T)0;
      if (idx[s] >= 0) {
        const int i = idx[s];
        const T iq = (T)1 / (T)__ldg(qd + i);
        const T ri = r_in[i], sn = w_in[i] + bt * s_in[i];
        const T pn = ri * iq + bt * p[i];
        rn[s] = ri - a * sn;
        un[s] = rn[s] * iq;
        p[i] = pn;
        x[i] = x[i] + a * pn;
        s_out[i] = sn;
        r_out[i] = rn[s];
      }
      tile[own_tile(l)] = un[s];
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      int j, tp;
      halo_slot(sm, threadIdx.x + BT * s, &j, &tp);
      T u = (T)0;
      if (j >= 0) u = (r_in[j] - a * (w_in[j] + bt * s_in[j])) / (T)__ldg(qd + j);
      tile[tp] = u;
    }
    __syncthreads();
    T fa0 = 0, fa1 = 0, fa2 = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (idx[s] < 0) continue;
      const int c = own_tile(threadIdx.x + BT * s);
      const T wn = (T)__ldg(qd + idx[s]) * un[s] - (T)A->lam * nsum(tile, c);
      w_out[idx[s]] = wn;
      fa0 += rn[s] * un[s];
      fa1 += wn * un[s];
      fa2 += rn[s] * rn[s];
    }
    acc[0] += (double)fa0;
    acc[1] += (double)fa1;
    acc[2] += (double)fa2;
  }
  if (!publish<3>(acc, A->part, &st->cnt)) return;
  double tot[3];
  gather<3>(A->part, tot);
  if (threadIdx.x == 0) {
    const double g = tot[0], d = tot[1], rr = tot[2];
    st->iter += 1;
    st->rr = rr;
    if (!isfinite(g) || !isfinite(d) || !isfinite(rr)) {
      st->status = 2;
      st->done = 1;
    } else if (rr <= st->tol2 * st->bb) {
      st->done = 1;
    } else if (st->iter >= st->max_iter) {
      st->status = 1;
      st->done = 1;
    } else {
      const double beta = g / st->gamma;
      const double den = d - beta * g / st->alpha;
      if (!(den > 0.0) || !isfinite(den)) {
        st->status = 2;
        st->done = 1;
      } else {
        st->beta = beta;
        st->alpha = g / den;
        st->gamma = g;
      }
    }
    st->cnt = 0;
    if (st->done) cudaGraphSetConditional(handle, 0);
  }
}

template <class T>
__global__ void k_axpy(int N, const T* __restrict__ d, double* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) x[i] += (double)d[i];
}

__global__ void k_cast_out(int N, const double* __restrict__ x, float* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = (float)x[i];
}

__global__ void k_cast_in(int N, const float* __restrict__ x, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = (double)x[i];
}

__global__ void k_state_init(PcgState* st, double tol, int max_iter, double eta_min) {
  st->tol0 = tol;
  st->eta_min = eta_min;
  st->max_iter = max_iter;
  st->iter = 0;
  st->status = 0;
  st->done = 0;
  st->alpha = st->beta = 0.0;
  st->cnt = 0;
  st->guard = 0;
  st->nexec = 0;
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

struct SolveGraph {
  bool fp64 = false;
  int64_t cap = 0;
  SolveArgs<float> hf;
  SolveArgs<double> hd;
  void* h_pin = nullptr;   // pinned staging of the argument block
  void* d_args = nullptr;
  PcgState* st = nullptr;
  PcgState* h_st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capstream = nullptr;
};

template <class T>
static SolveArgs<T>& host_args(SolveGraph* g);
template <>
SolveArgs<float>& host_args<float>(SolveGraph* g) { return g->hf; }
template <>
SolveArgs<double>& host_args<double>(SolveGraph* g) { return g->hd; }

template <class T>
static void free_arrays(SolveGraph* g) {
  SolveArgs<T>& h = host_args<T>(g);
  void* ptrs[] = {h.r[0], h.r[1], h.w[0], h.w[1], h.s[0], h.s[1], h.p, h.x, h.x64, h.part};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  memset(&h, 0, sizeof(h));
  g->cap = 0;
}

void solve_graph_free(SolveGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->capstream) cudaStreamDestroy(g->capstream);
  if (g->fp64) free_arrays<double>(g);
  else free_arrays<float>(g);
  if (g->d_args) cudaFree(g->d_args);
  if (g->st) cudaFree(g->st);
  if (g->h_st) cudaFreeHost(g->h_st);
  if (g->h_pin) cudaFreeHost(g->h_pin);
  delete g;
}

template <class T>
static bf_status get_solver(bf_ctx* ctx, bf_band* b, SolveGraph** out, const float* rhs = nullptr) {
  const bool fp64 = sizeof(T) == 8;
  SolveGraph*& g = ctx->sgl[fp64 ? 1 : 0];
  cudaStream_t s = ctx->stream;
  if (!g) {
    g = new SolveGraph();
    g->fp64 = fp64;
    memset(&g->hf, 0, sizeof(g->hf));
    memset(&g->hd, 0, sizeof(g->hd));
    BF_CK(cudaMalloc(&g->d_args, sizeof(SolveArgs<T>)));
    BF_CK(cudaMallocHost(&g->h_pin, sizeof(SolveArgs<T>)));
    BF_CK(cudaMalloc(&g->st, sizeof(PcgState)));
    BF_CK(cudaMallocHost(&g->h_st, sizeof(PcgState)));
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
    BF_CK(cudaStreamCreateWithFlags(&g->capstream, cudaStreamNonBlocking));
    BF_CK(cudaStreamBeginCaptureToGraph(g->capstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const SolveArgs<T>* A = (const SolveArgs<T>*)g->d_args;
    k_cg<T><<<CG_NCTA, BT, 0, g->capstream>>>(A, 0, g->st, h);
    k_cg<T><<<CG_NCTA, BT, 0, g->capstream>>>(A, 1, g->st, h);
    cudaGraph_t ob;
    cudaError_t e = cudaStreamEndCapture(g->capstream, &ob);
    if (e != cudaSuccess) return bf_fail(ctx, BF_ECUDA, "capture PCG body", cudaGetErrorString(e));
    BF_CK(cudaGraphInstantiate(&g->exec, g->graph, 0));
  }
  SolveArgs<T>& h = host_args<T>(g);
  if (b->N > g->cap) {
    BF_CK(cudaStreamSynchronize(s));
    free_arrays<T>(g);
    const int64_t n = b->N + b->N / 8 + 1024;
    for (int k = 0; k < 2; ++k) {
      BF_CK(cudaMalloc(&h.r[k], n * sizeof(T)));
      BF_CK(cudaMalloc(&h.w[k], n * sizeof(T)));
      BF_CK(cudaMalloc(&h.s[k], n * sizeof(T)));
    }
    BF_CK(cudaMalloc(&h.p, n * sizeof(T)));
    BF_CK(cudaMalloc(&h.x, n * sizeof(T)));
    BF_CK(cudaMalloc(&h.x64, n * sizeof(double)));
    BF_CK(cudaMalloc(&h.part, (size_t)3 * (NCTA > CG_NCTA ? NCTA : CG_NCTA) * sizeof(double)));
    g->cap = n;
  }
  h.B = band_view(b);
  h.lam = (float)b->prm.lambda;
  h.qd = b->qd;
  h.rhs = rhs ? rhs : b->rhs;  // the band's h, or another right-hand side
  // the previous upload from h_pin has completed: every solve ends with a sync
  memcpy(g->h_pin, &h, sizeof(h));
  BF_CK(cudaMemcpyAsync(g->d_args, g->h_pin, sizeof(h), cudaMemcpyHostToDevice, s));
  *out = g;
  return BF_OK;
}

template <class T>
static bf_status solve_t(bf_ctx* ctx, bf_band* b, double tol, int max_iter, unsigned flags, float* mu, int* iters,
                         double* relres, const float* rhs = nullptr) {
  cudaStream_t s = ctx->stream;
  SolveGraph* g = nullptr;
  BF_TRY(get_solver<T>(ctx, b, &g, rhs));
  SolveArgs<T>& h = host_args<T>(g);
  const SolveArgs<T>* A = (const SolveArgs<T>*)g->d_args;
  const int N = (int)b->N;
  if (flags & BF_SOLVE_WARM) {
    k_cast_in<<<gsz(N), 256, 0, s>>>(N, mu, h.x64);
    count_launch();
  } else {
    BF_CK(cudaMemsetAsync(h.x64, 0, (size_t)N * sizeof(double), s));
  }
  k_state_init<<<1, 1, 0, s>>>(g->st, tol, max_iter, sizeof(T) == 8 ? 1e-14 : 1e-7);
  count_launch();
  if (flags & BF_SOLVE_WARM)
    k_outer<T><<<NCTA, BT, 0, s>>>(A, g->st);
  else
    k_outer<T, true><<<NCTA, BT, 0, s>>>(A, g->st);
  count_launch();
  k_cg_init<T><<<NCTA, BT, 0, s>>>(A, g->st);
  count_launch();
  BF_CK(cudaGetLastError());
  bool done = false;
  for (int outer = 0; outer < REFINE_MAX_PASSES; ++outer) {
    BF_CK(cudaMemcpyAsync(g->h_st, g->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    BF_CK(cudaStreamSynchronize(s));
    if (g->h_st->done) {
      done = true;
      break;
    }
    BF_CK(cudaGraphLaunch(g->exec, s));
    k_axpy<T><<<gsz(N), 256, 0, s>>>(N, h.x, h.x64);
    count_launch();
    k_outer<T><<<NCTA, BT, 0, s>>>(A, g->st);
    count_launch();
    k_cg_init<T><<<NCTA, BT, 0, s>>>(A, g->st);
    count_launch();
    BF_CK(cudaGetLastError());
  }
  k_cast_out<<<gsz(N), 256, 0, s>>>(N, h.x64, mu);
  count_launch();
  BF_CK(cudaGetLastError());
  if (!done) {  // the last pass's residual check has not been read back yet
    BF_CK(cudaMemcpyAsync(g->h_st, g->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  }
  BF_CK(cudaStreamSynchronize(s));
  if (!done) done = g->h_st->done;
  const PcgState& st = *g->h_st;
  count_launch(st.nexec);
  if (iters) *iters = st.iter;
  if (relres) *relres = st.bb0 > 0 ? sqrt(st.rr0 / st.bb0) : 0.0;
  if (st.status == 2) return bf_fail(ctx, BF_BREAKDOWN, "PCG breakdown (non-positive curvature or non-finite)");
  if (!done || st.status == 1) return bf_fail(ctx, BF_NOT_CONVERGED, "PCG iteration limit reached");
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

// Q x = rhs for another right-hand side (FP32 vectors, FP64 refinement), x0 = 0
bf_status solve_rhs_impl(bf_ctx* ctx, bf_band* b, const float* rhs, double tol, int max_iter, float* x, int* iters,
                         double* relres) {
  if (b->N == 0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return BF_OK;
  }
  return solve_t<float>(ctx, b, tol, max_iter, 0u, x, iters, relres, rhs);
}

bf_status device_wait_status(bf_ctx* ctx, const char* what) {
  if (!ctx->d_err) return BF_OK;
  BF_CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->h_pinned[0] == 0) return BF_OK;
  ctx->h_pinned[0] = 0;
  BF_CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  return bf_fail(ctx, BF_ECUDA, what, "a kernel's bounded wait for its bulk copies ran out (results not valid)");
}

bf_status spmv_launch(bf_ctx* ctx, const bf_band* b, const float* x, float* y) {
  if (b->N == 0) return BF_OK;
  if (b->obs_mode == 3) return tri_spmv(ctx, b, x, y);
  if ((((uintptr_t)x | (uintptr_t)b->qd) & 15u) == 0) {  // bulk copies need 16-byte aligned arrays
    const int nw = (b->NB + SPT - 1) / SPT;
    const int grid = nw < 152 * SPT_OCC ? nw : 152 * SPT_OCC;
    k_spmv_t<<<grid, 32 * SPT, 0, ctx->stream>>>(band_view(b), (float)b->prm.lambda, b->qd, x, y,
                                                   (int)(b->N & ~(int64_t)3), ctx->d_err);
  } else {
    const int grid = b->NB < 152 * SPMV_OCC ? b->NB : 152 * SPMV_OCC;
    k_spmv<<<grid, BT, 0, ctx->stream>>>(band_view(b), (float)b->prm.lambda, b->qd, x, y);
  }
  count_launch();
  BF_CK(cudaGetLastError());
  return BF_OK;
}
