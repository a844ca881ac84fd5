// Learned warm start and variance surrogate: a 4-layer 3x3x3 convolutional
// network on haloed brick tiles (not in the paper; its Sec. 6 names prior
// learning as future work).
//
// Definition (identical to the oracle's): per active brick a 10^3 tile (the
// brick and a 1-voxel halo), input channels tsdf/h and log(1 + d) at band
// voxels (0 elsewhere); convolutions 2 -> 32 -> 32 -> 32 -> 2 with bias, zero
// padding at the tile boundary, ReLU after the first three; outputs at the
// 8^3 centre: mu_hat = tsdf/h + o0 (voxels), log s_hat = o1 - log Q_ii (residuals
// on the TSDF and on the Jacobi lower bound 1/Q_ii of (Q^-1)_ii); loss = mean
// over band voxels of (mu_hat - mu)^2 + (log s_hat - log max(s, 1/Q_ii))^2.
//
// Kernels: implicit GEMM on tensor cores (bf16 x bf16 -> fp32).  A CTA stages
// one brick tile at a time in shared memory with a zero border (12^3 rows of
// C channels), so a tap shift is a row offset.
//   k_conv_tc<FWD>   y = relu(conv(x) + b)                 (layers 1-3; tcgen05, TMEM)
//   k_conv_tc<LAST>  o = conv(x) + b; predictions; loss and dL/do at band voxels
//   k_conv_tc<DGRAD> dx = conv(dy, W flipped and transposed) * [x_prev > 0]
//   k_wgrad          dW[tap][ci][co] += sum_v x[v + tap][ci] dy[v][co], db (mma.sync)
//   k_conv           the same convolutions on mma.sync m16n8k16 with ldmatrix
//                    operand loads (16-voxel output tiles per warp); timing only
// Weights: FP32 master copy (oracle layout W[tap][ci][co], b[co]) with Adam
// moments; bf16 copies packed as [tap][co][ci] (forward) and
// [tap'][ci][co] with tap' = 26 - tap (backward data).
#include <cuda_bf16.h>

#include <math_constants.h>

#include <cstring>

#include "internal.cuh"

namespace {

constexpr int NT = 256;           // threads per conv CTA (8 warps)
constexpr int TV = 1000;          // tile voxels (10^3)
constexpr int PV = 1728;          // padded tile rows (12^3)
constexpr int NMT = 63;           // 16-voxel output tiles (1008 rows)
constexpr int CI_PAD[4] = {16, 32, 32, 32};
constexpr int CO_PAD[4] = {32, 32, 32, 16};
constexpr int CI_REAL[4] = {2, 32, 32, 32};
constexpr int CO_REAL[4] = {32, 32, 32, 2};

constexpr int MODE_FWD = 0, MODE_LAST = 1, MODE_DGRAD = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// padded row of tile voxel v (clamped to the last voxel for rows >= 1000)
__device__ __forceinline__ int prow(int v) {
  v = v < TV ? v : TV - 1;
  int tx = v % 10, ty = (v / 10) % 10, tz = v / 100;
  return (tx + 1) + 12 * (ty + 1) + 144 * (tz + 1);
}
__device__ __forceinline__ int tap_off(int tap) { return (tap % 3 - 1) + 12 * ((tap / 3) % 3 - 1) + 144 * (tap / 9 - 1); }

// Element offset of 16-byte chunk `chunk` of row `row` in a shared array of
// rows of C bf16: chunks are XOR-swizzled so that the 8 rows one ldmatrix
// phase reads from consecutive rows fall in distinct bank groups.
template <int C>
__device__ __forceinline__ int sw(int row, int chunk) {
  constexpr int U = C / 8, L = 8 / U;
  return row * C + 8 * (chunk ^ ((row / L) & (U - 1)));
}

// stage tile [1000][C] (global, bf16) into xs [1728][C] with a zero border
template <int C>
__device__ __forceinline__ void stage_tile(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* xs) {
  constexpr int U = C / 8;  // uint4 per row
  const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll 4
  for (int q = threadIdx.x; q < PV * U; q += NT) {
    int p = q / U, u = q - p * U;
    int px = p % 12, py = (p / 12) % 12, pz = p / 144;
    uint4 val = z;
    if (px >= 1 && px <= 10 && py >= 1 && py <= 10 && pz >= 1 && pz <= 10) {
      int v = (px - 1) + 10 * (py - 1) + 100 * (pz - 1);
      val = reinterpret_cast<const uint4*>(src + (size_t)v * C)[u];
    }
    *reinterpret_cast<uint4*>(xs + sw<C>(p, u)) = val;
  }
}

struct LossArgs {
  BandView B;
  const float* tsdf;   // [N] metres (skip connection of mu_hat)
  const float* qd;     // [N] Q_ii (floor of the variance target)
  const float* mu_t;   // [N] targets or null
  const float* s_t;    // [N] variance targets (voxels^2); log max(s, 1/Q_ii) is fitted
  float* mu_hat;       // [N] predictions or null
  float* ls_hat;       // [N]
  double inv_m;        // 1 / (band voxels in the batch)
  double* loss;        // accumulated loss
};

// Implicit-GEMM convolution over `nb` brick tiles (CTAs stride over bricks).
//   x   [nb][1000][CIN] bf16; w [27][COUT][CIN] bf16; bias [nbias] fp32 (0 beyond)
//   FWD:   y [nb][1000][COUT] bf16 = relu(conv + b)
//   LAST:  o (2 real channels) -> predictions, loss, dy [nb][1000][COUT] bf16
//   DGRAD: y [nb][1000][COUT] bf16 = conv(x, w) * [mask > 0], mask [nb][1000][COUT]
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NT, 1) k_conv(int nb, const __nv_bfloat16* __restrict__ x,
                                                const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                                int nbias, __nv_bfloat16* __restrict__ y,
                                                const __nv_bfloat16* __restrict__ mask, LossArgs la) {
  extern __shared__ __align__(16) uint8_t smem[];
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* ws = xs + PV * CIN;
  float* bs = reinterpret_cast<float*>(ws + 27 * COUT * CIN);
  constexpr int NTN = COUT / 8;   // n8 tiles
  constexpr int NKC = CIN / 16;   // k16 chunks per tap
  constexpr int MT = 4;           // m16 tiles per warp per pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < 27 * COUT * CIN / 8; q += NT)
    *reinterpret_cast<uint4*>(ws + sw<CIN>(q / (CIN / 8), q % (CIN / 8))) = reinterpret_cast<const uint4*>(w)[q];
  for (int q = threadIdx.x; q < COUT; q += NT) bs[q] = (bias && q < nbias) ? bias[q] : 0.0f;
  double lsum = 0.0;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    __syncthreads();
    stage_tile<CIN>(x + (size_t)b * TV * CIN, xs);
    __syncthreads();
    for (int mt0 = warp * MT; mt0 < NMT; mt0 += 8 * MT) {
      float acc[MT][NTN][4];
#pragma unroll
      for (int q = 0; q < MT; ++q)
#pragma unroll
        for (int n = 0; n < NTN; ++n)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[q][n][k] = 0.0f;
      // this lane's A row (one per m-tile): row (lane % 8) + 8 ((lane / 8) % 2)
      int arow[MT];
#pragma unroll
      for (int q = 0; q < MT; ++q) arow[q] = prow(16 * (mt0 + q) + (lane & 7) + 8 * ((lane >> 3) & 1));
      const int akc = lane >> 4;
      for (int tap = 0; tap < 27; ++tap) {
        const int off = tap_off(tap);
#pragma unroll
        for (int kc = 0; kc < NKC; ++kc) {
          uint32_t bf[NTN][2];
#pragma unroll
          for (int np = 0; np < NTN / 2; ++np) {
            const int j = lane >> 3;
            const int n = np * 16 + (lane & 7) + 8 * (j >> 1);
            ldsm_x4(smem_u32(ws + sw<CIN>(tap * COUT + n, 2 * kc + (j & 1))), bf[2 * np][0], bf[2 * np][1],
                    bf[2 * np + 1][0], bf[2 * np + 1][1]);
          }
#pragma unroll
          for (int q = 0; q < MT; ++q) {
            if (mt0 + q >= NMT) break;
            uint32_t a0, a1, a2, a3;
            ldsm_x4(smem_u32(xs + sw<CIN>(arow[q] + off, 2 * kc + akc)), a0, a1, a2, a3);
#pragma unroll
            for (int n = 0; n < NTN; ++n) mma16816(acc[q][n], a0, a1, a2, a3, bf[n][0], bf[n][1]);
          }
        }
      }
      // epilogue: thread holds rows g, g+8 and columns 2 t, 2 t + 1 of each n8 tile
      const int g = lane >> 2, t = lane & 3;
#pragma unroll
      for (int q = 0; q < MT; ++q) {
        if (mt0 + q >= NMT) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = 16 * (mt0 + q) + g + 8 * h;
          if (v >= TV) continue;
#pragma unroll
          for (int n = 0; n < NTN; ++n) {
            const int co = n * 8 + 2 * t;
            float v0 = acc[q][n][2 * h] + bs[co], v1 = acc[q][n][2 * h + 1] + bs[co + 1];
            const size_t o = ((size_t)b * TV + v) * COUT + co;
            if (MODE == MODE_FWD) {
              v0 = fmaxf(v0, 0.0f);
              v1 = fmaxf(v1, 0.0f);
            } else if (MODE == MODE_DGRAD) {
              const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(mask + o);
              if (!(__bfloat162float(m2.x) > 0.0f)) v0 = 0.0f;
              if (!(__bfloat162float(m2.y) > 0.0f)) v1 = 0.0f;
            } else {  // MODE_LAST: channels 0, 1 are (o0, o1); the rest stay 0
              float d0 = 0.0f, d1 = 0.0f;
              if (co == 0) {
                const int tx = v % 10, ty = (v / 10) % 10, tz = v / 100;
                if (tx >= 1 && tx <= 8 && ty >= 1 && ty <= 8 && tz >= 1 && tz <= 8) {
                  const int l = (tx - 1) + 8 * (ty - 1) + 64 * (tz - 1);
                  const MetaWord m = la.B.meta[16 * b + (l >> 5)];
                  const uint32_t bit = 1u << (l & 31);
                  if (m.bits & bit) {
                    const int idx = m.base + __popc(m.bits & (bit - 1u));
                    const float mh = la.tsdf[idx] / la.B.h + v0;
                    const float lh = (float)((double)v1 - log((double)la.qd[idx]));
                    if (la.mu_hat) {
                      la.mu_hat[idx] = mh;
                      la.ls_hat[idx] = lh;
                    }
                    if (la.mu_t) {
                      const double st = fmax((double)la.s_t[idx], 1.0 / (double)la.qd[idx]);
                      const double e0 = (double)mh - (double)la.mu_t[idx], e1 = (double)lh - log(st);
                      lsum += (e0 * e0 + e1 * e1) * la.inv_m;
                      d0 = (float)(2.0 * e0 * la.inv_m);
                      d1 = (float)(2.0 * e1 * la.inv_m);
                    }
                  }
                }
              }
              v0 = d0;
              v1 = d1;
            }
            *reinterpret_cast<__nv_bfloat162*>(y + o) = __floats2bfloat162_rn(v0, v1);
          }
        }
      }
    }
  }
  if (MODE == MODE_LAST && la.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.0) atomicAdd(la.loss, lsum);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) form of the same convolution.
//
// One CTA per SM walks the bricks.  The input tile lives in shared memory in
// the canonical K-major, no-swizzle operand layout: plane c (channels
// 8c .. 8c+7) holds one 16-byte row per padded voxel row (12^3 tile with a
// zero border, padded row TC_PB + (x+1) + 12 (y+1) + 144 (z+1)), so the A
// operand of tap t for output rows p0 .. p0+127 is the 128 rows starting at
// p0 + off(t): an 8-row core matrix is 128 contiguous bytes (stride between
// core matrices along M: 128 B; along K: one plane).  The weights are staged
// once, per tap and 8-channel chunk a [C_out][8] block (the B operand,
// K-major).  One 128-row M tile per interior plane z: rows (x, y) = (-1..10,
// 0..9) of the plane (120 rows holding its 100 voxels) and 8 rows of its
// y = 10 border, 1.28 computed rows per voxel (the last layer, whose outputs
// are needed at the 8^3 centre only, takes planes 1..8).  Each tile
// accumulates in its own TMEM columns (D: 128 lanes x C_out FP32), over 27
// taps x C_in/16 MMAs of M128 x N(C_out) x K16 issued by two threads
// (alternate tiles; one thread issues too slowly): the first half of the
// planes completes on one mbarrier, the second on another,
// so the epilogue of the first half (bias, ReLU / loss / ReLU mask; TMEM read
// by tcgen05.ld, interior voxels written) runs while the second half's MMAs
// do; the next brick's input is read into registers meanwhile.
// (With 32 input channels every MMA reads its 4 KB A block from shared
// memory for 131 kFLOP, so the MMAs run at the shared-memory operand rate,
// about half the tensor peak, rather than at the tensor peak.)
constexpr int TC_PB = 16;                  // padded row offset (keeps the lowest tap row of plane 0 >= 0)
constexpr int TC_ROWS = 1856;              // padded rows held
constexpr int TC_NT = 256;                 // threads per CTA (two warpgroups)
static_assert(TC_PB + 156 - 157 >= 0 && TC_PB + 156 + 144 * 9 + 127 + 157 < TC_ROWS, "tile rows");

template <int CIN, int COUT>
__host__ __device__ constexpr size_t tc_smem() {
  return (size_t)TC_ROWS * CIN * 2 + (size_t)27 * CIN * COUT * 2 + COUT * 4 + 64;
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
  // offsets in 16-byte units, descriptor version 1, no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <int N>
__host__ __device__ constexpr uint32_t tc_idesc() {
  // kind::f16 instruction descriptor: D FP32, A and B bf16, both K-major, N, M = 128
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(mbar))
               : "memory");
}

__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
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

// 32 lanes x 16 consecutive 32-bit TMEM columns into 16 registers per thread
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TC_NT, 1) k_conv_tc(int nb, const __nv_bfloat16* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ bias, int nbias,
                                                      __nv_bfloat16* __restrict__ y,
                                                      const __nv_bfloat16* __restrict__ mask, LossArgs la,
                                                      int* __restrict__ err) {
  extern __shared__ __align__(16) uint8_t tsm[];
  constexpr int NPL = CIN / 8;  // 8-channel planes of the input tile
  constexpr int KS = CIN / 16;  // K16 steps per tap
  constexpr int Z0 = MODE == MODE_LAST ? 1 : 0, NTZ = MODE == MODE_LAST ? 8 : 10;  // planes computed
  constexpr int NH = NTZ / 2;                                                         // planes per half
  constexpr uint32_t TCOLS = NTZ * COUT > 256 ? 512 : (NTZ * COUT > 128 ? 256 : 128);
  __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(tsm);  // [NPL][TC_ROWS][8]
  __nv_bfloat16* wsm = act + (size_t)TC_ROWS * CIN;              // [27][NPL][COUT][8]
  float* bs = reinterpret_cast<float*>(wsm + (size_t)27 * CIN * COUT);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(bs + COUT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // zero tile (the border rows stay zero), weights in operand order, bias
  for (int q = tid; q < TC_ROWS * CIN / 8; q += TC_NT) reinterpret_cast<uint4*>(act)[q] = make_uint4(0, 0, 0, 0);
  for (int q = tid; q < 27 * COUT * NPL; q += TC_NT) {  // q: global 16-byte chunk of w[27][COUT][CIN]
    const int tap = q / (COUT * NPL), rem = q - tap * COUT * NPL, co = rem / NPL, c = rem - co * NPL;
    reinterpret_cast<uint4*>(wsm)[(tap * NPL + c) * COUT + co] = reinterpret_cast<const uint4*>(w)[q];
  }
  for (int q = tid; q < COUT; q += TC_NT) bs[q] = (bias && q < nbias) ? bias[q] : 0.0f;
  if (tid == 0) {  // two arrivals per phase (the commits of the two issuing threads), for each half of the planes
#pragma unroll
    for (int h = 0; h < 2; ++h)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"((uint32_t)__cvta_generic_to_shared(mbar + h))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(tslot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t act_s = (uint32_t)__cvta_generic_to_shared(act), w_s = (uint32_t)__cvta_generic_to_shared(wsm);
  double lsum = 0.0;
  // the next brick's input is loaded into registers while the tensor cores work on the current one
  constexpr int PER = (TV * NPL + TC_NT - 1) / TC_NT;  // 16-byte chunks per thread and brick
  uint4 pre[PER];
  auto load_brick = [&](int bb) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int q = tid + i * TC_NT;
      if (bb < nb && q < TV * NPL)
        pre[i] = __ldg(reinterpret_cast<const uint4*>(x + (size_t)bb * TV * CIN) + q);  // chunk q = (v, c)
    }
  };
  load_brick(blockIdx.x);
  const uint64_t ad0 = tc_desc(act_s, TC_ROWS * 16u, 128u), bd0 = tc_desc(w_s, COUT * 16u, 128u);
  // the brick's 1000 rows into the interior of the tile (the MMAs of the previous brick have read the tile)
  auto stage = [&]() {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int q = tid + i * TC_NT;
      if (q < TV * NPL) {
        const int v = q / NPL, c = q - v * NPL;
        reinterpret_cast<uint4*>(act)[(size_t)c * TC_ROWS + TC_PB + prow(v)] = pre[i];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  };
  // the MMAs of half h of the planes: two issuing threads, alternate tiles; descriptors in 16-byte units
  auto issue = [&](int h) {
    if ((tid & 127) == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int mt = h * NH + ((h * NH + (tid >> 7)) & 1); mt < (h + 1) * NH; mt += 2) {
        const int p0 = TC_PB + 156 + 144 * (Z0 + mt);  // row of (x, y, z) = (-1, 0, Z0 + mt)
        for (int tap = 0; tap < 27; ++tap) {
          const uint64_t ar = ad0 + (uint64_t)(p0 + tap_off(tap));
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)
            tc_mma(tmem + (uint32_t)(mt * COUT), ar + (uint64_t)(2 * ks * TC_ROWS),
                   bd0 + (uint64_t)((tap * NPL + 2 * ks) * COUT), tc_idesc<COUT>(), (tap | ks) != 0);
        }
      }
      tc_commit(mbar + h);
    }
  };
  // wait for half h of brick number `it`; a wait that runs out reports, waits once more for every MMA in
  // flight (halves h..1 of this brick) and returns false in all threads
  auto wait_half = [&](int h, int it) -> bool {
    const bool ok = tc_wait(mbar + h, (uint32_t)it & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, 1);
      for (int hh = h; hh < 2; ++hh) tc_wait(mbar + hh, (uint32_t)it & 1u);
      return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return true;
  };
  // epilogue of half h of brick b: warpgroup g takes the half's tiles g, g + 2, ...; warp w reads TMEM lanes
  // 32 (w % 4) ..
  auto epilogue = [&](int h, int b) {
    const int lq = warp & 3;
    for (int mt = h * NH + (warp >> 2); mt < (h + 1) * NH; mt += 2) {
      const int z = Z0 + mt, i = 32 * lq + lane;  // tile row i: (x, y) = (i % 12 - 1, i / 12)
      const uint32_t taddr = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(mt * COUT);
      float acc[COUT];
#pragma unroll
      for (int k0 = 0; k0 < COUT; k0 += 16) {
        float t[16];
        tc_ld16(taddr + (uint32_t)k0, t);
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k0 + k] = t[k];
      }
      if (i >= 120 || i % 12 == 0 || i % 12 == 11) continue;  // the x = -1, 10 columns and the y = 10 row
      const int v = (i % 12 - 1) + 10 * (i / 12) + 100 * z;
      const size_t o = ((size_t)b * TV + v) * COUT;
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] += bs[co];
      if (MODE == MODE_FWD) {
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaxf(acc[co], 0.0f);
      } else if (MODE == MODE_DGRAD) {
#pragma unroll
        for (int c8 = 0; c8 < COUT / 8; ++c8) {
          const uint4 m4 = reinterpret_cast<const uint4*>(mask + o)[c8];
          const __nv_bfloat16* mv = reinterpret_cast<const __nv_bfloat16*>(&m4);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (!(__bfloat162float(mv[k]) > 0.0f)) acc[8 * c8 + k] = 0.0f;
        }
      } else {  // MODE_LAST: channels 0, 1 are (o0, o1) -> predictions, loss, dL/do
        float d0 = 0.0f, d1 = 0.0f;
        const int tx = v % 10, ty = (v / 10) % 10, tz = v / 100;
        if (tx >= 1 && tx <= 8 && ty >= 1 && ty <= 8 && tz >= 1 && tz <= 8) {
          const int l = (tx - 1) + 8 * (ty - 1) + 64 * (tz - 1);
          const MetaWord m = la.B.meta[16 * b + (l >> 5)];
          const uint32_t bit = 1u << (l & 31);
          if (m.bits & bit) {
            const int idx = m.base + __popc(m.bits & (bit - 1u));
            const float mh = la.tsdf[idx] / la.B.h + acc[0];
            const float lh = (float)((double)acc[1] - log((double)la.qd[idx]));
            if (la.mu_hat) {
              la.mu_hat[idx] = mh;
              la.ls_hat[idx] = lh;
            }
            if (la.mu_t) {
              const double st = fmax((double)la.s_t[idx], 1.0 / (double)la.qd[idx]);
              const double e0 = (double)mh - (double)la.mu_t[idx], e1 = (double)lh - log(st);
              lsum += (e0 * e0 + e1 * e1) * la.inv_m;
              d0 = (float)(2.0 * e0 * la.inv_m);
              d1 = (float)(2.0 * e1 * la.inv_m);
            }
          }
        }
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = 0.0f;
        acc[0] = d0;
        acc[1] = d1;
      }
#pragma unroll
      for (int c8 = 0; c8 < COUT / 8; ++c8) {
        uint4 o4;
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&o4);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(acc[8 * c8 + 2 * k], acc[8 * c8 + 2 * k + 1]);
        reinterpret_cast<uint4*>(y + o)[c8] = o4;
      }
    }
  };
  // pipeline over the CTA's bricks: the first half of the next brick's planes runs on the tensor cores while
  // the epilogue of this brick's second half does
  int b = blockIdx.x, it = 0;
  if (b < nb) {
    stage();
    issue(0);
    issue(1);
    load_brick(b + gridDim.x);
  }
  for (; b < nb; b += gridDim.x, ++it) {
    if (!wait_half(0, it)) break;
    if (MODE == MODE_LAST) {  // dL/do is zero on planes 0 and 9, which the last layer does not compute
      for (int q = tid; q < 200 * COUT / 8; q += TC_NT) {
        const int vv = q / (COUT / 8), v = vv < 100 ? vv : vv + 800;
        reinterpret_cast<uint4*>(y + ((size_t)b * TV + v) * COUT)[q % (COUT / 8)] = make_uint4(0, 0, 0, 0);
      }
    }
    epilogue(0, b);
    if (!wait_half(1, it)) break;
    const int bn = b + gridDim.x;
    if (bn < nb) {
      stage();  // also: every thread is past the first half's epilogue, whose TMEM columns are reused
      issue(0);
      load_brick(bn + gridDim.x);
    }
    epilogue(1, b);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the second half's TMEM columns are read
    if (bn < nb) issue(1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  if (MODE == MODE_LAST && la.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && lsum != 0.0) atomicAdd(la.loss, lsum);
  }
}

// Weight and bias gradients: dW[tap][ci][co] += sum_v x[v + tap][ci] dy[v][co],
// db[co] += sum_v dy[v][co] (co < nbias), over the CTA's bricks, added into fp32 dW, db.
// Warp w owns taps w, w + 8, w + 16, w + 24; a k-step is 16 output voxels.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT, 1) k_wgrad(int nb, const __nv_bfloat16* __restrict__ x,
                                                 const __nv_bfloat16* __restrict__ dy, float* __restrict__ dW,
                                                 float* __restrict__ db, int nbias) {
  extern __shared__ __align__(16) uint8_t smem[];
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* ds = xs + PV * CIN;  // [1008][COUT], rows >= 1000 zero
  constexpr int NTN = COUT / 8, NMI = CIN / 16, NTAP = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NTAP][NMI][NTN][4];
#pragma unroll
  for (int a = 0; a < NTAP; ++a)
#pragma unroll
    for (int m = 0; m < NMI; ++m)
#pragma unroll
      for (int n = 0; n < NTN; ++n)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[a][m][n][k] = 0.0f;
  float dbacc = 0.0f;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    __syncthreads();
    stage_tile<CIN>(x + (size_t)b * TV * CIN, xs);
    constexpr int U = COUT / 8;
    for (int q = threadIdx.x; q < 1008 * U; q += NT) {
      int v = q / U, u = q - v * U;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v < TV) val = reinterpret_cast<const uint4*>(dy + ((size_t)b * TV + v) * COUT)[u];
      *reinterpret_cast<uint4*>(ds + sw<COUT>(v, u)) = val;
    }
    __syncthreads();
    {
      const int co = threadIdx.x % COUT;
      for (int v = threadIdx.x / COUT; v < TV; v += NT / COUT) dbacc += __bfloat162float(ds[sw<COUT>(v, co / 8) + co % 8]);
    }
    for (int kc = 0; kc < NMT; ++kc) {
      const int v0 = 16 * kc;
      uint32_t bf[NTN][2];
      const int j = lane >> 3;
#pragma unroll
      for (int np = 0; np < NTN / 2; ++np) {
        const int row = v0 + (lane & 7) + 8 * (j & 1);
        ldsm_x4_t(smem_u32(ds + sw<COUT>(row, 2 * np + (j >> 1))), bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0],
                  bf[2 * np + 1][1]);
      }
      const int arow = prow(v0 + (lane & 7) + 8 * (j >> 1));
#pragma unroll
      for (int a = 0; a < NTAP; ++a) {
        const int tap = warp + 8 * a;
        if (tap >= 27) break;
        const int off = tap_off(tap);
#pragma unroll
        for (int m = 0; m < NMI; ++m) {
          uint32_t a0, a1, a2, a3;
          ldsm_x4_t(smem_u32(xs + sw<CIN>(arow + off, 2 * m + (j & 1))), a0, a1, a2, a3);
#pragma unroll
          for (int n = 0; n < NTN; ++n) mma16816(acc[a][m][n], a0, a1, a2, a3, bf[n][0], bf[n][1]);
        }
      }
    }
  }
  // accumulator (m = ci, n = co): rows g, g+8, columns 2t, 2t+1
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int a = 0; a < NTAP; ++a) {
    const int tap = warp + 8 * a;
    if (tap >= 27) break;
#pragma unroll
    for (int m = 0; m < NMI; ++m)
#pragma unroll
      for (int n = 0; n < NTN; ++n)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int ci = m * 16 + g + 8 * h, co = n * 8 + 2 * t;
          atomicAdd(dW + ((size_t)tap * CIN + ci) * COUT + co, acc[a][m][n][2 * h]);
          atomicAdd(dW + ((size_t)tap * CIN + ci) * COUT + co + 1, acc[a][m][n][2 * h + 1]);
        }
  }
  if (threadIdx.x % COUT < nbias) atomicAdd(db + threadIdx.x % COUT, dbacc);
}

// input tiles: channel 0 = tsdf/h, channel 1 = log(1 + d) at band voxels
__global__ void k_features(BandView B, const float* __restrict__ tsdf, const float* __restrict__ d,
                           __nv_bfloat16* __restrict__ x0) {
  const int b = blockIdx.x;
  const int bi = B.bcoord[4 * b], bj = B.bcoord[4 * b + 1], bk = B.bcoord[4 * b + 2];
  for (int v = threadIdx.x; v < TV; v += blockDim.x) {
    const int tx = v % 10, ty = (v / 10) % 10, tz = v / 100;
    const int idx = band_lookup(B, 8 * bi + tx - 1, 8 * bj + ty - 1, 8 * bk + tz - 1);
    float c0 = 0.0f, c1 = 0.0f;
    if (idx >= 0) {
      c0 = tsdf[idx] / B.h;
      c1 = log1pf(fmaxf(d[idx], 0.0f));
    }
    __nv_bfloat16* o = x0 + ((size_t)b * TV + v) * 16;
    o[0] = __float2bfloat16(c0);
    o[1] = __float2bfloat16(c1);
#pragma unroll
    for (int c = 2; c < 16; ++c) o[c] = __float2bfloat16(0.0f);
  }
}

// pack fp32 master weights of layer l (W[tap][ci][co]) into the bf16 forward
// layout [tap][co][ci_pad] and the backward-data layout [26 - tap][ci][co_pad]
__global__ void k_pack(const float* __restrict__ W, int ci_r, int co_r, int ci_p, int co_p,
                       __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wb) {
  const int n = 27 * ci_p * co_p;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int tap = q / (ci_p * co_p), rem = q - tap * ci_p * co_p;
    const int co = rem / ci_p, ci = rem - co * ci_p;  // forward element [tap][co][ci]
    const float v = (ci < ci_r && co < co_r) ? W[((size_t)tap * ci_r + ci) * co_r + co] : 0.0f;
    wf[q] = __float2bfloat16(v);
    if (wb) wb[((size_t)(26 - tap) * ci_p + ci) * co_p + co] = __float2bfloat16(v);
  }
}

// padded fp32 gradient [27][ci_p][co_p] -> flat gradient in the oracle layout
__global__ void k_unpad_grad(const float* __restrict__ gp, int ci_r, int co_r, int ci_p, int co_p,
                             float* __restrict__ g) {
  const int n = 27 * ci_r * co_r;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int tap = q / (ci_r * co_r), rem = q - tap * ci_r * co_r;
    const int ci = rem / co_r, co = rem - ci * co_r;
    g[q] = gp[((size_t)tap * ci_p + ci) * co_p + co];
  }
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__device__ __forceinline__ uint64_t mix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// He-normal weights (std sqrt(2 / fan_in), last layer x0.1), zero biases
__global__ void k_init(float* __restrict__ p, int64_t n, uint64_t seed, int64_t w0, int64_t b0, int64_t w1, int64_t b1,
                       int64_t w2, int64_t b2, int64_t w3, int64_t b3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float std = 0.0f;
    if (i < b0) std = sqrtf(2.0f / (27 * 2));
    else if (i >= w1 && i < b1) std = sqrtf(2.0f / (27 * 32));
    else if (i >= w2 && i < b2) std = sqrtf(2.0f / (27 * 32));
    else if (i >= w3 && i < b3) std = 0.1f * sqrtf(2.0f / (27 * 32));
    const uint64_t h1 = mix(seed ^ (uint64_t)(2 * i)), h2 = mix(seed ^ (uint64_t)(2 * i + 1));
    const double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    p[i] = std * (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

// Surrogate judge, one CTA per brick.  From the sums s1 = sum_k t_k and sq = sum_k t_k^2
// of K_j probe values t_k = z_k (.) Q^-1 z_k:
// s_J = mean, se = sample std / sqrt(K_j), floor f = max(s_J, 1/Q_ii),
// e_i = |s_hat_i - s_J,i|; stat0 = median over the brick of e_i / f_i,
// stat1 = max over the brick of e_i / (3 se_i + 0.1 f_i); accepted iff
// stat0 <= 0.10 and stat1 <= 1.
__global__ void __launch_bounds__(256) k_judge(const int32_t* __restrict__ off, const float* __restrict__ qd,
                                               const float* __restrict__ lsh, const double* __restrict__ s1,
                                               const double* __restrict__ sq, int Kj, double* __restrict__ stat,
                                               uint8_t* __restrict__ acc, int* __restrict__ nacc) {
  __shared__ double rel[512];
  __shared__ double wmax[8];
  const int b = blockIdx.x, i0 = off[b], n = off[b + 1] - i0;
  double mx = 0.0;
  for (int l = threadIdx.x; l < 512; l += blockDim.x) {
    double rv = CUDART_INF;
    if (l < n) {
      const int i = i0 + l;
      const double sj = s1[i] / (double)Kj;
      const double var = fmax((sq[i] - sj * s1[i]) / (double)(Kj - 1), 0.0);
      const double se = sqrt(var / (double)Kj);
      const double f = fmax(sj, 1.0 / (double)qd[i]);
      const double e = fabs(exp((double)lsh[i]) - sj);
      rv = e / f;
      mx = fmax(mx, e / (3.0 * se + 0.1 * f));
    }
    rel[l] = rv;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  // bitonic sort of the 512 values (absent voxels are +inf, at the end)
  for (int k = 2; k <= 512; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int l = threadIdx.x; l < 512; l += blockDim.x) {
        const int p = l ^ j;
        if (p > l) {
          const double a = rel[l], c = rel[p];
          const bool up = (l & k) == 0;
          if ((a > c) == up) {
            rel[l] = c;
            rel[p] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < 8; ++w) m = fmax(m, wmax[w]);
    const double med = n == 0 ? 0.0 : ((n & 1) ? rel[n / 2] : 0.5 * (rel[n / 2 - 1] + rel[n / 2]));
    stat[2 * b] = med;
    stat[2 * b + 1] = m;
    const uint8_t ok = (med <= 0.10 && m <= 1.0) ? 1 : 0;
    acc[b] = ok;
    if (ok) atomicAdd(nacc, 1);
  }
}

// s = exp(log s_hat) on accepted bricks, else the K-probe mean (K_j s_J + rest) / K
__global__ void k_surrogate_fill(const int32_t* __restrict__ off, const float* __restrict__ lsh,
                                 const float* __restrict__ sJ, const float* __restrict__ rest,
                                 const uint8_t* __restrict__ acc, int Kj, int K, float* __restrict__ s) {
  const int b = blockIdx.x, i0 = off[b], i1 = off[b + 1];
  const bool ok = acc[b] != 0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    s[i] = ok ? (float)exp((double)lsh[i]) : (float)(((double)Kj * (double)sJ[i] + (double)rest[i]) / (double)K);
}

unsigned gs(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return (size_t)PV * CIN * 2 + (size_t)27 * COUT * CIN * 2 + COUT * 4;
}
template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return (size_t)PV * CIN * 2 + (size_t)1008 * COUT * 2;
}

}  // namespace

struct bf_net {
  int64_t P = 0;
  int64_t woff[4], boff[4];  // offsets in the flat parameter vector
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // fp32 master, grad, Adam moments
  __nv_bfloat16* wf[4] = {nullptr, nullptr, nullptr, nullptr};   // forward layout
  __nv_bfloat16* wb[4] = {nullptr, nullptr, nullptr, nullptr};   // backward-data layout
  float* gpad[4] = {nullptr, nullptr, nullptr, nullptr};         // padded weight grads
  int step = 0;
  // activations for the current batch
  int cap_nb = 0;
  __nv_bfloat16* act[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // x0, a1, a2, a3, dy4
  __nv_bfloat16* gact[3] = {nullptr, nullptr, nullptr};                   // dz1, dz2, dz3
  double* loss = nullptr;
  double* h_loss = nullptr;
  int* err = nullptr;  // set by a tensor-core kernel whose MMAs did not complete in time
  bool attr = false;
  int device = 0;      // device that holds the parameters and activations
};

static int64_t nparams_impl() {
  int64_t n = 0;
  for (int l = 0; l < 4; ++l) n += 27 * CI_REAL[l] * CO_REAL[l] + CO_REAL[l];
  return n;
}

static bf_status net_pack(bf_ctx* ctx, bf_net* net) {
  for (int l = 0; l < 4; ++l) {
    k_pack<<<gs(27 * CI_PAD[l] * CO_PAD[l]), 256, 0, ctx->stream>>>(net->p + net->woff[l], CI_REAL[l], CO_REAL[l],
                                                                     CI_PAD[l], CO_PAD[l], net->wf[l],
                                                                     l > 0 ? net->wb[l] : nullptr);
    count_launch();
  }
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// CTAs for a brick-striding kernel: as many as are resident at once (at most nb)
template <class K>
static int occ_grid(K kern, size_t smem, int nb) {
  int per = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, smem) != cudaSuccess || per < 1) per = 1;
  const int g = per * 152;
  return nb < g ? nb : g;
}

template <int CIN, int COUT>
constexpr int tc_launch_smem() {  // at least 120 KB, so that one CTA (and one TMEM allocation) fits per SM
  return tc_smem<CIN, COUT>() > 120 * 1024 ? (int)tc_smem<CIN, COUT>() : 120 * 1024;
}

// tensor-core convolution over the band's bricks (one CTA per SM)
template <int CIN, int COUT, int MODE>
static void conv_tc(cudaStream_t s, bf_net* net, int nb, const __nv_bfloat16* x, const __nv_bfloat16* w,
                    const float* bias, int nbias, __nv_bfloat16* y, const __nv_bfloat16* mask, const LossArgs& la) {
  const int grid = nb < 152 ? nb : 152;
  k_conv_tc<CIN, COUT, MODE><<<grid, TC_NT, tc_launch_smem<CIN, COUT>(), s>>>(nb, x, w, bias, nbias, y, mask, la,
                                                                              net->err);
  count_launch();
}

static bf_status set_attrs(bf_ctx* ctx, bf_net* net) {
  if (net->attr) return BF_OK;
  BF_CK(cudaFuncSetAttribute(k_conv_tc<16, 32, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_launch_smem<16, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv_tc<32, 32, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_launch_smem<32, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv_tc<32, 16, MODE_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_launch_smem<32, 16>()));
  BF_CK(cudaFuncSetAttribute(k_conv_tc<16, 32, MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_launch_smem<16, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv_tc<32, 32, MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_launch_smem<32, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv<16, 32, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem<16, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv<32, 32, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem<32, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv<32, 16, MODE_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem<32, 16>()));
  BF_CK(cudaFuncSetAttribute(k_conv<16, 32, MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem<16, 32>()));
  BF_CK(cudaFuncSetAttribute(k_conv<32, 32, MODE_DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv_smem<32, 32>()));
  BF_CK(cudaFuncSetAttribute(k_wgrad<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem<16, 32>()));
  BF_CK(cudaFuncSetAttribute(k_wgrad<32, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem<32, 32>()));
  BF_CK(cudaFuncSetAttribute(k_wgrad<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem<32, 16>()));
  net->attr = true;
  return BF_OK;
}

static bf_status ensure_batch(bf_ctx* ctx, bf_net* net, int nb) {
  if (nb <= net->cap_nb) return BF_OK;
  for (auto& a : net->act)
    if (a) cudaFree(a), a = nullptr;
  for (auto& a : net->gact)
    if (a) cudaFree(a), a = nullptr;
  const size_t cap = (size_t)nb + nb / 4 + 8;
  BF_CK(cudaMalloc(&net->act[0], cap * TV * 16 * 2));
  for (int l = 1; l <= 3; ++l) BF_CK(cudaMalloc(&net->act[l], cap * TV * 32 * 2));
  BF_CK(cudaMalloc(&net->act[4], cap * TV * 16 * 2));
  for (int l = 0; l < 3; ++l) BF_CK(cudaMalloc(&net->gact[l], cap * TV * 32 * 2));
  net->cap_nb = (int)cap;
  return BF_OK;
}

// forward over the band's bricks; with targets also the loss and dy of the last layer
static bf_status net_forward(bf_ctx* ctx, bf_net* net, const bf_band* b, const float* mu_t, const float* s_t,
                             float* mu_hat, float* ls_hat) {
  cudaStream_t s = ctx->stream;
  const int nb = b->NB;
  BF_TRY(set_attrs(ctx, net));
  BF_TRY(ensure_batch(ctx, net, nb));
  BandView bv = band_view(b);
  k_features<<<nb, 256, 0, s>>>(bv, b->tsdf, b->d, net->act[0]);
  count_launch();
  LossArgs none;
  memset(&none, 0, sizeof(none));
  conv_tc<16, 32, MODE_FWD>(s, net, nb, net->act[0], net->wf[0], net->p + net->boff[0], CO_REAL[0], net->act[1],
                            nullptr, none);
  conv_tc<32, 32, MODE_FWD>(s, net, nb, net->act[1], net->wf[1], net->p + net->boff[1], CO_REAL[1], net->act[2],
                            nullptr, none);
  conv_tc<32, 32, MODE_FWD>(s, net, nb, net->act[2], net->wf[2], net->p + net->boff[2], CO_REAL[2], net->act[3],
                            nullptr, none);
  LossArgs la;
  la.B = bv;
  la.tsdf = b->tsdf;
  la.qd = b->qd;
  la.mu_t = mu_t;
  la.s_t = s_t;
  la.mu_hat = mu_hat;
  la.ls_hat = ls_hat;
  la.inv_m = b->N > 0 ? 1.0 / (double)b->N : 0.0;
  la.loss = mu_t ? net->loss : nullptr;
  if (mu_t) BF_CK(cudaMemsetAsync(net->loss, 0, sizeof(double), s));
  conv_tc<32, 16, MODE_LAST>(s, net, nb, net->act[3], net->wf[3], net->p + net->boff[3], CO_REAL[3], net->act[4],
                             nullptr, la);
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// gradient of the loss of the last net_forward with targets, into net->g
static bf_status net_backward(bf_ctx* ctx, bf_net* net, const bf_band* b) {
  cudaStream_t s = ctx->stream;
  const int nb = b->NB;
  for (int l = 0; l < 4; ++l) BF_CK(cudaMemsetAsync(net->gpad[l], 0, (size_t)27 * CI_PAD[l] * CO_PAD[l] * 4, s));
  BF_CK(cudaMemsetAsync(net->g, 0, net->P * 4, s));
  LossArgs none;
  memset(&none, 0, sizeof(none));
  // layer 4 (dy = act[4], written by the forward pass)
  k_wgrad<32, 16><<<occ_grid(k_wgrad<32, 16>, wgrad_smem<32, 16>(), nb), NT, wgrad_smem<32, 16>(), s>>>(nb, net->act[3], net->act[4], net->gpad[3],
                                                         net->g + net->boff[3], CO_REAL[3]);
  conv_tc<16, 32, MODE_DGRAD>(s, net, nb, net->act[4], net->wb[3], nullptr, 0, net->gact[2], net->act[3], none);
  // layer 3
  k_wgrad<32, 32><<<occ_grid(k_wgrad<32, 32>, wgrad_smem<32, 32>(), nb), NT, wgrad_smem<32, 32>(), s>>>(nb, net->act[2], net->gact[2], net->gpad[2],
                                                         net->g + net->boff[2], CO_REAL[2]);
  conv_tc<32, 32, MODE_DGRAD>(s, net, nb, net->gact[2], net->wb[2], nullptr, 0, net->gact[1], net->act[2], none);
  // layer 2
  k_wgrad<32, 32><<<occ_grid(k_wgrad<32, 32>, wgrad_smem<32, 32>(), nb), NT, wgrad_smem<32, 32>(), s>>>(nb, net->act[1], net->gact[1], net->gpad[1],
                                                         net->g + net->boff[1], CO_REAL[1]);
  conv_tc<32, 32, MODE_DGRAD>(s, net, nb, net->gact[1], net->wb[1], nullptr, 0, net->gact[0], net->act[1], none);
  // layer 1
  k_wgrad<16, 32><<<occ_grid(k_wgrad<16, 32>, wgrad_smem<16, 32>(), nb), NT, wgrad_smem<16, 32>(), s>>>(nb, net->act[0], net->gact[0], net->gpad[0],
                                                         net->g + net->boff[0], CO_REAL[0]);
  count_launch(4);  // the weight-gradient launches (conv_tc counts its own)
  for (int l = 0; l < 4; ++l) {
    k_unpad_grad<<<gs(27 * CI_REAL[l] * CO_REAL[l]), 256, 0, s>>>(net->gpad[l], CI_REAL[l], CO_REAL[l], CI_PAD[l],
                                                                 CO_PAD[l], net->g + net->woff[l]);
    count_launch();
  }
  BF_CK(cudaGetLastError());
  return BF_OK;
}

// synchronise and report a tensor-core kernel whose MMAs did not complete in time
static bf_status net_sync_check(bf_ctx* ctx, bf_net* net) {
  int* h_err = reinterpret_cast<int*>(net->h_loss + 1);
  BF_CK(cudaMemcpyAsync(h_err, net->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  if (*h_err) {
    *h_err = 0;
    cudaMemsetAsync(net->err, 0, sizeof(int), ctx->stream);
    return bf_fail(ctx, BF_ECUDA, "network: tensor-core MMAs did not complete in time");
  }
  return BF_OK;
}

extern "C" {

int64_t bf_net_nparams(void) { return nparams_impl(); }

bf_status bf_net_create(bf_ctx* ctx, uint64_t seed, bf_net** out) {
  BF_ENTER(ctx);
  if (!ctx || !out) return BF_EINVAL;
  bf_net* net = new bf_net();
  net->device = ctx->device;
  net->P = nparams_impl();
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    net->woff[l] = o;
    o += 27 * CI_REAL[l] * CO_REAL[l];
    net->boff[l] = o;
    o += CO_REAL[l];
  }
  auto fail = [&](bf_status st) {
    bf_net_destroy(net);
    return st;
  };
  if (cudaMalloc(&net->p, net->P * 4) || cudaMalloc(&net->g, net->P * 4) || cudaMalloc(&net->m, net->P * 4) ||
      cudaMalloc(&net->v, net->P * 4) || cudaMalloc(&net->loss, sizeof(double)) || cudaMalloc(&net->err, sizeof(int)) ||
      cudaMallocHost(&net->h_loss, 2 * sizeof(double)))
    return fail(bf_fail(ctx, BF_ENOMEM, "bf_net_create: allocation failed"));
  for (int l = 0; l < 4; ++l) {
    const size_t nw = (size_t)27 * CI_PAD[l] * CO_PAD[l];
    if (cudaMalloc(&net->wf[l], nw * 2) || cudaMalloc(&net->wb[l], nw * 2) || cudaMalloc(&net->gpad[l], nw * 4))
      return fail(bf_fail(ctx, BF_ENOMEM, "bf_net_create: allocation failed"));
  }
  cudaStream_t s = ctx->stream;
  k_init<<<gs(net->P), 256, 0, s>>>(net->p, net->P, seed, net->woff[0], net->boff[0], net->woff[1], net->boff[1],
                                    net->woff[2], net->boff[2], net->woff[3], net->boff[3]);
  count_launch();
  cudaMemsetAsync(net->m, 0, net->P * 4, s);
  cudaMemsetAsync(net->v, 0, net->P * 4, s);
  cudaMemsetAsync(net->err, 0, sizeof(int), s);
  bf_status st = net_pack(ctx, net);
  if (st) return fail(st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(bf_fail(ctx, BF_ECUDA, "bf_net_create"));
  *out = net;
  return BF_OK;
}

void bf_net_destroy(bf_net* net) {
  if (!net) return;
  enter_device(net->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {net->p, net->g, net->m, net->v, net->loss, net->err};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (net->h_loss) cudaFreeHost(net->h_loss);
  for (int l = 0; l < 4; ++l) {
    if (net->wf[l]) cudaFree(net->wf[l]);
    if (net->wb[l]) cudaFree(net->wb[l]);
    if (net->gpad[l]) cudaFree(net->gpad[l]);
  }
  for (auto a : net->act)
    if (a) cudaFree(a);
  for (auto a : net->gact)
    if (a) cudaFree(a);
  delete net;
}

bf_status bf_net_get_params(bf_ctx* ctx, const bf_net* net, float* params) {
  BF_ENTER(ctx);
  if (!ctx || !net || !params) return BF_EINVAL;
  BF_CK(cudaMemcpyAsync(params, net->p, net->P * 4, cudaMemcpyDefault, ctx->stream));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return BF_OK;
}

bf_status bf_net_set_params(bf_ctx* ctx, bf_net* net, const float* params) {
  BF_ENTER(ctx);
  if (!ctx || !net || !params) return BF_EINVAL;
  BF_CK(cudaMemcpyAsync(net->p, params, net->P * 4, cudaMemcpyDefault, ctx->stream));
  BF_CK(cudaMemsetAsync(net->m, 0, net->P * 4, ctx->stream));
  BF_CK(cudaMemsetAsync(net->v, 0, net->P * 4, ctx->stream));
  net->step = 0;
  BF_TRY(net_pack(ctx, net));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return BF_OK;
}

bf_status bf_net_forward(bf_ctx* ctx, bf_net* net, const bf_band* b, float* mu_hat, float* log_s_hat) {
  BF_ENTER(ctx);
  if (!ctx || !net || !b || !mu_hat || !log_s_hat) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_net_forward: call bf_integrate_depth first");
  if (b->N == 0) return BF_OK;
  float *dm, *dl;
  bool hm, hl;
  BF_TRY(stage_out(ctx, mu_hat, b->N, WS_OUT0, &dm, &hm));
  BF_TRY(stage_out(ctx, log_s_hat, b->N, WS_OUT1, &dl, &hl));
  BF_TRY(net_forward(ctx, net, b, nullptr, nullptr, dm, dl));
  BF_TRY(net_sync_check(ctx, net));
  BF_TRY(copy_out(ctx, mu_hat, (const float*)dm, b->N, hm));
  BF_TRY(copy_out(ctx, log_s_hat, (const float*)dl, b->N, hl));
  return BF_OK;
}

bf_status bf_net_train_step(bf_ctx* ctx, bf_net* net, const bf_band* b, const float* mu_t, const float* s_t,
                            float lr, double* loss, float* grad_out) {
  BF_ENTER(ctx);
  if (!ctx || !net || !b || !mu_t || !s_t) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_net_train_step: call bf_integrate_depth first");
  if (!(lr >= 0.0f) || !(lr < 1.0f)) return bf_fail(ctx, BF_EINVAL, "bf_net_train_step: need 0 <= lr < 1");
  if (b->N == 0) {
    if (loss) *loss = 0.0;
    return BF_OK;
  }
  cudaStream_t s = ctx->stream;
  const float *dmu, *dst;
  BF_TRY(stage_in(ctx, mu_t, b->N, WS_STAGE2, &dmu));
  BF_TRY(stage_in(ctx, s_t, b->N, WS_STAGE3, &dst));
  BF_TRY(net_forward(ctx, net, b, dmu, dst, nullptr, nullptr));
  BF_TRY(net_backward(ctx, net, b));
  BF_CK(cudaGetLastError());
  if (grad_out) BF_CK(cudaMemcpyAsync(grad_out, net->g, net->P * 4, cudaMemcpyDefault, s));
  if (lr > 0.0f) {
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)net->step), c2 = 1.0f - powf(b2, (float)net->step);
    k_adam<<<gs(net->P), 256, 0, s>>>((int)net->P, net->p, net->g, net->m, net->v, lr, b1, b2, c1, c2, 1e-8f);
    count_launch();
    BF_TRY(net_pack(ctx, net));
  }
  BF_CK(cudaMemcpyAsync(net->h_loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  BF_TRY(net_sync_check(ctx, net));
  if (loss) *loss = *net->h_loss;
  return BF_OK;
}

bf_status bf_surrogate_variance(bf_ctx* ctx, bf_band* b, const float* log_s_hat, int K, int K_judge, uint64_t seed,
                                double rel_tol, int max_iter, int rhs_block, unsigned flags, float* s,
                                uint8_t* accepted, double* brick_stat, int* n_accepted, int* total_iters) {
  BF_ENTER(ctx);
  if (!ctx || !b || !log_s_hat || !s) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_surrogate_variance: call bf_integrate_depth first");
  if (b->obs_mode == 3) return bf_fail(ctx, BF_ESTATE, "bf_surrogate_variance: the band holds trilinear rows");
  if (K_judge < 2 || K <= K_judge || !(rel_tol > 0.0) || !(rel_tol < 1.0) || max_iter < 1 || max_iter > 10000000)
    return bf_fail(ctx, BF_EINVAL, "bf_surrogate_variance: need 2 <= K_judge < K, 0 < rel_tol < 1");
  if (rhs_block != 0 && rhs_block != 1 && rhs_block != 8 && rhs_block != 16 && rhs_block != 32)
    return bf_fail(ctx, BF_EINVAL, "bf_surrogate_variance: rhs_block must be 0, 1, 8, 16 or 32");
  if (n_accepted) *n_accepted = 0;
  if (total_iters) *total_iters = 0;
  if (b->N == 0) return BF_OK;
  cudaStream_t st = ctx->stream;
  const int N = (int)b->N, NB = b->NB;
  const float* dl;
  float* ds;
  bool hs;
  BF_TRY(stage_in(ctx, log_s_hat, N, WS_STAGE2, &dl));
  BF_TRY(stage_out(ctx, s, N, WS_OUT0, &ds, &hs));
  float *sJ = nullptr, *rest = nullptr;
  double *sq = nullptr, *s1 = nullptr, *stat = nullptr;
  uint8_t* acc = nullptr;
  int* nacc = nullptr;
  bf_status r = BF_OK;
  auto done = [&](bf_status x) {
    dev_free(st, sJ);
    dev_free(st, rest);
    dev_free(st, sq);
    dev_free(st, s1);
    dev_free(st, stat);
    dev_free(st, acc);
    dev_free(st, nacc);
    return x;
  };
  if ((r = dev_alloc_t(ctx, &sJ, N)) || (r = dev_alloc_t(ctx, &rest, N)) || (r = dev_alloc_t(ctx, &sq, N)) ||
      (r = dev_alloc_t(ctx, &s1, N)) ||
      (r = dev_alloc_t(ctx, &stat, 2 * (size_t)NB)) || (r = dev_alloc_t(ctx, &acc, NB)) ||
      (r = dev_alloc_t(ctx, &nacc, 1)))
    return done(r);
  if (cudaMemsetAsync(sq, 0, (size_t)N * 8, st) || cudaMemsetAsync(nacc, 0, 4, st))
    return done(bf_fail(ctx, BF_ECUDA, "bf_surrogate_variance: memset"));
  // judge: probes 0 .. K_judge - 1 (the first K_judge probes of the K-probe estimate)
  int it_j = 0, it_r = 0;
  r = variance_impl(ctx, b, 0, K_judge, 1.0 / K_judge, seed, rel_tol, max_iter, rhs_block, flags, sJ, &it_j, sq, s1);
  if (r) return done(r);
  k_judge<<<NB, 256, 0, st>>>(b->off, b->qd, dl, s1, sq, K_judge, stat, acc, nacc);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return done(bf_fail(ctx, BF_ECUDA, "k_judge launch"));
  int h_nacc = 0;
  if (cudaMemcpyAsync(ctx->h_pinned, nacc, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
    return done(bf_fail(ctx, BF_ECUDA, "bf_surrogate_variance: read acceptance count"));
  memcpy(&h_nacc, ctx->h_pinned, 4);
  // rejected bricks: the remaining probes K_judge .. K - 1
  if (h_nacc < NB) {
    r = variance_impl(ctx, b, K_judge, K, 1.0, seed, rel_tol, max_iter, rhs_block, flags, rest, &it_r, nullptr);
    if (r) return done(r);
  }
  k_surrogate_fill<<<NB, 256, 0, st>>>(b->off, dl, sJ, h_nacc < NB ? rest : nullptr, acc, K_judge, K, ds);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return done(bf_fail(ctx, BF_ECUDA, "k_surrogate_fill launch"));
  if (accepted && cudaMemcpyAsync(accepted, acc, NB, cudaMemcpyDefault, st))
    return done(bf_fail(ctx, BF_ECUDA, "bf_surrogate_variance: copy accepted"));
  if (brick_stat && cudaMemcpyAsync(brick_stat, stat, (size_t)NB * 16, cudaMemcpyDefault, st))
    return done(bf_fail(ctx, BF_ECUDA, "bf_surrogate_variance: copy brick_stat"));
  r = copy_out(ctx, s, (const float*)ds, N, hs);
  if (r) return done(r);
  if (cudaStreamSynchronize(st)) return done(bf_fail(ctx, BF_ECUDA, "bf_surrogate_variance"));
  if (n_accepted) *n_accepted = h_nacc;
  if (total_iters) *total_iters = it_j + it_r;
  return done(BF_OK);
}

bf_status bf_net_bench(bf_ctx* ctx, bf_net* net, const bf_band* b, int which, int reps, double* ms) {
  BF_ENTER(ctx);
  if (!ctx || !net || !b || !ms || reps < 1 || which < 0 || which > 4) return BF_EINVAL;
  if (!b->integrated) return bf_fail(ctx, BF_ESTATE, "bf_net_bench: call bf_integrate_depth first");
  *ms = 0.0;
  if (b->NB == 0) return BF_OK;
  cudaStream_t s = ctx->stream;
  const int nb = b->NB;
  // one forward with (arbitrary, finite) targets so that every buffer holds data
  BF_TRY(net_forward(ctx, net, b, b->tsdf, b->d, nullptr, nullptr));
  LossArgs none;
  memset(&none, 0, sizeof(none));
  cudaEvent_t e0, e1;
  BF_CK(cudaEventCreate(&e0));
  BF_CK(cudaEventCreate(&e1));
  BF_CK(cudaEventRecord(e0, s));
  for (int i = 0; i < reps; ++i) {
    if (which == BF_NET_BENCH_FORWARD) {
      BF_TRY(net_forward(ctx, net, b, nullptr, nullptr, nullptr, nullptr));
    } else if (which == BF_NET_BENCH_TRAIN) {
      BF_TRY(net_forward(ctx, net, b, b->tsdf, b->d, nullptr, nullptr));
      BF_TRY(net_backward(ctx, net, b));
    } else if (which == BF_NET_BENCH_CONV) {
      conv_tc<32, 32, MODE_FWD>(s, net, nb, net->act[1], net->wf[1], net->p + net->boff[1], CO_REAL[1], net->act[2],
                                nullptr, none);
    } else if (which == BF_NET_BENCH_CONV_MMA) {
      k_conv<32, 32, MODE_FWD><<<occ_grid(k_conv<32, 32, MODE_FWD>, conv_smem<32, 32>(), nb), NT, conv_smem<32, 32>(),
                                 s>>>(nb, net->act[1], net->wf[1], net->p + net->boff[1], CO_REAL[1], net->act[2],
                                      nullptr, none);
      count_launch();
    } else {
      k_wgrad<32, 32><<<occ_grid(k_wgrad<32, 32>, wgrad_smem<32, 32>(), nb), NT, wgrad_smem<32, 32>(), s>>>(nb, net->act[1], net->act[2], net->gpad[1],
                                                             net->g + net->boff[1], CO_REAL[1]);
      count_launch();
    }
  }
  BF_CK(cudaEventRecord(e1, s));
  BF_CK(cudaEventSynchronize(e1));
  float t = 0.0f;
  BF_CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return net_sync_check(ctx, net);
}

}  // extern "C"
