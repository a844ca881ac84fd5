// Internal declarations of the GB300 posterior-solver library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bfsdf.h"

// ------------------------------------------------------------- host side

#define BF_CK(call)                                                                    \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess) return bf_fail(ctx, BF_ECUDA, #call, cudaGetErrorString(e__)); \
  } while (0)

#define BF_TRY(call)                     \
  do {                                   \
    bf_status s__ = (call);              \
    if (s__ != BF_OK) return s__;        \
  } while (0)

// Every entry point that takes a context runs on the context's device: the
// calling thread's current device is switched to it (and left there).
inline cudaError_t enter_device(int device) {
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur == device) return cudaSuccess;
  return cudaSetDevice(device);
}
#define BF_ENTER(ctx)                                                                       \
  do {                                                                                      \
    if (!(ctx)) return BF_EINVAL;                                                           \
    cudaError_t e__ = enter_device((ctx)->device);                                          \
    if (e__ != cudaSuccess) return bf_fail(ctx, BF_ECUDA, "cudaSetDevice", cudaGetErrorString(e__)); \
  } while (0)

// Refinement passes (true-residual recomputation and restart) of the mean
// solvers before they report BF_NOT_CONVERGED.
constexpr int REFINE_MAX_PASSES = 64;

struct Workspace {
  void* p = nullptr;
  size_t cap = 0;
};

enum { WS_STAGE0 = 0, WS_STAGE1, WS_STAGE2, WS_STAGE3, WS_OUT0, WS_OUT1, WS_TMP0, WS_TMP1, WS_TMP2, WS_TMP3,
       WS_TMP4, WS_TMP5, WS_SCAN, WS_COUNT };

struct SolveGraph;  // solve.cu
struct BlockGraph;  // block.cu

// a tuned probe-block width: band size class, probe-count class, choice, ms per iteration at R = 8, 16, 32
struct TuneEntry {
  int n_log2, k_class, R;
  double ms[3];
};

struct bf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  Workspace ws[WS_COUNT];
  int32_t* h_pinned = nullptr;  // small pinned scratch for scalars read back
  int* d_err = nullptr;         // device word set by a kernel whose bounded wait ran out
  // last extracted mesh
  float* mesh_v = nullptr;
  int32_t* mesh_t = nullptr;
  int64_t mesh_nv = 0, mesh_nt = 0;
  size_t mesh_vcap = 0, mesh_tcap = 0;
  int8_t* mc_table = nullptr;   // device [256][16][3] edge triples, -1 padded
  int8_t* mc_ntri = nullptr;    // device [256]
  BlockGraph* blk[3] = {nullptr, nullptr, nullptr};  // probe solvers, R = 8, 16, 32
  SolveGraph* sgl[2] = {nullptr, nullptr};           // mean solvers, FP32 and FP64
  std::vector<TuneEntry> tune;                       // autotuned probe-block widths
  bool tune_loaded = false;
};

// Per-brick lookup entry: band bits of 32 local voxels and the compact index
// of the first of them (brick offset + band voxels in earlier words).
struct __align__(8) MetaWord {
  uint32_t bits;
  int32_t base;
};

struct bf_band {
  bf_grid grid;
  bf_params prm;
  int nb = 0;
  int32_t NB = 0;
  int64_t N = 0;
  int64_t ncand = 0;
  cudaStream_t stream = nullptr;  // stream the arrays were allocated on
  int device = 0;                 // device that holds them
  // directory and per-brick data
  int32_t* dir = nullptr;     // [nb^3] rank or -1
  int32_t* bcoord = nullptr;  // [NB][4] (bi, bj, bk, 0)
  MetaWord* meta = nullptr;   // [NB][16]
  int32_t* off = nullptr;     // [NB+1]
  int32_t* nbr = nullptr;     // [NB][6]  -x,+x,-y,+y,-z,+z
  // per-voxel data
  int32_t* lin = nullptr;     // [N]
  float* tsdf = nullptr;      // [N] metres
  int32_t* wcount = nullptr;  // [N]
  uint8_t* info = nullptr;    // [N] deg | bdry << 3
  float* d = nullptr;         // [N] sum w
  float* hd = nullptr;        // [N] sum w y
  // deterministic accumulation: sum w and sum w y as int64 in units of 2^-OBS_FIX_BITS (exact, order-free)
  int64_t* dfx = nullptr;
  int64_t* hfx = nullptr;
  int obs_mode = 0;           // observations accumulated since the last reset: 0 none, 1 FP32 atomics, 2 fixed point
  float* qd = nullptr;        // [N] Q_jj
  float* rhs = nullptr;       // [N] h_j
  bool integrated = false;
  int32_t* nb6 = nullptr;     // [N][6] face-neighbour indices (probe solver)
  int32_t* sp_ext = nullptr;  // probe-solver SpMM plan: external rows per tile
  int32_t* sp_ne = nullptr;   //   their count per tile
  int16_t* sp_slot = nullptr; //   [N][8] staged-row slot of each face neighbour
  // trilinear observation rows (obs_mode 3): the data term A^T W A on the 14 offsets o >= 13 of the 27-point
  // neighbourhood ([14][N], entry o - 13 of voxel j = the coupling of j with j + off(o)), and the assembled
  // 27-point precision ([27][N], coefficient o of voxel j = Q_{j, j + off(o)})
  float* c27 = nullptr;
  float* q27 = nullptr;
};

// POD view of a band passed to kernels.
struct BandView {
  int n, nb, NB, N;
  float h, o0, o1, o2;
  const int32_t* dir;
  const MetaWord* meta;
  const int32_t* off;
  const int32_t* nbr;
  const int32_t* bcoord;
  const int32_t* lin;
};

struct Intr {
  float fx, fy, cx, cy;
  int W, H;
};

bf_status bf_fail(bf_ctx* ctx, bf_status st, const char* what, const char* detail = nullptr);
void* ws_get(bf_ctx* ctx, int slot, size_t bytes, bf_status* st);
bool is_device_ptr(const void* p);
BandView band_view(const bf_band* b);
bf_status dev_alloc(bf_ctx* ctx, void** p, size_t bytes);
template <class T>
inline bf_status dev_alloc_t(bf_ctx* ctx, T** p, size_t count) {
  return dev_alloc(ctx, (void**)p, count * sizeof(T));
}
void dev_free(cudaStream_t s, void* p);

// Device view of a caller array: the array itself if it is device memory,
// else a staged copy in workspace slot `slot`.
template <class T>
inline bf_status stage_in(bf_ctx* ctx, const T* p, size_t count, int slot, const T** out) {
  if (is_device_ptr(p)) {
    *out = p;
    return BF_OK;
  }
  bf_status st;
  T* d = (T*)ws_get(ctx, slot, count * sizeof(T), &st);
  if (st) return st;
  BF_CK(cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  *out = d;
  return BF_OK;
}

// Output target: the caller array if device memory, else a workspace buffer
// that copy_out writes back.
template <class T>
inline bf_status stage_out(bf_ctx* ctx, T* p, size_t count, int slot, T** out, bool* host) {
  *host = !is_device_ptr(p);
  if (!*host) {
    *out = p;
    return BF_OK;
  }
  bf_status st;
  *out = (T*)ws_get(ctx, slot, count * sizeof(T), &st);
  return st;
}

template <class T>
inline bf_status copy_out(bf_ctx* ctx, T* user, const T* dev, size_t count, bool host) {
  if (!host) return BF_OK;
  BF_CK(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  BF_CK(cudaStreamSynchronize(ctx->stream));
  return BF_OK;
}

// Exclusive prefix sum of n int32 values (in and out may alias); *total
// (device, may be null) receives the sum.
bf_status scan_i32(bf_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, int32_t* total);

// Module entry points (host side of each .cu file).
bf_status band_build(bf_ctx* ctx, const float* depth, int T, const float* poses, const Intr& K, const bf_grid& g,
                     const bf_params& p, bf_band** out);
bf_status band_integrate(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses, const Intr& K,
                         bool fixed_point = false);
constexpr int OBS_FIX_BITS = 32;
bf_status band_assemble(bf_ctx* ctx, bf_band* b);
// trilinear observation rows (tri.cu)
bf_status tri_integrate(bf_ctx* ctx, bf_band* b, const float* depth, int T, const float* poses, const Intr& K);
bf_status tri_rows(bf_ctx* ctx, const bf_band* b, const float* depth, int T, const float* poses, const Intr& K,
                   int32_t* idx, float* wts, uint8_t* used);
bf_status tri_spmv(bf_ctx* ctx, const bf_band* b, const float* x, float* y);
bf_status tri_solve_mean(bf_ctx* ctx, bf_band* b, double tol, int max_iter, float* mu, int* iters, double* relres);
bf_status tri_variance(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                       int max_iter, float* s, int* total_iters);
constexpr int TRI_R = 8;  // probe columns per block of the trilinear probe solver
bf_status band_observations_f64(bf_ctx* ctx, const bf_band* b, double* d64, double* h64);
bf_status spmv_launch(bf_ctx* ctx, const bf_band* b, const float* x, float* y);
// After the stream has been synchronised: BF_ECUDA if a kernel's bounded wait ran out since the last check
// (the context's device error word, which is then cleared), else BF_OK.
bf_status device_wait_status(bf_ctx* ctx, const char* what);
bf_status spmm_launch(bf_ctx* ctx, bf_band* b, const float* X, int R, float* Y);
bf_status solve_mean_impl(bf_ctx* ctx, bf_band* b, double tol, int max_iter, unsigned flags, float* mu, int* iters,
                          double* relres);
bf_status solve_rhs_impl(bf_ctx* ctx, bf_band* b, const float* rhs, double tol, int max_iter, float* x, int* iters,
                         double* relres);
bf_status variance_impl(bf_ctx* ctx, bf_band* b, int kb, int ke, double scale, uint64_t seed, double tol,
                        int max_iter, int R, unsigned flags, float* s, int* total_iters, double* sq = nullptr,
                        double* s1 = nullptr);
bf_status bench_block_iter(bf_ctx* ctx, bf_band* b, int R, int reps, double* ms);
bf_status autotune_rhs_block(bf_ctx* ctx, bf_band* b, int K, bool force, int* R_out, double ms_out[3]);
void solve_graph_free(SolveGraph* g);
void block_graph_free(BlockGraph* g);
bf_status mc_impl(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt);
bf_status dc_impl(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt);
bf_status nbv_exact_impl(bf_ctx* ctx, bf_band* b, const float* mu, const float* cand, int V, const Intr& K,
                         double eps, int Kp, uint64_t seed, double tol, int max_iter, int R, double* U, int* best,
                         int* total_iters);
bf_status nbv_impl(bf_ctx* ctx, const bf_band* b, const float* mu, const float* s, const float* cand, int V,
                   const Intr& K, double eps, double* U, int* best);

// ---------------------------------------------------------- device side

#ifdef __CUDACC__

// FP32 specification arithmetic: each operation rounded separately (no FMA
// contraction), so discrete decisions are reproducible bit for bit.
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_div(float a, float b) { return __fdiv_rn(a, b); }

struct Pose {
  float R[9];
  float C[3];
};

__device__ __forceinline__ Pose load_pose(const float* __restrict__ P) {
  Pose q;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) q.R[3 * a + b] = P[4 * a + b];
    q.C[a] = P[4 * a + 3];
  }
  return q;
}

__device__ __forceinline__ bool depth_ok(float D) { return D > 0.0f && D < __int_as_float(0x7f800000); }

// voxel centre coordinate along one axis: org + (i + 1/2) h
__device__ __forceinline__ float vox_c(float org, float h, int i) {
  return f_add(org, f_mul(f_add((float)i, 0.5f), h));
}

// pixel ray: dw = R K^-1 (px+1/2, py+1/2, 1), nrm = |K^-1 u|, r = dw / nrm
struct Ray {
  float dw[3], r[3], nrm;
};

__device__ __forceinline__ Ray pixel_ray(const Pose& P, int px, int py, const Intr& K) {
  Ray q;
  float a = f_div(f_sub(f_add((float)px, 0.5f), K.cx), K.fx);
  float b = f_div(f_sub(f_add((float)py, 0.5f), K.cy), K.fy);
  q.nrm = __fsqrt_rn(f_add(f_add(f_mul(a, a), f_mul(b, b)), 1.0f));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q.dw[k] = f_add(f_add(f_mul(P.R[3 * k], a), f_mul(P.R[3 * k + 1], b)), P.R[3 * k + 2]);
    q.r[k] = f_div(q.dw[k], q.nrm);
  }
  return q;
}

// bring bytes of v[i0 .. i1) into L2 as whole lines (bulk prefetch of the 16-byte granules inside the range)
template <class E>
__device__ __forceinline__ void prefetch_range(const E* v, int64_t i0, int64_t i1) {
  const uint64_t a0 = ((uint64_t)(v + i0) + 15u) & ~(uint64_t)15u, a1 = (uint64_t)(v + i1) & ~(uint64_t)15u;
  if (a1 > a0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
}

// compact index of voxel (i,j,k) or -1 if outside the band
__device__ __forceinline__ int band_lookup(const BandView& B, int i, int j, int k) {
  if ((unsigned)i >= (unsigned)B.n || (unsigned)j >= (unsigned)B.n || (unsigned)k >= (unsigned)B.n) return -1;
  int r = __ldg(B.dir + ((i >> 3) + B.nb * ((j >> 3) + B.nb * (k >> 3))));
  if (r < 0) return -1;
  int l = (i & 7) + 8 * (j & 7) + 64 * (k & 7);
  MetaWord m = B.meta[16 * r + (l >> 5)];
  uint32_t bit = 1u << (l & 31);
  if (!(m.bits & bit)) return -1;
  return m.base + __popc(m.bits & (bit - 1u));
}

// FP32-spec 3-D DDA over s in [sp - tau, sp + tau]; calls f(i, j, k) for each
// voxel entered (ties broken x < y < z), at most max_steps voxels.
template <class F>
__device__ __forceinline__ void dda_walk(const float C[3], const float r[3], float sp, float tau, float h,
                                         const float org[3], int max_steps, F&& f) {
  float s0 = f_sub(sp, tau);
  if (s0 < 0.0f) s0 = 0.0f;
  float s1 = f_add(sp, tau);
  float P0[3], tmax[3], tdel[3];
  int idx[3], step[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P0[k] = f_add(C[k], f_mul(s0, r[k]));
    float g = f_div(f_sub(P0[k], org[k]), h);
    if (!(fabsf(g) < 1.0e6f)) return;
    idx[k] = (int)floorf(g);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (r[k] > 0.0f) {
      step[k] = 1;
      tdel[k] = f_div(h, r[k]);
      float bnd = f_add(org[k], f_mul((float)(idx[k] + 1), h));
      tmax[k] = f_add(s0, f_div(f_sub(bnd, P0[k]), r[k]));
    } else if (r[k] < 0.0f) {
      step[k] = -1;
      tdel[k] = f_div(h, -r[k]);
      float bnd = f_add(org[k], f_mul((float)idx[k], h));
      tmax[k] = f_add(s0, f_div(f_sub(bnd, P0[k]), r[k]));
    } else {
      step[k] = 0;
      tdel[k] = __int_as_float(0x7f800000);
      tmax[k] = __int_as_float(0x7f800000);
    }
  }
  for (int it = 0; it < max_steps; ++it) {
    f(idx[0], idx[1], idx[2]);
    int a = (tmax[0] <= tmax[1] && tmax[0] <= tmax[2]) ? 0 : (tmax[1] <= tmax[2] ? 1 : 2);
    float ta = a == 0 ? tmax[0] : (a == 1 ? tmax[1] : tmax[2]);
    if (ta > s1) break;
    if (a == 0) { idx[0] += step[0]; tmax[0] = f_add(tmax[0], tdel[0]); }
    else if (a == 1) { idx[1] += step[1]; tmax[1] = f_add(tmax[1], tdel[1]); }
    else { idx[2] += step[2]; tmax[2] = f_add(tmax[2], tdel[2]); }
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): the mixing function of the
// counter-based probe generator.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__host__ __device__ inline int dda_max_steps(double band_vox) {
  return 3 * (int)ceil(2.0 * band_vox) + 12;
}

__host__ __device__ inline int brick_radius(double trunc_vox) {
  return (int)floor((1.25 * trunc_vox + 2.0) / 8.0) + 1;
}

#endif  // __CUDACC__

// Kernels launched by this library (host launches plus graph-body kernel
// executions), process-wide.
void count_launch(int64_t n = 1);
int64_t launch_total();
