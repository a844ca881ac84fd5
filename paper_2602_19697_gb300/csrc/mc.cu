// Marching cubes on the posterior mean (Sec. 3.8 surface extraction;
// Algorithm 1 step 7).
//
// Case table (built on the host once per context): for each of the 256 sign
// cases, each cube face is walked counter-clockwise as seen from outside the
// cube (corners sorted by angle about the face centre in a frame whose
// normal points out); every run of inside corners contributes a directed
// segment from the crossed edge where the walk enters the run to the one
// where it leaves it (so an ambiguous face separates its inside corners).
// Segments chain into closed loops; each loop, started from its
// lowest-numbered edge, is fan-triangulated.  Edge e = 4 axis + u + 2 v with
// (u, v) the lower corner's coordinates on the other two axes in ascending
// axis order; corner c = x + 2 y + 4 z.
//
// Kernels: classify (case, triangle count, used edges) -> scans -> emit
// triangles and vertices.  Vertices are numbered by (compact index of the
// edge's lower voxel, axis); triangles by the compact index of the cube's
// lower corner voxel, then table order -- so topology is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

struct CaseTable {
  int8_t tri[256][16][3];
  int8_t n[256];
};

int edge_between(int ca, int cb) {
  int d = ca ^ cb;
  int axis = d == 1 ? 0 : (d == 2 ? 1 : 2);
  int lo = ca & cb;
  int other[2], m = 0;
  for (int a = 0; a < 3; ++a)
    if (a != axis) other[m++] = (lo >> a) & 1;
  return 4 * axis + other[0] + 2 * other[1];
}

void build_case_table(CaseTable& T) {
  // faces: 4 corners each, sorted counter-clockwise seen from outside
  std::vector<std::vector<int>> faces;
  for (int axis = 0; axis < 3; ++axis)
    for (int side = 0; side < 2; ++side) {
      double n[3] = {0, 0, 0};
      n[axis] = side ? 1.0 : -1.0;
      double e1[3] = {0, 0, 0};
      e1[(axis + 1) % 3] = 1.0;
      double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
      std::vector<std::pair<double, int>> cs;
      for (int c = 0; c < 8; ++c) {
        if (((c >> axis) & 1) != side) continue;
        double p[3] = {(c & 1) - 0.5, ((c >> 1) & 1) - 0.5, ((c >> 2) & 1) - 0.5};
        double x = p[0] * e1[0] + p[1] * e1[1] + p[2] * e1[2];
        double y = p[0] * e2[0] + p[1] * e2[1] + p[2] * e2[2];
        cs.push_back({std::atan2(y, x), c});
      }
      std::sort(cs.begin(), cs.end());
      std::vector<int> f;
      for (auto& q : cs) f.push_back(q.second);
      faces.push_back(f);
    }
  for (int cs = 0; cs < 256; ++cs) {
    auto inside = [&](int c) { return (cs >> c) & 1; };
    int next[12];
    for (int& x : next) x = -1;
    for (const auto& f : faces) {
      for (int m = 0; m < 4; ++m) {
        int a = f[m], b = f[(m + 1) % 4];
        if (inside(a) || !inside(b)) continue;  // look for outside -> inside
        int from = edge_between(a, b);
        for (int j = m + 1; j < m + 4; ++j) {
          int c0 = f[j % 4], c1 = f[(j + 1) % 4];
          if (inside(c0) && !inside(c1)) {
            next[from] = edge_between(c0, c1);
            break;
          }
        }
      }
    }
    int nt = 0;
    bool seen[12] = {false};
    for (int e0 = 0; e0 < 12; ++e0) {
      if (next[e0] < 0 || seen[e0]) continue;
      std::vector<int> loop;
      int e = e0;
      while (!seen[e] && (int)loop.size() < 12) {
        seen[e] = true;
        loop.push_back(e);
        e = next[e];
      }
      for (size_t i = 1; i + 1 < loop.size(); ++i) {
        T.tri[cs][nt][0] = (int8_t)loop[0];
        T.tri[cs][nt][1] = (int8_t)loop[i];
        T.tri[cs][nt][2] = (int8_t)loop[i + 1];
        ++nt;
      }
    }
    for (int t = nt; t < 16; ++t) T.tri[cs][t][0] = T.tri[cs][t][1] = T.tri[cs][t][2] = -1;
    T.n[cs] = (int8_t)nt;
  }
}

// corner of the edge's lower end, and the edge axis
__device__ __forceinline__ void edge_lower(int e, int* corner, int* axis) {
  int a = e >> 2, u = e & 1, v = (e >> 1) & 1;
  int c;
  if (a == 0) c = (u << 1) | (v << 2);
  else if (a == 1) c = u | (v << 2);
  else c = u | (v << 1);
  *corner = c;
  *axis = a;
}

__device__ __forceinline__ int cube_case(const BandView& B, const float* __restrict__ mu, int v, int ci[8]) {
  int L = B.lin[v];
  int i = L % B.n, j = (L / B.n) % B.n, k = L / (B.n * B.n);
  ci[0] = v;
  for (int c = 1; c < 8; ++c) {
    ci[c] = band_lookup(B, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1));
    if (ci[c] < 0) return -1;
  }
  int cs = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) cs |= (__ldg(mu + ci[c]) < 0.0f) << c;
  return cs;
}

__global__ void k_mc_classify(BandView B, const float* __restrict__ mu, const int8_t* __restrict__ table,
                              const int8_t* __restrict__ ntri, int32_t* __restrict__ tcount,
                              int32_t* __restrict__ vflag) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int ci[8];
    int cs = cube_case(B, mu, v, ci);
    int nt = cs < 0 ? 0 : ntri[cs];
    tcount[v] = nt;
    for (int t = 0; t < nt; ++t)
      for (int q = 0; q < 3; ++q) {
        int corner, axis;
        edge_lower(table[(cs * 16 + t) * 3 + q], &corner, &axis);
        vflag[3 * ci[corner] + axis] = 1;
      }
  }
}

__global__ void k_mc_emit(BandView B, const float* __restrict__ mu, const int8_t* __restrict__ table,
                          const int8_t* __restrict__ ntri, const int32_t* __restrict__ toff,
                          const int32_t* __restrict__ vid, int32_t* __restrict__ tris) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int ci[8];
    int cs = cube_case(B, mu, v, ci);
    if (cs < 0) continue;
    int nt = ntri[cs];
    int base = toff[v];
    for (int t = 0; t < nt; ++t)
      for (int q = 0; q < 3; ++q) {
        int corner, axis;
        edge_lower(table[(cs * 16 + t) * 3 + q], &corner, &axis);
        tris[3 * (base + t) + q] = vid[3 * ci[corner] + axis];
      }
  }
}

__global__ void k_mc_verts(BandView B, const float* __restrict__ mu, const int32_t* __restrict__ vflag,
                           const int32_t* __restrict__ vid, float* __restrict__ verts) {
  int64_t n3 = (int64_t)B.N * 3;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n3; q += (int64_t)gridDim.x * blockDim.x) {
    if (!vflag[q]) continue;
    int v = (int)(q / 3), a = (int)(q - 3 * (q / 3));
    int L = B.lin[v];
    int ijk[3] = {L % B.n, (L / B.n) % B.n, L / (B.n * B.n)};
    int up[3] = {ijk[0], ijk[1], ijk[2]};
    up[a] += 1;
    int vb = band_lookup(B, up[0], up[1], up[2]);
    float ma = mu[v], mb = vb >= 0 ? mu[vb] : ma;
    float t = ma / (ma - mb);
    float org[3] = {B.o0, B.o1, B.o2};
    float p[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) p[d] = org[d] + ((float)ijk[d] + 0.5f) * B.h;
    p[a] += t * B.h;
    int id = vid[q];
    verts[3 * id] = p[0];
    verts[3 * id + 1] = p[1];
    verts[3 * id + 2] = p[2];
  }
}

// ---- dual contouring (Sec. 3.8 "MC or DC") ---------------------------------
//
// Cells are the cubes of 8 band voxels (inside = mu < 0), as for marching
// cubes.  A crossed grid edge (a, b = a + e_axis) carries the point
// p = x_a + t e_axis, t = mu_a / (mu_a - mu_b), and the normal n = g / |g|,
// g = (1 - t) g_a + t g_b, where g_v is the voxel's central difference of mu
// over its band neighbours along each axis (one-sided with one neighbour, 0
// with none; an edge with g = 0 adds its point but no plane).  A cube with a
// crossed edge gets the vertex minimising sum_e (n_e . (x - p_e))^2 +
// eps |x - c|^2 (c = mean crossing point, eps = 0.01), clamped to the cube;
// every crossed edge whose four cubes exist gives a quad of their vertices,
// facing mu >= 0, split into two triangles.  Grid coordinates and FP64
// throughout; vertices are stored in metres as FP32.  Order: vertices by the
// compact index of the cube's lower corner, triangles by (edge's lower voxel,
// axis), two per quad.
constexpr double DC_EPS = 0.01;

__device__ __forceinline__ void voxel_ijk(const BandView& B, int v, int ijk[3]) {
  const int L = B.lin[v];
  ijk[0] = L % B.n;
  ijk[1] = (L / B.n) % B.n;
  ijk[2] = L / (B.n * B.n);
}

__global__ void k_dc_grad(BandView B, const float* __restrict__ mu, double* __restrict__ grad) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int c[3];
    voxel_ijk(B, v, c);
    const double m = mu[v];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int up[3] = {c[0], c[1], c[2]}, dn[3] = {c[0], c[1], c[2]};
      up[a] += 1;
      dn[a] -= 1;
      const int iu = band_lookup(B, up[0], up[1], up[2]), id = band_lookup(B, dn[0], dn[1], dn[2]);
      double g = 0.0;
      if (iu >= 0 && id >= 0) g = 0.5 * ((double)mu[iu] - (double)mu[id]);
      else if (iu >= 0) g = (double)mu[iu] - m;
      else if (id >= 0) g = m - (double)mu[id];
      grad[3 * (size_t)v + a] = g;
    }
  }
}

// compact indices of the 8 corners of the cube with lower corner v; false if one is off the band
__device__ __forceinline__ bool cube_corners(const BandView& B, int v, const int c[3], int ci[8]) {
  ci[0] = v;
  for (int k = 1; k < 8; ++k) {
    ci[k] = band_lookup(B, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + ((k >> 2) & 1));
    if (ci[k] < 0) return false;
  }
  return true;
}

__global__ void k_dc_cube(BandView B, const float* __restrict__ mu, const double* __restrict__ grad,
                          int32_t* __restrict__ vflag, double* __restrict__ vpos) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int c[3], ci[8];
    voxel_ijk(B, v, c);
    vflag[v] = 0;
    if (!cube_corners(B, v, c, ci)) continue;
    double A[6] = {0, 0, 0, 0, 0, 0};  // xx, xy, xz, yy, yz, zz
    double r[3] = {0, 0, 0}, cs[3] = {0, 0, 0};
    int cnt = 0;
    for (int k0 = 0; k0 < 8; ++k0)
      for (int a = 0; a < 3; ++a) {
        if ((k0 >> a) & 1) continue;
        const int ia = ci[k0], ib = ci[k0 | (1 << a)];
        const float ma = mu[ia], mb = mu[ib];
        if ((ma < 0.0f) == (mb < 0.0f)) continue;
        const double da = ma, db = mb;
        const double t = da / (da - db);
        double p[3] = {(double)(c[0] + (k0 & 1)), (double)(c[1] + ((k0 >> 1) & 1)), (double)(c[2] + ((k0 >> 2) & 1))};
        p[a] += t;
        double g[3], gn = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          g[d] = (1.0 - t) * grad[3 * (size_t)ia + d] + t * grad[3 * (size_t)ib + d];
          gn += g[d] * g[d];
        }
        gn = sqrt(gn);
        double n[3] = {0, 0, 0};
        if (gn > 0.0)
          for (int d = 0; d < 3; ++d) n[d] = g[d] / gn;
        const double np = n[0] * p[0] + n[1] * p[1] + n[2] * p[2];
        A[0] += n[0] * n[0]; A[1] += n[0] * n[1]; A[2] += n[0] * n[2];
        A[3] += n[1] * n[1]; A[4] += n[1] * n[2]; A[5] += n[2] * n[2];
        for (int d = 0; d < 3; ++d) {
          r[d] += n[d] * np;
          cs[d] += p[d];
        }
        ++cnt;
      }
    if (!cnt) continue;
    // (A + eps I) x = r + eps c by Cholesky
    double m[3];
    for (int d = 0; d < 3; ++d) m[d] = r[d] + DC_EPS * (cs[d] / cnt);
    const double a00 = A[0] + DC_EPS, a01 = A[1], a02 = A[2], a11 = A[3] + DC_EPS, a12 = A[4], a22 = A[5] + DC_EPS;
    const double l00 = sqrt(a00), l10 = a01 / l00, l20 = a02 / l00;
    const double l11 = sqrt(a11 - l10 * l10), l21 = (a12 - l20 * l10) / l11;
    const double l22 = sqrt(a22 - l20 * l20 - l21 * l21);
    const double y0 = m[0] / l00, y1 = (m[1] - l10 * y0) / l11, y2 = (m[2] - l20 * y0 - l21 * y1) / l22;
    double x[3];
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    for (int d = 0; d < 3; ++d) x[d] = fmin(fmax(x[d], (double)c[d]), (double)c[d] + 1.0);
    vflag[v] = 1;
    for (int d = 0; d < 3; ++d) vpos[3 * (size_t)v + d] = x[d];
  }
}

__global__ void k_dc_verts(BandView B, const int32_t* __restrict__ vflag, const int32_t* __restrict__ vid,
                           const double* __restrict__ vpos, float* __restrict__ verts) {
  const double org[3] = {B.o0, B.o1, B.o2};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    if (!vflag[v]) continue;
    const int id = vid[v];
    for (int d = 0; d < 3; ++d) verts[3 * (size_t)id + d] = (float)(org[d] + (vpos[3 * (size_t)v + d] + 0.5) * (double)B.h);
  }
}

// the quad of edge (v, v + e_a) if crossed with its four cubes present: their vertex cubes in quad order
__device__ __forceinline__ bool dc_quad(const BandView& B, const float* __restrict__ mu, const int32_t* __restrict__ vflag,
                                        int v, const int c[3], int a, int q[4], bool* in_v) {
  int up[3] = {c[0], c[1], c[2]};
  up[a] += 1;
  const int u = band_lookup(B, up[0], up[1], up[2]);
  if (u < 0) return false;
  const bool iv = mu[v] < 0.0f, iu = mu[u] < 0.0f;
  if (iv == iu) return false;
  const int au = (a + 1) % 3, av = (a + 2) % 3;
  const int du[4] = {-1, 0, 0, -1}, dv[4] = {-1, -1, 0, 0};
  for (int k = 0; k < 4; ++k) {
    int o[3] = {c[0], c[1], c[2]};
    o[au] += du[k];
    o[av] += dv[k];
    const int cv = band_lookup(B, o[0], o[1], o[2]);
    if (cv < 0 || !vflag[cv]) return false;
    q[k] = cv;
  }
  *in_v = iv;
  return true;
}

__global__ void k_dc_count(BandView B, const float* __restrict__ mu, const int32_t* __restrict__ vflag,
                           int32_t* __restrict__ tcount) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int c[3], q[4];
    bool in_v;
    voxel_ijk(B, v, c);
    int n = 0;
    for (int a = 0; a < 3; ++a) n += dc_quad(B, mu, vflag, v, c, a, q, &in_v) ? 2 : 0;
    tcount[v] = n;
  }
}

__global__ void k_dc_emit(BandView B, const float* __restrict__ mu, const int32_t* __restrict__ vflag,
                          const int32_t* __restrict__ vid, const int32_t* __restrict__ toff, int32_t* __restrict__ tris) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < B.N; v += gridDim.x * blockDim.x) {
    int c[3], q[4];
    bool in_v;
    voxel_ijk(B, v, c);
    int o = toff[v];
    for (int a = 0; a < 3; ++a) {
      if (!dc_quad(B, mu, vflag, v, c, a, q, &in_v)) continue;
      int w[4];
      for (int k = 0; k < 4; ++k) w[k] = vid[q[in_v ? k : 3 - k]];
      tris[3 * (size_t)o + 0] = w[0]; tris[3 * (size_t)o + 1] = w[1]; tris[3 * (size_t)o + 2] = w[2];
      tris[3 * (size_t)o + 3] = w[0]; tris[3 * (size_t)o + 4] = w[2]; tris[3 * (size_t)o + 5] = w[3];
      o += 2;
    }
  }
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

bf_status mc_impl(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt) {
  cudaStream_t s = ctx->stream;
  if (!ctx->mc_table) {
    CaseTable T;
    build_case_table(T);
    BF_CK(cudaMalloc(&ctx->mc_table, sizeof(T.tri)));
    BF_CK(cudaMalloc(&ctx->mc_ntri, sizeof(T.n)));
    BF_CK(cudaMemcpy(ctx->mc_table, T.tri, sizeof(T.tri), cudaMemcpyHostToDevice));
    BF_CK(cudaMemcpy(ctx->mc_ntri, T.n, sizeof(T.n), cudaMemcpyHostToDevice));
  }
  ctx->mesh_nv = ctx->mesh_nt = 0;
  *nv = *nt = 0;
  const int64_t N = b->N;
  if (N == 0) return BF_OK;
  bf_status st;
  int32_t* tcount = (int32_t*)ws_get(ctx, WS_TMP0, (size_t)(N + 1) * 4, &st);
  if (st) return st;
  int32_t* vflag = (int32_t*)ws_get(ctx, WS_TMP1, (size_t)(3 * N + 1) * 4, &st);
  if (st) return st;
  int32_t* vid = (int32_t*)ws_get(ctx, WS_TMP2, (size_t)(3 * N + 1) * 4, &st);
  if (st) return st;
  BandView bv = band_view(b);
  BF_CK(cudaMemsetAsync(vflag, 0, (size_t)3 * N * 4, s));
  k_mc_classify<<<gsz(N), 256, 0, s>>>(bv, mu, ctx->mc_table, ctx->mc_ntri, tcount, vflag); count_launch();
  BF_CK(cudaGetLastError());
  BF_TRY(scan_i32(ctx, tcount, tcount, N, tcount + N));
  BF_TRY(scan_i32(ctx, vflag, vid, 3 * N, vid + 3 * N));
  BF_CK(cudaMemcpyAsync(ctx->h_pinned, tcount + N, 4, cudaMemcpyDeviceToHost, s));
  BF_CK(cudaMemcpyAsync(ctx->h_pinned + 1, vid + 3 * N, 4, cudaMemcpyDeviceToHost, s));
  BF_CK(cudaStreamSynchronize(s));
  int64_t NT = ctx->h_pinned[0], NV = ctx->h_pinned[1];
  if ((size_t)NV * 12 > ctx->mesh_vcap) {
    if (ctx->mesh_v) cudaFree(ctx->mesh_v);
    ctx->mesh_vcap = (size_t)NV * 12 + 1024;
    BF_CK(cudaMalloc(&ctx->mesh_v, ctx->mesh_vcap));
  }
  if ((size_t)NT * 12 > ctx->mesh_tcap) {
    if (ctx->mesh_t) cudaFree(ctx->mesh_t);
    ctx->mesh_tcap = (size_t)NT * 12 + 1024;
    BF_CK(cudaMalloc(&ctx->mesh_t, ctx->mesh_tcap));
  }
  k_mc_emit<<<gsz(N), 256, 0, s>>>(bv, mu, ctx->mc_table, ctx->mc_ntri, tcount, vid, ctx->mesh_t); count_launch();
  k_mc_verts<<<gsz(3 * N), 256, 0, s>>>(bv, mu, vflag, vid, ctx->mesh_v); count_launch();
  BF_CK(cudaGetLastError());
  ctx->mesh_nv = NV;
  ctx->mesh_nt = NT;
  *nv = NV;
  *nt = NT;
  return BF_OK;
}

bf_status dc_impl(bf_ctx* ctx, const bf_band* b, const float* mu, int64_t* nv, int64_t* nt) {
  cudaStream_t s = ctx->stream;
  ctx->mesh_nv = ctx->mesh_nt = 0;
  *nv = *nt = 0;
  const int64_t N = b->N;
  if (N == 0) return BF_OK;
  bf_status st;
  int32_t* tcount = (int32_t*)ws_get(ctx, WS_TMP0, (size_t)(N + 1) * 4, &st);
  if (st) return st;
  int32_t* vflag = (int32_t*)ws_get(ctx, WS_TMP1, (size_t)(N + 1) * 4, &st);
  if (st) return st;
  int32_t* vid = (int32_t*)ws_get(ctx, WS_TMP2, (size_t)(N + 1) * 4, &st);
  if (st) return st;
  double* grad = (double*)ws_get(ctx, WS_TMP3, (size_t)N * 3 * sizeof(double), &st);
  if (st) return st;
  double* vpos = (double*)ws_get(ctx, WS_TMP4, (size_t)N * 3 * sizeof(double), &st);
  if (st) return st;
  const BandView bv = band_view(b);
  k_dc_grad<<<gsz(N), 256, 0, s>>>(bv, mu, grad); count_launch();
  k_dc_cube<<<gsz(N), 256, 0, s>>>(bv, mu, grad, vflag, vpos); count_launch();
  BF_CK(cudaGetLastError());
  BF_TRY(scan_i32(ctx, vflag, vid, N, vid + N));
  k_dc_count<<<gsz(N), 256, 0, s>>>(bv, mu, vflag, tcount); count_launch();
  BF_CK(cudaGetLastError());
  BF_TRY(scan_i32(ctx, tcount, tcount, N, tcount + N));
  BF_CK(cudaMemcpyAsync(ctx->h_pinned, tcount + N, 4, cudaMemcpyDeviceToHost, s));
  BF_CK(cudaMemcpyAsync(ctx->h_pinned + 1, vid + N, 4, cudaMemcpyDeviceToHost, s));
  BF_CK(cudaStreamSynchronize(s));
  const int64_t NT = ctx->h_pinned[0], NV = ctx->h_pinned[1];
  if ((size_t)NV * 12 > ctx->mesh_vcap) {
    if (ctx->mesh_v) cudaFree(ctx->mesh_v);
    ctx->mesh_vcap = (size_t)NV * 12 + 1024;
    BF_CK(cudaMalloc(&ctx->mesh_v, ctx->mesh_vcap));
  }
  if ((size_t)NT * 12 > ctx->mesh_tcap) {
    if (ctx->mesh_t) cudaFree(ctx->mesh_t);
    ctx->mesh_tcap = (size_t)NT * 12 + 1024;
    BF_CK(cudaMalloc(&ctx->mesh_t, ctx->mesh_tcap));
  }
  k_dc_verts<<<gsz(N), 256, 0, s>>>(bv, vflag, vid, vpos, ctx->mesh_v); count_launch();
  k_dc_emit<<<gsz(N), 256, 0, s>>>(bv, mu, vflag, vid, tcount, ctx->mesh_t); count_launch();
  BF_CK(cudaGetLastError());
  ctx->mesh_nv = NV;
  ctx->mesh_nt = NT;
  *nv = NV;
  *nt = NT;
  return BF_OK;
}
