"""Dual contouring of the posterior mean (Sec. 3.8: the surface is extracted
from mu by "MC or DC") -- TEST INFRASTRUCTURE: the plain FP64 reference of
the CUDA path's bf_extract_surface_dc.  Only tests may use this module.

Readings (the paper names dual contouring without details):
  * cells are the cubes of 8 band voxel centres (as for marching cubes);
    inside = mu < 0;
  * a grid edge between two band voxels a (lower) and b = a + e_axis is
    crossed when exactly one end is inside; its Hermite data are the
    crossing point p = x_a + t e_axis, t = mu_a / (mu_a - mu_b) (grid
    units), and the normal n = g / |g| with g = (1 - t) g_a + t g_b, where
    g_v is the voxel's gradient of mu by central differences over its two
    band neighbours along each axis (one-sided with one neighbour, 0 with
    none); an edge with g = 0 contributes its point but no plane;
  * each cube with a crossed edge among its 12 gets one vertex: the
    minimiser of sum_e (n_e . (x - p_e))^2 + eps |x - c|^2, c the mean of
    its crossing points, eps = 0.01 (a Tikhonov pull towards the mass point
    that keeps the 3 x 3 system definite where the normals do not span
    space), i.e. (A + eps I) x = sum_e n_e (n_e . p_e) + eps c with
    A = sum_e n_e n_e^T, then clamped to the cube;
  * each crossed edge whose 4 incident cubes all exist gives a quad of
    their vertices, in the order of the cube offsets (-1,-1), (0,-1), (0,0),
    (-1,0) along the two other axes (u, v) taken cyclically after the edge's
    axis, reversed when the edge's lower end is outside (so the triangles
    face towards mu >= 0); the quad is split into (q0, q1, q2), (q0, q2, q3);
  * vertices are ordered by the compact index of the cube's lower corner,
    triangles by (compact index of the edge's lower voxel, axis), two per
    quad; vertex positions are in metres: origin + (x + 1/2) h.
"""
from __future__ import annotations

import numpy as np

EPS = 0.01


def _index_grid(band):
    """Dense map (i, j, k) -> compact index, -1 off the band, with a one-voxel border of -1."""
    n = band.n
    g = np.full((n + 2, n + 2, n + 2), -1, np.int64)
    ijk = band.ijk()
    g[ijk[:, 0] + 1, ijk[:, 1] + 1, ijk[:, 2] + 1] = np.arange(band.N)
    return g, ijk


def gradients(band, mu):
    """g [N, 3]: central differences of mu over band neighbours (one-sided with one, 0 with none)."""
    mu = np.asarray(mu, np.float64)
    g, ijk = _index_grid(band)
    out = np.zeros((band.N, 3))
    for a in range(3):
        e = np.zeros(3, np.int64)
        e[a] = 1
        up = g[ijk[:, 0] + 1 + e[0], ijk[:, 1] + 1 + e[1], ijk[:, 2] + 1 + e[2]]
        dn = g[ijk[:, 0] + 1 - e[0], ijk[:, 1] + 1 - e[1], ijk[:, 2] + 1 - e[2]]
        hu, hd = up >= 0, dn >= 0
        mu_u = np.where(hu, mu[np.maximum(up, 0)], 0.0)
        mu_d = np.where(hd, mu[np.maximum(dn, 0)], 0.0)
        out[:, a] = np.where(hu & hd, 0.5 * (mu_u - mu_d),
                             np.where(hu, mu_u - mu, np.where(hd, mu - mu_d, 0.0)))
    return out


def dual_contour(band, mu):
    """(verts [V, 3] metres, tris [F, 3] int32, cube_of_vertex [V] compact index of each vertex's cube)."""
    mu = np.asarray(mu, np.float32).astype(np.float64)
    g, ijk = _index_grid(band)
    grad = gradients(band, mu)
    N = band.N
    inside = mu < 0

    def at(offset):
        o = np.asarray(offset)
        return g[ijk[:, 0] + 1 + o[0], ijk[:, 1] + 1 + o[1], ijk[:, 2] + 1 + o[2]]

    # cubes: all 8 corners in the band
    corners = np.stack([at((c & 1, (c >> 1) & 1, (c >> 2) & 1)) for c in range(8)], 1)   # [N, 8]
    cube = np.all(corners >= 0, axis=1)
    # the 12 edges of a cube as corner pairs (lower, upper) with their axis
    edges = []
    for c in range(8):
        for a in range(3):
            if not (c >> a) & 1:
                edges.append((c, c | (1 << a), a))
    verts = []
    vcube = []
    vid = np.full(N, -1, np.int64)
    for v in np.nonzero(cube)[0]:
        pts, nrm = [], []
        for c0, c1, a in edges:
            ia, ib = corners[v, c0], corners[v, c1]
            if inside[ia] == inside[ib]:
                continue
            t = mu[ia] / (mu[ia] - mu[ib])
            p = ijk[ia].astype(np.float64)
            p[a] += t
            gg = (1.0 - t) * grad[ia] + t * grad[ib]
            gn = np.linalg.norm(gg)
            pts.append(p)
            nrm.append(gg / gn if gn > 0 else np.zeros(3))
        if not pts:
            continue
        P, Nn = np.array(pts), np.array(nrm)
        c = P.mean(0)
        A = Nn.T @ Nn + EPS * np.eye(3)
        r = Nn.T @ np.sum(Nn * P, 1) + EPS * c
        x = np.linalg.solve(A, r)
        lo = ijk[v].astype(np.float64)
        x = np.minimum(np.maximum(x, lo), lo + 1.0)
        vid[v] = len(verts)
        verts.append(np.asarray(band.origin, np.float64) + (x + 0.5) * band.h)
        vcube.append(v)
    tris = []
    upper = [at(tuple(int(a == d) for d in range(3))) for a in range(3)]   # the band neighbour at +e_axis
    for v in range(N):
        for a in range(3):
            u = upper[a][v]
            if u < 0 or inside[v] == inside[u]:
                continue
            au, av = (a + 1) % 3, (a + 2) % 3
            quad = []
            for du, dv in ((-1, -1), (0, -1), (0, 0), (-1, 0)):
                o = [0, 0, 0]
                o[au], o[av] = du, dv
                cv = g[ijk[v, 0] + 1 + o[0], ijk[v, 1] + 1 + o[1], ijk[v, 2] + 1 + o[2]]
                quad.append(vid[cv] if cv >= 0 and cube[cv] else -1)
            if min(quad) < 0:
                continue
            if not inside[v]:
                quad = quad[::-1]
            tris.append((quad[0], quad[1], quad[2]))
            tris.append((quad[0], quad[2], quad[3]))
    V = np.array(verts, np.float64).reshape(-1, 3)
    F = np.array(tris, np.int32).reshape(-1, 3)
    return V, F, np.array(vcube, np.int64)
