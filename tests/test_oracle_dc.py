"""Pins of the dual-contouring oracle (oracle/dc.py; Sec. 3.8 surface
extraction by "MC or DC"): a linear field puts every vertex on its zero
plane exactly (the crossing points and central-difference normals of a
linear function are exact, so the QEF's minimiser is the mass point, on the
plane); the exact SDF of a sphere gives a closed, consistently oriented
genus-0 mesh whose vertices lie on the sphere; the quads are the crossed edges
marching cubes puts its vertices on."""
import numpy as np
import pytest

import oracle
from oracle import dc

from .scenes import frontal_plane, hollow_sphere


def _edges(F):
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    return np.unique(e, axis=0, return_counts=True)


def test_linear_field_vertices_lie_on_its_zero_plane():
    s = frontal_plane(n=24)
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    x = b.centres()
    nrm = np.array([0.3, -0.2, 0.93])
    nrm /= np.linalg.norm(nrm)
    d0 = float(nrm @ np.array([0.0, 0.0, s["Z0"]])) + 0.123 * s["h"]
    mu = ((x @ nrm) - d0) / b.h
    V, F, vc = dc.dual_contour(b, mu.astype(np.float32))
    assert len(V) > 100 and len(F) > 100
    # mu was rounded to float32: the plane holds to that precision
    dist = (V @ nrm - d0) / b.h
    assert np.abs(dist).max() <= 1e-5
    # triangles face the side where mu >= 0 (the normal's side)
    tn = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert np.all(tn @ nrm > 0)


@pytest.fixture(scope="module")
def sphere_field():
    s = hollow_sphere()   # cameras at the centre see every surface point: a band that encloses the sphere
    b = oracle.build_band(s["depth"], s["poses"], s["intr"], s["n"], s["h"], s["org"], s["band_vox"], s["trunc_vox"])
    r = s["R"]
    mu = (np.linalg.norm(b.centres(), axis=1) - r) / b.h
    return b, mu.astype(np.float32), r


def test_sphere_sdf_gives_a_closed_oriented_mesh_on_the_sphere(sphere_field):
    b, mu, r = sphere_field
    V, F, vc = dc.dual_contour(b, mu)
    rad = np.linalg.norm(V, axis=1)
    assert np.abs(rad - r).max() <= 0.05 * b.h
    assert np.sqrt(np.mean((rad - r) ** 2)) <= 0.02 * b.h
    _, cnt = _edges(F)
    assert np.all(cnt == 2)
    assert len(V) - len(cnt) + len(F) == 2
    cen = V[F].mean(1)
    tn = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    assert np.all(np.sum(tn * cen, 1) > 0)
    # every vertex lies in its cube, which spans [centre(v), centre(v) + h] per axis
    assert np.all(V >= b.centres()[vc] - 1e-12) and np.all(V <= b.centres()[vc] + b.h + 1e-12)


def test_quads_are_the_edges_marching_cubes_crosses(sphere_field):
    b, mu, r = sphere_field
    V, F, vc = dc.dual_contour(b, mu)
    Vm, Fm = oracle.marching_cubes(b, mu)
    # marching cubes puts one vertex on every crossed edge of an existing cube; on this closed surface every
    # such edge has its four cubes, and dual contouring turns each into one quad (two triangles)
    assert len(F) == 2 * len(Vm)
