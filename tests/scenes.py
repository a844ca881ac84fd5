"""Small analytic test scenes with closed-form answers (inputs only)."""
import numpy as np

import synth


def hollow_sphere(n=32, h=0.02, R=0.22, W=64, f=28.0, band_vox=3.0, trunc_vox=5.0):
    """Six cube-map cameras at the centre of a sphere of radius R: every pixel
    ray meets the surface at normal incidence (frusta overlap slightly)."""
    sc = synth.sphere_scene(R)
    dirs = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    P = np.stack([synth.look_at((0, 0, 0), target=d) for d in dirs])
    intr = (f, f, W / 2, W / 2, W, W)
    depth = synth.render(sc, P, W, W, f, f, W / 2, W / 2)
    org = (-n * h / 2,) * 3
    return dict(n=n, h=h, R=R, org=org, poses=P.astype(np.float32), intr=intr, depth=depth,
                band_vox=band_vox, trunc_vox=trunc_vox)


def frontal_plane(n=32, h=0.015, z0_off=0.37, band_vox=3.0, trunc_vox=5.0, W=48, f=120.0, dist=1.0):
    """Cameras looking along -z at the plane z = Z0 from a 3x3 lattice of
    positions; Z0 sits 0.37 h above a voxel centre so no voxel is at a tie."""
    org = (-n * h / 2,) * 3
    Z0 = org[2] + (n // 2 + 0.5 + z0_off) * h
    sc = synth.plane_scene((0, 0, 1), Z0)
    P = []
    span = n * h / 3
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            c = (a * span, b * span, Z0 + dist)
            P.append(synth.look_at(c, target=(a * span, b * span, Z0)))
    P = np.stack(P)
    intr = (f, f, W / 2, W / 2, W, W)
    depth = synth.render(sc, P, W, W, f, f, W / 2, W / 2)
    return dict(n=n, h=h, Z0=Z0, org=org, poses=P.astype(np.float32), intr=intr, depth=depth,
                band_vox=band_vox, trunc_vox=trunc_vox)


def exterior_sphere(n=64, h=0.015, R=0.3, views=400, W=96, f=700.0, dist=1.0, band_vox=4.0, trunc_vox=6.0):
    """A sphere of radius R at the origin seen, without noise, by `views`
    cameras on a Fibonacci sphere of radius `dist` looking at its centre, with
    a narrow field of view: a ray at angle phi off the optical axis meets the
    sphere at incidence theta with sin(theta) = dist sin(phi) / R (law of
    sines), so every ray meets the surface within theta_max of its normal."""
    sc = synth.sphere_scene(R)
    P = np.stack([synth.look_at(dist * v) for v in synth.fibonacci_sphere(views)])
    intr = (f, f, W / 2, W / 2, W, W)
    depth = synth.render(sc, P, W, W, f, f, W / 2, W / 2)
    phi = np.arctan(np.hypot(W / 2, W / 2) / f)
    theta_max = float(np.arcsin(dist * np.sin(phi) / R))
    org = (-n * h / 2,) * 3
    return dict(n=n, h=h, R=R, org=org, poses=P.astype(np.float32), intr=intr, depth=depth,
                band_vox=band_vox, trunc_vox=trunc_vox, theta_max=theta_max)
