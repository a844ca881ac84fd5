"""Seeded synthetic workloads: analytic scenes, camera paths and noisy depth.

This module is the one input source shared by the CUDA path and the CPU
oracle.  It renders depth maps; it contains none of the fusion method's
arithmetic (no TSDF, band, observation model or solver).

Workloads (grid, scene, views, noise) restate the five workload descriptions
the method is measured on:

* ``sphere64``  -- sphere r=0.3 m at the origin, 64^3 grid at 15 mm, band
  +-4 voxels, 20 views 160x120 on a ring of radius 1 m (fx=fy=140),
  sigma(z) = 0.002 + 0.004 z^2, 16 probes, FP64 PCG to 1e-8.
* ``union256``  -- union of a box (half-size 0.2 m), a sphere (r=0.2 m) and
  a torus (R=0.25 m, r=0.05 m) in a 256^3 grid at 4 mm, band +-5 voxels,
  100 views 640x480 on a Fibonacci hemisphere of radius 1.2 m (fx=fy=560),
  same noise plus 1 % dropout, FP32 PCG to 1e-6, 64 probes.
* ``sphere64_k256`` -- the sphere64 scene with 256 probes (block PCG).
* ``blob512``   -- star-shaped blob r(w) = 0.25 (1 + 0.15 g(w)/max|g|), g a
  random real spherical-harmonic series of degrees 1..6 (seed 1), 512^3 grid
  at 2 mm, 200 frames 512x384 (fx=fy=448) on a two-turn spiral of radius
  0.8 m from 60 deg to -20 deg elevation, sigma(z) = 0.001 + 0.003 z^2,
  2 mm pose jitter on the rendering camera, 128 probes.

Scene placements, camera paths and the intrinsics not given by the workload
descriptions are fixed here; the record of each choice is in the design notes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lib = None

SC_SPHERE, SC_UNION, SC_BLOB, SC_PLANE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the generator (gcc, OpenMP) in-tree; returns the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_render.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
        lib.synth_scene_sdf_many.argtypes = [ctypes.c_int, dp, ctypes.c_int64, dp, dp]
        lib.synth_blob_stats.argtypes = [dp, ctypes.c_int, dp, dp]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------- cameras

def look_at(center, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    """World<-camera pose [3,4] (OpenCV axes: x right, y down, z forward)."""
    c = np.asarray(center, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(np.dot(f, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    P = np.zeros((3, 4))
    P[:, 0], P[:, 1], P[:, 2], P[:, 3] = x, y, f, c
    return P


def fibonacci_sphere(n: int, zmin: float = -1.0) -> np.ndarray:
    """n unit vectors on the spherical cap z >= zmin, Fibonacci spiral."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (i + 0.5) / n * (1.0 - zmin)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ph = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)


def ring_poses(n: int, radius: float, z: float = 0.0, phase: float = 0.0) -> np.ndarray:
    a = phase + 2 * math.pi * np.arange(n) / n
    return np.stack([look_at((radius * math.cos(t), radius * math.sin(t), z)) for t in a])


def hemisphere_poses(n: int, radius: float, zmin_frac: float = 0.1) -> np.ndarray:
    return np.stack([look_at(radius * v) for v in fibonacci_sphere(n, zmin_frac)])


def spiral_poses(n: int, radius: float, turns: float = 2.0, el0: float = 60.0, el1: float = -20.0):
    f = np.arange(n, dtype=np.float64)
    az = 2 * math.pi * turns * f / n
    el = np.radians(el0 + (el1 - el0) * f / max(n - 1, 1))
    c = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1) * radius
    return np.stack([look_at(p) for p in c])


# ------------------------------------------------------------------ scenes

@dataclass
class Scene:
    type: int
    params: np.ndarray

    def sdf(self, pts: np.ndarray) -> np.ndarray:
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        out = np.empty(len(pts), np.float64)
        _load().synth_scene_sdf_many(self.type, _dp(self.params), len(pts), _dp(pts), _dp(out))
        return out


def sphere_scene(r=0.3, c=(0.0, 0.0, 0.0)) -> Scene:
    return Scene(SC_SPHERE, np.array([*c, r], np.float64))


def union_scene() -> Scene:
    p = [-0.2, 0.0, 0.0, 0.2, 0.2, 0.2,      # box centre, half-size
         0.22, 0.0, 0.05, 0.2,               # sphere centre, radius
         0.05, 0.0, -0.25, 0.25, 0.05]       # torus centre, R, r (axis z)
    return Scene(SC_UNION, np.array(p, np.float64))


def blob_scene(seed: int = 1, r0: float = 0.25, amp: float = 0.15) -> Scene:
    coef = np.random.Generator(np.random.PCG64(seed)).standard_normal(48)
    gmax, gradmax = ctypes.c_double(), ctypes.c_double()
    _load().synth_blob_stats(_dp(coef), 100000, ctypes.byref(gmax), ctypes.byref(gradmax))
    rmin = r0 * (1 - amp)
    lip = math.sqrt(1.0 + (r0 * amp * gradmax.value / gmax.value / rmin) ** 2) * 1.25
    p = np.concatenate([[0.0, 0.0, 0.0, r0, amp, gmax.value, lip, 0.0], coef])
    return Scene(SC_BLOB, p.astype(np.float64))


def plane_scene(normal, c) -> Scene:
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    return Scene(SC_PLANE, np.array([*n, c], np.float64))


def render(scene: Scene, poses: np.ndarray, W: int, H: int, fx: float, fy: float, cx: float, cy: float,
           sig_a: float = 0.0, sig_b: float = 0.0, dropout: float = 0.0, seed: int = 0,
           threads: int = 0) -> np.ndarray:
    poses = np.ascontiguousarray(poses, np.float64)
    T = poses.shape[0]
    depth = np.empty((T, H, W), np.float32)
    _load().synth_render(scene.type, _dp(scene.params), T, H, W, _dp(poses), fx, fy, cx, cy,
                         sig_a, sig_b, dropout, seed, threads,
                         depth.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return depth


# --------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    n: int
    h: float
    origin: tuple
    depth: np.ndarray            # float32 [T,H,W], 0 = invalid
    poses: np.ndarray            # float32 [T,3,4] world<-camera used for fusion
    intr: tuple                  # (fx, fy, cx, cy, W, H)
    band_vox: float
    trunc_vox: float
    lam: float = 1.0
    lam_b: float = 1.0
    sig_a: float = 0.002
    sig_b: float = 0.004
    sig_pose: float = 0.0
    sig_model: float = 0.0
    tol: float = 1e-6
    fp64: bool = False
    K: int = 16
    seed: int = 0
    scene: Scene = None
    cand_poses: np.ndarray = None  # float32 [V,3,4]
    cand_intr: tuple = None
    extra: dict = field(default_factory=dict)

    @property
    def T(self):
        return self.depth.shape[0]

    def params(self) -> dict:
        return dict(band_vox=self.band_vox, trunc_vox=self.trunc_vox, lam=self.lam, lam_b=self.lam_b,
                    sig_a=self.sig_a, sig_b=self.sig_b, sig_pose=self.sig_pose, sig_model=self.sig_model)


def _grid(n: int, h: float):
    o = -0.5 * n * h
    return (o, o, o)


def make_workload(name: str, *, n: int | None = None, frames: int | None = None,
                  image_scale: float = 1.0, noise: bool = True, seed: int = 0,
                  band_vox: float | None = None, threads: int = 0, n_cand: int = 64,
                  variant: int | None = None) -> Workload:
    """Build one of the named workloads.  ``n``, ``frames`` and ``image_scale``
    shrink it for fast tests (the voxel size scales so the scene still fits).

    ``variant`` (sphere workloads only) draws one instance of the family used
    to train the learned warm start: sphere radius U(0.22, 0.34) m, centre
    offset U(-0.03, 0.03) m per axis and ring phase U(0, 2 pi / frames) from
    a generator seeded by the variant number, which is also the noise seed."""
    if name in ("sphere64", "sphere64_k256"):
        n0, h0, b, tc = 64, 0.015, 4.0, 6.0
        T = frames or 20
        if variant is None:
            scene = sphere_scene(0.3)
            P = ring_poses(T, 1.0)
        else:
            g = np.random.Generator(np.random.PCG64(10007 + int(variant)))
            r = float(g.uniform(0.22, 0.34))
            c = tuple(float(x) for x in g.uniform(-0.03, 0.03, 3))
            scene = sphere_scene(r, c)
            P = ring_poses(T, 1.0, phase=float(g.uniform(0.0, 2 * math.pi / T)))
            seed = int(variant)
        W, H, f = 160, 120, 140.0
        sa, sb, drop, sp = 0.002, 0.004, 0.0, 0.0
        cand_r = 1.0
        K, tol, fp64 = (256 if name.endswith("k256") else 16), (1e-6 if name.endswith("k256") else 1e-8), not name.endswith("k256")
    elif name == "union256":
        n0, h0, b, tc = 256, 0.004, 5.0, 7.0
        scene = union_scene()
        T = frames or 100
        P = hemisphere_poses(T, 1.2)
        W, H, f = 640, 480, 560.0
        sa, sb, drop, sp = 0.002, 0.004, 0.01, 0.0
        cand_r = 1.2
        K, tol, fp64 = 64, 1e-6, False
    elif name == "blob512":
        n0, h0 = 512, 0.002
        b = band_vox if band_vox is not None else 24.0
        tc = b + 2.0
        scene = blob_scene(1)
        T = frames or 200
        P = spiral_poses(T, 0.8)
        W, H, f = 512, 384, 448.0
        sa, sb, drop, sp = 0.001, 0.003, 0.0, 0.002
        cand_r = 0.8
        K, tol, fp64 = 128, 1e-6, False
    else:
        raise ValueError(f"unknown workload {name!r}")
    if variant is not None and not name.startswith("sphere"):
        raise ValueError("variant applies to the sphere workloads only")
    if band_vox is not None and name != "blob512":
        b, tc = float(band_vox), float(band_vox) + 2.0
    nn = n or n0
    h = h0 * n0 / nn
    W, H = int(round(W * image_scale)), int(round(H * image_scale))
    f = f * image_scale
    cx, cy = W / 2.0, H / 2.0
    Prender = P.copy()
    if sp > 0 and noise:
        jit = np.random.Generator(np.random.PCG64(seed + 7)).normal(0.0, sp, (T, 3))
        Prender[:, :, 3] += jit
    depth = render(scene, Prender, W, H, f, f, cx, cy, sa if noise else 0.0, sb if noise else 0.0,
                   drop if noise else 0.0, seed, threads)
    cand = np.stack([look_at(cand_r * v) for v in fibonacci_sphere(n_cand)]).astype(np.float32)
    Wc, Hc = max(W // 4, 1), max(H // 4, 1)
    return Workload(name=name, n=nn, h=h, origin=_grid(nn, h), depth=depth, poses=P.astype(np.float32),
                    intr=(f, f, cx, cy, W, H), band_vox=b, trunc_vox=tc, sig_a=sa, sig_b=sb,
                    sig_pose=sp, tol=tol, fp64=fp64, K=K, seed=seed, scene=scene,
                    cand_poses=cand, cand_intr=(f / 4, f / 4, Wc / 2.0, Hc / 2.0, Wc, Hc))
