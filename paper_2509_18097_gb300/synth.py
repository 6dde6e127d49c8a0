"""Seeded synthetic inputs shaped like the workloads of Preconditioned Deformation Grids.

This module only builds geometry: template meshes, point clouds sampled on analytic
surfaces and analytic deformations of them.  It holds none of the method's arithmetic
(no grid evaluation, nearest neighbours, losses, preconditioning or optimiser), so both
the CUDA path and the FP64 oracle can consume its arrays without sharing method code.

The paper's datasets (DFAUST, DT4D, AMA; Sec. 4) are not available here; these
generators stand in for them with the sizes the paper works at (2 500 - 20 000 points
per frame, Table 3; 17 - 80 frames, Sec. 4 and Table 2; noise as a fraction of the
bounding-box diagonal, Table 5).  Every array is float32 (points) or int32 (indices)
and every draw is from numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

F32 = np.float32

# --------------------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------------------


def _icosahedron():
    """The 12 vertices and 20 faces of a regular icosahedron on the unit sphere."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.asarray(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # faces = the triangles of the convex hull (every face of the icosahedron)
    from scipy.spatial import ConvexHull

    faces = ConvexHull(v).simplices.astype(np.int64)
    return v, faces


def edges_from_faces(faces: np.ndarray) -> np.ndarray:
    """Unique undirected edges (i < j), sorted lexicographically, as int32 [E, 2]."""
    f = np.asarray(faces, dtype=np.int64)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int32)


def icosphere(subdiv: int, radius: float = 1.0):
    """Icosphere by repeated midpoint subdivision with re-projection to the sphere.

    subdiv=3 gives 642 vertices, 1280 faces and 1920 edges.
    Returns (verts float32 [V,3], faces int32 [F,3], edges int32 [E,2]).
    """
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                verts.append(tuple(p))
                idx = len(verts) - 1
                cache[key] = idx
            return idx

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.asarray(nf, dtype=np.int64)
    verts = np.asarray(verts, dtype=np.float64) * radius
    return verts.astype(F32), f.astype(np.int32), edges_from_faces(f)


def geodesic_sphere(freq: int, axes=(1.0, 1.0, 1.0)):
    """Class-I geodesic sphere of frequency `freq`, scaled per axis to an ellipsoid.

    Each icosahedron face is split into freq^2 triangles on its barycentric lattice and
    the lattice points are projected to the unit sphere.  V = 10 freq^2 + 2,
    E = 30 freq^2, F = 20 freq^2 (freq=71: 50 412 / 151 230 / 100 820).
    """
    v0, f0 = _icosahedron()
    index: dict[tuple, int] = {}
    pos: list[np.ndarray] = []
    faces: list[tuple[int, int, int]] = []
    n = freq
    for a, b, c in f0:
        local = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                k = n - i - j
                # canonical key: (corner id, weight) pairs with non-zero weight, sorted
                key = tuple(sorted((cid, w) for cid, w in ((a, k), (b, i), (c, j)) if w))
                idx = index.get(key)
                if idx is None:
                    p = (k * v0[a] + i * v0[b] + j * v0[c]) / n
                    pos.append(p / np.linalg.norm(p))
                    idx = len(pos) - 1
                    index[key] = idx
                local[(i, j)] = idx
        for i in range(n):
            for j in range(n - i):
                faces.append((local[(i, j)], local[(i + 1, j)], local[(i, j + 1)]))
                if i + j < n - 1:
                    faces.append((local[(i + 1, j)], local[(i + 1, j + 1)], local[(i, j + 1)]))
    verts = np.asarray(pos) * np.asarray(axes, dtype=np.float64)
    faces = np.asarray(faces, dtype=np.int64)
    return verts.astype(F32), faces.astype(np.int32), edges_from_faces(faces)


def torus_mesh(nu: int, nv: int, R: float = 1.0, r: float = 0.3):
    """Torus in the xy-plane on an nu x nv parameter grid (two triangles per quad).

    nu=200, nv=100 gives V=20 000, F=40 000, E=60 000.
    """
    u = np.arange(nu) * (2 * np.pi / nu)
    v = np.arange(nv) * (2 * np.pi / nv)
    U, Vv = np.meshgrid(u, v, indexing="ij")
    verts = np.stack(
        [(R + r * np.cos(Vv)) * np.cos(U), (R + r * np.cos(Vv)) * np.sin(U), r * np.sin(Vv)], -1
    ).reshape(-1, 3)
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = ii * nv + jj
    b = ((ii + 1) % nu) * nv + jj
    c = ((ii + 1) % nu) * nv + (jj + 1) % nv
    d = ii * nv + (jj + 1) % nv
    faces = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    return verts.astype(F32), faces.astype(np.int32), edges_from_faces(faces)


# --------------------------------------------------------------------------------------
# point clouds
# --------------------------------------------------------------------------------------


def sphere_points(rng: np.random.Generator, n: int) -> np.ndarray:
    """n points uniform on the unit sphere (normalised Gaussians), float64."""
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def ellipsoid_points(rng: np.random.Generator, n: int, axes=(1.0, 0.7, 0.5)) -> np.ndarray:
    """n points area-uniform on an axis-aligned ellipsoid (rejection on the area element)."""
    a = np.asarray(axes, dtype=np.float64)
    jmax = 1.0 / a.min()
    out = []
    have = 0
    while have < n:
        u = sphere_points(rng, 2 * (n - have) + 64)
        jac = np.sqrt(((u / a) ** 2).sum(1))  # area scale / (abc)
        keep = rng.random(len(u)) * jmax < jac
        pts = u[keep] * a
        out.append(pts)
        have += len(pts)
    return np.concatenate(out)[:n]


def torus_points(rng: np.random.Generator, n: int, R: float = 1.0, r: float = 0.3) -> np.ndarray:
    """n points area-uniform on a torus (rejection on R + r cos v)."""
    out = []
    have = 0
    while have < n:
        m = 2 * (n - have) + 64
        u = rng.random(m) * 2 * np.pi
        v = rng.random(m) * 2 * np.pi
        keep = rng.random(m) * (R + r) < (R + r * np.cos(v))
        u, v = u[keep], v[keep]
        out.append(np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], -1))
        have += int(keep.sum())
    return np.concatenate(out)[:n]


# --------------------------------------------------------------------------------------
# analytic deformations
# --------------------------------------------------------------------------------------


def sinusoid(p: np.ndarray, amp: float, freq: float = 1.0) -> np.ndarray:
    """p + amp * [sin(2 pi f y), sin(2 pi f z), sin(2 pi f x)]."""
    p = np.asarray(p, dtype=np.float64)
    w = 2 * np.pi * freq
    return p + amp * np.stack([np.sin(w * p[:, 1]), np.sin(w * p[:, 2]), np.sin(w * p[:, 0])], -1)


def twist_bend(p: np.ndarray, s: float, tube_r: float = 0.3, R_bend: float = 1.3) -> np.ndarray:
    """Twist about z by (pi s / 2)(z / tube_r), then bend z += tube_r s x^2 / R_bend^2."""
    p = np.asarray(p, dtype=np.float64)
    ang = (np.pi * s / 2.0) * (p[:, 2] / tube_r)
    c, sn = np.cos(ang), np.sin(ang)
    x = c * p[:, 0] - sn * p[:, 1]
    y = sn * p[:, 0] + c * p[:, 1]
    z = p[:, 2] + tube_r * s * x**2 / R_bend**2
    return np.stack([x, y, z], -1)


# --------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    """One frame-pair fitting problem (all arrays float32 / int32)."""

    name: str
    template: np.ndarray  # [V,3] template vertices X_{t-1}
    edges: np.ndarray  # [E,2] int32
    source: np.ndarray  # [N,3] P_{t-1}
    target: np.ndarray  # [M,3] P_t
    res: tuple  # vertices per axis, coarse -> fine
    lo: tuple = (-1.5, -1.5, -1.5)
    hi: tuple = (1.5, 1.5, 1.5)
    steps: int = 200
    thetas: list | None = None  # optional initial grid values per level, [n,n,n,3] float32


def single_pair(seed: int = 0, n_pts: int = 2048) -> Workload:
    """Single frame pair on the unit sphere: icosphere(3) template, two independent
    uniform draws of `n_pts`, the second displaced by 0.1 [sin 2pi y, sin 2pi z, sin 2pi x];
    levels 8^3, 16^3, 32^3; 200 steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v, _, e = icosphere(3)
    src = sphere_points(rng, n_pts)
    tgt = sinusoid(sphere_points(rng, n_pts), 0.1)
    return Workload("single_pair_sphere_2k", v, e, src.astype(F32), tgt.astype(F32), (8, 16, 32), steps=200)


def ellipsoid_pair(seed: int = 0, n_pts: int = 100_000, freq: int = 71, res=(16, 32, 64, 128),
                   theta_sigma: float = 0.01) -> Workload:
    """Frame pair on the ellipsoid (1, 0.7, 0.5): geodesic template (freq 71: 50 412
    verts), 100k area-uniform source points, 100k target points deformed by
    0.05 [sin 2pi y, sin 2pi z, sin 2pi x]; grids 16^3..128^3 with N(0, 0.01^2) values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    axes = (1.0, 0.7, 0.5)
    v, _, e = geodesic_sphere(freq, axes)
    src = ellipsoid_points(rng, n_pts, axes)
    tgt = sinusoid(ellipsoid_points(rng, n_pts, axes), 0.05)
    thetas = None
    if theta_sigma:
        thetas = [(rng.standard_normal((n, n, n, 3)) * theta_sigma).astype(F32) for n in res]
    return Workload(f"ellipsoid_pair_{n_pts // 1000}k", v, e, src.astype(F32), tgt.astype(F32), tuple(res),
                    steps=100, thetas=thetas)


def torus_sequence_frame(k: int, n_frames: int = 100, n_pts: int = 20_000, seed: int = 0,
                         noise: float = 0.002, dropout: float = 0.1) -> np.ndarray:
    """Frame k of the twisted-and-bent torus sequence: n_pts area-uniform samples, the
    deformation at s = k / (n_frames - 1), Gaussian noise, Bernoulli dropout."""
    rng = np.random.Generator(np.random.PCG64(seed * 1000 + k))
    s = k / max(n_frames - 1, 1)
    p = twist_bend(torus_points(rng, n_pts), s)
    p = p + rng.standard_normal(p.shape) * noise
    keep = rng.random(len(p)) >= dropout
    p = p[keep]
    assert np.all(np.abs(p) < 1.45)
    return p.astype(F32)


def torus_sequence(n_frames: int = 100, n_pts: int = 20_000, seed: int = 0):
    """Template (200x100 torus mesh) and a generator of frames for the plain sequence fit."""
    v, _, e = torus_mesh(200, 100)
    return v, e, (lambda k: torus_sequence_frame(k, n_frames, n_pts, seed))


# grid sizes the preconditioner's radix-2/3 line transforms take: 2^a 3^b in 2..256
SMOOTH_SIZES = sorted({2**a * 3**b for a in range(9) for b in range(6) if 2 <= 2**a * 3**b <= 256})


def smooth23(n: float) -> int:
    """The size 2^a 3^b in 2..256 nearest to n on a log scale (ties to the smaller)."""
    ln = math.log(max(n, 2.0))
    return min(SMOOTH_SIZES, key=lambda m: (abs(math.log(m) - ln), m))


def batched_job(i: int, scale: float = 1.0, n_pts: int | None = None):
    """Job i of the batched / served workload: shape in {sphere, torus, ellipsoid},
    points per frame log-uniform in [5k, 200k] (times `scale`; `n_pts` overrides the draw,
    e.g. for the 500k-point frames of the served trace), 3-5 levels with the finest
    log-uniform in [32, 256] vertices per axis (rounded to the nearest 2^a 3^b, each coarser
    level half the next one, rounded the same way, at least 4), and an
    analytic deformation in {twist, bend, sinusoid}.  Returns a dict of arrays/params."""
    rng = np.random.Generator(np.random.PCG64(1000 + i))
    shape = ["sphere", "torus", "ellipsoid"][rng.integers(3)]
    drawn = int(math.exp(rng.uniform(math.log(5e3), math.log(2e5))) * scale)
    n_pts = max(drawn if n_pts is None else int(n_pts), 256)
    L = int(rng.integers(3, 6))
    finest = smooth23(math.exp(rng.uniform(math.log(32), math.log(256))))
    res = tuple(max(4, smooth23(finest / 2 ** (L - 1 - l))) for l in range(L))
    kind = ["twist", "bend", "sinusoid"][rng.integers(3)]
    amp = rng.uniform(0.05, 0.1)
    fr = rng.uniform(1.0, 3.0)
    n_tmpl = int(min(max(n_pts // 2, 642), 100_000))
    if shape == "sphere":
        freq = max(8, int(round(math.sqrt((n_tmpl - 2) / 10))))
        v, _, e = geodesic_sphere(freq)
        sampler = lambda r, n: sphere_points(r, n)
    elif shape == "ellipsoid":
        freq = max(8, int(round(math.sqrt((n_tmpl - 2) / 10))))
        v, _, e = geodesic_sphere(freq, (1.0, 0.7, 0.5))
        sampler = lambda r, n: ellipsoid_points(r, n)
    else:
        nv = max(8, int(round(math.sqrt(n_tmpl / 2))))
        v, _, e = torus_mesh(2 * nv, nv)
        sampler = lambda r, n: torus_points(r, n)

    def frame(k: int, n_frames: int = 10) -> np.ndarray:
        r = np.random.Generator(np.random.PCG64((1000 + i) * 1000 + k))
        s = k / max(n_frames - 1, 1)
        p = sampler(r, n_pts)
        if kind == "sinusoid":
            p = sinusoid(p, amp * s, fr)
        elif kind == "twist":
            p = twist_bend(p, s, tube_r=0.3, R_bend=1e9)
        else:
            p = twist_bend(p, 0.0) + np.stack([0 * p[:, 0], 0 * p[:, 0], 0.3 * s * p[:, 0] ** 2 / 1.69], -1)
        return np.clip(p, -1.45, 1.45).astype(F32)

    return dict(shape=shape, n_pts=n_pts, res=res, kind=kind, template=v, edges=e, frame=frame)
