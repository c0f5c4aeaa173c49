"""Seeded synthetic inputs for the Helmholtz MLFMA matvec.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It holds none of the method's arithmetic: only a counter-based
random stream (SplitMix64, Steele/Lea/Flood 2014), Box-Muller normals, and
point clouds shaped like the paper's workloads (sphere surfaces with leaves of
a quarter wavelength, Sec. 5; a cube surface with dense Gaussian clusters; random
ellipsoid surfaces).  Every function is a pure function of its seed.

Seeds follow the convention ``seed = 1000 * workload + stream``.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+n-1`` of the SplitMix64 stream seeded with ``seed``.

    Output i is mix(seed + (i+1)*gamma) (mod 2**64), with the published
    finaliser (shifts 30/27/31 and the two odd multipliers).
    """
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits of the stream."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, start: int = 0) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m, 2 * start)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:n]


def complex_normal(seed: int, n: int, nrhs: int = 1) -> np.ndarray:
    """i.i.d. (N(0,1) + i N(0,1)) / sqrt(2), shape ``[nrhs][n]`` complex128."""
    z = normal(seed, 2 * n * nrhs).reshape(nrhs, n, 2)
    return ((z[..., 0] + 1j * z[..., 1]) / math.sqrt(2.0)).astype(np.complex128)


def sphere(n: int, radius: float, seed: int, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """``n`` points uniform on a sphere surface: normalised Gaussian triplets."""
    g = normal(seed, 3 * n).reshape(n, 3)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g * radius + np.asarray(center, dtype=np.float64)


def cube_surface(n: int, half: float, seed: int) -> np.ndarray:
    """``n`` points uniform on the surface of the cube [-half, half]^3.

    Face = floor(6u); the two in-face coordinates are uniform.
    """
    u = uniform(seed, 3 * n).reshape(n, 3)
    face = np.minimum((u[:, 0] * 6.0).astype(np.int64), 5)
    a = (2.0 * u[:, 1] - 1.0) * half
    b = (2.0 * u[:, 2] - 1.0) * half
    axis = face // 2
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    pts = np.empty((n, 3))
    for ax in range(3):
        o1, o2 = (ax + 1) % 3, (ax + 2) % 3
        m = axis == ax
        pts[m, ax] = sign[m] * half
        pts[m, o1] = a[m]
        pts[m, o2] = b[m]
    return pts


def cube_surface_clusters(n: int, half: float = 16.0, frac_surface: float = 0.7,
                          nclusters: int = 64, sigma: float = 0.05, seed: int = 3000) -> np.ndarray:
    """floor(frac*n) points on the cube surface, the rest in Gaussian clusters.

    Point i of the clustered part goes to cluster (i mod nclusters); the cluster
    centres are uniform on the same cube surface.
    """
    ns = int(math.floor(frac_surface * n))
    nc = n - ns
    surf = cube_surface(ns, half, seed)
    centres = cube_surface(nclusters, half, seed + 1)
    g = normal(seed + 2, 3 * nc).reshape(nc, 3) * sigma
    cl = centres[np.arange(nc) % nclusters] + g
    return np.concatenate([surf, cl], axis=0)


def ellipsoid(n: int, a: float, b: float, c: float, seed: int) -> np.ndarray:
    """``n`` points area-uniform on the ellipsoid with semi-axes (a, b, c).

    A unit-sphere point u maps to (a u_x, b u_y, c u_z) and is accepted with
    probability sqrt((b c u_x)^2 + (a c u_y)^2 + (a b u_z)^2) / max(bc, ac, ab).
    Candidates are drawn in fixed batches from one stream, so the result is a
    pure function of the seed.
    """
    out = []
    have = 0
    batch = max(1024, 2 * n)
    it = 0
    gmax = max(b * c, a * c, a * b)
    while have < n:
        g = normal(seed, 3 * batch, start=3 * batch * it).reshape(batch, 3)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        acc = uniform(seed + 7919, batch, start=batch * it)
        dens = np.sqrt((b * c * g[:, 0]) ** 2 + (a * c * g[:, 1]) ** 2 + (a * b * g[:, 2]) ** 2) / gmax
        keep = g[acc < dens]
        out.append(keep * np.array([a, b, c]))
        have += keep.shape[0]
        it += 1
    return np.concatenate(out, axis=0)[:n]


def ellipsoid_batch(n_geom: int, seed: int, nmin: int = 1000, nmax: int = 65536,
                    amin: float = 2.0, amax: float = 16.0):
    """Geometries with log-uniform sizes in [nmin, nmax] and U(amin, amax) semi-axes."""
    u = uniform(seed, 4 * n_geom).reshape(n_geom, 4)
    sizes = np.rint(np.exp(math.log(nmin) + u[:, 0] * (math.log(nmax) - math.log(nmin)))).astype(np.int64)
    axes = amin + u[:, 1:] * (amax - amin)
    geoms = [ellipsoid(int(sizes[g]), *axes[g], seed=seed + 10 + g) for g in range(n_geom)]
    return geoms, sizes, axes


# ---------------------------------------------------------------------------
# Named workloads (wavelength 1, k = 2 pi).
# ---------------------------------------------------------------------------
K_WAVE = 2.0 * math.pi


def workload(name: str):
    """Return (points [n,3] float64, charges [1][n] complex128, params dict)."""
    if name == "sphere4k":           # N = 4,096 on a sphere of radius 2 (diameter 4 wavelengths)
        pts = sphere(4096, 2.0, seed=1001)
        q = complex_normal(1002, 4096)
        return pts, q, dict(k=K_WAVE, digits=3, leaf_max=0)
    if name == "sphere1m":           # N = 2^20 on a sphere of radius 32 (diameter 64 wavelengths)
        n = 1 << 20
        pts = sphere(n, 32.0, seed=2001)
        q = complex_normal(2002, n)
        return pts, q, dict(k=K_WAVE, digits=3, leaf_max=0)
    if name == "sphere256k":         # N = 2^18 on a sphere of radius 16 (profiling-size case, 8 levels)
        n = 1 << 18
        pts = sphere(n, 16.0, seed=2101)
        q = complex_normal(2102, n)
        return pts, q, dict(k=K_WAVE, digits=3, leaf_max=0)
    if name == "ellipsoid256k":      # N = 262,144 on the (8, 4, 2) ellipsoid
        n = 262144
        pts = ellipsoid(n, 8.0, 4.0, 2.0, seed=5001)
        q = complex_normal(5002, n)
        return pts, q, dict(k=K_WAVE, digits=3, leaf_max=0)
    if name == "cubeclusters4m":     # N = 4,194,304: cube surface + 64 clusters
        n = 1 << 22
        pts = cube_surface_clusters(n, seed=3001)
        q = complex_normal(3002, n)
        return pts, q, dict(k=K_WAVE, digits=4, leaf_max=64)
    if name == "cubeclusters512k":   # N = 524,288, the same construction (profiling-size case)
        n = 1 << 19
        pts = cube_surface_clusters(n, seed=3101)
        q = complex_normal(3102, n)
        return pts, q, dict(k=K_WAVE, digits=4, leaf_max=64)
    raise KeyError(name)
