"""Seeded synthetic inputs: curved quadratic-triangle meshes, densities, directions.

This module holds no arithmetic of the boundary element method itself. It only
produces the geometry and the random data that the GPU path, the tests and the
benchmark feed in. The workloads mirror the paper's: spheres meshed with curved
6-node quadratic triangles (Sec. 5.2, 5.3), plus a prolate spheroid, random
ellipsoids and a torus of the same element type.

Mesh convention (shared by every consumer):
  nodes : (n_nodes, 3) float64
  elems : (n_elems, 6) int32, node order [v0, v1, v2, m01, m12, m20]
          (three vertices, then the mid-edge nodes of edges 0-1, 1-2, 2-0);
          the vertices run counter-clockwise seen from outside the body.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_PHI = (1.0 + math.sqrt(5.0)) / 2.0

_ICO_V = np.array([
    [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
    [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
    [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
], dtype=np.float64)

_ICO_F = np.array([
    [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
    [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
    [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
    [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
], dtype=np.int64)


@dataclass
class Mesh:
    nodes: np.ndarray   # (n_nodes, 3) float64
    elems: np.ndarray   # (n_elems, 6) int32
    name: str = ""

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])

    @property
    def n_dof(self) -> int:
        return 6 * int(self.elems.shape[0])


def _unit_icosphere(m: int):
    """Frequency-m geodesic subdivision of the icosahedron on the unit sphere.

    Each of the 20 faces carries a (2m+1)-point barycentric grid; even grid
    points are element vertices and odd ones the mid-edge nodes, so every
    face yields m*m curved 6-node triangles (20 m^2 in all). Returns unit
    vectors (before any projection) and the element table.
    """
    if m < 1:
        raise ValueError("icosphere frequency must be >= 1")
    M = 2 * m
    grid = [(a, b) for b in range(M + 1) for a in range(M + 1 - b)]
    gidx = {ab: t for t, ab in enumerate(grid)}
    gw = np.array(grid, dtype=np.float64)            # (G, 2)
    nodes = []
    elems = []
    V = _ICO_V / np.linalg.norm(_ICO_V, axis=1, keepdims=True)
    for f, (ia, ib, ic) in enumerate(_ICO_F):
        A, B, C = V[ia], V[ib], V[ic]
        pa = (M - gw[:, 0] - gw[:, 1])[:, None] * A + gw[:, 0:1] * B + gw[:, 1:2] * C
        pa = pa / np.linalg.norm(pa, axis=1, keepdims=True)
        base = f * len(grid)
        nodes.append(pa)
        for j in range(m):
            for i in range(m - j):
                a, b = 2 * i, 2 * j
                g = lambda da, db: base + gidx[(a + da, b + db)]
                elems.append([g(0, 0), g(2, 0), g(0, 2), g(1, 0), g(1, 1), g(0, 1)])
                if i + j < m - 1:
                    elems.append([g(2, 0), g(2, 2), g(0, 2), g(2, 1), g(1, 2), g(1, 1)])
    nodes = np.concatenate(nodes, axis=0)
    elems = np.asarray(elems, dtype=np.int32)
    return nodes, elems


def _orient_outward(nodes: np.ndarray, elems: np.ndarray, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Flip elements whose vertex order is clockwise seen from outside a star-shaped body."""
    v0, v1, v2 = nodes[elems[:, 0]], nodes[elems[:, 1]], nodes[elems[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    cen = (v0 + v1 + v2) / 3.0 - np.asarray(center)
    bad = np.einsum("ij,ij->i", nrm, cen) < 0
    e = elems.copy()
    # swap v1<->v2 and m01<->m20 (m12 stays): reverses orientation
    e[bad, 1], e[bad, 2] = elems[bad, 2], elems[bad, 1]
    e[bad, 3], e[bad, 5] = elems[bad, 5], elems[bad, 3]
    return e


def icosphere(m: int, radius: float = 0.5, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Sphere of the given radius: 20 m^2 curved quadratic triangles, N = 120 m^2 DOF."""
    u, e = _unit_icosphere(m)
    nodes = radius * u + np.asarray(center, dtype=np.float64)
    e = _orient_outward(nodes, e, center)
    return Mesh(nodes=np.ascontiguousarray(nodes), elems=e, name=f"sphere(a={radius},m={m})")


def ellipsoid(m: int, semi_axes=(1.0, 0.25, 0.25)) -> Mesh:
    """Ellipsoid with the given semi-axes; icosphere nodes moved radially onto its surface."""
    a, b, c = (float(s) for s in semi_axes)
    u, e = _unit_icosphere(m)
    t = 1.0 / np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2 + (u[:, 2] / c) ** 2)
    nodes = u * t[:, None]
    e = _orient_outward(nodes, e)
    return Mesh(nodes=np.ascontiguousarray(nodes), elems=e, name=f"ellipsoid({a},{b},{c},m={m})")


def torus(R: float = 0.5, r: float = 0.2, nu: int = 250, nv: int = 100) -> Mesh:
    """Torus from an nu x nv parametric quad grid, two curved triangles per quad.

    Every node (vertices and mid-edge nodes at parametric midpoints) lies
    exactly on the torus.
    """
    U, W = 2 * nu, 2 * nv
    uu = np.arange(U) * (2 * math.pi / U)
    vv = np.arange(W) * (2 * math.pi / W)
    UU, VV = np.meshgrid(uu, vv, indexing="ij")
    rho = R + r * np.cos(VV)
    nodes = np.stack([rho * np.cos(UU), rho * np.sin(UU), r * np.sin(VV)], axis=-1).reshape(-1, 3)
    idx = lambda a, b: (a % U) * W + (b % W)
    elems = []
    for i in range(nu):
        for j in range(nv):
            a, b = 2 * i, 2 * j
            # (a,b) -> (a+2,b) -> (a+2,b+2): counter-clockwise in (u,v) = outward
            elems.append([idx(a, b), idx(a + 2, b), idx(a + 2, b + 2),
                          idx(a + 1, b), idx(a + 2, b + 1), idx(a + 1, b + 1)])
            elems.append([idx(a, b), idx(a + 2, b + 2), idx(a, b + 2),
                          idx(a + 1, b + 1), idx(a + 1, b + 2), idx(a, b + 1)])
    return Mesh(nodes=np.ascontiguousarray(nodes), elems=np.asarray(elems, dtype=np.int32),
                name=f"torus(R={R},r={r},{nu}x{nv})")


def complex_gaussian(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian vector (real and imaginary parts i.i.d. N(0,1)), complex128."""
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs is None else (nrhs, n)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors on a Fibonacci sphere: z_j = 1-(2j+1)/n, phi_j = j*pi*(3-sqrt 5)."""
    j = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / n
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted distinct row indices, drawn without replacement."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)


def random_ellipsoid_params(count: int, seed: int = 1, kd_range=(20.0, 80.0), axes_range=(0.3, 1.0)):
    """Semi-axes U[0.3,1] and wavenumbers with kD in U[20,80], D = 2 * largest semi-axis."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ax = rng.uniform(axes_range[0], axes_range[1], size=3)
        kd = rng.uniform(kd_range[0], kd_range[1])
        D = 2.0 * float(ax.max())
        out.append((tuple(float(a) for a in ax), kd / D))
    return out


# Named workloads (the sizes and wavenumbers of the paper-shaped configurations)
def sphere_points(n: int, radius: float = 1.0):
    """n points on a sphere (Fibonacci lattice, nearly uniform) and their outward unit normals."""
    d = fibonacci_directions(n)
    return radius * d, d.copy()


def table1_k(n: int, points_per_wavelength: float = 20.0, radius: float = 1.0) -> float:
    """Wavenumber at which n uniform points on the sphere have about ppw points per wavelength."""
    h = math.sqrt(4.0 * math.pi * radius * radius / n)
    return 2.0 * math.pi / (points_per_wavelength * h)


# particle summations of Sec. 5.1 (Table 1): unit sphere, ~20 points per wavelength, k = 8 pi ... 64 pi
TABLE1 = [(73728, 8 * math.pi), (294912, 16 * math.pi), (1179648, 32 * math.pi), (4718592, 64 * math.pi)]


WORKLOADS = {
    # sphere a=0.5 (D=1), kD=10, 320 elements, 1920 DOF
    "sphere_kd10": dict(kind="sphere", m=4, radius=0.5, k=10.0, eps=1e-6, leaf=64),
    # sphere a=0.5, kD=100, 16820 elements, 100920 DOF
    "sphere_kd100": dict(kind="sphere", m=29, radius=0.5, k=100.0, eps=1e-4, leaf=64),
    # sphere a=0.5, kD=60, 8000 elements, 48000 DOF (profiling-sized: a few GB on the device)
    "sphere_kd60": dict(kind="sphere", m=20, radius=0.5, k=60.0, eps=1e-4, leaf=64),
    # sphere a=0.5, kD=200, 188180 elements, 1129080 DOF (h ~ lambda/5)
    "sphere_kd200": dict(kind="sphere", m=97, radius=0.5, k=200.0, eps=1e-4, leaf=64),
    # prolate spheroid (1, .25, .25), kD=200, 67280 elements, 403680 DOF
    "spheroid_kd200": dict(kind="ellipsoid", m=58, axes=(1.0, 0.25, 0.25), k=100.0, eps=1e-4, leaf=64),
    # torus R=.5 r=.2, kD=150 with D=1.4, 50000 elements, 300000 DOF
    "torus_kd150": dict(kind="torus", R=0.5, r=0.2, nu=250, nv=100, k=150.0 / 1.4, eps=1e-4, leaf=64),
    # sphere a=0.5, kD=1000, 669780 elements, 4018680 DOF
    "sphere_kd1000": dict(kind="sphere", m=183, radius=0.5, k=1000.0, eps=1e-4, leaf=64),
}


def make_mesh(spec: dict) -> Mesh:
    kind = spec["kind"]
    if kind == "sphere":
        return icosphere(spec["m"], spec.get("radius", 0.5))
    if kind == "ellipsoid":
        return ellipsoid(spec["m"], spec["axes"])
    if kind == "torus":
        return torus(spec["R"], spec["r"], spec["nu"], spec["nv"])
    raise ValueError(kind)
