"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the solver: it only builds the *inputs* of
the Laplace problem (Section 2, Eq. laplaceproblem) that the paper solves on
its own meshes, which are not available here:

* straight-sided triangulations of rectangles (quads split along the SW-NE
  diagonal), used as the 2D vertical slice and as the horizontal base of the
  sigma-extruded prism meshes (Section 3.1);
* free-surface elevations eta(x, y) given as sums of cosine modes;
* exact harmonic potentials (linear Airy / cosh modes) used as Dirichlet data
  on the free surface and as exact solutions for error checks;
* per-element boundary-face flags (Dirichlet on the free surface, homogeneous
  Neumann elsewhere, Eq. laplaceproblem).

Face numbering follows the element conventions used by both the oracle and
the CUDA library: triangle faces f0=(v0,v1), f1=(v1,v2), f2=(v2,v0); prism
faces f0..f2 are the lateral quads over those edges, f3 the bottom (t=-1) and
f4 the top (t=+1) triangle.  Prism e sits in column b = e // nlayers and layer
l = e % nlayers (layer 0 at the bottom).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 2009_00705


@dataclass
class Mesh:
    """Mesh description handed to both the oracle and the library.

    dim == 2: triangles in the (x, z) plane; ``vxy`` holds (x, z).
    dim == 3: prisms extruded in ``nlayers`` sigma layers over the base
    triangulation; ``vxy`` holds (x, y); flat bottom z = -depth; the free
    surface is z = eta(x, y) given by ``eta_modes``.
    """
    dim: int
    vxy: np.ndarray              # [nvert, 2] float64
    tri: np.ndarray              # [ntri, 3] int32, counter-clockwise
    nlayers: int = 0
    depth: float = 1.0
    eta_modes: list = field(default_factory=list)   # [(a, kx, ky, phase)]: eta = sum a*cos(kx*x+ky*y+phase)
    face_bc: np.ndarray | None = None               # [nelem, nfaces] int8, 1 = Dirichlet

    @property
    def nelem(self) -> int:
        return int(self.tri.shape[0]) * (self.nlayers if self.dim == 3 else 1)

    @property
    def nfaces(self) -> int:
        return 5 if self.dim == 3 else 3

    def eta(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for (a, kx, ky, ph) in self.eta_modes:
            out = out + a * np.cos(kx * x + ky * y + ph)
        return out


def rect_triangulation(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float):
    """Vertices of an (nx+1) x (ny+1) grid and 2*nx*ny CCW triangles.

    Quad (i, j) with corners a=(i,j), b=(i+1,j), c=(i+1,j+1), d=(i,j+1) is split
    along the SW-NE diagonal into (a, b, c) and (a, c, d)."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")          # [ny+1, nx+1]
    vxy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    tri = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b = a + 1
            d = a + (nx + 1)
            c = d + 1
            tri.append((a, b, c))
            tri.append((a, c, d))
    return vxy, np.asarray(tri, dtype=np.int32)


def slice2d(nx: int = 16, nz: int = 4, length: float = 2 * math.pi, depth: float = 1.0) -> Mesh:
    """2D vertical slice x in [0, length], z in [-depth, 0] (config: 16x4 quads -> 128 triangles).

    Dirichlet on the free surface z = 0 (top edges), homogeneous Neumann on the
    bottom and the side walls."""
    vxy, tri = rect_triangulation(nx, nz, 0.0, length, -depth, 0.0)
    m = Mesh(dim=2, vxy=vxy, tri=tri, depth=depth)
    top = 0.0
    fb = np.zeros((tri.shape[0], 3), dtype=np.int8)
    for e, (v0, v1, v2) in enumerate(tri):
        for f, (a, b) in enumerate(((v0, v1), (v1, v2), (v2, v0))):
            if abs(vxy[a, 1] - top) < 1e-12 and abs(vxy[b, 1] - top) < 1e-12:
                fb[e, f] = 1
    m.face_bc = fb
    return m


def box3d(nx: int, ny: int, nlayers: int, lx: float = 2 * math.pi, ly: float = 2 * math.pi,
          depth: float = 1.0, eta_modes=None) -> Mesh:
    """3D box [0,lx] x [0,ly] x [-depth, eta]: nx*ny quads -> 2*nx*ny base triangles,
    extruded into ``nlayers`` sigma layers of prisms.  Dirichlet on the top faces
    of the top layer (the free surface), homogeneous Neumann elsewhere."""
    vxy, tri = rect_triangulation(nx, ny, 0.0, lx, 0.0, ly)
    m = Mesh(dim=3, vxy=vxy, tri=tri, nlayers=nlayers, depth=depth,
             eta_modes=list(eta_modes or []))
    fb = np.zeros((m.nelem, 5), dtype=np.int8)
    fb[nlayers - 1::nlayers, 4] = 1
    m.face_bc = fb
    return m


def eta_sinx_cosy(amp: float = 0.1):
    """eta = amp*sin(x)*cos(y) written as two cosine modes:
    sin x cos y = (cos(x+y-pi/2) + cos(x-y-pi/2)) / 2."""
    return [(amp / 2, 1.0, 1.0, -math.pi / 2), (amp / 2, 1.0, -1.0, -math.pi / 2)]


def config_slice2d() -> Mesh:
    """2D slice, depth h=1, length 2*pi/k with kh=1, 16x4 quads split into 128 triangles."""
    return slice2d(16, 4, 2 * math.pi, 1.0)


def config_box3d(n: int = 64, nlayers: int = 4) -> Mesh:
    """3D box 2pi x 2pi x 1, n x n quads -> 2n^2 triangles, ``nlayers`` sigma layers,
    eta = 0.1 sin(x) cos(y)."""
    return box3d(n, n, nlayers, eta_modes=eta_sinx_cosy(0.1))


# ---------------------------------------------------------------- exact potentials
def airy2d(x, z, k: float = 1.0, h: float = 1.0):
    """Linear Airy potential cosh(k(z+h))/cosh(kh) * cos(kx): harmonic, zero normal
    derivative on z=-h and on the walls x=0 and x=2*pi/k (cos form; the sin form
    does not satisfy the homogeneous Neumann side walls)."""
    return np.cosh(k * (np.asarray(z) + h)) / np.cosh(k * h) * np.cos(k * np.asarray(x))


def cosh_mode3d(x, y, z, kx: float, ky: float, h: float = 1.0):
    """cosh(kappa(z+h))/cosh(kappa h) cos(kx x) cos(ky y), kappa = |(kx, ky)|: harmonic,
    zero normal derivative on z=-h and on the walls x, y in {0, 2pi} for integer kx, ky."""
    kap = math.hypot(kx, ky)
    return (np.cosh(kap * (np.asarray(z) + h)) / math.cosh(kap * h)
            * np.cos(kx * np.asarray(x)) * np.cos(ky * np.asarray(y)))


def potential3d(x, y, z, h: float = 1.0):
    """Exact potential used on the 3D box: modes (kx,ky) = (1,1) plus 0.5*(2,1)."""
    return cosh_mode3d(x, y, z, 1.0, 1.0, h) + 0.5 * cosh_mode3d(x, y, z, 2.0, 1.0, h)


def tank_potential(x, y, z, modes, h: float = 1.0):
    """Sum of cosh modes a * cosh_mode3d(kx, ky) (modes = [(a, kx, ky)]): harmonic,
    zero normal derivative on the bottom and the walls of [0, 2pi]^2."""
    out = np.zeros(np.broadcast(np.asarray(x), np.asarray(y), np.asarray(z)).shape)
    for (a, kx, ky) in modes:
        out = out + a * cosh_mode3d(x, y, z, kx, ky, h)
    return out


def random_vector(n: int, seed: int = SEED, dtype=np.float64) -> np.ndarray:
    """Seeded standard-normal vector (parity inputs for apply / V-cycle)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n).astype(dtype)


def random_tank(i: int, count_range=(500, 20000)):
    """Seeded batched-tank description: element count uniform in [500, 20000] prisms
    (4 layers), P uniform in {3,4,5,6}, eta a sum of 8 random cosine modes with
    sum |a| <= 0.1, Dirichlet data from 3 random cosh modes.  Returns (mesh, P, modes)."""
    rng = np.random.default_rng(SEED + i)
    count = int(rng.integers(count_range[0], count_range[1] + 1))
    P = int(rng.integers(3, 7))
    n = max(2, int(round(math.sqrt(count / 8.0))))
    amps = rng.uniform(0.0, 1.0, 8)
    amps = amps / amps.sum() * 0.1 * rng.uniform(0.5, 1.0)
    kk = rng.integers(1, 7, size=(8, 2)).astype(np.float64)
    ph = rng.uniform(0, 2 * math.pi, 8)
    modes = [(float(amps[j]), float(kk[j, 0]), float(kk[j, 1]), float(ph[j])) for j in range(8)]
    mesh = box3d(n, n, 4, eta_modes=modes)
    pm = [(float(rng.uniform(0.2, 1.0)), float(rng.integers(0, 4)), float(rng.integers(0, 4)))
          for _ in range(3)]
    return mesh, P, pm


def all_boundary_dirichlet(mesh: Mesh) -> Mesh:
    """Flag every boundary face of ``mesh`` Dirichlet (used for exact-reproduction tests).

    2D: edges used by a single triangle.  3D: bottom and top faces of the bottom /
    top layer, and lateral faces over base edges used by a single triangle."""
    from collections import Counter
    tri = mesh.tri
    cnt = Counter()
    for (v0, v1, v2) in tri:
        for (a, b) in ((v0, v1), (v1, v2), (v2, v0)):
            cnt[(min(a, b), max(a, b))] += 1
    nf = mesh.nfaces
    fb = np.zeros((mesh.nelem, nf), dtype=np.int8)
    nl = mesh.nlayers if mesh.dim == 3 else 1
    for bidx, (v0, v1, v2) in enumerate(tri):
        for f, (a, b) in enumerate(((v0, v1), (v1, v2), (v2, v0))):
            if cnt[(min(a, b), max(a, b))] == 1:
                for l in range(nl):
                    fb[bidx * nl + l, f] = 1
        if mesh.dim == 3:
            fb[bidx * nl, 3] = 1
            fb[bidx * nl + nl - 1, 4] = 1
    mesh.face_bc = fb
    return mesh
