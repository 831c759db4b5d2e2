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
f4 the top (t=+1) triangle.  Prisms are numbered column by column, bottom up:
on a full mesh prism e sits in column b = e // nlayers and layer l = e % nlayers
(layer 0 at the bottom); a mesh with ``col_layers`` (the hull tank) holds layers
0 .. col_layers[b]-1 over base triangle b.
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

    Optional 3D fields (all None on the plain sigma-layer meshes):
    ``col_layers`` [ntri]: layers present over each base triangle (from the bottom);
    ``z_iface`` [nlayers+1, 2]: layer interface k lies at z = a_k + b_k eta(x, y)
    (None: sigma layers, a_k = -depth (1 - k/nlayers), b_k = k/nlayers);
    ``edge_arc`` [ntri, 3, 3]: per base edge f (f0=(v0,v1), f1=(v1,v2), f2=(v2,v0))
    the circle (cx, cy, R) the edge follows between its vertices, R = 0 straight.
    """
    dim: int
    vxy: np.ndarray              # [nvert, 2] float64
    tri: np.ndarray              # [ntri, 3] int32, counter-clockwise
    nlayers: int = 0
    depth: float = 1.0
    eta_modes: list = field(default_factory=list)   # [(a, kx, ky, phase)]: eta = sum a*cos(kx*x+ky*y+phase)
    face_bc: np.ndarray | None = None               # [nelem, nfaces] int8, 1 = Dirichlet
    col_layers: np.ndarray | None = None            # [ntri] int32
    z_iface: np.ndarray | None = None               # [nlayers+1, 2] float64
    edge_arc: np.ndarray | None = None              # [ntri, 3, 3] float64

    @property
    def nelem(self) -> int:
        if self.dim == 3 and self.col_layers is not None:
            return int(np.sum(self.col_layers))
        return int(self.tri.shape[0]) * (self.nlayers if self.dim == 3 else 1)

    def columns(self):
        """(base triangle, layer) of every prism in element order (3D only)."""
        ntri = int(self.tri.shape[0])
        col = (np.full(ntri, self.nlayers, dtype=np.int64) if self.col_layers is None
               else np.asarray(self.col_layers, dtype=np.int64))
        b = np.repeat(np.arange(ntri), col)
        start = np.concatenate([[0], np.cumsum(col)[:-1]])
        l = np.arange(int(col.sum())) - np.repeat(start, col)
        return b, l

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

    2D: edges used by a single triangle.  3D: the bottom face of every column's lowest
    prism, the top face of its highest prism, and the lateral faces over base edges used
    by a single triangle or whose neighbour column is lower than the prism's layer."""
    tri = mesh.tri
    owners: dict = {}
    for t, (v0, v1, v2) in enumerate(tri):
        for (a, b) in ((v0, v1), (v1, v2), (v2, v0)):
            owners.setdefault((min(a, b), max(a, b)), []).append(t)
    nf = mesh.nfaces
    fb = np.zeros((mesh.nelem, nf), dtype=np.int8)
    if mesh.dim == 2:
        for t, (v0, v1, v2) in enumerate(tri):
            for f, (a, b) in enumerate(((v0, v1), (v1, v2), (v2, v0))):
                if len(owners[(min(a, b), max(a, b))]) == 1:
                    fb[t, f] = 1
        mesh.face_bc = fb
        return mesh
    cb, cl = mesh.columns()
    ntri = tri.shape[0]
    col = np.bincount(cb, minlength=ntri)
    for e in range(cb.size):
        t, l = int(cb[e]), int(cl[e])
        v0, v1, v2 = tri[t]
        for f, (a, b) in enumerate(((v0, v1), (v1, v2), (v2, v0))):
            nb = [o for o in owners[(min(a, b), max(a, b))] if o != t]
            if not nb or col[nb[0]] <= l:
                fb[e, f] = 1
        if l == 0:
            fb[e, 3] = 1
        if l == col[t] - 1:
            fb[e, 4] = 1
    mesh.face_bc = fb
    return mesh


# ---------------------------------------------------------------- hull tank
def _hull_axis(n: int, lo: float, hi: float, rc: float, length: float) -> np.ndarray:
    """n+1 grid coordinates on [0, length] with lines at lo, lo+rc, hi-rc, hi: about
    uniform cells, at least one cell per segment, the two corner segments alike."""
    c = max(1, int(round(n * rc / length)))
    m = max(1, int(round(n * (hi - lo - 2 * rc) / length)))
    if (n - 2 * c - m) % 2:
        m += 1
    o = (n - 2 * c - m) // 2
    if o < 1:
        raise ValueError("grid too coarse for the hull footprint")
    segs = [(0.0, lo, o), (lo, lo + rc, c), (lo + rc, hi - rc, m), (hi - rc, hi, c), (hi, length, o)]
    pts = [np.linspace(a, b, k + 1)[:-1] for (a, b, k) in segs]
    return np.concatenate(pts + [np.array([length])])


def eta_powerlaw(nmodes: int = 32, seed: int = SEED, kmax: int = 8, amax: float = 0.1):
    """Free surface as ``nmodes`` cosine modes with integer wavevectors (kx in 0..kmax,
    ky in -kmax..kmax, not both zero), amplitudes proportional to |k|^-1.5, uniform
    random phases; scaled so that sum |a| = amax (hence max |eta| <= amax)."""
    rng = np.random.default_rng(seed)
    modes = []
    while len(modes) < nmodes:
        kx = int(rng.integers(0, kmax + 1))
        ky = int(rng.integers(-kmax, kmax + 1))
        if kx == 0 and ky == 0:
            continue
        modes.append((math.hypot(kx, ky) ** -1.5, float(kx), float(ky), float(rng.uniform(0, 2 * math.pi))))
    tot = sum(a for a, _, _, _ in modes)
    return [(a * amax / tot, kx, ky, ph) for (a, kx, ky, ph) in modes]


def hull_tank(n: int = 64, length: float = 2 * math.pi, depth: float = 1.0, hull_len: float = 0.3,
              hull_width: float = 0.1, corner: float = 0.25, draft: float = 0.3, nl_lower: int = 2,
              nl_upper: int = 2, eta_modes=None) -> Mesh:
    """Wave tank [0, L]^2 x [-depth, eta] with a surface-piercing rounded-box hull.

    The hull's footprint is centred, ``hull_len`` L long in x and ``hull_width`` L wide
    in y, its corners rounded with radius ``corner`` x width; it reaches ``draft`` x depth
    below z = 0.  Two vertical zones: the lower zone [-depth, -draft] in ``nl_lower`` flat
    layers everywhere; the upper zone [-draft, eta] in ``nl_upper`` sigma layers outside
    the footprint only (the hull is cut out).  The n x n base grid is graded so that grid
    lines run along the footprint's straight sides and the corner arcs' end points; the
    footprint-boundary vertices inside each corner square are moved radially onto the
    arc, and the footprint-boundary edges between two arc points follow the arc.
    Dirichlet on the free surface (top faces of full columns); homogeneous Neumann on the
    bottom, the tank walls and the hull (its sides and its bottom)."""
    xa, xb = 0.5 * length * (1 - hull_len), 0.5 * length * (1 + hull_len)
    ya, yb = 0.5 * length * (1 - hull_width), 0.5 * length * (1 + hull_width)
    rc = corner * hull_width * length
    xs = _hull_axis(n, xa, xb, rc, length)
    ys = _hull_axis(n, ya, yb, rc, length)
    nx, ny = len(xs) - 1, len(ys) - 1
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    vxy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    tri, infoot = [], []
    tol = 1e-9 * length
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, d = a + 1, a + (nx + 1)
            c = d + 1
            foot = xs[i] >= xa - tol and xs[i + 1] <= xb + tol and ys[j] >= ya - tol and ys[j + 1] <= yb + tol
            tri += [(a, b, c), (a, c, d)]
            infoot += [foot, foot]
    tri = np.asarray(tri, dtype=np.int32)
    infoot = np.asarray(infoot)
    # corners: (corner point, arc centre)
    corners = [((xa, ya), (xa + rc, ya + rc)), ((xb, ya), (xb - rc, ya + rc)),
               ((xb, yb), (xb - rc, yb - rc)), ((xa, yb), (xa + rc, yb - rc))]
    on_side = (((np.abs(vxy[:, 0] - xa) < tol) | (np.abs(vxy[:, 0] - xb) < tol)) & (vxy[:, 1] > ya - tol)
               & (vxy[:, 1] < yb + tol)) | (((np.abs(vxy[:, 1] - ya) < tol) | (np.abs(vxy[:, 1] - yb) < tol))
                                             & (vxy[:, 0] > xa - tol) & (vxy[:, 0] < xb + tol))
    for (K, C) in corners:
        inside = on_side & (np.abs(vxy[:, 0] - K[0]) < rc - tol) & (np.abs(vxy[:, 1] - K[1]) < rc - tol)
        for v in np.flatnonzero(inside):
            d = vxy[v] - np.asarray(C)
            vxy[v] = np.asarray(C) + rc * d / np.linalg.norm(d)
    owners: dict = {}
    for t, (v0, v1, v2) in enumerate(tri):
        for (a, b) in ((v0, v1), (v1, v2), (v2, v0)):
            owners.setdefault((min(a, b), max(a, b)), []).append(t)
    arc = np.zeros((tri.shape[0], 3, 3))
    for t, (v0, v1, v2) in enumerate(tri):
        for f, (a, b) in enumerate(((v0, v1), (v1, v2), (v2, v0))):
            own = owners[(min(a, b), max(a, b))]
            if len(own) != 2 or infoot[own[0]] == infoot[own[1]]:
                continue
            for (K, C) in corners:
                near = all(abs(vxy[v, 0] - K[0]) <= rc + tol and abs(vxy[v, 1] - K[1]) <= rc + tol
                           and abs(np.linalg.norm(vxy[v] - np.asarray(C)) - rc) < tol for v in (a, b))
                if near:
                    arc[t, f] = (C[0], C[1], rc)
    nl = nl_lower + nl_upper
    col = np.where(infoot, nl_lower, nl).astype(np.int32)
    zif = np.zeros((nl + 1, 2))
    for k in range(nl_lower + 1):
        zif[k] = (-depth + k * (depth - draft * depth) / nl_lower, 0.0)
    for k in range(1, nl_upper + 1):
        zif[nl_lower + k] = (-draft * depth * (1.0 - k / nl_upper), k / nl_upper)
    m = Mesh(dim=3, vxy=vxy, tri=tri, nlayers=nl, depth=depth, eta_modes=list(eta_modes or []),
             col_layers=col, z_iface=zif, edge_arc=arc)
    cb, cl = m.columns()
    fb = np.zeros((m.nelem, 5), dtype=np.int8)
    fb[(cl == nl - 1), 4] = 1
    m.face_bc = fb
    return m


def config_hull(n: int = 64) -> Mesh:
    """The learned-smoother tank: 64 x 64 base grid, rounded-box hull 0.3 L long, 0.1 L
    wide, corner radius a quarter of the width, draft 0.3 h, 2 + 2 layers; eta a sum of
    32 cosine modes with power-law amplitudes (max |eta| <= 0.1 h)."""
    return hull_tank(n, eta_modes=eta_powerlaw(32))
