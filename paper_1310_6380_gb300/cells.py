"""Seeded synthetic unit cells and wavevector lists.

This module makes the inputs that every consumer (tests, the benchmark,
the smoke run, the oracle) feeds to the band-structure method: a lattice
(h1, h2), a pixel phase map, a per-phase table of Lame constants and
density, and lists of fractional wavevectors Q (k = Q1 q1 + Q2 q2).  It
holds none of the method's arithmetic: no form factors, no matrices, no
eigenvalues.  Everything is a deterministic function of its arguments.

Conventions (Sec. "Statement of the problem" of the paper):
  * phase[p, q]: p indexes pixels along h1, q along h2; pixel (p, q) covers
    fractional coordinates [p/P, (p+1)/P) x [q/P, (q+1)/P) and its centroid
    is H = ((p + 1/2)/P, (q + 1/2)/P), x = H1 h1 + H2 h2.
  * lam, mu are the Lame constants and rho the density of each phase.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Cell", "square", "hexagonal", "homogeneous_cell", "circle_cell",
    "bilayer_cell", "voronoi_cell", "ellipse_cell", "steel_epoxy_hex_cell",
    "ibz_path", "config0", "config1", "config3_cell", "CONFIGS",
    "MeshCell", "jittered_triangles", "mesh_circle_cell", "mesh_voronoi_cell", "pixel_mesh",
    "steel_epoxy_hex_mesh", "isotropic_stiffness", "rotate_stiffness", "rotated_orthotropic", "with_stiffness",
    "anisotropic_cell", "Cell3", "sphere_cell3", "voronoi_cell3", "extruded_cell3",
    "ibz_path_cubic",
]


@dataclass
class Cell:
    """A pixelated multi-phase 2-D unit cell."""

    h1: np.ndarray            # (2,) first unit-cell vector, Cartesian
    h2: np.ndarray            # (2,) second unit-cell vector
    phase: np.ndarray         # (P, P) uint16 phase index per pixel
    lam: np.ndarray           # (nphase,) Lame lambda per phase
    mu: np.ndarray            # (nphase,) Lame mu (shear modulus) per phase
    rho: np.ndarray           # (nphase,) density per phase
    name: str = "cell"
    lattice: str = "square"   # "square" or "hex": selects the IBZ path
    meta: dict = field(default_factory=dict)
    stiffness: np.ndarray = None   # optional (nphase, 3, 3) in-plane Voigt stiffness

    @property
    def P(self) -> int:
        return int(self.phase.shape[0])

    @property
    def nphase(self) -> int:
        return int(self.lam.shape[0])

    def shifted(self, s1: int, s2: int) -> "Cell":
        """The same cell translated by whole pixels (circular shift)."""
        return Cell(self.h1.copy(), self.h2.copy(),
                    np.roll(self.phase, (s1, s2), axis=(0, 1)).copy(),
                    self.lam.copy(), self.mu.copy(), self.rho.copy(),
                    self.name + f"+shift({s1},{s2})", self.lattice, dict(self.meta))

    def with_props(self, lam=None, mu=None, rho=None, h_scale: float = 1.0) -> "Cell":
        return Cell(self.h1 * h_scale, self.h2 * h_scale, self.phase.copy(),
                    self.lam.copy() if lam is None else np.asarray(lam, np.float64),
                    self.mu.copy() if mu is None else np.asarray(mu, np.float64),
                    self.rho.copy() if rho is None else np.asarray(rho, np.float64),
                    self.name, self.lattice, dict(self.meta))


def square(a: float = 1.0):
    return np.array([a, 0.0]), np.array([0.0, a])


def hexagonal(a: float = 1.0):
    return np.array([a, 0.0]), np.array([0.5 * a, np.sqrt(3.0) / 2.0 * a])


def _centroids(h1, h2, P):
    """Cartesian centroids (P, P, 2) of the pixels."""
    f = (np.arange(P) + 0.5) / P
    H1, H2 = np.meshgrid(f, f, indexing="ij")
    return H1[..., None] * h1 + H2[..., None] * h2


def _min_image_dist2(h1, h2, pts, centre):
    """Squared Cartesian distance from pts (..., 2) to the nearest periodic
    image of `centre` (2,), over the 9 neighbouring images."""
    best = None
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            c = centre + i * h1 + j * h2
            d2 = np.sum((pts - c) ** 2, axis=-1)
            best = d2 if best is None else np.minimum(best, d2)
    return best


def homogeneous_cell(P=16, lam=4.0, mu=1.5, rho=1.2, lattice="square", a=1.0):
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    return Cell(h1, h2, np.zeros((P, P), np.uint16), np.array([lam], float),
                np.array([mu], float), np.array([rho], float), "homogeneous", lattice)


def circle_cell(P=32, r=0.3, matrix=(4.0, 1.5, 1.2), inclusion=(110.0, 80.0, 7.8),
                lattice="square", a=1.0, name="circle"):
    """One circular inclusion of radius r*a centred in the cell; a pixel is
    in the inclusion iff its centroid lies within r*a of the cell centre
    (fractional (1/2, 1/2))."""
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    x = _centroids(h1, h2, P)
    centre = 0.5 * h1 + 0.5 * h2
    inside = _min_image_dist2(h1, h2, x, centre) <= (r * a) ** 2
    phase = inside.astype(np.uint16)
    lam, mu, rho = (np.array([matrix[i], inclusion[i]], float) for i in range(3))
    return Cell(h1, h2, phase, lam, mu, rho, name, lattice)


def bilayer_cell(P=64, n1=None, layer1=(4.0, 1.5, 1.2), layer2=(110.0, 80.0, 7.8), a=1.0):
    """Square cell of two layers normal to x1 (uniform along x2): pixels with
    p < n1 are phase 0, the rest phase 1.  Layer thicknesses are n1*a/P and
    (P-n1)*a/P, so the interfaces fall on pixel edges."""
    if n1 is None:
        n1 = P // 2
    h1, h2 = square(a)
    phase = np.zeros((P, P), np.uint16)
    phase[n1:, :] = 1
    lam, mu, rho = (np.array([layer1[i], layer2[i]], float) for i in range(3))
    return Cell(h1, h2, phase, lam, mu, rho, "bilayer", "square", {"n1": n1})


def _draw_props(rng, nphase, lam_rng=(2.0, 120.0), mu_rng=(1.0, 80.0), rho_rng=(1.0, 8.0)):
    """Per phase, in the order lambda, mu, rho (rows of a (nphase, 3) draw)."""
    u = rng.random((nphase, 3))
    lam = lam_rng[0] + (lam_rng[1] - lam_rng[0]) * u[:, 0]
    mu = mu_rng[0] + (mu_rng[1] - mu_rng[0]) * u[:, 1]
    rho = rho_rng[0] + (rho_rng[1] - rho_rng[0]) * u[:, 2]
    return lam, mu, rho


def voronoi_cell(P=256, nseeds=1132, seed=1310, lattice="square", a=1.0, name="voronoi"):
    """Periodic Voronoi tessellation: seeds uniform in the cell (fractional),
    each pixel takes the index of the nearest seed under the minimum-image
    Cartesian metric over the 9 neighbouring images."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    frac = rng.random((nseeds, 2))
    lam, mu, rho = _draw_props(rng, nseeds)
    pts = frac[:, :1] * h1 + frac[:, 1:] * h2
    images = np.concatenate([pts + i * h1 + j * h2 for i in (-1, 0, 1) for j in (-1, 0, 1)])
    tree = cKDTree(images)
    x = _centroids(h1, h2, P).reshape(-1, 2)
    _, idx = tree.query(x)
    phase = (idx % nseeds).astype(np.uint16).reshape(P, P)
    return Cell(h1, h2, phase, lam, mu, rho, name, lattice, {"seed": seed, "nseeds": nseeds})


def ellipse_cell(P=64, nellipse=3, seed=0, lattice="square", a=1.0, name="ellipses"):
    """A matrix (phase 0) holding `nellipse` random ellipses; ellipse i is
    phase i+1 and later ellipses cover earlier ones.  Centres uniform in the
    cell, semi-axes uniform in [0.05a, 0.25a], orientation uniform."""
    rng = np.random.default_rng(seed)
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    x = _centroids(h1, h2, P)
    phase = np.zeros((P, P), np.uint16)
    geo = rng.random((nellipse, 5))
    for i in range(nellipse):
        c = geo[i, 0] * h1 + geo[i, 1] * h2
        ax, bx = (0.05 + 0.2 * geo[i, 2]) * a, (0.05 + 0.2 * geo[i, 3]) * a
        th = np.pi * geo[i, 4]
        rot = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
        inside = np.zeros((P, P), bool)
        for s in (-1, 0, 1):
            for t in (-1, 0, 1):
                d = (x - (c + s * h1 + t * h2)) @ rot.T
                inside |= (d[..., 0] / ax) ** 2 + (d[..., 1] / bx) ** 2 <= 1.0
        phase[inside] = i + 1
    lam, mu, rho = _draw_props(rng, nellipse + 1)
    return Cell(h1, h2, phase, lam, mu, rho, name, lattice, {"seed": seed})


def steel_epoxy_hex_cell(P=64):
    """Steel cylinders (diameter 4 mm) in epoxy on a hexagonal lattice of
    constant 6.023 mm, SI units (Sec. "Example: hexagonal unit cell").
    Plane strain uses mu = C44 and lambda = C11 - 2 C44."""
    a = 6.023e-3
    steel = (264e9 - 2 * 81e9, 81e9, 7780.0)
    epoxy = (7.54e9 - 2 * 1.48e9, 1.48e9, 1142.0)
    return circle_cell(P, r=2.0e-3 / a, matrix=epoxy, inclusion=steel, lattice="hex",
                       a=a, name="steel_epoxy_hex")


# ---------------------------------------------------------------- meshes
@dataclass
class MeshCell:
    """A multi-phase 2-D unit cell given as a mesh (the paper's subdomains,
    Sec. III): each element carries its centroid in fractional coordinates
    (x = s h1 + t h2), its Cartesian area and a phase index."""

    h1: np.ndarray
    h2: np.ndarray
    centroid: np.ndarray      # (nel, 2) fractional (s, t)
    area: np.ndarray          # (nel,) Cartesian areas, summing to |det[h1; h2]|
    phase: np.ndarray         # (nel,) uint16
    lam: np.ndarray
    mu: np.ndarray
    rho: np.ndarray
    name: str = "mesh"
    lattice: str = "square"
    meta: dict = field(default_factory=dict)
    stiffness: np.ndarray = None   # optional (nphase, 3, 3) in-plane Voigt stiffness

    @property
    def nel(self) -> int:
        return int(self.phase.shape[0])

    @property
    def nphase(self) -> int:
        return int(self.lam.shape[0])

    def translated(self, ds: float, dt: float) -> "MeshCell":
        """The same mesh moved by (ds, dt) in fractional coordinates."""
        return MeshCell(self.h1.copy(), self.h2.copy(), self.centroid + np.array([ds, dt]),
                        self.area.copy(), self.phase.copy(), self.lam.copy(), self.mu.copy(),
                        self.rho.copy(), self.name + f"+({ds},{dt})", self.lattice,
                        dict(self.meta))

    def with_props(self, lam=None, mu=None, rho=None) -> "MeshCell":
        return MeshCell(self.h1.copy(), self.h2.copy(), self.centroid.copy(), self.area.copy(),
                        self.phase.copy(),
                        self.lam.copy() if lam is None else np.asarray(lam, np.float64),
                        self.mu.copy() if mu is None else np.asarray(mu, np.float64),
                        self.rho.copy() if rho is None else np.asarray(rho, np.float64),
                        self.name, self.lattice, dict(self.meta))


def jittered_triangles(n: int, jitter: float = 0.3, seed: int = 0):
    """A periodic triangulation of the unit torus in fractional coordinates:
    vertices ((i + dx)/n, (j + dy)/n) with dx, dy uniform in
    [-jitter/2, jitter/2] (one draw per vertex, shared by every triangle that
    uses it), each grid square split into two triangles along alternating
    diagonals.  Returns the vertices (2 n^2, 3, 2) of every triangle, with
    coordinates unwrapped so each triangle is contiguous.  jitter < 1/2 keeps
    every triangle positively oriented."""
    if not 0.0 <= jitter < 0.5:
        raise ValueError("jitter must lie in [0, 1/2)")
    rng = np.random.default_rng(seed)
    d = (rng.random((n, n, 2)) - 0.5) * jitter

    def v(i, j):
        return (np.array([i, j], float) + d[i % n, j % n]) / n

    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, e = v(i, j), v(i + 1, j), v(i + 1, j + 1), v(i, j + 1)
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, e)]
            else:
                tris += [(a, b, e), (b, c, e)]
    return np.array(tris)


def _mesh_from_triangles(tris, h1, h2):
    """Centroids (fractional) and Cartesian areas of triangles (nel, 3, 2)."""
    cen = tris.mean(axis=1)
    e1, e2 = tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]
    frac_area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    if (frac_area <= 0).any():
        raise ValueError("a triangle is not positively oriented")
    V = abs(h1[0] * h2[1] - h1[1] * h2[0])
    return cen, frac_area * V


def mesh_circle_cell(n=22, r=0.3, matrix=(4.0, 1.5, 1.2), inclusion=(110.0, 80.0, 7.8),
                     lattice="square", a=1.0, jitter=0.3, seed=0, name="mesh_circle"):
    """A circular inclusion on a jittered triangle mesh: an element is in the
    inclusion iff its centroid lies within r*a of the cell centre (minimum
    image), the rule of circle_cell."""
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    cen, area = _mesh_from_triangles(jittered_triangles(n, jitter, seed), h1, h2)
    x = cen[:, :1] * h1 + cen[:, 1:] * h2
    inside = _min_image_dist2(h1, h2, x, 0.5 * h1 + 0.5 * h2) <= (r * a) ** 2
    lam, mu, rho = (np.array([matrix[i], inclusion[i]], float) for i in range(3))
    return MeshCell(h1, h2, cen, area, inside.astype(np.uint16), lam, mu, rho, name, lattice,
                    {"n": n, "jitter": jitter, "seed": seed})


def mesh_voronoi_cell(n=24, nseeds=40, seed=5, lattice="square", a=1.0, jitter=0.3):
    """Periodic Voronoi phases (the rule of voronoi_cell) on a jittered
    triangle mesh; properties drawn per phase as there."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    h1, h2 = square(a) if lattice == "square" else hexagonal(a)
    frac = rng.random((nseeds, 2))
    lam, mu, rho = _draw_props(rng, nseeds)
    cen, area = _mesh_from_triangles(jittered_triangles(n, jitter, seed + 1), h1, h2)
    pts = frac[:, :1] * h1 + frac[:, 1:] * h2
    images = np.concatenate([pts + i * h1 + j * h2 for i in (-1, 0, 1) for j in (-1, 0, 1)])
    x = cen[:, :1] * h1 + cen[:, 1:] * h2
    _, idx = cKDTree(images).query(x)
    return MeshCell(h1, h2, cen, area, (idx % nseeds).astype(np.uint16), lam, mu, rho,
                    "mesh_voronoi", lattice, {"n": n, "seed": seed, "nseeds": nseeds})


def pixel_mesh(cell: Cell) -> MeshCell:
    """A pixel cell as a mesh of square elements (centroid = pixel centre,
    area = V / P^2): the same subdomains, so the same quadrature."""
    P = cell.P
    f = (np.arange(P) + 0.5) / P
    S, T = np.meshgrid(f, f, indexing="ij")
    V = abs(cell.h1[0] * cell.h2[1] - cell.h1[1] * cell.h2[0])
    return MeshCell(cell.h1.copy(), cell.h2.copy(), np.stack([S.ravel(), T.ravel()], axis=1),
                    np.full(P * P, V / (P * P)), cell.phase.reshape(-1).astype(np.uint16),
                    cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), cell.name + "_as_mesh",
                    cell.lattice)


def steel_epoxy_hex_mesh(n=22):
    """The hexagonal steel/epoxy cell (Sec. "Example: hexagonal unit cell")
    on a jittered triangle mesh of 2 n^2 elements (968 for n = 22, the size
    of the paper's 964-triangle mesh)."""
    a = 6.023e-3
    steel = (264e9 - 2 * 81e9, 81e9, 7780.0)
    epoxy = (7.54e9 - 2 * 1.48e9, 1.48e9, 1142.0)
    return mesh_circle_cell(n, r=2.0e-3 / a, matrix=epoxy, inclusion=steel, lattice="hex", a=a,
                            name="steel_epoxy_hex_mesh")


# ---------------------------------------------------------------- anisotropy
# In-plane Voigt notation: sigma = (s11, s22, s12), strain = (e11, e22, 2 e12),
# sigma = C strain with C symmetric positive definite (plane strain).
def isotropic_stiffness(lam, mu):
    """(n, 3, 3) Voigt stiffness of isotropic phases."""
    lam, mu = np.atleast_1d(np.asarray(lam, float)), np.atleast_1d(np.asarray(mu, float))
    C = np.zeros((lam.shape[0], 3, 3))
    C[:, 0, 0] = C[:, 1, 1] = lam + 2 * mu
    C[:, 0, 1] = C[:, 1, 0] = lam
    C[:, 2, 2] = mu
    return C


def rotate_stiffness(C, theta):
    """Voigt stiffness (3, 3) of a material turned by theta in the plane."""
    c, s = np.cos(theta), np.sin(theta)
    T = np.array([[c * c, s * s, 2 * s * c], [s * s, c * c, -2 * s * c],
                  [-s * c, s * c, c * c - s * s]])          # sigma' = T sigma
    R = np.diag([1.0, 1.0, 2.0])                            # strain Voigt <-> tensor
    Te = R @ T @ np.linalg.inv(R)                           # strain' = Te strain
    return T @ np.asarray(C, float) @ np.linalg.inv(Te)     # sigma' = T C Te^-1 strain'


def rotated_orthotropic(c11, c22, c12, c66, theta):
    """Voigt stiffness of an orthotropic material whose axes are turned by
    theta in the plane: C' = T^-T C T^-1 with the stress transformation T of
    a rotation by theta."""
    return rotate_stiffness(np.array([[c11, c12, 0.0], [c12, c22, 0.0], [0.0, 0.0, c66]]), theta)


def with_stiffness(cell, C):
    """A copy of a pixel or mesh cell with per-phase Voigt stiffness C (nphase, 3, 3)."""
    import copy
    out = copy.copy(cell)
    out.stiffness = np.asarray(C, float).copy()
    return out


def anisotropic_cell(cell, seed=0):
    """The cell with every phase replaced by a rotated orthotropic material:
    c11, c22 ~ U[20, 200], c66 ~ U[5, 60], c12 ~ U[0, 0.4 sqrt(c11 c22)],
    orientation ~ U[0, pi); densities kept."""
    rng = np.random.default_rng(seed)
    C = []
    for _ in range(cell.nphase):
        u = rng.random(5)
        c11, c22 = 20 + 180 * u[0], 20 + 180 * u[1]
        c66 = 5 + 55 * u[2]
        c12 = 0.4 * np.sqrt(c11 * c22) * u[3]
        C.append(rotated_orthotropic(c11, c22, c12, c66, np.pi * u[4]))
    return with_stiffness(cell, np.array(C))


# ---------------------------------------------------------------- 3-D cells
@dataclass
class Cell3:
    """A voxelated multi-phase 3-D unit cell: phase[p, q, r] along h1, h2, h3,
    voxel (p, q, r) centred at ((p + 1/2)/P, (q + 1/2)/P, (r + 1/2)/P) in
    fractional coordinates."""

    h1: np.ndarray            # (3,)
    h2: np.ndarray
    h3: np.ndarray
    phase: np.ndarray         # (P, P, P) uint16
    lam: np.ndarray
    mu: np.ndarray
    rho: np.ndarray
    name: str = "cell3"
    lattice: str = "cubic"
    meta: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return int(self.phase.shape[0])

    @property
    def nphase(self) -> int:
        return int(self.lam.shape[0])


def _cubic(a=1.0):
    return np.array([a, 0.0, 0.0]), np.array([0.0, a, 0.0]), np.array([0.0, 0.0, a])


def _voxel_centres(h1, h2, h3, P):
    f = (np.arange(P) + 0.5) / P
    S, T, U = np.meshgrid(f, f, f, indexing="ij")
    return S[..., None] * h1 + T[..., None] * h2 + U[..., None] * h3


def sphere_cell3(P=16, r=0.3, matrix=(4.0, 1.5, 1.2), inclusion=(110.0, 80.0, 7.8), a=1.0):
    """A spherical inclusion of radius r*a at the centre of a simple cubic
    cell: a voxel is inside iff its centre lies within r*a of the centre."""
    h1, h2, h3 = _cubic(a)
    x = _voxel_centres(h1, h2, h3, P)
    c = 0.5 * (h1 + h2 + h3)
    inside = np.sum((x - c) ** 2, axis=-1) <= (r * a) ** 2
    lam, mu, rho = (np.array([matrix[i], inclusion[i]], float) for i in range(3))
    return Cell3(h1, h2, h3, inside.astype(np.uint16), lam, mu, rho, "sphere")


def voronoi_cell3(P=16, nseeds=12, seed=3, a=1.0):
    """Periodic 3-D Voronoi phases (nearest seed over the 27 periodic images)
    on a simple cubic cell; properties drawn per phase as in 2-D."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    h1, h2, h3 = _cubic(a)
    frac = rng.random((nseeds, 3))
    lam, mu, rho = _draw_props(rng, nseeds)
    pts = frac @ np.array([h1, h2, h3])
    images = np.concatenate([pts + i * h1 + j * h2 + k * h3
                             for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)])
    x = _voxel_centres(h1, h2, h3, P).reshape(-1, 3)
    _, idx = cKDTree(images).query(x)
    return Cell3(h1, h2, h3, (idx % nseeds).astype(np.uint16).reshape(P, P, P), lam, mu, rho,
                 "voronoi3", "cubic", {"seed": seed})


def extruded_cell3(cell: Cell, a3=1.0):
    """A 2-D pixel cell extruded along x3 (uniform in the third direction),
    h3 = (0, 0, a3), P voxels along h3."""
    h1 = np.array([cell.h1[0], cell.h1[1], 0.0])
    h2 = np.array([cell.h2[0], cell.h2[1], 0.0])
    h3 = np.array([0.0, 0.0, a3])
    P = cell.P
    ph = np.repeat(cell.phase[:, :, None], P, axis=2).astype(np.uint16)
    return Cell3(h1, h2, h3, ph, cell.lam.copy(), cell.mu.copy(), cell.rho.copy(),
                 cell.name + "_extruded", "tetragonal")


def ibz_path_cubic(nk: int, a=1.0) -> np.ndarray:
    """nk fractional wavevectors (nk, 3) uniform in arc length along
    Gamma-X-M-R-Gamma of the simple cubic lattice (first and last Gamma)."""
    corners = np.array([(0, 0, 0), (0.5, 0, 0), (0.5, 0.5, 0), (0.5, 0.5, 0.5), (0, 0, 0)],
                       float)
    kc = corners * (2 * np.pi / a)
    seg = np.linalg.norm(np.diff(kc, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    out = np.empty((nk, 3))
    for i in range(nk):
        s_ = cum[-1] * i / (nk - 1)
        j = min(int(np.searchsorted(cum, s_, side="right")) - 1, len(seg) - 1)
        t = 0.0 if seg[j] == 0 else (s_ - cum[j]) / seg[j]
        out[i] = corners[j] + min(max(t, 0.0), 1.0) * (corners[j + 1] - corners[j])
    return out


# High-symmetry points in fractional coordinates Q (k = Q1 q1 + Q2 q2).
_PATHS = {
    "square": [(0.0, 0.0), (0.5, 0.0), (0.5, 0.5), (0.0, 0.0)],          # G-X-M-G
    "hex": [(0.0, 0.0), (0.5, 0.0), (2.0 / 3.0, 1.0 / 3.0), (0.0, 0.0)],  # G-M-K-G
}


def ibz_path(lattice: str, nk: int, h1=None, h2=None) -> np.ndarray:
    """nk fractional wavevectors (nk, 2) uniform in Cartesian arc length
    along the closed IBZ boundary; the first and last are both Gamma."""
    if nk < 2:
        raise ValueError("nk must be >= 2")
    if h1 is None:
        h1, h2 = square() if lattice == "square" else hexagonal()
    A = np.array([h1, h2], float)
    qmat = 2.0 * np.pi * np.linalg.inv(A)      # column i is q^i
    corners = np.array(_PATHS[lattice], float)
    kc = corners @ qmat.T
    seg = np.linalg.norm(np.diff(kc, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    out = np.empty((nk, 2))
    for i in range(nk):
        s = cum[-1] * i / (nk - 1)
        j = min(int(np.searchsorted(cum, s, side="right")) - 1, len(seg) - 1)
        t = 0.0 if seg[j] == 0 else (s - cum[j]) / seg[j]
        out[i] = corners[j] + min(max(t, 0.0), 1.0) * (corners[j + 1] - corners[j])
    return out


def config0():
    """32x32 circle r=0.3a, square a=1, M=3, 30 k on G-X-M-G, 8 bands."""
    cell = circle_cell(32, 0.3)
    return dict(cell=cell, M=3, Q=ibz_path("square", 30), nbands=8)


def config1():
    """256x256 periodic Voronoi with 1132 phases (seed 1310), square, M=10,
    90 k on G-X-M-G, 18 bands."""
    cell = voronoi_cell(256, 1132, 1310)
    return dict(cell=cell, M=10, Q=ibz_path("square", 90), nbands=18)


def c3_style_cell(seed: int, P: int = 64, tag: str = "c3"):
    """A cell of the ragged-batch style from one seed: square or hexagonal
    lattice with probability 1/2; half ellipse maps, half Voronoi; 2..16
    phases; truncation M uniform in {5..8}; 30 k on its lattice's path;
    10 bands."""
    rng = np.random.default_rng(seed)
    lattice = "square" if rng.random() < 0.5 else "hex"
    nphase = int(rng.integers(2, 17))
    M = int(rng.integers(5, 9))
    sub = int(rng.integers(0, 2**31 - 1))
    if rng.random() < 0.5:
        cell = ellipse_cell(P, nphase - 1, sub, lattice, name=f"{tag}_{seed}_ellipses")
    else:
        cell = voronoi_cell(P, nphase, sub, lattice, name=f"{tag}_{seed}_voronoi")
    return dict(cell=cell, M=M, Q=ibz_path(lattice, 30, cell.h1, cell.h2), nbands=10)


def config3_cell(i: int, P: int = 64):
    """Cell i of the 4096-cell ragged batch: seed 6380+i."""
    return c3_style_cell(6380 + i, P, tag=f"c3_{i}")


def config4_train_cell(i: int):
    """Training cell i of the learned warm start: seed 10^6 + i."""
    return c3_style_cell(1_000_000 + i, tag="c4train")


def config4_eval_cell(i: int):
    """Held-out evaluation cell i of the learned warm start: seed 2 10^6 + i."""
    return c3_style_cell(2_000_000 + i, tag="c4eval")


CONFIGS = {"c0": config0, "c1": config1}
