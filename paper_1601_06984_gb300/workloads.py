"""Seeded synthetic workloads for the multilevel lattice Boltzmann path.

This module only *generates inputs*: octree meshes as treeID lists, the
Taylor-Green closed-form initial fields, seeded perturbations and body forces.
It holds none of the method's arithmetic (no equilibrium, collision,
interpolation or streaming), so both the CUDA library and the CPU oracle can be
fed from it without sharing any of the method.

Mesh geometry follows the paper's workloads (arXiv:1601.06984): the periodic
Taylor-Green vortex of Sec. 4.1 (Eq. tgv), the 2D cylinder channel of Sec. 4.2
and the sphere of Sec. 4.3, resized to the synthetic configurations listed in
the project documentation (central refined blocks, nested refinement boxes,
half-way bounce-back obstacles).

treeIDs (Sec. 3.1): level L holds ids off(L) .. off(L+1)-1 with
off(L) = (2^{dL}-1)/(2^d-1); the remainder is the z-curve (Morton) index of the
element at that level with the x bit lowest, then y, then z.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_PERIODIC, BC_WALL, BC_VELOCITY_IN, BC_PRESSURE_OUT = 0, 1, 2, 3
TIME_LINEAR, TIME_TWO_LAYER, TIME_DIFFUSIVE = 0, 1, 2
SEED = 20160127


# ----------------------------------------------------------------- treeIDs
def level_offset(L: int, d: int) -> int:
    return ((1 << (d * L)) - 1) // ((1 << d) - 1)


def _spread(v: np.ndarray, d: int) -> np.ndarray:
    """Insert d-1 zero bits between the bits of v (v < 2^21 for d=3, < 2^31 for d=2)."""
    v = v.astype(np.uint64)
    if d == 2:
        for shift, mask in ((16, 0x0000FFFF0000FFFF), (8, 0x00FF00FF00FF00FF), (4, 0x0F0F0F0F0F0F0F0F),
                            (2, 0x3333333333333333), (1, 0x5555555555555555)):
            v = (v | (v << np.uint64(shift))) & np.uint64(mask)
    else:
        for shift, mask in ((32, 0x001F00000000FFFF), (16, 0x001F0000FF0000FF), (8, 0x100F00F00F00F00F),
                            (4, 0x10C30C30C30C30C3), (2, 0x1249249249249249)):
            v = (v | (v << np.uint64(shift))) & np.uint64(mask)
    return v


def morton(coords: np.ndarray, L: int, d: int) -> np.ndarray:
    """Interleave the bits of integer coordinates [n, d] at level L (x bit lowest)."""
    coords = np.asarray(coords, dtype=np.int64)
    if coords.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    m = np.zeros(coords.shape[0], dtype=np.uint64)
    for a in range(d):
        m |= _spread(coords[:, a], d) << np.uint64(a)
    return m.astype(np.int64)


def tree_ids(coords: np.ndarray, L: int, d: int) -> np.ndarray:
    return morton(coords, L, d) + np.int64(level_offset(L, d))


@dataclasses.dataclass
class Mesh:
    """A leaf list: treeID and level per element, plus the integer coordinates
    (at the element's own level) kept for building input fields."""

    d: int
    extent: tuple          # domain box in coarsest-level elements
    bc: tuple              # per face: x-, x+, y-, y+, z-, z+
    tree_ids: np.ndarray   # int64 [n]
    levels: np.ndarray     # int8 [n]
    coords: np.ndarray     # int64 [n, d]
    lmin: int

    @property
    def n(self) -> int:
        return int(self.tree_ids.shape[0])

    def centres(self) -> np.ndarray:
        """Element centres in coarsest-level lattice units, [n, d]."""
        scale = np.ldexp(1.0, -(self.levels.astype(np.int64) - self.lmin))
        return (self.coords + 0.5) * scale[:, None]

    def level_counts(self) -> dict:
        lv, cnt = np.unique(self.levels, return_counts=True)
        return {int(a): int(b) for a, b in zip(lv, cnt)}

    def updates_per_coarse_step(self, substeps: int = 2) -> int:
        """Fine-substep weighted element updates, sum_L N_L m^{L-Lmin} (the
        workload weights of Sec. 3.1, Eq. weight), m = 2 fine substeps per
        coarse step (acoustic scaling) or 4 (diffusive scaling)."""
        return int(sum(c * substeps ** (lv - self.lmin) for lv, c in self.level_counts().items()))


def _grid(lo, hi):
    axes = [np.arange(a, b, dtype=np.int64) for a, b in zip(lo, hi)]
    g = np.meshgrid(*axes, indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


def nested_boxes(d, lmin, extent, boxes, bc, solid=None):
    """Mesh of nested refinement boxes.  boxes[k] = (lo, hi) of the level
    lmin+k+1 region, in level lmin+k+1 cells (each box must be a union of its
    parent level's cells and lie inside the previous box).  solid(level,
    centres_in_finest_units) -> bool mask of cells to drop (obstacles)."""
    nlev = len(boxes) + 1
    finest = lmin + nlev - 1
    ids, lvls, crd = [], [], []
    regions = [((0,) * d, tuple(extent))] + [tuple(map(tuple, b)) for b in boxes]
    for k in range(nlev):
        L = lmin + k
        lo, hi = regions[k]
        c = _grid(lo, hi)
        if k + 1 < nlev:
            clo = np.array(regions[k + 1][0]) // 2
            chi = np.array(regions[k + 1][1]) // 2
            assert np.all(np.array(regions[k + 1][0]) % 2 == 0) and np.all(np.array(regions[k + 1][1]) % 2 == 0)
            inside = np.all((c >= clo) & (c < chi), axis=1)
            c = c[~inside]
        if solid is not None:
            cen = (c + 0.5) * float(1 << (finest - L))
            c = c[~solid(L, cen)]
        ids.append(tree_ids(c, L, d))
        lvls.append(np.full(c.shape[0], L, dtype=np.int8))
        crd.append(c)
    return Mesh(d=d, extent=tuple(extent), bc=tuple(bc), tree_ids=np.concatenate(ids),
                levels=np.concatenate(lvls), coords=np.concatenate(crd), lmin=lmin)


def uniform(d, L, extent, bc, solid=None):
    return nested_boxes(d, L, extent, [], bc, solid)


def two_level_block(d, n, lo, hi, bc=None):
    """Periodic n^d coarse box (n a power of two) with the coarse block
    [lo, hi)^d refined once."""
    L = int(round(math.log2(n)))
    assert 1 << L == n
    bc = bc or (BC_PERIODIC,) * (2 * d)
    return nested_boxes(d, L, (n,) * d, [((2 * lo,) * d, (2 * hi,) * d)], bc)


def half_refined_2d(n):
    """The paper's Taylor-Green convergence layout (Sec. 4.1): left half of the
    periodic square at level L (n = 2^L cells across), right half one level
    finer."""
    L = int(round(math.log2(n)))
    coarse = _grid((0, 0), (n // 2, n))
    fine = _grid((n, 0), (2 * n, 2 * n))
    ids = np.concatenate([tree_ids(coarse, L, 2), tree_ids(fine, L + 1, 2)])
    lv = np.concatenate([np.full(len(coarse), L, np.int8), np.full(len(fine), L + 1, np.int8)])
    return Mesh(d=2, extent=(n, n), bc=(BC_PERIODIC,) * 4, tree_ids=ids, levels=lv,
                coords=np.concatenate([coarse, fine]), lmin=L)


def shuffled(mesh: Mesh, seed: int = SEED) -> Mesh:
    """Same mesh with its elements in a seeded random order (the user order is
    arbitrary; the library must not depend on it)."""
    p = np.random.default_rng(seed).permutation(mesh.n)
    return dataclasses.replace(mesh, tree_ids=mesh.tree_ids[p], levels=mesh.levels[p], coords=mesh.coords[p])


# ----------------------------------------------------------------- configs
def config_tgv2d():
    """D2Q9 two-level Taylor-Green: periodic 32x32 coarse, central 16x16 coarse
    block refined to 32x32 fine."""
    return two_level_block(2, 32, 8, 24)


def config_tgv3d(n=64):
    """D3Q19 two-level Taylor-Green extruded in z: periodic n^3 coarse with the
    central (n/2)^3 block refined (n=64: 64^3 coarse, 32^3 block -> 64^3 fine)."""
    return two_level_block(3, n, n // 4, 3 * n // 4)


def config_cylinder(D=40, walls=True):
    """D2Q9 cylinder channel 40D x 20D; 4 levels from dx=D/5 to D/40 with
    nested boxes [5,25]x[5,15]D, [7.5,17.5]x[7.5,12.5]D, [8.5,13.5]x[8.75,11.25]D;
    cylinder of diameter D (finest cells) at (10D, 10D); velocity inlet at
    x-, pressure outlet at x+, walls (or periodic) on y."""
    assert D == 40, "the configured cylinder has D = 40 finest cells"
    nx, ny = 200, 100
    lmin = int(math.ceil(math.log2(max(nx, ny))))

    def box(lo_d, hi_d, k):
        # level lmin+k cell = D / (5 * 2^k)
        cells_per_d = 5 * (1 << k)
        return (tuple(int(round(v * cells_per_d)) for v in lo_d),
                tuple(int(round(v * cells_per_d)) for v in hi_d))

    boxes = [box((5, 5), (25, 15), 1), box((7.5, 7.5), (17.5, 12.5), 2),
             box((8.5, 8.75), (13.5, 11.25), 3)]
    finest_cells_per_d = 40
    cx = cy = 10 * finest_cells_per_d
    r = 0.5 * finest_cells_per_d

    def solid(L, cen):
        return (cen[:, 0] - cx) ** 2 + (cen[:, 1] - cy) ** 2 < r * r

    lat = BC_WALL if walls else BC_PERIODIC
    bc = (BC_VELOCITY_IN, BC_PRESSURE_OUT, lat, lat)
    return nested_boxes(2, lmin, (nx, ny), boxes, bc, solid)


def config_cylinder_schafer(D=40):
    """The paper's cylinder geometry (Sec. 4.2, the Schaefer-Turek channel):
    channel 2.2 x 0.41 with a cylinder of diameter 0.1 centred at (0.2, 0.2),
    in units where D is the cylinder diameter in finest cells.  Two levels: the
    bulk at dx = 2/D of a diameter, and one refined box [0.05, 0.35]^2 around
    the cylinder (the paper's ring of thickness 0.1 around it).  Velocity inlet
    at x-, pressure outlet at x+, walls on y.  D must be a multiple of 20."""
    assert D % 20 == 0, "D must be a multiple of 20 (whole cells for H = 4.1 D on the coarse level)"
    nx, ny = 22 * D // 2, 41 * D // 20          # coarse cells
    lmin = int(math.ceil(math.log2(max(nx, ny))))
    lo, hi = D // 2, 7 * D // 2                 # refined box [0.05, 0.35] in fine cells
    cx = cy = 2 * D                             # centre (0.2, 0.2) in fine cells
    r = 0.5 * D

    def solid(L, cen):
        return (cen[:, 0] - cx) ** 2 + (cen[:, 1] - cy) ** 2 < r * r

    return nested_boxes(2, lmin, (nx, ny), [((lo, lo), (hi, hi))],
                        (BC_VELOCITY_IN, BC_PRESSURE_OUT, BC_WALL, BC_WALL), solid)


_C27 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                 [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
                 [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1], [1, 1, 1], [-1, -1, -1],
                 [1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, -1], [-1, 1, 1], [1, -1, -1]])
_C9 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [1, 1, 0], [-1, -1, 0],
                [1, -1, 0], [-1, 1, 0]])


def wall_distance_ball(mesh: Mesh, elem, dirs, centre, radius, Q):
    """Geometry input of the interpolated bounce-back: for each link (element,
    direction i with x - c_i inside the ball), the fraction q in (0, 1] of the
    link from the element centre x to the surface, so that the wall lies at
    x - q c_i.  A circle in 2D, a sphere in 3D; centre and radius in finest
    cells; directions in the library's order."""
    c = (_C9 if Q == 9 else _C27)[np.asarray(dirs, dtype=np.int64)][:, :mesh.d].astype(float)
    elem = np.asarray(elem, dtype=np.int64)
    h = np.ldexp(1.0, int(mesh.levels.max()) - mesh.levels[elem].astype(np.int64))   # cell size, finest units
    x = (mesh.coords[elem].astype(float) + 0.5) * h[:, None]
    p = x - np.asarray(centre, float)[: mesh.d]
    v = -c * h[:, None]                         # from x toward x - c_i
    a = (v * v).sum(1)
    b = (p * v).sum(1)
    cc = (p * p).sum(1) - radius * radius
    q = (-b - np.sqrt(np.maximum(b * b - a * cc, 0.0))) / a
    return np.clip(q, 1e-6, 1.0)


def config_sphere(scale=1):
    """D3Q19 sphere: box 32D x 16D x 16D, sphere diameter D = 64/scale finest
    cells at (8D,8D,8D), 5 levels from D/4 to D/64 with nested boxes
    [2,28]x[2,14]^2 D, [4,24]x[3.5,12.5]^2 D, [5,20]x[4.5,11.5]^2 D,
    [6,16]x[5.5,10.5]^2 D; velocity inlet x-, pressure outlet x+, periodic
    lateral faces.  scale>1 shrinks every length by that factor (reduced
    cases for parity tests)."""
    cpd0 = 4 // 1  # coarse cells per D
    nx, ny = 32 * cpd0, 16 * cpd0
    # with scale>1 the coarse grid shrinks but keeps 5 levels
    nx //= scale
    ny //= scale
    lmin = int(math.ceil(math.log2(nx)))

    def box(lo_d, hi_d, k):
        cells_per_d = cpd0 * (1 << k) / scale
        lo = tuple(int(round(v * cells_per_d)) for v in lo_d)
        hi = tuple(int(round(v * cells_per_d)) for v in hi_d)
        return lo, hi

    boxes = [box((2, 2, 2), (28, 14, 14), 1), box((4, 3.5, 3.5), (24, 12.5, 12.5), 2),
             box((5, 4.5, 4.5), (20, 11.5, 11.5), 3), box((6, 5.5, 5.5), (16, 10.5, 10.5), 4)]
    Dfin = 64 / scale
    c = 8 * Dfin
    r = 0.5 * Dfin

    def solid(L, cen):
        return ((cen - c) ** 2).sum(axis=1) < r * r

    bc = (BC_VELOCITY_IN, BC_PRESSURE_OUT, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return nested_boxes(3, lmin, (nx, ny, ny), boxes, bc, solid)


# ----------------------------------------------------------------- fields
def tgv_fields(mesh: Mesh, u0: float, rho0: float = 1.0, t: float = 0.0, nu: float = 0.0,
               n_period: float | None = None):
    """Taylor-Green vortex closed form (Sec. 4.1, Eq. tgv) at the element
    centres, extruded in z for 3D.  Wavenumber k = 2 pi / N with N the periodic
    box length in coarsest-level cells; lattice units of the coarsest level for
    positions, time and viscosity.  Returns rho [n], u [n, d] and S [n, nS] with
    S in each element's own level lattice units (S_level = S_coarse / 2^{L-Lmin})
    and nS = 3 (xx, yy, xy) or 6 (xx, yy, zz, xy, yz, xz)."""
    N = n_period or mesh.extent[0]
    k = 2.0 * math.pi / N
    x = mesh.centres()
    X, Y = k * x[:, 0], k * x[:, 1]
    decay = math.exp(-2.0 * nu * k * k * t)
    ux = -u0 * np.cos(X) * np.sin(Y) * decay
    uy = u0 * np.sin(X) * np.cos(Y) * decay
    # p = p0 - rho u0^2/4 (cos 2x + cos 2y) e^{-2t/tD}; rho = rho0 + p'/c_s^2
    rho = rho0 - 3.0 * rho0 * u0 * u0 / 4.0 * (np.cos(2 * X) + np.cos(2 * Y)) * decay * decay
    sxx = u0 * k * np.sin(X) * np.sin(Y) * decay
    n = mesh.n
    lvl_scale = np.ldexp(1.0, -(mesh.levels.astype(np.int64) - mesh.lmin))
    if mesh.d == 2:
        u = np.stack([ux, uy], axis=1)
        S = np.stack([sxx, -sxx, np.zeros(n)], axis=1)
    else:
        u = np.stack([ux, uy, np.zeros(n)], axis=1)
        S = np.stack([sxx, -sxx, np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)], axis=1)
    S = S * lvl_scale[:, None]
    return rho, u, S


def diffusive_units(mesh: Mesh, rho, u, S, rho0: float = 1.0):
    """Fields given as the generators above return them (rho and u in the
    coarsest level's lattice units, S in each level's units of acoustic
    scaling, dt ~ dx) converted to each level's lattice units of diffusive
    scaling (dt ~ dx^2): per level below the coarsest, velocity / 2, strain
    rate / 4 (one more factor 1/2 here) and density deviation / 4."""
    l = (mesh.levels.astype(np.int64) - mesh.lmin)
    h = np.ldexp(1.0, -l)
    rho = rho0 + (np.asarray(rho) - rho0) * h * h
    u = np.asarray(u) * h[:, None]
    S = None if S is None else np.asarray(S) * h[:, None]
    return rho, u, S


def uniform_fields(mesh: Mesh, rho0=1.0, u=None):
    n = mesh.n
    uu = np.zeros((n, mesh.d)) if u is None else np.tile(np.asarray(u, float)[: mesh.d], (n, 1))
    ns = 3 if mesh.d == 2 else 6
    return np.full(n, rho0), uu, np.zeros((n, ns))


# ----------------------------------------------------------------- random numbers
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014), vectorised on uint64."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def counter_uniform(tree_ids: np.ndarray, ncomp: int, seed: int, stream: int = 0) -> np.ndarray:
    """U(-1, 1) numbers keyed by (treeID, component, seed, stream): independent
    of element order.  Returns [n, ncomp]."""
    t = np.asarray(tree_ids, dtype=np.int64).astype(np.uint64)
    comp = np.arange(ncomp, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = (t[:, None] * np.uint64(0x100000001B3) + comp[None, :] * np.uint64(0x9E3779B1)
               + np.uint64(seed) * np.uint64(0xD6E8FEB86659FD93) + np.uint64(stream)) & _M64
    r = splitmix64(splitmix64(key))
    return ((r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))) * 2.0 - 1.0


def pdf_perturbation(mesh: Mesh, Q: int, amplitude: float = 1e-6, seed: int = SEED) -> np.ndarray:
    """amplitude * U(-1,1) per element and discrete velocity, [n, Q]."""
    return amplitude * counter_uniform(mesh.tree_ids, Q, seed, stream=1)


def gaussian_force(mesh: Mesh, sigma: float = 1e-6, seed: int = SEED) -> np.ndarray:
    """N(0, sigma^2) body force per component per element (Box-Muller on two
    counter-based uniforms), [n, d]."""
    u1 = 0.5 * (counter_uniform(mesh.tree_ids, mesh.d, seed, stream=2) + 1.0)
    u2 = 0.5 * (counter_uniform(mesh.tree_ids, mesh.d, seed, stream=3) + 1.0)
    u1 = np.clip(u1, 1e-300, 1.0)
    return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def random_direction(shape, seed: int, stream: int) -> np.ndarray:
    """Seeded direction for directional-derivative checks."""
    return np.random.default_rng([seed, stream]).standard_normal(shape)


def config_sphere_small():
    """Reduced sphere-like case for oracle parity (about 17k elements): box
    24 x 12 x 12 coarse cells, three levels with nested boxes
    [4,20)x[2,10)^2 (coarse cells) and [7,15)x[4,8)^2 (coarse cells), a sphere
    of diameter 8 finest cells at the finest box centre, velocity inlet x-,
    pressure outlet x+, periodic lateral faces."""
    boxes = [((8, 4, 4), (40, 20, 20)), ((28, 16, 16), (60, 32, 32))]

    def solid(L, cen):
        return ((cen - np.array([44.0, 24.0, 24.0])) ** 2).sum(axis=1) < 16.0

    bc = (BC_VELOCITY_IN, BC_PRESSURE_OUT, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return nested_boxes(3, 5, (24, 12, 12), boxes, bc, solid)


def config_sphere_5level_small():
    """Reduced five-level D3Q19 sphere-like case for oracle parity (about 17k
    elements): channel 16 x 12 x 12 coarse cells, velocity inlet x-, pressure
    outlet x+, periodic lateral faces, four nested refinement boxes (each in
    its own level's cells) [8,24)x[4,20)^2, [24,40)x[16,32)^2,
    [56,72)x[40,56)^2 and [120,136)x[88,104)^2 (every box 4 cells of its
    parent level inside the previous one), and a sphere of diameter 5 finest
    cells at the finest box centre.  The same recursion depth as the full
    sphere workload (four interfaces) at a size the oracle runs in seconds."""
    boxes = [((8, 4, 4), (24, 20, 20)), ((24, 16, 16), (40, 32, 32)), ((56, 40, 40), (72, 56, 56)),
             ((120, 88, 88), (136, 104, 104))]

    def solid(L, cen):
        return ((cen - np.array([128.0, 96.0, 96.0])) ** 2).sum(axis=1) < 6.25

    bc = (BC_VELOCITY_IN, BC_PRESSURE_OUT, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return nested_boxes(3, 4, (16, 12, 12), boxes, bc, solid)


def omega_coarse_from_finest(omega_f: float, nlev: int) -> float:
    """Coarsest-level relaxation rate for a finest-level one under
    1/omega_f - 1/2 = m (1/omega_c - 1/2), m = 2 per level."""
    return 1.0 / (0.5 + (1.0 / omega_f - 0.5) / (1 << (nlev - 1)))


def omega_for_re(U: float, D: float, Re: float) -> float:
    """Finest-level relaxation rate for Re = U D / nu (lattice units)."""
    return 1.0 / (3.0 * U * D / Re + 0.5)
