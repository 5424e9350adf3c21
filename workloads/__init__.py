"""Seeded, synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds problem descriptions (mesh sizes, material phases, boundary
conditions, time-integration parameters), surface triangulations (icospheres and
boxes standing in for the CAD surfaces of the paper's Section 3) and seeded random
states.  It contains none of the method's arithmetic: no shape functions, no
residuals, no solvers, no distances or ray casts.  Both the CUDA path and the
oracle read these plain descriptions and implement the method independently.

Workloads (Section 5-6 of the paper, re-cast on uniform Q1 hexahedra):
  cavity16  - 3D lid-driven cavity, unit cube, 16^3 hexes, elastic sphere R=0.2
              at (0.6,0.5,0.5) (the rotating-sphere case of Section 5.2 with the
              material values of the 2D disk case: rho=1, mu=0.01, mu_L=0.1).
  cavity64  - the same cavity at 64^3 hexes (274,625 nodes).
  falling   - sphere (R=0.15, rho=2, mu_L=1e3) above an elastic block
              (rho=1.5, mu_L=50) in a 1x1x2 box, 96x96x192 hexes, gravity -9.81 z
              (a synthetic variant of Section 5.3).
  shipice   - water/air, a box hull and 8 seeded ice boxes, 4x2x1 box on
              256x128x64 hexes, 11 phase indicators (a synthetic variant of
              Section 6).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

Vec3 = Tuple[float, float, float]

# Face order used everywhere: x-, x+, y-, y+, z-, z+
FACES = ("x-", "x+", "y-", "y+", "z-", "z+")

# Boundary kinds for the velocity on a face.
BC_NATURAL = 0   # no Dirichlet condition (traction-free / outflow)
BC_DIRICHLET = 1  # prescribed velocity


@dataclass
class Phase:
    """One material phase: density, dynamic viscosity, shear modulus (0 for fluids)."""
    rho: float
    mu: float
    mu_L: float = 0.0
    solid: bool = False


@dataclass
class FaceBC:
    kind: int = BC_DIRICHLET
    vel: Vec3 = (0.0, 0.0, 0.0)
    priority: int = 0  # where Dirichlet faces meet, the highest priority wins


@dataclass
class MeshDesc:
    """Problem description on the uniform box [0,lx]x[0,ly]x[0,lz]."""
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    phases: List[Phase]
    gravity: Vec3 = (0.0, 0.0, 0.0)
    eps: float = 0.0
    eta: float = 0.2
    dt: float = 0.01
    rho_inf: float = 0.0
    c_i: float = 36.0
    faces: List[FaceBC] = field(default_factory=lambda: [FaceBC() for _ in range(6)])
    # interior box with prescribed velocity: (lo, hi, vel) or None
    prescribed_box: Optional[Tuple[Vec3, Vec3, Vec3]] = None
    pin_node: int = 0  # node whose pressure is fixed to 0; -1 for none

    @property
    def nn(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def ne(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_phase(self) -> int:
        return len(self.phases)

    @property
    def solid_phases(self) -> List[int]:
        return [i for i, p in enumerate(self.phases) if p.solid]

    @property
    def n_solid(self) -> int:
        return len(self.solid_phases)

    @property
    def ncomp(self) -> int:
        """Unknowns per node: v(3), p, phi(N), B(6 per solid)."""
        return 4 + self.n_phase + 6 * self.n_solid

    @property
    def h(self) -> Vec3:
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)


# ---------------------------------------------------------------- surfaces

@dataclass
class Surface:
    """Triangulated closed surface: vertices (n_v,3) float64, triangles (n_t,3) int32."""
    verts: np.ndarray
    tris: np.ndarray


def icosphere(center: Vec3, radius: float, h_target: float) -> Surface:
    """Icosahedron refined by edge midpoints until the edge length is <= h_target,
    vertices pushed to the sphere.  Deterministic vertex and triangle order."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    tris = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
            (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
            (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
            (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    edge = 1.0514622242382672 * radius  # icosahedron edge on the unit sphere x R
    while edge > h_target:
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        new = []
        for (a, b, c) in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = new
        edge *= 0.5
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return Surface(V.astype(np.float64), np.array(tris, dtype=np.int32))


def box_surface(lo: Vec3, hi: Vec3, h_target: float) -> Surface:
    """Axis-aligned box; each face split into a grid of squares, two triangles each,
    with vertices shared between faces."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    m = [max(1, int(math.ceil((hi[d] - lo[d]) / h_target))) for d in range(3)]
    index = {}
    verts = []

    def vid(ix, iy, iz):
        key = (ix, iy, iz)
        if key not in index:
            index[key] = len(verts)
            verts.append([lo[0] + (hi[0] - lo[0]) * ix / m[0],
                          lo[1] + (hi[1] - lo[1]) * iy / m[1],
                          lo[2] + (hi[2] - lo[2]) * iz / m[2]])
        return index[key]

    tris = []
    for d in range(3):
        a, b = [e for e in range(3) if e != d]
        for side in (0, m[d]):
            for ia in range(m[a]):
                for ib in range(m[b]):
                    def p(u, w):
                        c = [0, 0, 0]
                        c[d] = side
                        c[a] = u
                        c[b] = w
                        return vid(*c)
                    q00, q10, q01, q11 = p(ia, ib), p(ia + 1, ib), p(ia, ib + 1), p(ia + 1, ib + 1)
                    tris.append((q00, q10, q11))
                    tris.append((q00, q11, q01))
    return Surface(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32))


# Phase rules for the fluid indicators (what fsi_init_phases does after the solids).
RULE_SURFACE = 0      # phase takes the signed-distance field of a surface
RULE_COMPLEMENT = 1   # alpha = max(0, 1 - sum of solid alphas) * plane factor


@dataclass
class PhaseRule:
    kind: int
    surface: int = -1         # RULE_SURFACE: index into the surface list
    plane_z: float = 0.0      # RULE_COMPLEMENT: plane z = plane_z ...
    plane_side: int = 0       # 0: no plane, +1: keep z < plane_z, -1: keep z > plane_z


@dataclass
class Workload:
    name: str
    desc: MeshDesc
    surfaces: List[Surface]
    rules: List[PhaseRule]
    grid_cells: Tuple[int, int, int]
    steps: int
    k_max: int


def _cavity(n: int, name: str, steps: int, k_max: int, center: Vec3 = (0.6, 0.5, 0.5), radius: float = 0.2,
            mu_L: float = 0.1) -> Workload:
    h = 1.0 / n
    phases = [Phase(rho=1.0, mu=0.01), Phase(rho=1.0, mu=0.01, mu_L=mu_L, solid=True)]
    faces = [FaceBC(BC_DIRICHLET, (0.0, 0.0, 0.0), 0) for _ in range(5)]
    faces.append(FaceBC(BC_DIRICHLET, (1.0, 0.0, 0.0), 1))  # lid at z=1 wins on its edges
    desc = MeshDesc(n, n, n, 1.0, 1.0, 1.0, phases, (0.0, 0.0, 0.0), eps=1.5 * h,
                    eta=0.2, dt=0.01, rho_inf=0.0, c_i=36.0, faces=faces, pin_node=0)
    surf = icosphere(center, radius, h)
    rules = [PhaseRule(RULE_COMPLEMENT), PhaseRule(RULE_SURFACE, surface=0)]
    g = max(1, n // 4)
    return Workload(name, desc, [surf], rules, (g, g, g), steps, k_max)


def cavity16() -> Workload:
    return _cavity(16, "cavity16", steps=5, k_max=5)


def cavity64() -> Workload:
    return _cavity(64, "cavity64", steps=100, k_max=5)


def cavity(n: int) -> Workload:
    return _cavity(n, f"cavity{n}", steps=5, k_max=5)


def cavity_batch(count: int = 64, seed: int = 0) -> List[Workload]:
    """Uneven independent cavity instances: cube size s ~ U{16, 24, 32, 40, 48}, sphere
    centre ~ U[0.3, 0.7]^3, radius ~ U[0.1, 0.25], shear modulus 10^U[-2, 1]; instance
    k draws from its own stream numpy.random.default_rng([seed, k])."""
    out = []
    for k in range(count):
        rng = np.random.default_rng([seed, k])
        n = int(rng.choice([16, 24, 32, 40, 48]))
        c = tuple(float(v) for v in rng.uniform(0.3, 0.7, size=3))
        r = float(rng.uniform(0.1, 0.25))
        mu_L = float(10.0 ** rng.uniform(-2.0, 1.0))
        out.append(_cavity(n, f"batch{k}_n{n}", steps=20, k_max=5, center=c, radius=r, mu_L=mu_L))
    return out


def falling(scale: int = 1) -> Workload:
    """Sphere falling on an elastic block; scale=1 is 96x96x192."""
    nx, ny, nz = 96 // scale, 96 // scale, 192 // scale
    h = 1.0 / nx
    eps = 1.5 * h
    phases = [Phase(rho=1.0, mu=0.01),
              Phase(rho=2.0, mu=0.01, mu_L=1e3, solid=True),
              Phase(rho=1.5, mu=0.01, mu_L=50.0, solid=True)]
    faces = [FaceBC(BC_DIRICHLET, (0.0, 0.0, 0.0), 0) for _ in range(5)]
    faces.append(FaceBC(BC_NATURAL))
    desc = MeshDesc(nx, ny, nz, 1.0, 1.0, 2.0, phases, (0.0, 0.0, -9.81), eps=eps,
                    eta=0.1, dt=1e-3, faces=faces, pin_node=-1)
    pad = 6.0 * eps  # block faces that lie on the walls are pushed outside the box
    surfs = [icosphere((0.5, 0.5, 1.5), 0.15, h),
             box_surface((-pad, -pad, -pad), (1.0 + pad, 1.0 + pad, 0.3), h)]
    rules = [PhaseRule(RULE_COMPLEMENT), PhaseRule(RULE_SURFACE, surface=0),
             PhaseRule(RULE_SURFACE, surface=1)]
    return Workload("falling", desc, surfs, rules, (nx // 4, ny // 4, nz // 4), 500, 5)


def shipice(scale: int = 1, seed: int = 0) -> Workload:
    """Water/air, box hull at +x 0.5, 8 seeded non-overlapping ice boxes."""
    nx, ny, nz = 256 // scale, 128 // scale, 64 // scale
    h = 4.0 / nx
    eps = 1.5 * h
    phases = [Phase(rho=1000.0, mu=1e-3), Phase(rho=1.0, mu=1.8e-5),
              Phase(rho=500.0, mu=1e-3, mu_L=1e6, solid=True)]
    phases += [Phase(rho=900.0, mu=1e-3, mu_L=1e6, solid=True) for _ in range(8)]
    hull_lo = (0.75 - 0.5, 1.0 - 0.15, 0.5 - 0.1)
    hull_hi = (0.75 + 0.5, 1.0 + 0.15, 0.5 + 0.1)
    rng = np.random.default_rng(seed)
    ice = []
    while len(ice) < 8:
        sx, sy = rng.uniform(0.1, 0.3, size=2)
        cx, cy = rng.uniform(1.4, 3.8), rng.uniform(0.1, 1.9)
        lo = (cx - sx / 2, cy - sy / 2, 0.48 - 0.025)
        hi = (cx + sx / 2, cy + sy / 2, 0.48 + 0.025)
        if lo[1] < 0.0 or hi[1] > 2.0:
            continue
        ok = all(lo[0] > b[1][0] + 2 * eps or hi[0] < b[0][0] - 2 * eps or
                 lo[1] > b[1][1] + 2 * eps or hi[1] < b[0][1] - 2 * eps for b in ice)
        if ok:
            ice.append((lo, hi))
    faces = [FaceBC(BC_DIRICHLET, (0.0, 0.0, 0.0), 0) for _ in range(5)]
    faces.append(FaceBC(BC_NATURAL))
    desc = MeshDesc(nx, ny, nz, 4.0, 2.0, 1.0, phases, (0.0, 0.0, -9.81), eps=eps,
                    eta=1000.0, dt=1e-3, faces=faces,
                    prescribed_box=(hull_lo, hull_hi, (0.5, 0.0, 0.0)), pin_node=-1)
    surfs = [box_surface(hull_lo, hull_hi, h)] + [box_surface(lo, hi, h) for lo, hi in ice]
    rules = [PhaseRule(RULE_COMPLEMENT, plane_z=0.5, plane_side=+1),
             PhaseRule(RULE_COMPLEMENT, plane_z=0.5, plane_side=-1)]
    rules += [PhaseRule(RULE_SURFACE, surface=s) for s in range(9)]
    return Workload("shipice", desc, surfs, rules, (nx // 4, ny // 4, nz // 4), 200, 5)


# ---------------------------------------------------------------- random states

def node_coords(desc: MeshDesc) -> np.ndarray:
    """(3, nn) node coordinates, x fastest: x = i*hx etc."""
    hx, hy, hz = desc.h
    i = np.arange(desc.nx + 1, dtype=np.float64) * hx
    j = np.arange(desc.ny + 1, dtype=np.float64) * hy
    k = np.arange(desc.nz + 1, dtype=np.float64) * hz
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()])


def random_state(desc: MeshDesc, seed: int, amp_v: float = 1.0, amp_B: float = 0.05,
                 noise: float = 0.05, phi_range: float = 1.0, independent: bool = False):
    """Seeded smooth random state (x^{n+1}, x^n, xdot^n), each (ncomp, nn) float64.

    Velocities and pressure: a few random Fourier modes plus nodal noise.
    Phase indicators: tanh profiles of random spheres (values in [-1,1] scaled by
    phi_range) plus noise.  B: identity plus a small random symmetric perturbation.
    By default the phase fractions sum to one; with `independent` every phase i >= 1
    is its own sphere profile and phase 0 is 1 - s/2 for a further sphere profile s,
    so the fractions overlap (their sum ranges over about [0.5, 2.5]) while phase 0
    never drops below one half (the independently evolved indicators of N > 2 phases).
    """
    rng = np.random.default_rng(seed)
    X = node_coords(desc)
    L = np.array([desc.lx, desc.ly, desc.lz])[:, None]
    xs = X / L
    nc, nn = desc.ncomp, desc.nn

    def smooth(amp):
        out = np.zeros(nn)
        for _ in range(3):
            kv = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            c = rng.normal()
            out += c * np.sin(np.pi * kv[0] * xs[0] + ph[0]) * np.sin(np.pi * kv[1] * xs[1] + ph[1]) \
                * np.sin(np.pi * kv[2] * xs[2] + ph[2])
        out += noise * rng.normal(size=nn)
        return amp * out

    def one():
        x = np.zeros((nc, nn))
        for k in range(3):
            x[k] = smooth(amp_v)
        x[3] = smooth(1.0)
        eps = desc.eps if desc.eps > 0 else 1.5 * min(desc.h)
        # phase fractions that sum to one (phase 0 takes what the others leave), each
        # phase i >= 1 a tanh profile of a random sphere, then small nodal noise
        remaining = np.ones(nn)
        alphas = [None] * desc.n_phase
        for i in range(1, desc.n_phase):
            c = rng.uniform(0.3, 0.7, size=3) * L[:, 0]
            r = rng.uniform(0.15, 0.3) * float(L.min())
            d = r - np.sqrt(((X - c[:, None]) ** 2).sum(0))
            s = (1.0 + phi_range * np.tanh(d / (math.sqrt(2.0) * eps))) / 2.0
            alphas[i] = s if independent else s * remaining
            remaining = remaining - alphas[i]
        alphas[0] = remaining
        if independent:
            c = rng.uniform(0.3, 0.7, size=3) * L[:, 0]
            r = rng.uniform(0.15, 0.3) * float(L.min())
            d = r - np.sqrt(((X - c[:, None]) ** 2).sum(0))
            alphas[0] = 1.0 - 0.25 * (1.0 + np.tanh(d / (math.sqrt(2.0) * eps)))
        for i in range(desc.n_phase):
            x[4 + i] = 2.0 * alphas[i] - 1.0 + 0.4 * noise * rng.normal(size=nn)
        base = 4 + desc.n_phase
        for s in range(desc.n_solid):
            for c in range(6):
                x[base + 6 * s + c] = (1.0 if c < 3 else 0.0) + amp_B * smooth(1.0)
        return x

    x1 = one()
    xn = x1 + 0.1 * (one() - x1)
    xdn = one() * 0.5
    return x1, xn, xdn


def kuhn_corners() -> np.ndarray:
    """(6, 4) cell corners (bit 0 x, bit 1 y, bit 2 z) of the six tetrahedra around the
    cell diagonal 0 -> 7: 0 -> e_p1 -> e_p1 + e_p2 -> 7 for each permutation p of the axes."""
    import itertools
    out = []
    for p in itertools.permutations(range(3)):
        c1 = 1 << p[0]
        c2 = c1 | (1 << p[1])
        out.append([0, c1, c2, 7])
    return np.array(out)


def tet_box_mesh(desc: MeshDesc, jitter: float = 0.0, seed: int = 0):
    """Linear tetrahedra on a box grid's nodes: (X (3, nn) coordinates, conn (ne, 4) int64),
    six tetrahedra per cell (element e = 6 x cell + t, cells x fastest), interior nodes
    moved by uniform offsets in [-jitter, jitter] x h per axis (numpy.random.default_rng(seed)),
    each element's corners ordered for a positive volume."""
    nx, ny, nz = desc.nx, desc.ny, desc.nz
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    h = desc.h
    n = np.arange(nn)
    i, j, k = n % (nx + 1), (n // (nx + 1)) % (ny + 1), n // ((nx + 1) * (ny + 1))
    X = np.stack([i * h[0], j * h[1], k * h[2]]).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        inner = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
        d = rng.uniform(-jitter, jitter, size=(3, nn)) * np.array(h)[:, None]
        X[:, inner] += d[:, inner]
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ex, ey, ez = (a.transpose(2, 1, 0).ravel() for a in (ex, ey, ez))
    cells = np.empty((ex.size, 8), dtype=np.int64)
    for a in range(8):
        cells[:, a] = (ex + (a & 1)) + (nx + 1) * ((ey + ((a >> 1) & 1)) + (ny + 1) * (ez + ((a >> 2) & 1)))
    conn = cells[:, kuhn_corners()].reshape(-1, 4)
    e1, e2, e3 = (X[:, conn[:, a]] - X[:, conn[:, 0]] for a in (1, 2, 3))
    det = np.einsum("ie,ie->e", e1, np.cross(e2.T, e3.T).T)
    neg = det < 0
    conn[neg] = conn[neg][:, [0, 2, 1, 3]]
    return X, conn


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).normal(size=n)


def he_normal_weights(fan: list, seed: int, last_scale: float = 0.1) -> np.ndarray:
    """Seeded initial weights for a stack of 3x3x3 convolutions.

    `fan` lists (out channels, in channels) per convolution in storage order; each
    convolution gets co*ci*27 normal draws with std sqrt(2 / (27 ci)) (He et al. 2015),
    the last one scaled by `last_scale` so that an untrained network starts close to
    zero output."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (co, ci) in enumerate(fan):
        std = math.sqrt(2.0 / (27 * ci)) * (last_scale if k == len(fan) - 1 else 1.0)
        parts.append(rng.normal(scale=std, size=co * ci * 27))
    return np.concatenate(parts)
