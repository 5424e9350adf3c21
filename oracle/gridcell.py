"""Phase-field initialisation from a triangulated surface (oracle).

Test infrastructure only (see oracle/__init__.py).

Section 3:
  phi = tanh(d / (sqrt(2) eps)), d the signed distance, positive inside.
Distance (Section 3.1, Algorithm 1):
  grid cells: bounding box of the Eulerian nodes split into gx x gy x gz cells of size
    hc = (x_max - x_min)/gx; node cell i = floor((x_p - x_min)/hc), clamped to gx-1
    (nodes on the upper face of the box belong to the last cell);
  each triangle is assigned to every cell of its bounding box expanded by 3 eps,
    index range floor((min - 3eps - x_min)/hc) .. floor((max + 3eps - x_min)/hc),
    clamped to the grid;
  a node in a cell that holds triangles gets |d| = the smallest Euclidean distance to
    the vertices of those triangles (ties: lowest vertex id) and
    |phi| = tanh(|d|/(sqrt(2) eps)); every node in a cell without triangles gets
    |phi| = 1.
Sign (Section 3.2-3.3, Algorithm 2):
  a ray from the node in +x; triangles of the cells [i, gx) x {j} x {k} are tested,
    in cell i only those with a vertex x_v > x_p;
  projected on the y-z plane, A0 = area of the triangle, A_m = area of (node, edge
    opposite vertex m); triangles with A0 <= chi are skipped (parallel to the ray);
    the ray crosses when A1 + A2 + A3 - A0 <= 2 chi and the crossing point
    x_c = (A1 x1 + A2 x2 + A3 x3)/A0 lies beyond the node (x_c > x_p);
  non-duplicated plane partitioning: with n_small = #{m : A_m < chi} the crossing is
    an element crossing (key: the three vertex ids) when n_small = 0 or 3, an edge
    crossing (key: the two vertices of the edge opposite the small area) when 1, a
    node crossing (key: the remaining vertex) when 2; the crossing number is the
    number of distinct keys; odd means inside;
  in a cell without triangles only its lowest-index node is cast and its sign is
    given to every node of the cell;
  chi = 1e-12 L^2 with L the diagonal of the box (the paper gives no value).
All arithmetic is IEEE float64 elementwise (numpy never contracts to FMA):
  area(a,b,c) = 0.5 * |(b_y - a_y)*(c_z - a_z) - (b_z - a_z)*(c_y - a_y)|
  d^2 = (dx*dx + dy*dy) + dz*dz.
"""
from __future__ import annotations

import math

import numpy as np

from workloads import RULE_COMPLEMENT, RULE_SURFACE, MeshDesc, Surface


def _node_xyz(desc: MeshDesc):
    hx, hy, hz = desc.lx / desc.nx, desc.ly / desc.ny, desc.lz / desc.nz
    n = np.arange(desc.nn)
    i = n % (desc.nx + 1)
    j = (n // (desc.nx + 1)) % (desc.ny + 1)
    k = n // ((desc.nx + 1) * (desc.ny + 1))
    return np.stack([i * hx, j * hy, k * hz]), (hx, hy, hz)


class GridCells:
    def __init__(self, desc: MeshDesc, surf: Surface, eps: float, grid):
        self.desc = desc
        self.g = tuple(int(v) for v in grid)
        X, h = _node_xyz(desc)
        self.X = X
        self.xmin = np.array([0.0, 0.0, 0.0])
        self.xmax = np.array([desc.nx * h[0], desc.ny * h[1], desc.nz * h[2]])
        self.hc = np.array([(self.xmax[d] - self.xmin[d]) / self.g[d] for d in range(3)])
        self.eps = eps
        self.V = surf.verts
        self.T = surf.tris.astype(np.int64)
        # node cells
        c = np.empty((3, desc.nn), dtype=np.int64)
        for d in range(3):
            c[d] = np.minimum(np.floor((X[d] - self.xmin[d]) / self.hc[d]).astype(np.int64), self.g[d] - 1)
        self.node_cell = c
        self.node_cell_id = c[0] + self.g[0] * (c[1] + self.g[1] * c[2])
        # triangle cells
        three_eps = 3.0 * eps
        cells = {}
        self.tri_lo = np.empty((3, len(self.T)), dtype=np.int64)
        for t, tri in enumerate(self.T):
            rng = []
            for d in range(3):
                lo = min(self.V[tri[0], d], self.V[tri[1], d], self.V[tri[2], d])
                hi = max(self.V[tri[0], d], self.V[tri[1], d], self.V[tri[2], d])
                a = int(math.floor(((lo - three_eps) - self.xmin[d]) / self.hc[d]))
                b = int(math.floor(((hi + three_eps) - self.xmin[d]) / self.hc[d]))
                a = min(max(a, 0), self.g[d] - 1)
                b = min(max(b, 0), self.g[d] - 1)
                rng.append((a, b))
                self.tri_lo[d, t] = a
            for cz in range(rng[2][0], rng[2][1] + 1):
                for cy in range(rng[1][0], rng[1][1] + 1):
                    for cx in range(rng[0][0], rng[0][1] + 1):
                        cells.setdefault(cx + self.g[0] * (cy + self.g[1] * cz), []).append(t)
        self.cells = {k: np.array(v, dtype=np.int64) for k, v in cells.items()}
        L2 = desc.lx * desc.lx + desc.ly * desc.ly + desc.lz * desc.lz
        self.chi = 1e-12 * L2

    def cell_id(self, cx, cy, cz):
        return cx + self.g[0] * (cy + self.g[1] * cz)

    # ------------------------------------------------------------ distance
    def nearest_vertex(self, p: int):
        """(d^2, vertex id) of the nearest vertex among the node's cell triangles."""
        tris = self.cells[int(self.node_cell_id[p])]
        vids = np.unique(self.T[tris].ravel())  # ascending ids
        dx = self.X[0, p] - self.V[vids, 0]
        dy = self.X[1, p] - self.V[vids, 1]
        dz = self.X[2, p] - self.V[vids, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        a = int(np.argmin(d2))  # first minimum = lowest id
        return d2[a], int(vids[a])

    # ------------------------------------------------------------ ray cast
    def crossings(self, p: int) -> int:
        xp, yp, zp = self.X[0, p], self.X[1, p], self.X[2, p]
        cx, cy, cz = (int(v) for v in self.node_cell[:, p])
        cand = []
        for c in range(cx, self.g[0]):
            tris = self.cells.get(self.cell_id(c, cy, cz))
            if tris is None:
                continue
            if c == cx:
                vx = self.V[self.T[tris], 0]
                tris = tris[(vx > xp).any(axis=1)]
            cand.append(tris)
        if not cand:
            return 0
        tris = np.concatenate(cand)
        v1, v2, v3 = self.V[self.T[tris, 0]], self.V[self.T[tris, 1]], self.V[self.T[tris, 2]]

        def area(ay, az, by, bz, cy_, cz_):
            return 0.5 * np.abs((by - ay) * (cz_ - az) - (bz - az) * (cy_ - ay))

        A0 = area(v1[:, 1], v1[:, 2], v2[:, 1], v2[:, 2], v3[:, 1], v3[:, 2])
        A1 = area(yp, zp, v2[:, 1], v2[:, 2], v3[:, 1], v3[:, 2])
        A2 = area(yp, zp, v3[:, 1], v3[:, 2], v1[:, 1], v1[:, 2])
        A3 = area(yp, zp, v1[:, 1], v1[:, 2], v2[:, 1], v2[:, 2])
        chi = self.chi
        ok = A0 > chi
        ok &= ((A1 + A2) + A3) - A0 <= 2.0 * chi
        safeA0 = np.where(A0 > 0.0, A0, 1.0)
        xc = ((A1 * v1[:, 0] + A2 * v2[:, 0]) + A3 * v3[:, 0]) / safeA0
        ok &= xc > xp
        keys = set()
        for t_local in np.nonzero(ok)[0]:
            ids = [int(v) for v in self.T[tris[t_local]]]
            small = [A1[t_local] < chi, A2[t_local] < chi, A3[t_local] < chi]
            ns = sum(small)
            if ns == 1:
                m = small.index(True)
                key = tuple(sorted(ids[q] for q in range(3) if q != m))
            elif ns == 2:
                m = small.index(False)
                key = (ids[m],)
            else:
                key = tuple(sorted(ids))
            keys.add(key)
        return len(keys)


def signed_distance_phi(desc: MeshDesc, surf: Surface, eps: float, grid, nodes=None):
    """phi (nn,) and tags (4, nn) int32 = [cell id, nearest vertex or -1, crossing
    number, inside flag].  With `nodes` only those entries are computed (others 0)."""
    gc = GridCells(desc, surf, eps, grid)
    nn = desc.nn
    phi = np.zeros(nn)
    tags = np.zeros((4, nn), dtype=np.int32)
    todo = np.arange(nn) if nodes is None else np.asarray(nodes)
    scale = math.sqrt(2.0) * eps
    # representative (lowest index) node of each cell without triangles
    rep = {}
    for cid in np.unique(gc.node_cell_id):
        if int(cid) not in gc.cells:
            rep[int(cid)] = int(np.nonzero(gc.node_cell_id == cid)[0][0])
    rep_count = {}
    for p in todo:
        p = int(p)
        cid = int(gc.node_cell_id[p])
        tags[0, p] = cid
        if cid in gc.cells:
            d2, vid = gc.nearest_vertex(p)
            cross = gc.crossings(p)
            mag = math.tanh(math.sqrt(d2) / scale)
            tags[1, p] = vid
        else:
            r = rep[cid]
            if r not in rep_count:
                rep_count[r] = gc.crossings(r)
            cross = rep_count[r]
            mag = 1.0
            tags[1, p] = -1
        inside = cross % 2 == 1
        tags[2, p] = cross
        tags[3, p] = int(inside)
        phi[p] = mag if inside else -mag
    return phi, tags


def apply_rules(desc: MeshDesc, surface_phi: dict, rules, eps: float) -> np.ndarray:
    """(N, nn) phase indicators: surface phases from their signed-distance phi, the
    complement phases alpha = max(0, 1 - sum of surface alphas) x plane factor."""
    nn = desc.nn
    X, _ = _node_xyz(desc)
    out = np.zeros((len(rules), nn))
    solid_alpha = np.zeros(nn)
    for i, r in enumerate(rules):
        if r.kind == RULE_SURFACE:
            out[i] = surface_phi[r.surface]
            solid_alpha = solid_alpha + (1.0 + out[i]) / 2.0
    for i, r in enumerate(rules):
        if r.kind == RULE_COMPLEMENT:
            a = np.maximum(0.0, 1.0 - solid_alpha)
            if r.plane_side != 0:
                pp = np.tanh((r.plane_z - X[2]) / (math.sqrt(2.0) * eps))
                a = a * ((1.0 + pp) / 2.0 if r.plane_side > 0 else (1.0 - pp) / 2.0)
            out[i] = 2.0 * a - 1.0
    return out
