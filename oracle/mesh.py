"""Background mesh, cell classification, DOFs, subdomains and coarse objects.

Oracle (test infrastructure only).  Follows Sect. 2.1 (cell partition and
subdomain partition), Sect. 3.2 (geometric objects), Sect. 4.4 (first variant of
the improved coarse objects) and the strong Dirichlet / pinned-node treatment of
Sect. 5.1.  Readings of passages the paper leaves open (numbered as in the
design notes):

  R1  a node is inside iff phi < 0 (strict); phi == 0 counts as outside;
  R2  a cell is internal iff its 8 vertices are inside, external iff none is,
      cut otherwise; active = internal or cut; no volume-fraction threshold;
  R3  DOFs are the nodes of active cells, minus nodes constrained by a strong
      Dirichlet box face, minus the pinned node; numbered in node order;
  R4  the pinned node (when no box face constrains any node) is the node whose 8
      incident cells are all internal with the smallest phi (ties: lowest index);
  R5  a subdomain is a connected component (cells sharing a DOF) of the active
      cells of one cubic block; subdomains are ordered by (block index, smallest
      cell index);
  R6  neigh(xi) = subdomains owning an active cell that contains xi; the
      interface Gamma = DOFs with |neigh| >= 2;
  R7  objects = connected components, through FE edges (grid edges of active
      cells), of interface DOFs with identical neigh sets; |neigh| = 2 -> face,
      otherwise a single DOF -> corner and several DOFs -> edge; objects are
      ordered by their smallest DOF id;
  R8  variant 1: an FE edge of an edge object is cut iff its end nodes lie on
      different sides (phi < 0 vs phi >= 0); DOFs on cut FE edges become corners;
      the rest form connected sub-edges over the uncut FE edges (single DOFs
      become corners).

Parity: every function here is integer work and pinned by hand-counted cases,
brute-force recomputation and the closed-form object counts of an uncut
box partition (tests/test_oracle_mesh.py).
"""
from __future__ import annotations

from collections import deque

import numpy as np

EXTERNAL, CUT, INTERNAL = 0, 1, 2
CORNER, EDGE, FACE = 0, 1, 2

# local vertex a of a cell has offsets (a & 1, (a >> 1) & 1, (a >> 2) & 1)
VERTEX_OFFSETS = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]


class Grid:
    """Cartesian background mesh of the box [lo, hi] with uniform cubic cells."""

    def __init__(self, box_lo, box_hi, cells, sub_cells):
        self.lo = np.asarray(box_lo, dtype=np.float64)
        self.hi = np.asarray(box_hi, dtype=np.float64)
        self.n = np.asarray(cells, dtype=np.int64)
        self.s = np.asarray(sub_cells, dtype=np.int64)
        hs = (self.hi - self.lo) / self.n
        if not np.allclose(hs, hs[0], rtol=1e-12, atol=0):
            raise ValueError("cells must be cubes")
        if np.any(self.n % self.s):
            raise ValueError("sub_cells must divide cells")
        self.h = float(hs[0])
        self.nn = self.n + 1
        self.n_nodes = int(np.prod(self.nn))
        self.n_cells = int(np.prod(self.n))
        self.nb = self.n // self.s
        self.n_blocks = int(np.prod(self.nb))

    def node_id(self, i, j, k):
        return i + self.nn[0] * (j + self.nn[1] * k)

    def node_ijk(self, v):
        v = np.asarray(v)
        return v % self.nn[0], (v // self.nn[0]) % self.nn[1], v // (self.nn[0] * self.nn[1])

    def cell_id(self, i, j, k):
        return i + self.n[0] * (j + self.n[1] * k)

    def cell_ijk(self, c):
        c = np.asarray(c)
        return c % self.n[0], (c // self.n[0]) % self.n[1], c // (self.n[0] * self.n[1])

    def cell_nodes(self, c):
        """The 8 node ids of cell c in local vertex order."""
        i, j, k = self.cell_ijk(c)
        return [int(self.node_id(i + a, j + b, k + d)) for (a, b, d) in VERTEX_OFFSETS]

    def block_of_cell(self, c):
        i, j, k = self.cell_ijk(c)
        bi, bj, bk = i // self.s[0], j // self.s[1], k // self.s[2]
        return bi + self.nb[0] * (bj + self.nb[1] * bk)

    def node_xyz(self, v):
        i, j, k = self.node_ijk(v)
        return self.lo + self.h * np.stack([i, j, k], axis=-1)

    def cells_of_node(self, v):
        """Cell ids of the (up to 8) cells containing node v."""
        i, j, k = (int(x) for x in self.node_ijk(v))
        out = []
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    ci, cj, ck = i + di, j + dj, k + dk
                    if 0 <= ci < self.n[0] and 0 <= cj < self.n[1] and 0 <= ck < self.n[2]:
                        out.append(int(self.cell_id(ci, cj, ck)))
        return out


# ---------------------------------------------------------------------------
# Sect. 2.1: cell classification
# ---------------------------------------------------------------------------

def classify_cells(grid: Grid, phi: np.ndarray) -> np.ndarray:
    """Cell type per cell: EXTERNAL (0), CUT (1) or INTERNAL (2) (readings R1, R2)."""
    nx, ny, nz = (int(x) for x in grid.n)
    inside = (np.asarray(phi).reshape(nz + 1, ny + 1, nx + 1) < 0)
    count = np.zeros((nz, ny, nx), dtype=np.int64)
    for (a, b, d) in VERTEX_OFFSETS:
        count += inside[d:d + nz, b:b + ny, a:a + nx]
    t = np.full((nz, ny, nx), CUT, dtype=np.uint8)
    t[count == 0] = EXTERNAL
    t[count == 8] = INTERNAL
    return t.ravel()


def active_nodes(grid: Grid, cell_type: np.ndarray) -> np.ndarray:
    nx, ny, nz = (int(x) for x in grid.n)
    act = (cell_type.reshape(nz, ny, nx) != EXTERNAL)
    node = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    for (a, b, d) in VERTEX_OFFSETS:
        node[d:d + nz, b:b + ny, a:a + nx] |= act
    return node.ravel()


def box_face_nodes(grid: Grid, face_mask: int) -> np.ndarray:
    nx, ny, nz = (int(x) for x in grid.n)
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    if face_mask & 1:
        m[:, :, 0] = True
    if face_mask & 2:
        m[:, :, nx] = True
    if face_mask & 4:
        m[:, 0, :] = True
    if face_mask & 8:
        m[:, ny, :] = True
    if face_mask & 16:
        m[0, :, :] = True
    if face_mask & 32:
        m[nz, :, :] = True
    return m.ravel()


def auto_pin(grid: Grid, cell_type: np.ndarray, phi: np.ndarray) -> int:
    """Reading R4: deepest node (min phi) whose 8 incident cells are all internal."""
    nx, ny, nz = (int(x) for x in grid.n)
    internal = (cell_type.reshape(nz, ny, nx) == INTERNAL)
    all8 = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    inner = np.ones((nz - 1, ny - 1, nx - 1), dtype=bool)
    for (a, b, d) in VERTEX_OFFSETS:          # cell (i-1+a, j-1+b, k-1+d) of node (i, j, k)
        inner &= internal[d:d + nz - 1, b:b + ny - 1, a:a + nx - 1]
    all8[1:nz, 1:ny, 1:nx] = inner
    cand = all8.ravel()
    if not cand.any():
        raise ValueError("no node with 8 internal cells to pin")
    return int(np.argmin(np.where(cand, phi, np.inf)))    # first minimum = lowest index


def number_dofs(grid: Grid, cell_type, phi, face_mask: int, pin_node: int):
    """Reading R3.  Returns (dof_of_node, constrained_mask, pin) with -1 for non-DOFs."""
    act = active_nodes(grid, cell_type)
    constrained = act & box_face_nodes(grid, face_mask)
    pin = -1
    if pin_node == -2:
        if not constrained.any():
            pin = auto_pin(grid, cell_type, phi)
    elif pin_node >= 0:
        pin = int(pin_node)
        if not act[pin]:
            raise ValueError("pinned node is not active")
    if pin >= 0:
        constrained[pin] = True
    free = act & ~constrained
    dof = np.full(grid.n_nodes, -1, dtype=np.int64)
    dof[free] = np.arange(int(free.sum()))
    return dof, constrained, pin


# ---------------------------------------------------------------------------
# Sect. 2.1: subdomains by aggregation of active cells (reading R5)
# ---------------------------------------------------------------------------

def subdomains(grid: Grid, cell_type, dof_of_node):
    """Return sub_of_cell (-1 for external cells) and the list of cells per subdomain."""
    sub_of_cell = np.full(grid.n_cells, -1, dtype=np.int64)
    sub_cells = []
    block_cells = [[] for _ in range(grid.n_blocks)]
    for c in np.flatnonzero(cell_type != EXTERNAL):
        block_cells[grid.block_of_cell(c)].append(int(c))
    for b in range(grid.n_blocks):
        cells = block_cells[b]
        if not cells:
            continue
        by_node = {}
        for c in cells:
            for v in grid.cell_nodes(c):
                if dof_of_node[v] >= 0:
                    by_node.setdefault(v, []).append(c)
        seen = set()
        for c0 in cells:                      # ascending: each new component starts at its min cell
            if c0 in seen:
                continue
            comp = []
            queue = deque([c0])
            seen.add(c0)
            while queue:
                c = queue.popleft()
                comp.append(c)
                for v in grid.cell_nodes(c):
                    for c2 in by_node.get(v, ()):
                        if c2 not in seen:
                            seen.add(c2)
                            queue.append(c2)
            sid = len(sub_cells)
            sub_cells.append(sorted(comp))
            sub_of_cell[comp] = sid
    return sub_of_cell, sub_cells


def neighbour_sets(grid: Grid, sub_of_cell, dof_of_node):
    """neigh(xi) per DOF (reading R6), as sorted tuples; index = DOF id."""
    n_dof = int(dof_of_node.max()) + 1 if (dof_of_node >= 0).any() else 0
    neigh = [None] * n_dof
    for v in np.flatnonzero(dof_of_node >= 0):
        s = sorted({int(sub_of_cell[c]) for c in grid.cells_of_node(v) if sub_of_cell[c] >= 0})
        neigh[dof_of_node[v]] = tuple(s)
    return neigh


def local_dofs(grid: Grid, sub_cells, dof_of_node):
    """Sorted DOF ids of each subdomain (nodes of its cells that are DOFs)."""
    out = []
    for cells in sub_cells:
        s = set()
        for c in cells:
            for v in grid.cell_nodes(c):
                if dof_of_node[v] >= 0:
                    s.add(int(dof_of_node[v]))
        out.append(np.array(sorted(s), dtype=np.int64))
    return out


def fe_edge_exists(grid: Grid, cell_type, v, w):
    """True iff nodes v, w span a grid edge of an active cell."""
    cv = set(grid.cells_of_node(v))
    cw = set(grid.cells_of_node(w))
    common = cv & cw
    vi, vj, vk = (int(x) for x in grid.node_ijk(v))
    wi, wj, wk = (int(x) for x in grid.node_ijk(w))
    if abs(vi - wi) + abs(vj - wj) + abs(vk - wk) != 1:
        return False
    return any(cell_type[c] != EXTERNAL for c in common)


def _axis_neighbours(grid: Grid, v):
    i, j, k = (int(x) for x in grid.node_ijk(v))
    out = []
    for (di, dj, dk) in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        a, b, c = i + di, j + dj, k + dk
        if 0 <= a < grid.nn[0] and 0 <= b < grid.nn[1] and 0 <= c < grid.nn[2]:
            out.append(int(grid.node_id(a, b, c)))
    return out


def _components(members, adjacent):
    """Connected components of ``members`` (sorted list) under ``adjacent(u)``."""
    mset = set(members)
    seen = set()
    comps = []
    for m in members:
        if m in seen:
            continue
        comp = []
        queue = deque([m])
        seen.add(m)
        while queue:
            u = queue.popleft()
            comp.append(u)
            for w in adjacent(u):
                if w in mset and w not in seen:
                    seen.add(w)
                    queue.append(w)
        comps.append(sorted(comp))
    return comps


def standard_objects(grid: Grid, cell_type, dof_of_node, neigh):
    """Sect. 3.2 objects (reading R7).  Returns a list of dicts sorted by min DOF id:
    {"dofs": sorted DOF ids, "neigh": tuple of subdomains, "kind": CORNER/EDGE/FACE}."""
    node_of_dof = np.flatnonzero(dof_of_node >= 0)
    groups = {}
    for d, ns in enumerate(neigh):
        if len(ns) >= 2:
            groups.setdefault(ns, []).append(d)

    def adjacent(d):
        v = node_of_dof[d]
        out = []
        for w in _axis_neighbours(grid, v):
            if dof_of_node[w] >= 0 and fe_edge_exists(grid, cell_type, v, w):
                out.append(int(dof_of_node[w]))
        return out

    objs = []
    for ns, members in groups.items():
        for comp in _components(sorted(members), adjacent):
            if len(ns) == 2:
                kind = FACE
            elif len(comp) == 1:
                kind = CORNER
            else:
                kind = EDGE
            objs.append({"dofs": comp, "neigh": ns, "kind": kind})
    objs.sort(key=lambda o: o["dofs"][0])
    return objs


def variant1_objects(grid: Grid, cell_type, dof_of_node, phi, std_objs):
    """Sect. 4.4: split each edge object at its cut FE edges (reading R8)."""
    node_of_dof = np.flatnonzero(dof_of_node >= 0)
    inside = np.asarray(phi) < 0
    out = []
    for o in std_objs:
        if o["kind"] != EDGE:
            out.append(o)
            continue
        members = set(o["dofs"])
        edges = []
        for d in o["dofs"]:
            v = node_of_dof[d]
            for w in _axis_neighbours(grid, v):
                e = int(dof_of_node[w])
                if e > d and e in members and fe_edge_exists(grid, cell_type, v, w):
                    edges.append((d, e, bool(inside[v]) != bool(inside[w])))
        corners = set()
        for (a, b, cut) in edges:
            if cut:
                corners.add(a)
                corners.add(b)
        uncut_adj = {}
        for (a, b, cut) in edges:
            if not cut and a not in corners and b not in corners:
                uncut_adj.setdefault(a, []).append(b)
                uncut_adj.setdefault(b, []).append(a)
        for c in sorted(corners):
            out.append({"dofs": [c], "neigh": o["neigh"], "kind": CORNER})
        rest = sorted(members - corners)
        for comp in _components(rest, lambda u: uncut_adj.get(u, [])):
            out.append({"dofs": comp, "neigh": o["neigh"], "kind": CORNER if len(comp) == 1 else EDGE})
    out.sort(key=lambda o: o["dofs"][0])
    return out


V2_WEIGHT_TOL = 1e-8


def variant2_objects(grid: Grid, cell_type, dof_of_node, std_objs, weights):
    """Sect. 4.5: split each edge object into runs of FE-edge-adjacent DOFs with the same
    stiffness weights; DOFs left alone become corners (reading R22: weights "the same" when
    every subdomain's weight differs by at most V2_WEIGHT_TOL; weights[d] maps each
    subdomain of neigh(d) to A^w_dd / sum_w' A^w'_dd)."""
    node_of_dof = np.flatnonzero(dof_of_node >= 0)
    out = []
    for o in std_objs:
        if o["kind"] != EDGE:
            out.append(o)
            continue
        members = set(o["dofs"])

        def same(a, b):
            return max(abs(weights[a][w] - weights[b][w]) for w in o["neigh"]) <= V2_WEIGHT_TOL

        def adjacent(d):
            v = node_of_dof[d]
            res = []
            for w in _axis_neighbours(grid, v):
                e = int(dof_of_node[w])
                if e in members and fe_edge_exists(grid, cell_type, v, w) and same(d, e):
                    res.append(e)
            return res

        for comp in _components(sorted(members), adjacent):
            out.append({"dofs": comp, "neigh": o["neigh"], "kind": CORNER if len(comp) == 1 else EDGE})
    out.sort(key=lambda o: o["dofs"][0])
    return out


def coarse_objects(objs, coarse: str):
    """Lambda_O: 'c' corners, 'ce' corners+edges, 'cef' all (Sect. 3.2)."""
    keep = {"c": (CORNER,), "ce": (CORNER, EDGE), "cef": (CORNER, EDGE, FACE)}[coarse]
    return [o for o in objs if o["kind"] in keep]


class Mesh:
    """Everything integer about one problem, in the oracle's plain form."""

    def __init__(self, problem):
        p = problem
        self.grid = Grid(p.box_lo, p.box_hi, p.cells, p.sub_cells)
        self.phi = np.asarray(p.phi, dtype=np.float64)
        self.cell_type = classify_cells(self.grid, self.phi)
        self.dof_of_node, self.constrained, self.pin = number_dofs(
            self.grid, self.cell_type, self.phi, p.dirichlet_face_mask, p.pin_node)
        self.node_of_dof = np.flatnonzero(self.dof_of_node >= 0)
        self.n_dof = self.node_of_dof.size
        self.sub_of_cell, self.sub_cells = subdomains(self.grid, self.cell_type, self.dof_of_node)
        self.n_sub = len(self.sub_cells)
        self.neigh = neighbour_sets(self.grid, self.sub_of_cell, self.dof_of_node)
        self.sub_dofs = local_dofs(self.grid, self.sub_cells, self.dof_of_node)
        self.is_gamma = np.array([len(ns) >= 2 for ns in self.neigh], dtype=bool)
        self._objects = {}

    def objects(self, variant: str = "v1", weights=None):
        """Objects of variant 'std', 'v1' or 'v2' (v2 needs the stiffness weights per DOF)."""
        if "std" not in self._objects:
            self._objects["std"] = standard_objects(self.grid, self.cell_type, self.dof_of_node, self.neigh)
        if variant == "v1" and "v1" not in self._objects:
            self._objects["v1"] = variant1_objects(self.grid, self.cell_type, self.dof_of_node,
                                                   self.phi, self._objects["std"])
        if variant == "v2":
            return variant2_objects(self.grid, self.cell_type, self.dof_of_node, self._objects["std"], weights)
        return self._objects[variant]
