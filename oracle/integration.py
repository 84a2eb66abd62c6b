"""Cut-cell integration by marching tetrahedra (oracle; test infrastructure only).

Sect. 2.2 bulk form: A_e(u, v) = int_{e cap Omega} grad u . grad v (Neumann on the
unfitted boundary, so no Nitsche terms); loads int_{e cap Omega} f_h phi_a and
int_{Gamma_N cap e} (q_h . n) phi_a with f_h, q_h the Q1 interpolants of nodal
data.  The paper integrates cut cells on "integration cells" (Fig. 1c) without
fixing the algorithm; the reading used here (R9):

  * every cube is split into the 6 Kuhn tetrahedra v000 -> v000+e_a ->
    v000+e_a+e_b -> v111 over the 6 axis orders (a, b, c); the split is
    conforming across cells, so the discrete boundary is watertight;
  * phi is linear on each tetrahedron (phi_h); the part {phi_h < 0} is cut out
    with the edge crossing points x_u + phi_u/(phi_u - phi_v) (x_v - x_u):
    1 inside vertex -> one small tet; 2 -> a prism; 3 -> the tet minus a corner,
    also a prism; each prism is split into 3 tets;
  * the boundary facet is one triangle (1 or 3 inside vertices) or a planar quad
    split into 2 triangles (2 inside vertices), with unit normal grad(phi_h)/|.|;
  * volumes use the degree-7 Grundmann-Moeller tet rule and facets the degree-7
    triangle rule: the integrands (products of two trilinears) have degree <= 6,
    so every cut-cell integral is exact up to rounding.

Internal cells use the closed forms  K = h Khat,  Khat_ab = sum_d k(a_d, b_d)
prod_{d' != d} m(a_d', b_d')  and  M = h^3 prod_d m(a_d, b_d)  with
k(same) = 1, k(diff) = -1, m(same) = 1/3, m(diff) = 1/6.

Parity: pinned (tests/test_oracle_integration.py) by exact volumes of plane
cuts, the closed form of an uncut cell recovered through the tet machinery,
zero row sums and positive semi-definiteness of every K_e, the divergence
theorem on the cut facets, the convergence of the sphere volume, and the
quadrature's own exactness on simplex moments.
"""
from __future__ import annotations

import itertools

import numpy as np

from .mesh import CUT, INTERNAL, VERTEX_OFFSETS
from .quadrature import TET_BARY, TET_W, TRI_BARY, TRI_W

UNIT_VERTS = np.array(VERTEX_OFFSETS, dtype=np.float64)          # (8, 3)
BITS = np.array(VERTEX_OFFSETS, dtype=np.int64)                  # (8, 3)

# Kuhn tetrahedra as local vertex ids (vertex id = x + 2y + 4z)
KUHN_TETS = []
for perm in itertools.permutations(range(3)):
    a, b = perm[0], perm[1]
    KUHN_TETS.append((0, 1 << a, (1 << a) | (1 << b), 7))


def q1_shape(xi):
    """Trilinear shape functions N_a at local points xi (m, 3) in [0,1]^3 -> (m, 8)."""
    xi = np.atleast_2d(xi)
    out = np.ones((xi.shape[0], 8))
    for a in range(8):
        for d in range(3):
            out[:, a] *= xi[:, d] if BITS[a, d] else 1.0 - xi[:, d]
    return out


def q1_grad(xi):
    """Gradients dN_a/dxi_d at local points (m, 3) -> (m, 8, 3)."""
    xi = np.atleast_2d(xi)
    g = np.ones((xi.shape[0], 8, 3))
    for a in range(8):
        for d in range(3):
            for e in range(3):
                if e == d:
                    g[:, a, d] *= 1.0 if BITS[a, e] else -1.0
                else:
                    g[:, a, d] *= xi[:, e] if BITS[a, e] else 1.0 - xi[:, e]
    return g


def reference_stiffness():
    """Khat (8x8): unit-cube stiffness of Q1 (closed form)."""
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            s = 0.0
            for d in range(3):
                t = 1.0 if BITS[a, d] == BITS[b, d] else -1.0
                for e in range(3):
                    if e != d:
                        t *= (1.0 / 3.0) if BITS[a, e] == BITS[b, e] else (1.0 / 6.0)
                s += t
            K[a, b] = s
    return K


def reference_mass():
    """Mhat (8x8): unit-cube mass matrix of Q1 (closed form)."""
    M = np.ones((8, 8))
    for a in range(8):
        for b in range(8):
            for d in range(3):
                M[a, b] *= (1.0 / 3.0) if BITS[a, d] == BITS[b, d] else (1.0 / 6.0)
    return M


KHAT = reference_stiffness()
MHAT = reference_mass()


def _edge_point(P, F, u, v):
    t = F[u] / (F[u] - F[v])
    return P[u] + t * (P[v] - P[u])


def clip_tet(P, F):
    """Part {phi < 0} of the tet with vertices P (4,3), values F (4,).

    Returns (list of sub-tets (4,3), list of boundary triangles (3,3), normal)."""
    neg = [m for m in range(4) if F[m] < 0]
    pos = [m for m in range(4) if not F[m] < 0]
    k = len(neg)
    if k == 0:
        return [], [], None
    if k == 4:
        return [P.copy()], [], None
    D = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]])
    g = np.linalg.solve(D, np.array([F[1] - F[0], F[2] - F[0], F[3] - F[0]]))
    normal = g / np.linalg.norm(g)
    if k == 1:
        a = neg[0]
        b, c, d = pos
        pab, pac, pad = (_edge_point(P, F, a, x) for x in (b, c, d))
        return [np.stack([P[a], pab, pac, pad])], [np.stack([pab, pac, pad])], normal
    if k == 3:
        a, b, c = neg
        d = pos[0]
        pad, pbd, pcd = (_edge_point(P, F, x, d) for x in (a, b, c))
        A0, A1, A2, B0, B1, B2 = P[a], P[b], P[c], pad, pbd, pcd
        tets = [np.stack([A0, A1, A2, B0]), np.stack([A1, A2, B0, B1]), np.stack([A2, B0, B1, B2])]
        return tets, [np.stack([pad, pbd, pcd])], normal
    # k == 2
    a, b = neg
    c, d = pos
    pac, pad = _edge_point(P, F, a, c), _edge_point(P, F, a, d)
    pbc, pbd = _edge_point(P, F, b, c), _edge_point(P, F, b, d)
    A0, A1, A2, B0, B1, B2 = P[a], pac, pad, P[b], pbc, pbd
    tets = [np.stack([A0, A1, A2, B0]), np.stack([A1, A2, B0, B1]), np.stack([A2, B0, B1, B2])]
    tris = [np.stack([pac, pad, pbd]), np.stack([pac, pbd, pbc])]
    return tets, tris, normal


def integrate_cut_cell(phi8, f8, q8, h):
    """Element data of one cut cell.

    phi8: (8,) nodal level set; f8: (8,) nodal source; q8: (8,3) nodal flux or None.
    Returns (K (8,8), load (8,), eta) with K = int grad N_a . grad N_b over e cap Omega_h,
    load = int f_h N_a + int_{Gamma_h cap e} (q_h . n) N_a, eta = |e cap Omega_h| / |e|.
    """
    K, load, vol, _ = _cut_cell(phi8, f8, q8, h, None)
    return K, load, vol


def integrate_cut_cell_nitsche(phi8, f8, g8, h):
    """Element data of one cut cell whose unfitted boundary carries weak Dirichlet data
    (Sect. 2.2, Nitsche): K and load gain the Nitsche terms of oracle.nitsche with the Q1
    interpolant of g8.  Returns (K, load, eta, beta_e)."""
    return _cut_cell(phi8, f8, None, h, g8)


def _cut_cell(phi8, f8, q8, h, g8):
    K = np.zeros((8, 8))
    load = np.zeros(8)
    vol = 0.0
    facets = []
    for tet in KUHN_TETS:
        P = UNIT_VERTS[list(tet)]
        F = phi8[list(tet)]
        subtets, tris, normal = clip_tet(P, F)
        facets.extend((T, normal) for T in tris)
        for T in subtets:
            v = abs(np.linalg.det(np.stack([T[1] - T[0], T[2] - T[0], T[3] - T[0]]))) / 6.0
            if v == 0.0:
                continue
            xq = TET_BARY @ T                     # (m, 3)
            wq = TET_W * v
            G = q1_grad(xq)                       # (m, 8, 3)
            N = q1_shape(xq)                      # (m, 8)
            K += np.einsum("q,qad,qbd->ab", wq, G, G)
            load += (wq * (N @ f8)) @ N * h ** 3
            vol += v
        if q8 is not None:
            for T in tris:
                area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
                if area == 0.0:
                    continue
                xq = TRI_BARY @ T
                wq = TRI_W * area
                N = q1_shape(xq)
                gq = (N @ q8) @ normal            # (m,) q_h . n
                load += (wq * gq) @ N * h ** 2
    beta = 0.0
    if g8 is not None:
        from .nitsche import nitsche_cell
        Nmat, nload, beta = nitsche_cell(K, facets, np.asarray(g8, dtype=np.float64), h)
        return K * h + Nmat, load + nload, vol, beta
    return K * h, load, vol, beta


class Integration:
    """Element data of every active cell of a mesh (Sect. 2.2).

    ``map_fn(func, args)`` (default: the builtin map over argument tuples) evaluates
    integrate_cut_cell over the cut cells; a process pool's starmap runs the cells on
    several host cores with the same arithmetic per cell."""

    def __init__(self, mesh, problem, map_fn=None):
        g = mesh.grid
        self.h = g.h
        phi = mesh.phi
        f = np.asarray(problem.f, dtype=np.float64)
        q = None if problem.q is None else np.asarray(problem.q, dtype=np.float64)
        self.cut_cells = np.flatnonzero(mesh.cell_type == CUT)
        n_cut = self.cut_cells.size
        self.K_cut = np.zeros((n_cut, 8, 8))
        self.load_cut = np.zeros((n_cut, 8))
        self.eta = np.zeros(n_cut)
        weak = bool(getattr(problem, "weak_dirichlet", False))
        gd = None if not weak else np.asarray(problem.dirichlet_values, dtype=np.float64)
        args = []
        for c in self.cut_cells:
            nodes = g.cell_nodes(c)
            if weak:
                args.append((phi[nodes], f[nodes], gd[nodes], g.h))
            else:
                args.append((phi[nodes], f[nodes], None if q is None else q[nodes], g.h))
        fn = integrate_cut_cell_nitsche if weak else integrate_cut_cell
        if map_fn is None:
            results = [fn(*a) for a in args]
        else:
            results = map_fn(fn, args)
        self.beta = np.zeros(n_cut)
        for idx, res in enumerate(results):
            self.K_cut[idx] = res[0]
            self.load_cut[idx] = res[1]
            self.eta[idx] = res[2]
            if weak:
                self.beta[idx] = res[3]
        self.cut_index = {int(c): i for i, c in enumerate(self.cut_cells)}
        self.f = f
        self.kappa = (np.ones(g.n_cells) if problem.kappa is None
                      else np.asarray(problem.kappa, dtype=np.float64))
        self.cell_type = mesh.cell_type
        self.grid = g

    def unit_stiffness(self, c):
        """K_e without the coefficient (h Khat for internal cells)."""
        if self.cell_type[c] == INTERNAL:
            return self.h * KHAT
        return self.K_cut[self.cut_index[int(c)]]

    def stiffness(self, c):
        return self.kappa[c] * self.unit_stiffness(c)

    def load(self, c):
        if self.cell_type[c] == INTERNAL:
            nodes = self.grid.cell_nodes(c)
            return self.h ** 3 * (MHAT @ self.f[nodes])
        return self.load_cut[self.cut_index[int(c)]]
