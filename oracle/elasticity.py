"""Unfitted Q1 linear elasticity (oracle; test infrastructure only).

The paper treats the Poisson problem only.  The vector-valued variant is the
same unfitted discretisation (Sect. 2.2: bulk form integrated over the cut part
of each active cell, natural boundary condition on the unfitted boundary, no
Nitsche terms) with the isotropic linear-elastic form in place of the Laplacian
(reading R19):

    a_e(u, v) = int_{e cap Omega_h}  lambda div u div v + 2 mu eps(u) : eps(v),
    lambda = E nu / ((1 + nu)(1 - 2 nu)),  mu = E / (2 (1 + nu)),

with u in Q1^3; the element DOF of vertex a (a = x + 2y + 4z) and component c
is 3 a + c, and the global DOF of free node d and component c is 3 d + c.
Loads: int f_h . N_a over the cut part (f_h the Q1 interpolant of nodal body
forces) plus int_{Gamma_h cap e} (sigma_h n) . N_a for a nodal stress field
sigma_h (the elastic analogue of the flux q of the Poisson problem; zero for a
traction-free boundary).

Internal cells use the closed form K = h Khat_el(lambda, mu), built from the 1-D
integrals int n_a' n_b' = s_a s_b, int n_a' n_b = s_a / 2, int n_a n_b = 1/3 or
1/6 (n_0 = 1 - x, n_1 = x, s_0 = -1, s_1 = +1); cut cells are integrated on the
same clipped Kuhn tetrahedra as the Poisson problem with the degree-7 tet rule
(the integrand has degree <= 4 there, so the integrals are exact up to rounding).

Parity: pinned (tests/test_oracle_elasticity.py) by the closed form against the
tet machinery on an uncut cell, the six rigid-body modes in the kernel of every
element matrix, symmetry and positive semi-definiteness, and the patch test: a
linear displacement with uniform stress is reproduced exactly on a plane-cut
mesh when its traction is prescribed on the cut boundary.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .integration import KUHN_TETS, UNIT_VERTS, clip_tet, q1_grad, q1_shape
from .mesh import CUT, EXTERNAL, INTERNAL, VERTEX_OFFSETS as BITS_OF_VERTEX
from .quadrature import TET_BARY, TET_W, TRI_BARY, TRI_W

NCOMP = 3


def lame(E, nu):
    """(lambda, mu) of an isotropic material."""
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def _one_d(a_bit, b_bit, da, db):
    """int_0^1 n_a^(da) n_b^(db) dx for the linear 1-D shape functions."""
    sa = 1.0 if a_bit else -1.0
    sb = 1.0 if b_bit else -1.0
    if da and db:
        return sa * sb
    if da:
        return sa / 2.0
    if db:
        return sb / 2.0
    return 1.0 / 3.0 if a_bit == b_bit else 1.0 / 6.0


def grad_grad_unit(a, b, i, j):
    """int over the unit cube of dN_a/dx_i dN_b/dx_j (tensor product of 1-D integrals)."""
    v = 1.0
    for d in range(3):
        v *= _one_d(BITS_OF_VERTEX[a][d], BITS_OF_VERTEX[b][d], d == i, d == j)
    return v


def reference_stiffness(lam, mu):
    """Khat_el (24x24) on the unit cube: closed form."""
    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            lap = sum(grad_grad_unit(a, b, d, d) for d in range(3))
            for i in range(3):
                for j in range(3):
                    # lambda d_i N_a d_j N_b + mu (d_j N_a d_i N_b + delta_ij grad N_a . grad N_b)
                    v = lam * grad_grad_unit(a, b, i, j) + mu * grad_grad_unit(a, b, j, i)
                    if i == j:
                        v += mu * lap
                    K[3 * a + i, 3 * b + j] = v
    return K


def _element_from_gradients(G, w, lam, mu):
    """sum_q w_q B_q^T D B_q for gradients G (m, 8, 3) of the shape functions."""
    lap = np.einsum("q,qad,qbd->ab", w, G, G)
    gij = np.einsum("q,qai,qbj->abij", w, G, G)        # int d_i N_a d_j N_b
    K = np.zeros((24, 24))
    for i in range(3):
        for j in range(3):
            blk = lam * gij[:, :, i, j] + mu * gij[:, :, j, i]
            if i == j:
                blk = blk + mu * lap
            K[i::3, j::3] = blk
    return K


def integrate_cut_cell(phi8, f8, s8, h, lam, mu):
    """Element data of one cut cell.

    phi8 (8,) nodal level set; f8 (8, 3) nodal body force; s8 (8, 3, 3) nodal
    stress for the boundary traction sigma n, or None.  Returns (K (24,24),
    load (24,), eta) with K = int B^T D B over e cap Omega_h and eta the volume
    fraction."""
    K = np.zeros((24, 24))
    load = np.zeros(24)
    vol = 0.0
    for tet in KUHN_TETS:
        P = UNIT_VERTS[list(tet)]
        F = phi8[list(tet)]
        subtets, tris, normal = clip_tet(P, F)
        for T in subtets:
            v = abs(np.linalg.det(np.stack([T[1] - T[0], T[2] - T[0], T[3] - T[0]]))) / 6.0
            if v == 0.0:
                continue
            xq = TET_BARY @ T
            wq = TET_W * v
            K += _element_from_gradients(q1_grad(xq), wq, lam, mu)
            N = q1_shape(xq)                               # (m, 8)
            fq = N @ f8                                    # (m, 3)
            load += np.einsum("q,qa,qc->ac", wq, N, fq).ravel() * h ** 3
            vol += v
        if s8 is not None:
            for T in tris:
                area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
                if area == 0.0:
                    continue
                xq = TRI_BARY @ T
                wq = TRI_W * area
                N = q1_shape(xq)
                sq = np.einsum("qa,aij->qij", N, s8)       # (m, 3, 3)
                tq = sq @ normal                           # traction sigma n
                load += np.einsum("q,qa,qc->ac", wq, N, tq).ravel() * h ** 2
    return K * h, load, vol


class ElasticIntegration:
    """Element data of every active cell (24x24 stiffness, 24 loads)."""

    def __init__(self, mesh, problem):
        g = mesh.grid
        self.h = g.h
        E, nu = problem.lame
        self.lam, self.mu = lame(E, nu)
        self.khat = reference_stiffness(self.lam, self.mu)
        phi = mesh.phi
        f = np.asarray(problem.f, dtype=np.float64).reshape(g.n_nodes, 3)
        s = None if problem.q is None else np.asarray(problem.q, dtype=np.float64).reshape(g.n_nodes, 3, 3)
        self.f = f
        self.cut_cells = np.flatnonzero(mesh.cell_type == CUT)
        n_cut = self.cut_cells.size
        self.K_cut = np.zeros((n_cut, 24, 24))
        self.load_cut = np.zeros((n_cut, 24))
        self.eta = np.zeros(n_cut)
        for idx, c in enumerate(self.cut_cells):
            nodes = g.cell_nodes(c)
            Ke, le, eta = integrate_cut_cell(phi[nodes], f[nodes], None if s is None else s[nodes], g.h,
                                             self.lam, self.mu)
            self.K_cut[idx] = Ke
            self.load_cut[idx] = le
            self.eta[idx] = eta
        self.cut_index = {int(c): i for i, c in enumerate(self.cut_cells)}
        self.kappa = (np.ones(g.n_cells) if problem.kappa is None
                      else np.asarray(problem.kappa, dtype=np.float64))
        self.cell_type = mesh.cell_type
        self.grid = g

    def unit_stiffness(self, c):
        if self.cell_type[c] == INTERNAL:
            return self.h * self.khat
        return self.K_cut[self.cut_index[int(c)]]

    def stiffness(self, c):
        return self.kappa[c] * self.unit_stiffness(c)

    def load(self, c):
        if self.cell_type[c] == INTERNAL:
            nodes = self.grid.cell_nodes(c)
            M = _unit_mass()
            return (self.h ** 3 * (M @ self.f[nodes])).ravel()
        return self.load_cut[self.cut_index[int(c)]]


def _unit_mass():
    M = np.ones((8, 8))
    for a in range(8):
        for b in range(8):
            for d in range(3):
                M[a, b] *= (1.0 / 3.0) if BITS_OF_VERTEX[a][d] == BITS_OF_VERTEX[b][d] else (1.0 / 6.0)
    return M


def element_dofs(nodes):
    """Global-node element DOF ids (3 node + c) in element order 3 a + c."""
    nodes = np.asarray(nodes, dtype=np.int64)
    return (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()


class ElasticSystem:
    """Assembled FP64 elasticity system over the free DOFs (3 per free node)."""

    ncomp = NCOMP

    def __init__(self, mesh, integ, problem):
        g = mesh.grid
        rows, cols, vals = [], [], []
        bfull = np.zeros(3 * g.n_nodes)
        for c in np.flatnonzero(mesh.cell_type != EXTERNAL):
            ed = element_dofs(g.cell_nodes(c))
            Ke = integ.stiffness(c)
            rows.append(np.repeat(ed, 24))
            cols.append(np.tile(ed, 24))
            vals.append(Ke.ravel())
            bfull[ed] += integ.load(c)
        n3 = 3 * g.n_nodes
        A_full = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(n3, n3)).tocsr()
        free = element_dofs(mesh.node_of_dof)              # 3 d + c over the free nodes
        cons_nodes = np.flatnonzero(mesh.constrained)
        cons = element_dofs(cons_nodes)
        gvals = (np.zeros(cons.size) if problem.dirichlet_values is None
                 else np.asarray(problem.dirichlet_values, dtype=np.float64).reshape(g.n_nodes, 3)[cons_nodes].ravel())
        self.A = A_full[free][:, free].tocsr()
        self.b = bfull[free] - A_full[free][:, cons] @ gvals
        self.constrained_nodes = cons_nodes
        self.constrained_values = gvals.reshape(-1, 3)
        self.n = free.size

    def apply(self, x):
        return self.A @ x

    def full_solution(self, mesh, x):
        """Nodal (n_nodes, 3) displacement with the free values x and the constrained values."""
        u = np.full((mesh.grid.n_nodes, 3), np.nan)
        u[mesh.node_of_dof] = x.reshape(-1, 3)
        u[self.constrained_nodes] = self.constrained_values
        return u


def rigid_body_modes(points):
    """(3 m, 6) translations and infinitesimal rotations at points (m, 3), DOF order 3 i + c."""
    m = points.shape[0]
    R = np.zeros((3 * m, 6))
    for c in range(3):
        R[c::3, c] = 1.0
    x, y, z = points[:, 0], points[:, 1], points[:, 2]
    # rotation about x: (0, -z, y); about y: (z, 0, -x); about z: (-y, x, 0)
    R[1::3, 3], R[2::3, 3] = -z, y
    R[0::3, 4], R[2::3, 4] = z, -x
    R[0::3, 5], R[1::3, 5] = -y, x
    return R
