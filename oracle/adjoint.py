"""Adjoint gradient with respect to per-cell coefficients (oracle; test infrastructure only).

No counterpart in the paper.  With A(kappa) = sum_e kappa_e Khat_e over the free
DOFs, the residual R(u, kappa) = A_FF u_F + A_FC g_C - b_F = 0 and an objective
J(u_F), the adjoint lambda solves A_FF lambda = dJ/du_F (A is symmetric) and

    dJ/dkappa_e = -lambda_e^T Khat_e ubar_e,

ubar holding u at the free DOFs and the Dirichlet values g at constrained nodes,
lambda vanishing at constrained nodes.  The objective used for the coefficient
workload is the lumped-mass weighted misfit J = 1/2 sum_xi m_xi (u_xi - u_d,xi)^2,
m_xi = int_Omega phi_xi (a discrete L2(Omega) norm, reading R14): nodal values of
DOFs with tiny support are ill-determined (k(A) ~ eta^-7/3, Eq. finite-cell-estimate)
and the weights make J insensitive to them.  dJ/du = m (u - u_d).

Parity: pinned by central finite differences of J computed with direct solves
(tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .mesh import EXTERNAL


def objective(x, u_d, m=None):
    e = x - u_d
    return 0.5 * float(e @ e) if m is None else 0.5 * float(e @ (m * e))


def lumped_mass(mesh, integ):
    """m_xi = int_Omega phi_xi over the free DOFs (row sums of the cut mass matrix)."""
    from .integration import INTERNAL, MHAT, integrate_cut_cell
    g = mesh.grid
    m = np.zeros(g.n_nodes)
    for c in np.flatnonzero(mesh.cell_type != EXTERNAL):
        nodes = g.cell_nodes(c)
        if mesh.cell_type[c] == INTERNAL:
            m[nodes] += g.h ** 3 * MHAT.sum(axis=1)
        else:
            _, load, _ = integrate_cut_cell(mesh.phi[nodes], np.ones(8), None, g.h)
            m[nodes] += load
    return m[mesh.node_of_dof]


def kappa_gradient(mesh, integ, system, x, lam):
    """dJ/dkappa per cell (0 on external cells) from the forward and adjoint solutions."""
    g = mesh.grid
    ubar = np.zeros(g.n_nodes)
    ubar[mesh.node_of_dof] = x
    ubar[system.constrained_nodes] = system.constrained_values
    lbar = np.zeros(g.n_nodes)
    lbar[mesh.node_of_dof] = lam
    out = np.zeros(g.n_cells)
    for c in np.flatnonzero(mesh.cell_type != EXTERNAL):
        nodes = g.cell_nodes(c)
        out[c] = -(lbar[nodes] @ integ.unit_stiffness(c) @ ubar[nodes])
    return out


def direct_solve(system, rhs=None):
    return spla.spsolve(system.A.tocsc(), system.b if rhs is None else rhs)
