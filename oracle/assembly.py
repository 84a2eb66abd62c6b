"""Global operator and right-hand side (oracle; test infrastructure only).

Sect. 2.2: A = sum_e A_e and b = f + g^N summed element by element over the
active cells; strong Dirichlet values on box-face nodes and the pinned node
(Sect. 5.1) are moved to the right-hand side:  b_F = (sum_e b_e)_F - A_FC g_C.
Box faces without a Dirichlet condition carry homogeneous Neumann data.

Parity: the linear patch test (a linear u with matching flux data is reproduced
exactly on plane-cut meshes) and symmetry / positive definiteness of A pin this
module (tests/test_oracle_integration.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import EXTERNAL


class System:
    """Assembled FP64 system over the free DOFs."""

    def __init__(self, mesh, integ, problem):
        g = mesh.grid
        rows, cols, vals = [], [], []
        bfull = np.zeros(g.n_nodes)
        for c in np.flatnonzero(mesh.cell_type != EXTERNAL):
            nodes = np.array(g.cell_nodes(c))
            Ke = integ.stiffness(c)
            rows.append(np.repeat(nodes, 8))
            cols.append(np.tile(nodes, 8))
            vals.append(Ke.ravel())
            bfull[nodes] += integ.load(c)
        A_full = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(g.n_nodes, g.n_nodes)).tocsr()
        free = mesh.node_of_dof
        cons = np.flatnonzero(mesh.constrained)
        gvals = (np.zeros(cons.size) if problem.dirichlet_values is None
                 else np.asarray(problem.dirichlet_values, dtype=np.float64)[cons])
        self.A = A_full[free][:, free].tocsr()
        self.b = bfull[free] - A_full[free][:, cons] @ gvals
        self.constrained_nodes = cons
        self.constrained_values = gvals
        self.n = free.size

    def apply(self, x):
        return self.A @ x

    def full_solution(self, mesh, x):
        """Nodal vector with the free values x and the constrained values."""
        u = np.full(mesh.grid.n_nodes, np.nan)
        u[mesh.node_of_dof] = x
        u[self.constrained_nodes] = self.constrained_values
        return u
