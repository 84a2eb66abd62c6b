"""Pins for the oracle's adjoint gradient: central finite differences of J."""
import numpy as np

from oracle import adjoint as AD
from oracle.assembly import System
from oracle.integration import Integration
from oracle.mesh import Mesh
from paper_1703_06323_gb300 import inputs


def _kappa_problem(seed=0):
    p = inputs.sphere_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), centre=(0.51, 0.48, 0.5), radius=0.37,
                              dirichlet_face_mask=0, pin_node=inputs.PIN_AUTO)
    p.kappa = inputs.random_field_kappa(p.cells, seed=seed, ell=0.3)
    p.f = np.ones(p.n_nodes)
    p.q = None
    p.dirichlet_values = np.full(p.n_nodes, 0.25)     # nonzero pin value exercises the lift
    return p


def _J(p, u_d_nodal, weights=None):
    m = Mesh(p)
    integ = Integration(m, p)
    S = System(m, integ, p)
    x = AD.direct_solve(S)
    w = AD.lumped_mass(m, integ) if weights is None else weights
    return AD.objective(x, u_d_nodal[m.node_of_dof], w), (m, integ, S, x, w)


def test_lumped_mass_sums_to_domain_volume():
    p = _kappa_problem()
    p.dirichlet_values = None
    m = Mesh(p)
    integ = Integration(m, p)
    w = AD.lumped_mass(m, integ)
    vol = ((m.cell_type == 2).sum() + integ.eta.sum()) * m.grid.h ** 3
    # the pinned node is not a DOF: its share is missing from the sum
    assert 0 < vol - w.sum() < 8 * m.grid.h ** 3 / 8 + 1e-15
    assert (w > 0).all()


def test_adjoint_gradient_matches_central_differences():
    p = _kappa_problem()
    X, Y, Z = inputs.node_coords(p.box_lo, p.box_hi, p.cells)
    u_d = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    J0, (m, integ, S, x, w) = _J(p, u_d)
    lam = AD.direct_solve(S, w * (x - u_d[m.node_of_dof]))
    grad = AD.kappa_gradient(m, integ, S, x, lam)
    rng = np.random.default_rng(4)
    active = np.flatnonzero(m.cell_type != 0)
    cells = rng.choice(active, 8, replace=False)
    cut = np.flatnonzero(m.cell_type == 1)
    cells = np.concatenate([cells, cut[:3]])
    for c in cells:
        d = 1e-5 * p.kappa[c]
        kp, km = p.kappa.copy(), p.kappa.copy()
        kp[c] += d
        km[c] -= d
        p.kappa = kp
        Jp, _ = _J(p, u_d, w)
        p.kappa = km
        Jm, _ = _J(p, u_d, w)
        p.kappa = (kp + km) / 2
        fd = (Jp - Jm) / (2 * d)
        # central differences: O(d^2) truncation plus rounding of J / d
        assert abs(fd - grad[c]) <= 1e-5 * abs(fd) + 1e-6 * np.abs(grad).max(), (c, fd, grad[c])
    assert np.all(grad[m.cell_type == 0] == 0)
