"""Pins for the oracle's quadrature and cut-cell integration."""
import itertools
import math

import numpy as np
import pytest

from oracle import integration as IN
from oracle import quadrature as Q
from oracle.assembly import System
from oracle.mesh import Mesh, INTERNAL
from paper_1703_06323_gb300 import inputs


@pytest.mark.parametrize("n,bary,w", [(3, Q.TET_BARY, Q.TET_W), (2, Q.TRI_BARY, Q.TRI_W)])
def test_gm_rule_exact_on_simplex_moments(n, bary, w):
    """mean of prod lambda_j^a_j over the simplex = n! prod a_j! / (|a| + n)!  for |a| <= 7."""
    for a in itertools.product(range(8), repeat=n + 1):
        if sum(a) > 7:
            continue
        exact = math.factorial(n) * math.prod(math.factorial(x) for x in a) / math.factorial(sum(a) + n)
        q = float(w @ np.prod(bary ** np.array(a), axis=1))
        assert abs(q - exact) <= 1e-13 * exact


def test_closed_forms_match_direct_quadrature():
    """Khat and Mhat against quadrature on the unit cube (tensor Gauss, independent)."""
    g, gw = np.polynomial.legendre.leggauss(3)
    g = 0.5 * (g + 1)
    gw = 0.5 * gw
    pts = np.array(list(itertools.product(g, g, g)))
    wts = np.array([a * b * c for a, b, c in itertools.product(gw, gw, gw)])
    G = IN.q1_grad(pts)
    N = IN.q1_shape(pts)
    K = np.einsum("q,qad,qbd->ab", wts, G, G)
    Mm = np.einsum("q,qa,qb->ab", wts, N, N)
    assert np.allclose(K, IN.KHAT, atol=1e-15)
    assert np.allclose(Mm, IN.MHAT, atol=1e-15)
    # 27-point stencil of a node: centre 8/3 h, face 0, edge -1/6 h, corner -1/12 h
    assert np.isclose(8 * IN.KHAT[0, 0], 8.0 / 3.0)
    assert np.isclose(4 * IN.KHAT[0, 1], 0.0)
    assert np.isclose(2 * IN.KHAT[0, 3], -1.0 / 6.0)
    assert np.isclose(IN.KHAT[0, 7], -1.0 / 12.0)


def test_full_cell_through_tets_equals_closed_form():
    f8 = np.arange(8.0) - 3.0
    K, load, eta = IN.integrate_cut_cell(-np.ones(8), f8, None, 0.25)
    assert np.allclose(K, 0.25 * IN.KHAT, atol=1e-15)
    assert np.allclose(load, 0.25 ** 3 * IN.MHAT @ f8, atol=1e-15)
    assert abs(eta - 1.0) < 1e-14


@pytest.mark.parametrize("a", [0.1, 0.37, 0.5, 0.93])
def test_axis_plane_volume_exact(a):
    """phi = x - a inside one unit cell: the cut piece is the slab x < a, eta = a."""
    phi8 = np.array([x - a for (x, y, z) in IN.UNIT_VERTS])
    K, _, eta = IN.integrate_cut_cell(phi8, np.zeros(8), None, 1.0)
    assert abs(eta - a) < 1e-14
    # stiffness of the slab [0,a] x [0,1]^2: tensor closed form
    k1 = np.array([[1, -1], [-1, 1]]) / a              # int_0^a of dN/dx products (linear in x over [0,1]) scaled
    # direct check by 1D integrals: N_a = l_ax(x) l_ay(y) l_az(z) with l0 = 1-t, l1 = t
    def mx(i, j):
        f = lambda t: ((1 - t) if i == 0 else t) * ((1 - t) if j == 0 else t)
        return a * (f(0) + 4 * f(a / 2) + f(a)) / 6      # Simpson, exact for quadratics
    def kx(i, j):
        return a * ((-1 if i == 0 else 1) * (-1 if j == 0 else 1))
    m1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    Kx = np.zeros((8, 8))
    for p_, q_ in itertools.product(range(8), range(8)):
        bp, bq = IN.BITS[p_], IN.BITS[q_]
        Kx[p_, q_] = (kx(bp[0], bq[0]) * m1[bp[1], bq[1]] * m1[bp[2], bq[2]]
                      + mx(bp[0], bq[0]) * (1 if bp[1] == bq[1] else -1) * m1[bp[2], bq[2]]
                      + mx(bp[0], bq[0]) * m1[bp[1], bq[1]] * (1 if bp[2] == bq[2] else -1))
    assert np.allclose(K, Kx, atol=1e-14)
    del k1


@pytest.mark.parametrize("s", [0.05, 0.4, 1.0])
def test_corner_plane_volume_exact(s):
    """phi = x + y + z - s: the corner tet has volume s^3 / 6 (s <= 1)."""
    phi8 = np.array([x + y + z - s for (x, y, z) in IN.UNIT_VERTS])
    _, _, eta = IN.integrate_cut_cell(phi8, np.zeros(8), None, 1.0)
    assert abs(eta - s ** 3 / 6) < 1e-15


def test_tiny_corner_cut_fraction():
    s = 1e-3
    phi8 = np.array([x + y + z - s for (x, y, z) in IN.UNIT_VERTS])
    K, _, eta = IN.integrate_cut_cell(phi8, np.zeros(8), None, 1.0)
    assert abs(eta - s ** 3 / 6) < 1e-24
    assert abs(K.sum()) < 1e-18


def test_cut_matrices_zero_row_sums_and_psd():
    p = inputs.manufactured_sphere(0)
    m = Mesh(p)
    integ = IN.Integration(m, p)
    for K in integ.K_cut:
        scale = np.abs(K).max()
        assert np.abs(K.sum(axis=1)).max() <= 1e-13 * max(scale, 1e-300) + 1e-300
        assert np.allclose(K, K.T, rtol=0, atol=1e-14 * max(scale, 1e-300))
        assert np.linalg.eigvalsh(K).min() >= -1e-12 * scale
    assert (integ.eta > 0).all() and (integ.eta < 1).all()


def test_divergence_theorem_on_cut_facets():
    """sum_a of the Neumann load = int_Gamma q.n; for q = (x - x0, 0, 0) it equals |Omega_h|,
    for constant q it vanishes (closed surface strictly inside the box)."""
    p = inputs.manufactured_sphere(0)
    m = Mesh(p)
    g = m.grid
    X, Y, Z = inputs.node_coords(p.box_lo, p.box_hi, p.cells)
    total_vol = (m.cell_type == INTERNAL).sum() * g.h ** 3
    for qfield, expect in ((np.stack([X - 0.3, 0 * X, 0 * X], axis=1), "vol"),
                           (np.tile([0.3, -1.0, 0.7], (X.size, 1)), 0.0)):
        p2 = inputs.Problem(name="q", box_lo=p.box_lo, box_hi=p.box_hi, cells=p.cells, sub_cells=p.sub_cells,
                            phi=p.phi, f=np.zeros_like(X), q=qfield, pin_node=inputs.PIN_NONE)
        integ = IN.Integration(Mesh(p2), p2)
        flux = integ.load_cut.sum()
        if expect == "vol":
            vol = total_vol + integ.eta.sum() * g.h ** 3
            assert abs(flux - vol) < 1e-13
        else:
            assert abs(flux) < 1e-13


def test_sphere_volume_converges_second_order():
    errs = []
    for n in (16, 32):
        p = inputs.sphere_problem(cells=(n, n, n), centre=(0.5, 0.5, 0.5), radius=0.4)
        m = Mesh(p)
        integ = IN.Integration(m, p)
        vol = ((m.cell_type == INTERNAL).sum() + integ.eta.sum()) * m.grid.h ** 3
        errs.append(abs(vol - 4.0 / 3.0 * np.pi * 0.4 ** 3))
    assert errs[1] < errs[0] / 3.0


def test_linear_patch_test_on_plane_cut():
    """u = a + b.x with f = 0, g = b.n on the cut boundary and u = a + b.x on the box
    faces is reproduced exactly (Galerkin on the polyhedral Omega_h)."""
    import scipy.sparse.linalg as spla
    p = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(0.6, 0.8, 0.0), offset=0.53,
                             dirichlet_face_mask=inputs.ALL_FACES)
    m = Mesh(p)
    integ = IN.Integration(m, p)
    S = System(m, integ, p)
    ue = p.u_exact[m.node_of_dof]
    assert np.abs(S.A @ ue - S.b).max() < 1e-14 * np.abs(S.b).max() + 1e-15
    x = spla.spsolve(S.A.tocsc(), S.b)
    assert np.abs(x - ue).max() < 1e-9


def test_assembled_operator_symmetric_positive_definite():
    """A = sum_e A_e over the free DOFs is symmetric (to rounding: element entries
    (a, b) and (b, a) are summed separately) and positive definite.  With box
    Dirichlet data and cut fractions >= 1.8e-3 (plane cut) the smallest eigenvalue is
    clearly positive; on the pinned sphere, whose cut fractions reach 3e-9, it sits at
    the rounding level of the largest (the ill-conditioning of Sect. 4.1), so there
    the test is positive semi-definiteness to rounding."""
    plane = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(0.6, 0.8, 0.1), offset=0.61,
                                 dirichlet_face_mask=inputs.ALL_FACES)
    for p, floor in ((plane, 1e-10), (inputs.manufactured_sphere(0), -1e-14)):
        m = Mesh(p)
        integ = IN.Integration(m, p)
        A = System(m, integ, p).A.toarray()
        assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
        w = np.linalg.eigvalsh(0.5 * (A + A.T))
        assert w[0] > floor * w[-1]
