"""Pins of the weak-Dirichlet (Nitsche) oracle, Sect. 2.2.

* C_e (the largest eigenvalue of B_e x = lambda D_e x on the complement of the
  constants) against an independent computation: the largest eigenvalue of
  pinv(D_e) B_e, whose nonzero spectrum is the same; no random vector has a larger
  Rayleigh quotient;
* the constants lie in the kernel of D_e and of B_e (n . grad of a constant is zero);
* beta_e = 2 C_e makes every cut-cell form coercive with A_e - D_e / 2 >= 0 (Young's
  inequality with the constant C_e);
* consistency: a linear u with its own values as weak Dirichlet data on a plane cut (and
  strong data on the box faces) is reproduced exactly by the discrete solution;
* a manufactured solution on a sphere with weak Dirichlet data everywhere on the
  unfitted boundary converges at second order in the nodal error.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import integration as IN
from oracle import nitsche as NI
from oracle.assembly import System
from oracle.integration import Integration
from oracle.mesh import Mesh
from paper_1703_06323_gb300 import inputs


def _cut_cells(seed, count):
    """Random cut cells: nodal level sets of random planes and spheres through the unit cube."""
    rng = np.random.default_rng(seed)
    V = IN.UNIT_VERTS
    out = []
    while len(out) < count:
        if rng.random() < 0.5:
            n = rng.normal(size=3)
            phi = V @ n - (0.5 * n.sum() + rng.uniform(-0.6, 0.6) * np.linalg.norm(n))
        else:
            c = rng.uniform(-0.5, 1.5, 3)
            phi = np.linalg.norm(V - c, axis=1) - rng.uniform(0.3, 1.2)
        if (phi < 0).any() and not (phi < 0).all():
            out.append(phi)
    return out


def _forms(phi8):
    """(D_unit, facets) of one cut cell through the oracle's marching tetrahedra."""
    facets = []
    for tet in IN.KUHN_TETS:
        _, tris, normal = IN.clip_tet(IN.UNIT_VERTS[list(tet)], phi8[list(tet)])
        facets.extend((T, normal) for T in tris)
    D, _, _ = IN.integrate_cut_cell(phi8, np.zeros(8), None, 1.0)
    return D, facets


def test_nitsche_constant_against_pseudo_inverse_and_rayleigh_quotients():
    rng = np.random.default_rng(5)
    for phi8 in _cut_cells(1, 25):
        D, facets = _forms(phi8)
        M, C, B = NI.facet_forms(facets)
        if not np.any(B):
            continue
        ce = NI.nitsche_constant(D, B)
        ref = np.max(np.linalg.eigvals(np.linalg.pinv(D, rcond=1e-13) @ B).real)
        assert ce > 0 and abs(ce - ref) <= 1e-7 * ref, (ce, ref)
        X = rng.normal(size=(400, 8))
        rq = np.einsum("ia,ab,ib->i", X, B, X) / np.einsum("ia,ab,ib->i", X, D, X)
        assert rq.max() <= ce * (1 + 1e-10)


def test_constants_in_the_kernel_and_coercivity_with_beta_two_ce():
    for phi8 in _cut_cells(2, 25):
        D, facets = _forms(phi8)
        M, C, B = NI.facet_forms(facets)
        one = np.ones(8)
        scale = np.abs(D).max()
        assert np.abs(D @ one).max() <= 1e-12 * scale
        assert np.abs(B @ one).max() <= 1e-12 * max(np.abs(B).max(), 1e-300)
        assert np.abs(C @ one).max() <= 1e-12 * max(np.abs(C).max(), 1e-300)   # n . grad 1 = 0
        if not np.any(B):
            continue
        Nmat, _, beta = NI.nitsche_cell(D, facets, np.zeros(8), 1.0)
        assert beta == pytest.approx(2.0 * NI.nitsche_constant(D, B), rel=1e-14)
        A = D + Nmat
        w = np.linalg.eigvalsh(A - 0.5 * D)
        assert w.min() >= -1e-10 * np.abs(A).max()


def test_weak_dirichlet_linear_patch():
    """u = a + b.x is reproduced exactly: Nitsche's form is consistent (Sect. 2.2)."""
    p = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(0.6, 0.8, 0.1), offset=0.61,
                             dirichlet_face_mask=inputs.ALL_FACES, pin_node=inputs.PIN_NONE)
    p.q = None
    p.weak_dirichlet = True
    m = Mesh(p)
    integ = Integration(m, p)
    S = System(m, integ, p)
    u = p.u_exact[m.node_of_dof]
    # the linear u satisfies the discrete equations to rounding (a wrong sign or a missing
    # symmetric term in the boundary form leaves an O(1) residual) ...
    assert np.linalg.norm(S.A @ u - S.b) <= 1e-13 * np.linalg.norm(S.b)
    # ... and the solve returns it up to the conditioning of the small cuts
    x = spla.spsolve(S.A.tocsc(), S.b)
    assert np.abs(x - u).max() <= 1e-8
    assert np.all(integ.beta[np.abs(integ.beta) > 0] > 0)


def test_weak_dirichlet_sphere_second_order():
    errs = []
    for n in (16, 32):
        p = inputs.sphere_problem(cells=(n, n, n), sub_cells=(8, 8, 8), centre=(0.51, 0.49, 0.5), radius=0.4,
                                  dirichlet_face_mask=inputs.ALL_FACES, pin_node=inputs.PIN_NONE)
        p.q = None
        p.weak_dirichlet = True
        m = Mesh(p)
        S = System(m, Integration(m, p), p)
        x = spla.spsolve(S.A.tocsc(), S.b)
        inside = p.phi[m.node_of_dof] < 0
        errs.append(np.abs(x - p.u_exact[m.node_of_dof])[inside].max())
    assert errs[1] < errs[0] / 3.0, errs


def test_variant2_objects():
    """Sect. 4.5 objects: on an uncut box the stiffness weights are constant along every
    edge, so variant 2 leaves the standard objects unchanged; on a sphere with weak
    Dirichlet data the split edges make BDDC no worse than the standard and variant-1
    objects (the paper's robust choice for Nitsche, Sect. 5.2), and every variant-2
    edge carries constant weights."""
    from oracle.bddc import BDDC, stiffness_weights
    from oracle.mesh import EDGE
    from oracle.pcg import pcg
    box = inputs.box_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4))
    m = Mesh(box)
    integ = Integration(m, box)
    w = stiffness_weights(m, integ)
    assert m.objects("v2", weights=w) == m.objects("std")

    p = inputs.sphere_problem(cells=(16, 16, 16), sub_cells=(4, 4, 4), centre=(0.51, 0.49, 0.5), radius=0.4,
                              dirichlet_face_mask=inputs.ALL_FACES, pin_node=inputs.PIN_NONE)
    p.q = None
    p.weak_dirichlet = True
    m = Mesh(p)
    integ = Integration(m, p)
    S = System(m, integ, p)
    w = stiffness_weights(m, integ)
    v2 = m.objects("v2", weights=w)
    assert len(v2) > len(m.objects("std"))
    for o in v2:
        if o["kind"] == EDGE:
            for d in o["dofs"][1:]:
                assert max(abs(w[d][s] - w[o["dofs"][0]][s]) for s in o["neigh"]) <= 2e-8
    its = {ob: pcg(S.apply, S.b, BDDC(m, integ, S, objects=ob, coarse="cef").apply, rtol=1e-8)["iterations"]
           for ob in ("std", "v1", "v2")}
    assert its["v2"] <= its["v1"] <= its["std"], its
