"""Pins for the oracle's three-level BDDC (reading R26 of the multilevel construction).

* the level-2 objects of a full box, counted by hand: 16^3 cells in 4^3-cell blocks
  (64 subdomains, 279 coarse DOFs: 27 corners, 108 edges, 144 faces), groups of
  2 x 2 x 2 blocks: the three mid planes carry 127 coarse DOFs, split into the centre
  corner, 6 half-lines (edges of 3 coarse DOFs: two first-level edges and the corner
  between them) and 12 quadrants (faces of 9: four first-level faces, four edges and
  one corner);
* one level-2 subdomain (no level-2 interface) and the all-corner level-2 space both
  make M_2 = A_c^-1, so the three-level M is the two-level M;
* C_2 Phi_2 = I on every level-2 subdomain and the level-2 weights sum to one;
* M_2 is symmetric with lambda_min(M_2 A_c) >= 1 (the Sect. 3.4 argument one level
  up), so M_3 >= M and the eigenvalues of M_3 A bound those of M A from above in order;
* the option keeping first-level corners as level-2 corners, counted by hand on the
  same box;
* elasticity: one type of first-level coarse DOF per level-2 object, and the same
  properties on three elastic cases.
"""
import numpy as np
import pytest

from oracle.assembly import System
from oracle.bddc import BDDC
from oracle.integration import Integration
from oracle.mesh import CORNER, EDGE, FACE, Mesh
from oracle.multilevel import CoarseBDDC, ThreeLevelBDDC
from oracle.pcg import pcg
from paper_1703_06323_gb300 import inputs


def _bddc(p, **kw):
    m = Mesh(p)
    integ = Integration(m, p)
    S = System(m, integ, p)
    return m, S, BDDC(m, integ, S, **kw)


@pytest.fixture(scope="module")
def box():
    return _bddc(inputs.box_problem(cells=(16, 16, 16), sub_cells=(4, 4, 4), dirichlet_face_mask=inputs.ALL_FACES))


@pytest.fixture(scope="module")
def tiny():
    """Sphere in 8^3 cells with 4^3-cell blocks: 8 subdomains, each its own group."""
    p = inputs.sphere_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), centre=(0.52, 0.47, 0.5), radius=0.41)
    return _bddc(p)


@pytest.fixture(scope="module")
def sbox():
    """Whole box, 8^3 cells in 2^3-cell blocks (64 subdomains, 343 DOFs): with groups of
    2^3 blocks the level-2 objects hold several coarse DOFs (an inexact level 2)."""
    return _bddc(inputs.box_problem(cells=(8, 8, 8), sub_cells=(2, 2, 2), dirichlet_face_mask=inputs.ALL_FACES))


@pytest.fixture(scope="module")
def tower():
    """A wavy cylinder through 8 z layers of 4^3-cell blocks (pure Neumann, pinned)."""
    from tests.oracle_cache import small_problems
    return _bddc(small_problems()["tower"])


def test_full_box_objects_by_hand(box):
    m, S, B = box
    assert m.n_sub == 64 and B.n_coarse == 27 + 108 + 144
    L2 = CoarseBDDC(B, group=2)
    assert L2.n_sub2 == 8
    assert int(L2.is_gamma.sum()) == 127
    kinds = [o["kind"] for o in L2.objs]
    sizes = sorted(len(o["dofs"]) for o in L2.objs)
    assert kinds.count(CORNER) == 1 and kinds.count(EDGE) == 6 and kinds.count(FACE) == 12
    assert sizes == [1] + [3] * 6 + [9] * 12
    assert all(len(o["neigh"]) == {CORNER: 8, EDGE: 4, FACE: 2}[o["kind"]] for o in L2.objs)
    assert CoarseBDDC(B, group=2, coarse="ce").n_coarse == 7
    assert CoarseBDDC(B, group=2, coarse="c").n_coarse == 1
    # first-level corners kept as level-2 corners: the 3 x 3 block vertices of each mid
    # plane, 3 x 9 - 3 x 3 + 1 = 19 distinct (the centre lines' 3 each lie on two planes,
    # the centre on three): the centre, 6 on the half-lines, 12 quadrant centres.  The
    # two first-level edges of a half-line were joined only through the corner between
    # them, so each becomes a one-DOF corner (12 more); each quadrant keeps its 4 faces
    # and 4 edges as one face of 8
    L2c = CoarseBDDC(B, group=2, level1_corners=True)
    got = sorted((o["kind"], len(o["dofs"]), len(o["neigh"])) for o in L2c.objs)
    assert got == sorted([(CORNER, 1, 8)] + [(CORNER, 1, 4)] * 18 + [(CORNER, 1, 2)] * 12 + [(FACE, 8, 2)] * 12)
    assert int(L2c.is_gamma.sum()) == 127


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["tiny", "tower"])
def test_exact_level2_reproduces_two_level(case, request):
    m, S, B = request.getfixturevalue(case)
    r = np.random.default_rng(1).normal(size=m.n_dof)
    ref = B.apply(r)
    one = ThreeLevelBDDC(B, group=64)
    assert one.level2.n_sub2 == 1 and not one.level2.is_gamma.any()
    assert _rel(one.apply(r), ref) <= 1e-12
    corners = ThreeLevelBDDC(B, group=1, all_interface_corners=True)
    assert corners.level2.n_sub2 > 1
    assert _rel(corners.apply(r), ref) <= 1e-10


@pytest.mark.parametrize("case,group", [("tiny", 1), ("tower", 1), ("tower", 2), ("box", 2)])
@pytest.mark.parametrize("level1_corners", [False, True])
def test_constraints_and_weights(case, group, level1_corners, request):
    m, S, B = request.getfixturevalue(case)
    L2 = CoarseBDDC(B, group=group, level1_corners=level1_corners)
    assert L2.n_sub2 > 1 and L2.n_coarse > 0
    for L in L2.local:
        if L["cids"].size:
            assert np.abs(L["C"] @ L["Phi"] - np.eye(L["cids"].size)).max() <= 1e-11
    assert np.abs(L2.weight_sums() - 1.0).max() <= 1e-14


@pytest.mark.parametrize("case,group", [("sbox", 2), ("tower", 1), ("tower", 2)])
@pytest.mark.parametrize("level1_corners", [False, True])
def test_level2_spectrum(case, group, level1_corners, request):
    """M_2 symmetric positive definite with lambda_min(M_2 A_c) >= 1 (and > 1 somewhere:
    these level-2 spaces are genuinely smaller than the assembled one)."""
    m, S, B = request.getfixturevalue(case)
    L2 = CoarseBDDC(B, group=group, level1_corners=level1_corners)
    n = L2.n
    M2 = np.column_stack([L2.apply(e) for e in np.eye(n)])
    assert np.abs(M2 - M2.T).max() <= 1e-10 * np.abs(M2).max()
    ev = np.sort(np.linalg.eigvals(M2 @ B.Ac).real)
    assert ev[0] >= 1.0 - 1e-9
    if any(len(o["dofs"]) > 1 for o in L2.objs):
        assert ev[-1] > 1.0 + 1e-3   # means over several coarse DOFs: a genuinely inexact coarse solve
    else:
        assert ev[-1] <= 1.0 + 1e-9  # every level-2 object a single coarse DOF: M_2 = A_c^-1


def test_three_level_dominates_two_level(sbox):
    """M_3 >= M: the ordered eigenvalues of M_3 A are at least those of M A, and
    both start at 1; PCG with M_3 reaches the same solution."""
    m, S, B = sbox
    T = ThreeLevelBDDC(B, group=2)
    A = S.A.toarray() if hasattr(S.A, "toarray") else np.asarray(S.A)
    n = m.n_dof
    E = np.eye(n)
    M = np.column_stack([B.apply(e) for e in E])
    M3 = np.column_stack([T.apply(e) for e in E])
    assert np.abs(M3 - M3.T).max() <= 1e-9 * np.abs(M3).max()
    e2 = np.sort(np.linalg.eigvals(M @ A).real)
    e3 = np.sort(np.linalg.eigvals(M3 @ A).real)
    assert e2[0] >= 1.0 - 1e-8 and e3[0] >= 1.0 - 1e-8
    assert np.all(e3 >= e2 - 1e-8 * e2[-1]) and e3[-1] > e2[-1] * (1 + 1e-3)
    r2 = pcg(S.apply, S.b, B.apply, rtol=1e-10)
    r3 = pcg(S.apply, S.b, T.apply, rtol=1e-10)
    assert r3["converged"] and r3["iterations"] > r2["iterations"]
    assert np.linalg.norm(r3["x"] - r2["x"]) <= 1e-8 * np.linalg.norm(r2["x"])


@pytest.mark.parametrize("name,group", [("el_sphere8", 1), ("el_wall", 1), ("el_wall", 2)])
def test_elastic_level2(name, group):
    """Elasticity (reading R20 rows: component means, rotation moments): every level-2
    object holds first-level coarse DOFs of one type only, C_2 Phi_2 = I, the weights
    sum to one, M_2 is symmetric with lambda_min(M_2 A_c) >= 1, and PCG with the
    three-level preconditioner reaches the two-level solution."""
    from oracle.multilevel import coarse_dof_types
    from tests.oracle_cache import oracle_run
    orc = oracle_run(name)
    B = orc.bddc()
    L2 = CoarseBDDC(B, group=group)
    types = coarse_dof_types(B)
    assert set(types) <= set(range(6)) and {0, 1, 2} <= set(types)
    assert all(len({types[k] for k in o["dofs"]}) == 1 for o in L2.objs)
    for L in L2.local:
        if L["cids"].size:
            assert np.abs(L["C"] @ L["Phi"] - np.eye(L["cids"].size)).max() <= 1e-10
    assert np.abs(L2.weight_sums() - 1.0).max() <= 1e-14
    M2 = np.column_stack([L2.apply(e) for e in np.eye(L2.n)])
    assert np.abs(M2 - M2.T).max() <= 1e-8 * np.abs(M2).max()
    ev = np.sort(np.linalg.eigvals(M2 @ B.Ac).real)
    assert ev[0] >= 1.0 - 1e-8 and ev[-1] > 1.0 + 1e-3
    T = ThreeLevelBDDC(B, group=group)
    r2 = pcg(orc.sys.apply, orc.sys.b, B.apply, rtol=1e-10, maxit=2000)
    r3 = pcg(orc.sys.apply, orc.sys.b, T.apply, rtol=1e-10, maxit=2000)
    assert r3["converged"]
    assert np.linalg.norm(r3["x"] - r2["x"]) <= 1e-7 * np.linalg.norm(r2["x"])
