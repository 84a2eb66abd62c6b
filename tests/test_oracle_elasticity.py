"""Pins for the oracle's unfitted Q1 elasticity and its BDDC (vector DOFs)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import elasticity as EL
from oracle.bddc import BDDC, object_rows
from oracle.mesh import CORNER, EDGE, FACE, Mesh
from oracle.pcg import pcg
from paper_1703_06323_gb300 import inputs


def _small_sphere(cells=(8, 8, 8), sub=(4, 4, 4), centre=(0.2, 0.5, 0.5), radius=0.42):
    """A sphere crossing the clamped face x = 0, body force (0, 0, -1)."""
    X, Y, Z = inputs.node_coords((0, 0, 0), (1, 1, 1), cells)
    c = np.asarray(centre)
    phi = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - radius
    f = np.zeros((X.size, 3))
    f[:, 2] = -1.0
    return inputs.Problem(name="el_small", box_lo=np.zeros(3), box_hi=np.ones(3), cells=cells, sub_cells=sub,
                          phi=phi, f=f, q=None, dirichlet_face_mask=inputs.FACE_XLO, pin_node=inputs.PIN_NONE,
                          dirichlet_values=np.zeros((X.size, 3)), ncomp=3, lame=(1.0, 0.3))


def _build(p):
    m = Mesh(p)
    integ = EL.ElasticIntegration(m, p)
    S = EL.ElasticSystem(m, integ, p)
    return m, integ, S


def test_closed_form_matches_tet_quadrature_on_an_uncut_cell():
    lam, mu = EL.lame(2.5, 0.27)
    K = EL.reference_stiffness(lam, mu)
    Kq, load, vol = EL.integrate_cut_cell(-np.ones(8), np.zeros((8, 3)), None, 1.0, lam, mu)
    assert vol == pytest.approx(1.0, abs=1e-14)
    assert np.abs(K - Kq).max() <= 1e-14 * np.abs(K).max()
    # a hand value: the diagonal entry of vertex 0, component x of the unit cube
    # lam * (1/3 * 1/3 * 1) / ... : d_x N_0 d_x N_0 integrates to 1 * 1/3 * 1/3 = 1/9;
    # K[0,0] = (lam + mu) / 9 + mu * (3 / 9) = (lam + 2 mu) / 9 + 2 mu / 9
    assert K[0, 0] == pytest.approx((lam + 2 * mu) / 9 + 2 * mu / 9, rel=1e-14)


def test_rigid_modes_symmetry_and_psd_of_every_cut_cell():
    p = _small_sphere()
    m, integ, _ = _build(p)
    pts = np.array(EL.BITS_OF_VERTEX, dtype=np.float64)
    R = EL.rigid_body_modes(pts)
    assert integ.K_cut.shape[0] > 50
    for Ke in integ.K_cut:
        scale = np.abs(Ke).max()
        assert np.abs(Ke - Ke.T).max() <= 1e-14 * scale
        assert np.abs(Ke @ R).max() <= 1e-12 * scale
        assert np.linalg.eigvalsh(Ke).min() >= -1e-12 * scale


def test_body_force_load_integrates_to_the_volume():
    p = _small_sphere()
    m, integ, S = _build(p)
    h = m.grid.h
    vol = ((m.cell_type == 2).sum() + integ.eta.sum()) * h ** 3
    tot = np.zeros(3)
    for c in np.flatnonzero(m.cell_type != 0):
        tot += integ.load(c).reshape(8, 3).sum(axis=0)
    assert tot[:2] == pytest.approx([0.0, 0.0], abs=1e-15)
    assert tot[2] == pytest.approx(-vol, rel=1e-13)


def test_patch_test_reproduces_a_linear_displacement():
    p = inputs.elastic_patch()
    m, integ, S = _build(p)
    ue = p.u_exact[m.node_of_dof].ravel()
    # Galerkin exactness: the linear field satisfies the discrete equations
    res = S.A @ ue - S.b
    assert np.abs(res).max() <= 1e-13 * np.abs(S.b).max()
    # and a direct solve recovers it (to the conditioning of the cut system)
    x = spla.spsolve(S.A.tocsc(), S.b)
    assert np.abs(x - ue).max() <= 1e-8 * np.abs(ue).max()
    # the same problem without the prescribed traction is not reproduced
    p.q = None
    m2, integ2, S2 = _build(p)
    assert np.abs(S2.A @ ue - S2.b).max() > 1e-4 * np.abs(S.b).max()


def test_object_rows_against_the_inertia_closed_form():
    p = _small_sphere()
    m = Mesh(p)
    objs = m.objects("v1")
    kinds = {CORNER: 0, EDGE: 0, FACE: 0}
    for o in objs:
        rows = object_rows(o, m.grid, m, 3)
        nodes = [int(d) for d in o["dofs"]]
        ijk = np.array([m.grid.node_ijk(int(m.node_of_dof[d])) for d in nodes], dtype=np.float64)
        y = ijk - ijk.mean(axis=0)
        n = len(nodes)

        def apply(row, field):            # field (n, 3) at the object's nodes
            return sum(wt * field[nodes.index(d), c] for (d, c), wt in row.items())

        # translations: the first three rows are the component means
        for c in range(3):
            t = np.zeros((n, 3))
            t[:, c] = 1.0
            assert [apply(r, t) for r in rows[:3]] == pytest.approx(np.eye(3)[c], abs=1e-15)
            assert all(abs(apply(r, t)) <= 1e-15 for r in rows[3:])
        # rotations: (1/n) sum y x (omega x y) = J omega / n with J = sum |y|^2 I - y y^T
        J = (np.sum(y * y) * np.eye(3) - y.T @ y) / n
        kept = [k for k in range(3) if not (np.all(ijk[:, (k + 1) % 3] == ijk[0, (k + 1) % 3])
                                            and np.all(ijk[:, (k + 2) % 3] == ijk[0, (k + 2) % 3]))]
        if n == 1:
            kept = []
        assert len(rows) == 3 + len(kept)
        for a in range(3):
            om = np.eye(3)[a]
            rot = np.cross(om[None, :], y)
            got = [apply(r, rot) for r in rows[3:]]
            assert got == pytest.approx([J[k, a] for k in kept], abs=1e-13)
        kinds[o["kind"]] += 1
        # corners carry 3 rows; edges lie on a grid line, so they carry 5
        if o["kind"] == CORNER:
            assert len(rows) == 3
        if o["kind"] == EDGE:
            assert len(rows) == 5
    assert min(kinds.values()) > 0


def test_one_subdomain_bddc_is_the_exact_inverse():
    p = _small_sphere(sub=(8, 8, 8))
    m, integ, S = _build(p)
    B = BDDC(m, integ, S)
    r = np.random.default_rng(0).normal(size=S.n)
    z = B.apply(r)
    x = spla.spsolve(S.A.tocsc(), r)
    assert np.linalg.norm(z - x) <= 1e-9 * np.linalg.norm(x)


@pytest.fixture(scope="module")
def small_bddc():
    p = _small_sphere(cells=(8, 8, 8), sub=(4, 4, 4))
    m, integ, S = _build(p)
    return p, m, integ, S


def test_all_corner_bddc_is_exact(small_bddc):
    p, m, integ, S = small_bddc
    B = BDDC(m, integ, S, all_interface_corners=True)
    r = np.random.default_rng(1).normal(size=S.n)
    x = spla.spsolve(S.A.tocsc(), r)
    assert np.linalg.norm(B.apply(r) - x) <= 1e-8 * np.linalg.norm(x)


def test_bddc_weights_constraints_and_spectrum(small_bddc):
    p, m, integ, S = small_bddc
    assert m.n_sub >= 6
    B = BDDC(m, integ, S, weighting="stiffness", objects="v1", coarse="cef")
    assert np.abs(B.weight_sums() - 1.0).max() <= 1e-14
    for L in B.local:
        if L["cids"].size:
            assert np.abs(L["C"] @ L["Phi"] - np.eye(L["cids"].size)).max() <= 1e-9
    M = B.dense_preconditioner()
    assert np.abs(M - M.T).max() <= 1e-9 * np.abs(M).max()
    A = S.A.toarray()
    ev = np.sort(np.real(sla.eigvals(M @ A)))
    assert ev[0] >= 1.0 - 1e-8, ev[:3]
    # PCG with this preconditioner reaches the direct solution
    b = S.b
    info = pcg(S.apply, b, B.apply, rtol=1e-10, maxit=200)
    x = info["x"]
    xd = spla.spsolve(S.A.tocsc(), b)
    # energy-norm error (nodal values on tiny-support DOFs are ill-determined)
    e = x - xd
    assert np.sqrt(e @ (S.A @ e)) <= 1e-8 * np.sqrt(xd @ (S.A @ xd))
    assert info["iterations"] <= 40
