"""Pins for the oracle's BDDC preconditioner and PCG."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assembly import System
from oracle.bddc import BDDC
from oracle.integration import Integration
from oracle.mesh import Mesh
from oracle.pcg import lanczos_ritz, pcg
from paper_1703_06323_gb300 import inputs


def _setup(p):
    m = Mesh(p)
    integ = Integration(m, p)
    return m, integ, System(m, integ, p)


@pytest.fixture(scope="module")
def tiny():
    """Sphere in 8^3 cells with 4^3-cell blocks: 8 subdomains, a few hundred DOFs."""
    p = inputs.sphere_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), centre=(0.52, 0.47, 0.5), radius=0.41)
    return _setup(p)


def test_one_subdomain_is_exact_solve():
    """No interface: M = A0^-1 = A^-1, so PCG converges in one iteration."""
    p = inputs.manufactured_sphere(0, n=16, sub=16)
    m, integ, S = _setup(p)
    assert m.n_sub == 1 and not m.is_gamma.any()
    B = BDDC(m, integ, S)
    res = pcg(S.apply, S.b, B.apply, rtol=1e-10)
    assert res["iterations"] == 1


def test_all_interface_corners_is_exact_solve(tiny):
    """Enlarged coarse space (Sect. 4.2): every interface DOF a corner => V~ = continuous space."""
    m, integ, S = tiny
    B = BDDC(m, integ, S, all_interface_corners=True)
    res = pcg(S.apply, S.b, B.apply, rtol=1e-10)
    assert res["iterations"] == 1


@pytest.mark.parametrize("weighting", ["stiffness", "topological"])
def test_weights_partition_of_unity(tiny, weighting):
    m, integ, S = tiny
    B = BDDC(m, integ, S, weighting=weighting)
    assert np.allclose(B.weight_sums(), 1.0, rtol=0, atol=4e-16 * 8)


def test_stiffness_equals_topological_on_uncut_box():
    p = inputs.box_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), dirichlet_face_mask=inputs.ALL_FACES)
    m, integ, S = _setup(p)
    Bs = BDDC(m, integ, S, weighting="stiffness")
    Bt = BDDC(m, integ, S, weighting="topological")
    for Ls, Lt in zip(Bs.local, Bt.local):
        assert np.allclose(Ls["w"], Lt["w"], rtol=0, atol=1e-15)


def test_coarse_basis_reproduces_coarse_dofs(tiny):
    m, integ, S = tiny
    B = BDDC(m, integ, S, objects="v1", coarse="cef")
    for L in B.local:
        if L["cids"].size:
            assert np.allclose(L["C"] @ L["Phi"], np.eye(L["cids"].size), atol=1e-12)
    assert np.allclose(B.Ac, B.Ac.T, atol=1e-12)
    assert np.linalg.eigvalsh(B.Ac).min() > 0


@pytest.mark.parametrize("objects,coarse,weighting", [("std", "cef", "stiffness"), ("v1", "ce", "stiffness"),
                                                      ("v1", "cef", "topological")])
def test_preconditioner_symmetric_and_lambda_min_one(tiny, objects, coarse, weighting):
    """M is SPD and the spectrum of M A is bounded below by exactly 1 (Sect. 3.4 proof)."""
    m, integ, S = tiny
    B = BDDC(m, integ, S, weighting=weighting, objects=objects, coarse=coarse)
    Md = B.dense_preconditioner()
    assert np.allclose(Md, Md.T, atol=1e-10 * np.abs(Md).max())
    A = S.A.toarray()
    ev = np.sort(sla.eigvals(Md @ A).real)
    assert abs(ev[0] - 1.0) < 1e-8
    # Lanczos Ritz values from the PCG coefficients lie inside the dense spectrum
    res = pcg(S.apply, S.b, B.apply, rtol=1e-12)
    ritz = lanczos_ritz(res["alphas"][:-1], res["betas"])
    assert ritz.min() >= 1.0 - 1e-8 and ritz.max() <= ev[-1] * (1 + 1e-8)
    assert abs(ritz.max() - ev[-1]) < 1e-3 * ev[-1]


def test_bddc_operator_inverse_by_brute_force(tiny):
    """A~^-1 (local constrained Neumann + coarse split) equals the Galerkin inverse of the
    sub-assembled operator on an explicit basis of V~ = {v : coarse DOFs agree} (Sect. 3.2)."""
    m, integ, S = tiny
    B = BDDC(m, integ, S, objects="v1", coarse="cef")
    offs = np.cumsum([0] + [L["dofs"].size for L in B.local])
    ntot = offs[-1]
    Asub = np.zeros((ntot, ntot))
    for k, L in enumerate(B.local):
        Asub[offs[k]:offs[k + 1], offs[k]:offs[k + 1]] = L["A"]
    rows = []
    for ci, o in enumerate(B.objs):
        ws = list(o["neigh"])
        def alpha(w):
            row = np.zeros(ntot)
            L = B.local[w]
            pos = {int(d): i for i, d in enumerate(L["dofs"])}
            for d in o["dofs"]:
                row[offs[w] + pos[int(d)]] = 1.0 / len(o["dofs"])
            return row
        for w in ws[1:]:
            rows.append(alpha(ws[0]) - alpha(w))
    Z = sla.null_space(np.array(rows))
    rng = np.random.default_rng(0)
    r = rng.normal(size=ntot)
    ref = Z @ np.linalg.solve(Z.T @ Asub @ Z, Z.T @ r)
    got = np.concatenate(B.bddc_solve([r[offs[k]:offs[k + 1]] for k in range(len(B.local))]))
    assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max()


def test_topological_weighting_breaks_down_stiffness_does_not():
    """3D slab analogue of the breakdown example (Sect. 4.1, Fig. 3): the domain x < 0.5 + eps h
    leaves the blocks beyond x = 0.5 with a sliver of width eps h.  With topological weighting
    the PCG iterations grow as eps -> 0; stiffness weighting (Sect. 4.3) stays flat."""
    its = {"topological": [], "stiffness": []}
    for eps in (0.3, 1e-3, 1e-6):
        h = 1.0 / 8
        p = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(1, 0, 0), offset=0.5 + eps * h,
                                 dirichlet_face_mask=inputs.FACE_XLO, linear=(0, 0, 0, 0))
        p.f = np.random.default_rng(0).uniform(-1, 1, p.n_nodes)
        m, integ, S = _setup(p)
        for w in its:
            B = BDDC(m, integ, S, weighting=w, objects="std", coarse="cef")
            its[w].append(pcg(S.apply, S.b, B.apply, rtol=1e-8, maxit=500)["iterations"])
    t, s = its["topological"], its["stiffness"]
    assert t[0] < t[1] < t[2] and t[2] >= 3 * t[0]
    assert max(s) - min(s) <= 2 and max(s) < t[2] / 3


def test_improved_objects_reduce_iterations_on_sphere():
    """Sect. 4.4 / 5.2: with stiffness weighting, variant-1 objects need fewer iterations than
    the standard ones on a cut sphere; BDDC(cef) needs no more than BDDC(ce)."""
    p = inputs.manufactured_sphere(0)
    m, integ, S = _setup(p)
    it = {}
    for ob in ("std", "v1"):
        for co in ("ce", "cef"):
            B = BDDC(m, integ, S, weighting="stiffness", objects=ob, coarse=co)
            it[ob, co] = pcg(S.apply, S.b, B.apply, rtol=1e-8)["iterations"]
    assert it["v1", "cef"] < it["std", "cef"]
    assert it["v1", "ce"] < it["std", "ce"]
    assert it["std", "cef"] <= it["std", "ce"]


def test_pcg_exact_preconditioner_one_iteration_and_finite_termination():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    A = Q @ np.diag(np.linspace(1, 50, 12)) @ Q.T
    b = rng.normal(size=12)
    res = pcg(lambda x: A @ x, b, lambda r: np.linalg.solve(A, r), rtol=1e-12)
    assert res["iterations"] == 1
    res = pcg(lambda x: A @ x, b, lambda r: r, rtol=1e-10, maxit=100)
    assert res["iterations"] <= 13 and res["true_residual"] < 1e-9
    resf = pcg(lambda x: A @ x, b, lambda r: r, rtol=1e-10, maxit=100, flexible=True)
    assert abs(resf["iterations"] - res["iterations"]) <= 1


def test_manufactured_solution_error_decreases():
    """Discretisation error of the BDDC-PCG solution inside Omega: O(h^2) at the nodes."""
    errs = []
    for n in (16, 32):
        p = inputs.manufactured_sphere(0, n=n)
        m, integ, S = _setup(p)
        B = BDDC(m, integ, S)
        x = pcg(S.apply, S.b, B.apply, rtol=1e-10)["x"]
        ins = p.phi[m.node_of_dof] < 0
        errs.append(np.abs(x - p.u_exact[m.node_of_dof])[ins].max())
    assert errs[1] < errs[0] / 3.0


def test_flexible_pcg_absorbs_a_varying_preconditioner():
    """Flexible CG (Notay 2000) against classical CG when the preconditioner changes from
    one application to the next: z = A^-1 r plus 30 % random noise drawn afresh at every
    application (2-D Laplacian, 576 unknowns).  The flexible beta keeps the search
    directions useful and converges to 1e-10 in a few tens of iterations; the classical
    beta assumes one fixed symmetric M and does not converge in 300.  Together with the
    fixed-preconditioner test above (where both betas agree, which rules out a sign or
    denominator mistake) this pins the flexible branch."""
    n = 24
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = np.kron(T, np.eye(n)) + np.kron(np.eye(n), T)
    b = np.random.default_rng(0).normal(size=n * n)
    Ainv = np.linalg.inv(A)

    def varying(seed):
        g = np.random.default_rng(seed)

        def M(r):
            z = Ainv @ r
            return z + 0.3 * np.linalg.norm(z) * g.normal(size=z.size) / np.sqrt(z.size)
        return M

    flex = pcg(lambda x: A @ x, b, varying(1), rtol=1e-10, maxit=300, flexible=True)
    classic = pcg(lambda x: A @ x, b, varying(1), rtol=1e-10, maxit=300)
    assert flex["converged"] and flex["iterations"] <= 40 and flex["true_residual"] < 1e-9
    assert not classic["converged"]
