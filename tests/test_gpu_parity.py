"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer work is compared bit for bit; floating point to the tolerances stated
per test (FP64: relative 1e-8 in the energy norm for solutions, rounding-level
for element data; mixed precision: 1e-6 for solutions).
"""
import numpy as np
import pytest

from tests.oracle_cache import energy_error, object_ids, oracle_run, small_problems

pytestmark = pytest.mark.gpu

SMALL = list(small_problems().keys())
SOLVABLE = [n for n in SMALL if n != "two_pieces"]
MESH_ONLY = {"two_pieces"}


@pytest.fixture(scope="module")
def ufe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import ufe as U
    return U


def _solver(ufe, p, **kw):
    from paper_1703_06323_gb300.solver import Solver
    return Solver(p, **kw)


def _oracle_bddc_or_none(orc, **kw):
    """The oracle's preconditioner, or None when the oracle refuses it as singular."""
    from oracle.bddc import SingularLocal
    try:
        return orc.bddc(**kw)
    except SingularLocal:
        return None


def _expect_singular(ufe, p, **kw):
    with pytest.raises(ufe.UfeError) as e:
        _solver(ufe, p, **kw)
    assert e.value.status == ufe.ERR_SINGULAR_LOCAL


# ---------------------------------------------------------------------------
# integer set-up: bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", SMALL)
def test_mesh_integers_bit_exact(ufe, name):
    orc = oracle_run(name)
    m = orc.mesh
    p = orc.p
    mesh = ufe.ufe_mesh_create(p.box_lo, p.box_hi, p.cells, p.sub_cells, p.phi, p.dirichlet_face_mask, p.pin_node)
    try:
        info = ufe.ufe_mesh_get_info(mesh)
        assert info["n_dof"] == m.n_dof
        assert info["n_subdomains"] == m.n_sub
        assert info["pinned_node"] == m.pin
        assert info["n_interface_dofs"] == int(m.is_gamma.sum())
        assert info["n_cut_cells"] == int((m.cell_type == 1).sum())
        assert np.array_equal(ufe.ufe_mesh_get_cell_types(mesh), m.cell_type)
        assert np.array_equal(ufe.ufe_mesh_get_dof_map(mesh).astype(np.int64), m.dof_of_node)
        assert np.array_equal(ufe.ufe_mesh_get_subdomains(mesh).astype(np.int64), m.sub_of_cell)
        neigh = ufe.ufe_mesh_get_neighbours(mesh)
        ref = -np.ones((m.n_dof, 8), dtype=np.int64)
        for d, ns in enumerate(m.neigh):
            ref[d, :len(ns)] = ns
        assert np.array_equal(neigh.astype(np.int64), ref)
    finally:
        ufe.ufe_mesh_destroy(mesh)


def test_floating_subdomain_without_coarse_dof_is_singular(ufe):
    """Islands with no interface and no constrained node: the oracle and the library refuse them."""
    from oracle.bddc import SingularLocal
    orc = oracle_run("two_pieces")
    with pytest.raises(SingularLocal):
        orc.bddc()
    with pytest.raises(ufe.UfeError) as e:
        _solver(ufe, orc.p)
    assert e.value.status == ufe.ERR_SINGULAR_LOCAL


@pytest.mark.parametrize("name", SOLVABLE)
@pytest.mark.parametrize("objects", ["std", "v1"])
def test_objects_bit_exact(ufe, name, objects):
    orc = oracle_run(name)
    m = orc.mesh
    objs = m.objects(objects)
    ref_ids, ref_kinds = object_ids(objs, m.n_dof)
    with _solver(ufe, orc.p, objects=objects, coarse="cef") as S:
        ids, kinds, coarse = ufe.ufe_bddc_get_objects(S.bddc, m.n_dof)
        assert np.array_equal(ids.astype(np.int64), ref_ids)
        assert np.array_equal(kinds.astype(np.int64), ref_kinds)
        assert np.array_equal(coarse, np.arange(len(objs)))
    # BDDC(ce): faces carry no coarse DOF, the others are numbered in object order
    if name == "one_subdomain":
        return
    if _oracle_bddc_or_none(orc, objects=objects, coarse="ce") is None:
        _expect_singular(ufe, orc.p, objects=objects, coarse="ce")
        return
    with _solver(ufe, orc.p, objects=objects, coarse="ce") as S:
        _, kinds, coarse = ufe.ufe_bddc_get_objects(S.bddc, m.n_dof)
        keep = ref_kinds != 2
        expect = np.where(keep, np.cumsum(keep) - 1, -1)
        assert np.array_equal(coarse.astype(np.int64), expect)


# ---------------------------------------------------------------------------
# integration, right-hand side, operator: rounding level
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", SOLVABLE)
def test_cut_cell_data(ufe, name):
    orc = oracle_run(name)
    integ = orc.integ
    with _solver(ufe, orc.p) as S:
        n_cut = S.info["n_cut_cells"]
        cells, K, load, eta = ufe.ufe_system_get_cut_data(S.system, n_cut)
        assert np.array_equal(cells.astype(np.int64), integ.cut_cells)
        for k in range(n_cut):
            scale = np.abs(integ.K_cut[k]).max()
            assert np.abs(K[k] - integ.K_cut[k]).max() <= 1e-12 * scale
        if n_cut:
            lscale = np.abs(integ.load_cut).max() + 1e-300
            assert np.abs(load - integ.load_cut).max() <= 1e-12 * lscale
            assert np.abs(eta - integ.eta).max() <= 1e-13


@pytest.mark.parametrize("name", SOLVABLE)
def test_rhs_and_operator(ufe, name):
    orc = oracle_run(name)
    with _solver(ufe, orc.p) as S:
        b = S.rhs()
        assert np.abs(b - orc.sys.b).max() <= 1e-12 * np.abs(orc.sys.b).max()
        x = np.random.default_rng(1).normal(size=S.n_dof)
        y = S.apply(x)
        ref = orc.sys.A @ x
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# preconditioner and solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["sphere16", "sphere_ragged", "plane", "slab_sliver", "one_subdomain", "u_shape"])
@pytest.mark.parametrize("weighting,objects,coarse", [("stiffness", "v1", "cef"), ("stiffness", "std", "ce"),
                                                      ("topological", "std", "cef")])
def test_preconditioner_fp64(ufe, name, weighting, objects, coarse):
    """z = M r (Eq. bddc) for random r: energy-norm difference at FP64 rounding level."""
    orc = oracle_run(name)
    B = _oracle_bddc_or_none(orc, weighting=weighting, objects=objects, coarse=coarse)
    if B is None:
        _expect_singular(ufe, orc.p, weighting=weighting, objects=objects, coarse=coarse)
        return
    r = np.random.default_rng(2).normal(size=orc.mesh.n_dof)
    ref = B.apply(r)
    with _solver(ufe, orc.p, weighting=weighting, objects=objects, coarse=coarse) as S:
        z = S.precondition(r)
    assert energy_error(orc.sys.A, z, ref) <= 1e-9


@pytest.mark.parametrize("name", ["sphere16", "sphere_ragged", "slab_sliver"])
def test_preconditioner_mixed(ufe, name):
    """Mixed precision M r: FP32 local operators, relative energy-norm error well below 1e-3."""
    orc = oracle_run(name)
    B = orc.bddc()
    r = np.random.default_rng(3).normal(size=orc.mesh.n_dof)
    ref = B.apply(r)
    with _solver(ufe, orc.p, precision="mixed") as S:
        z = S.precondition(r)
    assert energy_error(orc.sys.A, z, ref) <= 1e-3


def _local_energy_errors(B, z, ref):
    """Per subdomain w: |z - ref| / |ref| in the energy of its local Neumann matrix A^w
    over its own DOFs.  A wrong scaling of one subdomain's local solves by 1 % shows up
    here at 3e-4 to 8e-3 on these cases, where the global energy norm sees as little
    as 1e-7 of it (its share of the energy is small)."""
    out = []
    for L in B.local:
        d = L["dofs"]
        e = z[d] - ref[d]
        den = float(ref[d] @ (L["A"] @ ref[d]))
        out.append(np.sqrt(max(float(e @ (L["A"] @ e)), 0.0) / den) if den > 0 else 0.0)
    return np.array(out)


@pytest.mark.parametrize("name", ["sphere16", "sphere_ragged", "slab_sliver"])
def test_preconditioner_mixed_per_subdomain(ufe, name):
    """Mixed precision M r measured subdomain by subdomain (see _local_energy_errors):
    the FP32 operators stay within 1e-4 of the FP64 oracle in every subdomain's local
    energy, which a 1 % mis-scaling of any one subdomain's local solves would exceed."""
    orc = oracle_run(name)
    B = orc.bddc()
    r = np.random.default_rng(3).normal(size=orc.mesh.n_dof)
    ref = B.apply(r)
    with _solver(ufe, orc.p, precision="mixed") as S:
        z = S.precondition(r)
    le = _local_energy_errors(B, z, ref)
    print(name, "mixed M r, largest per-subdomain local energy error:", le.max())
    assert le.max() <= 1e-4


@pytest.mark.parametrize("name", ["tower", "sphere_ragged", "plane"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coarse_cyclic_reduction(ufe, name, precision):
    """The block cyclic reduction coarse solver (forced here; the default takes it above
    2048 coarse DOFs) solves the same coarse problem as the dense inverse: M r agrees
    with the dense-solver preconditioner to rounding, with the oracle as in the
    preconditioner tests, and PCG takes the same number of iterations."""
    orc = oracle_run(name)
    r = np.random.default_rng(4).normal(size=orc.mesh.n_dof)
    ref = orc.bddc().apply(r)
    out = {}
    for cs in ("cr", "dense"):
        with _solver(ufe, orc.p, precision=precision, coarse_solver=cs) as S:
            bi = S.bddc_info
            assert bi["coarse_solver"] == (ufe.COARSE_SOLVER_CR if cs == "cr" else ufe.COARSE_SOLVER_DENSE)
            z = S.precondition(r)
            x, info = S.solve(rtol=1e-8)
            out[cs] = (z, x, info, bi)
    zc, xc, ic, bc = out["cr"]
    zd, xd, idn, _ = out["dense"]
    nl = {"tower": 8, "sphere_ragged": 2, "plane": 2}[name]
    assert bc["coarse_layers"] == nl and bc["coarse_levels"] == int(np.ceil(np.log2(nl)))
    assert energy_error(orc.sys.A, zc, zd) <= (1e-11 if precision == "fp64" else 1e-6)
    assert energy_error(orc.sys.A, zc, ref) <= (1e-9 if precision == "fp64" else 1e-3)
    assert ic["converged"] == 1 and ic["true_rel_residual"] <= 1.5e-8
    assert abs(ic["iterations"] - idn["iterations"]) <= (0 if precision == "fp64" else 1)


@pytest.mark.parametrize("name", SOLVABLE)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_solution(ufe, name, precision):
    """PCG at the method's rtol 1e-8: converged, true residual within the tolerance,
    FP64 iteration counts within 1 of the oracle's.  Solution parity: both sides
    solve to rtol 1e-12, where each is the discrete solution to well below the
    stated tolerance, and the GPU solution must match the oracle's in the energy
    norm to 1e-8 (FP64) / 1e-6 (mixed), with no allowance for either solver's
    stopping point."""
    orc = oracle_run(name)
    ref = orc.solve(rtol=1e-12)
    ref8 = orc.solve(rtol=1e-8)
    tol = 1e-8 if precision == "fp64" else 1e-6
    with _solver(ufe, orc.p, precision=precision) as S:
        x, info = S.solve(rtol=1e-8)
        assert info["converged"] == 1
        assert info["true_rel_residual"] <= 1e-8 * 1.5
        # FP64: within 1 of the oracle; mixed (flexible PCG on FP32 local operators): within
        # 2, which a mis-scaled local operator in any subdomain would break
        assert abs(info["iterations"] - ref8["iterations"]) <= (1 if precision == "fp64" else 2)
        x12, info12 = S.solve(rtol=1e-12, maxit=3000)
    assert info12["converged"] == 1
    assert energy_error(orc.sys.A, x12, ref["x"]) <= tol


def test_pcg_initial_guess_and_zero_rhs(ufe):
    orc = oracle_run("sphere16")
    with _solver(ufe, orc.p) as S:
        x, info = S.solve(b=np.zeros(S.n_dof), x0=np.ones(S.n_dof))
        assert info["iterations"] == 0 and np.all(x == 0)
        ref = orc.solve(rtol=1e-12)["x"]
        x0 = ref.copy()
        x, info = S.solve(x0=x0)
        assert info["iterations"] == 0


def test_maxit_reports_no_convergence(ufe):
    orc = oracle_run("sphere16")
    from paper_1703_06323_gb300 import ufe as U
    with _solver(ufe, orc.p, weighting="topological", objects="std") as S:
        x, info = S.solve(maxit=2, raise_on_error=False)
        assert info["status"] == U.ERR_NO_CONVERGENCE
        assert info["iterations"] == 2 and not info["converged"]
