"""Elasticity at full size: the 96^3 union of 8 seeded spheres (1728 blocks of 8^3,
clamped at x = 0, body force (0, 0, -1)), FP64 and mixed, through the C ABI.

The oracle cannot solve this size in test time, so it checks what it can compute
one by one: the mesh integers and the coarse objects / coarse-row count (bit
exact), sampled cut-cell matrices, and sampled rows of the operator built from
the oracle's element matrices; the solve is then checked by its true residual
(the operator being pinned row by row) at the stated rtol.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    from oracle.mesh import Mesh
    p = inputs.elastic_spheres(0)
    return torch, ufe, p, Mesh(p)


def _oracle_row(m, p, d, x, cache):
    """(A x) at the three DOFs of free node d from the oracle's element matrices."""
    from oracle import elasticity as EL
    g = m.grid
    lam, mu = EL.lame(*p.lame)
    v = int(m.node_of_dof[d])
    y = np.zeros(3)
    for c in g.cells_of_node(v):
        if m.cell_type[c] == 0:
            continue
        nodes = g.cell_nodes(c)
        if c not in cache:
            if m.cell_type[c] == 2:
                cache[c] = g.h * EL.reference_stiffness(lam, mu)
            else:
                cache[c] = EL.integrate_cut_cell(m.phi[nodes], np.zeros((8, 3)), None, g.h, lam, mu)[0]
        K = cache[c]
        a = list(nodes).index(v)
        xe = np.zeros(24)
        for b, w in enumerate(nodes):
            e = m.dof_of_node[w]
            if e >= 0:
                xe[3 * b:3 * b + 3] = x[3 * e:3 * e + 3]
        y += K[3 * a:3 * a + 3] @ xe
    return y


def test_config3_integers_and_sampled_operator(env):
    torch, ufe, p, m = env
    from oracle.bddc import object_rows
    from oracle.mesh import coarse_objects
    from paper_1703_06323_gb300.solver import Solver
    from tests.oracle_cache import object_ids
    with Solver(p) as S:
        assert S.n_dof == 3 * m.n_dof
        assert np.array_equal(ufe.ufe_mesh_get_dof_map(S.mesh), m.dof_of_node)
        assert S.info["n_subdomains"] == m.n_sub
        objs = m.objects("v1")
        ids, kinds, first = ufe.ufe_bddc_get_objects(S.bddc, m.n_dof)
        ref_ids, ref_kinds = object_ids(objs, m.n_dof)
        assert np.array_equal(ids, ref_ids) and np.array_equal(kinds, ref_kinds)
        kept = coarse_objects(objs, "cef")
        assert S.bddc_info["n_coarse"] == sum(len(object_rows(o, m.grid, m, 3)) for o in kept)
        # sampled cut cells
        from oracle import elasticity as EL
        lam, mu = EL.lame(*p.lame)
        n_cut = S.info["n_cut_cells"]
        cells, K, load, eta = ufe.ufe_system_get_cut_data(S.system, n_cut)
        rng = np.random.default_rng(0)
        f = np.asarray(p.f).reshape(-1, 3)
        for k in rng.choice(n_cut, 48, replace=False):
            nodes = m.grid.cell_nodes(int(cells[k]))
            Ke, le, et = EL.integrate_cut_cell(m.phi[nodes], f[nodes], None, m.grid.h, lam, mu)
            assert np.abs(K[k] - Ke).max() <= 1e-12 * np.abs(Ke).max()
            assert np.abs(load[k] - le).max() <= 1e-12 * max(np.abs(le).max(), 1e-300)
            assert abs(eta[k] - et) <= 1e-13
        # sampled operator rows
        x = rng.normal(size=S.n_dof)
        y = S.apply(x)
        cache = {}
        for d in rng.choice(m.n_dof, 64, replace=False):
            ref = _oracle_row(m, p, int(d), x, cache)
            assert np.abs(y[3 * d:3 * d + 3] - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300) + 1e-14


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config3_solve(env, precision):
    torch, ufe, p, m = env
    from paper_1703_06323_gb300.solver import Solver
    with Solver(p, precision=precision) as S:
        if precision == "mixed":
            # genuinely mixed: most subdomains keep FP32 operators, those with tiny cut
            # fractions (failing the pivot or C Phi = I test) are factored in FP64
            bi = S.bddc_info
            assert bi["fp64_refactor"] == 0
            assert 0 < bi["fp64_subdomains"] < S.info["n_subdomains"] // 2
            assert bi["cphi_error"] <= 1e-2
        b = torch.from_numpy(S.rhs()).cuda()
        x = torch.zeros_like(b)
        info = ufe.ufe_pcg_solve(S.system, S.bddc, b, x, rtol=1e-8, maxit=2000)[1]
        assert info["converged"] == 1
        assert info["true_rel_residual"] <= 1.5e-8
        # recompute the residual with the (row-pinned) operator
        r = b - torch.from_numpy(S.apply(x.cpu().numpy())).cuda()
        assert float(r.norm() / b.norm()) <= 1.5e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config3_downscale_solution_against_the_oracle(precision):
    """The config-3 geometry at 32^3 (the same seeded union of 8 spheres, 29 subdomains,
    16,959 DOFs): the GPU solution at rtol 1e-12 against the FP64 elasticity oracle's in
    the energy norm, 1e-8 in FP64 and 1e-6 in mixed precision (both sides at rtol 1e-12,
    no allowance for the stopping point)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs
    from paper_1703_06323_gb300.solver import Solver
    from tests.oracle_cache import ElasticOracleRun, energy_error
    p = inputs.elastic_spheres(seed=0, n=32, sub=8)
    orc = _downscale_oracle(p)
    ref = orc.solve(rtol=1e-12)
    with Solver(p, precision=precision) as S:
        x, info = S.solve(rtol=1e-12, maxit=5000)
    assert info["converged"] == 1
    assert energy_error(orc.sys.A, x, ref["x"]) <= (1e-8 if precision == "fp64" else 1e-6)


_DOWNSCALE = {}


def _downscale_oracle(p):
    from tests.oracle_cache import ElasticOracleRun
    if "orc" not in _DOWNSCALE:
        _DOWNSCALE["orc"] = ElasticOracleRun(p)
    return _DOWNSCALE["orc"]
