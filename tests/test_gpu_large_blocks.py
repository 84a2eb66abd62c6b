"""Subdomain blocks of more than 8 cells per edge (Sect. 5.2 studies H/h in {4, 8, 16}).

With 16^3-cell blocks a subdomain holds up to 17^3 local nodes: the block labelling
and the local numbering walk their cells and nodes in chunks, and the FP64 operator
rows of a nearly full block (interior near 15^3) are too long for eight of them to be
streamed into one CTA's shared memory, so fewer go to a stage and warps split the
columns of a row.  Each case is compared with the FP64 oracle as in the other parity
tests: integers bit for bit, the preconditioner in the energy norm (FP64 1e-9, mixed
1e-3), solutions to rtol 1e-12 against the oracle's (FP64 1e-8, mixed 1e-6) and the
iteration counts at rtol 1e-8 (FP64 within 1, mixed within 2).
"""
import numpy as np
import pytest

from tests.oracle_cache import energy_error, large_block_problems, object_ids, oracle_run

pytestmark = pytest.mark.gpu

NAMES = list(large_block_problems().keys())


@pytest.fixture(scope="module")
def ufe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import ufe as U
    return U


def _solver(p, **kw):
    from paper_1703_06323_gb300.solver import Solver
    return Solver(p, **kw)


@pytest.mark.parametrize("name", NAMES)
def test_mesh_and_objects_bit_exact(ufe, name):
    orc = oracle_run(name)
    m, p = orc.mesh, orc.p
    mesh = ufe.ufe_mesh_create(p.box_lo, p.box_hi, p.cells, p.sub_cells, p.phi, p.dirichlet_face_mask, p.pin_node)
    try:
        info = ufe.ufe_mesh_get_info(mesh)
        assert info["n_dof"] == m.n_dof and info["n_subdomains"] == m.n_sub
        assert info["n_interface_dofs"] == int(m.is_gamma.sum())
        assert np.array_equal(ufe.ufe_mesh_get_dof_map(mesh).astype(np.int64), m.dof_of_node)
        assert np.array_equal(ufe.ufe_mesh_get_subdomains(mesh).astype(np.int64), m.sub_of_cell)
        neigh = ufe.ufe_mesh_get_neighbours(mesh)
        ref = -np.ones((m.n_dof, 8), dtype=np.int64)
        for d, ns in enumerate(m.neigh):
            ref[d, :len(ns)] = ns
        assert np.array_equal(neigh.astype(np.int64), ref)
        print(name, "largest interior / interface:", info["max_interior"], info["max_interface"])
    finally:
        ufe.ufe_mesh_destroy(mesh)
    objs = m.objects("v1")
    ref_ids, ref_kinds = object_ids(objs, m.n_dof)
    with _solver(p, objects="v1", coarse="cef") as S:
        ids, kinds, coarse = ufe.ufe_bddc_get_objects(S.bddc, m.n_dof)
        assert np.array_equal(ids.astype(np.int64), ref_ids)
        assert np.array_equal(kinds.astype(np.int64), ref_kinds)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_preconditioner(ufe, name, precision):
    orc = oracle_run(name)
    r = np.random.default_rng(11).normal(size=orc.mesh.n_dof)
    ref = orc.bddc().apply(r)
    with _solver(orc.p, precision=precision) as S:
        z = S.precondition(r)
    assert energy_error(orc.sys.A, z, ref) <= (1e-9 if precision == "fp64" else 1e-3)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solution(ufe, name, precision):
    orc = oracle_run(name)
    ref = orc.solve(rtol=1e-12)
    ref8 = orc.solve(rtol=1e-8)
    with _solver(orc.p, precision=precision) as S:
        x, info = S.solve(rtol=1e-8)
        assert info["converged"] == 1 and info["true_rel_residual"] <= 1.5e-8
        assert abs(info["iterations"] - ref8["iterations"]) <= (1 if precision == "fp64" else 2)
        x12, info12 = S.solve(rtol=1e-12, maxit=3000)
    assert info12["converged"] == 1
    assert energy_error(orc.sys.A, x12, ref["x"]) <= (1e-8 if precision == "fp64" else 1e-6)


def test_elasticity_beyond_shared_memory_is_refused(ufe):
    """Elasticity in 16^3-cell blocks (interiors near 3 x 15^3 values): a subdomain's
    vectors no longer fit one CTA's shared memory, and the set-up says so before it
    allocates any local operator."""
    from tests.oracle_cache import _elastic_sphere
    p = _elastic_sphere((32, 32, 32), (16, 16, 16), (0.3, 0.5, 0.5), 0.62, name="el_big")
    with pytest.raises(ufe.UfeError) as e:
        _solver(p)
    assert e.value.status == ufe.ERR_UNSUPPORTED
