"""Batched solves (ufe_pcg_solve_batched): many independent problems of uneven size in
one call, against the same problems solved one by one and against the oracle.

The batch runs the same graphs and kernels as the single solve, so solutions and
iteration counts must be bit-identical; the oracle check covers the batch's parity
with the paper's method on the small members.
"""
import numpy as np
import pytest

from tests.oracle_cache import energy_error, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    return torch, inputs, ufe


def _problems(inputs):
    """Seeded spheres of uneven size (the serving-style set at reduced count) plus
    two parity cases and one elasticity problem."""
    ps = inputs.batched_spheres(count=10, seed=3, sizes=(24, 32, 48))
    ps.append(oracle_run("sphere16").p)
    ps.append(oracle_run("sphere_ragged").p)
    ps.append(oracle_run("el_sphere8").p)
    return ps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_single_solves(env, precision):
    torch, inputs, ufe = env
    from paper_1703_06323_gb300.solver import Solver
    ps = _problems(inputs)
    solvers = [Solver(p, precision=precision) for p in ps]
    try:
        dev = torch.device("cuda", 0)
        singles = []
        for S in solvers:
            x = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, info = ufe.ufe_pcg_solve(S.system, S.bddc, None, x, rtol=1e-8, maxit=500)
            singles.append((x, info))
        xs = [torch.full((S.n_dof,), 0.0, dtype=torch.float64, device=dev) for S in solvers]
        st, infos = ufe.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers], None, xs,
                                              rtol=1e-8, maxit=500)
        assert st == ufe.OK
        for (xs1, i1), xb, ib in zip(singles, xs, infos):
            assert ib["converged"] == 1
            assert ib["iterations"] == i1["iterations"]
            assert torch.equal(xb, xs1)
            assert ib["true_rel_residual"] == i1["true_rel_residual"]
    finally:
        for S in solvers:
            S.close()


def test_batched_parity_with_the_oracle(env):
    torch, inputs, ufe = env
    from paper_1703_06323_gb300.solver import Solver
    names = ["sphere16", "sphere_ragged", "plane", "el_sphere8", "el_ragged"]
    runs = [oracle_run(n) for n in names]
    solvers = [Solver(r.p) for r in runs]
    try:
        xs = [np.zeros(S.n_dof) for S in solvers]
        # both sides at rtol 1e-12: solution parity with no allowance for the stopping point
        st, infos = ufe.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers],
                                              [None] * len(solvers), xs, rtol=1e-12, maxit=5000)
        assert st == ufe.OK
        for r, x, info in zip(runs, xs, infos):
            ref = r.solve(rtol=1e-12)
            assert energy_error(r.sys.A, x, ref["x"]) <= 1e-8
    finally:
        for S in solvers:
            S.close()


def test_batched_reports_every_problem(env):
    """One member capped at 2 iterations does not stop the others; the call returns
    NO_CONVERGENCE and every info is filled."""
    torch, inputs, ufe = env
    from paper_1703_06323_gb300.solver import Solver
    ps = _problems(inputs)[:4]
    solvers = [Solver(p) for p in ps]
    try:
        xs = [np.zeros(S.n_dof) for S in solvers]
        st, infos = ufe.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers], None, xs,
                                              rtol=1e-8, maxit=2, raise_on_error=False)
        assert st == ufe.ERR_NO_CONVERGENCE
        assert all(i["iterations"] == 2 and not i["converged"] for i in infos)
        xs = [np.zeros(S.n_dof) for S in solvers]
        st, infos = ufe.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers], None, xs,
                                              rtol=1e-8, maxit=500)
        assert st == ufe.OK and all(i["converged"] for i in infos)
        with pytest.raises(ufe.UfeError):
            ufe.ufe_pcg_solve_batched([solvers[0].system] * 2, [solvers[0].bddc] * 2, None,
                                      [np.zeros(solvers[0].n_dof)] * 2)
    finally:
        for S in solvers:
            S.close()
