"""The batched serving-style set at full size: 256 independent Poisson problems on
background meshes drawn from {24^3, 32^3, 48^3, 64^3} cells (8^3-cell blocks), each
a seeded sphere of radius U(0.25, 0.45), mixed precision, rtol 1e-8 each, solved by
one ufe_pcg_solve_batched call.

Checked: every problem converges with a true residual within the tolerance; sampled
members give bit-identical results when solved alone; the two smallest members match
the FP64 oracle in the energy norm.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_config4_batch(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver
    from tests.oracle_cache import OracleRun, energy_error

    ps = inputs.batched_spheres(count=256, seed=0)
    assert sorted({p.cells[0] for p in ps}) == [24, 32, 48, 64]
    dev = torch.device("cuda", 0)
    solvers = []
    try:
        for p in ps:
            solvers.append(Solver(p, precision="mixed"))
        xs = [torch.zeros(S.n_dof, dtype=torch.float64, device=dev) for S in solvers]
        st, infos = ufe.ufe_pcg_solve_batched([S.system for S in solvers], [S.bddc for S in solvers], None, xs,
                                              rtol=1e-8, maxit=1000)
        assert st == ufe.OK
        assert all(i["converged"] == 1 for i in infos)
        assert max(i["true_rel_residual"] for i in infos) <= 1.5e-8
        rng = np.random.default_rng(0)
        for k in rng.choice(len(ps), 6, replace=False):
            S = solvers[k]
            x = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, info = ufe.ufe_pcg_solve(S.system, S.bddc, None, x, rtol=1e-8, maxit=1000)
            assert info["iterations"] == infos[k]["iterations"]
            assert torch.equal(x, xs[k])
        sizes = [S.n_dof for S in solvers]
        for k in np.argsort(sizes)[:2]:
            orc = OracleRun(ps[k])
            ref = orc.solve(rtol=1e-12)["x"]
            S = solvers[k]
            x12 = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, info12 = ufe.ufe_pcg_solve(S.system, S.bddc, None, x12, rtol=1e-12, maxit=3000)
            assert info12["converged"] == 1
            # both sides at rtol 1e-12: no allowance for the stopping point
            assert energy_error(orc.sys.A, x12.cpu().numpy(), ref) <= 1e-6
    finally:
        for S in solvers:
            S.close()
