"""The adjoint workload at full size: Poisson with kappa = exp(g), g a Gaussian random
field (sigma 1, correlation length 0.1), on a sphere of radius 0.45 in 128^3 background
cells split into 16^3 subdomains of 8^3 cells; J = 1/2 sum_xi m_xi (u - u_d)^2 with the
lumped-mass weights and u_d = sin(pi x) sin(pi y) sin(pi z).  (The 32^3 downscale is
checked against the oracle gradient in test_gpu_adjoint.py.)

Checked here:
* dJ/dkappa from one forward and one adjoint FP64 BDDC-PCG solve against central
  finite differences on 32 random active cells, kappa_c (1 +- 1e-4).  Each difference
  keeps the preconditioner of kappa0 (ufe_system_set_kappa) and solves for the update
  Delta = u(kappa) - u0 from the residual of u0 (rtol 1e-10 of that residual), so
  J(kappa) - J(kappa0) = sum m (u0 - u_d) Delta + 1/2 sum m Delta^2 carries no
  cancellation against J itself;
* the mixed-precision gradient against the FP64 one;
* the coarse problem goes through the cyclic-reduction coarse solver (above 2048
  coarse DOFs).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_config5_gradient_fullsize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import autograd as AG
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver

    dev = torch.device("cuda", 0)
    p = inputs.coefficient_sphere(seed=0, n=128, sub=8, radius=0.45)
    kappa0 = torch.from_numpy(p.kappa).to(dev)
    arrays = {"phi": torch.from_numpy(p.phi).to(dev), "f": torch.from_numpy(p.f).to(dev),
              "g": torch.from_numpy(p.dirichlet_values).to(dev), "kappa": kappa0.clone()}
    w = AG.lumped_mass(p, dev)
    grads = {}
    for precision in ("fp64", "mixed"):
        with Solver(p, precision=precision, arrays=dict(arrays)) as S:
            bi = S.bddc_info
            assert S.info["n_subdomains"] > 1500 and bi["n_coarse"] > 2048
            assert bi["coarse_solver"] == ufe.COARSE_SOLVER_CR and bi["coarse_layers"] >= 14
            dof_of_node = ufe.ufe_mesh_get_dof_map(S.mesh)
            nodes = np.flatnonzero(dof_of_node >= 0)
            node_of_dof = np.empty(nodes.size, np.int64)
            node_of_dof[dof_of_node[nodes]] = nodes
            ud = torch.from_numpy(p.meta["u_d"][node_of_dof]).to(dev)
            u0 = torch.zeros(S.n_dof, dtype=torch.float64, device=dev)
            _, info = ufe.ufe_pcg_solve(S.system, S.bddc, None, u0, rtol=1e-12, maxit=3000)
            assert info["converged"] == 1
            lam = torch.zeros_like(u0)
            g = torch.empty(kappa0.numel(), dtype=torch.float64, device=dev)
            ufe.ufe_adjoint(S.system, S.bddc, u0, w * (u0 - ud), lam, g, rtol=1e-12, maxit=3000)
            grads[precision] = g.cpu().numpy()
            if precision != "fp64":
                continue
            g = grads["fp64"]
            gmax = np.abs(g).max()
            cell_type = ufe.ufe_mesh_get_cell_types(S.mesh)
            rng = np.random.default_rng(11)
            cells = rng.choice(np.flatnonzero(cell_type != ufe.CELL_EXTERNAL), 32, replace=False)
            b = torch.from_numpy(S.rhs()).to(dev)
            wr = w * (u0 - ud)
            for c in cells:
                d = 1e-4 * float(kappa0[c])
                dJ = []
                for sgn in (1.0, -1.0):
                    k = kappa0.clone()
                    k[c] += sgn * d
                    ufe.ufe_system_set_kappa(S.system, k)
                    r0 = b - ufe.ufe_system_apply(S.system, u0)
                    delta = torch.zeros_like(u0)
                    _, inf = ufe.ufe_pcg_solve(S.system, S.bddc, r0, delta, rtol=1e-10, maxit=3000)
                    assert inf["converged"] == 1
                    dJ.append(float((wr * delta).sum() + 0.5 * (w * delta * delta).sum()))
                fd = (dJ[0] - dJ[1]) / (2 * d)
                assert abs(fd - g[c]) <= 1e-5 * abs(g[c]) + 1e-8 * gmax, (int(c), fd, g[c])
            ufe.ufe_system_set_kappa(S.system, kappa0)
    g64, gm = grads["fp64"], grads["mixed"]
    assert np.linalg.norm(gm - g64) <= 1e-8 * np.linalg.norm(g64)
