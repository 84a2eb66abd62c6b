"""GPU adjoint: dJ/dkappa through torch.autograd against the oracle gradient and
against central finite differences of J computed with GPU solves.

Workload: sphere of radius 0.45, per-cell kappa = exp(Gaussian random field,
sigma 1, correlation length 0.1), f = 1, J = 1/2 sum_xi m_xi (u - u_d)^2 with the
lumped-mass weights m_xi and u_d = sin(pi x) sin(pi y) sin(pi z); the 32^3
downscale of the 128^3 coefficient workload.
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
    from paper_1703_06323_gb300 import autograd as AG
    from paper_1703_06323_gb300 import inputs
    p = inputs.coefficient_sphere(seed=0, n=32, sub=8, radius=0.45)
    return torch, AG, p


def _oracle(p, u_d):
    from oracle import adjoint as AD
    from oracle.assembly import System
    from oracle.integration import Integration
    from oracle.mesh import Mesh
    m = Mesh(p)
    integ = Integration(m, p)
    S = System(m, integ, p)
    x = AD.direct_solve(S)
    w = AD.lumped_mass(m, integ)
    ud = u_d[m.node_of_dof]
    lam = AD.direct_solve(S, w * (x - ud))
    return AD.kappa_gradient(m, integ, S, x, lam), w, m


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_matches_oracle(env, precision):
    torch, AG, p = env
    dev = torch.device("cuda", 0)
    u_d = p.meta["u_d"]
    ref, w_ref, m = _oracle(p, u_d)
    w = AG.lumped_mass(p, dev)
    assert torch.allclose(w.cpu(), torch.from_numpy(w_ref), rtol=1e-12, atol=1e-18)
    kappa = torch.from_numpy(p.kappa).to(dev).requires_grad_(True)
    x = AG.solve(kappa, p, rtol=1e-12, precision=precision)
    ud = torch.from_numpy(u_d[m.node_of_dof]).to(dev)
    J = 0.5 * (w * (x - ud) ** 2).sum()
    J.backward()
    g = kappa.grad.cpu().numpy()
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err
    assert np.all(g[m.cell_type == 0] == 0)


def test_gradient_matches_central_differences(env):
    torch, AG, p = env
    dev = torch.device("cuda", 0)
    from oracle.mesh import Mesh
    m = Mesh(p)
    u_d = p.meta["u_d"]
    w = AG.lumped_mass(p, dev)
    ud = torch.from_numpy(u_d[m.node_of_dof]).to(dev)

    def J_of(k):
        x = AG.solve(k, p, rtol=1e-13, precision="fp64")
        return 0.5 * float((w * (x - ud) ** 2).sum())

    kappa0 = torch.from_numpy(p.kappa).to(dev)
    k = kappa0.clone().requires_grad_(True)
    x = AG.solve(k, p, rtol=1e-13, precision="fp64")
    (0.5 * (w * (x - ud) ** 2).sum()).backward()
    g = k.grad.cpu().numpy()
    rng = np.random.default_rng(11)
    cells = rng.choice(np.flatnonzero(m.cell_type != 0), 32, replace=False)
    gmax = np.abs(g).max()
    for c in cells:
        d = 1e-5 * float(kappa0[c])
        kp, km = kappa0.clone(), kappa0.clone()
        kp[c] += d
        km[c] -= d
        fd = (J_of(kp) - J_of(km)) / (2 * d)
        assert abs(fd - g[c]) <= 1e-5 * abs(fd) + 1e-6 * gmax, (int(c), fd, g[c])
