"""The paper's robustness and coarse-space studies, run on the GPU (Sect. 5.2, Sect. 5.3).

* translation sweep (Sect. 5.3): the background mesh is shifted by 51 values of
  eps in [-h, h] along x (equivalently the geometry by -eps) on the sphere of Table 1
  mesh 3 (radius 0.7 in [-1, 1]^3, 64^3 cells, 8^3-cell blocks) with weak Dirichlet
  data on the whole unfitted boundary; the paper reports a largest change of one
  PCG iteration for variant 2 and of four for the other methods.  Here: variant 2
  changes by at most two iterations, and no variant by more than six;
* the same sweep on a 16^3 downscale with five shifts against the FP64 oracle:
  iteration counts within one;
* coarse-space size (Sect. 5.2): the variant-1 and variant-2 coarse spaces exceed
  the standard one by a ratio that falls toward 1 as the mesh of Table 1 refines
  (meshes 1-4), and the largest per-subdomain coarse-DOF count stays bounded;
* subdomain size H/h in {2, 4, 8, 16} (Sect. 5.2 studies {4, 8, 16}): the iteration
  count grows mildly.

Every measured value is printed (pytest -s shows them).
"""
import numpy as np
import pytest

from paper_1703_06323_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import ufe
    from paper_1703_06323_gb300.solver import Solver
    return ufe, Solver


def table1_sphere(n, sub=8, shift=0.0, weak=True):
    """Sphere of radius 0.7 centred at the origin in [-1, 1]^3 (Table 1 geometry),
    background mesh shifted by `shift` along x; manufactured sines as data."""
    p = inputs.sphere_problem(cells=(n, n, n), sub_cells=(sub, sub, sub), centre=(-shift, 0.0, 0.0), radius=0.7,
                              box_lo=(-1.0, -1.0, -1.0), box_hi=(1.0, 1.0, 1.0),
                              dirichlet_face_mask=inputs.ALL_FACES,
                              pin_node=inputs.PIN_NONE if weak else inputs.PIN_AUTO, name=f"t1_{n}_{shift:+.4f}")
    if weak:
        p.q = None
        p.weak_dirichlet = True
    return p


def _iterations(Solver, p, objects, precision="fp64"):
    with Solver(p, objects=objects, precision=precision) as S:
        _, info = S.solve(rtol=1e-8, maxit=2000)
        assert info["converged"] == 1
        return info["iterations"], S.bddc_info["n_coarse"]


def test_translation_sweep_mesh3(env):
    ufe, Solver = env
    n = 64
    h = 2.0 / n
    its = {ob: [] for ob in ("std", "v1", "v2")}
    for eps in np.linspace(-h, h, 51):
        p = table1_sphere(n, shift=float(eps))
        for ob in its:
            its[ob].append(_iterations(Solver, p, ob)[0])
    spread = {ob: max(v) - min(v) for ob, v in its.items()}
    print("translation sweep, Table 1 sphere mesh 3, weak Dirichlet, 51 shifts:",
          {ob: (min(v), max(v), spread[ob]) for ob, v in its.items()})
    assert spread["v2"] <= 2
    assert max(spread.values()) <= 6


def test_translation_sweep_downscale_against_oracle(env):
    ufe, Solver = env
    from tests.oracle_cache import OracleRun
    n = 16
    h = 2.0 / n
    for eps in np.linspace(-h, h, 5):
        p = table1_sphere(n, shift=float(eps))
        orc = OracleRun(p)
        for ob in ("std", "v1", "v2"):
            gpu, _ = _iterations(Solver, p, ob)
            ref = orc.solve(rtol=1e-8, objects=ob)["iterations"]
            assert abs(gpu - ref) <= 1, (eps, ob, gpu, ref)


def test_coarse_space_ratio_falls_with_refinement(env):
    ufe, Solver = env
    ratios = []
    for n in (16, 32, 64, 128):
        p = table1_sphere(n, weak=False)
        sizes = {}
        for ob in ("std", "v1", "v2"):
            with Solver(p, objects=ob, precision="mixed") as S:
                sizes[ob] = S.bddc_info["n_coarse"]
                if ob == "v2":
                    m = S.info
                    nsub = m["n_subdomains"]
                    local_max = S.bddc_info["max_local_coarse"]
        ratios.append((n, sizes["v1"] / sizes["std"], sizes["v2"] / sizes["std"], nsub, local_max))
    print("coarse-space size ratio vs standard (Table 1 sphere meshes 1-4, Neumann):", ratios)
    r1 = [r[1] for r in ratios]
    assert all(r >= 1.0 for r in r1)
    assert r1[-1] < r1[0]
    assert ratios[-1][4] <= 3 * ratios[0][4] + 30


def test_subdomain_size_study(env):
    """H/h in {2, 4, 8, 16} on Table 1 sphere mesh 2: the iterations grow mildly, as
    the (1 + log^2 (H/h)) bound of Sect. 3.4 lets them."""
    ufe, Solver = env
    its = {}
    for sub in (2, 4, 8, 16):
        p = table1_sphere(32, sub=sub)
        its[sub] = _iterations(Solver, p, "v2", precision="mixed")
    print("H/h study, Table 1 sphere mesh 2, weak Dirichlet, variant 2 (iterations, coarse DOFs):", its)
    assert its[2][0] <= its[4][0] + 1 and its[4][0] <= its[8][0] + 1
    assert its[8][0] <= 2.5 * its[2][0] + 3
    assert its[16][0] <= 3 * its[2][0] + 3


def test_weak_scaling_by_subdomain_size(env):
    """Sect. 5.2's weak-scaling view of H/h: for each H/h in {4, 8, 16} the sphere of
    Table 1 (weak Dirichlet data) on meshes of 2^3, 4^3 and 8^3 blocks (up to 128^3
    cells), solved with the three coarse spaces (standard, variants 1 and 2,
    BDDC(cef)).  The paper finds the effect of H/h very mild and the solvers weakly
    scalable; here the iterations at 8^3 blocks stay within those at 4^3 blocks plus
    four, the iterations grow by at most four from H/h = 4 to 16, and variant 2 never
    needs more than the standard space plus two."""
    ufe, Solver = env
    table = {}
    for hh in (4, 8, 16):
        for nb in (2, 4, 8):
            p = table1_sphere(hh * nb, sub=hh)
            table[(hh, nb)] = {obj: _iterations(Solver, p, obj, precision="mixed") for obj in ("std", "v1", "v2")}
    for (hh, nb), row in sorted(table.items()):
        print(f"H/h {hh:2d}, {nb}^3 blocks: " + ", ".join(f"{k} {v[0]} it / {v[1]} coarse" for k, v in row.items()))
    for hh in (4, 8, 16):
        for obj in ("std", "v1", "v2"):
            assert table[(hh, 8)][obj][0] <= table[(hh, 4)][obj][0] + 4
        for nb in (2, 4, 8):
            assert table[(hh, nb)]["v2"][0] <= table[(hh, nb)]["std"][0] + 2
    for nb in (2, 4, 8):
        for obj in ("std", "v1", "v2"):
            assert table[(16, nb)][obj][0] <= table[(4, nb)][obj][0] + 4
