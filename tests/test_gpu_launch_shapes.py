"""Launch shapes of the per-iteration preconditioner kernels: every cluster size (2, 4,
8 CTAs per subdomain) and stage count gives the same z = M r (the slices of the dense
GEMVs change, the arithmetic of each row does not; the coarse restriction sums its
slices in a different order, in FP64 for FP64 operators and from FP32 partial sums
over each CTA's rows for FP32 ones, so mixed precision agrees to FP32 rounding) and
the same PCG iterations (within one in mixed precision); the tuner reports a shape
from its candidate set and reuses it for a second problem of the same size class."""
import os

import numpy as np
import pytest

from tests.oracle_cache import small_problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver
    return inputs, ufe, Solver


@pytest.mark.parametrize("name", ["sphere16", "sphere_ragged", "tower", "bumpy64"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_launch_shape_gives_the_same_preconditioner(env, name, precision):
    inputs, ufe, Solver = env
    p = inputs.bumpy_sphere(0) if name == "bumpy64" else small_problems()[name]
    out = {}
    saved = os.environ.get("UFE_PREC_SHAPE")
    try:
        for shape in ("4,0", "2,1", "2,4", "8,1", "8,2", "4,4"):
            os.environ["UFE_PREC_SHAPE"] = shape
            with Solver(p, precision=precision) as S:
                bi = S.bddc_info
                assert (bi["prec_cluster"], bi["prec_stages"]) == tuple(int(v) for v in shape.split(","))
                r = np.random.default_rng(9).normal(size=S.n_dof)
                z = S.precondition(r)
                _, info = S.solve(rtol=1e-8)
                out[shape] = (z, info["iterations"])
    finally:
        if saved is None:
            os.environ.pop("UFE_PREC_SHAPE", None)
        else:
            os.environ["UFE_PREC_SHAPE"] = saved
    z0, it0 = out["4,0"]
    tol, dit = (1e-12, 0) if precision == "fp64" else (1e-5, 1)
    for shape, (z, it) in out.items():
        assert np.linalg.norm(z - z0) <= tol * np.linalg.norm(z0), shape
        assert abs(it - it0) <= dit, shape


def test_tuner_picks_a_candidate_and_caches_it(env):
    inputs, ufe, Solver = env
    os.environ.pop("UFE_PREC_SHAPE", None)
    shapes = []
    for seed in (0, 1):
        with Solver(inputs.bumpy_sphere(seed), precision="mixed") as S:
            bi = S.bddc_info
            shapes.append((bi["prec_cluster"], bi["prec_stages"]))
    assert shapes[0][0] in (2, 4, 8) and shapes[0][1] in (1, 2, 4)
    assert shapes[1] == shapes[0]
