"""FP32 local inversions on the tensor cores (tcgen05 kind::tf32, 3xTF32 split products)
against the SIMT FP32 Gauss-Jordan (UFE_FP32_GJ=simt) and the FP64 operators.

The mixed-precision preconditioner z = M r must stay as close to the FP64 one as the
SIMT FP32 inversion keeps it (3xTF32 carries about FP32 accuracy: a few times the
SIMT error at most, and within the mixed tolerance), on the parity geometries (matrices
of one to seven 64-wide blocks, ragged last blocks, 4^3 and 8^3 subdomain blocks) and
on the 64^3 bench workload; PCG takes the same iterations.
"""
import os

import numpy as np
import pytest

from tests.oracle_cache import small_problems

pytestmark = pytest.mark.gpu

NAMES = ["sphere16", "sphere_ragged", "plane", "tower", "slab_sliver", "u_shape", "box_dirichlet", "one_subdomain"]


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


def _compare(env, p):
    inputs, ufe, Solver = env
    out = {}
    saved = os.environ.get("UFE_FP32_GJ")
    try:
        with Solver(p, precision="fp64") as S64:
            r = np.random.default_rng(3).normal(size=S64.n_dof)
            z64 = S64.precondition(r)
            _, i64 = S64.solve(rtol=1e-8)
            for mode in ("simt", "tc"):
                if mode == "simt":
                    os.environ["UFE_FP32_GJ"] = "simt"
                else:
                    os.environ.pop("UFE_FP32_GJ", None)
                with Solver(p, precision="mixed") as S:
                    z = S.precondition(r)
                    _, info = S.solve(rtol=1e-8)
                    bi = S.bddc_info
                e = z - z64
                err = float(np.sqrt(abs(e @ S64.apply(e)) / abs(z64 @ S64.apply(z64))))
                out[mode] = (err, bi, info)
    finally:
        if saved is None:
            os.environ.pop("UFE_FP32_GJ", None)
        else:
            os.environ["UFE_FP32_GJ"] = saved
    return out, i64


def _check(out):
    (e_simt, bi_simt, it_simt), (e_tc, bi_tc, it_tc) = out["simt"], out["tc"]
    if bi_tc["fp64_refactor"]:
        assert bi_tc["local_tensor_cores"] == 0
        return
    assert bi_tc["local_tensor_cores"] == 1 and bi_simt["local_tensor_cores"] == 0
    assert e_tc <= max(4.0 * e_simt, 1e-6), (e_tc, e_simt)
    assert e_tc <= 1e-4
    assert it_tc["converged"] == 1 and it_tc["iterations"] == it_simt["iterations"]


@pytest.mark.parametrize("name", NAMES)
def test_tensor_core_inverse_matches_simt(env, name):
    out, _ = _compare(env, small_problems()[name])
    _check(out)


def test_tensor_core_inverse_on_bench_workload(env):
    inputs, _, _ = env
    out, i64 = _compare(env, inputs.bumpy_sphere(0))
    _check(out)
    assert out["tc"][2]["iterations"] <= i64["iterations"] + 1
