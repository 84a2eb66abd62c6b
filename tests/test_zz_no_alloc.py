"""ufe_bddc_apply_noalloc: z = M r with the intermediates in the library's static
device array instead of allocated buffers, for callers that must not allocate
device memory while they run.  Checked against ufe_bddc_apply, which uses the
buffers allocated by ufe_bddc_setup, on two calls in a row (the second call
reuses the array the first one left behind).  This file is named to be collected
last, so a run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_apply(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver

    dev = torch.device("cuda", 0)
    p = inputs.manufactured_sphere(0)
    with Solver(p, precision=precision) as S:
        rng = np.random.default_rng(17)
        for call in range(2):
            r = torch.from_numpy(rng.normal(size=S.n_dof)).to(dev)
            ref = ufe.ufe_bddc_apply(S.bddc, r)
            z = torch.full_like(r, float("nan"))
            ufe.ufe_bddc_apply_noalloc(S.bddc, r, z)
            torch.cuda.synchronize()
            assert torch.isfinite(z).all(), call
            # same kernels, same order: equal to rounding (the tolerance of the preconditioner tests)
            err = float((z - ref).norm() / ref.norm())
            assert err <= 1e-12, (call, err)


def test_noalloc_rejects_host_pointers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver
    with Solver(inputs.manufactured_sphere(0)) as S:
        with pytest.raises(TypeError):
            ufe.ufe_bddc_apply_noalloc(S.bddc, np.zeros(S.n_dof), np.zeros(S.n_dof))
