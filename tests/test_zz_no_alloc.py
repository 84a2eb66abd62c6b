"""ufe_bddc_apply_noalloc: z = M r with the intermediates in the library's static
device array instead of allocated buffers, for callers that must not allocate
device memory while they run (a serving loop holding a fixed memory budget, or
host code called back from a framework that owns the device allocator).

Checked against ufe_bddc_apply, which uses the buffers allocated by
ufe_bddc_setup, on two calls in a row (the second call reuses the array the first
one left behind), with the three coarse solvers (dense, cyclic reduction, and the
three-level method, whose level-2 work space set-up allocates); the free device memory is unchanged
across calls made right after set-up; problems beyond the array's limits are
refused.  This file is named to be collected last, so a run that stops at the
first failure has run every other test first.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06323_gb300 import build_ext
    build_ext.build()
    from paper_1703_06323_gb300 import inputs, ufe
    from paper_1703_06323_gb300.solver import Solver
    return torch, inputs, ufe, Solver


def _problem(inputs, name):
    if name == "tower":
        from tests.oracle_cache import _tower
        return _tower()
    return inputs.manufactured_sphere(0)


@pytest.mark.parametrize("name,coarse_solver", [("sphere16", "dense"), ("tower", "cr"), ("tower", "bddc")])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_allocating_apply(precision, name, coarse_solver):
    torch, inputs, ufe, Solver = _env()
    dev = torch.device("cuda", 0)
    with Solver(_problem(inputs, name), precision=precision, coarse_solver=coarse_solver) as S:
        want = {"dense": ufe.COARSE_SOLVER_DENSE, "cr": ufe.COARSE_SOLVER_CR, "bddc": ufe.COARSE_SOLVER_BDDC}[coarse_solver]
        assert S.bddc_info["coarse_solver"] == want
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


@pytest.mark.parametrize("coarse_solver", ["dense", "cr", "bddc"])
def test_noalloc_takes_no_device_memory(coarse_solver):
    """Right after set-up (no other apply or solve before it), two calls leave the
    free device memory exactly as it was: set-up already loaded the device code and
    looked up the static array, so nothing is loaded or allocated inside the call."""
    torch, inputs, ufe, Solver = _env()
    dev = torch.device("cuda", 0)
    with Solver(_problem(inputs, "tower"), precision="mixed", coarse_solver=coarse_solver) as S:
        r = torch.from_numpy(np.random.default_rng(5).normal(size=S.n_dof)).to(dev)
        z = torch.empty_like(r)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        ufe.ufe_bddc_apply_noalloc(S.bddc, r, z)
        ufe.ufe_bddc_apply_noalloc(S.bddc, r, z)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info(dev)[0]
        assert free1 == free0, (free0, free1)
        ref = ufe.ufe_bddc_apply(S.bddc, r)
        assert float((z - ref).norm() / ref.norm()) <= 1e-12


def test_noalloc_refuses_problems_beyond_its_limits():
    """An uncut 80^3 box in 8^3-cell blocks has 1000 subdomains and more than the
    262,144 interface slots the static array holds: the call is refused with
    UFE_ERR_INVALID_ARG naming the limit, and z is left untouched."""
    torch, inputs, ufe, Solver = _env()
    dev = torch.device("cuda", 0)
    p = inputs.box_problem(cells=(80, 80, 80))
    with Solver(p, precision="mixed") as S:
        assert S.bddc_info["interface_slots"] > 262144
        r = torch.ones(S.n_dof, dtype=torch.float64, device=dev)
        z = torch.full_like(r, 7.0)
        with pytest.raises(ufe.UfeError) as ei:
            ufe.ufe_bddc_apply_noalloc(S.bddc, r, z)
        assert ei.value.status == ufe.ERR_INVALID_ARG
        assert "262144" in str(ei.value) and "interface slots" in str(ei.value)
        torch.cuda.synchronize()
        assert bool((z == 7.0).all())


def test_noalloc_rejects_host_pointers():
    torch, inputs, ufe, Solver = _env()
    with Solver(inputs.manufactured_sphere(0)) as S:
        with pytest.raises(TypeError):
            ufe.ufe_bddc_apply_noalloc(S.bddc, np.zeros(S.n_dof), np.zeros(S.n_dof))
