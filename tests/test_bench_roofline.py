"""The roofline arithmetic of bench.py (host logic, no GPU): achieved = algorithmic
work per launch / average launch time, frac = achieved / peak, the dominant kernel is
the instrumented kernel with a work count and the largest time per step, and the
per-iteration kernels count one launch per PCG iteration plus the initial one."""
import math

import bench


def _binfo(**kw):
    b = {"inverse_flops_local": 0.0, "inverse_flops_coarse": 1075.0 ** 3, "fp64_refactor": 0,
         "local_tensor_cores": 1}
    b.update(kw)
    return b


PEAKS = {"bf16_tflops_sustained": 1700.9, "source": "measured"}
FMA = {"fp64": 1.06, "fp32": 77.9}


def test_coarse_update_is_counted_as_a_cholesky_spread_over_its_launches():
    steps = 10
    kt = {"gj_update_f64": (1.19 * steps, 34 * steps)}   # 1.19 ms and 34 launches per step
    out = bench.roofline_block(kt, steps, _binfo(), None, 12, FMA, PEAKS, 0)
    work = 1075.0 ** 3 / 3.0 / 34.0
    t = 1.19e-3 / 34.0
    assert out["kernel"] == "gj_update_f64" and out["bound"] == "alu" and out["unit"] == "TFLOP/s"
    assert math.isclose(out["work_per_launch"], work, rel_tol=1e-12)
    assert math.isclose(out["achieved"], work / t / 1e12, rel_tol=1e-12)
    assert math.isclose(out["frac"], out["achieved"] / 1.06, rel_tol=1e-12)


def test_dominant_kernel_is_the_slowest_one_with_a_work_count():
    steps = 5
    kt = {"gj_update_f64": (1.0 * steps, 34 * steps),
          "gj_lookahead_f64": (9.0 * steps, 33 * steps),       # slower, but listed with its time only
          "integrate_cut": (2.0 * steps, 1 * steps)}
    out = bench.roofline_block(kt, steps, _binfo(), None, 12, FMA, PEAKS, n_subtets=1000)
    assert out["kernel"] == "integrate_cut"
    assert math.isclose(out["work_per_launch"], 54.0 * 35 * 1000, rel_tol=1e-12)
    names = [r["kernel"] for r in out["kernels"]]
    assert names[0] == "gj_lookahead_f64" and "achieved" not in out["kernels"][0]


def test_per_iteration_kernels_count_iterations_plus_one_launches():
    per_iter = {"peak_gbs": 6755.5, "peak_source": "measured",
                "prec_interior": {"us": 35.0, "bytes": 53.8e6}}
    out = bench.roofline_block({}, 1, _binfo(), per_iter, 12, FMA, PEAKS, 0)
    row = out["kernels"][0]
    assert row["kernel"] == "prec_interior" and row["launches_per_step"] == 13
    assert math.isclose(row["achieved"], 53.8e6 / 35e-6 / 1e9, rel_tol=1e-12)
    assert math.isclose(row["frac"], row["achieved"] / 6755.5, rel_tol=1e-12)


def test_fp32_tensor_update_uses_the_sustained_tf32_peak():
    steps = 2
    kt = {"gj_update_f32": (0.78 * steps, 14 * steps)}
    out = bench.roofline_block(kt, steps, _binfo(inverse_flops_local=3.0e11, inverse_flops_coarse=0.0), None, 12,
                               FMA, PEAKS, 0)
    tf32 = 1700.9 * bench.NOMINAL_TENSOR["tf32"] / bench.NOMINAL_TENSOR["bf16"]
    assert out["kernel"] == "gj_update_f32" and out["bound"] == "tensor"
    assert math.isclose(out["peak"], tf32, rel_tol=1e-12)
    assert math.isclose(out["work_per_launch"], 1.0e11 / 14, rel_tol=1e-12)


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reads_median_clock_and_throttle_reasons():
    """The clocks record of the bench line: median SM clock over the samples taken
    during the timed steps, the maximum clock, and every throttle reason seen Active
    (hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown reject a run; sw_power_cap
    is kept and noted)."""
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    c2 = bench.ClockSampler(0)
    c2.proc = _FakeProc()
    c2.lines = ["0, 1500, 2070, 1000, 0x40, Not Active, Active, Not Active, Not Active"]
    assert c2.stop()["reasons"] == ["hw_thermal_slowdown"]
