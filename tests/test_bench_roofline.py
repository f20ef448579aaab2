"""The arithmetic of the benchmark's roofline object (host logic, no GPU):
the step kernel's gathered bytes count 20 B per FP32 source voxel (five FP32
channels) and 8 B per FP16 one (channels c0..c3 in half precision), over the
kernel's own time, against the measured copy bandwidth; the per-evaluation
unit counts a whole 125-voxel FP32 patch; and the DRAM traffic per launch is
the captured bytes per gathered voxel scaled by this run's gathered voxels,
reported only for the configuration it was captured on."""
from types import SimpleNamespace

import pytest

import bench


def _args(**kw):
    a = dict(storage="fp16", sub_sweeps=2, lanes=0, realign=False, rs_mode="eq3")
    a.update(kw)
    return SimpleNamespace(**a)


def test_gathered_bytes_and_fraction():
    # 1e9 FP32 voxels and 5e8 FP16 voxels in 0.5 s against a 10,000 GB/s peak
    r = bench.step_roofline(gathered=1e9, gathered_h=5e8, step_evals=2e8, step_ms=500.0, wall_ms=1000.0,
                            peak=10000.0, peak_kind="measured", kernel="k", traffic=None, launches=100)
    gbytes = 1e9 * 20 + 5e8 * 8
    assert r["achieved"] == pytest.approx(gbytes / 0.5 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 10000.0)
    assert r["gathered_bytes_per_launch"] == pytest.approx(gbytes / 100)
    assert r["gathered_voxels_per_eval"] == pytest.approx(1.5e9 / 2e8)
    assert r["kernel_ms_share"] == pytest.approx(0.5)
    # a whole FP32 patch per counted evaluation: 125 voxels x 5 channels x 4 B
    assert bench.BYTES_PER_EVAL_FP32_C5 == 2500
    assert r["per_evaluation_unit"]["achieved"] == pytest.approx(2e8 * 2500 / 0.5 / 1e9)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_no_roofline_without_kernel_time():
    assert bench.step_roofline(1.0, 0.0, 1.0, 0.0, 1.0, 1.0, "measured", "k", None, 1) is None


def test_traffic_scales_the_captured_figure_by_gathered_voxels():
    per_voxel = bench.NCU_STEP_TRAFFIC[("batch48", "fp16", 2)]
    got = bench.step_traffic(_args(), "batch48", gathered=3e10, gathered_h=4e9, launches=1800)
    assert got == pytest.approx(per_voxel * 3.4e10 / 1800)
    # the FP32 capture for FP32 storage
    got32 = bench.step_traffic(_args(storage="fp32"), "batch48", 1e10, 0.0, 1000)
    assert got32 == pytest.approx(bench.NCU_STEP_TRAFFIC[("batch48", "fp32", 2)] * 1e10 / 1000)


@pytest.mark.parametrize("kw", [dict(storage="fp16-all"), dict(sub_sweeps=1), dict(lanes=8), dict(realign=True),
                                dict(rs_mode="multi")])
def test_traffic_is_null_off_the_captured_configuration(kw):
    assert bench.step_traffic(_args(**kw), "batch48", 3e10, 4e9, 1800) is None


def test_traffic_is_null_for_another_workload_or_no_launches():
    assert bench.step_traffic(_args(), "layered_1280x720x100", 3e10, 4e9, 1800) is None
    assert bench.step_traffic(_args(), "batch48", 3e10, 4e9, 0) is None
