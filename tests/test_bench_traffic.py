"""Host logic of the bench's captured-traffic table: volume scaling, system-count match, source check."""
import numpy as np

import bench


def test_traffic_scales_with_volume_for_the_captured_system_count():
    e = bench.KERNEL_TRAFFIC["dirac_f32"]
    got = bench.kernel_traffic("dirac_f32", e["L"], e["nsys"])
    assert got == e["bytes"]
    L2 = tuple(2 * v for v in e["L"])
    assert bench.kernel_traffic("dirac_f32", L2, e["nsys"]) == int(e["bytes"] * 16)


def test_traffic_is_null_for_another_system_count_or_an_unknown_kernel():
    e = bench.KERNEL_TRAFFIC["sap_mr"]
    assert bench.kernel_traffic("sap_mr", e["L"], e["nsys"] + 1) is None
    assert bench.kernel_traffic("no_such_kernel", e["L"], e["nsys"]) is None


def test_traffic_is_null_once_the_sources_change(monkeypatch):
    e = dict(bench.KERNEL_TRAFFIC["dirac_f32"])
    e["sha1"] = {"dirac.cu": "0" * 40}
    monkeypatch.setitem(bench.KERNEL_TRAFFIC, "dirac_f32", e)
    assert bench.kernel_traffic("dirac_f32", e["L"], e["nsys"]) is None


def test_stencil_bytes_formula():
    # 4 links (18 reals) + clover (72 reals) + every system read and written (24 reals each)
    assert bench.dirac_bytes_per_site(16, 32) == 576 + 192 * 16
    assert bench.dirac_bytes_per_site(1, 64) == 1152 + 384
    assert np.isclose(bench.FP32_ALU_PEAK_TFLOPS, 152 * 128 * 2 * 2.070e9 / 1e12)
