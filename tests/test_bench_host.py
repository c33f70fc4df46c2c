"""Host-side pieces of bench.py that need no GPU: the DRAM-traffic ratio read
from the committed ncu summary of the sweep tiles (the `traffic` figure of the
roofline object), and the FP32 SIMT peak derived from the SM count."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_ratio_from_profile(tmp_path, monkeypatch):
    # the committed summary carries the ratio only while it was measured on the current kernels
    r = bench.fronts_traffic("overthrust5", 1.0)
    assert r is None or 1.0 < r < 3.0
    prof = tmp_path / "k_mf_tile.md"
    prof.write_text("# summary\n| quantity | value |\n|---|---|\n| dram_over_algorithmic | 1.48 |\n")
    monkeypatch.setattr(bench, "TILE_PROFILE", str(prof))
    assert abs(bench.fronts_traffic("overthrust5", 2.0) - 2.96) < 1e-12   # DRAM bytes per application
    assert bench.fronts_traffic("cube", 1.0) is None   # the cube's factors fit in L2
    monkeypatch.setattr(bench, "TILE_PROFILE", str(tmp_path / "absent.md"))
    assert bench.fronts_traffic("overthrust5", 1.0) is None


def test_simt_peak_formula():
    class Props:
        multi_processor_count = 152

    class Cuda:
        @staticmethod
        def get_device_properties(_):
            return Props()

        @staticmethod
        def current_device():
            return 0

    class Torch:
        cuda = Cuda()

    tf, sms, mhz = bench.fp32_simt_tflops(Torch(), 2070.0)
    assert sms == 152 and mhz == 2070.0
    assert abs(tf - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
