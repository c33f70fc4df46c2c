"""Host-side pieces of bench.py that need no GPU: the DRAM-traffic ratio read
from the committed ncu summary of the sweep tiles (the `traffic` figure of the
roofline object), and the FP32 SIMT peak derived from the SM count."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_ratio_from_profile():
    r = bench.fronts_traffic("overthrust5", 1.0)
    assert r is not None and 1.0 < r < 3.0      # DRAM bytes / algorithmic bytes of one application
    assert bench.fronts_traffic("overthrust5", 2.0) == 2.0 * r
    assert bench.fronts_traffic("cube", 1.0) is None   # the cube's factors fit in L2


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
