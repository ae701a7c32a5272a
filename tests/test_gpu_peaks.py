"""The library's peak micro-benchmarks (mvs_measure_peaks) give plausible
figures on the GPU: the FFMA rate below the FP32 units' limit at the maximum
SM clock and above half of it, L1 gathers above the L2 stream's rate in
8-byte loads, an L2 bandwidth above the HBM copy bandwidth."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible(mvs_lib):
    import torch
    p = torch.cuda.get_device_properties(0)
    f, g, b = mvs_lib.mvs_measure_peaks(0)
    limit = p.multi_processor_count * 128 * 2 * 2.1e9        # FP32 lanes x 2 flop x a clock above the maximum
    print(f"FFMA {f / 1e12:.1f} TFLOP/s, L1 gathers {g / 1e12:.2f} T/s, L2 {b / 1e9:.0f} GB/s")
    assert 0.5 * limit < f < limit
    assert g > b / 8
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as fh:
            hbm = float(json.load(fh)["hbm_gbs"]) * 1e9
    except (OSError, KeyError, ValueError):
        hbm = 5e12
    assert b > hbm
    with pytest.raises(mvs_lib.MvsError):
        mvs_lib.mvs_measure_peaks(torch.cuda.device_count())
