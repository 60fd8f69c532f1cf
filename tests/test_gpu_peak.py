"""The FP32 FMA calibration kernel: a plausible rate, bounded by the unit-count
limit (SMs x 128 lanes x 2 flop x maximum SM clock, times 2 for the packed
two-lane form), and argument checks."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fp32_peak_plausible():
    import paper_2609_30644_gb300 as mp
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12   # 2.2 GHz > any SM clock
    s = mp.fp32_peak(False, iters=4096)
    p = mp.fp32_peak(True, iters=4096)
    assert 0.2 * bound < s <= bound
    assert 0.2 * bound < p <= 2 * bound
    with pytest.raises(mp.MrpopError):
        mp.fp32_peak(False, iters=0)
