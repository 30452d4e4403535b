"""The LOP3 throughput probe (kpz_alu_peak) against the ALU pipe's derived
peak: 16 lanes per SM sub-partition per clock, 4 sub-partitions per SM."""
import pytest

from tests.gpu_util import engine

pytestmark = pytest.mark.gpu


def test_alu_probe_is_near_the_derived_peak():
    import torch
    eng = engine()
    r = eng._lib.alu_peak()
    props = torch.cuda.get_device_properties(0)
    max_hz = 2.2e9   # above any GB300 SM clock: the probe cannot exceed this bound
    assert 0 < r["lane_ops_per_s"] < props.multi_processor_count * 64 * max_hz
    # at least a third of the pipe's rate even at a reduced clock
    assert r["lane_ops_per_s"] > props.multi_processor_count * 64 * 1.0e9 / 3
    assert r["kernel_ms"] > 0
