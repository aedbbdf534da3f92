"""Failure handling on the GPU without a fault: a bounded mbarrier wait that runs out
records code 1 in the device status word, the host reads and clears it, and the
context stays usable for the next call."""
import numpy as np
import pytest
import torch

from metrics import check_float_output, conv_reference
from paper_1605_06399_gb300 import ImclError, _abi, ops, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    assert ops.device_status() == 0


def test_bounded_wait_times_out_and_reports():
    assert ops.device_status() == 0
    ops.selftest_wait_timeout(1000)
    assert ops.device_status() == 1, "the wait that cannot complete did not report its timeout"
    assert ops.device_status() == 0, "reading the status word clears it"
    g = np.random.default_rng(31)
    x = synth.uniform_f32(g, 64, 80)
    w = synth.normal_filter_l1(g, 5)
    y = ops.conv2d(torch.from_numpy(x).cuda(), w)
    ref, s = conv_reference(x, w)
    check_float_output(y, ref, s, torch.float32, "conv2d after a timed-out wait")
    assert ops.device_status() == 0


def test_selftest_rejects_unbounded_rounds():
    for bad in (0, -1, (1 << 20) + 1):
        with pytest.raises(ImclError) as ei:
            ops.selftest_wait_timeout(bad)
        assert ei.value.status == _abi.ERR_INVALID
