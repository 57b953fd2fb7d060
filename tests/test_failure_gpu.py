"""Failure detection on the GPU without a fault: a bounded wait that cannot
succeed (an mbarrier nothing arrives on) gives up after its limit, the
device status word reports it, and the context stays usable."""
import time

import numpy as np
import pytest

import oracle
from paper_1708_02645_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports(spo_lib):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert spo_lib.selftest_wait(50_000_000) is True
    dt = time.perf_counter() - t0
    assert dt >= 0.045, dt          # the probe really waited its 50 ms
    assert spo_lib.device_status() == 0   # read and cleared by the self-test
    # the context is still usable: an evaluation runs and matches the oracle
    c = inputs.uniform_coefs(8, 9, 10, 12, seed=101).astype(np.float32)
    pos = inputs.uniform_positions(200, 102)
    with spo_lib.OrbitalSet(c) as s:
        got = s.eval(torch.from_numpy(pos).cuda(), "v").cpu().numpy()
    ref = oracle.spo_eval(c.astype(np.float64), pos.astype(np.float64), oracle.KIND_V)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_selftest_rejects_long_limits(spo_lib):
    with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
        spo_lib.selftest_wait(2_000_000_000)
