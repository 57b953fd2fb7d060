"""spo_eval_noalloc — the entry point for callers that must not have the
library allocate device memory (its scratch is a fixed per-device array).

Checked through the C ABI against the regular entry point (spo_eval_ex),
within the parity tolerance of the other tests, on two calls in a row with
different positions (the second call must not see the first call's binning).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1708_02645_gb300 import inputs
from parity import MAX_REL, errors

pytestmark = pytest.mark.gpu


def _call(lib, s, k, pos, out, stream=None):
    return lib.spo_eval_noalloc(s.handle, k, ctypes.c_void_p(pos.data_ptr()), int(pos.shape[0]),
                                ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("N,storage", [(96, "f32"), (40, "f32"), (130, "bf16")])
def test_noalloc_matches_regular_entry_point(spo_lib, N, storage):
    import torch
    lib = spo_lib.load()
    c = inputs.plane_wave_coefs(24, 20, 28, N, seed=23)
    with spo_lib.OrbitalSet(c, storage=storage) as s:
        for call, (P, seed) in enumerate(((50000, 31), (7777, 32))):
            pos = torch.from_numpy(inputs.wide_positions(P, seed)).cuda()
            for k, kind in ((2, "vgh"), (1, "vgl"), (0, "v")):
                ref = s.eval(pos, kind, algo="auto")
                out = torch.full_like(ref, float("nan"))
                assert _call(lib, s, k, pos, out) == 0, lib.spo_last_error()
                torch.cuda.synchronize()
                e = errors(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64), k)
                assert all(v["max_rel"] <= MAX_REL for v in e.values()), (call, kind, e)


def test_noalloc_rejects_requests_beyond_its_limits(spo_lib):
    import torch
    lib = spo_lib.load()
    c = inputs.uniform_coefs(8, 8, 8, 64, seed=3).astype(np.float32)
    with spo_lib.OrbitalSet(c) as s:
        too_many = torch.zeros((262145, 3), device="cuda")
        out = torch.empty((1, 1), device="cuda")
        assert _call(lib, s, 2, too_many, out) == 1
        assert b"SPO_NOALLOC_MAX_POSITIONS" in lib.spo_last_error()
    big = np.zeros((264, 264, 264, 1), dtype=np.float32)   # 66^3 bricks > 65,536
    with spo_lib.OrbitalSet(big) as s:
        pos = torch.zeros((16, 3), device="cuda")
        out = torch.empty((16, 10, 1), device="cuda")
        assert _call(lib, s, 2, pos, out) == 1
        assert b"SPO_NOALLOC_MAX_BRICKS" in lib.spo_last_error()
        assert _call(lib, s, 2, pos[:0], out) == 0   # empty batch: nothing to do
