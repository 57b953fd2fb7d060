"""spo_eval_noalloc — the entry point for callers that must not have the
library allocate device memory (its scratch is a fixed per-device array).

Checked through the C ABI against the regular entry point (spo_eval_ex with
SPO_ALGO_AUTO, the strategy the no-allocation call also takes): the outputs
must be equal bit for bit, on two calls in a row with different positions
(the second call must not see the first call's binning), and repeated calls
must leave the device's free memory unchanged.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1708_02645_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = ((2, "vgh"), (1, "vgl"), (0, "v"))


def _call(lib, s, k, pos, out, stream=None):
    return lib.spo_eval_noalloc(s.handle, k, ctypes.c_void_p(pos.data_ptr()), int(pos.shape[0]),
                                ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("N,storage", [(96, "f32"), (40, "f32"), (130, "bf16")])
def test_noalloc_matches_regular_entry_point(spo_lib, N, storage):
    import torch
    lib = spo_lib.load()
    c = inputs.plane_wave_coefs(24, 20, 28, N, seed=23)
    with spo_lib.OrbitalSet(c, storage=storage) as s:
        # 50,000 positions take the brick kernel (VGH) or the binned gather
        # kernel, 7,777 the binned gather kernel, 600 the unbinned one
        for call, (P, seed) in enumerate(((50000, 31), (7777, 32), (600, 33))):
            pos = torch.from_numpy(inputs.wide_positions(P, seed)).cuda()
            for k, kind in KINDS:
                ref = s.eval(pos, kind, algo="auto")
                out = torch.full_like(ref, float("nan"))
                assert _call(lib, s, k, pos, out) == 0, lib.spo_last_error()
                torch.cuda.synchronize()
                assert torch.equal(out, ref), (call, kind, P, (out - ref).abs().max().item())


def test_noalloc_allocates_nothing(spo_lib):
    import torch
    lib = spo_lib.load()
    c = inputs.plane_wave_coefs(32, 32, 32, 64, seed=29)
    with spo_lib.OrbitalSet(c, storage="f32") as s:
        pos = [torch.from_numpy(inputs.uniform_positions(60000, 40 + i)).cuda() for i in range(2)]
        outs = {k: torch.empty(s.out_shape(60000, kind), device="cuda") for k, kind in KINDS}
        # the first calls look up the scratch array and load the kernels'
        # code on first use (lazy module loading), which may take memory
        for k, _ in KINDS:
            assert _call(lib, s, k, pos[1], outs[k]) == 0, lib.spo_last_error()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for rep in range(3):
            for k, _ in KINDS:
                assert _call(lib, s, k, pos[rep % 2], outs[k]) == 0, lib.spo_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        # and the results are still those of the regular entry point
        for k, kind in KINDS:
            assert torch.equal(outs[k], s.eval(pos[0], kind, algo="auto")), kind


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
