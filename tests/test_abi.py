"""The C-ABI library loads and exports every symbol include/spo.h declares;
host-side argument checks reject bad calls before touching CUDA.  No compute
calls: these run without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1708_02645_gb300 import build as spo_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "spo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spo_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    spo_build.build()
    from paper_1708_02645_gb300 import spo
    return spo.load()


def test_header_declares_expected_api():
    names = header_functions()
    for required in ("spo_create", "spo_destroy", "spo_eval_v", "spo_eval_vgl", "spo_eval_vgh",
                     "spo_eval", "spo_eval_host", "spo_footprint", "spo_status_str"):
        assert required in names


def test_library_exports_every_header_symbol(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, f"libspo.so lacks {missing}"


def test_binding_covers_every_header_symbol():
    from paper_1708_02645_gb300 import spo
    bound = {name for name, _, _ in spo.SIGNATURES}
    assert set(header_functions()) == bound


def test_host_only_queries(lib):
    assert lib.spo_abi_version() == 1
    assert [lib.spo_rows(k) for k in (0, 1, 2, 7)] == [1, 5, 10, 0]
    for s in range(6):
        assert lib.spo_status_str(s).startswith(b"SPO_")
    assert lib.spo_status_str(99) == b"unknown spo_status"


def test_create_rejects_bad_arguments_before_cuda(lib):
    from paper_1708_02645_gb300 import spo
    h = ctypes.c_void_p()
    buf = (ctypes.c_double * 64)()
    grid = spo._Grid(4, 4, 4)
    small = spo._Grid(3, 4, 4)
    # NULL out / grid / coefs, too-small grid, N < 1, bad dtypes, F64 storage
    assert lib.spo_create(ctypes.byref(grid), buf, 0, 1, 1, 0, None) == 1
    assert lib.spo_create(None, buf, 0, 1, 1, 0, ctypes.byref(h)) == 1
    assert lib.spo_create(ctypes.byref(grid), None, 0, 1, 1, 0, ctypes.byref(h)) == 1
    assert lib.spo_create(ctypes.byref(small), buf, 0, 1, 1, 0, ctypes.byref(h)) == 1
    assert b"n_d must be >= 4" in lib.spo_last_error()
    assert lib.spo_create(ctypes.byref(grid), buf, 0, 0, 1, 0, ctypes.byref(h)) == 1
    assert lib.spo_create(ctypes.byref(grid), buf, 9, 1, 1, 0, ctypes.byref(h)) == 1
    assert lib.spo_create(ctypes.byref(grid), buf, 0, 1, 0, 0, ctypes.byref(h)) == 5
    assert lib.spo_create(ctypes.byref(grid), buf, 0, 1, 7, 0, ctypes.byref(h)) == 1
    assert h.value is None


def test_eval_rejects_bad_arguments_before_cuda(lib):
    fake = ctypes.c_void_p(0)
    assert lib.spo_eval(None, 2, fake, 1, fake, None) == 1
    assert lib.spo_eval_vgh(None, fake, 1, fake, None) == 1
    assert lib.spo_eval_host(None, 2, fake, 1, fake, None) == 1
    b = ctypes.c_size_t()
    assert lib.spo_footprint(None, ctypes.byref(b)) == 1
    a = ctypes.c_int(-1)
    assert lib.spo_auto_algo(None, 2, 100, ctypes.byref(a)) == 1 and a.value == -1
    assert lib.spo_destroy(None) == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1708_02645_gb300 import spo
    monkeypatch.setattr(spo, "_lib", None)
    monkeypatch.setattr(spo, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        spo.load()


def test_newer_entry_points_reject_bad_arguments_before_cuda(lib):
    """Surrogate, prefilter, batch and self-test calls check their
    arguments on the host and return SPO_EINVAL (1) before any CUDA call."""
    from paper_1708_02645_gb300 import spo
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    bad = spo._SurrogateSpec(0, 19, 2, 16, 512, 128, 3, 0, 384)         # no levels
    good = spo._SurrogateSpec(16, 19, 2, 16, 512, 128, 3, 0, 384)
    assert lib.spo_surrogate_create(ctypes.byref(bad), 0, ctypes.byref(h)) == 1
    assert lib.spo_surrogate_create(ctypes.byref(good), 0, None) == 1
    wide = spo._SurrogateSpec(16, 19, 2, 16, 512, 128, 9, 0, 384)        # too many layers
    assert lib.spo_surrogate_create(ctypes.byref(wide), 0, ctypes.byref(h)) == 1
    assert h.value is None
    loss = ctypes.c_float()
    assert lib.spo_surrogate_eval(None, 1, fake, 1, fake, 1, None) == 1
    assert lib.spo_surrogate_train(None, None, 1, 1, 1e-3, None, 0, None, ctypes.byref(loss)) == 1
    assert lib.spo_surrogate_grad(None, fake, fake, 1, None, 0, ctypes.byref(loss), fake, fake, fake,
                                  None) == 1
    b = ctypes.c_size_t()
    assert lib.spo_surrogate_footprint(None, ctypes.byref(b)) == 1
    assert lib.spo_surrogate_set_optimizer(None, 0.9, 0.99, 1e-15, 1.0) == 1
    assert lib.spo_surrogate_set_train_precision(None, 1) == 1
    assert lib.spo_surrogate_set_level_lr(None, 2.0) == 1
    n = ctypes.c_int64()
    assert lib.spo_surrogate_nparams(None, ctypes.byref(n)) == 1
    assert lib.spo_surrogate_destroy(None) == 0
    grid = spo._Grid(8, 8, 8)
    assert lib.spo_prefilter(None, 4, fake, 0, None) == 1
    assert lib.spo_prefilter(ctypes.byref(grid), 0, fake, 0, None) == 1
    assert lib.spo_prefilter(ctypes.byref(grid), 4, fake, 3, None) == 1       # FP16 data
    t = ctypes.c_int()
    assert lib.spo_selftest_wait(2_000_000_000, None, ctypes.byref(t)) == 1
    assert lib.spo_selftest_wait(1000, None, None) == 1
    assert lib.spo_eval_batch(None, 0, None, 0, 2, None) == 1
    assert lib.spo_batch_create(None, 0, 1, 1, ctypes.byref(h)) == 1


def test_bounds_checked_units_compile():
    """The index-checking debug flavour (-DSPO_CHECK_BOUNDS) of the gather
    and binning units compiles (cross-compiled here; the GPU test builds and
    runs the whole checked library)."""
    import subprocess
    import tempfile
    from paper_1708_02645_gb300 import build
    with tempfile.TemporaryDirectory() as d:
        for src in ("spo_eval.cu", "spo_bin.cu"):
            cmd = [build.nvcc(), *build.ARCH, *build.NVCC_FLAGS, "-DSPO_CHECK_BOUNDS", "-c",
                   os.path.join(build.CSRC, src), "-o", os.path.join(d, src + ".o")]
            r = subprocess.run(cmd, capture_output=True, text=True)
            assert r.returncode == 0, r.stderr[-2000:]
