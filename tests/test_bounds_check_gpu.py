"""The index-checking debug build (-DSPO_CHECK_BOUNDS).

In that build the kernels check the indices they are about to use (a
position's cell against the brick its CTA staged, a sorted slot, a
permutation entry, the window's table rows) and, when one fails, set bit 1
of the device status word and skip the access.  On valid inputs it must
change nothing: the checked library, built into a temporary directory and
run in a subprocess, gives the regular library's outputs bit for bit for
every strategy and kind, and leaves the status word clean.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1708_02645_gb300 import build

pytestmark = pytest.mark.gpu

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    from paper_1708_02645_gb300 import inputs, spo
    out = {}
    coefs = inputs.plane_wave_coefs(24, 20, 28, 96, seed=5)
    pos = torch.from_numpy(inputs.wide_positions(20000, 6)).cuda()
    with spo.OrbitalSet(coefs) as s:
        for kind in ("v", "vgl", "vgh"):
            for algo in ("gather", "sorted_gather", "brick"):
                out[kind + "_" + algo] = s.eval(pos, kind, algo=algo).cpu().numpy()
    torch.cuda.synchronize()
    out["status"] = np.array([spo.device_status()])   # raises if a check failed
    out["library"] = np.array([spo.library_path()])
    np.savez(sys.argv[1], **out)
""")


def _run_child(path, library, root):
    env = dict(os.environ)
    env.pop("SPO_LIBRARY", None)
    if library:
        env["SPO_LIBRARY"] = library
    r = subprocess.run([sys.executable, "-c", CHILD, str(path)], cwd=root, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_checked_build_changes_nothing_on_valid_inputs(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    checked = build.build(extra_flags=["-DSPO_CHECK_BOUNDS"], out_dir=str(tmp_path / "checked"))
    ref = _run_child(tmp_path / "ref.npz", None, root)
    chk = _run_child(tmp_path / "chk.npz", checked, root)
    assert str(chk["library"][0]) == checked and str(ref["library"][0]) != checked
    assert int(chk["status"][0]) == 0
    for k in ref.files:
        if k not in ("status", "library"):
            assert np.array_equal(ref[k], chk[k]), k
