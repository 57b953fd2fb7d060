"""spo_prefilter (interpolating coefficients) against the oracle's Fourier-space
prefilter, and end to end: a set built from prefiltered samples reproduces
the samples at the grid nodes.

Tolerances: FP64 data, 1e-12 of max |c| (two exact inversions of a
well-conditioned operator, eigenvalues in [1/3, 1], differing only in
rounding); FP32 data, 2e-6 of max |c| (the recursions keep FP64 state but
read and write FP32 between passes); node values of an FP32 table, 1e-5 of
max |f| (the FP32 kernel parity bound on V).  Shapes include a line of one
node and a line of 400 nodes."""
import numpy as np
import pytest

import oracle
from paper_1708_02645_gb300 import inputs

pytestmark = pytest.mark.gpu


def torch():
    import torch as t
    return t


@pytest.mark.parametrize("shape", [(4, 5, 6, 3), (16, 12, 20, 40), (48, 48, 48, 64), (3, 70, 1, 5),
                                   (400, 3, 2, 2)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_prefilter_matches_oracle(spo_lib, oracle_lib, shape, dtype):
    t = torch()
    f = inputs.plane_wave_coefs(*shape, seed=73) if shape[0] > 3 else inputs.uniform_coefs(*shape, seed=74)
    want = oracle.prefilter(f)
    tdt = t.float64 if dtype == "f64" else t.float32
    d = t.from_numpy(f).to(tdt).cuda()
    spo_lib.prefilter(d)
    got = d.cpu().double().numpy()
    tol = 1e-12 if dtype == "f64" else 2e-6
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_prefiltered_set_interpolates_samples(spo_lib, oracle_lib):
    t = torch()
    ns, N = (24, 20, 28), 48
    f = inputs.plane_wave_coefs(*ns, N, seed=75)
    d = t.from_numpy(f).cuda()
    spo_lib.prefilter(d)
    with spo_lib.OrbitalSet(d, src_dtype="f64") as s:
        nodes = np.stack(np.meshgrid(*[np.arange(n) / n for n in ns], indexing="ij"), -1).reshape(-1, 3)
        v = s.eval(t.from_numpy(nodes.astype(np.float32)).cuda(), "v").cpu().numpy()
    assert np.abs(v - f.reshape(-1, N)).max() <= 1e-5 * np.abs(f).max()


def test_prefilter_errors(spo_lib):
    t = torch()
    with pytest.raises(TypeError):
        spo_lib.prefilter(t.zeros((4, 4, 4, 2), dtype=t.float16, device="cuda"))
    with pytest.raises(TypeError):
        spo_lib.prefilter(t.zeros((4, 4, 4, 2), dtype=t.float64))
