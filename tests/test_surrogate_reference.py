"""Pins of the FP64 surrogate reference (oracle/surrogate.py).

The surrogate is a learned approximation; its error against the spline is
measured, not pinned.  What is pinned here is that the reference computes
the function it defines: the derivative channels are the derivatives of the
value channel (central finite differences), the Laplacian channel is the
trace of the second derivatives, the hand-derived backward is the gradient
of the loss (finite differences on every kind of parameter), and the
function is periodic on the unit cube.
"""
import numpy as np
import pytest

from oracle import surrogate as S
from paper_1708_02645_gb300 import inputs

SMALL = S.SurrogateSpec(levels=3, log2_table=7, features=2, r_min=4, r_max=9, hidden=8,
                        layers=2, N=3)


def small_params(seed=1, grid_scale=0.5):
    return S.init_params(SMALL, seed=seed, grid_scale=grid_scale)


def test_resolutions_and_slots():
    spec = S.SurrogateSpec()
    R = spec.resolutions()
    assert R[0] == 16 and R[-1] == 512 and len(R) == 16 and all(np.diff(R) > 0)
    # dense levels (R^3 <= T) index directly; hashed ones stay within the table
    assert S.corner_slot(16, spec.table, 1, 2, 3) == (1 * 16 + 2) * 16 + 3
    h = S.corner_slot(512, spec.table, np.arange(100), np.arange(100) * 3, np.arange(100) * 7)
    assert h.min() >= 0 and h.max() < spec.table


def test_jets_are_derivatives_of_the_value():
    p = small_params()
    pos = inputs.uniform_positions(40, 3).astype(np.float64) * 0.98 + 0.01
    out, _ = S.forward(p, pos)
    d = 1e-6
    lap_fd = np.zeros_like(out[:, 0])
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = d
        up, _ = S.forward(p, pos + e)
        dn, _ = S.forward(p, pos - e)
        g_fd = (up[:, 0] - dn[:, 0]) / (2 * d)
        assert np.abs(g_fd - out[:, 1 + ax]).max() < 1e-5 * max(1.0, np.abs(out[:, 1 + ax]).max())
        lap_fd += (up[:, 1 + ax] - dn[:, 1 + ax]) / (2 * d)
    assert np.abs(lap_fd - out[:, 4]).max() < 1e-4 * max(1.0, np.abs(out[:, 4]).max())


def test_backward_matches_finite_differences():
    p = small_params(seed=2)
    pos = inputs.uniform_positions(16, 4).astype(np.float64)
    target = np.random.default_rng(0).normal(size=(16, 5, SMALL.N))
    wch = [1.0, 0.3, 0.3, 0.3, 0.05]
    L0, gg, gW, gb = S.grads(p, pos, target, wch)
    rng = np.random.default_rng(1)
    eps = 1e-6

    def fd(arr, idx):
        old = arr[idx]
        arr[idx] = old + eps
        lp = S.loss(S.forward(p, pos)[0], target, wch)
        arr[idx] = old - eps
        lm = S.loss(S.forward(p, pos)[0], target, wch)
        arr[idx] = old
        return (lp - lm) / (2 * eps)

    # grid entries actually touched by the positions, weights and biases
    _, cache = S.encode(p, pos)
    for l, (slots, _) in enumerate(cache):
        for q in rng.choice(slots.reshape(-1), size=3, replace=False):
            for f in range(SMALL.features):
                assert abs(fd(p.grid[l], (q, f)) - gg[l][q, f]) < 1e-6 * max(1.0, abs(gg[l][q, f]))
    for l in range(len(p.W)):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in p.W[l].shape)
            assert abs(fd(p.W[l], idx) - gW[l][idx]) < 1e-6 * max(1.0, abs(gW[l][idx]))
        j = int(rng.integers(0, p.b[l].shape[0]))
        assert abs(fd(p.b[l], (j,)) - gb[l][j]) < 1e-6 * max(1.0, abs(gb[l][j]))


def test_periodic_on_the_unit_cube():
    p = small_params(seed=3)
    pos = inputs.uniform_positions(30, 5).astype(np.float64)
    a, _ = S.forward(p, pos)
    b, _ = S.forward(p, pos + np.array([1.0, -2.0, 3.0]))
    assert np.array_equal(a, b)


def test_c2_across_cell_faces():
    """Values and derivatives are continuous across grid faces (the quintic
    weights are C2), also at the coarsest level's faces."""
    p = small_params(seed=4)
    base = inputs.uniform_positions(10, 6).astype(np.float64)
    base[:, 0] = 0.25                                  # a face of the R = 4 level
    e = np.array([1e-10, 0, 0])
    a, _ = S.forward(p, base - e)
    b, _ = S.forward(p, base + e)
    assert np.abs(a - b).max() < 1e-6


def test_rounding_helpers_match_library_conversions():
    """round_bf16 / round_fp16 agree with torch's bfloat16 and numpy's
    float16 conversions (round to nearest even) on FP32 inputs, including
    ties, subnormals of binary16 and large magnitudes."""
    torch = pytest.importorskip("torch")
    x = np.concatenate([
        (inputs.normal(7, 4000) * 10.0 ** (inputs.uniform01(8, 4000) * 12 - 6)),
        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 3e-6, -7e-7, 65504.0, 0.0]),
    ]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.round_bf16(x.astype(np.float64)), want)
    assert S.round_bf16(1.0 + 2.0 ** -8) == 1.0          # tie to even
    assert S.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    xh = x[np.abs(x) <= 65504.0]
    half = xh.astype(np.float16).astype(np.float64)
    assert np.array_equal(S.round_fp16(xh.astype(np.float64)), half)


def test_quantised_forward_is_close_and_rounds_inputs():
    """The inference reading (FP16 grid, BF16 weights, BF16 layer inputs)
    stays within a few bfloat16 roundings of the exact function, and with
    the identity as act_round and unquantised parameters it is the exact
    function bit for bit."""
    p = small_params(seed=5)
    pos = inputs.uniform_positions(50, 9).astype(np.float64)
    exact, _ = S.forward(p, pos)
    same, _ = S.forward(p, pos, act_round=lambda h: h)
    assert np.array_equal(exact, same)
    q, _ = S.forward(S.quantised(p), pos, act_round=S.round_bf16)
    for c in range(5):
        scale = np.abs(exact[:, c]).max()
        assert np.abs(q[:, c] - exact[:, c]).max() < 0.05 * scale
        assert np.abs(q[:, c] - exact[:, c]).max() > 0.0


def test_gemm_rounding_reading():
    """The tensor-core training reading (both operands of every product
    rounded to bfloat16): with the identity as rounding it is the exact
    backward bit for bit; with bfloat16 it stays within a few roundings."""
    p = small_params(seed=6)
    pos = inputs.uniform_positions(24, 10).astype(np.float64)
    target = np.random.default_rng(3).normal(size=(24, 5, SMALL.N))
    wch = [1.0, 0.3, 0.3, 0.3, 0.05]
    exact = S.grads(p, pos, target, wch)
    same = S.grads(p, pos, target, wch, gemm_round=lambda x: x)
    assert exact[0] == same[0]
    for a, b in zip([exact[1]] + exact[2] + exact[3], [same[1]] + same[2] + same[3]):
        assert np.array_equal(a, b)
    bf = S.grads(p, pos, target, wch, gemm_round=S.round_bf16)
    assert abs(bf[0] - exact[0]) < 0.05 * abs(exact[0])
    for a, b in zip(exact[2], bf[2]):
        assert 0 < np.abs(a - b).max() < 0.1 * np.abs(a).max()
