"""GPU surrogate (spo_surrogate_*) against the FP64 reference oracle/surrogate.py.

Tolerances, per output channel c, relative to max |ref_c| over the batch:
* FP32 master path: 2e-4.  The sums are at most K = 128 terms long (the
  encode adds 8 corners), so the FP32 error is below K u sum|terms| with
  u = 2^-24 and sum|terms| a few times max|out_c|: about 1e-5; the margin
  covers the cancelling Laplacian sums of the finest levels.
* inference path (FP16 grid, BF16 weights and layer inputs): 4e-3 against
  the reference's quantised reading.  Both round the same layer inputs to
  bfloat16; an FP32 accumulation difference can flip one rounding by one
  bfloat16 step (2^-8 relative) in a handful of activations.
* gradients: 1e-3 of max |ref| per parameter array (FP32 sums of up to 5P
  terms in atomic order).
"""
import numpy as np
import pytest

from oracle import surrogate as S
from paper_1708_02645_gb300 import inputs

pytestmark = pytest.mark.gpu

# ragged shapes: two dense and two hashed levels, widths that are not
# multiples of the GEMM tiles
RAGGED = S.SurrogateSpec(levels=4, log2_table=10, features=2, r_min=4, r_max=40, hidden=80,
                         layers=2, N=72)
# the full-size surrogate of the 384-orbital set (fused tensor-core inference)
FULL = S.SurrogateSpec()
# also served by the fused tensor-core kernel: one and two hidden layers, 16
# and 48 encoded features, output chunks of 128 + 128 + 16 and of 48
TC_ONE = S.SurrogateSpec(levels=8, log2_table=12, features=2, r_min=4, r_max=64, hidden=128,
                         layers=1, N=48)
TC_TWO = S.SurrogateSpec(levels=24, log2_table=14, features=2, r_min=4, r_max=128, hidden=128,
                         layers=2, N=272)


def torch():
    import torch as t
    return t


def load(spo_lib, spec, params):
    s = spo_lib.Surrogate(spec, seed=0)
    s.set_params(params.grid, params.W, params.b)
    return s


def channel_errors(got, ref):
    return [np.abs(got[:, c] - ref[:, c]).max() / max(np.abs(ref[:, c]).max(), 1e-30) for c in range(5)]


@pytest.mark.parametrize("spec,P,grid_scale", [(RAGGED, 333, 0.5), (FULL, 96, 0.05)])
def test_fp32_forward_matches_reference(spo_lib, spec, P, grid_scale):
    t = torch()
    p = S.as_float32(S.init_params(spec, seed=11, grid_scale=grid_scale))
    pos = np.concatenate([inputs.uniform_positions(P - 20, 12), inputs.wide_positions(20, 13)])
    ref, _ = S.forward(p, pos.astype(np.float64))
    with load(spo_lib, spec, p) as s:
        got = s.eval(t.from_numpy(pos).cuda(), precision=0).cpu().numpy().astype(np.float64)
        v = s.eval(t.from_numpy(pos).cuda(), kind="v", precision=0).cpu().numpy()
    err = channel_errors(got, ref)
    assert max(err) < 2e-4, err
    assert np.array_equal(v, got[:, 0].astype(np.float32))


@pytest.mark.parametrize("spec,P,grid_scale", [(RAGGED, 333, 0.5), (FULL, 96, 0.05),
                                               (FULL, 3001, 0.05), (TC_ONE, 333, 0.5),
                                               (TC_TWO, 250, 0.3)])
def test_inference_forward_matches_quantised_reference(spo_lib, spec, P, grid_scale):
    t = torch()
    p = S.as_float32(S.init_params(spec, seed=14, grid_scale=grid_scale))
    pos = np.concatenate([inputs.uniform_positions(P - 10, 15), inputs.wide_positions(10, 16)])
    ref, _ = S.forward(S.quantised(p), pos.astype(np.float64), act_round=S.round_bf16)
    with load(spo_lib, spec, p) as s:
        got = s.eval(t.from_numpy(pos).cuda(), precision=1).cpu().numpy().astype(np.float64)
        v = s.eval(t.from_numpy(pos).cuda(), kind="v", precision=1).cpu().numpy()
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    err = channel_errors(got, ref)
    assert max(err) < 4e-3, err
    assert np.array_equal(v, got[:, 0].astype(np.float32))


@pytest.mark.parametrize("P", [1, 129, 152 * 128 + 1])
def test_fused_tile_sizing_edges(spo_lib, P):
    """One position; one more than a tile; one more than a full wave of
    128-position tiles on 152 SMs (two waves of 65-position tiles)."""
    t = torch()
    p = S.as_float32(S.init_params(FULL, seed=32, grid_scale=0.05))
    pos = inputs.uniform_positions(P, 33)
    ref, _ = S.forward(S.quantised(p), pos.astype(np.float64), act_round=S.round_bf16)
    with load(spo_lib, FULL, p) as s:
        got = s.eval(t.from_numpy(pos).cuda(), precision=1).cpu().numpy().astype(np.float64)
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    err = channel_errors(got, ref)
    assert max(err) < 4e-3, err


# widths that are not multiples of 8 (the GEMM's scalar epilogue) and odd
# row counts
ODD = S.SurrogateSpec(levels=3, log2_table=9, features=2, r_min=3, r_max=11, hidden=36, layers=2, N=20)


@pytest.mark.parametrize("spec,P", [(RAGGED, 257), (FULL, 200), (ODD, 131)])
def test_tensor_core_gradients_match_rounded_reference(spo_lib, spec, P):
    """precision 1: the forward, weight-gradient and data-gradient products
    on the tensor cores with BF16 operands against the reference that rounds
    the same operands (tolerance 2e-3 of max |ref| per array: FP32
    accumulation order, and an operand whose FP32 and FP64 values straddle a
    bfloat16 rounding boundary now and then)."""
    t = torch()
    p = S.as_float32(S.init_params(spec, seed=34, grid_scale=0.3))
    pos = inputs.uniform_positions(P, 35)
    target = inputs.normal(36, P * 5 * spec.N).reshape(P, 5, spec.N).astype(np.float32)
    wch = [1.0, 0.25, 0.25, 0.25, 0.01]
    L, gg, gW, gb = S.grads(p, pos.astype(np.float64), target.astype(np.float64), wch,
                            gemm_round=S.round_bf16)
    with load(spo_lib, spec, p) as s:
        loss, ggot, Wgot, bgot = s.grad(t.from_numpy(pos).cuda(), t.from_numpy(target).cuda(),
                                        channel_weights=wch, precision=1)
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    assert abs(loss - L) < 1e-4 * abs(L)
    for got, ref in [(ggot, gg)] + list(zip(Wgot, gW)) + list(zip(bgot, gb)):
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 2e-3, err


@pytest.mark.parametrize("given", [True, False])
def test_gradients_match_reference(spo_lib, given):
    t = torch()
    spec = RAGGED
    p = S.as_float32(S.init_params(spec, seed=16, grid_scale=0.5))
    P = 257
    pos = inputs.uniform_positions(P, 17)
    target = inputs.normal(18, P * 5 * spec.N).reshape(P, 5, spec.N).astype(np.float32)
    tg = target.astype(np.float64)
    wch = [1.0, 0.25, 0.25, 0.25, 0.01] if given else \
        [1.0 / np.mean(tg[:, c] ** 2) for c in range(5)]
    L, gg, gW, gb = S.grads(p, pos.astype(np.float64), tg, wch)
    with load(spo_lib, spec, p) as s:
        loss, ggot, Wgot, bgot = s.grad(t.from_numpy(pos).cuda(), t.from_numpy(target).cuda(),
                                        channel_weights=wch if given else None)
        # the parameters are left as they were
        g2, W2, b2 = s.get_params()
        assert np.array_equal(g2, p.grid.astype(np.float32))
    assert abs(loss - L) < 1e-5 * abs(L)
    pairs = [(ggot, gg)] + list(zip(Wgot, gW)) + list(zip(bgot, gb))
    for got, ref in pairs:
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-3, err


def test_params_round_trip_and_footprint(spo_lib):
    spec = RAGGED
    p = S.init_params(spec, seed=19, grid_scale=0.5)
    with load(spo_lib, spec, p) as s:
        g, W, b = s.get_params()
        assert np.array_equal(g, p.grid.astype(np.float32))
        for a, r in zip(W + b, p.W + p.b):
            assert np.array_equal(a, r.astype(np.float32))
        T = 1 << spec.log2_table
        widths = spec.widths()
        nw = sum(i * o for i, o in zip(widths[:-1], widths[1:]))
        assert s.footprint() == 2 * spec.levels * T * spec.features + 2 * nw + 4 * sum(widths[1:])
    with spo_lib.Surrogate(FULL, seed=0) as s:
        # FP16 grid 32 MiB + BF16 weights + FP32 biases: about 33.9 MB
        assert s.footprint() < 34_000_000


def test_errors_and_empty(spo_lib):
    t = torch()
    with spo_lib.Surrogate(RAGGED, seed=0) as s:
        pos = t.zeros((0, 3), device="cuda")
        assert s.eval(pos).shape == (0, 5, RAGGED.N)
        pos = t.rand((4, 3), device="cuda")
        with pytest.raises(spo_lib.SpoError, match="SPO_EUNSUPPORTED"):
            s.eval(pos, kind="vgh")
        with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
            s.eval(pos, precision=2)
    # the fused tensor-core kernel writes 32-byte vectors: a misaligned output
    # is refused (this spec qualifies for it: 16 encoded features, width 128)
    tc = S.SurrogateSpec(levels=8, log2_table=12, features=2, r_min=2, r_max=16, hidden=128, layers=2, N=32)
    with spo_lib.Surrogate(tc, seed=0) as s:
        pos = t.rand((4, 3), device="cuda")
        base = t.empty(4 * 5 * tc.N + 8, device="cuda")
        with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
            s.eval(pos, out=base[4:4 + 4 * 5 * tc.N].view(4, 5, tc.N), precision=1)
        ok = s.eval(pos, out=base[8:8 + 4 * 5 * tc.N].view(4, 5, tc.N), precision=1)
        t.cuda.synchronize()
        assert t.equal(ok, s.eval(pos, precision=1))
    bad = S.SurrogateSpec(levels=0)
    with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
        spo_lib.Surrogate(bad)


def test_training_fits_the_spline(spo_lib):
    """Adam on spline VGL targets (16 low-frequency plane-wave orbitals)
    lowers the variance-normalised loss several times; the trained
    surrogate's error against the spline on held-out positions is measured
    for both precisions (reported; bounded loosely: a learned fit has no
    a-priori error bound)."""
    t = torch()
    N = 16
    coefs = inputs.plane_wave_coefs(16, 16, 16, N, seed=20, kmax=2.0).astype(np.float32)
    spec = S.SurrogateSpec(levels=8, log2_table=14, features=2, r_min=2, r_max=16, hidden=64,
                           layers=2, N=N)
    with spo_lib.OrbitalSet(coefs) as teacher, spo_lib.Surrogate(spec, seed=21) as s:
        first = s.train(teacher, steps=1, batch=4096, lr=1e-2, seed=22)
        last = s.train(teacher, steps=1000, batch=4096, lr=1e-2, seed=23)
        assert last < 0.25 * first, (first, last)
        pos = t.from_numpy(inputs.uniform_positions(5000, 24)).cuda()
        want = teacher.eval(pos, kind="vgl").cpu().numpy()
        for prec in (0, 1):
            got = s.eval(pos, precision=prec).cpu().numpy()
            rel = [np.sqrt(np.mean((got[:, c] - want[:, c]) ** 2) / np.mean(want[:, c] ** 2))
                   for c in range(5)]
            print(f"precision {prec}: relative RMS error V {rel[0]:.3g} G {max(rel[1:4]):.3g} "
                  f"L {rel[4]:.3g}")
            assert rel[0] < 0.35 and max(rel[1:4]) < 0.45, rel


def test_checkpoint_round_trip(spo_lib, tmp_path):
    """save() / load_checkpoint() restore parameters, Adam moments and the
    step count exactly; training resumes from the restored state."""
    t = torch()
    coefs = inputs.plane_wave_coefs(12, 12, 12, 16, seed=26, kmax=2.0).astype(np.float32)
    spec = S.SurrogateSpec(levels=6, log2_table=12, features=2, r_min=2, r_max=16, hidden=32,
                           layers=1, N=16)
    path = str(tmp_path / "surrogate.bin")
    with spo_lib.OrbitalSet(coefs) as teacher, spo_lib.Surrogate(spec, seed=27) as a, \
            spo_lib.Surrogate(spec, seed=28) as b:
        a.train(teacher, steps=20, batch=1024, lr=1e-2, seed=29)
        a.save(path, note="test")
        head = b.load_checkpoint(path)
        assert head["step"] == 20 and head["meta"]["note"] == "test"
        pa, ma, va, sa = a.state()
        pb, mb, vb, sb = b.state()
        assert sa == sb == 20
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb) and np.array_equal(va, vb)
        pos = t.from_numpy(inputs.uniform_positions(300, 30)).cuda()
        assert t.equal(a.eval(pos, precision=1), b.eval(pos, precision=1))
        la = a.train(teacher, steps=1, batch=1024, lr=1e-2, seed=31)
        lb = b.train(teacher, steps=1, batch=1024, lr=1e-2, seed=31)
        assert abs(la - lb) <= 1e-5 * abs(la)
    bad = S.SurrogateSpec(levels=6, log2_table=12, features=2, r_min=2, r_max=16, hidden=32,
                          layers=1, N=8)
    with spo_lib.Surrogate(bad, seed=0) as c:
        with pytest.raises(ValueError):
            c.load_checkpoint(path)


def test_initial_parameters_follow_the_generator_definition(spo_lib):
    """spo_surrogate_create draws the same splitmix64 streams as the
    reference's init_params (grid U(-1e-4, 1e-4), weights U(+-1/sqrt(in)),
    biases 0), rounded once to FP32."""
    ref = S.as_float32(S.init_params(RAGGED, seed=25))
    with spo_lib.Surrogate(RAGGED, seed=25) as s:
        g, W, b = s.get_params()
    assert np.array_equal(g, ref.grid.astype(np.float32))
    for a, r in zip(W + b, ref.W + ref.b):
        assert np.array_equal(a, r.astype(np.float32))


def test_level_learning_rates(spo_lib):
    """spo_surrogate_set_level_lr: Adam's first step moves every parameter
    with a gradient by its rate (to rounding: the grid gradients are summed
    with atomics), so the largest first-step change of level l's features is
    lr (R_0 / R_l)^power; resolutions 4, 8, 16, 32 here.  Power 0 is the
    default; out-of-range powers are refused."""
    t = torch()
    teacher_c = inputs.plane_wave_coefs(16, 16, 16, 32, seed=91).astype(np.float32)
    spec = S.SurrogateSpec(levels=4, log2_table=12, features=2, r_min=4, r_max=32, hidden=128, layers=2, N=32)
    with spo_lib.OrbitalSet(teacher_c) as teacher:
        states = []
        for power in (None, 0.0, 2.0):
            with spo_lib.Surrogate(spec, seed=5) as s:
                if power is not None:
                    s.set_level_lr(power)
                g0, _, _ = s.get_params()
                s.train(teacher, steps=1, batch=1024, lr=1e-2, seed=7)
                g1, _, _ = s.get_params()
                states.append(np.abs(g1 - g0).reshape(spec.levels, -1).max(axis=1))
        R = np.array([4.0, 8.0, 16.0, 32.0])
        np.testing.assert_allclose(states[0], 1e-2, rtol=1e-5)
        np.testing.assert_allclose(states[1], 1e-2, rtol=1e-5)
        np.testing.assert_allclose(states[2], 1e-2 * (R[0] / R) ** 2, rtol=1e-5)
        with spo_lib.Surrogate(spec, seed=5) as s:
            with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
                s.set_level_lr(5.0)
            with pytest.raises(spo_lib.SpoError, match="SPO_EINVAL"):
                s.set_level_lr(-1.0)


def _training_draw(seed, step, batch):
    """Positions of step `step` of a training call, from the documented
    stream: coordinate i is the top 24 bits of splitmix64(seed + (3 batch
    step + i + 1) 0x9E3779B97F4A7C15) over 2^24."""
    m64 = (1 << 64) - 1
    out = np.empty(3 * batch, dtype=np.float32)
    for i in range(3 * batch):
        z = (seed + (3 * batch * step + i + 1) * 0x9E3779B97F4A7C15) & m64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m64
        z ^= z >> 31
        out[i] = np.float32(z >> 40) / np.float32(16777216.0)
    return out.reshape(batch, 3)


def test_sparse_grid_updates_and_recapture(spo_lib):
    """The grid's Adam step is sparse: in a training call, a grid entry moves
    only if the call's batch gives it a gradient (dense Adam would also move
    the entries only the previous call touched, whose first moment is not
    zero); the perceptron's step is dense.  Calls that change the batch size
    or the per-level rates between replays of the captured step keep
    training, and the step count follows every step."""
    t = torch()
    coefs = inputs.plane_wave_coefs(12, 12, 12, 16, seed=41, kmax=2.0).astype(np.float32)
    spec = S.SurrogateSpec(levels=4, log2_table=10, features=2, r_min=2, r_max=16, hidden=32, layers=1, N=16)
    with spo_lib.OrbitalSet(coefs) as teacher, spo_lib.Surrogate(spec, seed=42) as s:
        s.train(teacher, steps=1, batch=64, lr=1e-2, seed=43)
        g1, W1, _ = s.get_params()
        pos = t.from_numpy(_training_draw(44, 0, 64)).cuda()
        _, gg, _, _ = s.grad(pos, teacher.eval(pos, kind="vgl"), precision=1)
        s.train(teacher, steps=1, batch=64, lr=1e-2, seed=44)
        g2, W2, _ = s.get_params()
        moved, touched = g2 != g1, gg != 0
        assert moved.any() and touched.sum() < 0.5 * touched.size
        assert not (moved & ~touched).any(), int((moved & ~touched).sum())
        for a, b in zip(W2, W1):
            assert (a != b).mean() > 0.9
        losses = [s.train(teacher, steps=4, batch=64, lr=1e-2, seed=45),
                  s.train(teacher, steps=4, batch=128, lr=5e-3, seed=46)]
        s.set_level_lr(1.0)
        losses.append(s.train(teacher, steps=4, batch=128, lr=5e-3, seed=47))
        assert np.all(np.isfinite(losses)), losses
        assert s.state()[3] == 14
