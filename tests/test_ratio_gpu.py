"""GPU determinant ratios (spo_eval_ratio) against the FP64 oracle.

rho_p = (row r(p) of A^-1) . phi(pos_p), eq. md_lemma; the oracle's ratio is
pinned to det(A')/det(A) in test_oracle_pins.py.  Tolerance: |d| <= 1e-5 x
sum_j |a_j| beta_j (beta: the condition sums of the values), which covers the
FP32 value error (64 2^-24 beta_j per orbital) and the FP32 dot product.
"""
import numpy as np
import pytest

import oracle
from paper_1708_02645_gb300 import inputs

pytestmark = pytest.mark.gpu


def torch():
    import torch as t
    return t


def check(got, coefs32, pos, rows, row_of):
    vals = coefs32.astype(np.float64)
    ref = oracle.spo_ratio(vals, pos.astype(np.float64), rows, row_of)
    cond = oracle.spo_ratio_condition(vals, pos.astype(np.float64), rows, row_of)
    d = np.abs(got.astype(np.float64) - ref)
    bad = d > 1e-5 * cond
    assert not bad.any(), f"{bad.sum()} ratios off; worst {(d / cond).max():.3g}"
    return (d / cond).max()


@pytest.mark.parametrize("grid,N,P,nrows", [((48, 48, 48), 192, 12288, 384),
                                            ((20, 22, 24), 100, 5000, 5000),
                                            ((9, 10, 11), 13, 2000, 64),
                                            ((16, 16, 16), 40, 300, 300)])
def test_ratio_matches_oracle(spo_lib, oracle_lib, grid, N, P, nrows):
    """Brick path (fused epilogue) for the first two shapes, value + dot
    kernels for the small set and the small batch; shared rows via row_of."""
    t = torch()
    c = inputs.plane_wave_coefs(*grid, N, seed=61).astype(np.float32)
    pos = inputs.wide_positions(P, seed=62)
    rows = (2.0 * inputs.uniform01(63, nrows * N) - 1.0).astype(np.float32).reshape(nrows, N)
    row_of = None if nrows == P else (inputs.uniform01(64, P) * nrows).astype(np.int32)
    with spo_lib.OrbitalSet(c) as s:
        ro = None if row_of is None else t.from_numpy(row_of).cuda()
        got = s.eval_ratio(t.from_numpy(pos).cuda(), t.from_numpy(rows).cuda(), ro)
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    check(got.cpu().numpy(), c, pos, rows, row_of)


def test_ratio_values_and_paths_agree(spo_lib):
    """v_out of the fused kernel equals the V evaluation bit for bit; the
    fused and unfused paths agree within the tolerance."""
    t = torch()
    c = inputs.plane_wave_coefs(24, 24, 24, 128, seed=65).astype(np.float32)
    P = 20000
    pos = t.from_numpy(inputs.uniform_positions(P, 66)).cuda()
    rows = t.from_numpy((2 * inputs.uniform01(67, P * 128) - 1).astype(np.float32).reshape(P, 128)).cuda()
    with spo_lib.OrbitalSet(c) as s:
        v = t.empty((P, 128), device="cuda")
        fused = s.eval_ratio(pos, rows, v_out=v)
        ref_v = s.eval(pos, "v", algo="gather")
        t.cuda.synchronize()
        assert t.equal(v, ref_v)
        small = s.eval_ratio(pos[:500], rows[:500])          # below the brick threshold
        t.cuda.synchronize()
        num = (small - fused[:500]).abs()
        den = (rows[:500].abs() * ref_v[:500].abs()).sum(1) + 1e-30
        assert (num / den).max().item() < 1e-5


def test_ratio_clamps_row_indices(spo_lib):
    t = torch()
    c = inputs.uniform_coefs(8, 8, 8, 64, seed=68).astype(np.float32)
    P, R = 2048, 16
    pos = t.from_numpy(inputs.uniform_positions(P, 69)).cuda()
    rows = t.from_numpy((2 * inputs.uniform01(70, R * 64) - 1).astype(np.float32).reshape(R, 64)).cuda()
    idx = np.arange(P, dtype=np.int32) % R
    idx[3], idx[7] = -5, R + 7
    with spo_lib.OrbitalSet(c) as s:
        got = s.eval_ratio(pos, rows, t.from_numpy(idx).cuda())
        clamped = s.eval_ratio(pos, rows, t.from_numpy(np.clip(idx, 0, R - 1)).cuda())
        t.cuda.synchronize()
    assert t.equal(got, clamped)


def test_ratio_rejects_bad_arguments(spo_lib):
    t = torch()
    c = inputs.uniform_coefs(8, 8, 8, 32, seed=71).astype(np.float32)
    with spo_lib.OrbitalSet(c) as s:
        pos = t.zeros((10, 3), device="cuda")
        with pytest.raises(spo_lib.SpoError, match="ld >= N"):
            s.eval_ratio(pos, t.zeros((10, 16), device="cuda"))
        with pytest.raises(spo_lib.SpoError, match="nrows < P"):
            s.eval_ratio(pos, t.zeros((4, 32), device="cuda"))


def test_ratio_nio64_full_batch_sampled(spo_lib, oracle_lib):
    """The benchmark's ratio call: all 98,304 positions of the NiO-64-shaped
    workload against 384 orbitals in one launch (brick path, fused epilogue),
    one random row of A^-1 per position; a seeded sample of 1024 ratios
    against the oracle."""
    t = torch()
    cfg = inputs.NIO64
    c = cfg.make_coefs(np.float32)
    pos = cfg.make_positions()
    P = pos.shape[0]
    rows = (2.0 * inputs.uniform01(65, P * cfg.N) - 1.0).astype(np.float32).reshape(P, cfg.N)
    with spo_lib.OrbitalSet(c) as s:
        got = s.eval_ratio(t.from_numpy(pos).cuda(), t.from_numpy(rows).cuda())
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    sample = np.sort(np.unique((inputs.uniform01(66, 1024) * P).astype(np.int64)))
    check(got.cpu().numpy()[sample], c, pos[sample], rows[sample], None)


def test_ratio_nlpp_quadrature_batch_sampled(spo_lib, oracle_lib):
    """Ratios at the non-local pseudopotential quadrature points of the
    NiO-64-shaped crowd (12 points per electron within r_cut of one of 64
    ions: clustered positions, half of the bricks empty), the points of an
    electron sharing its row of A^-1; a seeded sample against the oracle."""
    t = torch()
    cfg, nl = inputs.NIO64, inputs.NLPP
    c = cfg.make_coefs(np.float32)
    pts, row_of = nl.make_points()
    rows = (2.0 * inputs.uniform01(nl.seed + 2, nl.n_electrons * cfg.N) - 1.0).astype(np.float32)
    rows = rows.reshape(nl.n_electrons, cfg.N)
    with spo_lib.OrbitalSet(c) as s:
        got = s.eval_ratio(t.from_numpy(pts).cuda(), t.from_numpy(rows).cuda(), t.from_numpy(row_of).cuda())
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    sample = np.sort(np.unique((inputs.uniform01(67, 1024) * len(pts)).astype(np.int64)))
    check(got.cpu().numpy()[sample], c, pts[sample], rows, row_of[sample])


def test_ratio_on_column_clusters(spo_lib, oracle_lib):
    """The fused ratio on clustered positions (rows shared through row_of)
    against the oracle; its values equal the gather kernel's."""
    import test_parity_gpu as tp
    t = torch()
    grid, N = (24, 20, 28), 72
    c = inputs.plane_wave_coefs(*grid, N, seed=73).astype(np.float32)
    pos = tp.column_clusters(grid, 500, 1500, 74)
    P, nrows = pos.shape[0], 300
    rows = (2.0 * inputs.uniform01(75, nrows * N) - 1.0).astype(np.float32).reshape(nrows, N)
    row_of = (inputs.uniform01(76, P) * nrows).astype(np.int32)
    with spo_lib.OrbitalSet(c) as s:
        p = t.from_numpy(pos).cuda()
        v = t.empty((P, N), device="cuda")
        got = s.eval_ratio(p, t.from_numpy(rows).cuda(), t.from_numpy(row_of).cuda(), v_out=v)
        ref_v = s.eval(p, "v", algo="gather")
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
        assert t.equal(v, ref_v)
    check(got.cpu().numpy(), c, pos, rows, row_of)
