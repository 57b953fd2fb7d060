"""GPU (libspo, sm_103a) vs FP64 oracle, element by element, through the C ABI.

Inputs come from the seeded recipes in paper_1708_02645_gb300.inputs; every
expected value comes from the oracle.  Kernel parity runs the oracle on the
coefficients exactly as the table stores them; the storage-format error runs
it on the original FP64 coefficients.  Tolerances are in tests/parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1708_02645_gb300 import inputs
from parity import (assert_format_error, assert_kernel_parity, errors, stored_values)

pytestmark = pytest.mark.gpu

KINDS = {"v": 0, "vgl": 1, "vgh": 2}


def torch():
    import torch as t
    return t


ALGOS = ["gather", "sorted_gather", "brick", "brick4", "brick_t32", "brick4_t32", "pipe",
         "pipe_t32"]


def gpu_eval(spo, coefs_upload, pos, kind, storage, src_dtype=None, out=None, algos=("auto",)):
    """Outputs of every requested strategy; all must be bit-identical."""
    t = torch()
    res = {}
    with spo.OrbitalSet(coefs_upload, storage=storage, src_dtype=src_dtype) as s:
        p = t.from_numpy(np.ascontiguousarray(pos, dtype=np.float32)).cuda()
        for a in algos:
            s.set_param("brick_vec", 4 if a.startswith("brick4") else 2)
            s.set_param("brick_tile", 32 if a.endswith("_t32") else 64)
            s.set_param("brick_schedule", 1 if a.startswith("pipe") else 0)
            brick = a.startswith("brick") or a.startswith("pipe")
            if brick and s.info()["Np"] < 32:
                continue
            o = s.eval(p, kind, out=out, algo="brick" if brick else a)
            t.cuda.synchronize()
            res[a] = o.cpu().numpy()
        assert spo.device_status() == 0
    first = next(iter(res.values()))
    for a, o in res.items():
        assert np.array_equal(o, first, equal_nan=True), f"strategy {a} differs from {next(iter(res))}"
    return first


def check_case(spo, coefs64, pos, kind, storage, sample=None, what="", algos=("auto",)):
    """Kernel parity (and the format error for reduced precision)."""
    k = KINDS[kind]
    vals, upload, sd = stored_values(coefs64, storage)
    got = gpu_eval(spo, upload, pos, kind, storage, sd, algos=algos)
    idx = np.arange(len(pos)) if sample is None else sample
    pos64 = np.asarray(pos, dtype=np.float64)[idx]
    ref = oracle.spo_eval(vals, pos64, k)
    beta = oracle.condition(vals, pos64, k)
    err = assert_kernel_parity(got[idx], ref, beta, k, what)
    if storage != "f32":
        ref64 = oracle.spo_eval(coefs64, pos64, k)
        beta64 = oracle.condition(coefs64, pos64, k)
        wsum = oracle.condition(np.ones(coefs64.shape[:3] + (1,)), pos64, k)
        wsum = np.broadcast_to(wsum, ref64.shape)
        assert_format_error(got[idx], ref64, beta64, wsum, k, storage, what)
    return err


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
def test_uniform16_vgh(spo_lib, oracle_lib):
    cfg = inputs.UNIFORM16
    c = cfg.make_coefs()
    check_case(spo_lib, c, cfg.make_positions(), "vgh", "f32", what=cfg.name,
               algos=("auto", "gather", "sorted_gather"))


@pytest.mark.parametrize("kind", ["vgl", "vgh", "v"])
def test_nio32_full(spo_lib, oracle_lib, kind):
    cfg = inputs.NIO32
    c = cfg.make_coefs()
    check_case(spo_lib, c, cfg.make_positions(), kind, "f32", what=f"{cfg.name} {kind}",
               algos=["auto"] + ALGOS)


@pytest.fixture(scope="module")
def nio64():
    cfg = inputs.NIO64
    return cfg, cfg.make_coefs(), cfg.make_positions()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_nio64_full_batch_sampled(spo_lib, oracle_lib, nio64, storage):
    """All 98,304 positions in one launch (the benchmark's launch); the oracle
    checks a seeded sample of 2048 of them element by element."""
    cfg, c, pos = nio64
    sample = np.sort(np.unique((inputs.uniform01(99, 2048) * len(pos)).astype(np.int64)))
    check_case(spo_lib, c, pos, "vgh", storage, sample=sample, what=f"{cfg.name} {storage}",
               algos=["auto"] + ALGOS)


@pytest.mark.parametrize("kind", ["v", "vgl"])
def test_nio64_full_batch_sampled_other_kinds(spo_lib, oracle_lib, nio64, kind):
    """V and VGL of all 98,304 positions in one launch (FP32), every strategy
    bit for bit; the oracle checks a seeded sample of 2048 positions."""
    cfg, c, pos = nio64
    sample = np.sort(np.unique((inputs.uniform01(98, 2048) * len(pos)).astype(np.int64)))
    check_case(spo_lib, c, pos, kind, "f32", sample=sample, what=f"{cfg.name} {kind}",
               algos=["auto", "gather", "sorted_gather", "brick4_t32"])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("grid,N", [((4, 4, 4), 1), ((5, 9, 7), 13), ((4, 6, 5), 7),
                                    ((8, 8, 8), 33), ((7, 4, 11), 4), ((6, 6, 6), 1024),
                                    ((9, 10, 11), 100), ((4, 5, 6), 65), ((13, 6, 9), 64),
                                    ((12, 10, 20), 40)])
@pytest.mark.parametrize("kind", ["v", "vgl", "vgh"])
def test_ragged_shapes(spo_lib, oracle_lib, grid, N, kind):
    """Grids that are not multiples of the brick edge (partial bricks at the
    far faces), N that is not a multiple of the tile (partial last tile, odd
    N: scalar stores), every strategy."""
    c = inputs.uniform_coefs(*grid, N, seed=grid[0] * 100 + N)
    pos = np.concatenate([inputs.uniform_positions(1301, 5), inputs.wide_positions(1200, 6)])
    check_case(spo_lib, c, pos, kind, "f32", what=f"{grid} N={N} {kind}", algos=["auto"] + ALGOS)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("N", [21, 130])
def test_ragged_reduced_precision(spo_lib, oracle_lib, storage, N):
    c = inputs.plane_wave_coefs(9, 10, 11, N, seed=3)
    pos = inputs.wide_positions(2057, 8)
    check_case(spo_lib, c, pos, "vgh", storage, what=f"ragged {storage}", algos=["auto"] + ALGOS)


@pytest.mark.parametrize("kind", ["v", "vgh"])
def test_f16_special_values(spo_lib, oracle_lib, kind):
    """FP16 tables holding zeros of both signs, subnormals, the smallest and
    largest normals and values that round into the subnormal range, mixed
    with ordinary ones: every strategy widens each stored half exactly."""
    rng = np.random.default_rng(23)
    special = np.array([0.0, -0.0, 2.0 ** -24, -(2.0 ** -24), 3 * 2.0 ** -24, 2.0 ** -15,
                        2.0 ** -14, -(2.0 ** -14), 2.0 ** -14 - 2.0 ** -24, 65504.0, -65504.0,
                        1e-5, -3e-6, 0.75, -1.5])
    grid, N = (8, 9, 10), 40
    c = rng.choice(special, size=grid + (N,))
    ordinary = rng.uniform(-2.0, 2.0, size=c.shape)
    c = np.where(rng.uniform(size=c.shape) < 0.5, c, ordinary)
    pos = np.concatenate([inputs.uniform_positions(3001, 21), inputs.wide_positions(500, 22)])
    check_case(spo_lib, c, pos, kind, "f16", what=f"f16 special values {kind}",
               algos=["auto"] + ALGOS)


def test_degenerate_position_clouds(spo_lib, oracle_lib):
    """All positions in one cell (one brick holds every position), all at one
    point, and a single position: every strategy."""
    c = inputs.plane_wave_coefs(16, 12, 20, 96, seed=17)
    rng = np.random.default_rng(3)
    one_cell = (np.array([5, 7, 9]) + rng.uniform(0, 1, size=(3000, 3))) / np.array([16, 12, 20])
    same = np.tile(np.array([[0.3, 0.6, 0.9]]), (1500, 1))
    for pos, what in ((one_cell, "one cell"), (same, "one point"), (same[:1], "one position")):
        check_case(spo_lib, c, pos.astype(np.float32), "vgh", "f32", what=what,
                   algos=["auto"] + ALGOS)


def column_clusters(grid, nclusters, nuniform, seed):
    """Positions in clusters along z columns of cells: per cluster, members
    in the cluster's cell (twice), 1, 2 and 3 cells above it and 1 below
    (each at its own fraction within the cell): many positions share a
    cell or a column of one brick; plus uniform positions.  FP32."""
    n = np.array(grid, dtype=np.float64)
    u = inputs.uniform01(seed, 3 * nclusters).reshape(nclusters, 3)
    base = np.floor(u * n)
    dz = np.array([0, 0, 1, 2, 3, -1], dtype=np.float64)
    f = inputs.uniform01(seed + 1, nclusters * len(dz) * 3).reshape(nclusters, len(dz), 3)
    cells = np.repeat(base[:, None, :], len(dz), axis=1)
    cells[:, :, 2] += dz
    pos = ((cells + f) / n).reshape(-1, 3)
    return np.concatenate([pos, inputs.uniform_positions(nuniform, seed + 2).astype(np.float64)]).astype(np.float32)


@pytest.mark.parametrize("grid,N,storage", [((24, 20, 28), 40, "f32"), ((16, 16, 32), 96, "f32"),
                                            ((24, 20, 28), 40, "bf16")])
def test_values_on_column_clusters(spo_lib, oracle_lib, grid, N, storage):
    """Clustered positions (an odd number of bricks along z in the first
    grid, a ragged last orbital tile for N = 40): every strategy bit for bit
    and the oracle element by element."""
    pos = column_clusters(grid, 500, 1500, 71)
    c = inputs.plane_wave_coefs(*grid, N, seed=72)
    check_case(spo_lib, c, pos, "v", storage, algos=ALGOS, what=f"clusters {grid} N={N}")


def test_binning_reused_for_several_kinds(spo_lib):
    """spo_bin once, then V, VGL and VGH from the same binning (the ratio and
    derivative evaluations of one move) equal the one-call results."""
    t = torch()
    c = inputs.plane_wave_coefs(20, 20, 20, 128, seed=19).astype(np.float32)
    pos = t.from_numpy(inputs.uniform_positions(20000, 20)).cuda()
    with spo_lib.OrbitalSet(c) as s:
        s.bin(pos)
        staged = {k: s.eval_binned(pos, k, algo=a) for k, a in
                  (("v", "brick"), ("vgl", "sorted_gather"), ("vgh", "brick"))}
        direct = {k: s.eval(pos, k, algo="gather") for k in staged}
        t.cuda.synchronize()
        for k in staged:
            assert t.equal(staged[k], direct[k]), k
        other = t.from_numpy(inputs.uniform_positions(20000, 21)).cuda()
        with pytest.raises(spo_lib.SpoError, match="differ from the last spo_bin"):
            s.eval_binned(other, "vgh")


def test_special_positions(spo_lib, oracle_lib):
    """Grid nodes, cell faces, 1.0, negative and large coordinates."""
    grid = (8, 12, 10)
    c = inputs.uniform_coefs(*grid, 72, seed=12)
    g = np.array(grid, dtype=np.float64)
    nodes = np.array([[0, 0, 0], [7, 11, 9], [3, 6, 5], [8, 12, 10]]) / g
    pts = np.concatenate([nodes, [[1.0, 1.0, 1.0], [-1.0, -0.5, 2.0], [0.99999994, 0.0, 0.5],
                                  [-1e-7, 1e-7, -0.99999994], [123.25, -77.5, 1000.125]],
                          nodes - 1e-7, nodes + 1e-7]).astype(np.float32)
    check_case(spo_lib, c, pts, "vgh", "f32", what="special positions", algos=["auto"] + ALGOS)


@pytest.mark.parametrize("algo", ["auto", "gather", "sorted_gather", "brick"])
def test_nonfinite_positions_do_not_fault(spo_lib, oracle_lib, algo):
    """NaN/Inf give unspecified values for that position only."""
    t = torch()
    c = inputs.uniform_coefs(6, 6, 6, 64, seed=1)
    pos = inputs.uniform_positions(2048, 2)
    bad = pos.copy()
    bad[5] = [np.nan, 0.5, 0.5]
    bad[9] = [np.inf, -np.inf, 0.25]
    bad[17] = [3e38, -3e38, np.nan]
    with spo_lib.OrbitalSet(c.astype(np.float32)) as s:
        o = s.eval(t.from_numpy(bad).cuda(), "vgh", algo=algo)
        t.cuda.synchronize()
        got = o.cpu().numpy()
        assert spo_lib.device_status() == 0
    good = np.setdiff1d(np.arange(len(pos)), [5, 9, 17])
    vals = c.astype(np.float32).astype(np.float64)
    ref = oracle.spo_eval(vals, pos[good].astype(np.float64), 2)
    beta = oracle.condition(vals, pos[good].astype(np.float64), 2)
    assert_kernel_parity(got[good], ref, beta, 2, "finite neighbours of NaN positions")


def test_empty_batch(spo_lib):
    t = torch()
    c = inputs.uniform_coefs(4, 4, 4, 3, seed=1).astype(np.float32)
    with spo_lib.OrbitalSet(c) as s:
        o = s.eval(t.empty((0, 3), device="cuda"), "vgh")
        assert o.shape == (0, 10, 3)
        h = s.eval_host(np.empty((0, 3), np.float32), "vgl")
        assert h.shape == (0, 5, 3)


@pytest.mark.parametrize("algo", ["gather", "brick"])
def test_misaligned_output_uses_scalar_stores(spo_lib, oracle_lib, algo):
    t = torch()
    c = inputs.uniform_coefs(5, 6, 7, 64, seed=4)
    pos = inputs.uniform_positions(1100, 3)
    with spo_lib.OrbitalSet(c.astype(np.float32)) as s:
        big = t.full((1100 * 10 * 64 + 1,), float("nan"), device="cuda")
        view = big[1:]   # 4-byte aligned, not 8- or 16-byte aligned
        s.eval(t.from_numpy(pos).cuda(), "vgh", out=view, algo=algo)
        t.cuda.synchronize()
        got = view.cpu().numpy().reshape(1100, 10, 64)
        assert np.isnan(big[0].item())
    vals = c.astype(np.float32).astype(np.float64)
    ref = oracle.spo_eval(vals, pos, 2)
    assert_kernel_parity(got, ref, oracle.condition(vals, pos, 2), 2, "misaligned out")


def test_table_beyond_2_31_elements(spo_lib):
    """A 128^3 x 1024 FP32 table (2^31 coefficients, 8.6 GB): element offsets
    beyond int32.  Coefficients c[m][j] = (j mod 5) + m_x + 2 m_y + 3 m_z are
    linear in m, so by polynomial reproduction (pinned in the oracle tests)
    V = (j mod 5) + u_x + 2 u_y + 3 u_z, G = (n_x, 2 n_y, 3 n_z), H = 0 in
    cells whose window does not wrap.  Addressing errors would break this."""
    t = torch()
    n, N = 128, 1024
    ar = t.arange(n, device="cuda", dtype=t.float32)
    coefs = (ar[:, None, None, None] + 2 * ar[None, :, None, None] + 3 * ar[None, None, :, None]
             + (t.arange(N, device="cuda") % 5).float()[None, None, None, :])
    coef_max = coefs.abs().max().item()
    P = 2048
    u = 0.999 * inputs.uniform01(81, 3 * P).reshape(P, 3)   # stay inside the cell
    cells = 1 + np.floor(inputs.uniform01(82, 3 * P).reshape(P, 3) * (n - 3))
    pos = ((cells + u) / n).astype(np.float32)
    with spo_lib.OrbitalSet(coefs) as s:
        del coefs
        t.cuda.empty_cache()
        got = s.eval_vgh(t.from_numpy(pos).cuda()).cpu().numpy().astype(np.float64)
    uu = pos.astype(np.float64) * n
    v = (np.arange(N) % 5)[None, :] + (uu[:, 0] + 2 * uu[:, 1] + 3 * uu[:, 2])[:, None]
    # FP32 rounding bound 64 * 2^-24 * beta with beta <= max|c| * sum|W|, and
    # sum|W| <= 1 (V), n (G), 4 n^2 (H); an addressing error shifts V by >= 1
    # and G by >= n
    unit = 64 * 2.0 ** -24 * float(coef_max)
    assert np.abs(got[:, 0] - v).max() <= unit
    for d, g in enumerate((n, 2 * n, 3 * n)):
        assert np.abs(got[:, 1 + d] - g).max() <= unit * n
    assert np.abs(got[:, 4:]).max() <= unit * 4 * n * n


# ---------------------------------------------------------------------------
# consistency between entry points
# ---------------------------------------------------------------------------
def test_kinds_consistent(spo_lib):
    t = torch()
    c = inputs.plane_wave_coefs(12, 12, 12, 40, seed=9).astype(np.float32)
    pos = t.from_numpy(inputs.wide_positions(500, 10)).cuda()
    with spo_lib.OrbitalSet(c) as s:
        v, g, h = s.eval_v(pos), s.eval_vgl(pos), s.eval_vgh(pos)
        t.cuda.synchronize()
    v, g, h = v.cpu().numpy(), g.cpu().numpy(), h.cpu().numpy()
    # identical z/y/x stages for the value: bitwise equal
    assert np.array_equal(v, h[:, 0]) and np.array_equal(g[:, :4], h[:, :4])
    lap = h[:, 4].astype(np.float64) + h[:, 7] + h[:, 9]
    assert np.abs(g[:, 4] - lap).max() <= 1e-5 * np.abs(lap).max()


def test_host_path_matches_device_path(spo_lib):
    """spo_eval_host gives the device path's bits: pinned buffers (zero-copy:
    kernels read and write host memory), pageable buffers (chunked copies on
    two streams, ragged last chunk), and pinned positions with a pageable
    output (chunked)."""
    t = torch()
    c = inputs.plane_wave_coefs(8, 8, 8, 384, seed=11).astype(np.float32)
    pos = inputs.wide_positions(10001, 12)   # > 2 chunks of 4369 VGH positions
    with spo_lib.OrbitalSet(c) as s:
        dev = s.eval(t.from_numpy(pos).cuda(), "vgh").cpu().numpy()
        pinned = t.empty((10001, 10, 384), dtype=t.float32).pin_memory()
        host = s.eval_host(t.from_numpy(pos).pin_memory(), "vgh", out=pinned).numpy()
        pageable = s.eval_host(pos, "vgh")
        mixed = s.eval_host(t.from_numpy(pos).pin_memory(), "vgh")
    assert np.array_equal(dev, host) and np.array_equal(dev, pageable)
    assert np.array_equal(dev, mixed)


def test_deterministic(spo_lib):
    t = torch()
    c = inputs.plane_wave_coefs(16, 16, 16, 64, seed=13).astype(np.float32)
    pos = t.from_numpy(inputs.uniform_positions(3000, 14)).cuda()
    with spo_lib.OrbitalSet(c) as s:
        a = s.eval_vgh(pos).cpu().numpy()
        b = s.eval_vgh(pos).cpu().numpy()
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# upload and conversion
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_library_conversion_rounds_once_to_nearest_even(spo_lib, storage):
    """F64 coefficients converted by the library give the same outputs, bit
    for bit, as coefficients rounded on the host with one RNE step."""
    t = torch()
    c = inputs.plane_wave_coefs(8, 9, 10, 24, seed=15)
    _, upload, sd = stored_values(c, storage)
    pos = t.from_numpy(inputs.uniform_positions(700, 16)).cuda()
    with spo_lib.OrbitalSet(c, storage=storage) as a, \
            spo_lib.OrbitalSet(upload, storage=storage, src_dtype=sd) as b, \
            spo_lib.OrbitalSet(t.from_numpy(c).cuda(), storage=storage) as d:
        oa, ob, od = a.eval_vgh(pos), b.eval_vgh(pos), d.eval_vgh(pos)
        t.cuda.synchronize()
        assert t.equal(oa, ob) and t.equal(oa, od)
        assert a.info()["Np"] == 24
        assert a.footprint() == 11 * 12 * 13 * 24 * (4 if storage == "f32" else 2)


def test_tuning_parameters(spo_lib):
    c = inputs.uniform_coefs(4, 4, 4, 64, seed=1).astype(np.float32)
    with spo_lib.OrbitalSet(c) as s:
        assert s.get_param("brick_vec") == 4
        s.set_param("brick_vec", 2)
        assert s.get_param("brick_vec") == 2
        with pytest.raises(spo_lib.SpoError, match="must be 2 or 4"):
            s.set_param("brick_vec", 3)
        assert s.get_param("brick_tile") == 32
        s.set_param("brick_tile", 64)
        assert s.get_param("brick_tile") == 64
        with pytest.raises(spo_lib.SpoError, match="must be 32 or 64"):
            s.set_param("brick_tile", 48)


def test_footprint_and_padding(spo_lib):
    c = inputs.uniform_coefs(4, 5, 6, 13, seed=1).astype(np.float32)
    with spo_lib.OrbitalSet(c, storage="bf16") as s:
        info = s.info()
        assert info["grid"] == (4, 5, 6) and info["N"] == 13 and info["Np"] == 16
        assert s.footprint() == 7 * 8 * 9 * 16 * 2   # 3 ghost nodes per axis
        with pytest.raises(spo_lib.SpoError, match="SPO_EUNSUPPORTED"):
            s.eval(torch().zeros((2048, 3), device="cuda"), "vgh", algo="brick")


def test_errors_are_reported_not_launched(spo_lib):
    t = torch()
    c = inputs.uniform_coefs(4, 4, 4, 4, seed=1).astype(np.float32)
    with spo_lib.OrbitalSet(c) as s:
        host_pos = t.zeros((4, 3))
        out = t.empty((4, 10, 4), device="cuda")
        import ctypes
        lib = spo_lib.load()
        st = lib.spo_eval(s.handle, 2, ctypes.c_void_p(host_pos.data_ptr()), 4,
                          ctypes.c_void_p(out.data_ptr()), None)
        assert st == 1 and b"device memory" in lib.spo_last_error()
        st = lib.spo_eval(s.handle, 2, ctypes.c_void_p(out.data_ptr()), -1,
                          ctypes.c_void_p(out.data_ptr()), None)
        assert st == 1
        st = lib.spo_eval(s.handle, 2, ctypes.c_void_p(out.data_ptr()), 1 << 40,
                          ctypes.c_void_p(out.data_ptr()), None)
        assert st == 1 and b"too large" in lib.spo_last_error()
        with pytest.raises(spo_lib.SpoError):
            spo_lib.OrbitalSet(c, storage="f64")
        # the context is still healthy
        o = s.eval_vgh(t.from_numpy(inputs.uniform_positions(8, 1)).cuda())
        t.cuda.synchronize()
        assert t.isfinite(o).all()


def test_nio32_errors_reported(spo_lib, oracle_lib):
    """max and RMS relative error per output group, FP32 storage (reported)."""
    cfg = inputs.NIO32
    c = cfg.make_coefs()
    pos = cfg.make_positions()[:2048]
    got = gpu_eval(spo_lib, c.astype(np.float32), pos, "vgl", "f32")
    ref = oracle.spo_eval(c, pos.astype(np.float64), 1)
    e = errors(got, ref, 1)
    assert all(v["max_rel"] < 1e-5 for v in e.values()), e


def test_autotune_picks_a_strategy_and_keeps_outputs(spo_lib, tmp_path, monkeypatch):
    """spo_autotune times the strategies, applies the fastest (outputs stay
    bit-identical), caches the result in the process and in SPO_TUNE_CACHE."""
    t = torch()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SPO_TUNE_CACHE", str(cache))
    c = inputs.plane_wave_coefs(20, 18, 22, 72, seed=27).astype(np.float32)
    pos = t.from_numpy(inputs.uniform_positions(6000, 28)).cuda()
    with spo_lib.OrbitalSet(c) as s:
        before = s.eval(pos, "vgl", algo="gather")
        best = s.autotune("vgl", 6000)
        assert best["algo"] in ("gather", "sorted_gather", "brick") and best["ms"] > 0
        assert not best["from_cache"]
        after = s.eval(pos, "vgl")                     # AUTO now follows the tuning
        t.cuda.synchronize()
        assert t.equal(before, after)
        again = s.autotune("vgl", 7000)                # same power-of-two bucket
        assert again["from_cache"] and again["algo"] == best["algo"]
    assert cache.exists() and "kind=1" in cache.read_text()


@pytest.mark.parametrize("kind", ["vgh", "v"])
def test_reserved_evaluation_replays_in_a_cuda_graph(spo_lib, kind):
    """After spo_reserve on a stream, an evaluation on that stream (binning
    and brick kernel) can be captured in a CUDA graph; each replay evaluates
    the positions the buffer holds then, bit for bit as a direct call."""
    import torch as t
    c = inputs.plane_wave_coefs(16, 12, 20, 64, seed=19).astype(np.float32)
    P = 6000
    with spo_lib.OrbitalSet(c) as s:
        stream = t.cuda.Stream()
        pos = t.from_numpy(inputs.uniform_positions(P, 31)).cuda()
        out = t.empty(s.out_shape(P, kind), device="cuda")
        s.reserve(P, stream=stream)
        t.cuda.synchronize()
        g = t.cuda.CUDAGraph()
        with t.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
            s.eval(pos, kind, out=out, algo="brick")
        for step in range(2):
            pos.copy_(t.from_numpy(inputs.uniform_positions(P, 40 + step)))
            g.replay()
            t.cuda.synchronize()
            assert spo_lib.device_status() == 0
            assert t.equal(out, s.eval(pos, kind, algo="brick"))


def test_auto_strategy_follows_positions_per_brick(spo_lib):
    """spo_auto_algo: gather below 1.5 positions per brick (or P < 1024),
    the brick kernel from 5 (VGH), 7 (VGL) or 8 (V) per brick, the gather in
    binned order between; sets with fewer than 32 padded orbitals never take
    the brick kernel."""
    c = inputs.uniform_coefs(64, 64, 64, 40, seed=5).astype(np.float32)   # 16^3 = 4096 bricks
    with spo_lib.OrbitalSet(c) as s:
        expect = [(1000, "vgh", "gather"), (4096, "v", "gather"), (8192, "vgh", "sorted_gather"),
                  (16384, "vgh", "sorted_gather"), (20480, "vgh", "brick"), (24576, "vgl", "sorted_gather"),
                  (28672, "vgl", "brick"), (28672, "v", "sorted_gather"), (32768, "v", "brick"),
                  (98304, "v", "brick")]
        for P, kind, algo in expect:
            assert s.auto_algo(kind, P) == algo, (P, kind)
        with pytest.raises(Exception):
            s.auto_algo("vgh", -1)
    small = inputs.uniform_coefs(64, 64, 64, 8, seed=6).astype(np.float32)
    with spo_lib.OrbitalSet(small) as s:
        assert s.auto_algo("vgh", 98304) == "sorted_gather"

