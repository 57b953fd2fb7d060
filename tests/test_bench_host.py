"""Host logic of bench.py: byte accounting, traffic records, and the
multi-rank timing reduction (world size 2, gloo, CPU processes)."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_algorithmic_bytes_per_eval():
    # 64 coefficients + output rows per (position, orbital), 12 B per position
    assert bench.algorithmic_bytes(1, 1, "f32", "vgh") == 64 * 4 + 40 + 12
    assert bench.algorithmic_bytes(1, 1, "bf16", "vgh") == 64 * 2 + 40 + 12
    assert bench.algorithmic_bytes(1, 1, "f16", "vgl") == 64 * 2 + 20 + 12
    assert bench.algorithmic_bytes(1, 1, "f32", "v") == 64 * 4 + 4 + 12
    assert bench.algorithmic_bytes(98304, 384, "f32", "vgh") == 98304 * 384 * 296 + 12 * 98304


def test_traffic_record_is_dropped_when_kernel_changes(tmp_path, monkeypatch):
    rec = {"kernel_source_sha256_16": bench.kernel_source_digest(),
           "entries": [{"workload": "w", "storage": "f32", "kind": "vgh", "tuning": "brick/t32/v4/s0",
                        "dram_bytes_per_launch": 123}]}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.recorded_traffic("w", "f32", "vgh", "brick/t32/v4/s0") == 123
    assert bench.recorded_traffic("w", "bf16", "vgh", "brick/t32/v4/s0") is None
    assert bench.recorded_traffic("w", "f32", "vgh", "gather/t32/v4/s0") is None
    rec["kernel_source_sha256_16"] = "0" * 16
    path.write_text(json.dumps(rec))
    assert bench.recorded_traffic("w", "f32", "vgh", "brick/t32/v4/s0") is None


def test_brick_smem_bytes_count_padded_tiles():
    # 64 staged coefficients per (position, orbital), the last tile padded
    assert bench.brick_smem_bytes(1, 32, "f32", 32) == 32 * 64 * 4
    assert bench.brick_smem_bytes(1, 33, "f32", 32) == 64 * 64 * 4
    assert bench.brick_smem_bytes(2, 40, "bf16", 64) == 2 * 64 * 64 * 2
    assert bench.brick_smem_bytes(98304, 384, "f32", 32) == 98304 * 384 * 256


def test_smem_peak_is_derived_from_bank_count_and_clock():
    gbs, src = bench.smem_peak_gbs(152)
    assert abs(gbs - 152 * 128 * 2070e6 / 1e9) < 1e-6 or "MEASURED" in src
    assert "banks" in src


def test_fp32_peak_is_derived_from_unit_counts_and_clock():
    tf, src = bench.fp32_peak_tflops(152)
    assert abs(tf - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-6 or "MEASURED" in src
    assert "SMs" in src


def test_shard_seeds_differ_per_rank():
    seeds = {bench.shard_seed(100, r) for r in range(8)}
    assert len(seeds) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, _ = bench.dist_env()
    bench.dist_init("gloo")
    bench.barrier(w)
    # each rank "measured" a different time; every rank must see the max
    m = bench.max_over_ranks(10.0 + 5.0 * r, w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, m))


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 15.0, 1: 15.0}


def test_reference_arm_rank_nonzero_exits_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert capsys.readouterr().out == ""


@pytest.mark.slow
def test_reference_arm_prints_one_line(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    bench.main(["--impl", "reference", "--steps", "2", "--warmup", "3",
                "--workload", "uniform16_n16"])
    line = capsys.readouterr().out.strip()
    d = json.loads(line)
    assert d["impl"] == "reference" and d["unit"] == "evals/s" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_compulsory_bytes_are_table_positions_and_outputs():
    assert bench.compulsory_bytes(10, 3, "f32", "vgh", 1000) == 1000 + 12 * 10 + 4 * 10 * 10 * 3
    assert bench.compulsory_bytes(10, 3, "bf16", "v", 500) == 500 + 12 * 10 + 4 * 1 * 10 * 3


def test_hbm_peak_is_measured_else_fallback(monkeypatch, tmp_path):
    gbs, src = bench.measured_hbm_peak()
    assert gbs > 0 and src in ("measured", "fallback")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))   # no MEASURED_PEAKS.json there
    assert bench.measured_hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    assert bench.measured_hbm_peak() == (1234.5, "measured")


def test_oracle_timing_is_bounded_and_counts_evaluations():
    import numpy as np
    from paper_1708_02645_gb300 import inputs
    c = inputs.uniform_coefs(8, 8, 8, 16, seed=3)
    pos = inputs.uniform_positions(300, 4)
    rate, n, reps, cores, dt = bench.oracle_throughput(c, pos, "vgh", 0.05)
    assert 0 < n <= len(pos) and reps >= 1 and cores >= 1 and dt > 0
    assert abs(rate - reps * n * 16 / dt) <= 1e-6 * rate
    rate1, n1, dt1 = bench.oracle_single_thread(c, pos, "v", 0.05)
    assert rate1 > 0 and 0 < n1 <= len(pos) and dt1 > 0


def test_workload_config_names_the_bench_shapes():
    from paper_1708_02645_gb300 import inputs
    cfg = bench.workload_config(inputs.NIO64.name)
    assert cfg.grid == (64, 64, 64) and cfg.N == 384 and cfg.P == 98304
    c = bench.base_config(cfg, "f32", "vgh", cfg.P)
    assert c["workload"] == "nio64_64cubed_n384" and c["positions"] == 98304 and c["orbitals"] == 384


def test_variant_names_and_surrogate_recipe():
    """--variants accepts the surrogate-inference timing and refuses unknown
    names; the specified surrogate is 16 levels x 2^19 x 2, resolutions
    2..64, 3 x 128 hidden units, with the value channel's loss weight
    doubled."""
    import pytest
    assert "surrogate_inference" in bench.VARIANTS and "all" in bench.VARIANTS
    with pytest.raises(SystemExit):
        bench.main(["--variants", "no_such_variant"])
    spec = bench.surrogate_spec(384)
    assert (spec.levels, spec.log2_table, spec.features, spec.r_min, spec.r_max, spec.hidden, spec.layers,
            spec.N) == (16, 19, 2, 2, 64, 128, 3, 384)
    assert bench.surrogate_spec(384, 16, 512).r_max == 512
    assert tuple(bench.SURROGATE_CHANNEL_SCALE) == (2.0, 1.0, 1.0, 1.0, 1.0)
