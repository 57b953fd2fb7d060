#!/usr/bin/env python
"""Throughput of periodic tricubic B-spline orbital evaluation on GB300.

Metric: orbital VGH evaluations per second (positions x orbitals), with the
evaluation kernel's fraction of the measured HBM bandwidth (roofline on
algorithmic bytes).  One step = one spo_eval_vgh call over the whole batch
(wrap and reduce, basis weights, 64-corner gather, tensor-product reduction
and store, all in one kernel).

Default workload: the NiO-64-shaped orbital set (64^3 grid, N = 384
plane-wave orbitals, FP32 table of 403 MB) at 128 walkers x 768 electron
positions (P = 98,304) - the table and the 1.51 GB of outputs per step are
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own positions against its own
replica of the table (weak scaling, no data-path collective); only the timing
uses a barrier and a max-over-ranks reduction.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1708_02645_gb300 import inputs  # noqa: E402

STORAGE_BYTES = {"f32": 4, "bf16": 2, "f16": 2}
ROWS = {"v": 1, "vgl": 5, "vgh": 10}
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = os.path.join(ROOT, "paper_1708_02645_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


# ---------------------------------------------------------------------------
# accounting
# ---------------------------------------------------------------------------
def algorithmic_bytes(P: int, N: int, storage: str, kind: str) -> int:
    """Bytes one evaluation of P positions must move at minimum per its
    definition with no cache reuse: 64 corner coefficients and the output
    rows per (position, orbital), plus 12 bytes of position per position."""
    return P * N * (64 * STORAGE_BYTES[storage] + 4 * ROWS[kind]) + 12 * P


def compulsory_bytes(P: int, N: int, storage: str, kind: str, table_bytes: int) -> int:
    """The least any implementation must move per launch: the table once,
    the positions and the outputs."""
    return table_bytes + 12 * P + 4 * ROWS[kind] * P * N


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the files the brick kernel is compiled from (its recorded DRAM traffic goes
# stale when any of them changes)
BRICK_SOURCES = ("spo_brick.cu", "spo_brick.cuh", "spo_brick_f32.cu", "spo_brick_bf16.cu", "spo_brick_f16.cu",
                 "spo_device.cuh", "spo_tma.cuh", "spo_internal.h", "spo_batch.h")


def kernel_source_digest() -> str:
    """Digest of the brick kernel's source files."""
    h = hashlib.sha256()
    for name in BRICK_SOURCES:
        with open(os.path.join(KERNEL_SOURCES, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def resolve_algo(name: str, s, P: int, kind: str) -> str:
    """The strategy a call with algo=name takes (the library's answer for
    "auto"), so that the launch count and the timed kernel are known."""
    return s.auto_algo(kind, P) if name == "auto" else name


def recorded_traffic(workload: str, storage: str, kind: str, tuning: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("kernel_source_sha256_16") != kernel_source_digest():
        return None
    for e in rec.get("entries", []):
        if (e.get("workload") == workload and e.get("storage") == storage and e.get("kind") == kind
                and e.get("tuning") == tuning):
            return e.get("dram_bytes_per_launch")
    return None


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; the data path has no collective)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(backend: str):
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend, init_method="env://")
    return dist


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_seed(base: int, rank: int) -> int:
    """Each rank draws its own electron positions (weak scaling)."""
    return base + 7919 * rank


# ---------------------------------------------------------------------------
# GPU clocks during the timed region (NVML through ctypes, read only)
# ---------------------------------------------------------------------------
REASONS = [(0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
           (0x40, "hw_thermal_slowdown"), (0x80, "hw_power_brake_slowdown"),
           (0x2, "applications_clocks_setting"), (0x10, "sync_boost")]


def pci_bus_string(props):
    """NVML bus id ("dddddddd:bb:dd.0") of a CUDA device, or None."""
    try:
        return "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        return None


class ClockSampler:
    def __init__(self, pci_bus_id: str | None, period_s: float = 0.005):
        self.samples = []
        self.max_mhz = None
        self.period = period_s
        self._stop = threading.Event()
        self._thread = None
        self.error = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = ctypes.c_void_p()
            if pci_bus_id is None or nv.nvmlDeviceGetHandleByPciBusId_v2(
                    pci_bus_id.encode(), ctypes.byref(h)) != 0:
                if nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    raise RuntimeError("no NVML device handle")
            self.nv, self.h = nv, h
            m = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = int(m.value)
            self._reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except Exception as e:  # no NVML: report clocks as unavailable
            self.nv = None
            self.error = str(e)

    def _sample(self):
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        p = ctypes.c_uint()
        ok = self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0
        self._reasons_fn(self.h, ctypes.byref(r))
        self.nv.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(p))
        if ok:
            self.samples.append((int(c.value), int(r.value), int(p.value) / 1000.0))

    def _run(self):
        while not self._stop.is_set():
            self._sample()
            time.sleep(self.period)

    def start(self):
        if self.nv is None:
            return
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    def stop(self):
        if self.nv is None:
            return
        self._stop.set()
        self._thread.join()
        self._sample()

    def summary(self):
        if self.nv is None or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [],
                    "note": f"clocks unavailable: {self.error}"}
        mhz = [s[0] for s in self.samples]
        bits = 0
        for s in self.samples:
            bits |= s[1]
        return {"sm_mhz": float(statistics.median(mhz)), "sm_max_mhz": self.max_mhz,
                "reasons": [name for b, name in REASONS if bits & b],
                "samples": len(self.samples),
                "power_w_max": max(s[2] for s in self.samples)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, bounded sample
# ---------------------------------------------------------------------------
def oracle_throughput(coefs64, pos, kind: str, target_s: float):
    """Time the oracle (as it stands) on a sample of the workload's positions
    sized for about target_s seconds of CPU work (the whole batch, repeated,
    when one pass is shorter than that).  Returns (evals/s, positions per
    pass, passes, cores, seconds)."""
    import oracle
    k = {"v": oracle.KIND_V, "vgl": oracle.KIND_VGL, "vgh": oracle.KIND_VGH}[kind]
    N = coefs64.shape[3]
    n0 = min(len(pos), 4096)
    oracle.spo_eval(coefs64, pos[:64].astype(np.float64), k)   # thread pool warm-up
    t0 = time.perf_counter()
    oracle.spo_eval(coefs64, pos[:n0].astype(np.float64), k)
    per_pos = max((time.perf_counter() - t0) / n0, 1e-9)
    n = int(min(len(pos), max(n0, target_s / per_pos)))
    reps = max(1, int(round(target_s / (per_pos * n))))
    sample = pos[:n].astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.spo_eval(coefs64, sample, k)
    dt = time.perf_counter() - t0
    return reps * n * N / dt, n, reps, oracle.num_threads(), dt


def oracle_single_thread(coefs64, pos, kind: str, target_s: float):
    """The oracle on one thread, on a sample sized for about target_s."""
    import oracle
    k = {"v": oracle.KIND_V, "vgl": oracle.KIND_VGL, "vgh": oracle.KIND_VGH}[kind]
    N = coefs64.shape[3]
    n0 = min(len(pos), 256)
    t0 = time.perf_counter()
    oracle.spo_eval(coefs64, pos[:n0].astype(np.float64), k, nthreads=1)
    per_pos = max((time.perf_counter() - t0) / n0, 1e-9)
    n = int(min(len(pos), max(n0, target_s / per_pos)))
    t0 = time.perf_counter()
    oracle.spo_eval(coefs64, pos[:n].astype(np.float64), k, nthreads=1)
    dt = time.perf_counter() - t0
    return n * N / dt, n, dt


PRECISION_SAMPLE = 4096


def cpu_baseline_leg(args, cfg, pos_np, kind: str):
    """The FP64 oracle on the host cores.  Returns the cpu_baseline entry
    (its throughput on a bounded sample, all threads and one thread) and its
    FP64 outputs (VGH and VGL, from the FP64 coefficients) at a seeded sample
    of PRECISION_SAMPLE of the workload's positions: the reference against
    which each storage format's error is reported."""
    import oracle
    P = len(pos_np)
    coefs64 = cfg.make_coefs(np.float64)
    v, n, reps, cores, dt = oracle_throughput(coefs64, pos_np, kind, args.cpu_seconds)
    v1, n1, dt1 = oracle_single_thread(coefs64, pos_np, kind, min(3.0, args.cpu_seconds))
    baseline = {"value": v, "unit": "evals/s", "cores": cores, "kind": "oracle",
                "sample": f"{n} of the {P} positions x {cfg.N} orbitals, "
                          f"{reps} pass(es) ({kind.upper()}, FP64 oracle, "
                          f"{dt:.1f} s on {cores} threads)",
                "single_thread": {"value": v1, "unit": "evals/s",
                                  "sample": f"{n1} positions x {cfg.N} orbitals, "
                                            f"{dt1:.1f} s on 1 thread"}}
    idx = np.sort(np.random.default_rng(cfg.seed + 4096).choice(
        P, size=min(P, PRECISION_SAMPLE), replace=False))
    sp = pos_np[idx].astype(np.float64)
    ref = {"vgh": oracle.spo_eval(coefs64, sp, oracle.KIND_VGH),
           "vgl": oracle.spo_eval(coefs64, sp, oracle.KIND_VGL)}
    return baseline, {"idx": idx, "ref": ref}


def error_vs_reference(sv, pos_sample, ref):
    """Max and RMS relative error per output group (V, G, H from VGH; L from
    VGL) of the set sv at the sampled positions against FP64 values:
    max|d| / max|ref| and ||d|| / ||ref|| over positions x orbitals x
    components.  Every strategy gives the same bits, so these are the rows
    of the full-size launch at those positions."""
    out = {}
    for kd, groups in (("vgh", {"V": (0, 1), "G": (1, 4), "H": (4, 10)}), ("vgl", {"L": (4, 5)})):
        got = sv.eval(pos_sample, kd, algo="auto").cpu().numpy().astype(np.float64)
        r = ref[kd]
        for g, (lo, hi) in groups.items():
            d, rr = got[:, lo:hi] - r[:, lo:hi], r[:, lo:hi]
            out[g] = {"max_rel": float(np.abs(d).max() / np.abs(rr).max()),
                      "rms_rel": float(np.linalg.norm(d) / np.linalg.norm(rr))}
    return out


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def workload_config(name: str):
    cfg = inputs.CONFIGS[name]
    return cfg


def base_config(cfg, storage, kind, P):
    return {"workload": cfg.name, "grid": list(cfg.grid), "orbitals": cfg.N, "positions": P,
            "walkers": cfg.walkers, "electrons_per_walker": cfg.per_walker,
            "storage": storage, "kind": kind, "coefficients": "plane waves (8 per orbital, |k|<=4)",
            "l2": "inputs larger than L2 (table %.0f MB, outputs %.0f MB per step)" % (
                cfg.grid[0] * cfg.grid[1] * cfg.grid[2] * ((cfg.N + 7) // 8 * 8)
                * STORAGE_BYTES[storage] / 1e6, P * cfg.N * ROWS[kind] * 4 / 1e6)}


def measure_e2e(args, s, pos_np, out, kind, evals_per_step, world, dev):
    """Same metric through spo_eval_host: pinned host positions in, pinned
    host outputs back, both copies inside the timed region."""
    import torch
    pos_h = torch.from_numpy(pos_np).pin_memory()
    out_h = torch.empty(tuple(out.shape), dtype=torch.float32).pin_memory()
    for _ in range(max(1, min(args.warmup, 2))):
        s.eval_host(pos_h, kind, out=out_h)
    e2e_steps = max(1, min(args.steps, 10))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.eval_host(pos_h, kind, out=out_h)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, dev)
    e2e = {"value": world * evals_per_step / e2e_s, "unit": "evals/s",
           "h2d_bytes_per_step": int(pos_h.numel() * 4), "d2h_bytes_per_step": int(out_h.numel() * 4),
           "ms_per_step": round(e2e_s * 1e3, 4),
           "api": "spo_eval_host (pinned host buffers: kernels read positions from and write "
                  "outputs to host memory over NVLink-C2C)"}
    return e2e


# 2 x the FMA-pipe operations of the factored z -> y -> x sums per evaluation
# (each sum's first term is a multiply, which the FMA pipe takes like an FMA)
FLOPS_PER_EVAL = {"v": 168, "vgl": 600, "vgh": 656}
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(num_sms: int):
    """FP32 FMA peak: SMs x 128 lanes x 2 flop x the maximum SM clock (the
    clock measured under load on this machine, MEASURED_PEAKS.json)."""
    mhz, src = 2070.0, "nominal max SM clock"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        pass
    return num_sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, \
        f"{num_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:.0f} MHz ({src})"


def smem_peak_gbs(num_sms: int):
    """Shared-memory bandwidth: SMs x 32 banks x 4 bytes per clock x the
    maximum SM clock (MEASURED_PEAKS.json)."""
    mhz, src = 2070.0, "nominal max SM clock"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        pass
    return num_sms * 128 * mhz * 1e6 / 1e9, f"{num_sms} SMs x 32 banks x 4 B x {mhz:.0f} MHz ({src})"


def brick_smem_bytes(P: int, N: int, storage: str, tile: int) -> int:
    """Shared-memory bytes the brick kernel's window sums read per launch:
    64 staged coefficients per (position, orbital of every tile, the last
    one padded to the tile)."""
    return P * (-(-N // tile) * tile) * 64 * STORAGE_BYTES[storage]


def configure(s, args):
    s.set_param("brick_vec", args.brick_vec)
    s.set_param("brick_tile", args.brick_tile)
    s.set_param("brick_schedule", args.brick_schedule)


def time_steps(s, pos, out, kind, algo, steps, warmup):
    """ms per full evaluation (binning included), CUDA events on the stream."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        s.eval(pos, kind, out=out, algo=algo)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s.eval(pos, kind, out=out, algo=algo)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def time_kernel(s, pos, out, kind, algo, steps):
    """ms per launch of the evaluation kernel alone (binned strategies: bin
    once, then time only the evaluation launches)."""
    import torch
    if algo == "gather":
        return time_steps(s, pos, out, kind, algo, steps, 1)
    stream = torch.cuda.current_stream()
    s.bin(pos)
    s.eval_binned(pos, kind, out=out, algo=algo)
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(steps):
        s.eval_binned(pos, kind, out=out, algo=algo)
    k1.record(stream)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / steps


def max_rel_diff(a, b, kind):
    """max |a - b| / max |b| per output group (GPU tensors)."""
    groups = {"v": {"V": (0, 1)}, "vgl": {"V": (0, 1), "G": (1, 4), "L": (4, 5)},
              "vgh": {"V": (0, 1), "G": (1, 4), "H": (4, 10)}}[kind]
    if a.dim() == 2:
        a, b = a[:, None, :], b[:, None, :]
    return {g: float((a[:, lo:hi] - b[:, lo:hi]).abs().max()
                     / b[:, lo:hi].abs().max().clamp_min(1e-30))
            for g, (lo, hi) in groups.items()}


def run_ours(args):
    import torch
    from paper_1708_02645_gb300 import spo

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist_init("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    cfg = workload_config(args.workload)
    kind, storage = args.kind, args.storage
    coefs32 = cfg.make_coefs(np.float32)
    P = args.positions if args.positions > 0 else cfg.P
    pos_np = inputs.uniform_positions(P, shard_seed(cfg.seed + 1000, rank))
    pos = torch.from_numpy(pos_np).to(dev)
    rows = ROWS[kind]
    out = torch.empty((P, rows, cfg.N) if rows > 1 else (P, cfg.N), dtype=torch.float32, device=dev)
    s = spo.OrbitalSet(coefs32, storage=storage)
    configure(s, args)
    stream = torch.cuda.current_stream()

    algo = resolve_algo(args.algo, s, P, kind)
    for _ in range(args.warmup):
        s.eval(pos, kind, out=out, algo=algo)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(pci_bus_string(props))
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        s.eval(pos, kind, out=out, algo=algo)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, dev)
    ms_per_step = ms_max / args.steps
    evals_per_step = P * cfg.N
    value = world * evals_per_step / (ms_per_step * 1e-3)

    # roofline of the dominant kernel (its own launches, events on its stream)
    kernel_ms = time_kernel(s, pos, out, kind, algo, args.steps)
    kernel_name = ("spo_brick_pipe_kernel" if args.brick_schedule == 1 else "spo_brick_kernel") \
        if algo == "brick" else ("spo_gather_kernel" if algo == "gather"
                                 else "spo_gather_kernel (binned order)")
    flops = FLOPS_PER_EVAL[kind] * evals_per_step
    tf_peak, tf_src = fp32_peak_tflops(props.multi_processor_count)
    achieved_tf = flops / (kernel_ms * 1e-3) / 1e12
    alg = algorithmic_bytes(P, cfg.N, storage, kind)
    achieved_gbs = alg / (kernel_ms * 1e-3) / 1e9
    hbm_peak, hbm_src = measured_hbm_peak()
    comp = compulsory_bytes(P, cfg.N, storage, kind, s.footprint())
    tuning = f"{algo}/t{args.brick_tile}/v{args.brick_vec}/s{args.brick_schedule}"
    roofline = {
        "bound": "alu", "achieved": round(achieved_tf, 3), "peak": round(tf_peak, 2),
        "unit": "TFLOP/s", "frac": round(achieved_tf / tf_peak, 4),
        "peak_source": tf_src + "; FP32 FMA issue is what limits this kernel (ncu)",
        "flop_note": "2 per FMA-pipe operation of the factored sums (a sum's first term is a multiply, "
                     "which occupies the FMA pipe as an FMA): frac is the share of FMA-pipe slots "
                     "doing algorithmic work",
        "traffic": recorded_traffic(cfg.name, storage, kind, tuning),
        "kernel": f"{kernel_name}<{storage},{kind}>", "kernel_ms": round(kernel_ms, 5),
        "flops_per_launch": flops, "flops_per_eval": FLOPS_PER_EVAL[kind],
        "hbm": {"achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved_gbs / hbm_peak, 4),
                "peak_source": hbm_src + " (hbm_gbs, burst copy)",
                "algorithmic_bytes_per_launch": alg,
                "note": "algorithmic bytes (64 corner coefficients + outputs per eval); the "
                        "staged blocks are read from DRAM about 1.6 times per launch, so the "
                        "DRAM traffic is far below them",
                "compulsory_bytes_per_launch": comp,
                "compulsory_achieved": round(comp / (kernel_ms * 1e-3) / 1e9, 1),
                "compulsory_frac": round(comp / (kernel_ms * 1e-3) / 1e9 / hbm_peak, 4)},
    }
    if algo == "brick" and args.brick_schedule == 0:
        tile = args.brick_tile if s.info()["Np"] >= 64 else 32
        sb = brick_smem_bytes(P, cfg.N, storage, tile)
        sp, ssrc = smem_peak_gbs(props.multi_processor_count)
        roofline["smem"] = {"achieved": round(sb / (kernel_ms * 1e-3) / 1e9, 1), "peak": round(sp, 1),
                            "unit": "GB/s", "frac": round(sb / (kernel_ms * 1e-3) / 1e9 / sp, 4),
                            "peak_source": ssrc, "bytes_per_launch": sb,
                            "note": "coefficient reads of the window sums from the staged blocks "
                                    "(64 per evaluation); the bound of the V kernel, where each "
                                    "read feeds one FMA"}
    assert spo.device_status() == 0, "a bounded device-side wait gave up"

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None if args.no_e2e else measure_e2e(args, s, pos_np, out, kind, evals_per_step, world, dev)

    result = {
        "metric": "orbital VGH evals/s (positions x orbitals)" if kind == "vgh"
        else f"orbital {kind.upper()} evals/s (positions x orbitals)",
        "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16 storage, f32 accumulate",
                  "f16": "f16 storage, f32 accumulate"}[storage],
        "data": "synthetic (seeded plane-wave orbitals, uniform positions)",
        "config": dict(base_config(cfg, storage, kind, P), algo=algo, brick_vec=args.brick_vec,
                       brick_tile=args.brick_tile, brick_schedule=args.brick_schedule),
        "roofline": roofline, "e2e": e2e,
        # binning (count with its scan, scatter, weight records) and the evaluation
        "gpu_launches": args.steps * (1 if algo == "gather" else 4),
        "clocks": sampler.summary(),
    }
    if world > 1:
        result["config"]["parallelism"] = f"replicas x{world} (positions sharded per rank)"

    oracle_sample = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"], oracle_sample = cpu_baseline_leg(args, cfg, pos_np, kind)

    if rank == 0 and world == 1 and not args.no_variants:
        result["variants"] = measure_variants(args, cfg, coefs32, s, pos, out, kind, storage, algo,
                                              oracle_sample)
    s.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


VARIANTS = ("all", "storage", "ratio", "nlpp", "autotune", "crowd", "surrogate", "surrogate_specified",
            "surrogate_inference", "prefilter", "nio32")


def measure_variants(args, cfg, coefs32, s32, pos, out32, kind, storage, algo, oracle_sample=None):
    """Reduced-precision storage on the same positions (throughput, table
    bytes, the error of every storage format against the FP64 oracle on the
    FP64 coefficients at a seeded sample of the positions, and the
    difference from the FP32-storage outputs), and the NiO-32-shaped set
    (V, VGL, VGH)."""
    import torch
    from paper_1708_02645_gb300 import spo
    res = {}
    steps = max(5, min(args.steps, 50))
    chosen = set(args.variants.split(","))

    def want(name):
        return "all" in chosen or name in chosen

    if storage == "f32" and want("storage"):
        ref = out32.clone()
        psample = None
        if oracle_sample is not None:
            psample = pos[torch.from_numpy(oracle_sample["idx"]).to(pos.device)]
            res["precision_sample"] = (f"{len(oracle_sample['idx'])} positions drawn without "
                                       f"replacement (seed {cfg.seed + 4096}) from the {pos.shape[0]}; "
                                       "reference: the FP64 oracle on the FP64 coefficients")
            res["f32_error_vs_oracle"] = error_vs_reference(s32, psample, oracle_sample["ref"])
        for st in ("bf16", "f16"):
            with spo.OrbitalSet(coefs32, storage=st) as sv:
                configure(sv, args)
                o = torch.empty_like(out32)
                step_ms = time_steps(sv, pos, o, kind, algo, steps, 3)
                k_ms = time_kernel(sv, pos, o, kind, algo, steps)
                sv.eval(pos, kind, out=o, algo=algo)
                torch.cuda.synchronize()
                res[st] = {"value": pos.shape[0] * cfg.N / (step_ms * 1e-3), "unit": "evals/s",
                           "ms_per_step": round(step_ms, 5), "kernel_ms": round(k_ms, 5),
                           "table_bytes": sv.footprint(),
                           "max_rel_diff_vs_f32_storage": max_rel_diff(o, ref, kind)}
                if psample is not None:
                    res[st]["error_vs_oracle"] = error_vs_reference(sv, psample, oracle_sample["ref"])
        res["f32_table_bytes"] = s32.footprint()
    if want("ratio"):
        res["ratio_fused_v"] = measure_ratio(cfg, s32, pos, steps)
    if want("nlpp") and cfg.name == inputs.NIO64.name:
        res["nlpp_ratio"] = measure_nlpp(cfg, s32, pos.device, steps)
    if want("autotune"):
        res["autotune"] = s32.autotune(kind, pos.shape[0])
        configure(s32, args)   # back to the command line's tuning
    if want("crowd"):
        res["crowd"] = measure_crowd(args, kind, steps)
    if cfg.N == 384 and (want("surrogate") or "surrogate_specified" in chosen):
        res["surrogate"] = measure_surrogate(cfg, s32, pos, steps, coarse_run=want("surrogate"))
    if cfg.N == 384 and "surrogate_inference" in chosen:
        res["surrogate_inference"] = measure_surrogate_inference(cfg, pos, steps)
    if want("prefilter"):
        res["prefilter"] = measure_prefilter(cfg)
    if want("nio32"):
        n32 = inputs.NIO32
        c = n32.make_coefs(np.float32)
        p32 = torch.from_numpy(n32.make_positions()).to(pos.device)
        with spo.OrbitalSet(c, storage="f32") as sv:
            configure(sv, args)
            for kd in ("v", "vgl", "vgh"):
                o = torch.empty(sv.out_shape(n32.P, kd), dtype=torch.float32, device=pos.device)
                a = resolve_algo(args.algo, sv, n32.P, kd)
                # a step is about 0.06 ms, launched from Python: the median of
                # three runs of 200 keeps a host stall from entering the number
                step_ms = float(np.median([time_steps(sv, p32, o, kd, a, 200, 3) for _ in range(3)]))
                res[f"{n32.name}_{kd}"] = {"value": n32.P * n32.N / (step_ms * 1e-3), "unit": "evals/s",
                                           "ms_per_step": round(step_ms, 5), "algo": a}
    return res


def measure_ratio(cfg, s32, pos, steps):
    """Fused value + determinant ratio: one row of A^-1 per position."""
    import torch
    P = pos.shape[0]
    rows = (2.0 * torch.rand((P, cfg.N), device=pos.device, dtype=torch.float32,
                             generator=torch.Generator(device=pos.device).manual_seed(7)) - 1.0)
    ratio = torch.empty((P,), device=pos.device)
    for _ in range(3):
        s32.eval_ratio(pos, rows, ratio=ratio)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        s32.eval_ratio(pos, rows, ratio=ratio)
    e1.record()
    torch.cuda.synchronize()
    r_ms = e0.elapsed_time(e1) / steps
    return {"value": P * cfg.N / (r_ms * 1e-3), "unit": "evals/s",
            "ratios_per_s": P / (r_ms * 1e-3), "ms_per_step": round(r_ms, 5),
            "what": "spo_eval_ratio: V of all orbitals dotted with an A^-1 row per position, "
                    "values not stored"}


def measure_nlpp(cfg, s32, dev, steps):
    """Determinant ratios at the non-local pseudopotential quadrature points
    of 128 walkers x 768 electrons (12 points per electron within r_cut of an
    ion, 64 ions), one A^-1 row per electron shared by its points."""
    import torch
    nl = inputs.NLPP
    pts, row_of = nl.make_points()
    Q = pts.shape[0]
    rows = (2.0 * inputs.uniform01(nl.seed + 2, nl.n_electrons * cfg.N) - 1.0).astype(np.float32)
    rows = torch.from_numpy(rows.reshape(nl.n_electrons, cfg.N)).to(dev)
    q = torch.from_numpy(pts).to(dev)
    ro = torch.from_numpy(row_of).to(dev)
    ratio = torch.empty((Q,), device=dev)
    for _ in range(3):
        s32.eval_ratio(q, rows, ro, ratio=ratio)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        s32.eval_ratio(q, rows, ro, ratio=ratio)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g = np.asarray(cfg.grid)
    cells = np.minimum((pts.astype(np.float64) * g).astype(np.int64), g - 1) // 4
    nb = -(-g // 4)
    occupied = len(np.unique((cells[:, 0] * nb[1] + cells[:, 1]) * nb[2] + cells[:, 2]))
    return {"workload": nl.name, "points": Q, "electrons_near_ions": Q // 12,
            "bricks_occupied": f"{occupied} of {int(nb.prod())}",
            "value": Q * cfg.N / (ms * 1e-3), "unit": "evals/s", "ratios_per_s": Q / (ms * 1e-3),
            "ms_per_step": round(ms, 5),
            "what": "spo_eval_ratio at the 12-point quadrature points, row_of = electron"}


def measure_prefilter(cfg):
    """spo_prefilter on the workload's samples in FP64 ([nx, ny, nz, N]):
    interpolating coefficients, three recursive passes in place."""
    import torch
    from paper_1708_02645_gb300 import spo
    d = torch.from_numpy(cfg.make_coefs(np.float64)).cuda()
    work = d.clone()
    for _ in range(2):
        work.copy_(d)
        spo.prefilter(work)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps, ms = 3, 0.0
    for _ in range(reps):
        work.copy_(d)
        e0.record()
        spo.prefilter(work)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    ms /= reps
    nbytes = d.numel() * 8
    return {"ms": round(ms, 4), "table_bytes_f64": nbytes,
            "gbs_per_pass": round(2 * nbytes / (ms / 3 * 1e-3) / 1e9, 1),
            "what": "FP64 samples [64,64,64,384] -> interpolating B-spline coefficients "
                    "(3 axis passes, each reading and writing the table at least once)"}


def time_surrogate_inference(sg, pos, N, steps):
    """CUDA-event time of the fused tensor-core inference (VGL and V) of
    surrogate sg at positions pos, after 3 untimed calls."""
    import torch
    P = pos.shape[0]
    res = {}
    out = torch.empty((P, 5, N), dtype=torch.float32, device=pos.device)
    outv = torch.empty((P, N), dtype=torch.float32, device=pos.device)
    for kd, o in (("vgl", out), ("v", outv)):
        for _ in range(3):
            sg.eval(pos, out=o, kind=kd, precision=1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            sg.eval(pos, out=o, kind=kd, precision=1)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[f"inference_{kd}"] = {"value": P * N / (ms * 1e-3), "unit": "evals/s",
                                  "ms_per_step": round(ms, 5),
                                  "kernels": "encode_image_kernel + surrogate_fused_kernel "
                                             "(tcgen05, BF16 x BF16 -> FP32)"}
    return res


def surrogate_spec(N, r_min=2, r_max=64):
    """The specified surrogate: 16 levels x 2^19 x 2 FP16 hashed grid,
    32-128-128-128-N BF16 perceptron."""
    from types import SimpleNamespace
    return SimpleNamespace(levels=16, log2_table=19, features=2, r_min=r_min, r_max=r_max, hidden=128,
                           layers=3, N=N)


def measure_surrogate_inference(cfg, pos, steps):
    """Inference time of the specified surrogate, untrained (its weights'
    values do not change the work): the short command the inference kernel
    is profiled with."""
    from paper_1708_02645_gb300 import spo
    spec = surrogate_spec(cfg.N)
    with spo.Surrogate(spec, seed=20170808) as sg:
        res = {"spec": vars(spec), "weights": "initial (untrained)"}
        res.update(time_surrogate_inference(sg, pos, cfg.N, steps))
    return res


def surrogate_run(spec, teacher, pos, steps, lr, train_steps, batch, warm, grid_lr_mult=10.0,
                  channel_scale=(1.0, 1.0, 1.0, 1.0, 1.0), seed=20170808):
    """Train one surrogate on spline VGL samples with the variance-normalised
    V, G, L loss (channel weights channel_scale_c / mean(target_c^2) over
    16,384 uniform teacher samples), Adam with a linear warm-up over `warm` steps and a
    cosine decay of the learning rate to 0 (stepped every 16 steps), then
    time its fused tensor-core inference (VGL and V) and measure its error
    against the spline and its footprint."""
    import math
    import time
    import torch
    from paper_1708_02645_gb300 import spo
    P = pos.shape[0]
    N = spec.N
    res = {"spec": vars(spec), "batch": batch, "grid_lr_mult": grid_lr_mult,
           "schedule": {"peak_lr": lr, "steps": train_steps, "warmup_steps": warm,
                        "decay": "cosine to 0, the rate stepped every 16 steps"}}
    sp = torch.from_numpy(inputs.uniform_positions(16384, 20170810)).to(pos.device)
    t = teacher.eval(sp, "vgl").double()
    cw = [float(channel_scale[c] / (t[:, c] ** 2).mean()) for c in range(5)]
    res["channel_weights"] = cw
    chunk = 16
    with spo.Surrogate(spec, seed=seed) as sg:
        sg.set_optimizer(0.9, 0.99, 1e-15, grid_lr_mult)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = None
        for k in range(0, train_steps, chunk):
            f = (k + chunk / 2) / train_steps
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * f))
            if k < warm:
                cur *= (k + chunk) / warm
            loss = sg.train(teacher, steps=min(chunk, train_steps - k), batch=batch, lr=cur,
                            channel_weights=cw, seed=20170809 + k)
        torch.cuda.synchronize()
        res["train_samples"] = train_steps * batch
        res["train_s"] = round(time.perf_counter() - t0, 3)
        res["final_loss"] = loss
        res.update(time_surrogate_inference(sg, pos, N, steps))
        out = torch.empty((P, 5, N), dtype=torch.float32, device=pos.device)
        sg.eval(pos, out=out, kind="vgl", precision=1)
        want = torch.empty_like(out)
        teacher.eval(pos, "vgl", out=want)
        torch.cuda.synchronize()
        err = {}
        for c, name in enumerate(("V", "Gx", "Gy", "Gz", "L")):
            d = (out[:, c] - want[:, c]).double()
            w = want[:, c].double()
            err[name] = {"rms_rel": float(torch.sqrt((d * d).mean() / (w * w).mean())),
                         "max_rel": float(d.abs().max() / w.abs().max())}
        res["error_vs_spline"] = err
        res["footprint_bytes"] = sg.footprint()
        res["spline_table_bytes"] = teacher.footprint()
        res["footprint_ratio"] = round(teacher.footprint() / sg.footprint(), 2)
        # Eckart-Young: no linear read-out of `hidden` features (+ the bias)
        # can beat the truncated SVD of the sampled values
        vals = want[:8192, 0].double().cpu().numpy()
        sv = np.linalg.svd(vals, compute_uv=False)
        k = spec.hidden + 1
        res["rank_floor_rms_rel_V"] = float(np.sqrt((sv[k:] ** 2).sum() / (sv ** 2).sum()))
    return res


# Loss weight of each channel (V, Gx, Gy, Gz, L) relative to 1 / mean(target^2):
# the value enters every determinant ratio, the derivatives only the drift
# and the local energy, so it counts twice.
SURROGATE_CHANNEL_SCALE = (2.0, 1.0, 1.0, 1.0, 1.0)


def measure_surrogate(cfg, teacher, pos, steps, coarse_run=True):
    """Learned surrogates of the 384-orbital set, both with the specified
    capacity (16 levels x 2^19 x 2 FP16 hashed grid, 32-128-128-128-384 BF16
    perceptron) and 2^22 training samples: level resolutions 2..64 (the
    finest at the spline's own 64^3 grid; the reading this network is
    reported on) and, for comparison, 16..512 (the hashed-grid default,
    whose finest levels keep the Laplacian term from training)."""
    res = {"loss": "sum over V, Gx, Gy, Gz, L of w_c mean squared error, w_c = s_c / mean(target_c^2), "
                   "s = (2, 1, 1, 1, 1): the value counted twice",
           "rank_floor_what": "relative RMS error of the best rank-(hidden + 1) approximation of "
                              "the [8192 positions x N] matrix of spline values: a lower bound for "
                              "any output layer reading the hidden units"}
    spec = surrogate_spec(cfg.N)
    res["specified"] = surrogate_run(spec, teacher, pos, steps, 1.5e-2, 8192, 512, 128,
                                     channel_scale=SURROGATE_CHANNEL_SCALE)
    if not coarse_run:
        return res
    fine = surrogate_spec(cfg.N, 16, 512)
    res["resolutions_16_512"] = surrogate_run(fine, teacher, pos, steps, 1.5e-2, 8192, 512, 128,
                                              channel_scale=SURROGATE_CHANNEL_SCALE)
    return res


def measure_crowd(args, kind, steps):
    """Batched crowds: 3 orbital sets (32^3/64, 48^3/192, 64^3/384, FP32),
    512 walkers with U{64..768} electrons, walker w on set w mod 3; one graph
    replay per step (binning + one brick-kernel launch over all sets)."""
    import torch
    from paper_1708_02645_gb300 import spo
    cr = inputs.CROWD
    dev = torch.device("cuda", torch.cuda.current_device())
    sets = [spo.OrbitalSet(cr.make_coefs(k, np.float32)) for k in range(len(cr.sets))]
    sizes = cr.sizes()
    which = cr.set_of_walker()
    items, evals = [], 0
    for w in range(cr.walkers):
        k = int(which[w])
        p = torch.from_numpy(cr.make_positions(w, int(sizes[w]))).to(dev)
        o = torch.empty(sets[k].out_shape(p.shape[0], kind), dtype=torch.float32, device=dev)
        items.append((k, p, o))
        evals += p.shape[0] * sets[k].N
    total = int(sizes.sum())
    out = {"workload": cr.name, "walkers": cr.walkers, "positions": total,
           "sets": [list(x) for x in cr.sets], "evals_per_step": evals}
    stream = torch.cuda.current_stream()

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    with spo.Batch(sets, total, cr.walkers) as b:
        b.graph(items, kind)
        g_ms = timed(b.launch, steps)
        e_ms = timed(lambda: b.eval(items, kind), steps)
    w_ms = timed(lambda: [sets[k].eval(p, kind, out=o) for k, p, o in items], max(1, steps // 10))
    out.update({"value": evals / (g_ms * 1e-3), "unit": "evals/s",
                "graph_ms_per_step": round(g_ms, 5), "batch_eval_ms_per_step": round(e_ms, 5),
                "per_walker_calls_ms_per_step": round(w_ms, 5),
                "gpu_launches_per_step": "1 graph (item_of, count, scan, scatter, records, brick kernel "
                                         "+ 1 memset)"})
    for st in sets:
        st.close()
    return out


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is a bounded
    sample of the same workload; same metric and unit as our arm."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cfg = workload_config(args.workload)
    kind = args.kind
    coefs64 = cfg.make_coefs(np.float64)
    pos = inputs.uniform_positions(cfg.P, cfg.seed + 1000).astype(np.float64)
    k = {"v": oracle.KIND_V, "vgl": oracle.KIND_VGL, "vgh": oracle.KIND_VGH}[kind]
    # size one step for ~ 150 s / (steps + warmup) of oracle time
    t0 = time.perf_counter()
    oracle.spo_eval(coefs64, pos[:64], k)
    per_pos = (time.perf_counter() - t0) / 64
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(max(16, min(cfg.P, budget / max(per_pos, 1e-9))))
    for w in range(args.warmup):
        oracle.spo_eval(coefs64, pos[:n], k)
    times = []
    for st in range(args.steps):
        lo = (st * n) % max(1, cfg.P - n)
        t0 = time.perf_counter()
        oracle.spo_eval(coefs64, pos[lo:lo + n], k)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * n * cfg.N / total
    cores = oracle.num_threads()
    sample = f"{n} of the {cfg.P} positions x {cfg.N} orbitals per step ({kind.upper()}, FP64)"
    result = {
        "impl": "reference", "metric": "orbital VGH evals/s (positions x orbitals)" if kind == "vgh"
        else f"orbital {kind.upper()} evals/s (positions x orbitals)",
        "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded plane-wave orbitals, uniform positions)",
        "config": base_config(cfg, "f32", kind, cfg.P),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(result), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(inputs.CONFIGS), default=inputs.NIO64.name)
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--kind", choices=["v", "vgl", "vgh"], default="vgh")
    ap.add_argument("--algo", choices=["auto", "gather", "sorted_gather", "brick"], default="auto")
    ap.add_argument("--brick-vec", type=int, choices=[2, 4], default=4)
    ap.add_argument("--brick-tile", type=int, choices=[32, 64], default=32)
    ap.add_argument("--brick-schedule", type=int, choices=[0, 1], default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the BF16/FP16 and NiO-32-shaped sub-results")
    ap.add_argument("--variants", default="all",
                    help="comma list of the sub-results to measure: storage, ratio, autotune, crowd, "
                         "surrogate (both networks), surrogate_specified (the specified network "
                         "only), surrogate_inference (the specified network untrained, inference "
                         "timing only; not part of all), prefilter, nio32 (default all)")
    ap.add_argument("--positions", type=int, default=0,
                    help="evaluate this many positions instead of the workload's (profiling)")
    args = ap.parse_args(argv)
    unknown = set(args.variants.split(",")) - set(VARIANTS)
    if unknown:
        ap.error(f"unknown --variants {sorted(unknown)}; choose from {VARIANTS}")
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
