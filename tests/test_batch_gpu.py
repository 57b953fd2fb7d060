"""Batched crowds (spo_batch_*): many walkers with uneven electron counts
against several orbital sets in one binning and one launch, and the same
work recorded into a CUDA graph.  Every walker's outputs must equal an
spo_eval of that walker alone (bit for bit: one FMA order everywhere), and a
sample is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1708_02645_gb300 import inputs
from parity import assert_kernel_parity

pytestmark = pytest.mark.gpu

SETS = ((12, 64), (16, 96), (20, 130))   # (grid edge, N)


def torch():
    import torch as t
    return t


def make_crowd(spo, nwalk=40, seed=81, lo=0, hi=300):
    t = torch()
    sets, coefs = [], []
    for k, (n, N) in enumerate(SETS):
        c = inputs.plane_wave_coefs(n, n, n, N, seed=seed + k).astype(np.float32)
        coefs.append(c)
        sets.append(spo.OrbitalSet(c))
    counts = inputs.walker_sizes(nwalk, lo, hi, seed + 10)
    walkers = []
    for w in range(nwalk):
        pos = t.from_numpy(inputs.wide_positions(int(counts[w]), seed + 100 + w)).cuda()
        walkers.append((w % len(SETS), pos))
    return sets, coefs, walkers


def outputs_for(sets, walkers, kind):
    t = torch()
    return [t.full(sets[k].out_shape(p.shape[0], kind), float("nan"), device="cuda")
            for k, p in walkers]


@pytest.mark.parametrize("kind", ["vgh", "vgl", "v"])
def test_batch_equals_single_set_evaluations(spo_lib, oracle_lib, kind):
    t = torch()
    sets, coefs, walkers = make_crowd(spo_lib)
    outs = outputs_for(sets, walkers, kind)
    total = sum(p.shape[0] for _, p in walkers)
    with spo_lib.Batch(sets, total, len(walkers)) as b:
        b.eval([(k, p, o) for (k, p), o in zip(walkers, outs)], kind)
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    for (k, p), o in zip(walkers, outs):
        if p.shape[0] == 0:
            continue
        ref = sets[k].eval(p, kind)
        t.cuda.synchronize()
        assert t.equal(o, ref)
    # a sample of walkers against the oracle
    kk = {"v": 0, "vgl": 1, "vgh": 2}[kind]
    for w in (1, 2, 3):
        k, p = walkers[w]
        pn = p.cpu().numpy().astype(np.float64)
        vals = coefs[k].astype(np.float64)
        assert_kernel_parity(outs[w].cpu().numpy(), oracle.spo_eval(vals, pn, kk),
                             oracle.condition(vals, pn, kk), kk, f"walker {w}")
    for s in sets:
        s.close()


def test_batch_graph_replays_new_positions(spo_lib):
    """Record once; change the positions in place; each replay evaluates the
    current positions (as a DMC step would)."""
    t = torch()
    sets, _, walkers = make_crowd(spo_lib, nwalk=25, seed=91, lo=50, hi=400)
    outs = outputs_for(sets, walkers, "vgh")
    total = sum(p.shape[0] for _, p in walkers)
    with spo_lib.Batch(sets, total, len(walkers)) as b:
        b.graph([(k, p, o) for (k, p), o in zip(walkers, outs)], "vgh")
        for step in range(2):
            for w, (k, p) in enumerate(walkers):
                p.copy_(t.from_numpy(inputs.wide_positions(p.shape[0], 1000 * step + w)))
            b.launch()
            t.cuda.synchronize()
            for (k, p), o in zip(walkers, outs):
                assert t.equal(o, sets[k].eval(p, "vgh"))
    for s in sets:
        s.close()


def test_batch_rejects_bad_plans_and_items(spo_lib):
    t = torch()
    sets, _, walkers = make_crowd(spo_lib, nwalk=4)
    small = spo_lib.OrbitalSet(inputs.uniform_coefs(8, 8, 8, 13, seed=1).astype(np.float32))
    with pytest.raises(spo_lib.SpoError, match="SPO_EUNSUPPORTED"):
        spo_lib.Batch([small], 100, 4)
    with spo_lib.Batch(sets, 10, 4) as b:
        pos = t.zeros((11, 3), device="cuda")
        out = t.empty(sets[0].out_shape(11, "v"), device="cuda")
        with pytest.raises(spo_lib.SpoError, match="exceed"):
            b.eval([(0, pos, out)], "v")
        with pytest.raises(spo_lib.SpoError, match="set 7 invalid"):
            b.eval([(7, pos[:2], out)], "v")
        with pytest.raises(spo_lib.SpoError, match="no graph"):
            b.launch()
    for s in sets + [small]:
        s.close()


@pytest.mark.parametrize("small_set", [False, True])
def test_one_call_eval_batch(spo_lib, small_set):
    """spo_eval_batch equals per-walker evaluations bit for bit, through a
    temporary plan (sets the plan takes) and through per-walker calls (a set
    with fewer than 32 padded orbitals, which the plan cannot take)."""
    t = torch()
    sets, coefs, walkers = make_crowd(spo_lib, nwalk=17, seed=91)
    if small_set:
        c = inputs.plane_wave_coefs(9, 10, 11, 13, seed=95).astype(np.float32)
        sets.append(spo_lib.OrbitalSet(c))
        walkers = [(w % 4, p) for w, (_, p) in enumerate(walkers)]
    outs = outputs_for(sets, walkers, "vgh")
    spo_lib.eval_batch(sets, [(k, p, o) for (k, p), o in zip(walkers, outs)], "vgh")
    t.cuda.synchronize()
    assert spo_lib.device_status() == 0
    for (k, p), o in zip(walkers, outs):
        if p.shape[0] == 0:
            continue
        assert t.equal(o, sets[k].eval(p, "vgh"))


def test_crowd_full_size_graph(spo_lib, oracle_lib):
    """The benchmark's crowd in its launch form: 3 sets (32^3 x 64, 48^3 x
    192, 64^3 x 384 orbitals), 512 walkers of 64..768 electrons, VGH through
    one recorded graph.  Every walker equals its own spo_eval bit for bit, and
    a seeded sample of positions of 6 walkers matches the FP64 oracle."""
    t = torch()
    cr = inputs.CROWD
    coefs = [cr.make_coefs(k, np.float32) for k in range(len(cr.sets))]
    sets = [spo_lib.OrbitalSet(c) for c in coefs]
    sizes, which = cr.sizes(), cr.set_of_walker()
    items = []
    for w in range(cr.walkers):
        k = int(which[w])
        p = t.from_numpy(cr.make_positions(w, int(sizes[w]))).cuda()
        o = t.full(sets[k].out_shape(p.shape[0], "vgh"), float("nan"), device="cuda")
        items.append((k, p, o))
    with spo_lib.Batch(sets, int(sizes.sum()), cr.walkers) as b:
        b.graph(items, "vgh")
        b.launch()
        t.cuda.synchronize()
        assert spo_lib.device_status() == 0
    for k, p, o in items:
        assert t.equal(o, sets[k].eval(p, "vgh"))
    for w in (0, 1, 2, 257, 258, 511):
        k, p, o = items[w]
        idx = np.sort(np.unique((inputs.uniform01(500 + w, 48) * p.shape[0]).astype(np.int64)))
        pn = p.cpu().numpy().astype(np.float64)[idx]
        vals = coefs[k].astype(np.float64)
        assert_kernel_parity(o.cpu().numpy()[idx], oracle.spo_eval(vals, pn, 2),
                             oracle.condition(vals, pn, 2), 2, f"crowd walker {w}")
    for s in sets:
        s.close()
