"""The workload configurations at their stated sizes, GPU against the oracle
or against closed forms derived by hand.

  * host-loop sweep: all 64 bindings (N = 2^8 .. 2^20, up to 10^8 instances
    each), plain and batched, against the strided kernel's closed form;
  * kernel corpus: 30 kernels spread log-uniformly over 10^3 .. 10^7
    instances, plain and batched, against the oracle;
  * learned-ranker workload: the 2,000 held-out kernels, batched, against the
    oracle verdicts stored in tests/golden/c5_heldout_verdicts.json (written
    by the script beside it, which calls only the oracle).
"""
import json
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import closed_forms as cf
import paper_2604_02106_b300 as hg
import workloads

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _bind(w):
    return hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)


def _pairs(ws):
    out = {}
    for w in ws:
        out[(w[3], w[4])] = out.get((w[3], w[4]), 0) | w[5]
    return out


def test_sweep_all_64_bindings_against_the_closed_form():
    items = workloads.config3()
    assert len(items) == 64 and items[-1].binding.params[0] == 1 << 20
    ks = [_bind(w) for w in items]
    want = []
    for w in items:
        N, S = w.binding.params
        bd, g = w.binding.block[0], w.binding.grid[0]
        b, lo, hi, k = cf.stride_witnesses(N, S, bd)
        wl = list(zip([0] * len(b), [0] * len(b), b.tolist(), lo.tolist(), hi.tolist(), k.tolist()))
        want.append((wl, cf.stride_keys(N, g, bd), g * bd * 8 * 12))
    for w, k, (wl, nkeys, ninst) in zip(items, ks, want):
        r = k.check(cap=max(1, len(wl)), flags=hg.NO_PAIR)
        assert r.witnesses == wl, w.name
        assert r.n_witness == len(wl) and r.n_keys == nkeys and r.n_oob == 0 and r.n_instances == ninst
        assert r.n_by_kind == tuple(sum(1 for x in wl if x[5] >> t & 1) for t in range(3))
        assert r.racy == (w.binding.params[1] < 8) and r.pairs == _pairs(wl)
    res = hg.Batch(ks, witness_cap=256).check()
    for w, r, (wl, nkeys, ninst) in zip(items, res, want):
        assert r.status == 0 and r.n_witness == len(wl) and r.n_keys == nkeys, w.name
        assert r.witnesses == wl[:256] and r.pairs == _pairs(wl)


def _inst(w):
    loops = [int(l.split()[2]) for l in w.text.splitlines() if l.startswith("loop ")]
    nacc = sum(1 for l in w.text.splitlines() if l.startswith("access "))
    return math.prod(w.binding.grid) * math.prod(w.binding.block) * math.prod(loops) * nacc


def corpus_log_spaced(nbins=30, pool=2000):
    """The first corpus item in each of `nbins` equal bins of log10(instances)
    over [3, 7]."""
    picks = {}
    for i in range(pool):
        w = workloads.config4(i)
        b = min(nbins - 1, int((math.log10(_inst(w)) - 3) / 4 * nbins))
        if b >= 0 and b not in picks:
            picks[b] = i
    return [picks[b] for b in sorted(picks)]


def _oracle_item(i):
    import oracle
    w = workloads.config4(i)
    return oracle.check(w.text, w.binding, cap=1 << 22, pair=False)


def test_corpus_across_its_size_range_against_the_oracle():
    items = corpus_log_spaced()
    ws = [workloads.config4(i) for i in items]
    ns = [_inst(w) for w in ws]
    assert len(items) == 30 and min(ns) < 2000 and max(ns) > 5e6
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as p:
        orc = p.map(_oracle_item, items)
    ks = [_bind(w) for w in ws]
    for w, k, o in zip(ws, ks, orc):
        r = k.check(cap=1 << 22, flags=hg.NO_PAIR)
        assert (r.witnesses, r.n_witness, r.n_by_kind, r.n_keys, r.n_oob, r.n_instances) == \
               (o.witnesses, o.n_witness, o.n_by_kind, o.n_keys, o.n_oob, o.n_instances), w.name
        assert r.min_w == o.min_w and r.pairs == _pairs(o.witnesses)
    assert any(o.racy for o in orc) and any(not o.racy for o in orc)
    res = hg.Batch(ks, witness_cap=64).check()
    for w, r, o in zip(ws, res, orc):
        assert r.status == 0 and r.n_witness == o.n_witness and r.n_by_kind == o.n_by_kind, w.name
        assert r.n_keys == o.n_keys and r.n_oob == o.n_oob and r.witnesses == o.witnesses[:64]
        assert r.pairs == _pairs(o.witnesses)


def heldout_verdicts():
    with open(os.path.join(HERE, "golden", "c5_heldout_verdicts.json")) as f:
        return json.load(f)["verdicts"]


def test_ranker_heldout_kernels_against_the_oracle_verdicts():
    rows = heldout_verdicts()
    assert len(rows) == 2000
    ws = [workloads.config4(r["item"], hi_exp=6.0) for r in rows]
    ks = [_bind(w) for w in ws]
    res = hg.Batch(ks, witness_cap=16).check()
    reruns = 0
    for row, k, r in zip(rows, ks, res):
        if r.status == -6:  # more per-run witnesses than the batch keeps: the plain check decides
            r = k.check(cap=16, flags=hg.NO_PAIR)
            reruns += 1
        assert (r.racy, r.n_witness, list(r.n_by_kind), r.n_instances, r.n_keys, r.n_oob) == \
               (row["racy"], row["n_witness"], row["n_by_kind"], row["n_instances"], row["n_keys"],
                row["n_oob"]), row["item"]
        assert {f"{a},{b}": m for (a, b), m in r.pairs.items()} == row["pairs"]
    assert reruns < 100
