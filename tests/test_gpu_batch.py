"""Batched check (hgrd_batch_*) against the CPU oracle, item by item.

Corpus kernels of uneven size (config-4 shapes, capped so the oracle stays
fast) and host-loop parameter sweeps (config-3 tuples) run as one batch; every
item's counts, kinds and first canonical witnesses must equal the oracle's.
Both size classes (on-chip items, device-wide items) are covered, as are the
CUDA-graph replay and the autotuner.
"""
import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads

pytestmark = pytest.mark.gpu


def _kernels(ws):
    return [hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params) for w in ws]


def _same_item(r, o, cap):
    assert r.status == 0
    assert r.n_witness == o.n_witness
    assert r.n_by_kind == o.n_by_kind
    assert r.n_keys == o.n_keys and r.n_oob == o.n_oob and r.n_instances == o.n_instances
    assert r.witnesses == o.witnesses[:cap]
    if len(o.witnesses) == o.n_witness:
        pairs = {}
        for w in o.witnesses:
            pairs[(w[3], w[4])] = pairs.get((w[3], w[4]), 0) | w[5]
        assert r.pairs == pairs


def _check_batch(ws, **kw):
    b = hg.Batch(_kernels(ws), **kw)
    res = b.check()
    for w, r in zip(ws, res):
        _same_item(r, oracle.check(w.text, w.binding), b.witness_cap)
    return b, res


def test_corpus_batch_matches_oracle():
    ws = [workloads.config4(i, hi_exp=4.6) for i in range(150)]
    b, res = _check_batch(ws)
    assert any(r.small for r in res) and any(not r.small for r in res)
    assert sum(r.racy for r in res) == sum(1 for w in ws if w.meta["planted"])


def test_sweep_batch_matches_oracle():
    ws = workloads.config3()[:15]
    _check_batch(ws, witness_cap=256)


def test_batch_with_specialised_kernels_matches_oracle():
    # large items on specialised expansion kernels (compiled at creation, one
    # module per program structure), in a replayed CUDA graph
    ws = workloads.config3()[:15] + [workloads.config4(i, hi_exp=4.6) for i in range(150, 190)]
    b, res = _check_batch(ws, witness_cap=256, jit=True, graph=True)
    assert any(not r.small for r in res)
    again = b.check()
    assert [i for i in range(len(ws)) if res[i] != again[i]] == []


def test_all_large_and_all_small_classes():
    ws = [workloads.config4(i, hi_exp=3.6) for i in range(200, 260)] + [workloads.config1(0)]
    _check_batch(ws, small_keys=1)      # everything through the device-wide path
    _check_batch(ws, small_keys=4096)   # everything that fits on chip


def test_graph_replay_and_tuning_keep_results():
    ws = [workloads.config4(i, hi_exp=4.3) for i in range(300, 360)]
    b = hg.Batch(_kernels(ws), graph=True)
    first = b.check()
    second = b.check()
    assert [i for i in range(len(ws)) if first[i] != second[i]] == [], "graph replay changed items"
    choice = b.tune()
    assert choice["streams"] in (2, 4, 8, 16)
    third = b.check()
    assert [i for i in range(len(ws)) if first[i] != third[i]] == [], f"tuned plan {choice} changed items"
    for w, r in zip(ws, first):
        _same_item(r, oracle.check(w.text, w.binding), b.witness_cap)
