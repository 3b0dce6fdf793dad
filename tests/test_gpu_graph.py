"""Checks replayed as one CUDA graph (HGRD_GRAPH) against the direct launch
and the oracle: the first check of a binding captures the graph, the later
ones replay it (counter clearing, expansion, sort, scans and the conditional
witness merge all inside the graph; the program in the graph's own device
copy)."""
import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads
from test_gpu_parity import _same

pytestmark = pytest.mark.gpu


def _bind(w):
    return hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)


CASES = {
    "stencil_planted": lambda: workloads.config2(0, planted=True, W=256, H=256, K=8),
    "stencil_clean": lambda: workloads.config2(0, planted=False, W=128, H=128, K=4),
    "shared": lambda: workloads.random_shared(5003),
    "tiny_small_path": lambda: workloads.random_tiny(1003, max_instances=500),
    "warp_barriers": lambda: workloads.warp_exchange(4, 3, "warp", False, grid=8, space="global"),
    "sweep_item": lambda: workloads.config3()[5],
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("flags", [0, hg.NO_JIT | hg.NO_SMALL, hg.JIT])
def test_graph_replays_match_direct_launch(name, flags):
    w = CASES[name]()
    k = _bind(w)
    direct = k.check(cap=1 << 20, flags=flags)
    first = k.check(cap=1 << 20, flags=flags | hg.GRAPH)   # capture
    second = k.check(cap=1 << 20, flags=flags | hg.GRAPH)  # replay
    assert first == direct and second == direct
    _same(second, oracle.check(w.text, w.binding, cap=1 << 20))


def test_graph_survives_other_checks_in_the_same_workspace():
    # the replay reads its own device program and clears its counters itself
    a = _bind(workloads.config2(0, planted=True, W=128, H=128, K=4))
    b = _bind(workloads.random_shared(5011))
    need = max(a.workspace_size(), b.workspace_size())
    import torch
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    ra = a.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH)
    rb = b.check(cap=1 << 20, workspace=buf)
    assert a.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH) == ra
    assert b.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH) == rb
    assert a.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH) == ra


def test_graph_enqueue_keeps_its_program_between_other_checks():
    # enqueued replays read the graph's own device program (copied in once):
    # another binding's checks in the same workspace between them change
    # nothing (collect reports no instance pair; hgrd_check does)
    import torch
    wa = workloads.config2(0, planted=True, W=128, H=128, K=4)
    wb = workloads.random_shared(5011)
    a, b = _bind(wa), _bind(wb)
    buf = torch.empty(max(a.workspace_size(), b.workspace_size()), dtype=torch.uint8, device="cuda")
    oa = oracle.check(wa.text, wa.binding, cap=1 << 20)
    ob = oracle.check(wb.text, wb.binding, cap=1 << 20)
    for _ in range(2):
        a.enqueue(buf, flags=hg.GRAPH)
        _same(a.collect(buf, cap=1 << 20, flags=hg.GRAPH), oa, pair=False)
        b.enqueue(buf)  # direct launches: its program goes into the workspace
        _same(b.collect(buf, cap=1 << 20), ob, pair=False)
        b.enqueue(buf, flags=hg.GRAPH)
        _same(b.collect(buf, cap=1 << 20, flags=hg.GRAPH), ob, pair=False)
        a.enqueue(buf)
        _same(a.collect(buf, cap=1 << 20), oa, pair=False)
    _same(a.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH), oa)
    _same(b.check(cap=1 << 20, workspace=buf, flags=hg.GRAPH), ob)


def test_graph_enqueue_collect_and_rebind():
    w = workloads.config2(0, planted=True, W=128, H=128, K=4)
    k = _bind(w)
    ws = k.workspace()
    for _ in range(3):
        k.enqueue(ws, flags=hg.GRAPH)
    r = k.collect(ws, cap=1 << 20, flags=hg.GRAPH)
    assert r.n_witness == w.meta["expected_witnesses"]
    # a rebind is a new binding: its own graph, its own verdict
    w2 = workloads.config2(0, planted=False, W=128, H=128, K=4)
    k.bind(w2.binding.grid, w2.binding.block, w2.binding.params)
    r2 = k.check(cap=1 << 20, flags=hg.GRAPH)
    assert w2.text == w.text
    _same(r2, oracle.check(w2.text, w2.binding, cap=1 << 20))


def test_graph_with_profile_runs_directly():
    k = _bind(workloads.config2(0, planted=True, W=128, H=128, K=4))
    r = k.check(cap=1 << 20, flags=hg.GRAPH | hg.PROFILE)
    assert len(hg.last_profile()) > 3
    assert r == k.check(cap=1 << 20)
