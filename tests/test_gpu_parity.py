"""GPU path (through the C ABI) against the CPU oracle, bit for bit.

Every case compares the canonical witness list, the per-kind counts, the
instance / key / out-of-bounds counts, the minimal witness and the canonical
instance pair.  Sizes run from tiny launches to the full 64x64x(16x16)
stencil the bench times, where the oracle checks a sample of the address
space and closed forms check the rest.
"""
import math

import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads
from workloads import Binding

pytestmark = pytest.mark.gpu


def _same(g, o, pair=True):
    assert g.witnesses == o.witnesses
    assert g.n_witness == o.n_witness
    assert g.n_by_kind == o.n_by_kind
    assert g.n_instances == o.n_instances
    assert g.n_keys == o.n_keys
    assert g.n_oob == o.n_oob
    assert g.racy == o.racy
    assert g.min_w == o.min_w
    if pair and o.racy:
        assert g.min_x == o.min_x and g.min_y == o.min_y
    if g.pairs is not None and not g.truncated and len(o.witnesses) == o.n_witness:
        assert g.pairs == oracle_pairs(o)


def oracle_pairs(o):
    """Racy access pairs with their kinds, from the oracle's witness list."""
    out = {}
    for w in o.witnesses:
        out[(w[3], w[4])] = out.get((w[3], w[4]), 0) | w[5]
    return out


def _both(text, binding, cap=1 << 20, **kw):
    # a small binding runs whole in one CTA by default; the device-wide
    # pipeline (NO_SMALL) must give the same result
    g = hg.check(text, binding, cap=cap, **kw)
    flags = kw.pop("flags", 0)
    g2 = hg.check(text, binding, cap=cap, flags=flags | hg.NO_SMALL, **kw)
    assert hg.stats()["small"] == 0
    assert g2 == g
    # with and without the per-cell pre-filter of the sorted keys
    g3 = hg.check(text, binding, cap=cap, flags=flags | hg.NO_SMALL | hg.CELL_FILTER, **kw)
    g4 = hg.check(text, binding, cap=cap, flags=flags | hg.NO_SMALL | hg.NO_CELL_FILTER, **kw)
    assert g3 == g and g4 == g
    # the first scan phase as 32-key warp steps instead of tensor-copied rows
    g5 = hg.check(text, binding, cap=cap, flags=flags | hg.NO_SMALL | hg.SCAN_BALLOT, **kw)
    assert g5 == g
    o = oracle.check(text, binding, cap=cap)
    return g, o


@pytest.mark.parametrize("seed", range(60))
def test_tiny_random_launches(seed):
    w = workloads.random_tiny(1000 + seed, max_instances=500)
    _same(*_both(w.text, w.binding))


@pytest.mark.parametrize("seed", range(40))
def test_small_random_launches(seed):
    w = workloads.random_tiny(20000 + seed, max_instances=20000)
    _same(*_both(w.text, w.binding))


@pytest.mark.parametrize("item", range(6))
def test_config1_plain(item):
    w = workloads.config1(item)
    g, o = _both(w.text, w.binding)
    _same(g, o)
    # the planted write is the kernel's only race
    assert g.n_witness == 1 and g.pairs == {(5, 5): 1}


@pytest.mark.parametrize("item", range(4))
def test_config1_shape_with_unconstrained_accesses(item):
    w = workloads.plain_random(item)
    _same(*_both(w.text, w.binding))


def test_paper_fixtures():
    import json, os
    gold = os.path.join(os.path.dirname(__file__), "golden")
    for name in sorted(os.listdir(gold)):
        if not name.startswith("fig"):
            continue  # the paper's figures; other files hold stored verdicts of other tests
        g = json.load(open(os.path.join(gold, name)))
        for case in g["cases"]:
            if case["expect"] == "EHOSTCONSTRAINT":
                continue
            text = g["descriptor"] if case.get("assert", True) else g["descriptor_without_assert"]
            b = Binding(tuple(case["grid"]), tuple(case["block"]), tuple(case["params"]))
            gr, orr = _both(text, b)
            _same(gr, orr)
            assert gr.racy == (case["expect"] == "racy")


@pytest.mark.parametrize("W,K,planted", [(64, 4, True), (64, 4, False), (128, 8, True), (256, 6, True)])
def test_stencil_small(W, K, planted):
    w = workloads.config2(0, planted=planted, W=W, H=W, K=K)
    g, o = _both(w.text, w.binding)
    _same(g, o)
    assert g.n_witness == (W - 1 if planted else 0)


@pytest.mark.parametrize("item", [0, 1, 2, 5, 6, 7, 10, 11, 12])
def test_stride_sweep_items(item):
    w = workloads.config3()[item]
    _same(*_both(w.text, w.binding))


def test_stride_sweep_large_closed_form():
    # N = 2^16, stride 3: thread g writes A[3g .. 3g+7]; elements touched by
    # two or more threads are exactly 3 <= e < 3(N-1)+8 except the first three
    from test_oracle import _stride_closed_form
    items = [w for w in workloads.config3() if w.meta["N"] == 1 << 14]
    for w in items:
        g = hg.check(w.text, w.binding, cap=1 << 22)
        want = sorted(_stride_closed_form(w.meta["N"], w.meta["stride"], w.binding.block[0]))
        assert g.witnesses == want
        assert g.n_instances == w.binding.grid[0] * w.binding.block[0] * 8 * 12


def test_full_stencil_sampled_against_oracle():
    # the full 1024x1024 stencil in the bench's launch shape: closed form for
    # the witness set, the oracle on every instance for the counts and on the
    # Out rows holding the planted collisions plus a band of In
    w = workloads.config2(0, planted=True)
    g = hg.check(w.text, w.binding, cap=1 << 16)
    want = [(0, 2, 4 * (r + 1) * 1023, 15, 15, 1) for r in range(1023)]
    assert g.witnesses == want
    assert g.n_instances == 536870912
    o = oracle.check(w.text, w.binding, filter_array=2, gran_lo=1023 * 500, gran_hi=1023 * 540)
    assert g.n_keys == o.n_keys and g.n_oob == o.n_oob
    assert [x for x in g.witnesses if 1023 * 500 <= x[2] // 4 < 1023 * 540] == o.witnesses
    assert g.min_x == (0, 16, 0, 0, 0, 0, 15) and g.min_y == (63, 15, 0, 0, 0, 0, 15)
    o2 = oracle.check(w.text, w.binding, filter_array=1, gran_lo=300000, gran_hi=301000)
    assert o2.witnesses == []


def test_full_stencil_clean():
    w = workloads.config2(0, planted=False)
    g = hg.check(w.text, w.binding)
    assert not g.racy and g.n_witness == 0


# ---------------------------------------------------------------- edge cases

EDGE = {
    "empty_loop": ("kernel e\nparam U\nloop i U\narray a global 64\naccess W a ; width 4 ; idx 0\n",
                   Binding((2, 1, 1), (32, 1, 1), (0,))),
    "dead_guard": ("kernel e\narray a global 64\naccess W a ; width 4 ; idx 0 ; if tx > 100\n",
                   Binding((2, 1, 1), (32, 1, 1), ())),
    "single_thread": ("kernel e\nloop i 5\narray a global 64\naccess W a ; width 4 ; idx i % 2\n",
                      Binding((1, 1, 1), (1, 1, 1), ())),
    "ragged_warps": ("kernel e\narray a global 4096\naccess W a ; width 4 ; idx tx / 3\n",
                     Binding((3, 1, 1), (45, 1, 1), ())),
    "grid_3d": ("kernel e\narray a global 4096\narray s shared 256\n"
                "access W a ; width 4 ; idx (bx + 2*by + 4*bz) * 8 + tx / 4\n"
                "access W s ; width 4 ; idx tz * 4 + tx % 4 ; iv 1\n",
                Binding((2, 2, 2), (8, 2, 3), ())),
    "all_oob": ("kernel e\narray a global 16\naccess W a ; width 4 ; idx tx + 8\n",
                Binding((2, 1, 1), (32, 1, 1), ())),
    "wide_int64": ("kernel e\nparam BIG\narray a global 64\n"
                   "access W a ; width 4 ; idx (tx * BIG) % 3 + BIG - BIG\n",
                   Binding((2, 1, 1), (64, 1, 1), (1 << 40,))),
    "float4_mixed": ("kernel e\narray a global 1024\naccess W a ; width 16 ; idx tx\n"
                     "access R a ; width 4 ; idx 4*tx + 5\n", Binding((2, 1, 1), (32, 1, 1), ())),
    "atomics": ("kernel e\narray a global 64\naccess A a ; width 4 ; idx tx % 2 ; scope block\n"
                "access A a ; width 4 ; idx tx % 2 ; scope device\naccess R a ; width 4 ; idx 1 ; iv 1\n",
                Binding((3, 1, 1), (64, 1, 1), ())),
    "negative_mod": ("kernel e\narray a global 400\naccess W a ; width 4 ; idx 50 + (tx - 40) % 7\n"
                     "access W a ; width 4 ; idx 50 + (tx - 40) / 7 ; iv 2\n",
                     Binding((1, 1, 1), (80, 1, 1), ())),
    "one_hot_address_long_run": ("kernel e\nloop i 4\narray a global 64\naccess W a ; width 4 ; idx 3\n",
                                 Binding((64, 1, 1), (256, 1, 1), ())),
    "many_intervals": ("kernel e\nloop i 40\narray s shared 512\naccess W s ; width 4 ; iv i ; idx (tx + i) % 128\n"
                       "access R s ; width 4 ; iv i ; idx (tx + i + 1) % 128\n", Binding((2, 1, 1), (128, 1, 1), ())),
}


@pytest.mark.parametrize("name", sorted(EDGE))
def test_edge_cases(name):
    text, b = EDGE[name]
    _same(*_both(text, b))


def test_truncation_keeps_exact_counts():
    w = workloads.plain_random(0)
    full = hg.check(w.text, w.binding, cap=1 << 20)
    part = hg.check(w.text, w.binding, cap=7)
    assert part.truncated and part.witnesses == full.witnesses[:7]
    assert part.n_witness == full.n_witness and part.n_by_kind == full.n_by_kind


def test_raw_witness_buffer_retry():
    # more per-run witnesses than a tiny raw buffer: ENOMEM then an automatic retry
    w = workloads.plain_random(0)
    g = hg.check(w.text, w.binding, cap=1 << 20, max_raw_witness=64)
    o = oracle.check(w.text, w.binding)
    _same(g, o)


def test_deterministic_and_enqueue_collect():
    import torch
    w = workloads.config1(3)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    a = k.check(cap=1 << 20)
    b = k.check(cap=1 << 20)
    assert a == b
    ws = k.workspace()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        k.enqueue(ws, stream=s)
        c = k.collect(ws, cap=1 << 20, stream=s)
    assert c.witnesses == a.witnesses and c.n_by_kind == a.n_by_kind
    st = hg.stats()
    assert st["kernel_launches"] > 0


@pytest.mark.parametrize("seed", range(12))
def test_restricted_and_stop_first(seed):
    # a check of a subset of the accesses finds exactly the oracle's witnesses
    # among those accesses; stop-at-first keeps the verdict and reports real races
    w = workloads.random_tiny(30000 + seed, max_instances=20000)
    o = oracle.check(w.text, w.binding)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    nacc = w.meta["n_access"]
    mask = 0b101 & ((1 << nacc) - 1) or 1
    want = [x for x in o.witnesses if (mask >> x[3]) & 1 and (mask >> x[4]) & 1]
    full = {x[:5]: x[5] for x in o.witnesses}
    for extra in (0, hg.NO_SMALL):
        r = k.check(cap=1 << 20, only_accesses=mask, flags=extra)
        assert r.witnesses == want
        f = k.check(cap=1 << 20, flags=hg.STOP_FIRST | extra)
        assert f.racy == o.racy
        for x in f.witnesses:
            assert x[:5] in full and (x[5] & ~full[x[:5]]) == 0


@pytest.mark.parametrize("bounds", [(300,), (7, 130), (3, 5, 7, 11)])
def test_long_loops_few_threads(bounds):
    # loop vectors of one simulated warp are split into chunks; the chunk seams
    # must keep emission order and the counters exact
    loops = "".join(f"loop i{l} {b}\n" for l, b in enumerate(bounds))
    off = "i0"
    for l, b in enumerate(bounds[1:], 1):
        off = f"({off})*{b} + i{l}"
    text = ("kernel ll\n" + loops + "array a global 1048576\narray s shared 4096\n"
            f"access W a ; width 4 ; idx ({off}) % 997 + tx\n"
            f"access R a ; width 4 ; iv 1 ; idx ({off}) % 13\n"
            f"access W s ; width 4 ; idx ({off}) % 64 + tx\n")
    _same(*_both(text, Binding((1, 1, 1), (3, 1, 1), ())))


def test_every_sort_shape_gives_the_same_result():
    # the sort autotuner chooses among onesweep CTA shapes; each must be exact
    cur, n = hg.sort_variant()
    try:
        ws = [workloads.config1(2), workloads.config2(0, planted=True, W=128, H=128, K=8)]
        want = [oracle.check(w.text, w.binding) for w in ws]
        for v in range(n):
            hg.sort_variant(v)
            for w, o in zip(ws, want):
                _same(hg.check(w.text, w.binding, cap=1 << 20), o)
                # every key through the sort: every live key written, one
                # global sort, no cell filter
                _same(hg.check(w.text, w.binding, cap=1 << 20,
                               flags=hg.NO_SMALL | hg.NO_SPLIT | hg.NO_CELL_FILTER | hg.ALL_KEYS), o)
                if w is ws[1]:
                    assert hg.stats()["n_sorted_keys"] > 100000
    finally:
        hg.sort_variant(cur)


# ---------------------------------------------------------------- block-local shared bins

@pytest.mark.parametrize("seed", range(48))
def test_shared_bins_against_oracle(seed):
    # shared-memory keys checked in per-block (granule, interval) bins and the
    # same check with one global sort must both equal the oracle
    w = workloads.random_shared(5000 + seed)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    g = k.check(cap=1 << 20, flags=hg.NO_SMALL)
    st = hg.stats()
    _same(g, o)
    _same(k.check(cap=1 << 20), o)
    if st["shared_bins"]:
        assert st["n_sorted_keys"] + st["n_binned_keys"] <= g.n_keys
    n = k.check(cap=1 << 20, flags=hg.NO_SPLIT | hg.NO_SMALL)
    assert hg.stats()["shared_bins"] == 0 and hg.stats()["n_sorted_keys"] <= n.n_keys
    _same(n, o)


def test_shared_bins_are_used():
    used = 0
    for seed in range(48):
        w = workloads.random_shared(5000 + seed)
        hg.check(w.text, w.binding, cap=16, flags=hg.NO_SMALL)
        used += hg.stats()["shared_bins"]
    assert used >= 12


@pytest.mark.parametrize("seed", range(12))
def test_shared_bins_restricted_and_stop_first(seed):
    w = workloads.random_shared(7000 + seed)
    o = oracle.check(w.text, w.binding)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    mask = 0b1011 & ((1 << w.meta["n_access"]) - 1)
    for extra in (0, hg.NO_SMALL):
        r = k.check(cap=1 << 20, only_accesses=mask, flags=extra)
        assert r.witnesses == [x for x in o.witnesses if (mask >> x[3]) & 1 and (mask >> x[4]) & 1]
        f = k.check(cap=1 << 20, flags=hg.STOP_FIRST | extra)
        assert f.racy == o.racy
        full = {x[:5]: x[5] for x in o.witnesses}
        for x in f.witnesses:
            assert x[:5] in full and (x[5] & ~full[x[:5]]) == 0


def test_stencil_bins_skip_the_sort():
    # the shared tile's keys never enter the sort; the clean tile has no
    # candidate bin.  The tile's first staging write goes through a
    # permutation of its 256 cells (a remainder: no bind-time test proves its
    # threads disjoint), so its keys are kept and counted in bins
    w = workloads.config2(0, planted=True, W=256, H=256, K=8)
    text = w.text.replace("; idx lin ;", "; idx (lin*5) % 256 ;")
    assert text != w.text
    g = hg.check(text, w.binding, cap=1 << 20)
    st = hg.stats()
    assert st["shared_bins"] == 1 and st["n_binned_keys"] == 0
    assert st["n_sorted_keys"] < g.n_keys // 4
    n = hg.check(text, w.binding, cap=1 << 20, flags=hg.NO_SPLIT)
    assert n == g
    _same(g, oracle.check(text, w.binding, cap=1 << 20))


# ---------------------------------------------------------------- accesses that cannot race

def test_keys_of_accesses_without_partners_are_counted_not_sorted():
    # reads of a read-only array and device-scope atomics among themselves can
    # race with nothing (pair rule E): counted in n_keys, never written
    text = ("kernel d\narray a global 4096\narray c global 64\narray w global 4096\n"
            "access R a ; width 4 ; idx tx\naccess R a ; width 4 ; idx tx + 1\n"
            "access A c ; width 4 ; idx 0 ; scope device\naccess A c ; width 4 ; idx 1 ; scope device\n"
            "access W w ; width 4 ; idx tx / 2\n")
    b = Binding((4, 1, 1), (64, 1, 1), ())
    for flags in (hg.NO_SMALL, hg.JIT | hg.NO_SMALL):
        g = hg.check(text, b, cap=1 << 20, flags=flags)
        _same(g, oracle.check(text, b, cap=1 << 20))
        assert hg.stats()["n_sorted_keys"] == 4 * 64
    assert g.n_keys == 5 * 4 * 64


@pytest.mark.parametrize("space", ["shared", "global"])
@pytest.mark.parametrize("jit", [0, hg.JIT])
def test_accesses_in_disjoint_barrier_intervals(space, jit):
    # reads whose interval range meets no write's race with nothing inside a
    # block (shared memory: with nothing at all); loop-dependent intervals
    # that meet still race; the verdict is the oracle's either way
    text = (f"kernel iv\nloop k 4\narray S {space} 4096\n"
            "access W S ; width 4 ; iv 0 ; idx tx + 64*bx\n"
            "access R S ; width 4 ; iv 1 ; idx tx + 1 + 64*bx\n"
            "access W S ; width 4 ; iv 2*k + 2 ; idx (tx + k) % 64 + 64*bx\n"
            "access R S ; width 4 ; iv 4 ; idx (tx + 2) % 64 + 64*bx\n"
            "access R S ; width 4 ; iv 9 ; idx tx + 64*bx\n")
    b = Binding((8, 1, 1), (64, 1, 1), ())
    g, o = _both(text, b, flags=jit)
    _same(g, o)
    assert o.racy and g.n_keys == 5 * 8 * 64 * 4


def test_stencil_sorts_only_the_output_keys():
    w = workloads.config2(0, planted=True, W=256, H=256, K=8)
    g = hg.check(w.text, w.binding, cap=1 << 20, flags=hg.NO_CELL_FILTER)
    st = hg.stats()
    assert st["n_sorted_keys"] == 256 * 256  # one Out write per thread; the In reads race with nothing
    _same(g, oracle.check(w.text, w.binding, cap=1 << 20))


def test_room_for_shared_keys_reports_and_retries():
    # every thread of a block writes and reads one of 8 shared cells: 2048 keys
    # in candidate bins; a smaller room is an HGRD_ENOMEM naming the count,
    # and the synchronous call retries with it
    text = "kernel s\narray S shared 1024\naccess W S ; width 4 ; idx tx % 8\naccess R S ; width 4 ; idx tx % 8 ; iv 0\n"
    b = Binding((4, 1, 1), (256, 1, 1), ())
    o = oracle.check(text, b, cap=1 << 20)
    k = hg.Kernel(text).bind(b.grid, b.block, b.params)
    ws = k.workspace(max_shared_keys=100)
    k.enqueue(ws, max_shared_keys=100, flags=hg.NO_SMALL)
    with pytest.raises(hg.HgrdError) as e:
        k.collect(ws, cap=1 << 20, max_shared_keys=100, flags=hg.NO_SMALL)
    assert "ENOMEM" in str(e.value) and "need 2048" in str(e.value)
    g = k.check(cap=1 << 20, max_shared_keys=100, flags=hg.NO_SMALL)
    assert hg.stats()["shared_bins"] == 1 and hg.stats()["n_binned_keys"] == 2048
    _same(g, o)


# ---------------------------------------------------------------- one-CTA path of small checks

@pytest.mark.parametrize("seed", range(4))
def test_small_checks_run_in_one_cta(seed):
    # at most 4096 keys: one CTA (two launches), plus the pair search when racy
    w = workloads.random_tiny(1000 + seed, max_instances=500)
    g = hg.check(w.text, w.binding, cap=1 << 20)
    assert hg.stats()["small"] == 1 and hg.stats()["kernel_launches"] <= 3
    _same(g, oracle.check(w.text, w.binding, cap=1 << 20))


def test_small_check_falls_back_when_it_keeps_too_few_witnesses():
    # 512 runs of two writers and two accesses: 1536 per-run witnesses, more
    # than the one-CTA path keeps; the device-wide pipeline takes over
    text = "kernel f\narray a global 4096\naccess W a ; width 4 ; idx tx / 2\naccess W a ; width 4 ; idx tx / 2\n"
    b = Binding((1, 1, 1), (1024, 1, 1), ())
    g = hg.check(text, b, cap=1 << 20)
    assert hg.stats()["small"] == 0
    _same(g, oracle.check(text, b, cap=1 << 20))


@pytest.mark.parametrize("n_loc", [1, 31, 1000, 1024, 1025, 2000, 2048, 2049, 3500, 4096, 4097, 5000])
def test_witness_merge_sizes(n_loc):
    # n_loc locations, each written by two threads of one access: one raw
    # witness per location.  Up to 1024, 2048 and 4096 raw witnesses the
    # one-CTA merge holds one, two and four per thread; above, the
    # device-wide merge runs.
    text = (f"kernel wm\narray a global {4 * n_loc}\n"
            f"access W a ; width 4 ; idx (bx*512 + tx) / 2 ; if bx*512 + tx < {2 * n_loc}\n")
    b = Binding(((2 * n_loc + 511) // 512, 1, 1), (512, 1, 1), ())
    g = hg.check(text, b, cap=1 << 20, flags=hg.NO_SMALL)
    assert hg.stats()["n_raw_witness"] == n_loc
    o = oracle.check(text, b, cap=1 << 20)
    assert o.n_witness == n_loc
    _same(g, o)


# ---------------------------------------------------------------- warp barriers (Sec. 5.2)

@pytest.mark.parametrize("seed", range(60))
def test_warp_barrier_random_launches(seed):
    w = workloads.random_warp(3000 + seed)
    _same(*_both(w.text, w.binding))


@pytest.mark.parametrize("seed", range(12))
def test_warp_barrier_random_specialised(seed):
    w = workloads.random_warp(3500 + seed, max_instances=20000)
    g = hg.check(w.text, w.binding, cap=1 << 20, flags=hg.JIT)
    _same(g, oracle.check(w.text, w.binding, cap=1 << 20))


@pytest.mark.parametrize("space", ["shared", "global"])
@pytest.mark.parametrize("sync,cross", [("none", False), ("warp", False), ("warp2", False), ("warp2", True),
                                        ("block", True)])
def test_warp_exchange_many_blocks(space, sync, cross):
    # 48 blocks of 32 warps, 4 loop iterations: keys span many sort tiles and
    # every block's exchange is checked; both expansion paths
    w = workloads.warp_exchange(32, 4, sync, cross, grid=48, space=space)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    for flags in (0, hg.NO_JIT | hg.NO_SMALL, hg.JIT):
        g = hg.check(w.text, w.binding, cap=1 << 20, flags=flags)
        _same(g, o)
    # warp intervals change the key layout: the sort covers block and warp interval
    if sync in ("warp", "warp2"):
        assert hg.stats()["sort_passes"] >= 3


@pytest.mark.parametrize("grid", [2047, 2100])
def test_many_units_one_access(grid):
    # ~65k simulated warps of one write access, neighbouring blocks overlapping
    # by one element: grid - 1 inter-block witnesses
    text = "kernel bigscan\narray a global 8800000\naccess W a ; width 4 ; idx bx*1023 + tx\n"
    b = Binding((grid, 1, 1), (1024, 1, 1), ())
    o = oracle.check(text, b, cap=1 << 20)
    assert o.n_witness == grid - 1
    for flags in (hg.NO_SMALL, hg.JIT):
        _same(hg.check(text, b, cap=1 << 20, flags=flags), o)


@pytest.mark.parametrize("planted", [True, False])
def test_cell_filter_sorts_only_shared_cells(planted):
    # stencil 256x256: 256x256x8 possible output keys; with the planted row
    # stride only the 255 cells two blocks write keep their 2 keys each.
    # Without it no key is written at all (below), so there is nothing to filter
    w = workloads.config2(0, planted=planted, W=256, H=256, K=8)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    for flags in (hg.NO_JIT, hg.JIT):
        g = hg.check(w.text, w.binding, cap=1 << 20, flags=flags)
        st = hg.stats()
        assert st["cell_filter"] == (1 if planted else 0)
        assert st["n_sorted_keys"] == (2 * 255 if planted else 0)
        assert st["n_written_keys"] == (256 * 256 if planted else 0) and st["n_binned_keys"] == 0
        _same(g, o)
        _same(hg.check(w.text, w.binding, cap=1 << 20, flags=flags | hg.NO_CELL_FILTER), o)
        # without the planted stride every thread writes its own output
        # element: the write races with nothing (thread-tile pruning) and no
        # global key is written at all
        assert hg.stats()["cell_filter"] == 0 and hg.stats()["n_sorted_keys"] == (256 * 256 if planted else 0)


# ---------------------------------------------------------------- acquire-release guards (Sec. 6.5)

@pytest.mark.parametrize("seed", range(40))
def test_acquire_release_random_against_oracle(seed):
    # guards of the forms decided at bind time (constant elements, or each
    # access's own index), block or device scope, global or shared data
    w = workloads.random_sync(9000 + seed, supported=True)
    _same(*_both(w.text, w.binding))


@pytest.mark.parametrize("seed", range(80))
def test_acquire_release_per_instance_against_oracle(seed):
    # guard elements mixed per kernel (constants, per-thread tx, per-block bx,
    # each access's own index): pairs whose elements can differ between
    # instances are decided instance pair by instance pair in the exact scan
    w = workloads.random_sync(11000 + seed, supported=False)
    _same(*_both(w.text, w.binding))
    _same(hg.check(w.text, w.binding, cap=1 << 20, flags=hg.NO_SMALL | hg.JIT),
          oracle.check(w.text, w.binding, cap=1 << 20))


_RMW = "kernel c\narray c global 4\narray L global 64\narray F global 64\n"
_R, _W = "access R c ; width 4 ; idx 0", "access W c ; width 4 ; idx 0"


@pytest.mark.parametrize("text", [
    _RMW + f"{_R}\n{_W}\n",
    _RMW + f"{_R} ; sync L 0\n{_W} ; sync L 0\n",
    _RMW + f"{_R} ; sync L 0 ; syncscope block\n{_W} ; sync L 0 ; syncscope block\n",
    _RMW + f"{_R} ; sync L 0 ; syncscope block\n{_W} ; sync L 0\n",
    _RMW + f"{_R}\n{_W} ; sync L 0\n",
    _RMW + f"{_R} ; sync L 0\n{_W} ; sync L 1\n",
    "kernel h\narray h global 64\narray L global 64\n"
    "access R h ; width 4 ; idx tx % 4 ; sync L tx % 4\naccess W h ; width 4 ; idx tx % 4 ; sync L tx % 4\n",
    "kernel p\narray d global 4\narray F global 64\naccess W d ; width 4 ; idx 0 ; if tx == 0 ; sync F 0\n"
    "access R d ; width 4 ; idx 0 ; if tx > 0 ; sync F 0\n",
    "kernel p\narray d global 4\narray F global 64\naccess W d ; width 4 ; idx 0 ; if tx == 0 ; sync F 0\n"
    "access R d ; width 4 ; idx 0 ; if tx > 0 ; sync F 1\n",
    # a lock per block: ordered inside a block, not across blocks
    _RMW + f"{_R} ; sync L bx\n{_W} ; sync L bx\n",
    # a lock per thread orders nothing between threads
    _RMW + f"{_R} ; sync L tx\n{_W} ; sync L tx\n",
    # a lock per block in block scope
    _RMW + f"{_R} ; sync L bx + 4 ; syncscope block\n{_W} ; sync L bx + 4 ; syncscope block\n",
    # two lock families on one pair: equal elements only where tx == bx
    _RMW + f"{_R} ; sync L tx\n{_W} ; sync L bx\n",
])
@pytest.mark.parametrize("jit", [0, hg.JIT])
def test_acquire_release_fixtures(text, jit):
    # counter read-modify-write under no lock, one lock (device or block
    # scope), a lock on one side, two locks; per-element locks; producer /
    # consumer flags: each result equals the oracle's
    b = Binding((4, 1, 1), (64, 1, 1), ())
    g, o = _both(text, b, flags=jit)
    _same(g, o)


# ---------------------------------------------------------------- block-pair pruning

@pytest.mark.parametrize("text", [
    # own slices: the neighbour read races inside a block only
    "kernel s\narray G global 4096\naccess W G ; width 4 ; idx bx*64 + tx\n"
    "access R G ; width 4 ; idx bx*64 + (tx + 1) % 64\n",
    # slices that meet through the loop: an inter-block race at every seam
    "kernel m\nloop i 2\narray G global 4096\naccess W G ; width 4 ; idx bx*64 + tx + i\n",
    # own slices in another interval: the read races with nothing
    "kernel o\narray G global 4096\naccess W G ; width 4 ; idx bx*64 + tx\n"
    "access R G ; width 4 ; iv 1 ; idx bx*64 + tx\naccess W G ; width 4 ; iv 1 ; idx bx*64 + 63 - tx\n",
])
def test_block_pair_pruning_against_oracle(text):
    b = Binding((8, 1, 1), (64, 1, 1), ())
    for jit in (0, hg.JIT):
        g, o = _both(text, b, flags=jit)
        _same(g, o)


@pytest.mark.parametrize("seed", range(12))
def test_every_key_through_the_sort(seed):
    # HGRD_ALL_KEYS: the keys the pair rule would drop are written, sorted and
    # scanned as well; the result is the oracle's all the same
    w = workloads.random_tiny(5000 + seed, max_instances=20000)
    g = hg.check(w.text, w.binding, cap=1 << 20, flags=hg.ALL_KEYS)
    st = hg.stats()
    assert st["shared_bins"] == 0 and st["jit"] == 0 and st["small"] == 0
    _same(g, oracle.check(w.text, w.binding, cap=1 << 20))
    assert hg.check(w.text, w.binding, cap=1 << 20, flags=hg.ALL_KEYS | hg.SCAN_BALLOT) == g


def test_every_key_through_the_sort_on_the_stencil():
    w = workloads.config2(0, planted=True, W=128, H=128, K=8)
    g = hg.check(w.text, w.binding, cap=1 << 20, flags=hg.ALL_KEYS | hg.NO_CELL_FILTER)
    assert hg.stats()["n_sorted_keys"] == g.n_keys  # every live key went through the sort
    _same(g, oracle.check(w.text, w.binding, cap=1 << 20))
    assert hg.check(w.text, w.binding, cap=1 << 20, flags=hg.ALL_KEYS | hg.NO_CELL_FILTER | hg.SCAN_BALLOT) == g


def test_sort_shapes_chosen_per_pass():
    # each pass of the key sort on its own shape (the tuner's per-pass
    # choice): the stable LSD sort composes, the result is the oracle's
    w = workloads.config2(0, planted=True, W=128, H=128, K=8)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    _, n = hg.sort_variant()
    try:
        for shapes in ((0, 4, 7), (4, 2, 0), (6, 5, 11)):
            for p, v in enumerate(shapes):
                hg.sort_pass_variant(p, v % n)
            assert [hg.sort_pass_variant(p) for p in range(3)] == [v % n for v in shapes]
            g = hg.check(w.text, w.binding, cap=1 << 20, flags=hg.ALL_KEYS | hg.NO_CELL_FILTER)
            assert hg.stats()["sort_passes"] == 3
            _same(g, o)
    finally:
        for p in range(3):
            hg.sort_pass_variant(p, -1)
    assert hg.sort_pass_variant(0) == -1


@pytest.mark.parametrize("pairs_of_writers", [100, 2047, 2048, 6000])
def test_cell_filter_compact_form_and_fallback(pairs_of_writers):
    # two threads write each element: with the cell filter every written key
    # is kept; up to 4096 kept keys one CTA sorts them whole from the write
    # pass's compact buffer, beyond that the filter and the sort passes run
    n = 2 * pairs_of_writers
    text = (f"kernel pairs\narray a global {4 * pairs_of_writers}\narray r global {4 * n}\n"
            "access W a ; width 4 ; idx (bx*256 + tx)/2\n"
            "access R r ; width 4 ; idx bx*256 + tx\n"
            "access W a ; width 4 ; idx 0 ; if 0 - bx*256 - tx >= 0\n")
    b = Binding(((n + 255) // 256, 1, 1), (256, 1, 1), ())
    o = oracle.check(text, b, cap=1 << 20)
    for flags in (hg.CELL_FILTER | hg.NO_SMALL, hg.CELL_FILTER | hg.NO_SMALL | hg.JIT):
        g = hg.check(text, b, cap=1 << 20, flags=flags)
        st = hg.stats()
        assert st["cell_filter"] == 1
        assert st["n_sorted_keys"] == n + 1  # every write of `a` (the lone write of a[0] included)
        _same(g, o)
