"""Pins for the CPU oracle: nothing here compares the oracle with itself.

* pairwise brute force (tests/brute.py) on tiny random launches;
* the paper's worked examples (tests/golden/, each with its citation);
* closed forms worked out by hand for the stride sweep, the planted stencil
  row stride and the all-threads-one-address kernel;
* invariants of the race definition (an extra barrier, a removed access or a
  write turned into a read never adds a witness; relabelling threads inside a
  block keeps the witness set).
"""
import json
import math
import os
import re

import pytest

import oracle
import workloads
from workloads import Binding
import brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cmp_brute(w):
    r = oracle.check(w.text, w.binding)
    b = brute.check(w.text, w.binding)
    assert r.witnesses == b["witnesses"]
    assert r.n_witness == len(b["witnesses"])
    assert r.n_keys == b["n_keys"] and r.n_oob == b["n_oob"]
    assert r.n_instances == b["n_instances"]
    for k in range(3):
        assert r.n_by_kind[k] == sum(1 for x in b["witnesses"] if x[5] >> k & 1)
    if b["witnesses"]:
        assert r.min_w == b["witnesses"][0]
        kx, ky = b["min_pair"]
        assert r.min_x[:6] == kx and r.min_y[:6] == ky
        assert r.min_x[6] == r.min_w[3] and r.min_y[6] == r.min_w[4]
    else:
        assert not r.racy


@pytest.mark.parametrize("seed", range(60))
def test_oracle_matches_brute_force_tiny(seed):
    w = workloads.random_tiny(1000 + seed, max_instances=500)
    _cmp_brute(w)


def test_oracle_matches_brute_force_config1():
    _cmp_brute(workloads.config1(0))
    _cmp_brute(workloads.plain_random(0))


def test_config1_holds_exactly_the_planted_race():
    # the five drawn accesses are race free by construction (read-only G,
    # thread-owned S slots in intervals with an S write); the planted write
    # of thread 0 in every block is the one race, inter-block write-write
    for item in range(24):
        w = workloads.config1(item)
        o = oracle.check(w.text, w.binding)
        assert o.n_witness == 1 and o.n_by_kind == (1, 0, 0), item
        assert (o.witnesses[0][3], o.witnesses[0][4], o.witnesses[0][5]) == (5, 5, 1)


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", sorted(n for n in os.listdir(GOLD) if n.startswith("fig")))
def test_paper_worked_examples(name):
    g = _gold(name)
    for case in g["cases"]:
        text = g["descriptor"] if case.get("assert", True) else g["descriptor_without_assert"]
        b = Binding(tuple(case["grid"]), tuple(case["block"]), tuple(case["params"]))
        if case["expect"] == "EHOSTCONSTRAINT":
            with pytest.raises(oracle.OracleError) as ei:
                oracle.check(text, b)
            assert ei.value.code == -4
            continue
        r = oracle.check(text, b)
        assert r.racy == (case["expect"] == "racy"), (name, case)
        if "kind_bits_include" in case:
            assert any(w[5] & case["kind_bits_include"] for w in r.witnesses)
        if "witnesses" in case:
            assert [list(w) for w in r.witnesses] == case["witnesses"]


# ---------------------------------------------------------------- closed forms

def test_all_threads_one_address():
    text = "kernel one\narray res global 64\naccess W res ; width 4 ; idx 0\n"
    # 3 blocks x 40 threads: threads 0..39 span warps 0 and 1
    r = oracle.check(text, Binding((3, 1, 1), (40, 1, 1), ()))
    assert r.witnesses == [(0, 0, 0, 0, 0, 7)]
    # one warp per block: no intra-block (different warp) pair exists
    r = oracle.check(text, Binding((2, 1, 1), (32, 1, 1), ()))
    assert r.witnesses == [(0, 0, 0, 0, 0, 5)]
    # a single thread cannot race with itself
    r = oracle.check(text, Binding((1, 1, 1), (1, 1, 1), ()))
    assert not r.racy
    # shared memory: per-block copies, so no inter-block bit
    text_s = "kernel one\narray res shared 64\naccess W res ; width 4 ; idx 0\n"
    r = oracle.check(text_s, Binding((3, 1, 1), (40, 1, 1), ()))
    assert r.witnesses == [(1, 0, 0, 0, 0, 6)]


def test_atomics_and_scopes():
    base = "kernel at\narray a global 64\narray s shared 64\n"
    # device-scope atomics never race (Appendix A, trivially race free)
    t = base + "access A a ; width 4 ; idx 0 ; scope device\n"
    assert not oracle.check(t, Binding((2, 1, 1), (64, 1, 1), ())).racy
    # block-scope atomics race across blocks only (insufficient scope)
    t = base + "access A a ; width 4 ; idx 0 ; scope block\n"
    assert oracle.check(t, Binding((2, 1, 1), (64, 1, 1), ())).witnesses == [(0, 0, 0, 0, 0, 1)]
    assert not oracle.check(t, Binding((1, 1, 1), (64, 1, 1), ())).racy
    # a read against an atomic is a race
    t = base + "access A a ; width 4 ; idx 0\naccess R a ; width 4 ; idx 0\n"
    r = oracle.check(t, Binding((1, 1, 1), (64, 1, 1), ()))
    assert r.witnesses == [(0, 0, 0, 0, 1, 6)]
    # shared-memory block-scope atomics never race
    t = base + "access A s ; width 4 ; idx 0 ; scope block\n"
    assert not oracle.check(t, Binding((4, 1, 1), (64, 1, 1), ())).racy


def _stride_closed_form(N, S, bd):
    """Witnesses of the A array of the strided sweep kernel, derived by hand.

    Thread g (g < N) writes A[g*S + i], i < 8, in interval 0 (access 0) and
    reads the same elements in interval 1 (access 1).  Element e is touched by
    the threads g in [ceil((e-7)/S), floor(e/S)] ∩ [0, N).  (0,0) races when at
    least two threads touch e; (0,1) only across blocks (the reads follow a
    barrier inside a block); (1,1) never (two loads).
    """
    out = []
    for e in range(0, (N - 1) * S + 8):
        lo = max(0, -((7 - e) // S) if e >= 7 else 0)
        lo = max(0, math.ceil((e - 7) / S))
        hi = min(N - 1, e // S)
        gs = list(range(lo, hi + 1))
        if len(gs) < 2:
            continue
        blocks = {g // bd for g in gs}
        m = 0
        if len(blocks) > 1:
            m |= 1
        for b in blocks:
            ws = [g % bd // 32 for g in gs if g // bd == b]
            if len(ws) > 1:
                if len(set(ws)) > 1:
                    m |= 2
                if any(ws.count(x) > 1 for x in set(ws)):
                    m |= 4
        out.append((0, 0, 4 * e, 0, 0, m))
        if len(blocks) > 1:
            out.append((0, 0, 4 * e, 0, 1, 1))
    return out


@pytest.mark.parametrize("N,S,bd", [(96, 1, 64), (100, 3, 64), (64, 4, 32), (70, 8, 64), (40, 32, 64), (130, 2, 128)])
def test_stride_sweep_closed_form(N, S, bd):
    text = workloads.config3_kernel_text()
    grid = (N + bd - 1) // bd
    r = oracle.check(text, Binding((grid, 1, 1), (bd, 1, 1), (N, S)))
    want = sorted(_stride_closed_form(N, S, bd))
    assert r.witnesses == want
    assert r.racy == (S < 8)


@pytest.mark.parametrize("planted", [False, True])
def test_stencil_planted_row_stride(planted):
    # the tiled stencil on a 64x64 image with a 4-row window: the planted row
    # stride R = W - 1 collides (r, W-1) with (r+1, 0), W-1 inter-block pairs
    w = workloads.config2(0, planted=planted, W=64, H=64, K=4)
    r = oracle.check(w.text, w.binding)
    if planted:
        want = [(0, 2, 4 * (rr + 1) * 63, 15, 15, 1) for rr in range(63)]
        assert r.witnesses == want
        assert r.n_by_kind == (63, 0, 0)
    else:
        assert not r.racy
    assert r.n_instances == 4 * 4 * 256 * 4 * 16
    assert r.n_oob == 0


def test_host_classes_reject_bindings():
    t = workloads.fig1_copy_upp_low(with_assert=True)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.check(t, Binding((1, 1, 1), (4, 4, 1), (4,)))
    assert ei.value.code == -3  # missing parameter
    bad_div = "kernel d\nparam Q\narray a global 64\naccess W a ; width 4 ; idx tx / Q\n"
    with pytest.raises(oracle.OracleError) as ei:
        oracle.check(bad_div, Binding((1, 1, 1), (4, 1, 1), (0,)))
    assert ei.value.code == -3
    with pytest.raises(oracle.OracleError) as ei:
        oracle.check("kernel d\narray a global 64\naccess W a ; width 4 ; idx tx*ty\n",
                     Binding((1, 1, 1), (4, 1, 1), ()))
    assert ei.value.code == -2


def test_c_division_truncates_toward_zero():
    # idx = (tx - 5) / 2 and (tx - 5) % 3 evaluated for tx < 10 with C semantics
    t = ("kernel neg\narray a global 4096\n"
         "access W a ; width 4 ; idx 100 + (tx - 5) / 2\n"
         "access W a ; width 4 ; idx 200 + (tx - 5) % 3 ; iv 1\n")
    r = oracle.check(t, Binding((1, 1, 1), (10, 1, 1), ()))
    # truncation: tx=3,4 -> -1,0; tx=5,6 -> 0,0 ... elements hit by two threads
    q = [int((x - 5) / 2) for x in range(10)]
    m = [(x - 5) - 3 * int((x - 5) / 3) for x in range(10)]
    want = []
    for v in sorted(set(q)):
        if q.count(v) > 1:
            want.append((0, 0, 4 * (100 + v), 0, 0, 4))
    for v in sorted(set(m)):
        if m.count(v) > 1:
            want.append((0, 0, 4 * (200 + v), 1, 1, 4))
    assert r.witnesses == sorted(want)


# ---------------------------------------------------------------- invariants

def _acc_lines(text):
    return [i for i, l in enumerate(text.splitlines()) if l.startswith("access")]


def _set_of(r):
    return {w[:5]: w[5] for w in r.witnesses}


@pytest.mark.parametrize("seed", range(25))
def test_invariant_more_barriers_never_add_races(seed):
    w = workloads.random_tiny(5000 + seed, max_instances=600)
    lines = w.text.splitlines()
    base = _set_of(oracle.check(w.text, w.binding))
    # split every interval: give access k its own interval k (a barrier between all)
    for k, li in enumerate(_acc_lines(w.text)):
        f = [x for x in lines[li].split(" ; ") if not x.startswith("iv ")]
        f.insert(1, f"iv {k}")
        lines[li] = " ; ".join(f)
    split = _set_of(oracle.check("\n".join(lines) + "\n", w.binding))
    for key, m in split.items():
        assert key in base and (m & ~base[key]) == 0


@pytest.mark.parametrize("seed", range(25))
def test_invariant_removal_and_read_only(seed):
    w = workloads.random_tiny(7000 + seed, max_instances=600)
    base = _set_of(oracle.check(w.text, w.binding))
    lines = w.text.splitlines()
    acc = _acc_lines(w.text)
    # writes turned into reads: a subset (witness access ids unchanged)
    ro = list(lines)
    for li in acc:
        ro[li] = re.sub(r"^access [WA] ", "access R ", ro[li])
        ro[li] = ro[li].replace(" ; scope block", "").replace(" ; scope device", "")
    assert _set_of(oracle.check("\n".join(ro) + "\n", w.binding)) == {}
    # drop the last access: witnesses of the remaining pairs only, none new
    drop = [l for i, l in enumerate(lines) if i != acc[-1]]
    last = len(acc) - 1
    sub = _set_of(oracle.check("\n".join(drop) + "\n", w.binding))
    want = {k: m for k, m in base.items() if k[3] != last and k[4] != last}
    assert sub == want


@pytest.mark.parametrize("seed", range(20))
def test_invariant_thread_relabelling(seed):
    # tx -> bdx-1-tx is a bijection of the threads of a block; the witness set
    # is unchanged, the inter-block bit is unchanged, and "some same-block race"
    # (intra-block or intra-warp) is unchanged
    w = workloads.random_tiny(9000 + seed, max_instances=600)
    lines = w.text.splitlines()
    for li in _acc_lines(w.text):
        lines[li] = re.sub(r"\btx\b", "(bdx - 1 - tx)", lines[li])
    a = _set_of(oracle.check(w.text, w.binding))
    b = _set_of(oracle.check("\n".join(lines) + "\n", w.binding))
    assert a.keys() == b.keys()
    for k in a:
        assert (a[k] & 1) == (b[k] & 1)
        assert bool(a[k] & 6) == bool(b[k] & 6)


# ---------------------------------------------------------------- warp barriers (Sec. 5.2, Sec. 6.1)

@pytest.mark.parametrize("seed", range(40))
def test_oracle_matches_brute_force_warp_barriers(seed):
    _cmp_brute(workloads.random_warp(3000 + seed))


# warp_exchange closed forms: the write of S[t] and the neighbour's read race
# on every granule of S unless the barriers order them; the kind is
# intra-warp for the lane + 1 neighbour, intra-block for the next warp.
# In a loop with one barrier per iteration the read of iteration i and the
# write of iteration i + 1 stay unordered (a loop-carried race).
@pytest.mark.parametrize("sync,loops,cross,racy", [
    ("none", 0, False, True), ("none", 0, True, True), ("none", 3, False, True),
    ("warp", 0, False, False), ("warp", 0, True, True), ("warp", 3, False, True), ("warp", 3, True, True),
    ("warp2", 0, False, False), ("warp2", 3, False, False), ("warp2", 3, True, True),
    ("block", 0, False, False), ("block", 0, True, False), ("block", 3, False, True), ("block", 3, True, True),
])
@pytest.mark.parametrize("n_warps", [1, 2, 3])
def test_warp_exchange_closed_form(sync, loops, cross, racy, n_warps):
    if cross and n_warps == 1:
        racy = False  # the "next warp" is the warp itself: thread t reads S[t]
    w = workloads.warp_exchange(n_warps, loops, sync, cross)
    r = oracle.check(w.text, w.binding)
    kind = 4 if not cross else 2
    want = [(1, 0, 4 * g, 0, 1, kind) for g in range(32 * n_warps)] if racy else []
    assert r.witnesses == want
    if racy:
        # the smallest racing pair: writer thread of granule 0 against its reader
        rd = (32 * n_warps - 32) if cross else 31
        assert r.min_x[:2] == (0, 0) and r.min_y[:2] == (0, rd)


@pytest.mark.parametrize("seed", range(25))
def test_invariant_distinct_warp_intervals_drop_only_intra_warp(seed):
    # a warp barrier between every two accesses (access k in warp interval k)
    # orders same-warp pairs of different accesses; it leaves pairs of one
    # access with itself (other loop vectors, same interval), and every other
    # kind, as they were
    w = workloads.random_tiny(11000 + seed, max_instances=600)
    lines = w.text.splitlines()
    base = _set_of(oracle.check(w.text, w.binding))
    for k, li in enumerate(_acc_lines(w.text)):
        f = lines[li].split(" ; ")
        f.insert(1, f"wv {k}")
        lines[li] = " ; ".join(f)
    got = _set_of(oracle.check("\n".join(lines) + "\n", w.binding))
    want = {}
    for key, m in base.items():
        m2 = m if key[3] == key[4] else m & ~4
        if m2:
            want[key] = m2
    assert got == want


@pytest.mark.parametrize("space", ["shared", "global"])
def test_warp_exchange_expected_counts(space):
    # the witness count the bench asserts for its warp-barrier workload
    for nw in (1, 2, 3):
        for loops in (0, 1, 3):
            for sync in ("none", "warp", "warp2", "block"):
                for cross in (False, True):
                    w = workloads.warp_exchange(nw, loops, sync, cross, grid=2, space=space)
                    assert oracle.check(w.text, w.binding).n_witness == w.meta["expected_witnesses"]


# ---------------------------------------------------------------- acquire-release (Sec. 6.5)

@pytest.mark.parametrize("seed", range(60))
def test_oracle_matches_brute_force_acquire_release(seed):
    _cmp_brute(workloads.random_sync(7000 + seed))


def _kinds(text, grid=(2, 1, 1), block=(64, 1, 1)):
    """{(acc_lo, acc_hi): OR of the kind masks of that pair's witnesses}"""
    r = oracle.check(text, Binding(grid, block, ()), cap=1 << 20)
    out = {}
    for w in r.witnesses:
        out[(w[3], w[4])] = out.get((w[3], w[4]), 0) | w[5]
    return out


def test_acquire_release_closed_forms():
    # a read-modify-write of one counter by every thread of two blocks of two
    # warps: every race type between the read and the write and among writes
    rmw = "kernel c\narray c global 4\narray L global 64\narray F global 64\n"
    R, W = "access R c ; width 4 ; idx 0", "access W c ; width 4 ; idx 0"
    assert _kinds(rmw + f"{R}\n{W}\n") == {(0, 1): 7, (1, 1): 7}
    # both inside one device-scope lock (Sec. 6.5 "Lock/unlock"): no race
    assert _kinds(rmw + f"{R} ; sync L 0\n{W} ; sync L 0\n") == {}
    # a block-scope lock orders one block's threads only (Appendix A): with
    # both guards block scoped every inter-block pair races; with the read's
    # block scoped, the read-write pairs do, the writes (device) do not
    assert _kinds(rmw + f"{R} ; sync L 0 ; syncscope block\n{W} ; sync L 0 ; syncscope block\n") == \
        {(0, 1): 1, (1, 1): 1}
    assert _kinds(rmw + f"{R} ; sync L 0 ; syncscope block\n{W} ; sync L 0 ; syncscope device\n") == {(0, 1): 1}
    # only the write guarded: the read still races with it; writes do not
    assert _kinds(rmw + f"{R}\n{W} ; sync L 0\n") == {(0, 1): 7}
    # locks of different addresses do not order (Table 2, addr(syn) differ)
    assert _kinds(rmw + f"{R} ; sync L 0\n{W} ; sync L 1\n") == {(0, 1): 7}
    # a lock per thread: other threads hold other locks
    assert _kinds(rmw + f"{R} ; sync L tx\n{W} ; sync L tx\n") == {(0, 1): 7, (1, 1): 7}
    # a lock per block: one block's threads are ordered, blocks are not
    assert _kinds(rmw + f"{R} ; sync L bx\n{W} ; sync L bx\n") == {(0, 1): 1, (1, 1): 1}
    # per-element locks of a histogram (any function of the element) order it;
    # a lock index that two threads of one element do not share does not
    h = "kernel h\narray h global 16\narray L global 64\n"
    for lk, racy in (("tx % 4", False), ("tx % 2", False), ("(tx + 1) % 4", False), ("tx % 8", True)):
        t = h + f"access R h ; width 4 ; idx tx % 4 ; sync L {lk}\naccess W h ; width 4 ; idx tx % 4 ; sync L {lk}\n"
        assert bool(_kinds(t, grid=(1, 1, 1), block=(32, 1, 1))) == racy, lk
    # producer / consumer (Sec. 6.5): the producer's write released at flag
    # F[0], the consumers' reads acquired at it
    pc = "kernel p\narray d global 4\narray F global 64\naccess W d ; width 4 ; idx 0 ; if tx == 0 ; sync F 0\n"
    assert _kinds(pc + "access R d ; width 4 ; idx 0 ; if tx > 0 ; sync F 0\n") == {}
    # (the two blocks' producers stay ordered by their common flag)
    assert _kinds(pc + "access R d ; width 4 ; idx 0 ; if tx > 0 ; sync F 1\n") == {(0, 1): 7}


@pytest.mark.parametrize("seed", range(40))
def test_invariant_guards_never_add_races(seed):
    # dropping every acquire-release guard keeps every witness and may add
    # some; a witness keeps every kind it had
    w = workloads.random_sync(8000 + seed)
    g = oracle.check(w.text, w.binding, cap=1 << 20)
    bare = "\n".join(" ; ".join(f for f in l.split(" ; ") if not f.startswith(("sync ", "syncscope ")))
                     for l in w.text.splitlines()) + "\n"
    u = oracle.check(bare, w.binding, cap=1 << 20)
    full = {x[:5]: x[5] for x in u.witnesses}
    for x in g.witnesses:
        assert x[:5] in full and (x[5] & ~full[x[:5]]) == 0
    assert g.n_keys == u.n_keys and g.n_oob == u.n_oob


def test_acquire_release_with_barriers_and_widths():
    # barrier intervals still order one block; guards decide the rest
    rmw = "kernel c\narray c global 4\narray L global 64\n"
    t = (rmw + "access R c ; width 4 ; iv 0 ; idx 0 ; sync L 0 ; syncscope {s}\n"
         "access W c ; width 4 ; iv 1 ; idx 0 ; sync L 0 ; syncscope {s}\n")
    assert _kinds(t.format(s="block")) == {(0, 1): 1, (1, 1): 1}
    assert _kinds(t.format(s="device")) == {}
    # a float4 write guarded at its element, int reads of its words guarded at
    # the word's element (another address) or at the float4's (the same one);
    # thread t reads the word written by thread t / 4: the same warp for
    # t < 32, the other warp beyond
    v = ("kernel v\narray d global 1024\narray L global 1024\n"
         "access W d ; width 16 ; idx tx ; sync L tx\n"
         "access R d ; width 4 ; idx tx ; sync L {r}\n")
    assert _kinds(v.format(r="tx"), grid=(1, 1, 1), block=(64, 1, 1)) == {(0, 1): 6}
    assert _kinds(v.format(r="tx / 4"), grid=(1, 1, 1), block=(64, 1, 1)) == {}


def test_vectorised_stride_closed_form_matches_hand_form_and_oracle():
    # the array form of the strided sweep's closed form (used at N up to 2^20
    # on the GPU) against the per-element hand form and the oracle
    import closed_forms as cf
    for N, S, bd in [(96, 1, 64), (100, 3, 64), (64, 4, 32), (70, 8, 64), (40, 32, 64), (1000, 1, 64),
                     (513, 3, 256), (777, 2, 96)]:
        b, lo, hi, k = cf.stride_witnesses(N, S, bd)
        got = [(0, 0, int(x), int(y), int(z), int(m)) for x, y, z, m in zip(b, lo, hi, k)]
        assert got == sorted(_stride_closed_form(N, S, bd)), (N, S, bd)
    for w in workloads.config3()[:15]:
        N, S = w.binding.params
        bd, g = w.binding.block[0], w.binding.grid[0]
        o = oracle.check(w.text, w.binding, pair=False)
        b, lo, hi, k = cf.stride_witnesses(N, S, bd)
        assert o.witnesses == [(0, 0, int(x), int(y), int(z), int(m)) for x, y, z, m in zip(b, lo, hi, k)]
        assert o.n_keys == cf.stride_keys(N, g, bd) and o.n_oob == 0


def test_parallel_oracle_equals_the_oracle():
    # the bands partition the buckets (granule % jobs), so the merged result
    # of the banded runs is the whole-kernel result
    import multiprocessing as mp
    cases = [workloads.plain_random(1), workloads.config1(2), workloads.random_tiny(77, max_instances=4000),
             workloads.config2(0, planted=True, W=64, H=64, K=4), workloads.random_shared(5, max_instances=8000)]
    with mp.get_context("spawn").Pool(3) as pool:
        for w in cases:
            want = oracle.check(w.text, w.binding)
            got = oracle.check_parallel(w.text, w.binding, jobs=3, pool=pool)
            assert (got.witnesses, got.n_witness, got.n_by_kind, got.n_keys, got.n_oob, got.n_instances) == \
                   (want.witnesses, want.n_witness, want.n_by_kind, want.n_keys, want.n_oob, want.n_instances)
            assert (got.min_w, got.min_x, got.min_y) == (want.min_w, want.min_x, want.min_y)
