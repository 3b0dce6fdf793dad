"""Specialised expansion kernels (compiled at run time) against the oracle.

Same comparisons as the interpreted path: canonical witnesses, per-kind
counts, key / instance / out-of-bounds counts, minimal witness and instance
pair, on both pipelines (block-local shared bins and one global sort), the
int64 path, chunked long loops and restricted checks.
"""
import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads
from test_gpu_parity import EDGE, _same
from workloads import Binding

pytestmark = pytest.mark.gpu


def _jit_check(w_text, binding, flags=0, **kw):
    k = hg.Kernel(w_text).bind(binding.grid, binding.block, binding.params)
    r = k.check(cap=1 << 20, flags=flags | hg.JIT, **kw)
    assert hg.stats()["jit"] == 1
    return k, r


@pytest.mark.parametrize("seed", range(12))
def test_jit_random_tiny(seed):
    w = workloads.random_tiny(20000 + seed, max_instances=20000)
    _, r = _jit_check(w.text, w.binding)
    _same(r, oracle.check(w.text, w.binding, cap=1 << 20))


@pytest.mark.parametrize("seed", range(12))
def test_jit_random_shared_both_pipelines(seed):
    w = workloads.random_shared(5000 + seed)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    k, r = _jit_check(w.text, w.binding)
    _same(r, o)
    r2 = k.check(cap=1 << 20, flags=hg.JIT | hg.NO_SPLIT)
    assert hg.stats()["jit"] == 1 and hg.stats()["shared_bins"] == 0
    _same(r2, o)


@pytest.mark.parametrize("name", ["wide_int64", "negative_mod", "grid_3d", "ragged_warps", "many_intervals",
                                  "atomics", "float4_mixed"])
def test_jit_edge_cases(name):
    text, b = EDGE[name]
    _, r = _jit_check(text, b)
    _same(r, oracle.check(text, b, cap=1 << 20))


def test_jit_stencil_matches_oracle_and_interpreter():
    w = workloads.config2(0, planted=True, W=256, H=256, K=8)
    k, r = _jit_check(w.text, w.binding)
    _same(r, oracle.check(w.text, w.binding, cap=1 << 20))
    assert r == k.check(cap=1 << 20, flags=hg.NO_JIT)
    # once compiled, plain checks of the binding use the specialised kernels
    k.check(cap=16)
    assert hg.stats()["jit"] == 1


def test_jit_long_loops_and_restricted():
    text = ("kernel ll\nloop i0 7\nloop i1 130\narray a global 1048576\narray s shared 4096\n"
            "access W a ; width 4 ; idx (i0*130 + i1) % 997 + tx\n"
            "access R a ; width 4 ; iv 1 ; idx (i0*130 + i1) % 13\n"
            "access W s ; width 4 ; idx (i0*130 + i1) % 64 + tx\n")
    b = Binding((1, 1, 1), (3, 1, 1), ())
    o = oracle.check(text, b, cap=1 << 20)
    k, r = _jit_check(text, b)
    _same(r, o)
    r3 = k.check(cap=1 << 20, flags=hg.JIT, only_accesses=0b011)
    assert r3.witnesses == [x for x in o.witnesses if x[3] < 2 and x[4] < 2]


def test_jit_compile_reports_time_and_caches():
    w = workloads.config2(0, planted=False, W=64, H=64, K=4)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    k.jit_compile()
    k2 = hg.Kernel(w.text).bind((8, 8, 1), (16, 16, 1), (128, 128, 128))
    assert k2.jit_compile() == 0.0  # same structure: a cache hit


@pytest.mark.parametrize("block", [(40, 1, 1), (128, 2, 1)])
def test_jit_loop_invariant_accesses(block):
    # accesses whose guards, index and interval ignore the loop counters are
    # taken once per unit in the count pass (multiplicity = the unit's loop
    # vectors, chunked when the loops are long): counts, out-of-bounds
    # instances and bins must be those of the full walk
    # (reads of the read-only arrays r, q race with nothing: r's index moves
    # with the loops but stays in bounds, q's leaves them for some vectors)
    text = ("kernel inv\nloop i 100\nloop j 3\narray s shared 256\narray g global 4096\n"
            "array r global 4096\narray q global 64\n"
            "access W s ; width 4 ; idx tx % 5\n"
            "access R s ; width 4 ; idx tx + 60 ; iv 1\n"
            "access W s ; width 4 ; idx tx ; if tx < 3 ; iv 1\n"
            "access R s ; width 4 ; idx (i + j) % 64 ; iv 1\n"
            "access W g ; width 4 ; idx tx + 4*j\n"
            "access R r ; width 4 ; idx (tx + i) % 1000 ; if tx >= 2\n"
            "access R q ; width 4 ; idx tx + i\n")
    b = Binding((2, 1, 1), block, ())
    o = oracle.check(text, b, cap=1 << 20)
    k, r = _jit_check(text, b)
    assert hg.stats()["shared_bins"] == 1
    _same(r, o)
    assert r.n_oob == o.n_oob > 0
    _same(k.check(cap=1 << 20, flags=hg.JIT | hg.NO_SPLIT), o)


@pytest.mark.parametrize("block", [(40, 1, 1), (128, 2, 1)])
@pytest.mark.parametrize("bound", [32, 700])
def test_jit_loop_guard_ranges(block, bound):
    # accesses whose only loop dependence is a guard on the loop counter
    # (c0 + c*k >= 0) are taken once per unit over the counters the guards
    # admit (count pass; multiplicity = their number inside the unit's chunk,
    # chunked when the loop is long), and the write pass visits only the
    # counters where a kept access can be live; counts, out-of-bounds
    # instances, bins and the canonical pair (recorded at the first admitted
    # counter) must be those of the full walk
    text = (f"kernel lg\nparam C\nloop k {bound}\narray s shared 512\narray g global 8192\narray o global 1024\n"
            "access W s ; width 4 ; idx tx ; if k == C\n"
            "access R s ; width 4 ; idx tx / 2 ; if k >= C ; if 2*k < 3*C ; iv 0\n"
            "access W g ; width 4 ; idx bx*300 + tx / 3 ; if k > C - 3 ; if k <= C\n"
            "access R g ; width 4 ; idx bx*300 + tx + 1 ; if 5 - k >= 0\n"
            "access W o ; width 4 ; idx tx + 200 ; if k == 4\n"   # partly out of bounds
            "access A g ; width 4 ; idx 7 ; if -k + 3*C >= 0 ; scope block\n")
    for C in (5, 17):
        b = Binding((3, 1, 1), block, (C,))
        o = oracle.check(text, b, cap=1 << 20)
        k, r = _jit_check(text, b)
        _same(r, o)
        assert r.n_oob == o.n_oob and (o.n_oob > 0) == (block[0] * block[1] > 56)
        _same(k.check(cap=1 << 20, flags=hg.JIT | hg.NO_SPLIT), o)
        assert r == k.check(cap=1 << 20, flags=hg.NO_JIT | hg.NO_SMALL)
        r3 = k.check(cap=1 << 20, flags=hg.JIT, only_accesses=0b001100)
        assert r3.witnesses == [x for x in o.witnesses if x[3] in (2, 3) and x[4] in (2, 3)]


@pytest.mark.parametrize("seed", range(8))
def test_jit_with_cell_filter(seed):
    w = workloads.random_shared(5100 + seed)
    o = oracle.check(w.text, w.binding, cap=1 << 20)
    for extra in (hg.CELL_FILTER, hg.CELL_FILTER | hg.NO_SPLIT):
        k, r = _jit_check(w.text, w.binding, flags=extra)
        assert hg.stats()["cell_filter"] == 1
        _same(r, o)
