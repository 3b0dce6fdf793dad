"""hgrd_check_noalloc: the check on the library's built-in device scratch.

That entry point serves callers that cannot allocate device memory: code that
runs while another component (a caching allocator, a memory pool) owns all of
it, code called from inside such an allocator, and embedders with no access
to cudaMalloc.  It is called here through the C ABI on consecutive calls and
compared with the CPU oracle and with hgrd_check on a caller workspace.  The
check is exact integer work, so the results must be identical, also after the
shared scratch has held another descriptor's data.  The library's count of
CUDA objects it created (streams, events, graphs, pinned buffers, modules)
must not move across these calls, the first one included.  This file sorts
last, so a failure here comes after every other test has run; it also passes
alone in a fresh process.
"""
import pytest

import oracle
import paper_2604_02106_b300 as hg
import workloads

pytestmark = pytest.mark.gpu


def _fields(r):
    return (r.racy, r.n_witness, r.n_by_kind, r.n_instances, r.n_keys, r.n_oob, r.witnesses, r.min_w, r.truncated)


def _oracle_pairs(o):
    out = {}
    for w in o.witnesses:
        out[(w[3], w[4])] = out.get((w[3], w[4]), 0) | w[5]
    return out


def _kernel(w):
    return hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)


def _created():
    return hg.stats()["cuda_objects_created"]


def test_noalloc_matches_oracle_and_workspace_check_on_consecutive_calls():
    wa = workloads.plain_random(0)
    wb = workloads.config2(0, planted=True, W=64, H=64, K=4)
    a, b = _kernel(wa), _kernel(wb)
    before = _created()
    # the first calls of this process on this device come first: they look
    # up the scratch address and must not create anything either
    got_a0 = a.check_noalloc(cap=1 << 20)
    got_b0 = b.check_noalloc(cap=1 << 20)
    assert _created() == before
    oa = oracle.check(wa.text, wa.binding, cap=1 << 20)
    ob = oracle.check(wb.text, wb.binding, cap=1 << 20)
    assert oa.racy and ob.n_witness == 63
    for got, o in ((got_a0, oa), (got_b0, ob)):
        assert got.witnesses == o.witnesses
        assert (got.n_witness, got.n_by_kind, got.n_instances, got.n_keys, got.n_oob) == \
               (o.n_witness, o.n_by_kind, o.n_instances, o.n_keys, o.n_oob)
        assert got.min_w == o.min_w and got.racy == o.racy
        assert got.pairs == _oracle_pairs(o)
    # the same on a caller workspace (hgrd_check), then alternating calls
    want_a = a.check(cap=1 << 20)
    want_b = b.check(cap=1 << 20)
    for want in (want_a, want_b):
        assert want.pairs
    before = _created()
    for k, want in ((a, want_a), (a, want_a), (b, want_b), (a, want_a), (b, want_b)):
        got = k.check_noalloc(cap=1 << 20)
        assert _fields(got) == _fields(want)
        assert got.pairs == want.pairs
    assert _created() == before
    # truncation behaves as in hgrd_check
    got = a.check_noalloc(cap=5)
    assert got.truncated and got.witnesses == want_a.witnesses[:5] and got.n_witness == want_a.n_witness
    assert _created() == before


def test_noalloc_rejects_bindings_beyond_its_scratch():
    big = _kernel(workloads.config2(0, planted=True))  # needs over 1 GB of workspace
    with pytest.raises(hg.HgrdError) as ei:
        big.check_noalloc(cap=16)
    assert ei.value.code == -6 and "built-in array" in str(ei.value)


def test_noalloc_refuses_a_capturing_stream():
    import torch
    k = _kernel(workloads.config1(0))
    k.check_noalloc(cap=16)  # the scratch address is known before the capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            k.check_noalloc(cap=16, stream=s)
        except hg.HgrdError as e:
            err = e
        finally:
            g.capture_end()
    assert err is not None and err.code == -1 and "capturing" in str(err)
