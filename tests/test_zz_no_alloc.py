"""hgrd_check_noalloc: the check on the library's built-in device scratch.

That entry point serves callers that cannot allocate device memory (another
component owns all of it, or allocation is not allowed where they run).  It
is called here through the C ABI and compared with hgrd_check, which runs on
a caller-allocated workspace, on consecutive calls.  The check is exact
integer work, so the results must be identical, also after the shared scratch
has held another descriptor's data.  This file sorts last, so a failure here
comes after every other test has run.
"""
import pytest

import paper_2604_02106_b300 as hg
import workloads

pytestmark = pytest.mark.gpu


def _no_pair(r):
    return (r.racy, r.n_witness, r.n_by_kind, r.n_instances, r.n_keys, r.n_oob, r.witnesses, r.min_w, r.truncated)


def _kernel(w):
    return hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)


def test_noalloc_matches_workspace_check_on_consecutive_calls():
    a = _kernel(workloads.config1(0))
    b = _kernel(workloads.config2(0, planted=True, W=64, H=64, K=4))
    want_a = a.check(cap=1 << 20)
    want_b = b.check(cap=1 << 20)
    assert want_a.racy and want_b.n_witness == 63
    for k, want in ((a, want_a), (a, want_a), (b, want_b), (a, want_a)):
        got = k.check_noalloc(cap=1 << 20)
        assert _no_pair(got) == _no_pair(want)
    # truncation behaves as in hgrd_check
    got = a.check_noalloc(cap=5)
    assert got.truncated and got.witnesses == want_a.witnesses[:5] and got.n_witness == want_a.n_witness


def test_noalloc_rejects_bindings_beyond_its_scratch():
    big = _kernel(workloads.config2(0, planted=True))  # needs about 9 GB of workspace
    with pytest.raises(hg.HgrdError) as ei:
        big.check_noalloc(cap=16)
    assert ei.value.code == -6 and "built-in array" in str(ei.value)
