"""Symbolic-parameter mode: a race under some host-admissible input, decided
over generated admissible bindings on the batched path.  Every distinct
binding's verdict must equal the oracle's."""
import pytest

import oracle
import workloads
from paper_2604_02106_b300 import sweep
from workloads import Binding

pytestmark = pytest.mark.gpu


def _same_verdict(v, o, cap):
    assert v.racy == o.racy and v.n_witness == o.n_witness and v.n_by_kind == o.n_by_kind
    assert v.n_keys == o.n_keys and v.n_oob == o.n_oob and v.n_instances == o.n_instances
    assert v.witnesses == o.witnesses[:cap]


def test_strided_kernel_races_for_short_strides():
    text = workloads.config3_kernel_text()
    r = sweep.symbolic_check(text, lambda p: ((-(-p["N"] // 128), 1, 1), (128, 1, 1)),
                             values={"N": [256, 1000, 2048]}, free=(1, 40), per_param=6)
    assert r.admissible == 3 * 6 and r.rejected == 0
    assert r.racy
    seen = set()
    for (grid, block, p), v in zip(r.bindings, r.verdicts):
        assert v.racy == (p["STRIDE"] < 8)
        key = (grid, block, p["N"], p["STRIDE"])
        if key in seen:
            continue
        seen.add(key)
        o = oracle.check(text, Binding(grid, block, (p["N"], p["STRIDE"])))
        _same_verdict(v, o, 16)
    # racy and clean bindings fall into different verdict signatures
    assert len(r.groups) >= 2
    assert all(r.verdicts[i].racy == sig[0] for sig, idx in r.groups.items() for i in idx)


def test_asserts_reject_inadmissible_launches_and_equal_programs_run_once():
    # the stencil ties the grid to the image size: only matching launches are admissible;
    # R below W makes output rows overlap
    text = workloads.config2(0, planted=False, W=64, H=64, K=2).text
    shapes = [((4, 4, 1), (16, 16, 1)), ((8, 8, 1), (16, 16, 1))]
    r = sweep.symbolic_check(text, shapes, values={"W": [64, 128], "H": [64], "R": [63, 64, 65]})
    assert r.admissible == 3 and r.rejected == 2 * 2 * 3 - 3
    assert [p["R"] < p["W"] for _, _, p in r.bindings] == [v.racy for v in r.verdicts]
    assert r.racy and r.first_racy[0][2]["R"] == 63
    for (grid, block, p), v in zip(r.bindings, r.verdicts):
        o = oracle.check(text, Binding(grid, block, (p["W"], p["H"], p["R"])))
        _same_verdict(v, o, 16)
    # a parameter that folds away gives one program for all its values
    t2 = "kernel k\nparam N S\narray a global 4096\naccess W a ; width 4 ; idx (tx * S) % 64 + N - N\n"
    r2 = sweep.symbolic_check(t2, ((2, 1, 1), (64, 1, 1)), values={"N": [1, 2, 3, 4], "S": [1, 2]})
    assert r2.admissible == 8 and r2.distinct == 2
