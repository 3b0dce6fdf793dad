"""The conflict scan's first phase on long runs, through the C ABI.

Runs longer than 2^16 keys leave the first phase with their end unknown and
the exact scan finds it; a warp finishes the run open at the end of its range
past that range.  These kernels put one long run of writes to one address
after many one-key runs (reads of a thread's own element), so the long run
starts inside a range and crosses many, and compare both forms of the first
phase (lane rows, and 32-key warp steps with HGRD_SCAN_BALLOT) with the
closed form: the single written address is the only racing location, its
write races with itself in all three kinds.  The oracle checks the same
kernels at sizes where its pairwise check of one location stays small.
"""
import pytest

import oracle
import paper_2604_02106_b300 as hg
from workloads import Binding

pytestmark = pytest.mark.gpu

BD = 512  # threads per block


def _kernel(n_reads, n_writers, tail):
    """n_reads threads read their own element of `a`, n_writers threads write
    b[0]; with `tail`, every thread then reads its own element of `c`."""
    text = (f"kernel longrun\narray a global {4 * n_reads + 4}\narray b global 16\n"
            + (f"array c global {4 * (n_reads + n_writers) + 4}\n" if tail else "")
            + f"access R a ; width 4 ; idx bx*{BD} + tx ; if bx*{BD} + tx < {n_reads}\n"
            + f"access W b ; width 4 ; idx 0 ; if bx*{BD} + tx < {n_writers}\n")
    if tail:
        text += "access R c ; width 4 ; idx bx*512 + tx\n"
    nthr = max(n_reads, n_writers)
    grid = (nthr + BD - 1) // BD
    return text, Binding((grid, 1, 1), (BD, 1, 1), ())


def _closed_form(g, n_reads, n_writers, tail, grid):
    assert g.racy
    assert g.n_witness == 1
    w = g.witnesses[0]
    assert w[:5] == (0, 1, 0, 1, 1)  # global, array b, byte 0, the write with itself
    kinds = (1 if n_writers > BD else 0) | (2 if n_writers > 32 else 0) | (4 if n_writers > 1 else 0)
    assert w[5] == kinds
    assert g.n_instances == grid * BD * (3 if tail else 2)
    assert g.n_keys == n_reads + n_writers + (grid * BD if tail else 0)
    assert g.n_oob == 0


FORMS = [0, hg.SCAN_BALLOT, hg.ALL_KEYS | hg.NO_CELL_FILTER, hg.ALL_KEYS | hg.NO_CELL_FILTER | hg.SCAN_BALLOT]


@pytest.mark.parametrize("n_reads,n_writers,tail", [
    (131000, 100000, False),   # the long run (over 2^16 keys) ends the array
    (131000, 100000, True),    # ... and is followed by 231,424 one-key runs
    (70001, 65600, True),      # just over 2^16 keys
    (70001, 65000, True),      # just under: closed where it ends, past its range
    (99999, 5000, False),      # the array ends inside a warp's last run
])
def test_long_run_closed_form(n_reads, n_writers, tail):
    text, b = _kernel(n_reads, n_writers, tail)
    res = [hg.check(text, b, cap=64, flags=f | hg.NO_PAIR) for f in FORMS]
    for g in res:
        _closed_form(g, n_reads, n_writers, tail, b.grid[0])
    assert all(g == res[0] for g in res[1:])


@pytest.mark.parametrize("n_reads,n_writers,tail", [(3001, 1500, True), (5000, 700, False), (1025, 1024, True)])
def test_long_run_shape_against_oracle(n_reads, n_writers, tail):
    # the same kernels at sizes the oracle checks pair by pair
    text, b = _kernel(n_reads, n_writers, tail)
    o = oracle.check(text, b, cap=64)
    _closed_form(o, n_reads, n_writers, tail, b.grid[0])
    for f in FORMS:
        g = hg.check(text, b, cap=64, flags=f | hg.NO_SMALL)
        assert g.witnesses == o.witnesses and g.n_by_kind == o.n_by_kind and g.n_keys == o.n_keys
        assert g.min_x == o.min_x and g.min_y == o.min_y
