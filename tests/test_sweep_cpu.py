"""Host side of the symbolic-parameter mode: the bounds asserts put on single
parameters, the candidate values, and the bound-program hash."""
import pytest

import paper_2604_02106_b300 as hg
from paper_2604_02106_b300 import sweep

TEXT = ("kernel k\nparam N STRIDE M Q R\narray a global 4*(N*STRIDE+8)\n"
        "assert N > 0\nassert 2*N <= 8192\nassert STRIDE >= 1\nassert STRIDE < 64\nassert gdx*bdx >= N\n"
        "assert -M >= -100\nassert M*M < 100\nassert Q / 2 < 3\nassert 3 - R == 1\n"
        "access W a ; width 4 ; idx (bx*bdx+tx)*STRIDE\n")


def test_bounds_from_single_parameter_asserts():
    ps = {p.name: (p.lo, p.hi) for p in sweep.params(TEXT)}
    assert ps["N"] == (1, 4096)           # N > 0, 2N <= 8192
    assert ps["STRIDE"] == (1, 63)        # strict upper bound
    assert ps["M"] == (None, 100)         # negative coefficient flips the side
    assert ps["Q"] == (None, None)        # division and products of parameters are not bounds
    assert ps["R"] == (2, 2)              # equality
    assert list(ps) == ["N", "STRIDE", "M", "Q", "R"]


def test_rounding_of_bounds():
    t = "kernel k\nparam A B\nassert 3*A < 10\nassert 4*B >= 9\nassert -2*A > -9\n"
    ps = {p.name: (p.lo, p.hi) for p in sweep.params(t)}
    assert ps["A"] == (None, 3)           # 3A <= 9 -> A <= 3; -2A >= -8 -> A <= 4
    assert ps["B"] == (3, None)           # 4B >= 9 -> B >= ceil(9/4)


def test_candidate_values():
    assert sweep.candidate_values(sweep.Param("N", 1, 4096)) == [1, 2, 4, 8, 16, 32, 4095, 4096]
    assert sweep.candidate_values(sweep.Param("R", 2, 2)) == [2]
    assert sweep.candidate_values(sweep.Param("E", 5, 4)) == []
    v = sweep.candidate_values(sweep.Param("F", 10, 13), per_param=8)
    assert v == [10, 11, 12, 13]
    v = sweep.candidate_values(sweep.Param("G", None, None), free=(3, 20), per_param=6)
    assert v[0] == 3 and v[-1] == 20 and len(v) == 6 and v == sorted(set(v))


def test_bound_hash_separates_programs():
    t = "kernel k\nparam N S\narray a global 4096\naccess W a ; width 4 ; idx (tx * S) % 64 + N - N\n"
    def h(grid, block, params):
        return sweep.bound_hash(hg.Kernel(t).bind(grid, block, params))
    a = h((2, 1, 1), (64, 1, 1), (7, 3))
    assert a == h((2, 1, 1), (64, 1, 1), (7, 3))
    assert a == h((2, 1, 1), (64, 1, 1), (9, 3))   # N folds away: the same program
    assert a != h((2, 1, 1), (64, 1, 1), (7, 5))
    assert a != h((4, 1, 1), (64, 1, 1), (7, 3))
