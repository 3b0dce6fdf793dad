"""Host-side tests of the C ABI (no GPU): the library loads, exports every
symbol include/hgrd.h declares, and its parser / binder / division method
behave as documented."""
import os
import random
import re

import pytest

import paper_2604_02106_b300 as hg
import workloads
from workloads import Binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "hgrd.h")).read()
    declared = set(re.findall(r"\b(hgrd_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    L = hg.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(hg.EXPORTS)


def _err(text, grid=(1, 1, 1), block=(32, 1, 1), params=()):
    with pytest.raises(hg.HgrdError) as ei:
        hg.Kernel(text).bind(grid, block, params)
    return ei.value.code


def test_parse_errors():
    base = "kernel k\narray a global 64\n"
    assert _err(base + "access W a ; width 4 ; idx tx*ty\n") == -2          # not quasi-affine
    assert _err(base + "access W a ; width 4 ; idx 4 / tx\n") == -2         # divisor varies
    assert _err(base + "access W a ; width 4 ; idx q\n") == -2              # unknown name
    assert _err(base + "access W b ; width 4 ; idx 0\n") == -2              # unknown array
    assert _err(base + "access W a ; width 4 ; iv tx ; idx 0\n") == -2      # interval uses tid
    assert _err("kernel k\narray a global 64 ; granule 8\naccess W a ; width 4 ; idx 0\n") == -2  # width vs granule
    assert _err("array a global 4\n") == -2                                  # no kernel line
    assert _err(base + "access W a ; width 4 ; idx 0 ; if tx != 3\n") == -2  # != only in asserts


def test_bind_errors_match_host_classes():
    t = "kernel k\nparam Q\narray a global 4*Q\nassert Q > 2\naccess W a ; width 4 ; idx tx / Q\n"
    assert _err(t, params=()) == -3               # parameter count
    assert _err(t, params=(2,)) == -4             # host assert (class 1)
    assert _err(t, block=(0, 1, 1), params=(3,)) == -3
    assert _err(t, block=(64, 32, 1), params=(3,)) == -3   # > 1024 threads
    t2 = "kernel k\nparam Q\narray a global 64\naccess W a ; width 4 ; idx tx % Q\n"
    assert _err(t2, params=(0,)) == -3            # divisor <= 0
    t3 = "kernel k\nparam Q\narray a global 64\naccess W a ; width 4 ; idx tx * Q\n"
    assert _err(t3, params=(1 << 62,)) == -5      # int64 overflow
    hg.Kernel(t3).bind((1, 1, 1), (32, 1, 1), (3,))


def test_paper_fixtures_bind_like_the_oracle():
    import json
    gold = os.path.join(ROOT, "tests", "golden")
    for name in sorted(n for n in os.listdir(gold) if n.startswith("fig")):
        g = json.load(open(os.path.join(gold, name)))
        for case in g["cases"]:
            text = g["descriptor"] if case.get("assert", True) else g["descriptor_without_assert"]
            k = hg.Kernel(text)
            if case["expect"] == "EHOSTCONSTRAINT":
                with pytest.raises(hg.HgrdError) as ei:
                    k.bind(case["grid"], case["block"], case["params"])
                assert ei.value.code == -4
            else:
                k.bind(case["grid"], case["block"], case["params"])


def test_division_by_constant_method():
    # Granlund-Montgomery with C truncation, both widths, against exact integer division
    rnd = random.Random(7)
    def ref(n, d):
        q = abs(n) // d
        q = q if n >= 0 else -q
        return q, n - q * d
    for wide, N in ((False, 31), (True, 62)):
        ds = list(range(1, 200)) + [rnd.randrange(1, 1 << (N - 1)) for _ in range(200)] + [(1 << N) - 1, 1 << (N - 1)]
        for d in ds:
            ns = [0, 1, -1, d, -d, d - 1, 1 - d, (1 << N) - 1, 1 - (1 << N)] + \
                 [rnd.randrange(-(1 << N) + 1, 1 << N) for _ in range(20)]
            for n in ns:
                assert hg.debug_divmod(n, d, wide) == ref(n, d), (n, d, wide)


def test_workspace_scales_with_problem():
    w = workloads.config2(0)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    ws = k.workspace_size()
    # two 8-byte key buffers dominate, for the kept keys of the one global
    # write: the reads of the read-only input race with nothing, the ten
    # reads of the tile share no barrier interval with a write, the tile's
    # two staging writes cover the byte ranges [0, 1024) and [1024, 1296),
    # which never meet, and each maps distinct threads to distinct elements,
    # as does the centre write, so no shared-memory key is kept
    out_keys = 64 * 64 * 256 * 32
    shared_kept = 0
    keys = out_keys
    # (+ four raw-witness buffers of at most 2^24 words and small tables); the
    # cell filter adds 4 bytes per cell (3.4M cells)
    cells = 2 * 1024 * 1024 + 4096 * 324
    base = k.workspace_size(flags=hg.NO_CELL_FILTER)
    assert 16 * keys <= base < 16 * keys + 4 * 8 * (1 << 24) + (200 << 20)
    assert base + 4 * cells <= ws < base + 4 * cells + (1 << 20)
    # one global sort of every kept key needs buffers for all of them
    assert k.workspace_size(flags=hg.NO_SPLIT) >= 16 * (out_keys + shared_kept)
    # room for candidate shared-memory bins: all kept shared keys up to 2^24,
    # a sixteenth of them beyond, or a caller-given room
    text = ("kernel t\narray S shared 1024\naccess W S ; width 4 ; idx tx\n"
            "access R S ; width 4 ; idx (tx + 1) % 256\n")
    ks = hg.Kernel(text).bind((4096, 1, 1), (256, 1, 1), ())
    kept = 2 * 4096 * 256
    assert ks.workspace_size(flags=hg.NO_SPLIT) >= 16 * kept
    assert 16 * kept <= ks.workspace_size(flags=hg.NO_CELL_FILTER) < 16 * kept + 4 * 8 * (1 << 24) + (200 << 20)
    assert ks.workspace_size(max_shared_keys=1 << 10) < ks.workspace_size()


def test_acquire_release_guards_bind():
    # acquire-release guards (Sec. 6.5): decided at bind time when both guards
    # of a pair on one lock array are constant, or both the access's own index
    # (equal widths); decided per instance pair by the exact scan when each
    # guard element is constant, affine in thread and block ids, or the
    # access's own index; other forms guarding a pair are rejected (a loop
    # counter, or a division or remainder that is not the access's own
    # index); a guard without a guarded partner is fine; a lock array must be
    # global
    base = "kernel k\nloop i 2\narray d global 256\narray L global 64\narray S shared 64\n"
    ok = [("access W d ; width 4 ; idx 0 ; sync L 0", "access R d ; width 4 ; idx 0 ; sync L 1"),
          ("access W d ; width 4 ; idx tx % 4 ; sync L tx % 4", "access R d ; width 4 ; idx tx / 8 ; sync L tx / 8"),
          ("access R d ; width 4 ; idx 0 ; sync L tx", "access W d ; width 4 ; idx 0"),
          ("access W d ; width 4 ; idx 3 ; sync L 3", "access R d ; width 4 ; idx tx ; sync L tx"),
          ("access W d ; width 4 ; idx 0 ; sync L tx", "access R d ; width 4 ; idx 0"),
          ("access W d ; width 4 ; idx 0 ; sync L tx", "access R d ; width 4 ; idx 0 ; sync L 0"),
          ("access W d ; width 8 ; idx tx ; sync L tx", "access R d ; width 4 ; idx tx ; sync L tx"),
          ("access W d ; width 4 ; idx tx % 4 ; sync L tx % 4", "access R d ; width 4 ; idx 0 ; sync L bx + 2")]
    for a, b in ok:
        hg.Kernel(base + a + "\n" + b + "\n").bind((2, 1, 1), (32, 1, 1), ())
    bad = [("access W d ; width 4 ; idx tx % 4 ; sync L tx % 2", "access R d ; width 4 ; idx 0"),
           ("access W d ; width 4 ; idx 0 ; sync L i", "access R d ; width 4 ; idx 0 ; sync L 0"),
           ("access W d ; width 4 ; idx 0 ; sync L tx / 2", "access R d ; width 4 ; idx 0")]
    for a, b in bad:
        assert _err(base + a + "\n" + b + "\n", grid=(2, 1, 1)) == -9
    assert _err(base + "access W d ; width 4 ; idx 0 ; sync S 0\n") == -2   # shared lock array
    assert _err(base + "access W d ; width 4 ; idx 0 ; sync M 0\n") == -2   # unknown array
    assert _err(base + "access W d ; width 4 ; idx 0 ; sync L 0 ; syncscope grid\n") == -2


def test_acquire_release_pairs_leave_the_pair_rule():
    # both guarded at one device-scope lock: the pair is no longer eligible;
    # block scope keeps it for the inter-block kind only
    from paper_2604_02106_b300 import ranker
    base = "kernel k\narray c global 4\narray L global 64\n"
    for scope, want in (("device", []), ("block", [(0, 1), (1, 1)])):
        t = (base + f"access R c ; width 4 ; idx 0 ; sync L 0 ; syncscope {scope}\n"
             f"access W c ; width 4 ; idx 0 ; sync L 0 ; syncscope {scope}\n")
        k = hg.Kernel(t).bind((2, 1, 1), (64, 1, 1), ())
        assert ranker.pair_features(k)[1] == want
