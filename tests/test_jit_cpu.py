"""Specialised expansion kernels: the generated source compiles for sm_103a.

Without a GPU the compile runs in full and only loading the module fails, so
the error must come from the loader and not from the run-time compiler.  The
source depends on the program's structure only: bindings that differ in
values share one module.
"""
import pytest

import paper_2604_02106_b300 as hg
import workloads


def _compiles(k, **opts):
    try:
        k.jit_compile(**opts)
    except hg.HgrdError as e:
        msg = str(e)
        assert "nvrtcCompileProgram" not in msg and "cudaLibraryLoadData" in msg, msg[:2000]


def _bind(w):
    return hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)


@pytest.mark.parametrize("make", [
    lambda: workloads.config2(0, planted=True, W=64, H=64, K=4),
    lambda: workloads.config1(0),
    lambda: workloads.random_shared(5003),
    lambda: workloads.random_tiny(1007, max_instances=500),
    lambda: workloads.random_warp(3003),
    lambda: workloads.warp_exchange(4, 3, "warp2", False, grid=2, space="global"),
])
def test_generated_source_compiles(make):
    k = _bind(make())
    _compiles(k)
    _compiles(k, flags=hg.NO_SPLIT)


def test_source_depends_on_structure_only():
    # one sweep's items (N, block size) on one pipeline share their source
    # (items of one block excepted: with no second block nothing races across
    # blocks, which the pair rule, and so the source, records)
    items = [w for w in workloads.config3() if w.meta["stride"] == 3 and w.binding.grid[0] > 1]
    srcs = {_bind(w).jit_source(flags=hg.NO_SPLIT) for w in items[:4]}
    assert len(srcs) == 1
    a = _bind(workloads.config2(0, planted=True, W=64, H=64, K=4))
    b = _bind(workloads.config2(0, planted=True, W=128, H=128, K=8))
    assert a.jit_source() == b.jit_source()
    # no shared-memory key of the stencil is written (the tile's accesses race
    # with nothing), so it takes no block-local bins; a kernel with racing
    # shared accesses does
    assert a.jit_source() == a.jit_source(flags=hg.NO_SPLIT)
    r = _bind(workloads.random_shared(5000))
    assert r.jit_source() != r.jit_source(flags=hg.NO_SPLIT)
    # without the planted stride every thread writes its own output element:
    # the write races with nothing (thread-tile pruning), so its keys are
    # never written and the source says so
    c = _bind(workloads.config2(0, planted=False, W=128, H=128, K=8))
    assert c.jit_source() != b.jit_source()


def test_generated_source_covers_every_live_access():
    w = workloads.config2(0, planted=True, W=64, H=64, K=4)
    src = _bind(w).jit_source()
    for a in range(16):
        assert f"// access {a}\n" in src
    # no shared key is written: the plain count and write passes, no block-local ones
    assert "hgrd_jit_expand0" in src and "hgrd_jit_expand1" in src and "hgrd_jit_expand3" not in src
    r = _bind(workloads.random_shared(5000)).jit_source()
    assert "hgrd_jit_expand3" in r and "hgrd_jit_expand4" in r and "hgrd_jit_expand0" not in r


def test_warp_intervals_reach_the_key():
    # a program with warp-barrier intervals packs them next to the interval
    k = _bind(workloads.warp_exchange(4, 3, "warp2", False, grid=2))
    assert "pack_wv(" in k.jit_source()
    k0 = _bind(workloads.warp_exchange(4, 3, "none", False, grid=2))
    assert "pack_wv(" not in k0.jit_source()
