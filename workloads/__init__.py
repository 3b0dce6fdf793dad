"""Seeded synthetic inputs for the host-guided race check.

This module only *writes inputs*: kernel descriptors in the text format below
plus the host-side binding (grid, block, parameter values) a launch supplies.
It holds none of the checking arithmetic, so both the CPU oracle and the GPU
path can consume what it produces without sharing any of the method.

Descriptor text format (one directive per line, ``#`` starts a comment,
fields of ``array`` and ``access`` lines are separated by ``;``)::

    kernel NAME
    param P1 P2 ...                  kernel parameters, bound in this order
    loop VAR BOUND                   0 <= VAR < BOUND, outermost first, at most 4
    array NAME global|shared BYTES [; granule G]
    let NAME = EXPR                  textual macro over everything declared
    access R|W|A ARRAY ; width W [; iv EXPR] [; wv EXPR] ; idx EXPR [; if COND]* [; scope block|device]
           [; sync LOCKARRAY EXPR [; syncscope block|device]] [; line N]
    assert COND                      host-code fact over params and launch dims

Expressions use + - * / % (C semantics: division truncates toward zero),
unary minus, parentheses, integer literals and the names tx ty tz bx by bz
(threadIdx/blockIdx), bdx bdy bdz gdx gdy gdz (blockDim/gridDim), loop
variables, params and lets.  COND is ``EXPR op EXPR`` with op one of
``< <= > >= ==`` (and ``!=`` in asserts only).  ``idx`` is an element index
in units of the access width (C pointer arithmetic on a typed pointer), ``iv``
is the barrier-interval id (affine in loop variables), ``wv`` the warp-barrier
interval id, R/W/A = read, write, atomic.  ``sync`` names the acquire-release
guard of the access (a lock held around it, or a producer's release / a
consumer's acquire): the global array and element of its address;
``syncscope`` is the narrower scope of the guard's parts (default device).

The workload shapes follow the five benchmark configurations of this project
(plain 4x64 check, tiled 64x64x(16x16) stencil, 64-tuple host sweep,
10,000-kernel corpus, ranker corpus) and the paper's Fig. 1-5 listings.
Seeds are ``0x4847524400 + config*10000 + item``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

MASK64 = (1 << 64) - 1
SEED_BASE = 0x4847524400


def seed_for(config: int, item: int) -> int:
    return SEED_BASE + config * 10000 + item


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as published by Vigna."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) (rejection-free multiply-high)."""
        return (self.next() * n) >> 64

    def range(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def choice(self, seq):
        return seq[self.below(len(seq))]


@dataclass
class Binding:
    grid: tuple = (1, 1, 1)
    block: tuple = (1, 1, 1)
    params: tuple = ()

    def instances_per_access(self, loop_bounds) -> int:
        n = math.prod(self.grid) * math.prod(self.block)
        for b in loop_bounds:
            n *= max(0, b)
        return n


@dataclass
class Workload:
    name: str
    text: str
    binding: Binding
    meta: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# helpers to write descriptor text

class _Writer:
    def __init__(self, name):
        self.lines = [f"kernel {name}"]

    def add(self, line):
        self.lines.append(line)

    def access(self, kind, array, width, idx, iv=None, guards=(), scope=None, line=None, wv=None, sync=None,
               syncscope=None):
        f = [f"access {kind} {array}", f"width {width}"]
        if iv is not None:
            f.append(f"iv {iv}")
        if wv is not None:
            f.append(f"wv {wv}")
        f.append(f"idx {idx}")
        for g in guards:
            f.append(f"if {g}")
        if scope is not None:
            f.append(f"scope {scope}")
        if sync is not None:
            f.append(f"sync {sync}")
        if syncscope is not None:
            f.append(f"syncscope {syncscope}")
        if line is not None:
            f.append(f"line {line}")
        self.lines.append(" ; ".join(f))

    def text(self):
        return "\n".join(self.lines) + "\n"


def _lin(a, v):
    """Render coefficient*variable with sign handling."""
    if a == 0:
        return ""
    if a == 1:
        return f" + {v}"
    if a == -1:
        return f" - {v}"
    if a < 0:
        return f" - {-a}*{v}"
    return f" + {a}*{v}"


# --------------------------------------------------------------------------
# Config 1: plain check of one small kernel.
#   1D grid of 4 blocks x 64 threads, S = 256 int32 shared, G = 4096 int32
#   global, 6 accesses idx = a*tx + b*bx + c*i + d*N + e with a,b,c,d drawn
#   in [-4, 4], N = 64 bound by the host, loop i < 8, barrier intervals
#   {0,1,2}.  The offset e makes the smallest index of the access zero.  The
#   five drawn accesses are race free by construction:
#     * G is read only (reads never race with reads);
#     * in a barrier interval where S is written, every S access of that
#       interval uses one index expression with a nonzero thread coefficient
#       and no loop term, so each thread owns its slot (shared memory races
#       only inside a block, and a block's threads then never share a slot);
#     * S accesses in intervals without an S write are reads, drawn freely.
#   The sixth access is the planted race: thread 0 of every block writes one
#   G element (the shape of the paper's reduceFinal, Fig. 2) at index 1024 or
#   more, beyond every read of G (the largest read index is 4*63 + 4*3 + 4*7),
#   so the kernel has exactly one racy access pair, (5, 5), inter-block.

def _c1_expr(a, b, c, d, N, TB, GB, ITER):
    lo = min(0, a * (TB - 1)) + min(0, b * (GB - 1)) + min(0, c * (ITER - 1)) + d * N
    e = -lo
    expr = "0" + _lin(a, "tx") + _lin(b, "bx") + _lin(c, "i") + _lin(d, "N")
    return expr + (f" + {e}" if e >= 0 else f" - {-e}")


def config1(item: int = 0) -> Workload:
    rng = SplitMix64(seed_for(1, item) ^ 0xC1)
    N, TB, GB, ITER = 64, 64, 4, 8
    w = _Writer(f"plain_c1_{item}")
    w.add("param N")
    w.add("loop i 8")
    w.add("array S shared 1024")
    w.add("array G global 16384")
    draws = []
    for _ in range(5):
        arr = "S" if rng.below(2) == 0 else "G"
        kind = "W" if arr == "S" and rng.below(2) == 0 else "R"
        draws.append((arr, kind, rng.below(3)))
    slot = {}  # barrier interval with an S write -> the thread-owned index expression
    for arr, kind, iv in draws:
        if arr == "S" and kind == "W" and iv not in slot:
            a = rng.range(1, 4) * (1 if rng.below(2) else -1)
            b, d = rng.range(-4, 4), rng.range(-4, 4)
            slot[iv] = _c1_expr(a, b, 0, d, N, TB, GB, ITER)
    for a_id, (arr, kind, iv) in enumerate(draws):
        if arr == "S" and iv in slot:
            expr = slot[iv]
        else:
            expr = _c1_expr(*(rng.range(-4, 4) for _ in range(4)), N, TB, GB, ITER)
        w.access(kind, arr, 4, expr, iv=iv, line=10 + a_id)
    d = rng.range(-4, 4)
    e = -d * N + 1024 + rng.below(64)
    w.access("W", "G", 4, f"{d}*N + {e}", iv=rng.below(3), guards=["tx == 0"], line=20)
    return Workload(f"c1_{item}", w.text(), Binding((GB, 1, 1), (TB, 1, 1), (N,)),
                    {"config": 1, "loop_bounds": [ITER], "n_access": 6})


def plain_random(item: int = 0) -> Workload:
    """The config-1 launch shape with five unconstrained random accesses
    (racy almost everywhere) plus the Fig. 2 write: many witnesses on few
    instances, for tests of truncation and buffer retries."""
    rng = SplitMix64(seed_for(1, item))
    N, TB, GB, ITER = 64, 64, 4, 8
    w = _Writer(f"plain_random_{item}")
    w.add("param N")
    w.add("loop i 8")
    w.add("array S shared 1024")
    w.add("array G global 16384")
    for a_id in range(5):
        arr = "S" if rng.below(2) == 0 else "G"
        kind = "R" if rng.below(2) == 0 else "W"
        a, b, c, d = (rng.range(-4, 4) for _ in range(4))
        w.access(kind, arr, 4, _c1_expr(a, b, c, d, N, TB, GB, ITER), iv=rng.below(3), line=10 + a_id)
    d = rng.range(-4, 4)
    e = -d * N + rng.below(64)
    w.access("W", "G", 4, f"{d}*N + {e}", iv=rng.below(3), guards=["tx == 0"], line=20)
    return Workload(f"pr_{item}", w.text(), Binding((GB, 1, 1), (TB, 1, 1), (N,)),
                    {"config": 1, "loop_bounds": [ITER], "n_access": 6})


# --------------------------------------------------------------------------
# Config 2: tiled-stencil shape.
#   2D grid (W/16) x (H/16) of 16x16 threads, an 18x18 fp32 shared tile with
#   a one-cell halo, In/Out W x H fp32 global arrays, loop k < 32 (a 32-row
#   running window of In, rows and columns wrapping with mod H / mod W), 16
#   accesses over 4 barrier intervals.  The planted off-by-one race is an Out
#   row stride R = W - 1: element (r, W-1) collides with (r+1, 0), which lie in
#   blocks bx = W/16 - 1 and bx = 0, giving W - 1 inter-block write-write
#   witnesses.  Whether item `item` is planted is decided by its seed.

def config2(item: int = 0, planted=None, W: int = 1024, H: int = 1024, K: int = 32) -> Workload:
    rng = SplitMix64(seed_for(2, item))
    bit = rng.next() & 1
    if planted is None:
        planted = bool(bit)
    R = W - 1 if planted else W
    w = _Writer(f"stencil2d_window_{item}")
    w.add("param W H R")
    w.add(f"loop k {K}")
    w.add("array S shared 1296")
    w.add("array In global 4*W*H")
    w.add("array Out global 4*W*H")
    w.add("let lin = ty*16 + tx")
    w.add("let l2 = lin + 256")
    w.add("assert gdx*16 == W")
    w.add("assert gdy*16 == H")
    w.add("assert bdx == 16")
    w.add("assert bdy == 16")
    # iv 0: stage the halo tile (324 cells, two per thread) from a k-shifted row
    w.access("R", "In", 4, "((by*16 - 1 + lin/18 + k + H) % H)*W + (bx*16 - 1 + lin%18 + W) % W", iv=0, line=11)
    w.access("W", "S", 4, "lin", iv=0, line=11)
    w.access("R", "In", 4, "((by*16 - 1 + l2/18 + k + H) % H)*W + (bx*16 - 1 + l2%18 + W) % W", iv=0,
             guards=["l2 < 324"], line=12)
    w.access("W", "S", 4, "l2", iv=0, guards=["l2 < 324"], line=12)
    # iv 1: 3x3 neighbourhood reads of the tile
    for dy in range(3):
        for dx in range(3):
            w.access("R", "S", 4, f"(ty + {dy})*18 + tx + {dx}", iv=1, line=15)
    # iv 2: centre update on the last window row
    w.access("W", "S", 4, "(ty + 1)*18 + tx + 1", iv=2, guards=[f"k == {K - 1}"], line=18)
    # iv 3: read back the centre and store the output pixel
    w.access("R", "S", 4, "(ty + 1)*18 + tx + 1", iv=3, guards=["k == 0"], line=21)
    w.access("W", "Out", 4, "(by*16 + ty)*R + bx*16 + tx", iv=3, guards=["k == 0"], line=21)
    return Workload(f"c2_{item}", w.text(), Binding((W // 16, H // 16, 1), (16, 16, 1), (W, H, R)),
                    {"config": 2, "planted": planted, "loop_bounds": [K], "n_access": 16,
                     "expected_witnesses": (W - 1) if planted else 0})


# --------------------------------------------------------------------------
# Config 3: host-guided parameter sweep of one 12-access strided kernel.
#   Thread g = bx*bdx + tx (guard g < N) writes A[g*STRIDE + i] for i < 8 and
#   reads it back; STRIDE < 8 makes neighbouring threads overlap (racy),
#   STRIDE >= 8 keeps them disjoint (clean).  The other arrays follow
#   race-free patterns.  64 tuples: N = 2^8..2^20 x STRIDE in {1,2,3,4,32},
#   N-major, the first 64; blockDim drawn from {64,...,1024}, grid = ceil(N/bd).

C3_STRIDES = (1, 2, 3, 4, 32)


def config3_kernel_text() -> str:
    w = _Writer("strided_sweep")
    w.add("param N STRIDE")
    w.add("loop i 8")
    w.add("array A global 4*(N*STRIDE + 8)")
    w.add("array B global 32*N")
    w.add("array C global 32*N")
    w.add("array T shared 4*bdx")
    w.add("let g = bx*bdx + tx")
    w.add("assert N > 0")
    w.add("assert STRIDE > 0")
    w.add("assert gdx*bdx >= N")
    w.add("assert (gdx - 1)*bdx < N")
    w.access("W", "A", 4, "g*STRIDE + i", iv=0, guards=["g < N"], line=5)        # 0
    w.access("R", "A", 4, "g*STRIDE + i", iv=1, guards=["g < N"], line=6)        # 1
    w.access("R", "B", 4, "g*8 + i", iv=0, guards=["g < N"], line=7)             # 2
    w.access("R", "B", 4, "((g + 1) % N)*8 + i", iv=0, guards=["g < N"], line=8)  # 3
    w.access("W", "C", 4, "g*8 + i", iv=0, guards=["g < N"], line=9)             # 4
    w.access("R", "C", 4, "g*8 + 7 - i", iv=2, guards=["g < N"], line=10)        # 5
    w.access("W", "T", 4, "tx", iv=0, line=11)                                    # 6
    w.access("R", "T", 4, "(tx + 1) % bdx", iv=1, line=12)                        # 7
    w.access("R", "T", 4, "(tx + bdx - 1) % bdx", iv=1, line=13)                  # 8
    w.access("W", "T", 4, "tx", iv=2, guards=["i == 7"], line=14)                 # 9
    w.access("A", "C", 4, "g*8", iv=3, guards=["g < N", "i == 0"], scope="device", line=15)  # 10
    w.access("R", "B", 16, "g*2 + i/4", iv=1, guards=["g < N"], line=16)         # 11
    return w.text()


def config3(n_items: int = 64):
    text = config3_kernel_text()
    items = []
    for e in range(8, 21):
        for s in C3_STRIDES:
            if len(items) == n_items:
                break
            rng = SplitMix64(seed_for(3, len(items)))
            N = 1 << e
            bd = 64 * (1 << rng.below(5))  # 64..1024
            grid = (N + bd - 1) // bd
            items.append(Workload(f"c3_{len(items)}", text, Binding((grid, 1, 1), (bd, 1, 1), (N, s)),
                                  {"config": 3, "N": N, "stride": s, "loop_bounds": [8], "n_access": 12}))
    return items


# --------------------------------------------------------------------------
# Paper listings (Fig. 1-5) as descriptors, used as fixtures in the tests.

def fig1_copy_upp_low(with_assert=True) -> str:
    w = _Writer("copyUppLowKernel")
    w.add("param rows cols")
    w.add("array A global 4*rows*cols")
    w.add("let i = bx*bdx + tx")
    w.add("let j = by*bdy + ty")
    if with_assert:
        w.add("assert rows == cols")
    w.access("R", "A", 4, "i*cols + j", guards=["j > i", "j < rows"], line=7)
    w.access("W", "A", 4, "j*cols + i", guards=["j > i", "j < rows"], line=7)
    return w.text()


def fig2_reduce_final() -> str:
    w = _Writer("reduceFinal")
    w.add("param n")
    w.add("array res global 4*n")
    w.access("W", "res", 4, "0", guards=["tx == 0"], line=5)
    return w.text()


def fig3_tone_mapping(with_assert=True) -> str:
    w = _Writer("toneMapping")
    w.add("param width channels height")
    w.add("array output global 4*width*channels*height")
    w.add("let x = bx*bdx + tx")
    w.add("let y = by*bdy + ty")
    if with_assert:
        # grid.x = hWidth/16 and width = hWidth come from the same host variable
        w.add("assert gdx == width / 16")
    w.access("W", "output", 4, "width*channels*y + x*channels", line=7)
    return w.text()


def fig4_lud_internal() -> str:
    w = _Writer("ludInternal")
    w.add("param dim offset BS")
    w.add("array m global 4*dim*dim")
    w.add("let rid = offset + (by + 1)*BS")
    w.add("let cid = offset + (bx + 1)*BS")
    w.add("assert offset >= 0")
    w.access("W", "m", 4, "(rid + ty)*dim + cid + tx", line=7)
    return w.text()


def fig5_shift(with_assert=True) -> str:
    w = _Writer("shift")
    w.add("param rowSize width height")
    w.add("array matrix global 4*width*height")
    w.add("array tex global 4*width*height")
    w.add("let xid = bx*bdx + tx")
    w.add("let yid = by*bdy + ty")
    if with_assert:
        # rowSize is the pitch cudaMallocPitch returned for this allocation
        w.add("assert rowSize > 0")
    w.access("R", "tex", 4, "yid*width + xid", line=6)
    w.access("W", "matrix", 4, "yid*(rowSize/4) + xid", line=6)
    return w.text()


# --------------------------------------------------------------------------
# Tiny random kernels (a few hundred to a few thousand instances) used to pin
# the oracle against pairwise brute force.

def random_tiny(seed: int, max_instances: int = 2048) -> Workload:
    rng = SplitMix64(seed)
    ndim_g = rng.range(1, 2)
    ndim_b = rng.range(1, 2)
    grid = [1, 1, 1]
    block = [1, 1, 1]
    for d in range(ndim_g):
        grid[d] = rng.range(1, 3)
    for d in range(ndim_b):
        block[d] = rng.choice([1, 2, 3, 5, 8, 16, 33, 40])
    while math.prod(block) > 1024:
        block[block.index(max(block))] //= 2
    nthreads = math.prod(block) * math.prod(grid)
    nloops = rng.range(0, 2)
    bounds = [rng.range(1, 3) for _ in range(nloops)]
    nacc = rng.range(1, 5)
    while nthreads * math.prod(bounds) * nacc > max_instances and nacc > 1:
        nacc -= 1
    while nthreads * math.prod(bounds) * nacc > max_instances and bounds:
        bounds.pop()
    while nthreads * math.prod(bounds) * nacc > max_instances and block[0] > 1:
        block[0] = max(1, block[0] // 2)
    w = _Writer(f"tiny_{seed & 0xffff}")
    P = rng.range(1, 9)
    Q = rng.range(1, 5)
    w.add("param P Q")
    lv = ["i", "j"][:len(bounds)]
    for v, b in zip(lv, bounds):
        w.add(f"loop {v} {b}")
    w.add(f"array S shared {4 * rng.range(4, 40)} ; granule 4")
    w.add(f"array G global {4 * rng.range(4, 64)}")
    if rng.below(2):
        w.add("array H global 64")
    names = ["tx", "ty", "bx", "by"] + lv + ["P", "Q"]
    for a_id in range(nacc):
        arr = rng.choice(["S", "G", "G"])
        r = rng.below(10)
        kind = "R" if r < 4 else ("W" if r < 8 else "A")
        expr = str(rng.range(0, 3))
        for v in names:
            if rng.below(3) == 0:
                expr += _lin(rng.range(-3, 3), v)
        if rng.below(4) == 0:
            expr = f"({expr}) / {rng.range(1, 3)}"
        if rng.below(5) == 0:
            expr = f"({expr}) % {rng.choice(['P', 'Q', '3', '5'])}"
        width = rng.choice([4, 4, 4, 8, 16]) if arr != "S" else 4
        guards = []
        if rng.below(3) == 0:
            v = rng.choice(names[:4] + lv)
            guards.append(f"{v} {rng.choice(['<', '<=', '>', '>=', '=='])} {rng.range(0, 3)}")
        iv = None
        if rng.below(2):
            iv = str(rng.range(0, 2))
            if lv and rng.below(3) == 0:
                iv = f"{iv} + {rng.choice(lv)}"
        scope = None
        if kind == "A":
            scope = rng.choice(["block", "device"])
        w.access(kind, arr, width, expr, iv=iv, guards=guards, scope=scope, line=a_id + 1)
    params = (P, Q)
    return Workload(f"tiny_{seed}", w.text(), Binding(tuple(grid), tuple(block), params),
                    {"loop_bounds": bounds, "n_access": nacc})


def random_sync(seed: int, max_instances: int = 1500, supported: bool = False) -> Workload:
    """Tiny kernel whose accesses may be guarded by acquire-release (Sec. 6.5):
    `sync L <element>` with a global lock (a constant element), a lock per
    data element (the access's own index), a lock per thread or per block, in
    block or device scope; one data array (global or shared), reads, writes
    and atomics, barrier intervals.  With `supported`, guards are only of the
    forms the exhaustive check decides statically: constant elements, or each
    access's own index (accesses of one width), one family per kernel."""
    rng = SplitMix64(seed)
    grid = (rng.range(1, 3), 1, 1)
    block = (rng.choice([2, 3, 8, 16, 33, 40]), rng.range(1, 2), 1)
    nacc = rng.range(2, 4)
    while math.prod(grid) * math.prod(block) * nacc > max_instances and block[0] > 2:
        block = (block[0] // 2, block[1], 1)
    space = rng.choice(["global", "global", "shared"])
    w = _Writer(f"sync_{seed & 0xffff}")
    w.add("param Q")
    w.add(f"array D {space} 256")
    w.add("array L global 64")
    # the decided forms: constants only, or own indexes only, per kernel
    forms = ["0", "1", "tx", "bx", "own"] if not supported else rng.choice([["0", "1"], ["own"]])
    for a_id in range(nacc):
        r = rng.below(10)
        kind = "R" if r < 4 else ("W" if r < 8 else "A")
        idx = rng.choice(["0", "tx % Q", "tx / 2", "(tx + bx) % 4", "tx", "3"])
        iv = str(rng.range(0, 1)) if rng.below(3) == 0 else None
        sync = syncscope = None
        if rng.below(3) != 0:
            f = rng.choice(forms)
            sync = "L " + (idx if f == "own" else f)
            syncscope = rng.choice(["block", "device", None])
        scope = rng.choice(["block", "device"]) if kind == "A" else None
        w.access(kind, "D", 4, idx, iv=iv, scope=scope, sync=sync, syncscope=syncscope, line=a_id + 1)
    return Workload(f"sync_{seed}", w.text(), Binding(grid, block, (rng.range(1, 4),)), {"n_access": nacc})


def random_shared(seed: int, max_instances: int = 60000) -> Workload:
    """Random kernel dominated by shared-memory accesses on blocks of 4..32
    warps (1-2D), 1-2 loops, 1-3 shared arrays with 4- or 8-byte elements,
    barrier intervals that may follow a loop, block / device atomics and a
    few global accesses.  Index forms favour collisions between neighbouring
    threads and warps (tx / 2, tx % Q, lin + k, lin / 40) so that races of
    every intra-block kind occur in some seeds and not in others."""
    rng = SplitMix64(seed)
    bdx = rng.choice([32, 64, 128, 256, 40, 96])
    bdy = rng.choice([1, 1, 2, 3, 4])
    while bdx * bdy > 1024:
        bdy -= 1
    grid = (rng.range(1, 4), rng.range(1, 2), 1)
    nloops = rng.range(1, 2)
    bounds = [rng.range(1, 4) for _ in range(nloops)]
    nacc = rng.range(3, 12)
    nthr = bdx * bdy * math.prod(grid)
    while nthr * math.prod(bounds) * nacc > max_instances and nacc > 3:
        nacc -= 1
    while nthr * math.prod(bounds) * nacc > max_instances and len(bounds) > 1:
        bounds.pop()
    w = _Writer(f"shr_{seed & 0xffff}")
    Q = rng.range(2, 9)
    w.add("param Q")
    lv = ["i", "j"][:len(bounds)]
    for v, b in zip(lv, bounds):
        w.add(f"loop {v} {b}")
    nsh = rng.range(1, 3)
    sizes = []
    for k in range(nsh):
        el = rng.choice([4, 4, 8])
        n_el = rng.range(16, 600)
        sizes.append((el, n_el))
        w.add(f"array S{k} shared {el * n_el} ; granule 4")
    w.add("array G global 65536")
    w.add("let lin = ty*bdx + tx")
    forms = ["lin", "lin / 2", "tx / 2", "tx % Q", "lin + 1", "lin / 40", "(lin + {v}) % 97", "ty", "tx",
             "lin / 32 + {v}", "3"]
    # half the seeds follow a race-free discipline: a thread writes only its
    # own element (arrays at least a block long), in even intervals, and
    # reads others' elements only in odd ones
    disciplined = rng.below(2) == 0
    if disciplined:
        w.lines = [x for x in w.lines if not x.startswith("array S")]
        sizes = [(el, max(n_el, bdx * bdy)) for el, n_el in sizes]
        for k, (el, n_el) in enumerate(sizes):
            w.add(f"array S{k} shared {el * n_el} ; granule 4")
        w.lines.append(w.lines.pop(w.lines.index("array G global 65536")))
        w.lines.append(w.lines.pop(w.lines.index("let lin = ty*bdx + tx")))
    for a_id in range(nacc):
        if rng.below(6) == 0:
            kind = rng.choice(["R", "W"])
            w.access(kind, "G", 4, f"(bx*bdx*bdy + lin) % 16384", iv=str(rng.range(0, 2)), line=a_id + 1)
            continue
        k = rng.below(nsh)
        el, n_el = sizes[k]
        r = rng.below(10)
        kind = "R" if r < 5 else ("W" if r < 9 else "A")
        form = rng.choice(forms).replace("{v}", rng.choice(lv))
        iv = str(rng.range(0, 2))
        if disciplined:
            kind = "W" if kind == "A" else kind
            if kind == "W":
                form, iv = "lin", str(2 * rng.below(2))
            elif form != "lin":
                iv = str(2 * rng.below(2) + 1)
        expr = f"({form}) % {n_el}"
        if rng.below(3) == 0:
            iv = f"{iv} + 4*{rng.choice(lv)}"
        guards = []
        if rng.below(4) == 0:
            guards.append(f"{rng.choice(['tx', 'ty', 'lin'])} {rng.choice(['<', '>='])} {rng.range(1, 40)}")
        scope = rng.choice(["block", "device"]) if kind == "A" else None
        w.access(kind, f"S{k}", el, expr, iv=iv, guards=guards, scope=scope, line=a_id + 1)
    return Workload(f"shr_{seed}", w.text(), Binding(grid, (bdx, bdy, 1), (Q,)),
                    {"loop_bounds": bounds, "n_access": nacc})


def warp_exchange(n_warps: int = 2, loops: int = 0, sync: str = "none", cross_warp: bool = False,
                  grid: int = 1, space: str = "shared") -> Workload:
    """Threads publish a value in shared memory and read a neighbour's (the
    warp-exchange pattern that Sec. 5.2's warp barrier protects): thread t
    writes S[t], then reads S[t's lane + 1 mod 32 in its own warp] (or, with
    cross_warp, S[t + 32 mod blockDim], a thread of the next warp).

    sync: "none" (no barrier), "warp" (one syncwarp between the write and the
    read), "warp2" (one more syncwarp after the read, so the next loop
    iteration's write is ordered too), "block" (syncthreads between them).
    space "global": S is a global array, block b exchanging in S[b*n, b*n + n)
    (no two blocks share an element).
    With `loops` > 0 the pair sits in a loop `i < loops`; the interval ids
    count the barriers executed before each access.  Closed forms: race free
    iff the barriers order every conflicting pair; every granule of S holds
    one witness otherwise (see tests)."""
    n = 32 * n_warps
    w = _Writer(f"warpx_{n_warps}_{loops}_{sync}_{int(cross_warp)}_{space}")
    if loops:
        w.add(f"loop i {loops}")
    glob = space == "global"
    w.add(f"array S global {4 * n * grid}" if glob else f"array S shared {4 * n}")
    rd = f"(tx + 32) % {n}" if cross_warp else "tx / 32 * 32 + (tx + 1) % 32"
    base = f"bx * {n} + " if glob else ""
    i = "i" if loops else "0"
    per = {"none": 0, "warp": 1, "warp2": 2, "block": 1}[sync]
    if sync == "block":  # interval ids count the block barriers before the access
        w.access("W", "S", 4, base + "tx", iv=f"{i}" if loops else "0", line=1)
        w.access("R", "S", 4, base + f"({rd})", iv=f"{i} + 1" if loops else "1", line=2)
    else:
        w.access("W", "S", 4, base + "tx", wv=f"{per}*{i}" if loops else "0", line=1)
        w.access("R", "S", 4, base + f"({rd})", wv=(f"{per}*{i} + {min(per, 1)}" if loops else str(min(per, 1))),
                 line=2)
    # closed form (a thread of a one-warp block reading "the next warp" reads its own element)
    racy = not (cross_warp and n_warps == 1) and (
        sync == "none" or (cross_warp and sync != "block") or
        (loops > 1 and (sync == "block" or sync == "warp")))
    return Workload(w.lines[0].split()[1], w.text(), Binding((grid, 1, 1), (n, 1, 1), ()),
                    {"sync": sync, "loops": loops, "cross_warp": cross_warp,
                     "expected_witnesses": (n * (grid if glob else 1)) if racy else 0})


def random_warp(seed: int, max_instances: int = 4096) -> Workload:
    """Random kernel with warp barriers: 1D blocks of 1-4 warps (some with a
    partial last warp), 1-2 blocks, one loop of 1-3 iterations, shared and
    global accesses whose indices collide inside and across warps (tx,
    lane + 1, tx / 2, tx % 8, tx + 32, a constant), barrier intervals in
    {0, 1} and warp intervals in {0..3}, either of them possibly growing with
    the loop counter."""
    rng = SplitMix64(seed)
    bdx = rng.choice([32, 64, 96, 128, 40, 17])
    grid = (rng.range(1, 2), 1, 1)
    bound = rng.range(1, 3)
    nacc = rng.range(2, 6)
    while bdx * grid[0] * bound * nacc > max_instances and nacc > 2:
        nacc -= 1
    w = _Writer(f"warp_{seed & 0xffff}")
    w.add(f"loop i {bound}")
    w.add(f"array S shared {4 * 160}")
    w.add("array G global 4096")
    forms = ["tx", "tx / 32 * 32 + (tx + 1) % 32", "tx / 2", "tx % 8", "(tx + 32) % 160", "5", "tx + i"]
    for a_id in range(nacc):
        arr = rng.choice(["S", "S", "G"])
        r = rng.below(10)
        kind = "R" if r < 5 else ("W" if r < 9 else "A")
        idx = rng.choice(forms)
        if arr == "G" and rng.below(2):
            idx = f"bx * 200 + {idx}"
        iv = str(rng.range(0, 1))
        if rng.below(4) == 0:
            iv = f"{iv} + i"
        wv = str(rng.range(0, 3))
        if rng.below(3) == 0:
            wv = f"{wv} + {rng.range(1, 2)}*i"
        guards = [f"tx {rng.choice(['<', '>='])} {rng.range(1, 40)}"] if rng.below(4) == 0 else []
        scope = rng.choice(["block", "device"]) if kind == "A" else None
        w.access(kind, arr, 4, idx, iv=iv, wv=wv, guards=guards, scope=scope, line=a_id + 1)
    return Workload(f"warp_{seed}", w.text(), Binding(grid, (bdx, 1, 1), ()), {"n_access": nacc})


# --------------------------------------------------------------------------
# Config 4: corpus of seeded synthetic kernels of uneven size.
#   2..32 accesses, 1-3D grids and blocks, 1..4 nested loops (bounds <= 64),
#   affine guards, int32 and float4 widths, about 10% atomics and 30% with a
#   planted race; the instance count is drawn log-uniform on [1e3, 1e7] and
#   the launch dims are fitted to it.  Without the planted race every kernel
#   is race free by construction: each thread writes a private region of the
#   data arrays (idx = gid * SPAN + loop offset), reads go to read-only inputs
#   or to the thread's own region, shared-memory neighbour reads sit in a
#   later barrier interval than the writes, and atomics are device scoped on
#   their own counters.  The planted race is one of: a write that drops the
#   thread term, a private stride one too small, a neighbour read in the
#   writer's interval, block-scoped atomics on a grid-wide counter, or a
#   shared-memory neighbour read before the barrier.

PLANTS = ("shared_write", "short_stride", "neighbour_read", "block_atomic", "shared_early_read")


def _dims(total, rng, maxdims):
    nd = rng.range(1, maxdims)
    dims = [1, 1, 1]
    rest = max(1, total)
    for d in range(nd - 1):
        f = 1
        for _ in range(rng.range(0, 3)):
            if rest % 2 == 0 and rest > 1:
                f *= 2
                rest //= 2
        dims[d] = max(1, f)
    dims[nd - 1] = rest
    return dims


def _c4_lookalikes(w, item, nthr, nblk, span, has_shared, planted):
    """Append 0-3 blocks of two accesses whose addresses overlap across the
    threads of a block, so that no bind-time disjointness test can drop the
    pair and only the exact check decides it.  A block is a halo exchange on
    the global array H (each thread writes its own slot in iteration i at
    interval 2i, then reads the next thread's slot of its own block at 2i+1)
    or a broadcast through the shared array Bc (thread 0 writes at 2i+1,
    every thread reads at 2i+2).  Both are race free.  In a planted kernel
    one block may instead take its racy twin: the read in the writer's
    interval, or the halo read crossing the block edge (only with more than
    one block).  The draws come from a second generator stream, so the rest
    of the kernel is the same with or without these blocks.  Returns the
    racy twin's name or None."""
    rng = SplitMix64((seed_for(4, item) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & MASK64)
    used = sum(1 for l in w.lines if l.startswith("access"))
    blocks = []
    for _ in range(rng.below(4)):
        if used + 2 > 32:
            break
        blocks.append("broadcast" if has_shared and rng.below(2) else "halo")
        used += 2
    racy_at = rng.below(len(blocks)) if planted and blocks and rng.below(2) == 0 else -1
    if not blocks:
        return None
    decl = []
    if "halo" in blocks:
        decl.append(f"array H global {4 * (nthr * nblk + 1) * span}")
    if "broadcast" in blocks:
        decl.append(f"array Bc shared {4 * span}")
    at = next(n for n, l in enumerate(w.lines) if l.startswith("assert"))
    w.lines[at:at] = decl
    twin = None
    for n, b in enumerate(blocks):
        line = 200 + 2 * n
        if b == "halo":
            w.access("W", "H", 4, "gid*SPAN + off", iv="2*i", line=line)
            rd, iv = f"(lb*{nthr} + (lt + 1) % {nthr})*SPAN + off", "2*i + 1"
            if n == racy_at:
                if nblk > 1 and rng.below(2):
                    twin, rd = "halo_cross", "(gid + 1)*SPAN + off"
                else:
                    twin, iv = "halo_early", "2*i"
            w.access("R", "H", 4, rd, iv=iv, line=line + 1)
        else:
            w.access("W", "Bc", 4, "off", iv="2*i + 1", guards=["lt == 0"], line=line)
            iv = "2*i + 2"
            if n == racy_at:
                twin, iv = "broadcast_early", "2*i + 1"
            w.access("R", "Bc", 4, "off", iv=iv, line=line + 1)
    return twin


def config4(item: int, lo_exp: float = 3.0, hi_exp: float = 7.0, planted=None) -> Workload:
    rng = SplitMix64(seed_for(4, item))
    target = int(10 ** (lo_exp + (hi_exp - lo_exp) * rng.uniform()))
    nacc = rng.range(2, 32)
    nloops = rng.range(1, 4)
    bounds = [rng.choice([1, 2, 2, 3, 4, 4, 8, 16, 64]) for _ in range(nloops)]
    while math.prod(bounds) * nacc > max(target, nacc) and max(bounds) > 1:
        k = bounds.index(max(bounds))
        bounds[k] = max(1, bounds[k] // 2)
    span = math.prod(bounds)
    if planted is None:
        planted = rng.below(10) < 3
    threads = max(2 if planted else 1, target // (nacc * span))
    nthr = min(threads, rng.choice([32, 64, 128, 256, 512, 1024]))
    nthr = max(2 if planted else 1, nthr)
    nblk = max(1, (threads + nthr - 1) // nthr)
    block = _dims(nthr, rng, 3)
    while math.prod(block) > 1024:
        block[block.index(max(block))] //= 2
    grid = _dims(nblk, rng, 3)
    nthr = math.prod(block)
    nblk = math.prod(grid)
    plant = rng.choice(PLANTS) if planted else None
    lv = ["i", "j", "k", "l"][:nloops]
    w = _Writer(f"corpus_{item}")
    w.add("param SPAN NT")
    for v, b in zip(lv, bounds):
        w.add(f"loop {v} {b}")
    # linear ids and the loop offset inside the thread's private region
    w.add("let lt = (tz*bdy + ty)*bdx + tx")
    w.add("let lb = (bz*gdy + by)*gdx + bx")
    w.add("let gid = lb*(bdx*bdy*bdz) + lt")
    off = lv[0]
    for v, b in zip(lv[1:], bounds[1:]):
        off = f"({off})*{b} + {v}"
    w.add(f"let off = {off}")
    total_threads = nthr * nblk
    w.add(f"array D global {4 * (total_threads + 1) * span}")
    w.add(f"array E global {16 * (total_threads + 1) * span}")
    w.add(f"array In global {16 * 4096}")
    w.add("array Cnt global 256")
    has_shared = nthr * span <= 12288
    if has_shared:
        w.add(f"array S shared {4 * nthr * span}")
    w.add("assert SPAN > 0")
    w.add("assert NT > 0")
    nvalid = max(1, total_threads - rng.below(max(1, total_threads // 4)))
    kinds = []
    for a in range(nacc):
        r = rng.below(100)
        if r < 10:
            kinds.append("atomic")
        elif r < 30:
            kinds.append("input")
        elif r < 55:
            kinds.append("write_D")
        elif r < 70:
            kinds.append("read_D")
        elif r < 80:
            kinds.append("write_E")
        elif r < 88 and has_shared:
            kinds.append("shared_write")
        elif has_shared:
            kinds.append("shared_read")
        else:
            kinds.append("input")
    plant_at = rng.below(nacc) if planted else -1
    if plant == "block_atomic" and nblk < 2:
        plant = "shared_write"
    if plant == "shared_early_read" and not has_shared:
        plant = "neighbour_read"
    if plant in ("neighbour_read", "shared_early_read") and len(kinds) == 32:
        kinds.pop()  # the plant adds a second access; stay within 32
        plant_at = min(plant_at, len(kinds) - 1)
    for a, kind in enumerate(kinds):
        guards = []
        if rng.below(3) == 0:
            guards.append("gid < NT")
        if nloops and rng.below(5) == 0:
            v = rng.choice(lv)
            guards.append(f"{v} <= {rng.below(bounds[lv.index(v)])}")
        iv = rng.below(3)
        line = 100 + a
        if a == plant_at:
            # the planted race: unguarded so that it always fires
            if plant == "shared_write":
                w.access("W", "D", 4, "off", iv=iv, line=line)
            elif plant == "short_stride":
                w.access("W", "D", 4, "gid*(SPAN - 1) + off" if span > 1 else "gid / 2", iv=iv, line=line)
            elif plant == "neighbour_read":
                w.access("W", "D", 4, "gid*SPAN + off", iv=0, line=line)
                w.access("R", "D", 4, "(gid + 1)*SPAN + off", iv=0, line=line)
            elif plant == "block_atomic":
                w.access("A", "Cnt", 4, f"{rng.below(8)}", iv=iv, scope="block", line=line)
            else:  # shared_early_read
                w.access("W", "S", 4, "lt*SPAN + off", iv=1, line=line)
                w.access("R", "S", 4, f"((lt + 1) % {nthr})*SPAN + off", iv=1, line=line)
            continue
        if kind == "atomic":
            w.access("A", "Cnt", 4, f"gid % {rng.range(1, 64)}", iv=iv, guards=guards, scope="device", line=line)
        elif kind == "input":
            c1, c2 = rng.range(1, 7), rng.range(0, 5)
            wid = 16 if rng.below(3) == 0 else 4
            n_el = (16 * 4096) // wid
            w.access("R", "In", wid, f"(gid*{c1} + off*{c2} + {rng.below(97)}) % {n_el}", iv=iv, guards=guards,
                     line=line)
        elif kind == "write_D":
            w.access("W", "D", 4, "gid*SPAN + off", iv=iv, guards=guards, line=line)
        elif kind == "read_D":
            w.access("R", "D", 4, "gid*SPAN + off", iv=iv, guards=guards, line=line)
        elif kind == "write_E":
            w.access("W", "E", 16, "gid*SPAN + off", iv=iv, guards=guards, line=line)
        elif kind == "shared_write":
            w.access("W", "S", 4, "lt*SPAN + off", iv=1, guards=guards, line=line)
        elif kind == "shared_read":
            w.access("R", "S", 4, f"((lt + 1) % {nthr})*SPAN + off", iv=2, guards=guards, line=line)
    pattern_race = _c4_lookalikes(w, item, nthr, nblk, span, has_shared, plant is not None)
    inst = nblk * nthr * span * len([l for l in w.lines if l.startswith("access")])
    return Workload(f"c4_{item}", w.text(), Binding(tuple(grid), tuple(block), (span, nvalid)),
                    {"config": 4, "planted": plant, "pattern_race": pattern_race, "target": target, "instances": inst,
                     "n_access": sum(1 for l in w.lines if l.startswith("access"))})
