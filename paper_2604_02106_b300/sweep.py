"""A race under some host-admissible input.

The paper asks whether a kernel races for *some* input the host code admits
(Sec. 3 and Sec. 5.1: the host fixes some parameters, bounds others with
asserts and loops, and picks the launch shape).  The paper answers it
symbolically; this module answers it over a set of admissible bindings: the
parameter values come from the bounds the descriptor's asserts put on each
parameter (hgrd_desc_params) plus the values a caller supplies, every
combination is bound (asserts that relate several values, e.g. the launch
shape to a size, reject the inadmissible ones), bindings whose bound programs
are identical (hgrd_bound_hash) are checked once, and the distinct ones run
on the batched path.  The verdict of every binding is exact; "clean" means
clean for the bindings checked.
"""
from __future__ import annotations

import ctypes as C
import itertools
import random
from dataclasses import dataclass, field

from . import Batch, HgrdError, Kernel, ItemResult, _raise, lib

# bind-time refusals: not admissible (an assert failed, a divisor or size is
# out of range for the values), or admissible but beyond this checker (the
# values overflow the index arithmetic or the key)
_INADMISSIBLE = {"EHOSTCONSTRAINT", "EBIND"}
_UNSUPPORTED = {"EOVERFLOW", "EUNSUPPORTED"}


class ParamInfo(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("lo", C.c_int64), ("hi", C.c_int64), ("has_lo", C.c_uint32),
                ("has_hi", C.c_uint32)]


@dataclass
class Param:
    name: str
    lo: int | None   # from the asserts on this parameter alone; None = unbounded
    hi: int | None


def params(text: str) -> list:
    """The descriptor's parameters with the bounds its asserts put on each alone."""
    L = lib()
    L.hgrd_desc_params.argtypes = [C.c_void_p, C.POINTER(ParamInfo), C.c_uint32, C.POINTER(C.c_uint32)]
    L.hgrd_desc_params.restype = C.c_int
    k = Kernel(text)
    n = C.c_uint32()
    _raise(L.hgrd_desc_params(k._h, None, 0, C.byref(n)))
    buf = (ParamInfo * max(1, n.value))()
    _raise(L.hgrd_desc_params(k._h, buf, n.value, C.byref(n)))
    return [Param(buf[i].name.decode(), buf[i].lo if buf[i].has_lo else None, buf[i].hi if buf[i].has_hi else None)
            for i in range(n.value)]


def bound_hash(kernel: Kernel) -> int:
    """Hash of everything a check of the bound kernel reads (equal hash, equal verdict)."""
    L = lib()
    L.hgrd_bound_hash.argtypes = [C.c_void_p, C.POINTER(C.c_uint64)]
    L.hgrd_bound_hash.restype = C.c_int
    h = C.c_uint64()
    _raise(L.hgrd_bound_hash(kernel._h, C.byref(h)))
    return h.value


def candidate_values(p: Param, free=(1, 4096), per_param: int = 8, seed: int = 0) -> list:
    """Values tried for one parameter: the ends of its admissible range (the
    asserts' bounds, else `free`) and their neighbours, the powers of two in
    it, then seeded draws, at most per_param of them, in increasing order."""
    lo = p.lo if p.lo is not None else free[0]
    hi = p.hi if p.hi is not None else free[1]
    if lo > hi:
        return []
    first = [lo, hi, lo + 1, hi - 1]
    k = 1
    while k <= hi:
        if k >= lo:
            first.append(k)
        k <<= 1
    out = []
    for v in first:
        if lo <= v <= hi and v not in out:
            out.append(v)
    rng = random.Random(seed)
    while len(out) < per_param and len(out) < hi - lo + 1:
        v = rng.randint(lo, hi)
        if v not in out:
            out.append(v)
    return sorted(out[:per_param])


@dataclass
class SweepResult:
    racy: bool                 # some checked admissible binding races
    admissible: int            # bindings the asserts admitted
    rejected: int              # combinations the asserts (or binding rules) refused
    unsupported: int           # admissible combinations beyond this checker (not checked)
    distinct: int              # distinct bound programs checked
    instances: int             # instances over all admissible bindings
    bindings: list             # (grid, block, params) of every admissible binding
    verdicts: list             # ItemResult per admissible binding (shared by equal programs)
    groups: dict = field(default_factory=dict)  # verdict signature -> indices into bindings

    @property
    def racy_bindings(self) -> list:
        return [b for b, v in zip(self.bindings, self.verdicts) if v.racy]

    @property
    def first_racy(self):
        for b, v in zip(self.bindings, self.verdicts):
            if v.racy:
                return b, v
        return None


def _signature(v: ItemResult) -> tuple:
    """What the verdict says about the kernel: racy or not, and which access
    pairs race with which kinds."""
    return (bool(v.racy), tuple(sorted((v.pairs or {}).items())))


def symbolic_check(text: str, launch, values: dict | None = None, free=(1, 4096), per_param: int = 8,
                   max_bindings: int = 512, seed: int = 0, witness_cap: int = 16, stream=None) -> SweepResult:
    """Check `text` over admissible bindings.

    launch: the host's launch shape for a parameter assignment: a (grid,
        block) pair, a list of them, or a callable taking {name: value} and
        returning one pair or a list.
    values: {name: [values]} to try for a parameter instead of the generated
        candidates (host-loop values, say).
    Combinations beyond max_bindings are sampled (seeded)."""
    ps = params(text)
    values = values or {}
    cand = [values[p.name] if p.name in values else candidate_values(p, free, per_param, seed + i)
            for i, p in enumerate(ps)]
    combos = list(itertools.product(*cand)) if ps else [()]
    if len(combos) > max_bindings:
        combos = sorted(random.Random(seed).sample(combos, max_bindings))
    bindings, kernels, rejected, unsupported = [], [], 0, 0
    for combo in combos:
        assign = {p.name: v for p, v in zip(ps, combo)}
        shapes = launch(assign) if callable(launch) else launch
        if isinstance(shapes, tuple) and len(shapes) == 2 and isinstance(shapes[0], (tuple, list)):
            shapes = [shapes]
        for grid, block in shapes:
            try:
                k = Kernel(text).bind(tuple(grid), tuple(block), tuple(combo))
            except HgrdError as e:
                code = str(e).split(":")[0]
                if code in _INADMISSIBLE:
                    rejected += 1
                    continue
                if code in _UNSUPPORTED:
                    unsupported += 1
                    continue
                raise
            bindings.append((tuple(grid), tuple(block), dict(assign)))
            kernels.append(k)
    # one check per distinct bound program
    rep_of, reps = [], {}
    for k in kernels:
        h = bound_hash(k)
        if h not in reps:
            reps[h] = len(reps)
        rep_of.append(reps[h])
    first_of = {}
    for i, r in enumerate(rep_of):
        first_of.setdefault(r, i)
    distinct = [kernels[first_of[r]] for r in range(len(reps))]
    results = Batch(distinct, witness_cap=witness_cap).check(stream) if distinct else []
    for r, (res, k) in enumerate(zip(results, distinct)):
        if res.status != 0:  # a per-item buffer overflowed: the plain check retries with room
            full = k.check(cap=witness_cap)
            results[r] = ItemResult(status=0, racy=full.racy, small=False, n_witness=full.n_witness,
                                    n_by_kind=full.n_by_kind, n_instances=full.n_instances, n_keys=full.n_keys,
                                    n_oob=full.n_oob, witnesses=full.witnesses[:witness_cap], pairs=full.pairs)
    verdicts = [results[r] for r in rep_of]
    groups = {}
    for i, v in enumerate(verdicts):
        groups.setdefault(_signature(v), []).append(i)
    return SweepResult(any(v.racy for v in verdicts), len(bindings), rejected, unsupported, len(distinct),
                       sum(v.n_instances for v in verdicts), bindings, verdicts, groups)
