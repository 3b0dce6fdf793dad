"""CPU oracle for the host-guided race check — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct C++ implementation of the paper's race
definition (Sec. 2, Sec. 6.1, Tables 1-2, Appendix A) over every concrete
instance of a kernel descriptor under one host binding.  It shares no code with
the GPU library (own parser, own evaluator, own structs).  Only tests/,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may use it; the
product path never routes through it.

Parity status of each function (what pins it; the pins are in
tests/test_oracle.py and tests/test_ranker_cpu.py):
  * orc_check witness set / kind masks / counts / minimal witness / canonical
    instance pair: pinned by pairwise brute force over all instance pairs on
    tiny grids (tests/brute.py), by the paper's Fig. 1, 2, 3 and 5 verdicts
    (tests/golden/), by closed forms (stride sweep, planted stencil row
    stride, all-threads-one-address, the config-1 kernel's single planted
    race) and by invariants (an added barrier, a removed access or a write
    turned into a read never adds a witness; relabelling threads keeps the
    verdict).
  * mlp_ref (the ranker's FP64 reference): forward and loss pinned by a
    hand-worked network whose logits and weighted cross-entropy are written
    out in the test, and by the loss at logits 0 and +-40; gradients by
    central finite differences.
  * the Fig. 4 (ludInternal, offset < 0) race claim: parity unpinned — the
    printed listing alone cannot race under a uniform offset, so no verdict
    test uses it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgrd_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

ERRORS = {0: "OK", 1: "TRUNCATED", -1: "EINVAL", -2: "EPARSE", -3: "EBIND",
          -4: "EHOSTCONSTRAINT", -5: "EOVERFLOW"}


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU involved)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Binding(C.Structure):
    _fields_ = [("grid", C.c_int32 * 3), ("block", C.c_int32 * 3),
                ("nparams", C.c_uint32), ("params", C.POINTER(C.c_int64))]


class _Witness(C.Structure):
    _fields_ = [("space", C.c_uint8), ("array", C.c_uint8), ("acc_lo", C.c_uint8),
                ("acc_hi", C.c_uint8), ("kind_mask", C.c_uint8), ("pad", C.c_uint8 * 3),
                ("byte_addr", C.c_uint64)]


class _Inst(C.Structure):
    _fields_ = [("lin_block", C.c_uint32), ("lin_thread", C.c_uint32), ("iter", C.c_uint32 * 4),
                ("access", C.c_uint8), ("pad", C.c_uint8 * 3)]


class _Verdict(C.Structure):
    _fields_ = [("racy", C.c_int32), ("pad", C.c_int32), ("n_witness", C.c_uint64),
                ("n_by_kind", C.c_uint64 * 3), ("n_instances", C.c_uint64), ("n_keys", C.c_uint64),
                ("n_oob", C.c_uint64), ("min_w", _Witness), ("min_x", _Inst), ("min_y", _Inst)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_check.restype = C.c_int
        _lib.orc_check.argtypes = [C.c_char_p, C.POINTER(_Binding), C.c_int, C.c_uint64, C.c_uint64,
                                   C.POINTER(_Witness), C.c_uint64, C.POINTER(_Verdict),
                                   C.c_char_p, C.c_size_t, C.c_int]
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


@dataclass
class Result:
    code: int
    racy: bool
    n_witness: int
    n_by_kind: tuple
    n_instances: int
    n_keys: int
    n_oob: int
    witnesses: list            # tuples (space, array, byte_addr, acc_lo, acc_hi, kind_mask)
    min_w: tuple | None
    min_x: tuple | None        # (lin_block, lin_thread, i0, i1, i2, i3, access)
    min_y: tuple | None
    extra: dict = field(default_factory=dict)


def _wt(w):
    return (w.space, w.array, w.byte_addr, w.acc_lo, w.acc_hi, w.kind_mask)


def _it(i):
    return (i.lin_block, i.lin_thread, *i.iter, i.access)


def check(text: str, binding, cap: int = 1 << 20, filter_array: int = -1,
          gran_lo: int = 0, gran_hi: int = 0, pair: bool = True) -> Result:
    """Run the oracle.  ``binding`` has .grid, .block, .params.  pair=False
    skips the canonical instance pair (min_x / min_y are None): its search is
    quadratic in the instances on the minimal witness's granule."""
    lib = _load()
    params = (C.c_int64 * max(1, len(binding.params)))(*binding.params)
    b = _Binding((C.c_int32 * 3)(*binding.grid), (C.c_int32 * 3)(*binding.block),
                 len(binding.params), params)
    out = (_Witness * max(1, cap))()
    v = _Verdict()
    err = C.create_string_buffer(512)
    rc = lib.orc_check(text.encode(), C.byref(b), filter_array, gran_lo, gran_hi, out, cap,
                       C.byref(v), err, len(err), 0 if pair else 1)
    if rc < 0:
        raise OracleError(rc, err.value.decode())
    n = min(cap, v.n_witness)
    ws = [_wt(out[k]) for k in range(n)]
    return Result(rc, bool(v.racy), v.n_witness, tuple(v.n_by_kind), v.n_instances, v.n_keys, v.n_oob,
                  ws, _wt(v.min_w) if v.racy else None,
                  _it(v.min_x) if v.racy and pair else None, _it(v.min_y) if v.racy and pair else None)


def _band(args):
    text, grid, block, params, band, nbands, cap, pair = args
    from types import SimpleNamespace
    b = SimpleNamespace(grid=grid, block=block, params=params)
    return check(text, b, cap=cap, filter_array=-2, gran_lo=band, gran_hi=nbands, pair=pair)


def check_parallel(text: str, binding, jobs: int, cap: int = 1 << 20, pair: bool = True, pool=None) -> Result:
    """The oracle on `jobs` host processes: the buckets are split into `jobs`
    bands by granule (granule % jobs), each process enumerates every instance
    but buckets and checks only its band, and the witness lists are merged.
    The result equals check()'s (tests compare them).  Pass a process pool
    made with the 'spawn' start method, or one is made here."""
    import multiprocessing as mp
    args = [(text, tuple(binding.grid), tuple(binding.block), tuple(binding.params), j, jobs, cap, pair)
            for j in range(jobs)]
    if pool is None:
        with mp.get_context("spawn").Pool(jobs) as p:
            parts = p.map(_band, args)
    else:
        parts = pool.map(_band, args)
    ws = sorted(w for r in parts for w in r.witnesses)
    n_witness = sum(r.n_witness for r in parts)
    kinds = tuple(sum(r.n_by_kind[k] for r in parts) for k in range(3))
    first = min((r for r in parts if r.racy), key=lambda r: r.min_w, default=None)
    r0 = parts[0]
    return Result(1 if n_witness > cap else 0, n_witness > 0, n_witness, kinds, r0.n_instances, r0.n_keys,
                  r0.n_oob, ws[:cap], first.min_w if first else None, first.min_x if first else None,
                  first.min_y if first else None)
