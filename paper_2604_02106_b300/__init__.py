"""Python binding of libhgrd.so, the B300 exhaustive host-guided race check.

Argument marshalling only: every step of the check runs in the library's CUDA
kernels.  PyTorch provides the device workspace and the stream.  When the
compiled library is missing this module raises on use; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import struct
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhgrd.so")

OK, ETRUNCATED = 0, 1
ERRORS = {1: "ETRUNCATED", -1: "EINVAL", -2: "EPARSE", -3: "EBIND", -4: "EHOSTCONSTRAINT", -5: "EOVERFLOW",
          -6: "ENOMEM", -7: "EDEVICE", -8: "ETIMEOUT", -9: "EUNSUPPORTED"}
NO_PAIR = 1
PROFILE = 2
STOP_FIRST = 4
NO_SPLIT = 8
JIT = 16
NO_JIT = 32
NO_SMALL = 64
GRAPH = 128      # run the check as one CUDA graph launch (captured once per binding, workspace, options)
NO_CELL_FILTER = 256  # sort every kept key (no per-cell pre-filter)
CELL_FILTER = 512     # pre-filter keys by cell whenever the table fits (default: only for many keys)
ALL_KEYS = 1024       # write and sort the keys of every live access (one global sort, interpreted kernels)
SCAN_BALLOT = 2048    # first scan phase as 32-key warp steps instead of tensor-copied rows (same result)

# symbols include/hgrd.h declares
EXPORTS = ["hgrd_load_desc", "hgrd_bind_host_params", "hgrd_workspace_size", "hgrd_check", "hgrd_check_enqueue",
           "hgrd_check_collect", "hgrd_last_stats", "hgrd_last_profile", "hgrd_free_desc", "hgrd_last_error",
           "hgrd_debug_divmod", "hgrd_debug_lookback_timeout", "hgrd_check_noalloc", "hgrd_batch_create",
           "hgrd_batch_workspace_size",
           "hgrd_batch_run", "hgrd_batch_collect", "hgrd_batch_tune", "hgrd_batch_free", "hgrd_pair_features",
           "hgrd_mlp_model_bytes", "hgrd_mlp_workspace_bytes", "hgrd_mlp_init", "hgrd_mlp_predict", "hgrd_mlp_grad",
           "hgrd_mlp_train_step", "hgrd_mlp_params", "hgrd_mlp_sync_bf16", "hgrd_ranked_workspace_size",
           "hgrd_check_ranked", "hgrd_sort_tune", "hgrd_sort_variant", "hgrd_jit_compile", "hgrd_jit_source",
           "hgrd_desc_params", "hgrd_bound_hash", "hgrd_bound_info", "hgrd_batch_rank_prepare",
           "hgrd_batch_ranked_workspace_size", "hgrd_batch_check_ranked", "hgrd_sort_pass_variant"]
BATCH_GRAPH = 1
BATCH_JIT = 2


class HgrdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Binding(C.Structure):
    _fields_ = [("grid", C.c_int32 * 3), ("block", C.c_int32 * 3), ("nparams", C.c_uint32),
                ("params", C.POINTER(C.c_int64))]


class Witness(C.Structure):
    _fields_ = [("space", C.c_uint8), ("array", C.c_uint8), ("acc_lo", C.c_uint8), ("acc_hi", C.c_uint8),
                ("kind_mask", C.c_uint8), ("pad", C.c_uint8 * 3), ("byte_addr", C.c_uint64)]


def _witness_dtype():
    import numpy as np
    return np.dtype({"names": ["space", "array", "acc_lo", "acc_hi", "kind_mask", "byte_addr"],
                     "formats": ["u1", "u1", "u1", "u1", "u1", "<u8"],
                     "offsets": [Witness.space.offset, Witness.array.offset, Witness.acc_lo.offset,
                                 Witness.acc_hi.offset, Witness.kind_mask.offset, Witness.byte_addr.offset],
                     "itemsize": C.sizeof(Witness)})


_WITNESS_DTYPE = _witness_dtype()


class Inst(C.Structure):
    _fields_ = [("lin_block", C.c_uint32), ("lin_thread", C.c_uint32), ("iter", C.c_uint32 * 4),
                ("access", C.c_uint8), ("pad", C.c_uint8 * 3)]


class Verdict(C.Structure):
    _fields_ = [("racy", C.c_int32), ("pair_found", C.c_int32), ("n_witness", C.c_uint64),
                ("n_by_kind", C.c_uint64 * 3), ("n_instances", C.c_uint64), ("n_keys", C.c_uint64),
                ("n_oob", C.c_uint64), ("min_w", Witness), ("min_x", Inst), ("min_y", Inst),
                ("pair_kind", (C.c_uint32 * 32) * 3)]


class CheckOpts(C.Structure):
    _fields_ = [("max_raw_witness", C.c_uint64), ("pair_cap", C.c_uint32), ("flags", C.c_uint32),
                ("only_accesses", C.c_uint32), ("max_shared_keys", C.c_uint32)]


class BatchOpts(C.Structure):
    _fields_ = [("small_keys", C.c_uint32), ("streams", C.c_uint32), ("witness_cap", C.c_uint32),
                ("flags", C.c_uint32)]


class ItemVerdict(C.Structure):
    _fields_ = [("status", C.c_int32), ("racy", C.c_int32), ("small", C.c_int32), ("n_copied", C.c_int32),
                ("n_witness", C.c_uint64), ("n_by_kind", C.c_uint64 * 3), ("n_instances", C.c_uint64),
                ("n_keys", C.c_uint64), ("n_oob", C.c_uint64), ("pair_kind", (C.c_uint32 * 32) * 3)]


class BatchRankInfo(C.Structure):
    _fields_ = [("n_pairs", C.c_uint32), ("ranked", C.c_uint32), ("confirmed", C.c_uint32), ("second", C.c_uint32),
                ("ms_score", C.c_float), ("ms_stage1", C.c_float), ("ms_stage2", C.c_float), ("pad", C.c_float)]


class StageTime(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("ms", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("n_candidates", C.c_uint64), ("n_raw_witness", C.c_uint64),
                ("sort_passes", C.c_uint32), ("int64_path", C.c_uint32), ("h2d_bytes", C.c_uint64),
                ("d2h_bytes", C.c_uint64), ("n_sorted_keys", C.c_uint64), ("n_binned_keys", C.c_uint64),
                ("shared_bins", C.c_uint32), ("jit", C.c_uint32), ("eval_ops", C.c_uint64),
                ("small", C.c_uint32), ("cell_filter", C.c_uint32), ("n_written_keys", C.c_uint64),
                ("cuda_objects_created", C.c_uint64)]


_lib = None


def lib():
    """Load libhgrd.so (built in-tree by __graft_entry__.build / _build.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhgrd.so is not built ({LIB_PATH}); run paper_2604_02106_b300._build.build()")
        L = C.CDLL(LIB_PATH)
        vp, sz, u64 = C.c_void_p, C.c_size_t, C.c_uint64
        L.hgrd_load_desc.argtypes = [C.c_char_p, sz, C.POINTER(vp)]
        L.hgrd_bind_host_params.argtypes = [vp, C.POINTER(Binding)]
        L.hgrd_workspace_size.argtypes = [vp, C.POINTER(CheckOpts), C.POINTER(sz)]
        L.hgrd_check.argtypes = [vp, C.POINTER(CheckOpts), vp, sz, vp, C.POINTER(Witness), u64, C.POINTER(Verdict)]
        L.hgrd_check_enqueue.argtypes = [vp, C.POINTER(CheckOpts), vp, sz, vp]
        L.hgrd_check_collect.argtypes = [vp, C.POINTER(CheckOpts), vp, sz, vp, C.POINTER(Witness), u64,
                                         C.POINTER(Verdict)]
        L.hgrd_check_noalloc.argtypes = [vp, C.POINTER(CheckOpts), vp, C.POINTER(Witness), u64, C.POINTER(Verdict)]
        L.hgrd_check_noalloc.restype = C.c_int
        L.hgrd_batch_create.argtypes = [C.POINTER(vp), C.c_uint32, C.POINTER(BatchOpts), C.POINTER(vp)]
        L.hgrd_batch_workspace_size.argtypes = [vp, C.POINTER(sz)]
        L.hgrd_batch_run.argtypes = [vp, vp, sz, vp]
        L.hgrd_batch_collect.argtypes = [vp, vp, sz, vp, C.POINTER(ItemVerdict), C.POINTER(Witness), C.c_uint32]
        L.hgrd_batch_tune.argtypes = [vp, vp, sz, vp, C.POINTER(BatchOpts)]
        L.hgrd_batch_free.argtypes = [vp]
        L.hgrd_batch_free.restype = None
        L.hgrd_batch_rank_prepare.argtypes = [vp]
        L.hgrd_batch_ranked_workspace_size.argtypes = [vp, C.POINTER(sz)]
        L.hgrd_batch_check_ranked.argtypes = [vp, vp, C.c_uint32, C.c_float, vp, sz, vp, C.POINTER(ItemVerdict),
                                              C.POINTER(Witness), C.c_uint32, C.POINTER(C.c_uint8),
                                              C.POINTER(BatchRankInfo)]
        for f in ["hgrd_batch_create", "hgrd_batch_workspace_size", "hgrd_batch_run", "hgrd_batch_collect",
                  "hgrd_batch_tune", "hgrd_batch_rank_prepare", "hgrd_batch_ranked_workspace_size",
                  "hgrd_batch_check_ranked"]:
            getattr(L, f).restype = C.c_int
        L.hgrd_last_stats.argtypes = [C.POINTER(Stats)]
        L.hgrd_last_profile.argtypes = [C.POINTER(StageTime), C.c_uint32, C.POINTER(C.c_uint32)]
        L.hgrd_free_desc.argtypes = [vp]
        L.hgrd_free_desc.restype = None
        L.hgrd_last_error.restype = C.c_char_p
        L.hgrd_debug_divmod.argtypes = [C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.hgrd_jit_compile.argtypes = [vp, C.POINTER(CheckOpts), C.POINTER(C.c_double)]
        L.hgrd_jit_source.argtypes = [vp, C.POINTER(CheckOpts), C.c_char_p, sz, C.POINTER(sz)]
        L.hgrd_bound_info.argtypes = [vp, C.POINTER(u64), C.POINTER(u64)]
        for f in ["hgrd_load_desc", "hgrd_bind_host_params", "hgrd_workspace_size", "hgrd_check",
                  "hgrd_check_enqueue", "hgrd_check_collect", "hgrd_last_stats", "hgrd_last_profile",
                  "hgrd_debug_divmod", "hgrd_jit_compile", "hgrd_jit_source",
                  "hgrd_desc_params", "hgrd_bound_hash", "hgrd_bound_info"]:
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _raise(rc):
    if rc < 0:
        raise HgrdError(rc, lib().hgrd_last_error().decode(errors="replace"))


def _opts(max_raw_witness=0, pair_cap=0, flags=0, only_accesses=0, max_shared_keys=0):
    return CheckOpts(max_raw_witness, pair_cap, flags, only_accesses, max_shared_keys)


def _pairs(pk):
    """{(a, b): kind_mask} for a <= b from the three 32x32 bit matrices."""
    rows = struct.unpack("96I", bytes(pk))  # one copy out of the ctypes array
    out = {}
    for i, row in enumerate(rows):
        if not row:
            continue
        k, a = divmod(i, 32)
        row >>= a
        b = a
        while row:
            if row & 1:
                out[(a, b)] = out.get((a, b), 0) | (1 << k)
            row >>= 1
            b += 1
    return out


@dataclass
class Result:
    racy: bool
    n_witness: int
    n_by_kind: tuple
    n_instances: int
    n_keys: int
    n_oob: int
    witnesses: list        # (space, array, byte_addr, acc_lo, acc_hi, kind_mask), canonical order
    min_w: tuple | None
    min_x: tuple | None    # (lin_block, lin_thread, i0, i1, i2, i3, access)
    min_y: tuple | None
    truncated: bool = False
    pairs: dict = None     # {(acc_lo, acc_hi): kind_mask}: the racy access pairs


def _wt(w):
    return (w.space, w.array, w.byte_addr, w.acc_lo, w.acc_hi, w.kind_mask)


def _witness_list(out, n: int) -> list:
    """The first n hgrd_witness records of `out` as (space, array, byte_addr,
    acc_lo, acc_hi, kind_mask) tuples (one vectorised view, no per-record ctypes access)."""
    if n <= 0:
        return []
    import numpy as np
    a = np.frombuffer(out, dtype=_WITNESS_DTYPE, count=n)
    return list(zip(a["space"].tolist(), a["array"].tolist(), a["byte_addr"].tolist(), a["acc_lo"].tolist(),
                    a["acc_hi"].tolist(), a["kind_mask"].tolist()))


def _it(i):
    return (i.lin_block, i.lin_thread, *i.iter, i.access)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Kernel:
    """A kernel descriptor (library owned) plus its current host binding."""

    def __init__(self, text: str):
        h = C.c_void_p()
        b = text.encode()
        _raise(lib().hgrd_load_desc(b, len(b), C.byref(h)))
        self._h = h
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hgrd_free_desc(h)
            self._h = None

    def bind(self, grid, block, params):
        params = tuple(int(p) for p in params)
        arr = (C.c_int64 * max(1, len(params)))(*params)
        b = Binding((C.c_int32 * 3)(*grid), (C.c_int32 * 3)(*block), len(params), arr)
        _raise(lib().hgrd_bind_host_params(self._h, C.byref(b)))
        self.__dict__.pop("_ws_sizes", None)  # sizes follow the binding
        return self

    def info(self) -> tuple:
        """(instances, most keys) of the current binding (no device needed)."""
        n, k = C.c_uint64(), C.c_uint64()
        _raise(lib().hgrd_bound_info(self._h, C.byref(n), C.byref(k)))
        return n.value, k.value

    def workspace_size(self, **opts) -> int:
        key = tuple(sorted(opts.items()))
        cache = self.__dict__.setdefault("_ws_sizes", {})
        if key not in cache:
            n = C.c_size_t()
            o = _opts(**opts)
            _raise(lib().hgrd_workspace_size(self._h, C.byref(o), C.byref(n)))
            cache[key] = n.value
        return cache[key]

    def _out(self, cap: int):
        """A witness buffer of cap records, reused across calls (results copy out of it)."""
        cache = self.__dict__.setdefault("_outs", {})
        buf = cache.get(cap)
        if buf is None:
            buf = cache[cap] = (Witness * max(1, cap))()
        return buf

    def workspace(self, device="cuda", **opts):
        """A device workspace sized for the current binding (reused when large enough)."""
        import torch
        need = self.workspace_size(**opts)
        if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device(device):
            self._ws = None
            self._ws = torch.empty(need, dtype=torch.uint8, device=device)
        return self._ws

    def check(self, cap: int = 1 << 16, stream=None, workspace=None, **opts) -> Result:
        """Exhaustive check; synchronous.  Retries once with a larger raw-witness buffer."""
        for attempt in range(2):
            ws = workspace if workspace is not None else self.workspace(**opts)
            out = self._out(cap)
            v = Verdict()
            o = _opts(**opts)
            rc = lib().hgrd_check(self._h, C.byref(o), C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream),
                                  out, cap, C.byref(v))
            if rc == -6 and workspace is None and attempt == 0:
                # a buffer sized by default was short: retry once with the count the device reported
                st = stats()
                msg = lib().hgrd_last_error().decode(errors="replace")
                if "max_shared_keys" in msg:
                    opts = dict(opts, max_shared_keys=min(0xffffffff, int(st["n_binned_keys"] * 1.25) + 1024))
                    continue
                if st["n_raw_witness"] > opts.get("max_raw_witness", 0):
                    opts = dict(opts, max_raw_witness=int(st["n_raw_witness"] * 1.25) + 1024)
                    continue
            _raise(rc)
            n = min(cap, v.n_witness)
            return Result(bool(v.racy), v.n_witness, tuple(v.n_by_kind), v.n_instances, v.n_keys, v.n_oob,
                          _witness_list(out, n), _wt(v.min_w) if v.racy else None,
                          _it(v.min_x) if v.pair_found else None, _it(v.min_y) if v.pair_found else None,
                          rc == ETRUNCATED, _pairs(v.pair_kind))

    def jit_compile(self, **opts) -> float:
        """Compile (or find cached) the specialised expansion kernels for the
        pipeline `opts` selects; returns the milliseconds spent compiling.
        Later checks of this binding use them (unless flags has NO_JIT)."""
        ms = C.c_double()
        o = _opts(**opts)
        _raise(lib().hgrd_jit_compile(self._h, C.byref(o), C.byref(ms)))
        return ms.value

    def jit_source(self, **opts) -> str:
        """The generated source of the specialised expansion kernels."""
        n = C.c_size_t()
        o = _opts(**opts)
        _raise(lib().hgrd_jit_source(self._h, C.byref(o), None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        _raise(lib().hgrd_jit_source(self._h, C.byref(o), buf, n.value + 1, C.byref(n)))
        return buf.value.decode()

    def check_noalloc(self, cap: int = 1 << 16, stream=None, **opts) -> Result:
        """hgrd_check_noalloc: the check on the library's built-in 64 MiB device
        scratch, for callers that cannot allocate device memory.  No instance
        pair search (min_x / min_y are None)."""
        out = self._out(cap)
        v = Verdict()
        o = _opts(**opts)
        rc = lib().hgrd_check_noalloc(self._h, C.byref(o), _stream_ptr(stream), out, cap, C.byref(v))
        _raise(rc)
        n = min(cap, v.n_witness)
        return Result(bool(v.racy), v.n_witness, tuple(v.n_by_kind), v.n_instances, v.n_keys, v.n_oob,
                      _witness_list(out, n), _wt(v.min_w) if v.racy else None, None, None,
                      rc == ETRUNCATED, _pairs(v.pair_kind))

    def enqueue(self, workspace, stream=None, **opts):
        """Enqueue the device pipeline only (no host synchronisation)."""
        o = _opts(**opts)
        _raise(lib().hgrd_check_enqueue(self._h, C.byref(o), C.c_void_p(workspace.data_ptr()), workspace.numel(),
                                        _stream_ptr(stream)))

    def collect(self, workspace, cap: int = 1 << 16, stream=None, **opts) -> Result:
        out = self._out(cap)
        v = Verdict()
        o = _opts(**opts)
        rc = lib().hgrd_check_collect(self._h, C.byref(o), C.c_void_p(workspace.data_ptr()), workspace.numel(),
                                      _stream_ptr(stream), out, cap, C.byref(v))
        _raise(rc)
        n = min(cap, v.n_witness)
        return Result(bool(v.racy), v.n_witness, tuple(v.n_by_kind), v.n_instances, v.n_keys, v.n_oob,
                      _witness_list(out, n), _wt(v.min_w) if v.racy else None, None, None,
                      rc == ETRUNCATED, _pairs(v.pair_kind))


@dataclass
class ItemResult:
    status: int
    racy: bool
    small: bool
    n_witness: int
    n_by_kind: tuple
    n_instances: int
    n_keys: int
    n_oob: int
    witnesses: list   # first min(witness_cap, n_witness) canonical witnesses
    pairs: dict = None


class Batch:
    """Many bound kernels checked together (hgrd_batch_*).  Keeps its kernels alive."""

    def __init__(self, kernels, small_keys=0, streams=0, witness_cap=64, graph=False, jit=False):
        self.kernels = list(kernels)
        arr = (C.c_void_p * len(self.kernels))(*[k._h.value for k in self.kernels])
        o = BatchOpts(small_keys, streams, witness_cap, (BATCH_GRAPH if graph else 0) | (BATCH_JIT if jit else 0))
        h = C.c_void_p()
        _raise(lib().hgrd_batch_create(arr, len(self.kernels), C.byref(o), C.byref(h)))
        self._h = h
        self.witness_cap = witness_cap
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.hgrd_batch_free(h)
            self._h = None

    def workspace(self, device="cuda"):
        import torch
        n = C.c_size_t()
        _raise(lib().hgrd_batch_workspace_size(self._h, C.byref(n)))
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = None
            self._ws = torch.empty(n.value, dtype=torch.uint8, device=device)
        return self._ws

    def run(self, stream=None):
        ws = self.workspace()
        _raise(lib().hgrd_batch_run(self._h, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))

    def collect(self, stream=None):
        ws = self.workspace()
        n = len(self.kernels)
        v = (ItemVerdict * n)()
        wc = self.witness_cap
        w = (Witness * max(1, n * wc))()
        rc = lib().hgrd_batch_collect(self._h, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream), v, w, wc)
        if rc < 0 and rc != -6:
            _raise(rc)
        out = []
        for i in range(n):
            x = v[i]
            out.append(ItemResult(x.status, bool(x.racy), bool(x.small), x.n_witness, tuple(x.n_by_kind),
                                  x.n_instances, x.n_keys, x.n_oob,
                                  [_wt(w[i * wc + k]) for k in range(x.n_copied)], _pairs(x.pair_kind)))
        return out

    def check(self, stream=None):
        self.run(stream)
        return self.collect(stream)

    def rank_prepare(self):
        """hgrd_batch_rank_prepare: every item's eligible pairs and features (host, once)."""
        _raise(lib().hgrd_batch_rank_prepare(self._h))
        n = C.c_size_t()
        _raise(lib().hgrd_batch_ranked_workspace_size(self._h, C.byref(n)))
        import torch
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = None
            self._ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self._ranked = True

    def check_ranked(self, model, topk: int = 4, min_score: float = float("-inf"), stream=None):
        """hgrd_batch_check_ranked with a ranker's model buffer (a torch uint8
        tensor): (results, stages, info).  Verdicts are exact; an item a
        restricted check found racy lists the races found there."""
        if not getattr(self, "_ranked", False):
            self.rank_prepare()
        ws = self._ws
        n = len(self.kernels)
        v = (ItemVerdict * n)()
        wc = self.witness_cap
        w = (Witness * max(1, n * wc))()
        st = (C.c_uint8 * n)()
        info = BatchRankInfo()
        rc = lib().hgrd_batch_check_ranked(self._h, C.c_void_p(model.data_ptr()) if model is not None else None,
                                           topk, min_score, C.c_void_p(ws.data_ptr()), ws.numel(),
                                           _stream_ptr(stream), v, w, wc, st, C.byref(info))
        if rc < 0 and rc != -6:
            _raise(rc)
        out = []
        for i in range(n):
            x = v[i]
            out.append(ItemResult(x.status, bool(x.racy), bool(x.small), x.n_witness, tuple(x.n_by_kind),
                                  x.n_instances, x.n_keys, x.n_oob,
                                  [_wt(w[i * wc + k]) for k in range(x.n_copied)], _pairs(x.pair_kind)))
        return out, list(st), {k: getattr(info, k) for k, _ in BatchRankInfo._fields_ if k != "pad"}

    def tune(self, stream=None) -> dict:
        ws = self.workspace()
        o = BatchOpts()
        _raise(lib().hgrd_batch_tune(self._h, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream), C.byref(o)))
        return {"small_keys": o.small_keys, "streams": o.streams}


def sort_tune(workspace_bytes: int = 600 << 20, stream=None):
    """hgrd_sort_tune: time the onesweep CTA shapes, keep the fastest; returns (best, [ms...])."""
    import torch
    L = lib()
    L.hgrd_sort_tune.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_float),
                                 C.c_int]
    L.hgrd_sort_tune.restype = C.c_int
    ws = torch.empty(workspace_bytes, dtype=torch.uint8, device="cuda")
    best = C.c_int()
    ms = (C.c_float * 64)()
    _raise(L.hgrd_sort_tune(C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream), C.byref(best), ms, 64))
    n = C.c_int()
    L.hgrd_sort_variant.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    _raise(L.hgrd_sort_variant(-1, None, C.byref(n)))
    return best.value, [ms[i] for i in range(n.value)]


def sort_variant(v: int = -1):
    """Select (v >= 0) or query the onesweep CTA shape of the current device."""
    L = lib()
    L.hgrd_sort_variant.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.hgrd_sort_variant.restype = C.c_int
    cur, n = C.c_int(), C.c_int()
    _raise(L.hgrd_sort_variant(v, C.byref(cur), C.byref(n)))
    return cur.value, n.value


def sort_pass_variant(p: int, v: int = -2) -> int:
    """Select (v >= 0), reset (v == -1) or query (v < -1) the sort shape of key-sort pass p."""
    L = lib()
    L.hgrd_sort_pass_variant.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.hgrd_sort_pass_variant.restype = C.c_int
    cur = C.c_int()
    _raise(L.hgrd_sort_pass_variant(p, v, C.byref(cur)))
    return cur.value


def stats() -> dict:
    s = Stats()
    _raise(lib().hgrd_last_stats(C.byref(s)))
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def last_profile() -> list:
    """[(stage, ms)] of the last check enqueued with flags=PROFILE on this thread."""
    buf = (StageTime * 64)()
    n = C.c_uint32()
    _raise(lib().hgrd_last_profile(buf, 64, C.byref(n)))
    return [(buf[k].name.decode(), buf[k].ms) for k in range(min(64, n.value))]


def check(text: str, binding, cap: int = 1 << 16, **opts) -> Result:
    """Parse, bind and check in one call (binding has .grid, .block, .params)."""
    k = Kernel(text).bind(binding.grid, binding.block, binding.params)
    return k.check(cap=cap, **opts)


def debug_divmod(n: int, d: int, wide: bool):
    q, r = C.c_int64(), C.c_int64()
    _raise(lib().hgrd_debug_divmod(n, d, int(wide), C.byref(q), C.byref(r)))
    return q.value, r.value


def debug_lookback_timeout(stream=None) -> int:
    """hgrd_debug_lookback_timeout: a sort pass whose look-back waits on a tile
    nobody processes; returns the library's status code (HGRD_ETIMEOUT, -8,
    when the bounded wait ran out as it should)."""
    import torch
    L = lib()
    L.hgrd_debug_lookback_timeout.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p]
    L.hgrd_debug_lookback_timeout.restype = C.c_int
    ws = torch.empty(256 << 10, dtype=torch.uint8, device="cuda")
    rc = L.hgrd_debug_lookback_timeout(C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    torch.cuda.synchronize()
    return rc
