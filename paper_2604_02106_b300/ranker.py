"""Learned pair ranker: the MLP of libhgrd (hgrd_mlp_*) and the ranked check.

Argument marshalling only; the features, the network's forward and backward
passes, the optimizer and the checks all run inside libhgrd.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import (Kernel, Result, Witness, Verdict, CheckOpts, _opts, _raise, _stream_ptr, _wt, _pairs, lib,
               ETRUNCATED, HgrdError)

IN, HID, NPARAM = 96, 256, 90881
MAXPAIRS = 32 * 33 // 2


class RankInfo(C.Structure):
    _fields_ = [("n_pairs", C.c_uint32), ("stage", C.c_uint32), ("access_mask", C.c_uint32), ("pad", C.c_uint32),
                ("keys_ranked", C.c_uint64), ("keys_full", C.c_uint64), ("ms_rank", C.c_float),
                ("pad2", C.c_float)]


def _setup():
    L = lib()
    if getattr(L, "_ranker_ready", False):
        return L
    vp, sz, f32p = C.c_void_p, C.c_size_t, C.POINTER(C.c_float)
    L.hgrd_pair_features.argtypes = [vp, f32p, C.POINTER(C.c_uint8), C.c_uint32, C.POINTER(C.c_uint32)]
    L.hgrd_mlp_model_bytes.restype = sz
    L.hgrd_mlp_model_bytes.argtypes = []
    L.hgrd_mlp_workspace_bytes.restype = sz
    L.hgrd_mlp_workspace_bytes.argtypes = [C.c_uint32]
    L.hgrd_mlp_init.argtypes = [vp, C.c_uint64, vp]
    L.hgrd_mlp_predict.argtypes = [vp, vp, C.c_uint32, vp, vp, sz, vp]
    L.hgrd_mlp_grad.argtypes = [vp, vp, vp, vp, C.c_float, C.c_uint32, vp, sz, vp]
    L.hgrd_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_float, C.c_uint32, C.c_float, C.c_float, C.c_uint32, vp,
                                      sz, vp, vp]
    L.hgrd_mlp_sync_bf16.argtypes = [vp, vp]
    L.hgrd_ranked_workspace_size.argtypes = [vp, C.POINTER(CheckOpts), C.POINTER(sz)]
    L.hgrd_check_ranked.argtypes = [vp, C.POINTER(CheckOpts), vp, f32p, C.c_uint32, C.c_float, vp, sz, vp,
                                    C.POINTER(Witness), C.c_uint64, C.POINTER(Verdict), C.POINTER(RankInfo)]
    for f in ["hgrd_pair_features", "hgrd_mlp_init", "hgrd_mlp_predict", "hgrd_mlp_grad", "hgrd_mlp_train_step",
              "hgrd_mlp_sync_bf16", "hgrd_ranked_workspace_size", "hgrd_check_ranked"]:
        getattr(L, f).restype = C.c_int
    L._ranker_ready = True
    return L


def pair_features(kernel: Kernel):
    """(features [n, 96] float32, [(a, b), ...]) of the eligible pairs of a bound kernel."""
    L = _setup()
    out = np.zeros((MAXPAIRS, IN), dtype=np.float32)
    ab = np.zeros(2 * MAXPAIRS, dtype=np.uint8)
    n = C.c_uint32()
    rc = L.hgrd_pair_features(kernel._h, out.ctypes.data_as(C.POINTER(C.c_float)),
                              ab.ctypes.data_as(C.POINTER(C.c_uint8)), MAXPAIRS, C.byref(n))
    _raise(rc)
    k = n.value
    return out[:k].copy(), [(int(ab[2 * i]), int(ab[2 * i + 1])) for i in range(k)]


class Ranker:
    """Model buffer on the GPU plus the hgrd_mlp_* calls."""

    def __init__(self, seed: int = 0, device="cuda"):
        import torch
        L = _setup()
        self.model = torch.empty(L.hgrd_mlp_model_bytes(), dtype=torch.uint8, device=device)
        self._ws = None
        self.step = 0
        _raise(L.hgrd_mlp_init(C.c_void_p(self.model.data_ptr()), seed, _stream_ptr(None)))

    def _workspace(self, n):
        import torch
        need = _setup().hgrd_mlp_workspace_bytes(n)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.model.device)
        return self._ws

    def params(self):
        return self.model[:NPARAM * 4].view(__import__("torch").float32)

    def grads(self):
        off = (NPARAM * 4 + 255) // 256 * 256
        return self.model[off:off + NPARAM * 4].view(__import__("torch").float32)

    def load(self, flat):
        """Set the FP32 parameters (and their BF16 copies) from a flat vector."""
        import torch
        self.params().copy_(torch.as_tensor(flat, dtype=torch.float32, device=self.model.device))
        _raise(_setup().hgrd_mlp_sync_bf16(C.c_void_p(self.model.data_ptr()), _stream_ptr(None)))

    def predict(self, x):
        import torch
        x = x.contiguous().float()
        n = x.shape[0]
        z = torch.empty(n, dtype=torch.float32, device=x.device)
        ws = self._workspace(n)
        _raise(_setup().hgrd_mlp_predict(C.c_void_p(self.model.data_ptr()), C.c_void_p(x.data_ptr()), n,
                                         C.c_void_p(z.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                                         _stream_ptr(None)))
        return z

    def grad(self, x, y, w=None):
        x, y = x.contiguous().float(), y.contiguous().float()
        n = x.shape[0]
        ws = self._workspace(n)
        wsum = float(w.sum()) if w is not None else float(n)
        _raise(_setup().hgrd_mlp_grad(C.c_void_p(self.model.data_ptr()), C.c_void_p(x.data_ptr()),
                                      C.c_void_p(y.data_ptr()), C.c_void_p(w.data_ptr()) if w is not None else None,
                                      wsum, n, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(None)))
        return self.grads()

    def train_step(self, x, y, w=None, lr=1e-3, weight_decay=1e-4):
        import torch
        x, y = x.contiguous().float(), y.contiguous().float()
        n = x.shape[0]
        ws = self._workspace(n)
        wsum = float(w.sum()) if w is not None else float(n)
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        _raise(_setup().hgrd_mlp_train_step(C.c_void_p(self.model.data_ptr()), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(y.data_ptr()),
                                            C.c_void_p(w.data_ptr()) if w is not None else None, wsum, n, lr,
                                            weight_decay, self.step, C.c_void_p(ws.data_ptr()), ws.numel(),
                                            _stream_ptr(None), C.c_void_p(loss.data_ptr())))
        self.step += 1
        return loss

    def fit(self, X, y, epochs=4, batch=8192, lr=2e-3, weight_decay=1e-4, seed=0, pos_weight=None):
        """Minibatch training on (X [n, 96], y [n]); positives weighted to balance the classes."""
        import torch
        X = torch.as_tensor(X, dtype=torch.float32, device=self.model.device)
        y = torch.as_tensor(y, dtype=torch.float32, device=self.model.device)
        npos = float(y.sum())
        pw = pos_weight if pos_weight is not None else max(1.0, (len(y) - npos) / max(npos, 1.0))
        w = torch.where(y > 0.5, torch.tensor(pw, device=y.device), torch.tensor(1.0, device=y.device))
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(len(y), generator=g).to(y.device)
            for i in range(0, len(y), batch):
                idx = perm[i:i + batch]
                losses.append(self.train_step(X[idx], y[idx], w[idx], lr, weight_decay))
        return torch.cat(losses).cpu().numpy() if losses else np.zeros(0)


def ranked_workspace_size(kernel: Kernel) -> int:
    L = _setup()
    o = _opts()
    n = C.c_size_t()
    _raise(L.hgrd_ranked_workspace_size(kernel._h, C.byref(o), C.byref(n)))
    return n.value


def check_ranked(kernel: Kernel, ranker: Ranker | None = None, scores=None, topk: int = 4, cap: int = 1 << 16,
                 stream=None, min_score: float = float("-inf"), workspace=None, **opts):
    """hgrd_check_ranked: (Result, info dict).  With neither a ranker nor scores
    only the full check runs (stopping at its first race).  `opts` as for
    Kernel.check (e.g. flags=NO_SMALL ranks kernels one CTA would check)."""
    import torch
    L = _setup()
    o = _opts(**opts)
    ws = workspace
    if ws is None:
        n = C.c_size_t()
        _raise(L.hgrd_ranked_workspace_size(kernel._h, C.byref(o), C.byref(n)))
        ws = getattr(kernel, "_rws", None)
        if ws is None or ws.numel() < n.value:
            ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
            kernel._rws = ws
    out = kernel._out(cap)  # reused across calls, like the plain check's
    v = Verdict()
    info = RankInfo()
    sc = None
    if scores is not None:
        sc = np.ascontiguousarray(scores, dtype=np.float32)
    rc = L.hgrd_check_ranked(kernel._h, C.byref(o), C.c_void_p(ranker.model.data_ptr()) if ranker else None,
                             sc.ctypes.data_as(C.POINTER(C.c_float)) if sc is not None else None, topk,
                             min_score, C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream), out, cap, C.byref(v),
                             C.byref(info))
    _raise(rc)
    k = min(cap, v.n_witness)
    res = Result(bool(v.racy), v.n_witness, tuple(v.n_by_kind), v.n_instances, v.n_keys, v.n_oob,
                 [_wt(out[i]) for i in range(k)], _wt(v.min_w) if v.racy else None, None, None,
                 rc == ETRUNCATED, _pairs(v.pair_kind))
    return res, {"stage": info.stage, "n_pairs": info.n_pairs, "access_mask": info.access_mask,
                 "keys_ranked": info.keys_ranked, "keys_full": info.keys_full, "ms_rank": info.ms_rank}


def labelled_pairs(kernels, batch_results):
    """Training rows: features of every eligible pair, label 1 when the exact
    check (a batch result with its racy-pair matrices) reports the pair racy."""
    X, y = [], []
    for k, r in zip(kernels, batch_results):
        if r.status != 0:
            continue
        f, ab = pair_features(k)
        if not len(ab):
            continue
        X.append(f)
        y.append(np.array([1.0 if (a, b) in r.pairs else 0.0 for a, b in ab], dtype=np.float32))
    if not X:
        return np.zeros((0, IN), np.float32), np.zeros(0, np.float32)
    return np.concatenate(X), np.concatenate(y)
