"""Pairwise brute force of the race definition, for tiny launches.

Independent of both the oracle and the GPU library: its own tokenizer and
evaluator (Python ints, C truncating division), and no bucketing at all — it
compares every pair of live, in-bounds instances directly:

  * two instances conflict on every granule their byte ranges share, if they
    access the same array (and, for shared memory, come from the same block:
    each block owns its copy);
  * the pair is a race of type inter-block (different blocks), intra-block
    (same block and barrier interval, different warps) or intra-warp (same
    block, interval, warp and warp interval, different threads) — Sec. 2,
    Table 2, and Sec. 5.2 for the warp barrier;
  * two loads never race, nor do two device-scope atomics; two atomics of
    block scope or wider never race inside one block (Sec. 6.1, Appendix A);
  * two accesses both guarded by acquire-release at the same address do not
    race, if the guards' narrower scope covers the race type: device for
    inter-block, block or device otherwise (Sec. 6.5, Table 2, Appendix A).

Used only to pin the CPU oracle on launches of at most a few hundred instances.
"""
from __future__ import annotations

import itertools
import math
import re

_TOK = re.compile(r"\s*(?:(\d+)|([A-Za-z_]\w*)|(<=|>=|==|!=|[-+*/%()<>]))")


def _tokens(s):
    pos, out = 0, []
    s = s.strip()
    while pos < len(s):
        m = _TOK.match(s, pos)
        if not m or m.end() == pos:
            raise ValueError(f"cannot tokenize {s[pos:]!r}")
        if m.group(1) is not None:
            out.append(int(m.group(1)))
        else:
            out.append(m.group(2) or m.group(3))
        pos = m.end()
    return out


def _cdiv(a, b):
    q = abs(a) // abs(b)
    return q if (a >= 0) == (b > 0) else -q


def _cmod(a, b):
    return a - b * _cdiv(a, b)


class _Expr:
    """Recursive-descent parse into nested tuples; evaluated against a dict."""

    def __init__(self, text, lets):
        self.t = _tokens(text)
        self.i = 0
        self.lets = lets
        self.tree = self.sum()
        if self.i != len(self.t):
            raise ValueError(f"trailing tokens in {text!r}")

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def sum(self):
        x = self.prod()
        while self.peek() in ("+", "-"):
            op = self.t[self.i]
            self.i += 1
            x = (op, x, self.prod())
        return x

    def prod(self):
        x = self.unary()
        while self.peek() in ("*", "/", "%"):
            op = self.t[self.i]
            self.i += 1
            x = (op, x, self.unary())
        return x

    def unary(self):
        if self.peek() == "-":
            self.i += 1
            return ("neg", self.unary())
        tok = self.t[self.i]
        self.i += 1
        if tok == "(":
            x = self.sum()
            assert self.t[self.i] == ")"
            self.i += 1
            return x
        if isinstance(tok, int):
            return ("num", tok)
        if tok in self.lets:
            return self.lets[tok]
        return ("var", tok)


def _ev(t, env):
    k = t[0]
    if k == "num":
        return t[1]
    if k == "var":
        return env[t[1]]
    if k == "neg":
        return -_ev(t[1], env)
    a, b = _ev(t[1], env), _ev(t[2], env)
    if k == "+":
        return a + b
    if k == "-":
        return a - b
    if k == "*":
        return a * b
    if b <= 0:
        raise ValueError("divisor is not positive")
    return _cdiv(a, b) if k == "/" else _cmod(a, b)


_OPS = {"<": lambda a, b: a < b, "<=": lambda a, b: a <= b, ">": lambda a, b: a > b,
        ">=": lambda a, b: a >= b, "==": lambda a, b: a == b, "!=": lambda a, b: a != b}


def _cond(text, lets):
    for op in ("<=", ">=", "==", "!=", "<", ">"):
        if op in text:
            l, r = text.split(op, 1)
            return (op, _Expr(l, lets).tree, _Expr(r, lets).tree)
    raise ValueError(text)


def parse(text):
    d = {"params": [], "loops": [], "arrays": [], "acc": [], "asserts": [], "lets": {}}
    for raw in text.splitlines():
        line = raw.split("#")[0].strip()
        if not line:
            continue
        head, _, rest = line.partition(" ")
        if head == "kernel":
            continue
        if head == "param":
            d["params"] += rest.split()
        elif head == "loop":
            v, b = rest.split(None, 1)
            d["loops"].append((v, _Expr(b, d["lets"]).tree))
        elif head == "array":
            f = [x.strip() for x in rest.split(";")]
            name, space, size = f[0].split(None, 2)
            gran = None
            for x in f[1:]:
                k, val = x.split()
                assert k == "granule"
                gran = int(val)
            d["arrays"].append({"name": name, "shared": space == "shared",
                                "bytes": _Expr(size, d["lets"]).tree, "granule": gran})
        elif head == "let":
            n, e = rest.split("=", 1)
            d["lets"][n.strip()] = _Expr(e, d["lets"]).tree
        elif head == "assert":
            d["asserts"].append(_cond(rest, d["lets"]))
        elif head == "access":
            f = [x.strip() for x in rest.split(";")]
            kind, arr = f[0].split()
            a = {"kind": kind, "array": [x["name"] for x in d["arrays"]].index(arr), "iv": ("num", 0),
                 "wv": ("num", 0), "guards": [], "scope": "device", "sync": None, "syncscope": "device"}
            for x in f[1:]:
                k, _, body = x.partition(" ")
                if k == "width":
                    a["width"] = int(body)
                elif k == "iv":
                    a["iv"] = _Expr(body, d["lets"]).tree
                elif k == "wv":
                    a["wv"] = _Expr(body, d["lets"]).tree
                elif k == "idx":
                    a["idx"] = _Expr(body, d["lets"]).tree
                elif k == "if":
                    a["guards"].append(_cond(body, d["lets"]))
                elif k == "scope":
                    a["scope"] = body.strip()
                elif k == "sync":
                    sarr, sexpr = body.strip().split(None, 1)
                    a["sync"] = ([x["name"] for x in d["arrays"]].index(sarr), _Expr(sexpr, d["lets"]).tree)
                    assert not d["arrays"][a["sync"][0]]["shared"], "a sync array must be global"
                elif k == "syncscope":
                    a["syncscope"] = body.strip()
            d["acc"].append(a)
    for k, arr in enumerate(d["arrays"]):
        if arr["granule"] is None:
            ws = [a["width"] for a in d["acc"] if a["array"] == k]
            arr["granule"] = math.gcd(*ws) if ws else 4
    return d


def instances(d, binding):
    """All live, in-bounds instances: dicts with blk, thr, warp, it, acc, iv, granules."""
    env = {n: v for n, v in zip(d["params"], binding.params)}
    for c, n in zip("xyz", binding.grid):
        env["gd" + c] = n
    for c, n in zip("xyz", binding.block):
        env["bd" + c] = n
    for op, l, r in d["asserts"]:
        if not _OPS[op](_ev(l, env), _ev(r, env)):
            raise AssertionError("host assert violated")
    bounds = [max(0, _ev(b, env)) for _, b in d["loops"]]
    sizes = [_ev(a["bytes"], env) for a in d["arrays"]]
    gx, gy, gz = binding.grid
    bx_, by_, bz_ = binding.block
    out, n_oob = [], 0
    for bz, by, bx, tz, ty, tx in itertools.product(range(gz), range(gy), range(gx),
                                                    range(bz_), range(by_), range(bx_)):
        for it in itertools.product(*[range(b) for b in bounds]):
            e = dict(env, tx=tx, ty=ty, tz=tz, bx=bx, by=by, bz=bz)
            for (v, _), val in zip(d["loops"], it):
                e[v] = val
            for ai, a in enumerate(d["acc"]):
                if not all(_OPS[op](_ev(l, e), _ev(r, e)) for op, l, r in a["guards"]):
                    continue
                off = _ev(a["idx"], e) * a["width"]
                arr = d["arrays"][a["array"]]
                if off < 0 or off + a["width"] > sizes[a["array"]]:
                    n_oob += 1
                    continue
                g = arr["granule"]
                thr = tx + ty * bx_ + tz * bx_ * by_
                out.append({"blk": bx + by * gx + bz * gx * gy, "thr": thr, "warp": thr // 32,
                            "it": tuple(it) + (0,) * (4 - len(it)), "acc": ai, "iv": _ev(a["iv"], e),
                            "wv": _ev(a["wv"], e),
                            "sync": None if a["sync"] is None else (a["sync"][0], _ev(a["sync"][1], e)),
                            "array": a["array"], "shared": arr["shared"], "g": g,
                            "gran": set(range(off // g, (off + a["width"]) // g))})
    return out, n_oob


def race_kind(d, x, y):
    """Kind bit (1 inter-block, 2 intra-block, 4 intra-warp) of one instance pair, 0 if none."""
    if x["array"] != y["array"]:
        return 0
    if x["shared"] and x["blk"] != y["blk"]:
        return 0
    if x["blk"] == y["blk"] and x["thr"] == y["thr"]:
        return 0
    ka, kb = d["acc"][x["acc"]]["kind"], d["acc"][y["acc"]]["kind"]
    if ka == "R" and kb == "R":
        return 0
    if x["blk"] != y["blk"]:
        kind = 1
    elif x["iv"] != y["iv"]:
        return 0
    elif x["warp"] != y["warp"]:
        kind = 2
    elif x["wv"] != y["wv"]:  # a syncwarp between them
        return 0
    else:
        kind = 4
    if ka == "A" and kb == "A":
        block_scoped = "block" in (d["acc"][x["acc"]]["scope"], d["acc"][y["acc"]]["scope"])
        if kind != 1 or not block_scoped:
            return 0
    if x["sync"] is not None and x["sync"] == y["sync"]:  # one acquire-release address
        block_scoped = "block" in (d["acc"][x["acc"]]["syncscope"], d["acc"][y["acc"]]["syncscope"])
        if kind != 1 or not block_scoped:
            return 0
    return kind


def check(text, binding):
    """Witness dict {(space, array, byte_addr, lo, hi): mask}, canonical pair, counts."""
    d = parse(text)
    inst, n_oob = instances(d, binding)
    wit = {}
    best = {}
    for i in range(len(inst)):
        x = inst[i]
        for j in range(i + 1, len(inst)):
            y = inst[j]
            k = race_kind(d, x, y)
            if not k:
                continue
            common = x["gran"] & y["gran"]
            if not common:
                continue
            lo, hi = (x, y) if x["acc"] <= y["acc"] else (y, x)
            for gr in common:
                key = (1 if x["shared"] else 0, x["array"], gr * x["g"], lo["acc"], hi["acc"])
                wit[key] = wit.get(key, 0) | k
                kx = (lo["blk"], lo["thr"]) + lo["it"]
                ky = (hi["blk"], hi["thr"]) + hi["it"]
                if lo["acc"] == hi["acc"] and ky < kx:
                    kx, ky = ky, kx
                cand = (kx, ky)
                if key not in best or cand < best[key]:
                    best[key] = cand
    n_keys = sum(len(x["gran"]) for x in inst)
    n_inst = math.prod(binding.grid) * math.prod(binding.block) * len(d["acc"])
    env = {n: v for n, v in zip(d["params"], binding.params)}
    for c, n in zip("xyz", binding.grid):
        env["gd" + c] = n
    for c, n in zip("xyz", binding.block):
        env["bd" + c] = n
    for _, b in d["loops"]:
        n_inst *= max(0, _ev(b, env))
    keys = sorted(wit)
    min_pair = best[keys[0]] if keys else None
    return {"witnesses": [k + (wit[k],) for k in keys], "n_keys": n_keys, "n_oob": n_oob,
            "n_instances": n_inst, "min_pair": min_pair}
