"""GPU ranker: forward and gradients of the hand-written MLP kernels against
the FP64 CPU reference, training, and the ranked check against the oracle."""
import numpy as np
import pytest

import oracle
from oracle import mlp_ref
import paper_2604_02106_b300 as hg
from paper_2604_02106_b300 import ranker as rk
import workloads

pytestmark = pytest.mark.gpu


def _features(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1, (n, 96)).astype(np.float32)


def test_forward_matches_fp64_reference():
    import torch
    r = rk.Ranker(seed=3)
    p = r.params().cpu().double().numpy()
    x = _features(300, 1)
    z = r.predict(torch.tensor(x, device="cuda")).cpu().double().numpy()
    zr, _ = mlp_ref.forward(p, x, rnd=True)
    # the GPU sums in fp32 in another order; bf16 operands agree exactly
    assert np.max(np.abs(z - zr)) <= 1e-3 * max(1.0, np.max(np.abs(zr)))


def test_forward_and_loss_on_the_hand_worked_network():
    # every operand and activation exact in bf16, so the kernels must give
    # the hand-worked logits exactly (see the CPU pin of the reference)
    import math
    import torch
    from test_ranker_cpu import hand_network
    p, x, z_hand = hand_network()
    r = rk.Ranker(seed=0)
    r.load(p)
    z = r.predict(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().double().numpy()
    assert list(z) == list(z_hand)
    y, w = np.array([1.0, 0.0]), np.array([1.0, 3.0])
    loss = r.train_step(torch.tensor(x, dtype=torch.float32, device="cuda"),
                        torch.tensor(y, dtype=torch.float32, device="cuda"),
                        torch.tensor(w, dtype=torch.float32, device="cuda"), lr=0.0, weight_decay=0.0)
    s = [1 / (1 + math.exp(-v)) for v in z_hand]
    want = (-math.log(s[0]) - 3 * math.log(1 - s[1])) / 4
    assert abs(float(loss.item()) - want) <= 1e-6 * want


def _sum_bound(g, gr, base, flip, name):
    """Element-wise comparison of a GPU gradient (fp32 sums of bf16 products)
    with the fp64 reference that rounds at the same bf16 points.  `base`
    bounds the error of the fp32 sums (k terms: k * 2^-24 * sum|terms|) plus
    the error their inputs carry in from fp32 arithmetic before them.  A bf16
    rounding of an activation gradient can also land on the neighbouring
    bf16 value, since its fp32 input differs from the reference's in the
    last bits; `flip` bounds what such flips can move.  Every element must
    stay within both allowances together, and the elements beyond `base`
    alone (the rounding flips) must be rare."""
    err = np.abs(g - gr)
    base = base + 1e-30
    assert np.all(err <= base + flip), (name, float(np.max(err / (base + flip))))
    flips = int(np.count_nonzero(err > base))
    assert flips <= max(4, 0.01 * err.size), (name, flips, err.size)


def test_gradients_match_fp64_reference():
    import torch
    r = rk.Ranker(seed=5)
    p = r.params().cpu().double().numpy()
    n = 1000
    x = _features(n, 2)
    y = (np.random.default_rng(3).random(n) < 0.3).astype(np.float32)
    w = np.where(y > 0, 3.0, 1.0).astype(np.float32)
    g = r.grad(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"),
               torch.tensor(w, device="cuda")).cpu().double().numpy()
    _, gr = mlp_ref.loss_and_grad(p, x, y, w, rnd=True)
    # the magnitudes of every gradient sum's terms, from the reference's own
    # intermediates (bf16 at inputs, weights, hidden activations and
    # activation gradients)
    u = 2.0 ** -24
    q = mlp_ref.split(p)
    z, (xb, h1, h2) = mlp_ref.forward(p, x, rnd=True)
    wd = w.astype(np.float64)
    sig = 1 / (1 + np.exp(-z))
    dz = wd * (sig - y) / wd.sum()
    # the logit is an fp32 sum of 257 terms; the output gradient an fp32
    # sigmoid minus the label (a few units of 2^-24 absolute)
    dlogit = (257 + 8) * u * (np.abs(h2) @ np.abs(q["W3"]) + abs(q["b3"][0]))
    edz = wd / wd.sum() * (sig * (1 - sig) * dlogit + 8 * u)
    w2b = mlp_ref.bf16(q["W2"])
    dh2 = mlp_ref.bf16(np.where(h2 > 0, np.outer(dz, q["W3"]), 0))
    dh1 = mlp_ref.bf16(np.where(h1 > 0, dh2 @ w2b, 0))
    # a first-layer term moves with a flip of dh1 itself or of a dh2 it sums
    a1 = np.abs(dh1) + np.where(h1 > 0, np.abs(dh2) @ np.abs(w2b), 0)
    f = (n + 8) * u
    fl = 2.0 ** -7
    terms = {
        "W3": (f * (np.abs(h2).T @ np.abs(dz)) + np.abs(h2).T @ edz, np.zeros(256)),
        "b3": (np.array([f * np.abs(dz).sum() + edz.sum()]), np.zeros(1)),
        "W2": (f * (np.abs(dh2).T @ np.abs(h1)).ravel(), fl * (np.abs(dh2).T @ np.abs(h1)).ravel()),
        "b2": (f * np.abs(dh2).sum(0), fl * np.abs(dh2).sum(0)),
        "W1": (f * (np.abs(dh1).T @ np.abs(xb)).ravel(), fl * (a1.T @ np.abs(xb)).ravel()),
        "b1": (f * np.abs(dh1).sum(0), fl * a1.sum(0)),
    }
    o = 0
    for name, size in mlp_ref.SIZES:
        base, flip = terms[name]
        assert base.size == size and flip.size == size
        _sum_bound(g[o:o + size], gr[o:o + size], base, flip, name)
        o += size


def _corpus(first, n, hi=4.4):
    ws = [workloads.config4(i, hi_exp=hi) for i in range(first, first + n)]
    ks = [hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params) for w in ws]
    return ws, ks


@pytest.fixture(scope="module")
def trained():
    # training kernels: seeds disjoint from the held-out ones below
    ws, ks = _corpus(50000, 1000)
    res = hg.Batch(ks, witness_cap=1).check()
    X, y = rk.labelled_pairs(ks, res)
    assert y.sum() > 200 and len(y) - y.sum() > 1000
    r = rk.Ranker(seed=11)
    losses = r.fit(X, y, epochs=30, batch=256, lr=2e-3)
    return r, losses


def test_training_lowers_the_loss(trained):
    _, losses = trained
    k = max(1, len(losses) // 6)
    assert np.mean(losses[-k:]) < 0.7 * np.mean(losses[:k])


def test_ranked_verdicts_match_the_oracle(trained):
    r, _ = trained
    ws, ks = _corpus(60000, 80)
    for w, k in zip(ws, ks):
        o = oracle.check(w.text, w.binding)
        res, info = rk.check_ranked(k, r, topk=4)
        assert res.racy == o.racy
        full = {x[:5]: x[5] for x in o.witnesses}
        for x in res.witnesses:  # each witness is a real race of the kernel
            assert x[:5] in full and (x[5] & ~full[x[:5]]) == 0
        if not o.racy:
            assert info["stage"] == 2


def test_trained_network_beats_random_order(trained):
    # how often the ranked stage alone confirms a racy kernel from its single
    # top pair: trained scores against uniformly random scores for the same
    # pairs (random order finds about 69% of them on this corpus)
    r, _ = trained
    ws, ks = _corpus(70000, 300)
    rng = np.random.default_rng(0)
    hit_t = hit_r = racy = 0
    for w, k in zip(ws, ks):
        if not w.meta["planted"]:
            continue
        racy += 1
        _, info = rk.check_ranked(k, r, topk=1, flags=hg.NO_SMALL)
        hit_t += info["stage"] == 1
        n = info["n_pairs"]
        _, info_r = rk.check_ranked(k, scores=rng.random(n), topk=1, flags=hg.NO_SMALL)
        hit_r += info_r["stage"] == 1
    assert racy >= 40
    assert hit_t > hit_r + 0.15 * racy, (hit_t, hit_r, racy)


def test_restricted_check_small_enough_runs_in_one_cta():
    # 8192 keys in all, 4096 of the two checked accesses: the restricted check
    # runs whole in one CTA and finds exactly the oracle's races of that pair
    text = ("kernel r\narray a global 65536\narray b global 65536\n"
            "access W a ; width 4 ; idx tx + 64*bx\naccess R a ; width 4 ; idx tx + 1 + 64*bx\n"
            "access W b ; width 4 ; idx tx\naccess R b ; width 4 ; idx 2*tx + bx\n")
    from workloads import Binding
    bnd = Binding((32, 1, 1), (64, 1, 1), ())
    k = hg.Kernel(text).bind(bnd.grid, bnd.block, bnd.params)
    o = oracle.check(text, bnd, cap=1 << 20)
    sel = lambda m: [x for x in o.witnesses if (m >> x[3]) & 1 and (m >> x[4]) & 1]
    g = k.check(cap=1 << 20, only_accesses=0b1100)  # 128 witnesses
    assert hg.stats()["small"] == 1 and g.witnesses == sel(0b1100)
    # 2047 witnesses: more than one CTA keeps, so the full set comes from the
    # device-wide pipeline; stopping at the first races keeps the CTA's
    g = k.check(cap=1 << 20, only_accesses=0b0011)
    assert hg.stats()["small"] == 0 and g.witnesses == sel(0b0011)
    g = k.check(cap=1 << 20, only_accesses=0b0011, flags=hg.STOP_FIRST)
    assert hg.stats()["small"] == 1 and g.racy and g.witnesses
    full = {x[:5]: x[5] for x in sel(0b0011)}
    assert all(x[:5] in full and (x[5] & ~full[x[:5]]) == 0 for x in g.witnesses)
    k.check(cap=1 << 20)
    assert hg.stats()["small"] == 0


def test_ranked_check_of_few_pairs_is_one_restricted_check():
    # at most top-k eligible pairs: no scores, one restricted check covering
    # every eligible pair decides both verdicts (12288 and 16384 keys: more
    # than one CTA's check, which would skip the ranking altogether).  The
    # race-free write is injective only under its guard, so no bind-time
    # test drops its pair
    from workloads import Binding
    bnd = Binding((128, 1, 1), (64, 1, 1), ())
    for text, racy in ((("kernel c\narray a global 16384\narray r global 16384\n"
                         "access W a ; width 4 ; idx tx/2 + 32*bx ; if tx % 2 == 0\n"
                         "access R r ; width 4 ; idx tx\n"), False),
                       (("kernel d\narray a global 16384\narray r global 16384\n"
                         "access W a ; width 4 ; idx tx\naccess R r ; width 4 ; idx tx\n"), True)):
        k = hg.Kernel(text).bind(bnd.grid, bnd.block, bnd.params)
        res, info = rk.check_ranked(k, None, scores=[0.0], topk=4)
        assert res.racy == racy == oracle.check(text, bnd).racy
        assert info["n_pairs"] == 1 and info["access_mask"] == 1
        assert info["stage"] == (1 if racy else 2) and info["keys_full"] == 0
    # a kernel whose full check runs in one CTA is not ranked
    k = hg.Kernel(text).bind((4, 1, 1), (64, 1, 1), ())
    res, info = rk.check_ranked(k, None, scores=[0.0], topk=4)
    assert res.racy and info["n_pairs"] == 0 and info["stage"] == 2


def test_ranked_verdicts_on_all_heldout_kernels(trained):
    # the 2,000 held-out kernels of the learned-ranker workload: every ranked
    # verdict equals the oracle's (stored by tests/golden/c5_heldout_verdicts.py)
    import torch
    from test_gpu_configs import heldout_verdicts
    r, _ = trained
    rows = heldout_verdicts()
    ks = [hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
          for w in (workloads.config4(row["item"], hi_exp=6.0) for row in rows)]
    ws = torch.empty(max(rk.ranked_workspace_size(k) for k in ks), dtype=torch.uint8, device="cuda")
    stage1 = 0
    for row, k in zip(rows, ks):
        res, info = rk.check_ranked(k, r, topk=4, workspace=ws, cap=1 << 10)
        assert res.racy == row["racy"], row["item"]
        stage1 += info["stage"] == 1
    assert stage1 > 0


def test_ranked_batch_on_all_heldout_kernels(trained):
    # the batched ranked form: one inference over every pair of the 2,000
    # held-out kernels, restricted checks of the ranked large items, whole
    # checks of what they leave open; every verdict equals the oracle's and
    # every reported race is one of the oracle's
    from test_gpu_configs import heldout_verdicts
    r, _ = trained
    rows = heldout_verdicts()
    ks = [hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
          for w in (workloads.config4(row["item"], hi_exp=6.0) for row in rows)]
    b = hg.Batch(ks, witness_cap=16)
    res, stages, info = b.check_ranked(r.model, topk=4, min_score=0.0)
    reruns = 0
    for row, k, x, st in zip(rows, ks, res, stages):
        if x.status == -6:
            x = k.check(cap=16, flags=hg.NO_PAIR)
            reruns += 1
        assert x.racy == row["racy"], row["item"]
        full = {tuple(int(v) for v in p.split(",")): m for p, m in row["pairs"].items()}
        for pair, m in x.pairs.items():
            assert pair in full and (m & ~full[pair]) == 0, row["item"]
        if st in (0, 2):  # a whole check: the whole verdict
            assert x.n_witness == row["n_witness"] and x.pairs == full
    assert info["n_pairs"] > 1000 and info["ranked"] > 0 and info["confirmed"] > 0
    assert reruns < 100
