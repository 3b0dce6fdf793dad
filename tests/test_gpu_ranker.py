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


def test_gradients_match_fp64_reference():
    import torch
    r = rk.Ranker(seed=5)
    p = r.params().cpu().double().numpy()
    x = _features(1000, 2)
    y = (np.random.default_rng(3).random(1000) < 0.3).astype(np.float32)
    w = np.where(y > 0, 3.0, 1.0).astype(np.float32)
    g = r.grad(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"),
               torch.tensor(w, device="cuda")).cpu().double().numpy()
    _, gr = mlp_ref.loss_and_grad(p, x, y, w, rnd=True)
    cos = float(g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr)))
    assert cos > 0.999, cos
    # per tensor: a bf16 rounding of a gradient product can flip near zero,
    # so compare each tensor's error against its own scale
    o = 0
    for name, n in mlp_ref.SIZES:
        a, b = g[o:o + n], gr[o:o + n]
        assert np.max(np.abs(a - b)) <= 2e-2 * max(np.max(np.abs(b)), 1e-6), name
        o += n


def _corpus(first, n, hi=4.4):
    ws = [workloads.config4(i, hi_exp=hi) for i in range(first, first + n)]
    ks = [hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params) for w in ws]
    return ws, ks


@pytest.fixture(scope="module")
def trained():
    # training kernels: seeds disjoint from the held-out ones below
    ws, ks = _corpus(50000, 400)
    res = hg.Batch(ks, witness_cap=1).check()
    X, y = rk.labelled_pairs(ks, res)
    assert y.sum() > 20 and len(y) > 2000
    r = rk.Ranker(seed=11)
    losses = r.fit(X, y, epochs=6, batch=2048, lr=2e-3)
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
    # how often the ranked stage alone confirms a racy kernel: trained scores
    # against uniformly random scores for the same pairs
    r, _ = trained
    ws, ks = _corpus(70000, 300)
    rng = np.random.default_rng(0)
    hit_t = hit_r = racy = 0
    for w, k in zip(ws, ks):
        if not w.meta["planted"]:
            continue
        racy += 1
        _, info = rk.check_ranked(k, r, topk=2, flags=hg.NO_SMALL)
        hit_t += info["stage"] == 1
        n = info["n_pairs"]
        _, info_r = rk.check_ranked(k, scores=rng.random(n), topk=2, flags=hg.NO_SMALL)
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
    # every eligible pair decides both verdicts (16384 keys: more than one
    # CTA's check, which would skip the ranking altogether)
    from workloads import Binding
    bnd = Binding((128, 1, 1), (64, 1, 1), ())
    for text, racy in ((("kernel c\narray a global 16384\narray r global 16384\n"
                         "access W a ; width 4 ; idx tx + 64*bx\naccess R r ; width 4 ; idx tx\n"), False),
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
