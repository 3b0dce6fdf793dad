"""CPU tests of the ranker's pieces: the FP64 MLP reference is pinned by
central finite differences, and the host feature extractor lists exactly the
pairs the race rule allows."""
import numpy as np

import paper_2604_02106_b300 as hg
from paper_2604_02106_b300 import ranker
import workloads
from oracle import mlp_ref


def test_reference_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.15, mlp_ref.NPARAM)
    x = rng.normal(0, 1, (7, mlp_ref.IN))
    y = (rng.random(7) < 0.4).astype(float)
    w = rng.uniform(0.5, 2.0, 7)
    _, g = mlp_ref.loss_and_grad(p, x, y, w, rnd=False)
    idx = np.concatenate([rng.choice(mlp_ref.NPARAM - 600, 40, replace=False), np.arange(mlp_ref.NPARAM - 600,
                                                                                         mlp_ref.NPARAM, 37)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp_ref.loss_and_grad(p + e, x, y, w, rnd=False)
        lm, _ = mlp_ref.loss_and_grad(p - e, x, y, w, rnd=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def hand_network():
    """A network whose every weight and activation is a small binary fraction
    (exact in bf16), with values worked out by hand below.  Rows are output
    units, columns input units (W[out][in]); W2 is not symmetric, so a
    transposed W2 changes the logits."""
    q = {name: np.zeros(n) for name, n in mlp_ref.SIZES}
    W1 = q["W1"].reshape(mlp_ref.HID, mlp_ref.IN)
    W2 = q["W2"].reshape(mlp_ref.HID, mlp_ref.HID)
    W1[0, 0], W1[0, 1], q["b1"][0] = 1.0, -2.0, 0.5    # h1[0] = relu(x0 - 2 x1 + 0.5)
    W1[1, 2], q["b1"][1] = 3.0, -1.0                   # h1[1] = relu(3 x2 - 1)
    W1[2, 0] = -1.0                                    # h1[2] = relu(-x0)
    W2[0, 0], W2[0, 1], q["b2"][0] = 2.0, 1.0, -0.25   # h2[0] = relu(2 h1[0] + h1[1] - 0.25)
    W2[3, 2] = 1.0                                     # h2[3] = relu(h1[2])
    W2[5, 1], q["b2"][5] = -1.0, 0.5                   # h2[5] = relu(0.5 - h1[1])
    q["W3"][0], q["W3"][3], q["W3"][5], q["b3"][0] = 1.5, -2.0, 0.5, -0.75
    p = np.concatenate([q[name].ravel() for name, _ in mlp_ref.SIZES])
    x = np.zeros((2, mlp_ref.IN))
    x[0, :3] = (1.0, 0.5, 2.0)
    x[1, :3] = (-2.0, 1.0, 0.25)
    x[:, 95] = 7.0  # an input no weight reads
    # sample 0: h1 = (0.5, 5, 0), h2[0] = 5.75, h2[3] = 0, h2[5] = 0 -> z = 1.5*5.75 - 0.75
    # sample 1: h1 = (0, 0, 2),  h2[0] = 0, h2[3] = 2, h2[5] = 0.5 -> z = -4 + 0.25 - 0.75
    return p, x, np.array([7.875, -4.5])


def test_reference_forward_on_a_hand_worked_network():
    p, x, z_hand = hand_network()
    for rnd in (True, False):
        z, (_, h1, h2) = mlp_ref.forward(p, x, rnd=rnd)
        assert list(z) == list(z_hand)
        assert list(h1[0, :3]) == [0.5, 5.0, 0.0] and list(h1[1, :3]) == [0.0, 0.0, 2.0]
        assert (h2[0, 0], h2[0, 3], h2[0, 5]) == (5.75, 0.0, 0.0)
        assert (h2[1, 0], h2[1, 3], h2[1, 5]) == (0.0, 2.0, 0.5)
        assert not h1[:, 3:].any() and np.count_nonzero(h2) == 3


def test_reference_loss_is_weighted_binary_cross_entropy():
    # the textbook form -[y log s + (1 - y) log(1 - s)], s = 1 / (1 + e^-z),
    # weighted and divided by the weight sum
    import math
    p, x, z = hand_network()
    y, w = np.array([1.0, 0.0]), np.array([1.0, 3.0])
    s = [1 / (1 + math.exp(-v)) for v in z]
    want = (-w[0] * math.log(s[0]) - w[1] * math.log(1 - s[1])) / 4.0
    loss, g = mlp_ref.loss_and_grad(p, x, y, w, rnd=False)
    assert abs(loss - want) <= 1e-12 * abs(want)
    # d loss / d b3 = sum_i w_i (s_i - y_i) / sum w
    o = mlp_ref.NPARAM - 1
    assert abs(g[o] - (w[0] * (s[0] - 1) + w[1] * s[1]) / 4.0) <= 1e-12
    # d loss / d W3[3] = sum_i w_i (s_i - y_i) h2_i[3] / sum w: only sample 1 has h2[3] = 2
    assert abs(g[o - 256 + 3] - 3.0 * s[1] * 2.0 / 4.0) <= 1e-12
    # a logit fixed by the output bias alone (all weights zero)
    q = np.zeros(mlp_ref.NPARAM)
    for b3, yy, want in ((0.0, 1.0, math.log(2)), (0.0, 0.0, math.log(2)), (40.0, 1.0, math.exp(-40.0)),
                         (40.0, 0.0, 40.0 + math.exp(-40.0)), (-40.0, 1.0, 40.0 + math.exp(-40.0)),
                         (-40.0, 0.0, math.exp(-40.0))):
        q[-1] = b3
        loss, _ = mlp_ref.loss_and_grad(q, x[:1], np.array([yy]), None, rnd=True)
        assert abs(loss - want) <= 1e-12 * max(1.0, want), (b3, yy, loss, want)


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e38, 1e-30])
    r = mlp_ref.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] / 3.0e38 - 1) < 2 ** -8 and abs(r[5] / 1e-30 - 1) < 2 ** -8


def test_pair_features_list_the_eligible_pairs():
    w = workloads.plain_random(0)
    k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
    f, ab = ranker.pair_features(k)
    assert f.shape == (len(ab), 96) and np.isfinite(f).all()
    # accesses: array and kind per access line, pair rule of Sec. 6.1
    acc = [l.split(" ; ")[0].split()[1:] for l in w.text.splitlines() if l.startswith("access")]
    want = []
    for a in range(len(acc)):
        for b in range(a, len(acc)):
            if acc[a][1] == acc[b][1] and not (acc[a][0] == "R" and acc[b][0] == "R"):
                want.append((a, b))
    assert ab == want
    f2, ab2 = ranker.pair_features(k)
    assert ab2 == ab and (f2 == f).all()


def test_pairs_in_disjoint_barrier_intervals():
    # one block's instances in different barrier intervals are ordered
    # (Sec. 6.1, block barrier): in shared memory such a pair is never
    # eligible; in global memory it stays eligible for the inter-block kind
    text = ("kernel iv\nloop k 4\narray S shared 256\narray G global 256\n"
            "access W S ; width 4 ; iv 0 ; idx tx\n"          # 0
            "access R S ; width 4 ; iv 1 ; idx tx + 1\n"      # 1: no writer in interval 1
            "access W S ; width 4 ; iv 2*k + 2 ; idx tx\n"    # 2: intervals 2..8
            "access R S ; width 4 ; iv 5 ; idx tx + 2\n"      # 3: meets 2's range
            "access W G ; width 4 ; iv 0 ; idx tx\n"          # 4
            "access R G ; width 4 ; iv 1 ; idx tx + 1\n")     # 5
    k = hg.Kernel(text).bind((2, 1, 1), (32, 1, 1), ())
    _, ab = ranker.pair_features(k)
    # (0, 0) and (2, 2): each thread writes its own element of the block's
    # copy (thread-tile pruning); (4, 4): both blocks write G[tx]
    assert ab == [(2, 3), (4, 4), (4, 5)]


def test_block_pair_pruning_examples():
    # per-block hulls of affine global indexes: blocks writing their own
    # slices cannot race across blocks (inter kind pruned, intra kept); a
    # shared slice keeps it; a pair pruned of every kind leaves the list
    def pairs(text, grid=(4, 1, 1), block=(64, 1, 1)):
        k = hg.Kernel(text).bind(grid, block, ())
        f, ab = ranker.pair_features(k)
        return {p: (int(r[64 + 3]), int(r[64 + 4])) for p, r in zip(ab, f)}
    base = "kernel b\nloop i 2\narray G global 4096\n"
    # one element per thread (thread-tile pruning): no pair at all
    assert pairs(base + "access W G ; width 4 ; idx bx*64 + tx\n") == {}
    assert pairs(base + "access W G ; width 4 ; idx bx*128 + tx*2 + i\n") == {}
    assert pairs(base + "access W G ; width 4 ; idx bx*64 + tx*2 + i\n") == {(0, 0): (1, 1)}  # thread 32 meets block 1
    # two elements per thread, the write reaching the next thread's read
    assert pairs(base + "access W G ; width 4 ; idx (bx*64 + tx)*2 + i + 1\naccess R G ; width 4 ; idx bx*128 + tx*2\n") == \
        {(0, 1): (1, 1)}
    assert pairs(base + "access W G ; width 4 ; idx bx*64 + tx + i\n") == {(0, 0): (1, 1)}  # hulls meet
    assert pairs(base + "access W G ; width 4 ; idx bx*65 + tx + i\n") == {(0, 0): (0, 1)}
    assert pairs(base + "access W G ; width 4 ; idx tx\n") == {(0, 0): (1, 1)}
    assert pairs(base + "access W G ; width 4 ; idx bx*64 + tx\naccess R G ; width 4 ; iv 1 ; idx bx*64 + tx\n") == \
        {}  # every thread its own element, in both intervals
    assert pairs(base + "access W G ; width 16 ; idx bx*16 + tx / 4\n") == {(0, 0): (1, 1)}  # a division: not pruned
    # byte ranges that never meet: [0, 128) and [128, 256) by the remainders'
    # bounds (each access alone races: threads 0 and 32 share an element)
    two = "access W G ; width 4 ; idx tx % 32\naccess W G ; width 4 ; idx 32 + tx % 32\n"
    assert pairs(base + two) == {(0, 0): (1, 1), (1, 1): (1, 1)}
    # one element further and they meet (threads 32 and 63 against 0)
    assert pairs(base + two.replace("32 + tx", "31 + tx")) == {(0, 0): (1, 1), (0, 1): (1, 1), (1, 1): (1, 1)}
    # different widths: [0, 128) against bytes [128, 256) of 16-byte elements
    assert (0, 1) not in pairs(base + "access W G ; width 4 ; idx tx % 32\naccess R G ; width 16 ; idx 8 + tx % 8\n")
    assert (0, 1) in pairs(base + "access W G ; width 4 ; idx tx % 32\naccess R G ; width 16 ; idx 7 + tx % 8\n")


def test_block_pair_pruning_against_brute_force():
    # every global-memory pair whose inter-block kind was pruned (listed
    # without it, or not listed at all: byte ranges that never meet, or
    # threads that own disjoint elements) has no two instances of different
    # blocks on one granule (independent enumeration of tests/brute.py)
    import brute
    pruned = unlisted = 0
    for seed in range(120):
        w = workloads.random_tiny(4000 + seed, max_instances=400)
        k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
        f, ab = ranker.pair_features(k)
        inter = {p: r[64 + 3] for p, r in zip(ab, f)}
        d = brute.parse(w.text)
        inst, _ = brute.instances(d, w.binding)
        acc = d["acc"]
        for a in range(len(acc)):
            for b in range(a, len(acc)):
                if acc[a]["array"] != acc[b]["array"] or d["arrays"][acc[a]["array"]]["shared"]:
                    continue
                ka, kb = acc[a]["kind"], acc[b]["kind"]
                if (ka == "R" and kb == "R") or (ka == "A" and kb == "A"):
                    continue  # loads, and atomics (pruned by their scopes, not by addresses)
                if inter.get((a, b), 0):
                    continue
                pruned += 1
                unlisted += (a, b) not in inter
                xa = [x for x in inst if x["acc"] == a]
                xb = [x for x in inst if x["acc"] == b]
                for x in xa:
                    for y in xb:
                        assert x["blk"] == y["blk"] or not (x["gran"] & y["gran"]), (seed, a, b)
    assert pruned > 20 and 0 < unlisted < pruned, (pruned, unlisted)


def test_pair_rule_keeps_every_racing_pair():
    # the library's pair rule (with interval, block-pair and thread-tile
    # pruning) may drop only pairs that never race: every racy access pair of
    # the oracle is eligible; kernels whose threads own private regions lose
    # those pairs
    import oracle
    dropped = 0
    ws = [workloads.random_tiny(6000 + s, max_instances=3000) for s in range(80)] + \
         [workloads.config4(i, hi_exp=3.8) for i in range(60)]
    for w in ws:
        k = hg.Kernel(w.text).bind(w.binding.grid, w.binding.block, w.binding.params)
        _, ab = ranker.pair_features(k)
        o = oracle.check(w.text, w.binding, pair=False)
        assert {(x[3], x[4]) for x in o.witnesses} <= set(ab), w.name
        if w.name.startswith("c4") or "corpus" in w.text.splitlines()[0]:
            acc = [l for l in w.text.splitlines() if l.startswith("access")]
            for a, line in enumerate(acc):
                if line.startswith("access W D") and "gid*SPAN + off" in line and (a, a) not in ab:
                    dropped += 1
    assert dropped > 20


def test_block_pair_pruning_work_budget():
    # past the sweep budget (2^21 block hulls) the pair keeps its inter-block
    # kind: pruning is an optimisation, never required for exactness
    text = "kernel g\narray G global 4*64*4194304\naccess W G ; width 4 ; idx bx*64 + tx\n"
    for gx, inter in ((1 << 20, 0), ((1 << 21) + 1, 1)):
        # two threads (ty 0 and 1) share each element: no thread-tile pruning
        k = hg.Kernel(text).bind((gx, 1, 1), (64, 2, 1), ())
        f, ab = ranker.pair_features(k)
        assert ab == [(0, 0)] and int(f[0][64 + 3]) == inter and int(f[0][64 + 4]) == 1
