"""Pins for the CPU oracle: facts that do not come from the oracle itself.

Levenshtein: textbook values, metric axioms, closed forms, brute force over
all alignments.  NW: brute force pins both the optimal cost and the exact
tie-broken alignment; rescoring and de-gapping.  Partition: a closed-form
line metric and the invariants Alg. 1 implies.  Merge: a worked example by
hand and the postconditions of section "Merging".  MLP: finite differences,
a library bf16 cast, the first Adam step in closed form.
"""
import itertools
import os
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_2601_15458_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore")


def _golden_lev():
    rows = []
    with open(os.path.join(GOLDEN, "lev_textbook.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b, d = line.split()
            rows.append((b"" if a == "~" else a.encode(), b"" if b == "~" else b.encode(), int(d)))
    return rows


@pytest.mark.parametrize("a,b,d", _golden_lev())
def test_lev_textbook(a, b, d):
    assert oracle.lev(a, b) == d
    assert oracle.lev(b, a) == d


def _rand_dna(rng, n):
    return rng.choice(list(b"ACGT"), size=n).astype(np.uint8).tobytes()


def test_lev_metric_axioms():
    rng = np.random.default_rng(11)
    seqs = [_rand_dna(rng, int(rng.integers(0, 40))) for _ in range(25)]
    for x in seqs:
        assert oracle.lev(x, x) == 0
    for x, y in itertools.combinations(seqs, 2):
        d = oracle.lev(x, y)
        assert d == oracle.lev(y, x)
        assert abs(len(x) - len(y)) <= d <= max(len(x), len(y))
        if x != y:
            assert d > 0
    for x, y, z in itertools.islice(itertools.combinations(seqs, 3), 400):
        assert oracle.lev(x, z) <= oracle.lev(x, y) + oracle.lev(y, z)


def test_lev_closed_forms():
    rng = np.random.default_rng(12)
    for _ in range(20):
        b = _rand_dna(rng, int(rng.integers(0, 60)))
        k = int(rng.integers(0, len(b) + 1))
        assert oracle.lev(b"", b) == len(b)
        assert oracle.lev(b[:k], b) == len(b) - k       # prefix
        assert oracle.lev(b[k:], b) == k                # suffix
        # Hamming bound: equal lengths, d <= number of mismatching positions
        c = _rand_dna(rng, len(b))
        assert oracle.lev(b, c) <= sum(x != y for x, y in zip(b, c))
    # disjoint alphabets: d = max(m, n)
    assert oracle.lev(b"AAAA", b"CCCCCC") == 6


def test_lev_bruteforce_small():
    rng = np.random.default_rng(13)
    for _ in range(60):
        a = _rand_dna(rng, int(rng.integers(0, 7)))
        b = _rand_dna(rng, int(rng.integers(0, 7)))
        best = min(oracle.rescore(a, b, ops)[0] for ops in oracle.brute_alignments(a, b))
        assert oracle.lev(a, b) == best


def test_brute_alignment_count_is_delannoy():
    # number of alignments of strings of lengths m, n is the Delannoy number D(m, n)
    delannoy = {(1, 1): 3, (2, 2): 13, (3, 3): 63, (2, 3): 25, (6, 6): 8989}
    for (m, n), D in delannoy.items():
        assert len(oracle.brute_alignments(b"A" * m, b"C" * n)) == D


@pytest.mark.parametrize("costs", [(0, 1, 1), (0, 3, 2), (-1, 2, 3)])
def test_nw_bruteforce_exact_alignment(costs):
    rng = np.random.default_rng(14 + sum(costs))
    for _ in range(80):
        alpha = list(b"ACG-")
        a = rng.choice(alpha, size=int(rng.integers(0, 7))).astype(np.uint8).tobytes()
        b = rng.choice(alpha, size=int(rng.integers(0, 7))).astype(np.uint8).tobytes()
        score, ops = oracle.nw(a, b, *costs)
        bcost, bops = oracle.brute_best(a, b, *costs)
        assert score == bcost
        assert ops == bops


def test_nw_rescore_and_degap():
    rng = np.random.default_rng(15)
    for _ in range(40):
        a = _rand_dna(rng, int(rng.integers(0, 80)))
        b = _rand_dna(rng, int(rng.integers(0, 80)))
        score, ops = oracle.nw(a, b)
        cost, ra, rb = oracle.rescore(a, b, ops)
        assert cost == score
        assert ra.replace(b"-", b"") == a and rb.replace(b"-", b"") == b
        assert len(ra) == len(rb) == len(ops)
        assert score == oracle.lev(a, b)                  # unit costs: NW cost == f


def test_nw_worked_example():
    # kitten -> sitting: k/s substitution, e/i substitution, insert g
    score, ops = oracle.nw(b"kitten", b"sitting")
    assert score == 3
    assert ops == b"XMMMXMI"
    # empty operands
    assert oracle.nw(b"", b"ACG") == (3, b"III")
    assert oracle.nw(b"AC", b"") == (2, b"DD")


def test_pairs_versions_match_single():
    ds = synth.small_dna(seed=1, n=12)
    pairs = synth.all_pairs(ds.n)
    d = oracle.lev_pairs(ds.arena, ds.offs, pairs, nthreads=3)
    for (x, y), v in zip(pairs, d):
        assert v == oracle.lev(ds.seq(x), ds.seq(y))
    score, ops, off, ln = oracle.nw_pairs(ds.arena, ds.offs, pairs[:20], nthreads=2)
    for p, (x, y) in enumerate(pairs[:20]):
        s, o = oracle.nw(ds.seq(x), ds.seq(y))
        assert s == score[p] and o == ops[off[p]:off[p] + ln[p]].tobytes()


# ---------------------------------------------------------------------------
# Partition (Alg. 1) and merge
# ---------------------------------------------------------------------------

def test_partition_line_metric_closed_form():
    # "A"*k for k = 1..7: f(x, y) = |len x - len y|, so every step of Alg. 1
    # follows from the line.  Derived by hand:
    #   root {1..7}: medoid 4; l = argmax |4-x| -> tie 1, 7 -> smallest index -> 1;
    #   r = argmax |1-x| = 7; L = {x : |x-1| <= |x-7|} = {1,2,3,4}, R = {5,6,7}
    #   {1,2,3,4}: medoid sums 6,4,4,6 -> 2; l = 4; r = 1; L = {3,4}, R = {1,2}
    #   {5,6,7}: medoid 6; l = 5 (tie 5,7); r = 7; L = {5,6}, R = {7}
    seqs = [b"A" * k for k in range(1, 8)]
    nodes = oracle.partition(seqs)
    got = [(nd["members"], nd["center"]) for nd in nodes]
    idx = lambda *ks: [k - 1 for k in ks]  # noqa: E731
    assert got[0] == (idx(1, 2, 3, 4, 5, 6, 7), 3)
    assert got[1] == (idx(1, 2, 3, 4), 1)
    assert got[2] == (idx(5, 6, 7), 5)
    assert got[3] == (idx(3, 4), 2)
    assert got[4] == (idx(1, 2), 0)
    assert got[5] == (idx(5, 6), 4)
    assert got[6] == (idx(7), 6)


def _check_tree(nodes, n):
    leaves = [nd for nd in nodes if nd["left"] < 0]
    assert sorted(x for nd in leaves for x in nd["members"]) == list(range(n))
    for nd in leaves:
        assert len(nd["members"]) == 1
    for nd in nodes:
        if nd["left"] >= 0:
            L, R = nodes[nd["left"]]["members"], nodes[nd["right"]]["members"]
            assert L and R
            assert sorted(L + R) == nd["members"]
            assert nd["center"] in nd["members"]


def test_partition_invariants_random():
    ds = synth.small_dna(seed=3, n=24)
    nodes = oracle.partition(ds.seqs())
    _check_tree(nodes, ds.n)
    assert len(nodes) == 2 * ds.n - 1


def test_medoid_sample_rule():
    assert oracle.medoid_candidates(list(range(10))) == list(range(10))
    c = oracle.medoid_candidates(list(range(1000, 0, -1)))
    assert len(c) == 256 and c[0] == 1 and c == sorted(c)
    assert c[1] == 1 + (1000 // 256)


def test_merge_worked_example():
    # seqs AC, A: root medoid tie -> index 0 (AC); l = 1 (A); r = 0;
    # L = {1}, R = {0}; NW(A, AC) = 1 with script M then I (derived by hand);
    # the left block gains a gap column at the end.
    rows, order, merges = oracle.merge_tree([b"AC", b"A"], oracle.partition([b"AC", b"A"]))
    assert order == [1, 0]
    assert rows == [b"A-", b"AC"]
    assert merges[0] == (1, b"MI")


def test_merge_postconditions():
    ds = synth.small_dna(seed=4, n=20)
    seqs = ds.seqs()
    nodes = oracle.partition(seqs)
    rows, order, merges = oracle.merge_tree(seqs, nodes)
    assert sorted(order) == list(range(ds.n))
    w = len(rows[0])
    assert all(len(r) == w for r in rows)
    assert w >= max(len(s) for s in seqs)
    for r, s in zip(rows, order):
        assert r.replace(b"-", b"") == seqs[s]
    assert len(merges) == ds.n - 1


@pytest.mark.parametrize("maker", [lambda: synth.SeqSet.from_list([b"A" * k for k in range(1, 8)]),
                                   lambda: synth.small_dna(seed=1),
                                   lambda: synth.protein_families(seed=3, n_fam=3, per_fam=30)[0]])
def test_level_batched_partition_and_merge_equal_plain(maker):
    """The level-batched oracle (distances and alignments of one tree level
    gathered into one batch) gives node for node the tree of the per-pair
    partition and row for row its merge, scripts and scores included."""
    seqs = maker().seqs()
    plain = oracle.partition(seqs)
    assert oracle.partition_levels(seqs, nthreads=3) == plain
    assert oracle.merge_tree_levels(seqs, plain, nthreads=2) == oracle.merge_tree(seqs, plain)


def test_level_batched_single_step_with_sampled_medoid():
    """max_levels=1 is one application of Alg. 1: on 300 sequences the
    medoid comes from the 256-member sample, as in partition_step."""
    seqs = synth.tree_dna(seed=8, n=300, root_len=160).seqs()
    nodes = oracle.partition_levels(seqs, max_levels=1)
    c, l, r, L, R = oracle.partition_step(list(range(len(seqs))), oracle._default_dist(seqs))
    assert len(nodes) == 3 and nodes[0]["center"] == c
    assert nodes[1]["members"] == L and nodes[2]["members"] == R


# ---------------------------------------------------------------------------
# features and network
# ---------------------------------------------------------------------------

def test_kmer_counts_against_counter():
    rng = np.random.default_rng(16)
    for L in (0, 3, 4, 5, 57):
        s = _rand_dna(rng, L)
        c = oracle.kmer_counts(s)
        ref = Counter(s[i:i + 4] for i in range(len(s) - 3))
        assert c.sum() == max(0, L - 3)
        for kmer, cnt in ref.items():
            v = int("".join(str(b"ACGT".index(ch)) for ch in kmer), 4)
            assert c[v] == cnt
    assert oracle.kmer_counts(b"AAAA")[0] == 1
    assert oracle.kmer_counts(b"ACGT")[0b00011011] == 1


def test_kmer_l1_lower_bound():
    # one edit changes at most 4 windows out and 4 in: ||c_a - c_b||_1 <= 8 f(a, b)
    rng = np.random.default_rng(17)
    for _ in range(30):
        a = _rand_dna(rng, int(rng.integers(4, 120)))
        b = _rand_dna(rng, int(rng.integers(4, 120)))
        l1 = np.abs(oracle.kmer_counts(a) - oracle.kmer_counts(b)).sum()
        assert l1 <= 8 * oracle.lev(a, b)


def test_pair_feature_closed_forms():
    # AAAAAAA has 4 windows AAAA, AAAAA has 2: the only bin differs by 2, and
    # its feature is 2^2 / ((7 + 5) / 2) = 2/3 (squared, not 2 / 6)
    f = oracle.pair_feature(oracle.kmer_counts(b"AAAAAAA"), oracle.kmer_counts(b"AAAAA"), 7, 5)
    assert f[0] == oracle.bf16_round(np.float32(4.0) / np.float32(6.0))
    assert np.count_nonzero(f) == 1
    # a sequence against itself: all zero; the feature is symmetric in (a, b)
    rng = np.random.default_rng(19)
    a, b = _rand_dna(rng, 200), _rand_dna(rng, 180)
    ca, cb = oracle.kmer_counts(a), oracle.kmer_counts(b)
    assert not oracle.pair_feature(ca, ca, 200, 200).any()
    np.testing.assert_array_equal(oracle.pair_feature(ca, cb, 200, 180), oracle.pair_feature(cb, ca, 180, 200))
    # one substitution inside a run of distinct windows moves 4 windows out and
    # 4 in (8 bins off by one when all 8 are distinct): the sum is 8 / len
    s = bytearray(b"ACGTTGCAAGCTTCGAATGC")
    t = bytearray(s)
    t[10] = ord("A") if s[10] != ord("A") else ord("C")
    cs, ct = oracle.kmer_counts(bytes(s)), oracle.kmer_counts(bytes(t))
    assert np.abs(cs - ct).max() == 1 and np.abs(cs - ct).sum() == 8
    f = oracle.pair_feature(cs, ct, 20, 20)
    assert f.sum() == pytest.approx(8 / 20, rel=1e-2)


def test_bf16_round_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(18)
    x = np.concatenate([rng.standard_normal(1000).astype(np.float32) * 100,
                        np.float32([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, np.pi, 0.0, -2.5])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(x), ref)
    assert oracle.bf16_round(np.float32(1 + 2 ** -8)) == 1.0          # tie to even
    assert oracle.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def _params(rng, scale=0.2):
    return dict(W1=rng.standard_normal((256, 128)) * scale / 4, b1=rng.standard_normal(128) * 0.1,
                W2=rng.standard_normal((128, 64)) * scale, b2=rng.standard_normal(64) * 0.1,
                W3=rng.standard_normal((64, 1)) * scale, b3=rng.standard_normal(1) * 0.1)


def test_mlp_gradients_finite_differences(monkeypatch):
    # with bf16 rounding replaced by the identity the network is smooth almost
    # everywhere; central differences in float64 pin the analytic backward pass
    monkeypatch.setattr(oracle, "bf16_round", lambda x: np.asarray(x, dtype=np.float64))
    rng = np.random.default_rng(19)
    P = _params(rng)
    X = np.abs(rng.standard_normal((16, 256)))
    # targets kept at least 0.5 away from the prediction: no pinball kink in reach
    y0, _ = oracle.mlp_forward(P, X)
    y = y0 + np.where(rng.random(16) < 0.5, -1.0, 1.0) * (0.5 + rng.random(16))

    def loss_of(p):
        yh, _ = oracle.mlp_forward(p, X)
        return oracle.pinball_loss(yh, y)[0]

    yh, cache = oracle.mlp_forward(P, X)
    _, dy = oracle.pinball_loss(yh, y)
    G = oracle.mlp_backward(cache, dy)
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k].reshape(-1)[idx] += h
            Pm[k].reshape(-1)[idx] -= h
            fd = (loss_of(Pp) - loss_of(Pm)) / (2 * h)
            assert abs(fd - G[k].reshape(-1)[idx]) <= 1e-6 + 1e-4 * abs(fd), (k, idx)


def test_pinball_closed_form():
    loss, dy = oracle.pinball_loss(np.array([0.0, 2.0]), np.array([1.0, 1.0]), tau=0.9)
    assert loss == pytest.approx((0.9 * 1.0 + 0.1 * 1.0) / 2)
    np.testing.assert_allclose(dy, [-0.9 / 2, 0.1 / 2])


def _one_path(w1=1.0, b1=0.0, w2=1.0, b2=0.0, w3=1.0, b3=0.0):
    """Parameters whose only live path is x0 -> h1_0 -> h2_0 -> y."""
    P = dict(W1=np.zeros((256, 128)), b1=np.zeros(128), W2=np.zeros((128, 64)), b2=np.zeros(64),
             W3=np.zeros((64, 1)), b3=np.array([b3]))
    P["W1"][0, 0], P["b1"][0], P["W2"][0, 0], P["b2"][0], P["W3"][0, 0] = w1, b1, w2, b2, w3
    return P


@pytest.mark.parametrize("site,x0,kw,expect", [
    # the input is rounded to bf16: 1 + 2^-9 -> 1, so z1 = 1 - 15/16 = 2^-4
    # (unrounded: 2^-4 + 2^-9, itself a bf16 value, would come through)
    ("input", 1 + 2 ** -9, dict(b1=-0.9375), 2 ** -4),
    # W1, W2 and W3 are rounded to bf16 the same way
    ("weight1", 1.0, dict(w1=1 + 2 ** -9, b1=-0.9375), 2 ** -4),
    ("weight2", 1.0, dict(w2=1 + 2 ** -9, b2=-0.9375), 2 ** -4),
    ("weight3", 1.0, dict(w3=1 + 2 ** -9, b3=-0.9375), 2 ** -4),
    # h1 = bf16(1 + 2^-8 + 2^-10) = 1 + 2^-7 (above the half step 2^-8);
    # z2 = h1 - 1 = 2^-7 (unrounded h1 would give 2^-8 + 2^-10, a bf16 value)
    ("hidden1", 1.0, dict(b1=2 ** -8 + 2 ** -10, b2=-1.0), 2 ** -7),
    # h2 = bf16(1 + 2^-8 + 2^-10) = 1 + 2^-7, y = h2 - 1
    ("hidden2", 1.0, dict(b2=2 ** -8 + 2 ** -10, b3=-1.0), 2 ** -7),
    # ReLU: a negative pre-activation contributes nothing
    ("relu", 1.0, dict(b1=-2.0, b3=0.25), 0.25),
])
def test_mlp_forward_rounding_sites(site, x0, kw, expect):
    """Each place the forward pass rounds to bf16, shown by a hand-worked
    one-path network whose output changes if that rounding is left out."""
    X = np.zeros((1, 256))
    X[0, 0] = np.float32(x0)
    y, _ = oracle.mlp_forward(_one_path(**kw), X)
    assert y[0] == expect


def test_forward_tie_enumeration_finds_planted_flip():
    """The rounding-choice enumeration used by the GPU forward check: a row
    built to sit exactly on a bf16 boundary yields both outcomes, a row away
    from every boundary only the oracle's."""
    from mlp_ties import forward_candidates
    x = np.zeros(256)
    x[0] = 1.0
    cands, ties = forward_candidates(_one_path(b1=2 ** -8, b2=-0.5), x)   # z1 halfway between 1 and 1 + 2^-7
    assert ties == 1 and sorted(cands) == [0.5, 0.5 + 2 ** -7]
    cands, ties = forward_candidates(_one_path(b1=2 ** -6, b2=-0.5), x)
    assert ties == 0 and cands == [0.5 + 2 ** -6]


def test_adam_second_step_closed_form():
    # two steps from zero moments: m2 = (1 - b1)(b1 g1 + g2), v2 = (1 - b2)(b2 g1^2 + g2^2),
    # bias-corrected m2 / (1 - b1^2) = (b1 g1 + g2) / (1 + b1), v2 / (1 - b2^2) = (b2 g1^2 + g2^2) / (1 + b2)
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 1e-8
    g1 = np.array([0.5, -2.0, 1e-3, 0.3])
    g2 = np.array([0.5, 2.0, -1e-3, 0.0])
    p = {"w": np.zeros(4)}
    m = {"w": np.zeros(4)}
    v = {"w": np.zeros(4)}
    p1, m, v = oracle.adam_step(p, {"w": g1}, m, v, t=1, lr=lr)
    p2, m, v = oracle.adam_step(p1, {"w": g2}, m, v, t=2, lr=lr)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    step1 = -lr * g1 / (np.abs(g1) + eps)
    np.testing.assert_allclose(p2["w"], step1 - lr * mh / (np.sqrt(vh) + eps), rtol=1e-12, atol=1e-15)
    # a constant gradient keeps the step at lr (bias correction exact at t = 2)
    np.testing.assert_allclose(p2["w"][0], -2 * lr * 0.5 / (0.5 + eps), rtol=1e-12)
    # a reversed gradient: m2 / (1 - b1^2) = -g1 / 19, v2 / (1 - b2^2) = g1^2
    np.testing.assert_allclose(p2["w"][1] - p1["w"][1], -lr * (2.0 / 19) / (2.0 + eps), rtol=1e-12)
    np.testing.assert_allclose(m["w"], (1 - b1) * (b1 * g1 + g2), rtol=1e-12)
    np.testing.assert_allclose(v["w"], (1 - b2) * (b2 * g1 ** 2 + g2 ** 2), rtol=1e-12)


def test_adam_first_step_closed_form():
    # from zero moments the bias-corrected first step is -lr * g / (|g| + eps)
    g = {"w": np.array([0.5, -2.0, 1e-3])}
    p = {"w": np.zeros(3)}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    out, _, _ = oracle.adam_step(p, g, m, v, t=1, lr=0.01)
    np.testing.assert_allclose(out["w"], -0.01 * g["w"] / (np.abs(g["w"]) + 1e-8))


# ---------------------------------------------------------------------------
# alignment quality metrics (section "Evaluation")
# ---------------------------------------------------------------------------

def test_msa_metrics_hand_example():
    # rows AC-T / ACGT / A--T of ACT, ACGT, AT:
    # gaps 1, 0, 2 of 4 per row -> mean 25%;
    # compared columns (no gap in either row): pair 01 cols 0,1,3; pair 02 cols 0,3;
    # pair 12 cols 0,3 -> 7 columns, all equal -> p-score 0;
    # Hamming 1, 1, 2 against Levenshtein 1, 1, 2 -> distortion 1.
    rows = [b"AC-T", b"ACGT", b"A--T"]
    seqs = [b"ACT", b"ACGT", b"AT"]
    pct, p, dist, n = oracle.msa_metrics(rows, seqs)
    assert pct == pytest.approx(25.0) and p == 0.0 and dist == pytest.approx(1.0)
    assert n == dict(gaps=3, compared=7, mismatched=0, pairs=3)


def test_msa_metrics_mismatch_and_stretch():
    # A-CT / AG-T: the only compared columns are 0 and 3 (both equal);
    # Hamming 2 (columns 1, 2) against f(ACT, AGT) = 1 -> distortion 2.
    pct, p, dist, n = oracle.msa_metrics([b"A-CT", b"AG-T"], [b"ACT", b"AGT"])
    assert pct == pytest.approx(25.0) and p == 0.0 and dist == pytest.approx(2.0)
    # ACGT / AGGA: 4 compared columns, 2 differ -> p-score 50; Hamming 2 = f -> 1
    pct, p, dist, n = oracle.msa_metrics([b"ACGT", b"AGGA"], [b"ACGT", b"AGGA"])
    assert pct == 0.0 and p == pytest.approx(50.0) and dist == pytest.approx(1.0)
    assert n["compared"] == 4 and n["mismatched"] == 2


def test_msa_metrics_distortion_at_least_one():
    # an MSA restricted to two rows is an alignment of the two sequences, so
    # its Hamming distance (gap-gap columns dropped) is at least their
    # Levenshtein distance; a pairwise optimal alignment gives exactly 1
    rng = np.random.default_rng(20)
    seqs = [_rand_dna(rng, int(rng.integers(5, 30))) for _ in range(6)]
    a, b = seqs[0], seqs[1]
    score, ops = oracle.nw(a, b)
    ra, rb = bytearray(), bytearray()
    i = j = 0
    for op in ops:
        if op in b"MX":
            ra.append(a[i]); rb.append(b[j]); i += 1; j += 1
        elif op == ord("D"):
            ra.append(a[i]); rb.append(ord("-")); i += 1
        else:
            ra.append(ord("-")); rb.append(b[j]); j += 1
    _, _, dist, _ = oracle.msa_metrics([bytes(ra), bytes(rb)], [a, b])
    assert dist == pytest.approx(1.0)
    # a poor alignment of the same pair: everything against gaps
    rows = [a + b"-" * len(b), b"-" * len(a) + b]
    _, _, dist, _ = oracle.msa_metrics(rows, [a, b])
    assert dist == pytest.approx((len(a) + len(b)) / oracle.lev(a, b))


# ---------------------------------------------------------------------------
# affine gaps (Gotoh)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("costs", [(0, 1, 10, 1), (0, 3, 2, 1), (-1, 2, 3, 2), (0, 1, 0, 1)])
def test_nw_affine_bruteforce(costs):
    """Minimum affine cost over every alignment (rescored run by run) equals
    the DP score, and the DP's own script rescores to it."""
    rng = np.random.default_rng(sum(costs) + 50)
    for _ in range(60):
        a = rng.choice(list(b"ACG-"), size=int(rng.integers(0, 7))).astype(np.uint8).tobytes()
        b = rng.choice(list(b"ACG-"), size=int(rng.integers(0, 7))).astype(np.uint8).tobytes()
        best = min(oracle.rescore_affine(a, b, ops, *costs) for ops in oracle.brute_alignments(a, b))
        score, ops = oracle.nw_affine(a, b, *costs)
        assert score == best
        assert oracle.rescore_affine(a, b, ops, *costs) == score


def test_nw_affine_reduces_to_linear():
    # with open = 0 a run of L gaps costs L * ext: the linear model, same script
    rng = np.random.default_rng(51)
    for _ in range(40):
        a, b = _rand_dna(rng, int(rng.integers(0, 40))), _rand_dna(rng, int(rng.integers(0, 40)))
        assert oracle.nw_affine(a, b, 0, 1, 0, 1) == oracle.nw(a, b, 0, 1, 1)


def test_nw_affine_closed_forms():
    # one substitution (1) is cheaper than a deletion plus an insertion (2 x 11)
    assert oracle.nw_affine(b"ACGTACGT", b"ACGAACGT", 0, 1, 10, 1) == (1, b"MMMXMMMM")
    # one gap run of 3 costs open + 3 ext = 13, less than 3 substitutions at 5
    assert oracle.nw_affine(b"AAACCCGGG", b"AAAGGG", 0, 5, 10, 1) == (13, b"MMMDDDMMM")
    assert oracle.nw_affine(b"ACGT", b"AGGT", 0, 1, 10, 1) == (1, b"MXMM")
    assert oracle.nw_affine(b"", b"ACG", 0, 1, 10, 1) == (13, b"III")


def test_nw_affine_substitution_table_bruteforce():
    """With a substitution table the DP score is the minimum over every
    alignment rescored with that table, and its own script rescores to it
    (random integer tables, some entries negative like BLOSUM62 costs)."""
    rng = np.random.default_rng(52)
    for trial in range(12):
        T = np.zeros((256, 256), np.int32)
        letters = list(b"ACG-")
        for x in letters:
            for y in letters:
                T[x, y] = int(rng.integers(-4, 6))
        go, ge = int(rng.integers(0, 6)), int(rng.integers(1, 4))
        for _ in range(20):
            a = rng.choice(letters, size=int(rng.integers(0, 6))).astype(np.uint8).tobytes()
            b = rng.choice(letters, size=int(rng.integers(0, 6))).astype(np.uint8).tobytes()
            best = min(oracle.rescore_affine(a, b, ops, 0, 0, go, ge, sub=T) for ops in oracle.brute_alignments(a, b))
            score, ops = oracle.nw_affine(a, b, 0, 0, go, ge, sub=T)
            assert score == best
            assert oracle.rescore_affine(a, b, ops, 0, 0, go, ge, sub=T) == score


def test_nw_affine_flat_table_is_the_flat_model():
    rng = np.random.default_rng(53)
    T = np.full((256, 256), 3, np.int32)
    np.fill_diagonal(T, -1)
    for _ in range(30):
        a, b = _rand_dna(rng, int(rng.integers(0, 30))), _rand_dna(rng, int(rng.integers(0, 30)))
        assert oracle.nw_affine(a, b, -1, 3, 4, 1, sub=T) == oracle.nw_affine(a, b, -1, 3, 4, 1)


def test_blosum62_table():
    """Properties of the BLOSUM62 transcription: symmetric, the published
    diagonal, off-diagonal scores in [-4, 3] and below both residues' own
    scores; and the library's copy (its own transcription, in its code
    order) holds the same scores."""
    S = oracle.blosum62_scores()
    aa = "ARNDCQEGHILKMFPSTWYV"
    diag = dict(A=4, R=5, N=6, D=6, C=9, Q=5, E=5, G=6, H=8, I=4, L=4, K=5, M=5, F=6, P=7, S=4, T=5, W=11, Y=7, V=4)
    assert {x: S[(x, x)] for x in aa} == diag
    for x in aa:
        for y in aa:
            assert S[(x, y)] == S[(y, x)]
            if x != y:
                assert -4 <= S[(x, y)] <= 3 and S[(x, y)] < min(S[(x, x)], S[(y, y)])
    from paper_2601_15458_gb300 import substitution
    lib = substitution.blosum62_costs_by_code()
    order = substitution.PROTEIN_ORDER
    for i, x in enumerate(order):
        for j, y in enumerate(order):
            assert lib[i][j] == -S[(x, y)]
    T = oracle.blosum62_costs()
    g = len(order)
    assert lib[g][g] == T[ord("-"), ord("-")] and all(lib[g][i] == T[ord("-"), ord(x)] for i, x in enumerate(order))


# ---------------------------------------------------------------------------
# band policy and calibration
# ---------------------------------------------------------------------------

def test_band_policy_hand_examples():
    # gamma 0, yhat 0.25, lengths 1000/900: ceil(0.25 * 1000) + 8 = 258
    assert oracle.band_policy([0.25], [1000], [900], 0.0, 8)[0] == 258
    # the length difference dominates: max(500, ceil(0.01 * 1000) + 8)
    assert oracle.band_policy([0.01], [1000], [500], 0.0, 8)[0] == 500
    # negative outputs count as 0
    assert oracle.band_policy([-0.3], [64], [64], 0.5, 3)[0] == 3


def test_calibration_quantile_is_inverted_cdf():
    rng = np.random.default_rng(3)
    y = rng.random(1001).astype(np.float32)
    yhat = np.full(1001, 0.25, np.float32)            # every pair in bin 8
    for tau in (0.5, 0.9, 0.95, 1.0):
        knots = oracle.band_calibrate(yhat, y, tau)
        q = np.float32(np.quantile(y.astype(np.float64), tau, method="inverted_cdf"))
        assert knots[8] == q
        # bins 0..7 keep the identity, later bins the running maximum
        np.testing.assert_array_equal(knots[:8], np.arange(8, dtype=np.float32) / 32)
        np.testing.assert_array_equal(knots[9:], np.maximum(np.arange(9, 33, dtype=np.float32) / 32, q))


def test_calibration_sparse_bins_identity_and_monotone():
    rng = np.random.default_rng(4)
    yhat = rng.random(20000).astype(np.float32) * 0.6
    y = np.clip(yhat * 0.7 + rng.normal(0, 0.03, 20000), 0, None).astype(np.float32)
    yhat[:15] = 0.95                                  # 15 pairs in bin 30: too few
    knots = oracle.band_calibrate(yhat, y, 0.9)
    assert np.all(np.diff(knots) >= 0)
    assert knots[30] == max(np.float32(30) / 32, knots[29])
    # where the network runs high, the fitted map lies below the identity
    assert knots[16] < np.float32(16) / 32
    # bin edges: yhat just below (i + 0.5) / 32 belongs to bin i
    yb = np.array([np.nextafter(np.float32(8.5 / 32), np.float32(0))] * 16 + [np.float32(8.5 / 32)] * 16, np.float32)
    vals = np.array([0.5] * 16 + [0.7] * 16, np.float32)
    kb = oracle.band_calibrate(yb, vals, 1.0)
    assert kb[8] == np.float32(0.5) and kb[9] == np.float32(0.7)


def test_calibrated_policy_reductions():
    # identity knots reproduce the uncalibrated policy exactly on [0, 1]
    ident = np.arange(33, dtype=np.float32) / 32
    rng = np.random.default_rng(5)
    yhat = rng.uniform(-0.2, 1.0, 5000).astype(np.float32)
    la = rng.integers(1, 20000, 5000)
    lb = rng.integers(1, 20000, 5000)
    np.testing.assert_array_equal(oracle.band_policy(yhat, la, lb, 0.1, 8, knots=ident),
                                  oracle.band_policy(yhat, la, lb, 0.1, 8))
    # at a knot the map returns the knot; halfway between two it returns their mean
    knots = np.sort(rng.random(33).astype(np.float32))
    at = np.arange(33, dtype=np.float32) / 32
    np.testing.assert_array_equal(oracle.band_calibrated(knots, at), knots)
    mid = (np.arange(32, dtype=np.float32) + np.float32(0.5)) / 32
    np.testing.assert_allclose(oracle.band_calibrated(knots, mid), (knots[:-1] + knots[1:]) / 2, rtol=1e-6)
    # outputs above 1 use the last knot
    assert oracle.band_calibrated(knots, np.array([1.7], np.float32))[0] == knots[32]


# ---------------------------------------------------------------------------
# k-mer anchored NW (long pairs)
# ---------------------------------------------------------------------------

def test_kmer_anchors_definition():
    """Anchors are exactly the k-mers seen once in each sequence, counted
    with overlaps, at their positions."""
    rng = np.random.default_rng(61)
    for _ in range(30):
        a, b = _rand_dna(rng, int(rng.integers(0, 60))), _rand_dna(rng, int(rng.integers(0, 60)))
        k = int(rng.integers(2, 5))
        ref = []
        for i in range(len(a) - k + 1):
            w = a[i:i + k]
            ia = [t for t in range(len(a) - k + 1) if a[t:t + k] == w]
            jb = [t for t in range(len(b) - k + 1) if b[t:t + k] == w]
            if len(ia) == 1 and len(jb) == 1:
                ref.append((i, jb[0]))
        assert oracle.kmer_anchors(a, b, k) == ref


def test_anchor_chain_is_a_longest_increasing_chain():
    rng = np.random.default_rng(62)
    for _ in range(40):
        n = int(rng.integers(0, 9))
        anchors = sorted({(int(x), int(y)) for x, y in rng.integers(0, 12, (n, 2))})
        anchors = [(i, j) for t, (i, j) in enumerate(anchors) if t == 0 or i != anchors[t - 1][0]]
        chain = oracle.anchor_chain(anchors)
        assert all(p in anchors for p in chain)
        assert all(chain[t][0] < chain[t + 1][0] and chain[t][1] < chain[t + 1][1] for t in range(len(chain) - 1))
        best = 0
        for mask in range(1 << len(anchors)):
            sub = [anchors[t] for t in range(len(anchors)) if mask >> t & 1]
            if all(sub[t][1] < sub[t + 1][1] for t in range(len(sub) - 1)):
                best = max(best, len(sub))
        assert len(chain) == best


def test_nw_anchored_properties():
    """The split alignment is a valid alignment whose cost it reports, never
    below the optimum, equal to it for identical or anchor-free pairs, and
    its blocks are exact matches in order."""
    rng = np.random.default_rng(63)
    for _ in range(25):
        L = int(rng.integers(50, 600))
        a = _rand_dna(rng, L)
        b = bytearray(a)
        for _ in range(int(rng.integers(0, L // 10 + 1))):
            p = int(rng.integers(0, len(b)))
            b[p] = b"ACGT"[int(rng.integers(0, 4))]
        if rng.random() < 0.5 and len(b) > 20:
            del b[5:8]
        b = bytes(b)
        score, ops = oracle.nw_anchored(a, b, k=8)
        assert oracle.rescore(a, b, ops)[0] == score
        assert score >= oracle.nw(a, b)[0]
        blocks = oracle.anchor_blocks(oracle.anchor_chain(oracle.kmer_anchors(a, b, 8)), 8)
        for t, (sa, sb, ln) in enumerate(blocks):
            assert a[sa:sa + ln] == b[sb:sb + ln]
            if t:
                pa, pb, pl = blocks[t - 1]
                assert sa >= pa + pl and sb >= pb + pl
    a = _rand_dna(rng, 300)
    assert oracle.nw_anchored(a, a, k=8) == (0, b"M" * 300)
    # unrelated sequences over disjoint alphabets: no anchors, plain NW
    x, y = b"AC" * 40, b"GT" * 30
    assert oracle.nw_anchored(x, y, k=4) == oracle.nw(x, y)


def test_nw_anchored_hand_worked_split():
    # a = ACAGGGCCCTTT, b = AAGGGCCCTTAT.  The 6-mers seen once in each:
    # AGGGCC (2, 1), GGGCCC (3, 2), GGCCCT (4, 3), GCCCTT (5, 4), all on one
    # diagonal, so one block a[2:11] = b[1:10] (9 matches).  Left of it:
    # nw(AC, A) = 1 as M then D; right of it: nw(T, AT) = 1 as I then M.
    a = b"ACAGGGCCCTTT"
    b = b"AAGGGCCCTTAT"
    assert oracle.kmer_anchors(a, b, 6) == [(2, 1), (3, 2), (4, 3), (5, 4)]
    assert oracle.anchor_blocks(oracle.anchor_chain(oracle.kmer_anchors(a, b, 6)), 6) == [(2, 1, 9)]
    assert oracle.nw(b"AC", b"A") == (1, b"MD")
    assert oracle.nw(b"T", b"AT") == (1, b"IM")
    assert oracle.nw_anchored(a, b, k=6) == (2, b"MD" + b"M" * 9 + b"IM")


def test_nw_anchored_affine_hand_worked_and_properties():
    """Affine gaps in the anchored split (segments by nw_affine): the hand
    example above with open 2, extension 1 costs 3 + 0 + 3 (a deletion run
    of one, nine matches, an insertion run of one: each run pays open +
    extension); random related pairs, flat and with a table whose entries
    differ per pair of bytes: the script rescored under affine gaps gives the
    reported cost, which is never below the affine optimum; identical
    sequences cost the table's diagonal; without anchors the split is the
    plain affine alignment."""
    a, b = b"ACAGGGCCCTTT", b"AAGGGCCCTTAT"
    assert oracle.nw_anchored(a, b, k=6, gap=1, gap_open=2) == (6, b"MD" + b"M" * 9 + b"IM")
    rng = np.random.default_rng(71)
    T = rng.integers(-3, 6, size=(256, 256)).astype(np.int32)
    T = (T + T.T) // 2
    for x in b"ACGT":
        T[x, x] = -int(rng.integers(1, 4))
    for t in range(16):
        L = int(rng.integers(60, 400))
        a = _rand_dna(rng, L)
        b = bytearray(a)
        for _ in range(int(rng.integers(0, L // 12 + 1))):
            p = int(rng.integers(0, len(b)))
            b[p] = b"ACGT"[int(rng.integers(0, 4))]
        if len(b) > 30:
            del b[10:12 + t % 3]
        b = bytes(b)
        sub = T if t % 2 else None
        score, ops = oracle.nw_anchored(a, b, k=8, match=0, mismatch=2, gap=1, gap_open=3, sub=sub)
        assert oracle.rescore_affine(a, b, ops, 0, 2, 3, 1, sub) == score
        assert score >= oracle.nw_affine(a, b, 0, 2, 3, 1, sub)[0]
    a = _rand_dna(rng, 200)
    assert oracle.nw_anchored(a, a, k=8, gap=1, gap_open=3, sub=T) == (int(sum(T[x, x] for x in a)), b"M" * 200)
    x, y = b"AC" * 40, b"GT" * 30
    assert oracle.nw_anchored(x, y, k=4, gap=1, gap_open=3) == oracle.nw_affine(x, y, 0, 1, 3, 1)
