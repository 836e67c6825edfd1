"""Parity of Needleman-Wunsch fill + device traceback (A5, A6) with the oracle.

Scores and edit scripts must equal the oracle's byte for byte.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_15458_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_15458_gb300 import build
    build.build()
    c = api.Context(0, workspace_bytes=1 << 30)
    yield c
    c.close()


def _nw(ctx, rows, pairs, costs=(0, 1, 1)):
    seqs = api.ByteSeqs.from_list(rows)
    score, ops, off, ln = api.nw_align_batch(ctx, seqs, pairs, *costs)
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    return score, [ops[off[p]:off[p] + ln[p]].tobytes() for p in range(len(pairs))]


def _check(ctx, rows, pairs, costs=(0, 1, 1)):
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    score, scripts = _nw(ctx, rows, pairs, costs)
    ds = synth.SeqSet.from_list(rows)
    rs, rops, roff, rln = oracle.nw_pairs(ds.arena, ds.offs, pairs, *costs)
    for p, (x, y) in enumerate(pairs):
        ref = rops[roff[p]:roff[p] + rln[p]].tobytes()
        assert score[p] == rs[p], (p, len(rows[x]), len(rows[y]))
        assert scripts[p] == ref, (p, len(rows[x]), len(rows[y]))
        cost, ra, rb = oracle.rescore(rows[x], rows[y], scripts[p], *costs)
        assert cost == score[p]
    return score


def test_small_dna_pairs(ctx):
    ds = synth.small_dna(seed=1)
    pairs = synth.all_pairs(ds.n)[::7]
    _check(ctx, ds.seqs(), pairs)


@pytest.mark.parametrize("costs", [(0, 1, 1), (0, 2, 2), (0, 3, 2), (-1, 2, 3)])
def test_bruteforce_tiny(ctx, costs):
    rng = np.random.default_rng(sum(costs) + 40)
    rows = [rng.choice(list(b"ACG-"), size=int(rng.integers(0, 7))).astype(np.uint8).tobytes() for _ in range(40)]
    pairs = np.array([[i, (i * 7 + 3) % 40] for i in range(40)], np.int32)
    score, scripts = _nw(ctx, rows, pairs, costs)
    for p, (x, y) in enumerate(pairs):
        c, best = oracle.brute_best(rows[x], rows[y], *costs)
        assert score[p] == c and scripts[p] == best


EDGE = [0, 1, 15, 16, 17, 511, 512, 513, 1024, 1500, 3000]


def test_edge_lengths_and_gapped_rows(ctx):
    rng = np.random.default_rng(41)
    rows = []
    for L in EDGE:
        rows.append(rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes())
    for L in EDGE:
        a = np.frombuffer(rows[EDGE.index(L)], np.uint8).copy()
        if L:
            a[rng.integers(0, L, max(1, L // 8))] = ord("-")          # gapped center rows
        rows.append(a.tobytes())
    n = len(EDGE)
    pairs = [[i, n + j] for i in range(n) for j in range(n)]
    _check(ctx, rows, pairs)


def test_unit_cost_score_equals_levenshtein(ctx):
    ds = synth.tree_dna(seed=8, n=40, root_len=700)
    pairs = synth.random_pairs(3, ds.n, 60)
    seqs = api.upload_and_pack(ctx, ds)
    score, _, _, _ = api.nw_align_batch(ctx, seqs, pairs)
    d = api.lev_batch(ctx, seqs, pairs)
    ctx.check()
    np.testing.assert_array_equal(score.cpu().numpy(), d.cpu().numpy())
    # and both against the oracle
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.lev_pairs(ds.arena, ds.offs, pairs))


def test_protein_center_rows(ctx):
    members, roots = synth.protein_families(seed=3, n_fam=4, per_fam=10)
    rows = members.seqs() + roots.seqs()
    pairs = [[members.n + f, f * 10 + k] for f in range(4) for k in range(10)]
    _check(ctx, rows, pairs)


def test_unit_cost_many_symbols_and_absent_symbols(ctx):
    """Unit costs run bit-parallel over the distinct bytes of the row
    sequence; rows with more than 32 distinct bytes go to the plain DP in the
    same call; column bytes absent from the row sequence never match."""
    rng = np.random.default_rng(43)
    rows = []
    for L in (300, 2100, 40, 2049):
        rows.append(rng.integers(0, 256, size=L).astype(np.uint8).tobytes())          # many distinct bytes
        rows.append(rng.choice(list(b"ACGT-"), size=L).astype(np.uint8).tobytes())    # 5 symbols
        rows.append(rng.choice(list(b"acgtXYZ"), size=L // 2 + 1).astype(np.uint8).tobytes())  # disjoint
    n = len(rows)
    pairs = [[i, j] for i in range(n) for j in range(n) if (i + j) % 3 != 2]
    _check(ctx, rows, pairs)
    _check(ctx, rows, pairs[:40], (0, 2, 2))


def test_capacity_error(ctx):
    seqs = api.ByteSeqs.from_list([b"ACGT", b"ACG"])
    off = torch.tensor([0, 3], dtype=torch.int64, device="cuda")      # needs 7
    api.nw_align_batch(ctx, seqs, np.array([[0, 1]], np.int32), ops_off=off)
    with pytest.raises(api.MsaError):
        ctx.check()



# ---- affine gaps (Gotoh) -------------------------------------------------------

def _check_affine(ctx, rows, pairs, costs):
    match, mismatch, gap_open, gap_ext = costs
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    seqs = api.ByteSeqs.from_list(rows)
    score, ops, off, ln = api.nw_align_batch(ctx, seqs, pairs, match, mismatch, gap_ext, gap_open=gap_open)
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    for p, (x, y) in enumerate(pairs):
        rs, rops = oracle.nw_affine(rows[x], rows[y], *costs)
        got = ops[off[p]:off[p] + ln[p]].tobytes()
        assert score[p] == rs and got == rops, (p, len(rows[x]), len(rows[y]))
        assert oracle.rescore_affine(rows[x], rows[y], got, *costs) == score[p]


@pytest.mark.parametrize("costs", [(0, 1, 10, 1), (0, 3, 2, 1), (-1, 2, 3, 2), (0, 1, 0, 1)])
def test_affine_tiny_against_oracle_and_bruteforce(ctx, costs):
    rng = np.random.default_rng(sum(costs) + 60)
    rows = [rng.choice(list(b"ACG-"), size=int(rng.integers(0, 7))).astype(np.uint8).tobytes() for _ in range(40)]
    pairs = np.array([[i, (i * 7 + 3) % 40] for i in range(40)], np.int32)
    _check_affine(ctx, rows, pairs, costs)
    for x, y in pairs[:10]:
        best = min(oracle.rescore_affine(rows[x], rows[y], o, *costs) for o in oracle.brute_alignments(rows[x], rows[y]))
        assert oracle.nw_affine(rows[x], rows[y], *costs)[0] == best


def test_affine_edge_lengths(ctx):
    rng = np.random.default_rng(61)
    lens = [0, 1, 15, 16, 17, 511, 512, 513, 1024, 1500]
    rows = [rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes() for L in lens]
    for L in lens:
        a = bytearray(rows[lens.index(L)])
        for k in range(0, L, 37):
            a[k] = ord("-")
        rows.append(bytes(a[: max(0, L - L // 5)]))
    n = len(lens)
    pairs = [[i, n + j] for i in range(n) for j in range(n) if (i + j) % 2 == 0]
    _check_affine(ctx, rows, pairs, (0, 1, 10, 1))


def test_affine_protein_and_linear_reduction(ctx):
    members, roots = synth.protein_families(seed=3, n_fam=3, per_fam=10)
    rows = members.seqs() + roots.seqs()
    pairs = [[members.n + f, f * 10 + k] for f in range(3) for k in range(10)]
    _check_affine(ctx, rows, pairs, (0, 1, 10, 1))
    # open = 0: the linear model, same scores and scripts as the linear kernel
    seqs = api.ByteSeqs.from_list(rows)
    pr = np.asarray(pairs, np.int32)
    s0, o0, f0, l0 = api.nw_align_batch(ctx, seqs, pr, 0, 1, 1, gap_open=0)
    s1, o1, f1, l1 = api.nw_align_batch(ctx, seqs, pr, 0, 1, 1)
    ctx.check()
    np.testing.assert_array_equal(s0.cpu().numpy(), s1.cpu().numpy())
    np.testing.assert_array_equal(l0.cpu().numpy(), l1.cpu().numpy())
    np.testing.assert_array_equal(o0.cpu().numpy(), o1.cpu().numpy())


# ---------------------------------------------------------------------------
# substitution tables (BLOSUM62 for proteins, section "Implementation")
# ---------------------------------------------------------------------------

def _ascii_table(T_code, letters, gap=ord("-")):
    """The same costs as a 256 x 256 table over the oracle's ASCII bytes."""
    T = np.zeros((256, 256), np.int32)
    syms = list(letters) + [chr(gap)]
    for i, x in enumerate(syms):
        for j, y in enumerate(syms):
            T[ord(x), ord(y)] = T_code[i][j]
    return T


def test_affine_blosum62_protein_pairs(ctx):
    """BLOSUM62 costs with affine gaps (open 10, extend 1) on protein pairs:
    scores and scripts identical to the oracle's."""
    from paper_2601_15458_gb300 import substitution
    members, roots = synth.protein_families(seed=3, n_fam=4, per_fam=15)
    rows = members.seqs() + roots.seqs()
    ds = synth.SeqSet.from_list(rows, "protein")
    sq = api.upload_and_pack(ctx, ds)
    pairs = np.array([[members.n + f, f * 15 + k] for f in range(4) for k in range(15)] + [[0, 1], [5, 5], [7, 40]],
                     np.int32)
    score, ops, off, ln = api.nw_align_batch(ctx, sq, pairs, gap=1, gap_open=10, sub=api.blosum62_table())
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    assert oracle.blosum62_costs()[ord("W"), ord("W")] == -11
    T = _ascii_table(substitution.blosum62_costs_by_code(), substitution.PROTEIN_ORDER)
    np.testing.assert_array_equal(T, oracle.blosum62_costs())
    for p, (a, b) in enumerate(pairs):
        rs, rops = oracle.nw_affine(rows[a], rows[b], 0, 0, 10, 1, sub=T)
        assert score[p] == rs
        assert ops[off[p]:off[p] + ln[p]].tobytes() == rops


def test_affine_random_table_dna_with_gaps(ctx):
    """A random table over DNA codes and the gap code (some costs negative),
    on gapped rows: identical to the oracle."""
    rng = np.random.default_rng(31)
    T5 = rng.integers(-3, 6, (5, 5)).astype(np.int32)
    rows = [rng.choice(list(b"ACGT-"), size=int(rng.integers(0, 300))).astype(np.uint8).tobytes() for _ in range(40)]
    codes = [bytes(b"ACGT-".index(c) for c in r) for r in rows]
    bs = api.ByteSeqs.from_list(codes)
    pairs = np.array([[i, (i * 7 + 3) % 40] for i in range(40)], np.int32)
    score, ops, off, ln = api.nw_align_batch(ctx, bs, pairs, gap=2, gap_open=3,
                                             sub=torch.from_numpy(T5).cuda())
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    T = _ascii_table(T5.tolist(), "ACGT")
    for p, (a, b) in enumerate(pairs):
        rs, rops = oracle.nw_affine(rows[a], rows[b], 0, 0, 3, 2, sub=T)
        assert score[p] == rs
        assert ops[off[p]:off[p] + ln[p]].tobytes() == rops


def test_affine_table_rejects_codes_outside(ctx):
    bs = api.ByteSeqs.from_list([bytes([0, 1, 2]), bytes([0, 7, 1])])
    api.nw_align_batch(ctx, bs, np.array([[0, 1]], np.int32), gap=1, gap_open=2,
                       sub=torch.zeros((5, 5), dtype=torch.int32, device="cuda"))
    with pytest.raises(api.MsaError) as e:
        ctx.check()
    assert e.value.code == 6
