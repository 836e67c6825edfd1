"""Needleman-Wunsch split at unique k-mer anchors: scores and edit scripts
equal the oracle's (``oracle.nw_anchored``) byte for byte, on related long
pairs, repeat-rich pairs (most k-mers not unique), unrelated pairs (few or no
anchors), identical pairs (one block over everything), pairs shorter than k,
empty sequences, protein pairs and more pairs than resident blocks."""
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


def _mutate(rng, a, rate, alphabet=b"ACGT"):
    """Substitutions, insertions and deletions, each at rate/3 per residue."""
    out = []
    al = np.frombuffer(alphabet, np.uint8)
    for x in a:
        u = rng.random()
        if u < rate / 3:
            out.append(int(rng.choice(al)))
        elif u < 2 * rate / 3:
            out += [int(x), int(rng.choice(al))]
        elif u < rate:
            continue
        else:
            out.append(int(x))
    return bytes(out)


def _check(ctx, rows, pairs, k, costs=(0, 1, 1), packed=False):
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    if packed:
        ds = synth.SeqSet.from_list(rows)
        seqs = api.upload_and_pack(ctx, ds)
    else:
        seqs = api.ByteSeqs.from_list(rows)
    score, ops, off, ln = api.nw_align_batch_anchored(ctx, seqs, pairs, k, *costs)
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    full = []
    for p, (x, y) in enumerate(pairs):
        rs, rops = oracle.nw_anchored(rows[x], rows[y], k, *costs)
        got = ops[off[p]:off[p] + ln[p]].tobytes()
        assert score[p] == rs, (p, k, len(rows[x]), len(rows[y]))
        assert got == rops, (p, k, len(rows[x]), len(rows[y]))
        full.append(rs)
    return np.array(full)


@pytest.mark.parametrize("k", [8, 12, 20])
def test_related_long_pairs(ctx, k):
    rng = np.random.default_rng(70 + k)
    rows = []
    for L, rate in ((3000, 0.02), (5000, 0.05), (4000, 0.1), (6000, 0.15), (2500, 0.3)):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, rate)]
    pairs = [[2 * i, 2 * i + 1] for i in range(len(rows) // 2)] + [[2 * i + 1, 2 * i] for i in range(len(rows) // 2)]
    _check(ctx, rows, pairs, k)


@pytest.mark.parametrize("k", [4, 6])
def test_short_k_many_repeats(ctx, k):
    """With k = 4 or 6 most k-mers of a few-thousand-residue sequence occur
    more than once: the hash table holds many repeated keys and few anchors."""
    rng = np.random.default_rng(80 + k)
    rows = []
    for L in (300, 1200, 3000):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, 0.08)]
    _check(ctx, rows, [[0, 1], [2, 3], [4, 5], [5, 4], [0, 3]], k)


def test_tandem_repeats_and_unrelated(ctx):
    rng = np.random.default_rng(90)
    unit = rng.choice(list(b"ACGT"), size=60).astype(np.uint8).tobytes()
    flank = [rng.choice(list(b"ACGT"), size=800).astype(np.uint8).tobytes() for _ in range(4)]
    a = flank[0] + unit * 6 + flank[1]
    b = _mutate(rng, flank[0], 0.05) + unit * 4 + _mutate(rng, flank[1], 0.05)
    c = rng.choice(list(b"ACGT"), size=1500).astype(np.uint8).tobytes()
    d = rng.choice(list(b"ACGT"), size=1700).astype(np.uint8).tobytes()
    rows = [a, b, c, d, flank[2] + flank[3], flank[3] + flank[2]]      # swapped halves: crossing anchors
    _check(ctx, rows, [[0, 1], [1, 0], [2, 3], [0, 2], [4, 5]], 12)


def test_degenerate_pairs(ctx):
    rng = np.random.default_rng(91)
    x = rng.choice(list(b"ACGT"), size=2000).astype(np.uint8).tobytes()
    rows = [b"", b"A", b"ACGTACGTAC", b"ACGTACGTAG", x, x, x[:1000], x[500:], b"AAAAAAAAAAAAAAAAAAAAAAAA"]
    pairs = [[0, 0], [0, 4], [4, 0], [1, 2], [2, 3], [4, 5], [4, 6], [6, 4], [4, 7], [7, 6], [8, 8], [8, 2]]
    _check(ctx, rows, pairs, 12)
    _check(ctx, rows, pairs, 1)


def test_costs_and_packed_codes(ctx):
    rng = np.random.default_rng(92)
    rows = []
    for L in (700, 1500):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, 0.1)]
    pairs = [[0, 1], [2, 3], [3, 2]]
    for costs in ((0, 2, 2), (0, 3, 2), (-1, 2, 3)):
        _check(ctx, rows, pairs, 10, costs)
    _check(ctx, rows, pairs, 10, packed=True)


def test_protein_pairs(ctx):
    members, roots = synth.protein_families(seed=5, n_fam=3, per_fam=6)
    rows = members.seqs() + roots.seqs()
    pairs = [[members.n + f, f * 6 + j] for f in range(3) for j in range(6)] + [[0, 7], [1, 13]]
    _check(ctx, rows, pairs, 4)
    _check(ctx, rows, pairs, 6)


def test_more_pairs_than_blocks_and_upper_bound(ctx):
    """1,400 pairs (more than the resident pair blocks) of mixed lengths; the
    anchored cost is never below the plain NW optimum."""
    rng = np.random.default_rng(93)
    rows = []
    for i in range(1400):
        L = int(rng.integers(0, 600))
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, float(rng.choice([0.02, 0.1, 0.4])))]
    pairs = np.array([[2 * i, 2 * i + 1] for i in range(1400)], np.int32)
    got = _check(ctx, rows, pairs, 8)
    seqs = api.ByteSeqs.from_list(rows)
    opt, _, _, _ = api.nw_align_batch(ctx, seqs, pairs)
    ctx.check()
    assert np.all(got >= opt.cpu().numpy())


def test_bad_arguments(ctx):
    seqs = api.ByteSeqs.from_list([b"ACGT", b"ACGA"])
    for k in (0, 257):
        with pytest.raises(RuntimeError):
            api.nw_align_batch_anchored(ctx, seqs, np.array([[0, 1]], np.int32), k)
    with pytest.raises(RuntimeError):                  # negative gap opening
        api.nw_align_batch_anchored(ctx, seqs, np.array([[0, 1]], np.int32), 4, gap_open=-1)
    with pytest.raises(RuntimeError):                  # table wider than 32 symbols
        api.nw_align_batch_anchored(ctx, seqs, np.array([[0, 1]], np.int32), 4, gap_open=2,
                                    sub=torch.zeros(33, 33, dtype=torch.int32, device="cuda"))
    # a pair index past the set: the kernel records it (the host sizes the
    # scripts from offsets given here, so nothing indexes the lengths with it)
    off = torch.tensor([0, 8], dtype=torch.int64, device="cuda")
    api.nw_align_batch_anchored(ctx, seqs, np.array([[0, 2]], np.int32), 4, ops_off=off)
    with pytest.raises(RuntimeError):
        ctx.check()


# ---------------------------------------------------------------------------
# affine gaps in the segments (msa_nw_align_batch_anchored_affine / _sub)
# ---------------------------------------------------------------------------

def _ascii_table(T_code, letters):
    """A table over codes (letters in code order) as a 256 x 256 table over
    the oracle's bytes."""
    T = np.zeros((256, 256), np.int32)
    for i, x in enumerate(letters):
        for j, y in enumerate(letters):
            T[ord(x), ord(y)] = T_code[i][j]
    return T


@pytest.mark.parametrize("costs", [(0, 2, 3, 1), (0, 1, 10, 1), (-1, 2, 4, 2)])
def test_affine_related_pairs(ctx, costs):
    match, mismatch, gap_open, gap_ext = costs
    rng = np.random.default_rng(100 + gap_open)
    rows = []
    for L, rate in ((2500, 0.03), (4000, 0.1), (600, 0.2), (1200, 0.05)):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, rate)]
    rows += [b"", b"ACGTACGTACGT", b"ACGTACGTACGT"]
    pairs = np.array([[0, 1], [1, 0], [2, 3], [4, 5], [6, 7], [8, 9], [9, 10], [8, 0]], np.int32)
    seqs = api.ByteSeqs.from_list(rows)
    score, ops, off, ln = api.nw_align_batch_anchored(ctx, seqs, pairs, 12, match, mismatch, gap_ext,
                                                      gap_open=gap_open)
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    for p, (x, y) in enumerate(pairs):
        rs, rops = oracle.nw_anchored(rows[x], rows[y], 12, match, mismatch, gap_ext, gap_open=gap_open)
        assert score[p] == rs, (p, costs)
        assert ops[off[p]:off[p] + ln[p]].tobytes() == rops, (p, costs)


def test_affine_table_dna_codes(ctx):
    """A random table over DNA codes (some costs negative, diagonal
    included): segments by the table, block residues by its diagonal."""
    rng = np.random.default_rng(111)
    T4 = rng.integers(-3, 6, (4, 4)).astype(np.int32)
    rows = []
    for L, rate in ((1800, 0.05), (900, 0.15), (3000, 0.02)):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes()
        rows += [a, _mutate(rng, a, rate)]
    codes = [bytes(b"ACGT".index(c) for c in r) for r in rows]
    pairs = np.array([[0, 1], [2, 3], [4, 5], [5, 4]], np.int32)
    score, ops, off, ln = api.nw_align_batch_anchored(ctx, api.ByteSeqs.from_list(codes), pairs, 10, 0, 0, 1,
                                                      gap_open=4, sub=torch.from_numpy(T4).cuda())
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    T = _ascii_table(T4.tolist(), "ACGT")
    for p, (x, y) in enumerate(pairs):
        rs, rops = oracle.nw_anchored(rows[x], rows[y], 10, 0, 0, 1, gap_open=4, sub=T)
        assert score[p] == rs
        assert ops[off[p]:off[p] + ln[p]].tobytes() == rops


def test_affine_blosum62_protein(ctx):
    """BLOSUM62 with affine gaps (open 10, extend 1) on packed protein
    sequences: identical to the oracle's split over the same letters."""
    from paper_2601_15458_gb300 import substitution
    members, roots = synth.protein_families(seed=6, n_fam=3, per_fam=8)
    rows = members.seqs() + roots.seqs()
    ds = synth.SeqSet.from_list(rows, "protein")
    sq = api.upload_and_pack(ctx, ds)
    pairs = np.array([[members.n + f, f * 8 + j] for f in range(3) for j in range(8)] + [[0, 9]], np.int32)
    score, ops, off, ln = api.nw_align_batch_anchored(ctx, sq, pairs, 4, 0, 0, 1, gap_open=10,
                                                      sub=api.blosum62_table())
    ctx.check()
    score, ops, off, ln = score.cpu().numpy(), ops.cpu().numpy(), off.cpu().numpy(), ln.cpu().numpy()
    T = oracle.blosum62_costs()
    for p, (x, y) in enumerate(pairs):
        rs, rops = oracle.nw_anchored(rows[x], rows[y], 4, 0, 0, 1, gap_open=10, sub=T)
        assert score[p] == rs
        assert ops[off[p]:off[p] + ln[p]].tobytes() == rops


def test_affine_table_rejects_codes_outside(ctx):
    """A block residue outside the table is reported (the segments' check
    does not see block residues)."""
    a = bytes([0, 1, 2, 3] * 10)
    bs = api.ByteSeqs.from_list([a + bytes([9]) * 12 + a, a + bytes([9]) * 12 + a])
    api.nw_align_batch_anchored(ctx, bs, np.array([[0, 1]], np.int32), 6, 0, 0, 1, gap_open=2,
                                sub=torch.zeros(4, 4, dtype=torch.int32, device="cuda"))
    with pytest.raises(RuntimeError):
        ctx.check()
