"""Parity of the bit-vector Levenshtein path (A1-A3, A7) with the oracle.

Integer work: every distance must equal the oracle's exactly.
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


def _run(ctx, ds, pairs):
    seqs = api.upload_and_pack(ctx, ds)
    out = api.lev_batch(ctx, seqs, pairs)
    ctx.check()
    return out.cpu().numpy()


def test_small_dna_all_pairs(ctx):
    ds = synth.small_dna(seed=1)
    pairs = synth.all_pairs(ds.n)
    assert len(pairs) == 2016
    got = _run(ctx, ds, pairs)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    np.testing.assert_array_equal(got, ref)


def test_textbook_protein_alphabet(ctx):
    ds = synth.SeqSet.from_list([b"KITTEN", b"SITTING", b"", b"GAMMA"], "protein")
    pairs = np.array([[0, 1], [1, 0], [2, 1], [0, 2], [2, 2], [3, 0]], np.int32)
    got = _run(ctx, ds, pairs)
    np.testing.assert_array_equal(got, [3, 3, 7, 6, 0, oracle.lev(b"GAMMA", b"KITTEN")])


EDGE = [1, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 2047, 2048, 2049, 10000]


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
def test_edge_lengths_both_kernels(ctx, alphabet):
    rng = np.random.default_rng(7)
    letters = np.frombuffer(synth.DNA if alphabet == "dna" else synth.PROTEIN, np.uint8)
    seqs = [letters[rng.integers(0, len(letters), L)].tobytes() for L in EDGE]
    # mutated partners and a few random extra targets
    partners = []
    for s in seqs:
        a = np.frombuffer(s, np.uint8).copy()
        k = max(1, len(a) // 10)
        a[rng.integers(0, len(a), k)] = letters[rng.integers(0, len(letters), k)]
        partners.append(a[: max(0, len(a) - int(rng.integers(0, 5)))].tobytes())
    extra = [letters[rng.integers(0, len(letters), L)].tobytes() for L in (0, 5, 700, 3000)]
    allseq = seqs + partners + extra
    ds = synth.SeqSet.from_list(allseq, alphabet)
    n = len(seqs)
    pairs = [[i, n + i] for i in range(n)]                      # one target per query: warp kernel
    for i in range(n):                                          # many targets per query: lane kernel
        pairs += [[i, j] for j in range(len(allseq))]
    pairs = np.array(pairs, np.int32)
    got = _run(ctx, ds, pairs)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
def test_few_targets_per_query_slot_kernel(ctx, alphabet):
    """Queries with 1..40 targets: single targets go to the warp kernel, 2..31
    share warps in the slot kernel, 32+ take a warp each.  Query lengths span
    several word counts; empty query and target; the number of queries per
    bucket is not a multiple of the 8 a warp takes."""
    rng = np.random.default_rng(11)
    letters = np.frombuffer(synth.DNA if alphabet == "dna" else synth.PROTEIN, np.uint8)
    lens = [0, 1, 17, 32, 33, 100, 250, 700, 1100, 1530, 2100]
    seqs = [letters[rng.integers(0, len(letters), L)].tobytes() for L in lens]
    for i in range(90):
        L = int(rng.integers(1, 1600))
        seqs.append(letters[rng.integers(0, len(letters), L)].tobytes())
    n = len(seqs)
    pairs = []
    for q in range(n):
        c = int(rng.integers(1, 41)) if q >= len(lens) else 3 + q
        pairs += [[q, int(t)] for t in rng.integers(0, n, c)]
    pairs += [[1, 0], [0, 5], [0, 0]]
    pairs = np.array(pairs, np.int32)
    got = _run(ctx, synth.SeqSet.from_list(seqs, alphabet), pairs)
    ds = synth.SeqSet.from_list(seqs, alphabet)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    np.testing.assert_array_equal(got, ref)


def test_random_pairs_schedule_independent(ctx):
    ds = synth.tree_dna(seed=9, n=120, root_len=400)
    pairs = synth.random_pairs(5, ds.n, 3000)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    seqs = api.upload_and_pack(ctx, ds)
    got = api.lev_autotune(ctx, seqs, pairs)
    ctx.check()
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    np.testing.assert_array_equal(api.lev_batch(ctx, seqs, pairs).cpu().numpy(), ref)


def test_slot_kernel_full_warps(ctx):
    """Enough few-target queries for 8 queries per warp (the bucket holds more
    than 8 per resident warp: up to 16 blocks of 4 warps on each of 152 SMs
    for these short queries), with a ragged last task."""
    ds = synth.tree_dna(seed=13, n=90003, root_len=60)
    rng = np.random.default_rng(13)
    pairs = []
    for q in range(ds.n):
        c = int(rng.integers(2, 12))
        pairs += [[q, int(t)] for t in rng.integers(0, ds.n, c)]
    pairs = np.array(pairs, np.int32)
    seqs = api.upload_and_pack(ctx, ds)
    got = api.lev_batch(ctx, seqs, pairs).cpu().numpy()
    ctx.check()
    np.testing.assert_array_equal(got, oracle.lev_pairs(ds.arena, ds.offs, pairs))


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
def test_one_to_many(ctx, alphabet):
    """msa_lev_one_to_many equals the oracle for a query against repeated,
    empty and long targets; bad indices are reported; n = 0 is a no-op."""
    rng = np.random.default_rng(21)
    letters = np.frombuffer(synth.DNA if alphabet == "dna" else synth.PROTEIN, np.uint8)
    seqs = [letters[rng.integers(0, len(letters), L)].tobytes() for L in (700, 0, 1, 2049, 64, 1500)]
    seqs += [letters[rng.integers(0, len(letters), int(rng.integers(1, 1800)))].tobytes() for _ in range(300)]
    ds = synth.SeqSet.from_list(seqs, alphabet)
    sq = api.upload_and_pack(ctx, ds)
    for q, idx in [(0, np.arange(ds.n)), (1, np.array([0, 1, 3, 3, 3])), (3, rng.integers(0, ds.n, 5000))]:
        got = api.lev_one_to_many(ctx, sq, q, idx).cpu().numpy()
        ctx.check()
        pairs = np.stack([np.full(len(idx), q), idx], 1).astype(np.int32)
        np.testing.assert_array_equal(got, oracle.lev_pairs(ds.arena, ds.offs, pairs))
    assert api.lev_one_to_many(ctx, sq, 0, np.zeros(0, np.int32)).numel() == 0
    with pytest.raises(api.MsaError):
        api.lev_one_to_many(ctx, sq, ds.n, np.array([0], np.int32))
    api.lev_one_to_many(ctx, sq, 0, np.array([1, ds.n + 5], np.int32))
    with pytest.raises(api.MsaError):
        ctx.check()


def test_explicit_schedules_same_distances(ctx):
    """Every schedule gives the oracle's distances: slot kernel on and off,
    other thresholds, small tasks; the schedule in force is restored."""
    ds = synth.tree_dna(seed=12, n=300, root_len=700)
    pairs = synth.random_pairs(6, ds.n, 2500)             # ~8 targets per query
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    seqs = api.upload_and_pack(ctx, ds)
    keep = api.lev_schedule(ctx)
    try:
        for sched in [dict(lane_min_targets=32, slot_min_targets=2), dict(lane_min_targets=12, slot_min_targets=12),
                      dict(lane_min_targets=4, slot_min_targets=3), dict(lane_min_targets=1 << 30, slot_min_targets=1 << 30),
                      dict(lane_min_targets=1 << 30, slot_min_targets=1), dict(lane_per_task=32, warp_per_task=1)]:
            got = api.lev_schedule(ctx, **sched)
            for k, v in sched.items():
                assert got[k] == v
            np.testing.assert_array_equal(api.lev_batch(ctx, seqs, pairs).cpu().numpy(), ref, err_msg=str(sched))
        with pytest.raises(api.MsaError):
            api.lev_schedule(ctx, warp_per_task=0)
    finally:
        api.lev_schedule(ctx, **keep)
    ctx.check()


def test_protein_families_to_centers_sample(ctx):
    members, roots = synth.protein_families(seed=3, n_fam=6, per_fam=40)
    allseq = synth.SeqSet.from_list(members.seqs() + roots.seqs(), "protein")
    nm = members.n
    pairs = np.array([[nm + c, x] for c in range(roots.n) for x in range(nm)], np.int32)
    got = _run(ctx, allseq, pairs)
    ref = oracle.lev_pairs(allseq.arena, allseq.offs, pairs)
    np.testing.assert_array_equal(got, ref)


def test_bad_index_reports_edata(ctx):
    ds = synth.small_dna(seed=1, n=4)
    seqs = api.upload_and_pack(ctx, ds)
    api.lev_batch(ctx, seqs, np.array([[0, 1], [0, 9]], np.int32))
    with pytest.raises(api.MsaError) as e:
        ctx.check()
    assert e.value.code == 6
    ctx.check()    # cleared


@pytest.mark.parametrize("total", [1, 31, 32, 33, 4096 + 17, 100_003])
def test_pack_codes_and_planes(ctx, total):
    """Packed loader: byte codes (A0 C1 G2 T3) and the bit planes (plane p,
    bit k of word w = bit p of the code at 32 w + k), from their definition."""
    rng = np.random.default_rng(total)
    arena = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=total)
    offs = np.array([0, total // 3, total], np.int64)
    seqs = api.DeviceSeqs.from_host(arena, offs, "dna")
    api.pack(ctx, seqs)
    ctx.check()
    code = np.searchsorted(np.frombuffer(b"ACGT", np.uint8), arena)
    np.testing.assert_array_equal(seqs.codes.cpu().numpy()[:total], code)
    nw = (total + 31) // 32
    planes = seqs.planes.cpu().numpy().view(np.uint32)[: 2 * nw].reshape(nw, 2)
    padded = np.zeros(nw * 32, np.int64)
    padded[:total] = code
    bits = padded.reshape(nw, 32)
    for p in (0, 1):
        ref = ((bits >> p) & 1).astype(np.uint64) << np.arange(32, dtype=np.uint64)
        np.testing.assert_array_equal(planes[:, p], ref.sum(1).astype(np.uint32))


@pytest.mark.parametrize("rows", [[b"ACGT", b"ACNT"], [b"ACGT" * 20, b"ACGTACGTAC" * 3 + b"GGNAxA" + b"T" * 40]])
def test_bad_symbol_reports_edata(ctx, rows):
    ds = synth.SeqSet.from_list(rows, "dna")
    seqs = api.upload_and_pack(ctx, ds)
    with pytest.raises(api.MsaError, match="outside the alphabet"):
        ctx.check()
    # the valid residues keep their codes, the bad ones get code 0
    code = np.array([b"ACGT".find(bytes([c])) for c in ds.arena], np.int64)
    got = seqs.codes.cpu().numpy()[: len(ds.arena)].astype(np.int64)
    np.testing.assert_array_equal(got[code >= 0], code[code >= 0])
    assert np.all(got[code < 0] == 0)


def test_tree_dna_full_size_sampled(ctx):
    """The 2,000-sequence all-pairs workload, checked on a seeded sample."""
    ds = synth.tree_dna(seed=2)
    pairs = synth.all_pairs_balanced(ds.n)
    assert len(pairs) == ds.n * (ds.n - 1) // 2
    got = _run(ctx, ds, pairs)
    rng = np.random.default_rng(123)
    idx = rng.choice(len(pairs), size=1500, replace=False)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs[idx])
    np.testing.assert_array_equal(got[idx], ref)
    # properties that hold at any size
    lens = np.diff(ds.offs)
    a, b = lens[pairs[:, 0]], lens[pairs[:, 1]]
    assert np.all(got >= np.abs(a - b)) and np.all(got <= np.maximum(a, b)) and np.all(got > 0)


def test_protein_families_full_size_all_pairs(ctx):
    """10,000 protein members x 100 family roots (one-to-many by root): all
    1,000,000 distances against the oracle, and properties that hold for
    every pair."""
    members, roots = synth.protein_families(seed=3)
    allseq = synth.SeqSet.from_list(members.seqs() + roots.seqs(), "protein")
    nm = members.n
    pairs = np.array([[nm + c, x] for c in range(roots.n) for x in range(nm)], np.int32)
    assert len(pairs) == 1_000_000
    got = _run(ctx, allseq, pairs)
    np.testing.assert_array_equal(got, oracle.lev_pairs(allseq.arena, allseq.offs, pairs))
    lens = np.diff(allseq.offs)
    a, b = lens[pairs[:, 0]], lens[pairs[:, 1]]
    assert np.all(got >= np.abs(a - b)) and np.all(got <= np.maximum(a, b))
    # members are closer to their own family root than the typical other root
    fam = members.extra["family"]
    own = got.reshape(roots.n, nm)[fam, np.arange(nm)]
    assert np.median(own) < np.median(got)
