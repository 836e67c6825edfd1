"""Banded Levenshtein with certificate (A4): every distance equals the
oracle's whatever the starting band, and the band that certified it bounds
the distance."""
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


@pytest.fixture(scope="module")
def pairs_ds():
    ds = synth.divergent_pairs(seed=40, n_pairs=160, len_lo=200, len_hi=4000)
    pairs = np.stack([np.arange(0, ds.n, 2), np.arange(1, ds.n, 2)], axis=1).astype(np.int32)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    return ds, pairs, ref


@pytest.mark.parametrize("mode", ["zero", "exact", "below", "above", "huge", "random"])
def test_band_exact_for_any_start(ctx, pairs_ds, mode):
    ds, pairs, ref = pairs_ds
    rng = np.random.default_rng(5)
    lens = np.diff(ds.offs)
    mx = np.maximum(lens[pairs[:, 0]], lens[pairs[:, 1]])
    k0 = {"zero": np.zeros_like(ref), "exact": ref, "below": np.maximum(ref - 1, 0), "above": ref + 40,
          "huge": mx * 2, "random": rng.integers(0, 2000, len(ref))}[mode].astype(np.int32)
    seqs = api.upload_and_pack(ctx, ds)
    d, k_used = api.lev_banded_batch(ctx, seqs, pairs, k0)
    ctx.check()
    d, k_used = d.cpu().numpy(), k_used.cpu().numpy()
    np.testing.assert_array_equal(d, ref)
    assert np.all(k_used >= ref)
    assert np.all((k_used >= np.minimum(k0, mx)) | (k_used == mx))


def test_band_long_and_short_mix(ctx):
    rng = np.random.default_rng(6)
    seqs = []
    for L in (1, 31, 33, 64, 65, 700, 2048, 2049, 10000):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8)
        b = a.copy()
        k = max(1, L // 20)
        b[rng.integers(0, L, k)] = rng.choice(list(b"ACGT"), size=k).astype(np.uint8)
        b = np.concatenate([b[: L // 2], b[L // 2 + min(3, L // 3):]])
        seqs += [a.tobytes(), b.tobytes()]
    ds = synth.SeqSet.from_list(seqs)
    pairs = np.array([[2 * i, 2 * i + 1] for i in range(len(seqs) // 2)] +
                     [[2 * i + 1, 2 * i] for i in range(len(seqs) // 2)], np.int32)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    sq = api.upload_and_pack(ctx, ds)
    for k0 in (0, 16, 100, 5000):
        d, _ = api.lev_banded_batch(ctx, sq, pairs, np.full(len(pairs), k0, np.int32))
        ctx.check()
        np.testing.assert_array_equal(d.cpu().numpy(), ref)


def test_band_protein(ctx):
    members, roots = synth.protein_families(seed=3, n_fam=5, per_fam=20)
    rows = members.seqs() + roots.seqs()
    ds = synth.SeqSet.from_list(rows, "protein")
    pairs = np.array([[members.n + f, f * 20 + k] for f in range(5) for k in range(20)], np.int32)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    sq = api.upload_and_pack(ctx, ds)
    for k0 in (0, 50, 400):
        d, _ = api.lev_banded_batch(ctx, sq, pairs, np.full(len(pairs), k0, np.int32))
        ctx.check()
        np.testing.assert_array_equal(d.cpu().numpy(), ref)


LANE_CAPACITIES = [32 * w - 63 for w in (4, 8, 12, 16, 24, 32, 40, 48)]


def test_band_one_lane_windows(ctx):
    """DNA bands up to 1,473 rows run one pair per lane with a window of
    32-row words that moves down a word at 32-column boundaries: bands at
    and around every window size, column counts on and off those boundaries,
    rows far longer than columns, and bands started too narrow (retried in
    the lane when the retry band still fits the window, else in a later
    round) are all exact."""
    rng = np.random.default_rng(21)
    rows = []
    for L, div in ((32, 0.2), (64, 0.1), (95, 0.3), (640, 0.05), (1000, 0.3), (1024, 0.15), (1500, 0.25),
                   (2500, 0.12), (3000, 0.3), (4000, 0.08)):
        a = rng.choice(list(b"ACGT"), size=L).astype(np.uint8)
        b = a.copy()
        nsub = int(div * L)
        b[rng.integers(0, L, nsub)] = rng.choice(list(b"ACGT"), size=nsub).astype(np.uint8)
        cut = rng.integers(0, max(1, L // 3))
        b = np.concatenate([b[:L // 2], b[L // 2 + cut:]])      # rows longer than columns
        rows += [a.tobytes(), b.tobytes()]
    ds = synth.SeqSet.from_list(rows)
    pairs = np.array([[2 * i, 2 * i + 1] for i in range(len(rows) // 2)], np.int32)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    sq = api.upload_and_pack(ctx, ds)
    lens = np.diff(ds.offs)
    dl = np.abs(lens[pairs[:, 0]] - lens[pairs[:, 1]])
    starts = [np.full(len(pairs), c + e, np.int32) for c in LANE_CAPACITIES for e in (-1, 0, 1)]
    starts += [np.maximum(ref // 2, 0).astype(np.int32), np.maximum(ref - 3, 0).astype(np.int32),
               (ref + dl).astype(np.int32)]
    for k0 in starts:
        d, k_used = api.lev_banded_batch(ctx, sq, pairs, k0)
        ctx.check()
        np.testing.assert_array_equal(d.cpu().numpy(), ref)
        assert np.all(k_used.cpu().numpy() >= ref)


def test_divergent_pairs_full_size_every_pair(ctx):
    """The 100,000 pairs of the learned-band evaluation (lengths
    1,000-10,000, divergence 1-30%, seed 40), every one checked: the full DP
    equals the oracle on all of them (about 3.7e12 cells, some minutes on
    the host cores), and the certified banded DP equals the full DP from the
    narrowest start (|m - n|: every pair retries) and from the 4-mer L1
    lower bound."""
    ev = synth.divergent_pairs(seed=40, n_pairs=100000)
    pairs = np.stack([np.arange(0, ev.n, 2), np.arange(1, ev.n, 2)], 1).astype(np.int32)
    sq = api.upload_and_pack(ctx, ev)
    d_full = api.lev_batch(ctx, sq, pairs)
    ctx.check()
    lens = np.diff(ev.offs)
    dl = np.abs(lens[0::2] - lens[1::2]).astype(np.int32)
    prof = api.kmer_profile(ctx, sq)
    cnt = prof.int() & 0xFFFF
    pd = torch.from_numpy(pairs).cuda()
    l1 = (cnt[pd[:, 0].long()] - cnt[pd[:, 1].long()]).abs().sum(1)
    k_l1 = torch.maximum(torch.from_numpy(dl).cuda(), ((l1 + 7) // 8).int()).cpu().numpy().astype(np.int32)
    for k0 in (dl, k_l1):
        d, _ = api.lev_banded_batch(ctx, sq, pairs, k0)
        ctx.check()
        assert torch.equal(d, d_full)
    ref = oracle.lev_pairs(ev.arena, ev.offs, pairs)
    np.testing.assert_array_equal(d_full.cpu().numpy(), ref)
