"""Small fixed workloads that run one kernel family each, for profiling.

    python profile_cases.py lev     # lane kernel, 400 x 1,500 DNA all pairs
    python profile_cases.py lev_few # slot kernel, 20,000 x 1,500 DNA, 100,000 random pairs
    python profile_cases.py tree    # guide tree of 50,000 16S-like DNA sequences
    python profile_cases.py nw      # NW fill + traceback, 2,000 pairs of ~1,500
    python profile_cases.py band    # certified bands, 100,000 pairs 1,000-10,000
    python profile_cases.py band_small  # the same on 20,000 pairs (for ncu captures)
    python profile_cases.py pack    # packed loader, 1.1 GB arena
    python profile_cases.py mlp     # band network forward + one training step
    python profile_cases.py protein # 10,000 x 100 centre distances; guide tree and 9,999 merges of the 10,000
    python profile_cases.py nw_affine # NW with affine gaps (open 10, extend 1), 2,000 pairs
    python profile_cases.py metrics # MSA quality of a 3,000-sequence MSA, 2,000-row sample
    python profile_cases.py nw_long # 512 pairs of 6,000-10,000: plain NW against NW split at k-mer anchors

Each case runs its call a few times (the first warms up) and prints one
line with the call's device time.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2601_15458_gb300 import api, build, learned_band, synth


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def case_lev(ctx):
    ds = synth.tree_dna(seed=2, n=400)
    sq = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(synth.all_pairs_balanced(ds.n)).cuda()
    out = torch.empty(pairs.shape[0], dtype=torch.int32, device="cuda")
    return _time(lambda: api.lev_batch(ctx, sq, pairs, out))


def case_lev_few(ctx):
    """20,000 DNA sequences of ~1,500, 100,000 random pairs: ~5 targets per
    query, the slot kernel's batch shape."""
    ds = synth.tree_dna(seed=3, n=20000)
    sq = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(synth.random_pairs(7, ds.n, 100000)).cuda()
    out = torch.empty(pairs.shape[0], dtype=torch.int32, device="cuda")
    return _time(lambda: api.lev_batch(ctx, sq, pairs, out))


def case_tree(ctx):
    """Guide tree (Alg. 1) of 50,000 16S-like DNA sequences, one partition."""
    ds = synth.gg16s_dna(seed=5, n=50000)
    sq = api.upload_and_pack(ctx, ds)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = api.clam_partition(ctx, sq)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    print(f"guide tree: {tree.n_nodes} nodes, {ms:.1f} ms")
    return ms


def _nw_offsets(sq, pairs):
    lens = sq.offs[1:] - sq.offs[:-1]
    cap = lens[pairs[:, 0].long()] + lens[pairs[:, 1].long()]
    off = torch.zeros(len(pairs) + 1, dtype=torch.int64, device="cuda")
    torch.cumsum(cap, 0, out=off[1:])
    return off


def case_nw(ctx):
    ds = synth.tree_dna(seed=2, n=2000)
    sq = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(np.stack([np.arange(0, 2000, 2), np.arange(1, 2000, 2)], 1).astype(np.int32)).cuda()
    pairs = torch.cat([pairs, pairs.flip(1)])
    off = _nw_offsets(sq, pairs)          # output buffers made once, as a caller would
    ops = torch.empty(int(off[-1].item()), dtype=torch.uint8, device="cuda")
    return _time(lambda: api.nw_align_batch(ctx, sq, pairs, ops_off=off, ops=ops))


def case_nw_affine(ctx):
    ds = synth.tree_dna(seed=2, n=2000)
    sq = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(np.stack([np.arange(0, 2000, 2), np.arange(1, 2000, 2)], 1).astype(np.int32)).cuda()
    pairs = torch.cat([pairs, pairs.flip(1)])
    off = _nw_offsets(sq, pairs)
    ops = torch.empty(int(off[-1].item()), dtype=torch.uint8, device="cuda")
    return _time(lambda: api.nw_align_batch(ctx, sq, pairs, 0, 1, 1, ops_off=off, gap_open=10, ops=ops))


def case_metrics(ctx):
    ds = synth.gg16s_dna(seed=5, n=3000)
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    pos, width, score = api.merge_tree(ctx, sq, tree)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0]))
    t0 = time.perf_counter()
    api.msa_metrics(ctx, sq, tree, rows, sample=2000, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = api.msa_metrics(ctx, sq, tree, rows, sample=2000, seed=0)
    ms = (time.perf_counter() - t0) * 1e3
    print({k: v for k, v in m.items() if k != "sample"})
    return ms


def case_band(ctx):
    ev = synth.divergent_pairs(seed=40, n_pairs=100000)
    sq = api.upload_and_pack(ctx, ev)
    pairs = torch.from_numpy(np.stack([np.arange(0, ev.n, 2), np.arange(1, ev.n, 2)], 1).astype(np.int32)).cuda()
    d = api.lev_batch(ctx, sq, pairs)
    k0 = (d.float() * 1.2).int() + 8          # a band 20% above the distance
    full = _time(lambda: api.lev_batch(ctx, sq, pairs, d))
    print(f"full DP: {full:.3f} ms per call")
    return _time(lambda: api.lev_banded_batch(ctx, sq, pairs, k0))


def case_band_small(ctx):
    ev = synth.divergent_pairs(seed=40, n_pairs=20000)
    sq = api.upload_and_pack(ctx, ev)
    pairs = torch.from_numpy(np.stack([np.arange(0, ev.n, 2), np.arange(1, ev.n, 2)], 1).astype(np.int32)).cuda()
    d = api.lev_batch(ctx, sq, pairs)
    k0 = (d.float() * 1.2).int() + 8
    return _time(lambda: api.lev_banded_batch(ctx, sq, pairs, k0))


def case_pack(ctx):
    ev = synth.divergent_pairs(seed=40, n_pairs=100000)
    sq = api.DeviceSeqs.from_host(ev.arena, ev.offs, "dna")
    return _time(lambda: api.pack(ctx, sq))


def case_mlp(ctx):
    X, y, _ = learned_band.training_set(ctx, seed=4, n_per_tree=120)
    model = api.BandModel(ctx, seed=0)
    idx = torch.arange(4096, dtype=torch.int32, device="cuda") % X.shape[0]
    model.forward(X)
    return _time(lambda: model.train_step(X, y, idx, lr=1e-3))


def case_protein(ctx):
    members, roots = synth.protein_families(seed=3)
    allseq = synth.SeqSet.from_list(members.seqs() + roots.seqs(), "protein")
    nm = members.n
    sq = api.upload_and_pack(ctx, allseq)
    lens = np.diff(allseq.offs).astype(np.int64)
    cen = np.array([[nm + c, x] for c in range(roots.n) for x in range(nm)], np.int32)
    cen_d = torch.from_numpy(cen).cuda()
    out = torch.empty(len(cen), dtype=torch.int32, device="cuda")
    t_lev = _time(lambda: api.lev_batch(ctx, sq, cen_d, out))
    c_lev = int((lens[cen[:, 0]] * lens[cen[:, 1]]).sum())
    print(f"centre distances: {len(cen)} pairs, {t_lev:.3f} ms, {c_lev / t_lev / 1e9:.1f} TCUPS")
    # Alg. 1 over the 10,000 members and the 9,999 guide-tree merges
    msq = api.upload_and_pack(ctx, members)
    api.clam_partition(ctx, msq)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = api.clam_partition(ctx, msq)
    torch.cuda.synchronize()
    t_tree = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    pos, width, score = api.merge_tree(ctx, msq, tree)
    torch.cuda.synchronize()
    t_merge = (time.perf_counter() - t0) * 1e3
    print(f"guide tree: {t_tree:.1f} ms; 9,999 merges with traceback: {t_merge:.1f} ms, MSA width {int(width[0])}")
    return t_lev + t_tree + t_merge


def case_nw_long(ctx):
    """512 DNA pairs of 6,000-10,000 at 1-10 % divergence: plain NW against
    NW split at unique 12- and 16-mer anchors, with unit costs (the
    bit-parallel NW) and with mismatch 3 / gap 2 (the scoring DP), in a
    64 GB workspace (the plain traceback keeps about max_len^2 bits to 4
    bytes per cell of a pair in flight)."""
    big = api.Context(0, workspace_bytes=64 << 30)
    ds = synth.divergent_pairs(seed=44, n_pairs=512, len_lo=6000, len_hi=10000, div_lo=0.01, div_hi=0.10)
    sq = api.upload_and_pack(big, ds)
    pairs = torch.from_numpy(np.stack([np.arange(0, ds.n, 2), np.arange(1, ds.n, 2)], 1).astype(np.int32)).cuda()
    off = _nw_offsets(sq, pairs)
    ops = torch.empty(int(off[-1].item()), dtype=torch.uint8, device="cuda")
    out = 0.0
    for costs in ((0, 1, 1), (0, 3, 2)):
        t_plain = _time(lambda: api.nw_align_batch(big, sq, pairs, *costs, ops_off=off, ops=ops))
        opt = api.nw_align_batch(big, sq, pairs, *costs, ops_off=off, ops=ops)[0].cpu()
        res = {}
        for k in (12, 16):
            t = _time(lambda: api.nw_align_batch_anchored(big, sq, pairs, k, *costs, ops_off=off))
            sc = api.nw_align_batch_anchored(big, sq, pairs, k, *costs, ops_off=off)[0].cpu()
            big.check()
            res[k] = (t, float((sc == opt).float().mean()),
                      float(((sc - opt).float() / opt.clamp(min=1).float()).max()))
        print(f"costs {costs}: plain NW {t_plain:.2f} ms; " + "; ".join(
            f"anchored k={k}: {t:.2f} ms ({t_plain / t:.1f}x), optimal on {100 * eq:.1f} % of pairs, worst excess "
            f"{100 * ex:.2f} %" for k, (t, eq, ex) in res.items()))
        out = res[12][0]
    big.close()
    return out


CASES = dict(lev=case_lev, lev_few=case_lev_few, tree=case_tree, nw=case_nw, band=case_band, band_small=case_band_small, pack=case_pack, mlp=case_mlp,
             protein=case_protein, nw_affine=case_nw_affine, metrics=case_metrics,
             nw_long=case_nw_long)


def main(argv):
    build.build()
    ctx = api.Context(0, workspace_bytes=2 << 30)
    t0 = time.perf_counter()
    ms = CASES[argv[1]](ctx)
    ctx.check()
    print(f"case {argv[1]}: {ms:.3f} ms per call ({time.perf_counter() - t0:.1f} s total)")


if __name__ == "__main__":
    main(sys.argv)
