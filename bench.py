"""Benchmark of the batched alignment DP hot path on GB300.

Default workload (N=1): 2,000 DNA sequences simulated down a random binary
tree from a uniform root of length 1,500 (lengths ~1,200-1,800), all
1,999,000 pairwise unit-cost Levenshtein distances in one call.  One step =
pack the ASCII arena (A1) + the whole distance batch (A2, A3, A7).  The
metric is GCUPS = sum over pairs of m*n cells / seconds / 1e9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own copy of the batch (pairs are
independent; no collective on the data path), so scaling is weak and the
value is the cells of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# integer ops of one 32-row word step of the column recurrence on this ISA
# (3-input logic, add with carry, funnel shift): Eq & Pv, the add, the
# carry-in vector, 2 for Ph, the Ph shift, Xv, Pv', Mv'
ALU_OPS_PER_WORD = 9
# DRAM bytes per launch of the dominant kernel (lev_lane_kernel<48>) on this
# workload, from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum`
# (profiles/launches_tree_dna_allpairs_2000x1500.md); valid only while the
# kernel source is the one that was measured.
TRAFFIC = dict(kernel_sha256_16="8ee36c74ea96d418", bytes_per_launch=20.1e6)
WORKLOAD = "tree_dna_allpairs_2000x1500"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=2000, help="sequences (default: the 2,000-sequence workload)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule (for profiling)")
    ap.add_argument("--no-band", action="store_true", help="skip the learned-band measurement")
    ap.add_argument("--band-pairs", type=int, default=100000)
    ap.add_argument("--band-oracle-pairs", type=int, default=20000,
                    help="learned-band pairs checked against the oracle")
    ap.add_argument("--clam", type=int, default=50000, metavar="N",
                    help="guide tree and merges of N 16S-like sequences (0 skips)")
    ap.add_argument("--no-protein", action="store_true", help="skip the 10,000-protein section")
    ap.add_argument("--merge-checks", type=int, default=1000, help="guide-tree merges checked against the oracle")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, world):
    """Element-wise maximum over all ranks (gloo / nccl all_reduce); identity at N=1."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_gcups(cells_per_rank, steps, max_ms, world):
    """Cells of every rank over the slowest rank's time (weak scaling: each
    rank runs its own copy of the batch)."""
    return world * cells_per_rank * steps / (max_ms / 1e3) / 1e9


def make_workload(n):
    from paper_2601_15458_gb300 import synth
    ds = synth.tree_dna(seed=2, n=n)
    pairs = synth.all_pairs_balanced(ds.n)
    lens = np.diff(ds.offs)
    m = lens[pairs[:, 0]].astype(np.int64)
    nn = lens[pairs[:, 1]].astype(np.int64)
    cells = int((m * nn).sum())
    words = int((((m + 31) // 32) * nn).sum())
    return ds, pairs, cells, words


def cpu_oracle_sample(ds, pairs, seconds, seed=7, single=True):
    """Time the oracle on a seeded sample of pairs sized to about `seconds`
    on all host cores, and (single) on one thread over part of it.

    Returns ``(info, cells, seconds, sample_index, oracle_distances)``: the
    sample's oracle distances are kept so the caller can compare them with
    the GPU's output for the same pairs."""
    import oracle
    threads = oracle.cpu_threads()
    rng = np.random.default_rng(seed)
    lens = np.diff(ds.offs)
    calib = pairs[rng.choice(len(pairs), size=min(len(pairs), 4 * threads), replace=False)]
    t0 = time.perf_counter()
    oracle.lev_pairs(ds.arena, ds.offs, calib, nthreads=threads)
    dt = time.perf_counter() - t0
    per_pair = dt / len(calib)
    k = int(max(threads, min(len(pairs), seconds / max(per_pair, 1e-9))))
    idx = np.sort(rng.choice(len(pairs), size=k, replace=False))
    sample = pairs[idx]
    t0 = time.perf_counter()
    ref = oracle.lev_pairs(ds.arena, ds.offs, sample, nthreads=threads)
    dt = time.perf_counter() - t0
    cells = int((lens[sample[:, 0]].astype(np.int64) * lens[sample[:, 1]]).sum())
    info = dict(value=cells / dt / 1e9, unit="GCUPS", cores=threads, kind="oracle",
                sample=f"{k} random pairs of the workload ({cells:.3e} cells, {dt:.1f} s)")
    if not single:
        return info, cells, dt, idx, ref
    # the same oracle on one thread, over a sample of about a fifth of the time
    k1 = int(max(1, min(len(pairs), seconds / 5 / max(per_pair * threads, 1e-9))))
    s1 = sample[:k1]
    t0 = time.perf_counter()
    oracle.lev_pairs(ds.arena, ds.offs, s1, nthreads=1)
    dt1 = time.perf_counter() - t0
    cells1 = int((lens[s1[:, 0]].astype(np.int64) * lens[s1[:, 1]]).sum())
    info["single_thread"] = dict(value=cells1 / dt1 / 1e9, unit="GCUPS", cores=1,
                                 sample=f"the first {k1} of those pairs ({cells1:.3e} cells, {dt1:.1f} s)")
    return info, cells, dt, idx, ref


def distance_invariants(d, pairs, offs):
    """Pairs whose distance breaks |m - n| <= d <= max(m, n) (true for any f)."""
    lens = np.diff(offs)
    a, b = lens[pairs[:, 0]], lens[pairs[:, 1]]
    return int(np.sum((d < np.abs(a - b)) | (d > np.maximum(a, b))))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        fd, self.path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            if os.path.exists(self.path):
                os.remove(self.path)
            return None
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        os.remove(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in rows), sm_max_mhz=max(r["smax"] for r in rows),
                    reasons=sorted(reasons), samples=len(rows),
                    power_w_max=max(r["power"] for r in rows))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, sm_max_mhz=2070.0), "fallback"


HELD_OUT_PAIRS = 20000   # held-out pairs that fit the calibration


def band_bench(ctx, args, stream):
    """Learned band vs full DP on 100,000 fresh DNA pairs (lengths 1,000-10,000,
    divergence U(1%, 30%)), every distance checked against the full DP."""
    import torch
    from paper_2601_15458_gb300 import api, learned_band, synth
    t0 = time.perf_counter()
    X, y, tinfo = learned_band.training_set(ctx, seed=4)
    model, minfo = learned_band.train(ctx, X, y, epochs=8, batch=4096, lr=2e-3, tau=0.9)
    del X, y
    # calibration and band margin come from held-out pairs of two other
    # seeds, never from the evaluation pairs
    def held_out(seed, n_pairs):
        val = synth.divergent_pairs(seed=seed, n_pairs=n_pairs)
        vs = api.upload_and_pack(ctx, val)
        vp = torch.from_numpy(np.stack([np.arange(0, val.n, 2), np.arange(1, val.n, 2)], 1).astype(np.int32))
        return vs, api.kmer_profile(ctx, vs), vp.cuda()

    # the margin is timed on a held-out batch of the evaluation batch's size
    cal_set, gam_set = held_out(41, HELD_OUT_PAIRS), held_out(42, args.band_pairs)
    gamma_raw, _ = learned_band.pick_gamma(ctx, model, *gam_set)
    cal_tau, gamma, _ = learned_band.pick_band(ctx, model, cal_set, gam_set)
    setup_s = time.perf_counter() - t0
    ev = synth.divergent_pairs(seed=40, n_pairs=args.band_pairs)
    es = api.upload_and_pack(ctx, ev)
    prof = api.kmer_profile(ctx, es)
    P = ev.n // 2
    pairs = torch.from_numpy(np.stack([np.arange(0, ev.n, 2), np.arange(1, ev.n, 2)], 1).astype(np.int32)).cuda()
    lens = np.diff(ev.offs)
    cells = int((lens[0::2].astype(np.int64) * lens[1::2]).sum())
    d_full = api.lev_batch(ctx, es, pairs)
    knots = model.state[-64:].clone()
    model.calibrate(None, None)                    # the network alone, for comparison
    _, k_raw = model.predict_band(es, prof, pairs, gamma=gamma_raw, margin=8)
    model.state[-64:].copy_(knots)
    yhat, k = model.predict_band(es, prof, pairs, gamma=gamma, margin=8)
    d_raw, _ = api.lev_banded_batch(ctx, es, pairs, k_raw)
    d_band, k_used = api.lev_banded_batch(ctx, es, pairs, k)
    # non-learned start: the 4-mer L1 lower bound, ceil(L1 / 8) <= f
    cnt = prof.int() & 0xFFFF
    l1 = (cnt[pairs[:, 0].long()] - cnt[pairs[:, 1].long()]).abs().sum(1)
    del cnt
    dl = torch.from_numpy(np.abs(lens[0::2] - lens[1::2]).astype(np.int32)).cuda()
    k_l1 = torch.maximum(dl, ((l1 + 7) // 8).int())
    d_l1, _ = api.lev_banded_batch(ctx, es, pairs, k_l1)
    ctx.check()
    # every banded result (learned, network alone, L1 bound) against the full DP on all pairs
    mism_full = dict(learned=int((d_band != d_full).sum().item()), uncalibrated=int((d_raw != d_full).sum().item()),
                     l1_bound=int((d_l1 != d_full).sum().item()))
    band_share = float((k_used.cpu().numpy() < np.maximum(lens[0::2], lens[1::2])).mean())
    # cells of the band that certified each distance (about min(m, 2k + 1)
    # rows per column; m x n for pairs the full DP computed; the cells of
    # failed narrower attempts are not counted)
    ku = k_used.cpu().numpy().astype(np.int64)
    m_rows, n_cols = lens[0::2].astype(np.int64), lens[1::2].astype(np.int64)
    full_pairs = ku >= np.maximum(m_rows, n_cols)
    cells_band = int(np.where(full_pairs, m_rows * n_cols, np.minimum(m_rows, 2 * ku + 1) * n_cols).sum())

    def timed(fn, reps):
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sum(ts) / len(ts)

    reps = max(2, min(args.steps, 5))
    t_full = timed(lambda: api.lev_batch(ctx, es, pairs, d_full), reps)
    t_band = timed(lambda: (model.predict_band(es, prof, pairs, gamma=gamma, margin=8),
                            api.lev_banded_batch(ctx, es, pairs, k, d_band, k_used)), reps)
    t_l1 = timed(lambda: api.lev_banded_batch(ctx, es, pairs, k_l1, d_l1), reps)
    t_raw = timed(lambda: api.lev_banded_batch(ctx, es, pairs, k_raw, d_raw), reps)
    ctx.check()
    # the timed outputs against the oracle on a seeded sample of the pairs
    import oracle
    rng = np.random.default_rng(9)
    samp = np.sort(rng.choice(P, size=min(P, args.band_oracle_pairs), replace=False))
    host_pairs = pairs.cpu().numpy()
    t0 = time.perf_counter()
    ref = oracle.lev_pairs(ev.arena, ev.offs, host_pairs[samp])
    t_oracle = time.perf_counter() - t0
    mism_oracle = dict(learned=int((ref != d_band.cpu().numpy()[samp]).sum()),
                       full=int((ref != d_full.cpu().numpy()[samp]).sum()))
    mism = sum(mism_full.values()) + sum(mism_oracle.values())
    args.band_model = (model, gamma)
    return dict(workload=f"divergent_dna_pairs_{P}_len1000-10000_div1-30pct", pairs=P, cells=cells,
                pairs_per_s_learned=P / (t_band / 1e3), pairs_per_s_full=P / (t_full / 1e3),
                pairs_per_s_l1_bound=P / (t_l1 / 1e3), speedup_learned_vs_full=t_full / t_band,
                speedup_learned_vs_l1_bound=t_l1 / t_band,
                speedup_uncalibrated_vs_full=t_full / t_raw,
                calibration=dict(tau=cal_tau, pairs=HELD_OUT_PAIRS, margin_timing_pairs=args.band_pairs,
                                 gamma_uncalibrated=gamma_raw,
                                 k_mean_over_f=float((k.double() / d_full.double().clamp(min=1)).mean().item()),
                                 k_mean_over_f_uncalibrated=float(
                                     (k_raw.double() / d_full.double().clamp(min=1)).mean().item())),
                gcups_full=cells / (t_full / 1e3) / 1e9, gcups_equiv_learned=cells / (t_band / 1e3) / 1e9,
                cells_computed_learned=cells_band, computed_share_learned=cells_band / cells,
                gcups_computed_learned=cells_band / (t_band / 1e3) / 1e9,
                ms_learned=t_band, ms_full=t_full, mismatches=mism,
                parity=dict(oracle_pairs=int(len(samp)), oracle_seconds=t_oracle,
                            mismatches_vs_oracle=mism_oracle, mismatches_vs_full_dp_all_pairs=mism_full),
                share_certified_by_band=band_share, gamma=gamma, train_pairs=tinfo["pairs"],
                train_steps=minfo["steps"], val_pinball=minfo["val_loss"], setup_s=setup_s)


def _cols_of(tree, order, k, offs, pos_h):
    """Root-MSA columns of node k: those its members' residues occupy (a
    node's MSA has no all-gap column, so these are exactly its columns)."""
    mem = order[tree.lo[k]:tree.hi[k]]
    parts = [pos_h[offs[s]:offs[s + 1]] for s in mem]
    return np.unique(np.concatenate(parts)) if parts else np.zeros(0, np.int32)


def stepwise_merge_check(ds, tree, pos_h, width, score, nodes, gap=ord("-")):
    """Each sampled merge redone by the oracle on the same inputs.

    For merge k the two children's centre rows, as gapped rows of the
    children's MSAs, are read back from the root MSA (positions `pos`),
    aligned by oracle.nw, and the oracle's cost and edit script are compared
    with the GPU's cost and with the script the GPU's MSA realises (a column
    of both children is a diagonal move, one of the left child only D, of
    the right child only I).  Together with the same check one level down
    this is an inductive check of the whole merge."""
    import oracle
    order = tree.order.cpu().numpy()
    offs, arena = ds.offs, ds.arena
    rows, got_ops, bad_width = [], [], 0
    for k in nodes:
        L, R = int(tree.left[k]), int(tree.right[k])
        cl, cr = _cols_of(tree, order, L, offs, pos_h), _cols_of(tree, order, R, offs, pos_h)
        crow = []
        for child, cols in ((L, cl), (R, cr)):
            c = int(tree.center[child])
            row = np.full(len(cols), gap, np.uint8)
            row[np.searchsorted(cols, pos_h[offs[c]:offs[c + 1]])] = arena[offs[c]:offs[c + 1]]
            crow.append(row)
        u = np.union1d(cl, cr)
        inl, inr = np.isin(u, cl), np.isin(u, cr)
        il, ir = np.maximum(np.cumsum(inl) - 1, 0), np.maximum(np.cumsum(inr) - 1, 0)
        same = crow[0][il] == crow[1][ir]
        op = np.where(inl & inr, np.where(same, ord("M"), ord("X")), np.where(inl, ord("D"), ord("I")))
        got_ops.append(op.astype(np.uint8).tobytes())
        bad_width += int(len(u) != width[k] or len(cl) != width[L] or len(cr) != width[R])
        rows += [r.tobytes() for r in crow]
    lens = np.array([len(r) for r in rows], np.int64)
    roffs = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(lens, out=roffs[1:])
    rarena = np.frombuffer(b"".join(rows) + b"\0", np.uint8)
    sc, ops, ooff, oln = oracle.nw_pairs(rarena, roffs, np.arange(len(rows), dtype=np.int32).reshape(-1, 2))
    bad_score = bad_ops = 0
    for t, k in enumerate(nodes):
        bad_score += int(sc[t] != score[k])
        bad_ops += int(ops[ooff[t]:ooff[t] + oln[t]].tobytes() != got_ops[t])
    return dict(merges=len(nodes), score_mismatches=bad_score, script_mismatches=bad_ops,
                width_mismatches=bad_width, cells=int(sum(len(rows[2 * t]) * len(rows[2 * t + 1])
                                                          for t in range(len(nodes)))))


def cluster_checks(seqs, tree, picks):
    """Alg. 1 redone by the oracle (one batched application) on the GPU
    tree's clusters `picks`: centre and split must agree."""
    import oracle
    order = tree.order.cpu().numpy()
    bad = 0
    sizes = []
    for k in picks:
        mem = sorted(int(x) for x in order[tree.lo[k]:tree.hi[k]])
        nodes = oracle.partition_levels([seqs[x] for x in mem], max_levels=1)
        c = mem[nodes[0]["center"]]
        L = [mem[i] for i in nodes[1]["members"]]
        gl = sorted(int(x) for x in order[tree.lo[tree.left[k]]:tree.hi[tree.left[k]]])
        bad += int(c != int(tree.center[k]) or L != gl)
        sizes.append(len(mem))
    return dict(clusters=len(picks), mismatches=bad, sizes_checked=f"{min(sizes)}-{max(sizes)}" if sizes else "",
                sampled_medoid=int(sum(x > 256 for x in sizes)))


def pick_checks(tree, rng, n_merges, n_small=30, n_big=2):
    """Internal nodes to check: the root plus a seeded sample for merges;
    the two smallest clusters above 256 members (medoid from the 256-member
    sample) and a sample of clusters of 2-64 for Alg. 1."""
    internal = np.nonzero(tree.left[:tree.n_nodes] >= 0)[0]
    size = tree.hi[:tree.n_nodes] - tree.lo[:tree.n_nodes]
    merges = [0] + list(rng.choice(internal[1:], min(n_merges, len(internal) - 1), replace=False))
    big = sorted((int(size[k]), int(k)) for k in internal if size[k] > 256)[:n_big]
    small = [k for k in internal if 2 <= size[k] <= 64]
    small = list(rng.choice(small, min(n_small, len(small)), replace=False))
    return [int(k) for k in merges], [k for _, k in big] + [int(k) for k in small]


def rows_match_sequences(rows_h, order, ds, gap=ord("-")):
    """Every MSA row with its gaps removed is its sequence (one vectorised
    comparison over all rows)."""
    flat = rows_h[rows_h != gap]
    ref = np.concatenate([ds.arena[ds.offs[s]:ds.offs[s + 1]] for s in order])
    return bool(len(flat) == len(ref) and np.array_equal(flat, ref))


def clam_bench(ctx, args):
    """Guide tree (Alg. 1) and bottom-up merges on N 16S-like sequences
    (lengths 1,400-1,600), learned band on and off; Alg. 1 redone by the
    oracle on sampled clusters, sampled merges redone by the oracle on the
    same centre rows, every MSA row checked against its sequence."""
    import torch
    from paper_2601_15458_gb300 import api, synth
    from paper_2601_15458_gb300 import learned_band
    model, gamma = getattr(args, "band_model", (None, None))
    if model is None:
        X, y, _ = learned_band.training_set(ctx, seed=4)
        model, _ = learned_band.train(ctx, X, y, epochs=8, batch=4096, lr=2e-3, tau=0.9)
        del X, y
        gamma = 0.2
    t0 = time.perf_counter()
    ds = synth.gg16s_dna(seed=5, n=args.clam)
    gen_s = time.perf_counter() - t0
    sq = api.upload_and_pack(ctx, ds)
    prof = api.kmer_profile(ctx, sq)
    ctx.check()
    # learned band on: the same tree from banded distance batches
    api.clam_partition(ctx, api.upload_and_pack(ctx, synth.small_dna(seed=1)), band=model, gamma=gamma)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree_b = api.clam_partition(ctx, sq, band=model, prof=prof, gamma=gamma)
    torch.cuda.synchronize()
    t_part_b = time.perf_counter() - t0
    ctx.prof_read(reset=True)
    ctx.prof_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = api.clam_partition(ctx, sq)
    torch.cuda.synchronize()
    t_part = time.perf_counter() - t0
    part_dp_ms, part_launches = ctx.prof_read(reset=True)
    same_tree = bool(np.array_equal(tree.order.cpu().numpy(), tree_b.order.cpu().numpy())
                     and np.array_equal(tree.center, tree_b.center) and np.array_equal(tree.left, tree_b.left)
                     and np.array_equal(tree.lo, tree_b.lo))
    t0 = time.perf_counter()
    pos, width, score = api.merge_tree(ctx, sq, tree)
    torch.cuda.synchronize()
    t_merge = time.perf_counter() - t0
    merge_dp_ms, merge_launches = ctx.prof_read(reset=True)
    ctx.prof_enable(False)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0]))
    ctx.check()
    # alignment quality on a seeded 10,000-row sample (section "Evaluation")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    met = api.msa_metrics(ctx, sq, tree, rows, sample=min(10000, ds.n), seed=0)
    t_met = time.perf_counter() - t0
    # parity (outside every timed region)
    t0 = time.perf_counter()
    order = tree.order.cpu().numpy()
    rows_h = rows.cpu().numpy()
    rows_ok = rows_match_sequences(rows_h, order, ds)
    no_gap_col = not bool(np.any(np.all(rows_h == ord("-"), axis=0)))
    del rows_h
    rng = np.random.default_rng(0)
    merge_nodes, cluster_nodes = pick_checks(tree, rng, args.merge_checks)
    mcheck = stepwise_merge_check(ds, tree, pos.cpu().numpy(), width, score, merge_nodes)
    ccheck = cluster_checks(ds.seqs(), tree, cluster_nodes)
    check_s = time.perf_counter() - t0
    depth = np.zeros(tree.n_nodes, np.int64)
    for k in range(1, tree.n_nodes):
        depth[k] = depth[tree.parent[k]] + 1
    nw_cells = 0
    for k in range(tree.n_nodes):
        if tree.left[k] >= 0:
            nw_cells += int(width[tree.left[k]]) * int(width[tree.right[k]])
    mism = (mcheck["score_mismatches"] + mcheck["script_mismatches"] + mcheck["width_mismatches"]
            + ccheck["mismatches"] + int(not rows_ok) + int(not no_gap_col) + int(not same_tree))
    return dict(workload=f"gg16s_dna_{ds.n}_len1400-1600", n_seqs=ds.n, partition_s=t_part, merge_s=t_merge,
                partition_learned_band_s=t_part_b, learned_band_speedup=t_part / t_part_b,
                learned_band_gamma=gamma, learned_band_same_tree=same_tree,
                quality=dict(sample_rows=met["rows"], pct_gaps=met["pct_gaps"], p_score=met["p_score"],
                             distortion=met["distortion"], pairs=met["pairs"], seconds=t_met),
                partition_dp_ms=part_dp_ms, merge_dp_ms=merge_dp_ms, launches=part_launches + merge_launches,
                tree_depth=int(depth.max()), msa_width=int(width[0]), nw_cells=nw_cells,
                nw_gcups=nw_cells / (merge_dp_ms / 1e3) / 1e9 if merge_dp_ms else None,
                parity=dict(mismatches=mism, merges_vs_oracle=mcheck, clusters_vs_oracle=ccheck,
                            all_rows_degap_to_sequences=rows_ok, no_all_gap_column=no_gap_col, seconds=check_s),
                generate_s=gen_s)


def protein_bench(ctx, args, stream):
    """The 10,000-protein workload: 1,000,000 member-to-family-root distances
    (one-to-many by root) and the guide tree with its 9,999 merges; oracle
    checks on a 100,000-pair sample of the distances, on sampled clusters and
    on 1,000 sampled merges (the tests check every distance, node and row)."""
    import torch
    import oracle
    from paper_2601_15458_gb300 import api, synth
    members, roots = synth.protein_families(seed=3)
    allseq = synth.SeqSet.from_list(members.seqs() + roots.seqs(), "protein")
    nm = members.n
    pairs_h = np.array([[nm + c, x] for c in range(roots.n) for x in range(nm)], np.int32)
    lens = np.diff(allseq.offs)
    cells = int((lens[pairs_h[:, 0]].astype(np.int64) * lens[pairs_h[:, 1]]).sum())
    sq = api.upload_and_pack(ctx, allseq)
    pairs = torch.from_numpy(pairs_h).cuda()
    d = api.lev_batch(ctx, sq, pairs)

    def timed(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    # the schedule tuned for this batch (the headline's is for 2,000 x 1,500
    # all pairs), the headline's put back afterwards
    keep = api.lev_schedule(ctx)
    api.lev_autotune(ctx, sq, pairs, d)
    schedule = api.lev_schedule(ctx)
    t_dist = timed(lambda: api.lev_batch(ctx, sq, pairs, d))
    api.lev_schedule(ctx, **keep)
    msq = api.upload_and_pack(ctx, members)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = api.clam_partition(ctx, msq)
    torch.cuda.synchronize()
    t_part = time.perf_counter() - t0
    t0 = time.perf_counter()
    pos, width, score = api.merge_tree(ctx, msq, tree)
    torch.cuda.synchronize()
    t_merge = time.perf_counter() - t0
    rows = api.msa_rows(ctx, msq, tree, pos, int(width[0]))
    ctx.check()
    t0 = time.perf_counter()
    got = d.cpu().numpy()
    rng = np.random.default_rng(5)
    samp = np.sort(rng.choice(len(pairs_h), size=100000, replace=False))
    dmis = int((oracle.lev_pairs(allseq.arena, allseq.offs, pairs_h[samp]) != got[samp]).sum())
    inv = distance_invariants(got, pairs_h, allseq.offs)
    rows_ok = rows_match_sequences(rows.cpu().numpy(), tree.order.cpu().numpy(), members)
    merge_nodes, cluster_nodes = pick_checks(tree, rng, args.merge_checks)
    mcheck = stepwise_merge_check(members, tree, pos.cpu().numpy(), width, score, merge_nodes)
    ccheck = cluster_checks(members.seqs(), tree, cluster_nodes)
    check_s = time.perf_counter() - t0
    mism = (dmis + inv + mcheck["score_mismatches"] + mcheck["script_mismatches"] + mcheck["width_mismatches"]
            + ccheck["mismatches"] + int(not rows_ok))
    return dict(workload="protein_families_10000x100", pairs=len(pairs_h), cells=cells, ms_distances=t_dist,
                schedule=schedule,
                gcups_distances=cells / (t_dist / 1e3) / 1e9, partition_s=t_part, merge_s=t_merge,
                merges=int(tree.n_nodes - members.n), msa_width=int(width[0]),
                parity=dict(mismatches=mism, oracle_pairs=len(samp), distance_mismatches=dmis,
                            invariant_violations=inv, merges_vs_oracle=mcheck, clusters_vs_oracle=ccheck,
                            all_rows_degap_to_sequences=rows_ok, seconds=check_s))


def small_bench(ctx):
    """The 64-sequence DNA case checked in full: all 2,016 distances, the
    guide tree node for node and the 63 merges row for row."""
    import oracle
    from paper_2601_15458_gb300 import api, synth
    ds = synth.small_dna(seed=1)
    seqs = ds.seqs()
    sq = api.upload_and_pack(ctx, ds)
    pairs = synth.all_pairs(ds.n)
    d = api.lev_batch(ctx, sq, pairs).cpu().numpy()
    tree = api.clam_partition(ctx, sq)
    pos, width, score = api.merge_tree(ctx, sq, tree)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0])).cpu().numpy()
    ctx.check()
    ref_d = oracle.lev_pairs(ds.arena, ds.offs, pairs)
    ref_nodes = oracle.partition(seqs)
    ref_rows, ref_order, merges = oracle.merge_tree(seqs, ref_nodes)
    order = tree.order.cpu().numpy()
    node_mis = 0
    for k, nd in enumerate(ref_nodes):
        node_mis += int(sorted(int(x) for x in order[tree.lo[k]:tree.hi[k]]) != nd["members"]
                        or int(tree.center[k]) != nd["center"])
    return dict(workload="small_dna_64x150", pairs=len(pairs), distance_mismatches=int((d != ref_d).sum()),
                node_mismatches=node_mis + int(tree.n_nodes != len(ref_nodes)),
                merge_score_mismatches=int(sum(score[k] != sc for k, (sc, _) in merges.items())),
                row_mismatches=int(sum(r.tobytes() != q for r, q in zip(rows, ref_rows))) + int(list(order) != ref_order))


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step a bounded sample."""
    if rank != 0:
        return
    ds, pairs, cells, words = make_workload(args.n)
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    vals = []
    total_cells = 0
    total_t = 0.0
    info = None
    for s in range(args.warmup + args.steps):
        info, c, dt, _, _ = cpu_oracle_sample(ds, pairs, per_step, seed=100 + s, single=False)
        if s >= args.warmup:
            vals.append(info["value"])
            total_cells += c
            total_t += dt
    value = total_cells / total_t / 1e9
    line = dict(metric="GCUPS", value=value, unit="GCUPS", n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * total_t / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="int32", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, n_seqs=ds.n, pairs=len(pairs), cells=cells,
                            note="reference arm = the CPU oracle (full-matrix Wagner-Fischer) on seeded samples"),
                cpu_baseline=dict(info, value=value),
                e2e=dict(value=value, unit="GCUPS", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    from paper_2601_15458_gb300 import api, build
    build.build()
    ctx = api.Context(local, workspace_bytes=2 << 30)
    ds, pairs, cells, words = make_workload(args.n)
    stream = torch.cuda.current_stream()

    # device-resident inputs
    seqs = api.DeviceSeqs.from_host(ds.arena, ds.offs, ds.alphabet)
    pairs_d = torch.from_numpy(pairs).cuda()
    out = torch.empty(len(pairs), dtype=torch.int32, device="cuda")
    api.pack(ctx, seqs)
    if not args.no_autotune:
        api.lev_autotune(ctx, seqs, pairs_d, out)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        api.pack(ctx, seqs)
        api.lev_batch(ctx, seqs, pairs_d, out)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    ctx.check()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # integer-pipe throughput of this GPU (the roofline's denominator)
    probe = {op: api.probe_int_pipe(ctx, op) for op in api.PROBE_OPS}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.prof_read(reset=True)
    ctx.prof_enable(True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)          # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier()
    ctx.prof_enable(False)
    dp_ms, launches = ctx.prof_read(reset=True)
    ctx.check()
    out_timed = out.cpu().numpy()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms, dp_ms = max_over_ranks([total_ms, dp_ms], world)
    value = whole_job_gcups(cells, args.steps, total_ms, world)

    # end to end through the public API: host buffers, copies inside the timed region
    h_arena = torch.from_numpy(np.ascontiguousarray(np.concatenate(
        [ds.arena, np.zeros((-len(ds.arena)) % 16 + 16, np.uint8)]))).pin_memory()
    h_offs = torch.from_numpy(ds.offs.astype(np.int64)).pin_memory()
    h_pairs = torch.from_numpy(pairs).pin_memory()
    h_out = torch.empty(len(pairs), dtype=torch.int32).pin_memory()
    d_ascii = torch.empty_like(h_arena, device="cuda")
    d_offs = torch.empty_like(h_offs, device="cuda")
    d_pairs = torch.empty_like(h_pairs, device="cuda")
    e2e_seqs = api.DeviceSeqs(d_ascii, d_offs, "dna", int(np.diff(ds.offs).max()), int(ds.offs[-1]))

    def e2e_step():
        d_ascii.copy_(h_arena, non_blocking=True)
        d_offs.copy_(h_offs, non_blocking=True)
        d_pairs.copy_(h_pairs, non_blocking=True)
        api.pack(ctx, e2e_seqs)
        api.lev_batch(ctx, e2e_seqs, d_pairs, out)
        h_out.copy_(out, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    ctx.check()
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        eev[k][0].record(stream)
        e2e_step()
        eev[k][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    e2e_ms = sum(a.elapsed_time(b) for a, b in eev)
    (e2e_ms,) = max_over_ranks([e2e_ms], world)
    e2e_value = whole_job_gcups(cells, args.steps, e2e_ms, world)
    h2d = h_arena.numel() + h_offs.numel() * 8 + h_pairs.numel() * 4
    d2h = h_out.numel() * 4
    ok = np.array_equal(h_out.numpy(), out.cpu().numpy())

    # roofline of the DP kernels: bound by the integer ALU pipe, the unit that
    # executes 3-input logic, integer add and funnel shift.  The peak is
    # measured on this GPU by msa_probe_int_pipe (LOP3 chains at full
    # occupancy); the clock-derived figures are reported beside it.
    pk, pk_kind = peaks()
    props = torch.cuda.get_device_properties(local)
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    issue_peak = props.multi_processor_count * 4 * 32 * sm_max * 1e6 / 1e12   # T warp-lane instructions/s
    alu_pipe_derived = issue_peak / 2
    alu_pipe_peak = probe["lop3"]["ops_per_s"] / 1e12
    mix_peak = probe["word_step"]["ops_per_s"] / 1e12
    alg_ops = words * ALU_OPS_PER_WORD
    achieved = alg_ops * args.steps / (dp_ms / 1e3) / 1e12 if dp_ms > 0 else None
    import hashlib
    src = os.path.join(ROOT, "paper_2601_15458_gb300", "csrc", "lev_kernels.cuh")
    same_kernel = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == TRAFFIC["kernel_sha256_16"]
    roof = dict(bound="alu", kernel="lev_lane_kernel (all length buckets)", achieved=achieved, peak=alu_pipe_peak,
                unit="Tops/s (int32 lane-ops)", frac=(achieved / alu_pipe_peak) if achieved else None,
                traffic=TRAFFIC["bytes_per_launch"] if same_kernel else None,
                peak_source="measured: msa_probe_int_pipe LOP3 chains (8 per thread, full occupancy) on this GPU",
                probe={k: v["ops_per_s"] / 1e12 for k, v in probe.items()},
                op_mix_peak=mix_peak, frac_of_op_mix=(achieved / mix_peak) if achieved else None,
                alu_pipe_derived=alu_pipe_derived, issue_peak=issue_peak,
                frac_of_issue=(achieved / issue_peak) if achieved else None,
                derived_source=f"{props.multi_processor_count} SMs x 4 schedulers x 16 (ALU) / 32 (issue) lanes/clk "
                               f"x {sm_max:.0f} MHz ({pk_kind} max clock)",
                algorithmic=f"{ALU_OPS_PER_WORD} ops per 32-row word per column; "
                            f"{words:.4e} word-columns per launch set")

    clocks = clk.summary()
    band = None
    if not args.no_band:
        band = band_bench(ctx, args, stream)
    clam = clam_bench(ctx, args) if args.clam else None
    protein = None if args.no_protein else protein_bench(ctx, args, stream)
    small = small_bench(ctx)
    cpu = None
    parity = None
    if rank == 0:
        # the oracle on a seeded sample of the workload: timed as the CPU
        # baseline (one rank, N = 1) and compared with the timed GPU output
        secs = args.cpu_seconds if (world == 1 and not args.no_cpu_baseline) else 5.0
        info, _, _, idx, ref = cpu_oracle_sample(ds, pairs, secs, single=world == 1)
        if world == 1 and not args.no_cpu_baseline:
            cpu = info
        parity = dict(oracle_pairs=int(len(idx)), mismatches=int((out_timed[idx] != ref).sum()),
                      invariant_violations=distance_invariants(out_timed, pairs, ds.offs),
                      checked="the distances of the last timed step")
    if rank == 0:
        line = dict(metric="GCUPS", value=value, unit="GCUPS", n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=total_ms / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="int32", data="synthetic",
                    config=dict(workload=WORKLOAD, n_seqs=ds.n, pairs=len(pairs), cells=cells,
                                pairs_per_s=world * len(pairs) * args.steps / (total_ms / 1e3),
                                l2="flushed between timed steps (256 MB write)", step="msa_pack + msa_lev_batch",
                                schedule=dict(api.lev_schedule(ctx), autotuned=not args.no_autotune)),
                    roofline=roof, cpu_baseline=cpu, parity=parity,
                    e2e=dict(value=e2e_value, unit="GCUPS", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                             output_matches_device=bool(ok)),
                    gpu_launches=launches, dp_kernel_ms_per_step=dp_ms / args.steps, band=band, clam=clam,
                    protein=protein, small=small,
                    wall_s_timed=t_wall, clocks=clocks)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
