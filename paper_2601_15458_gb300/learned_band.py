"""Learned band proposer pipeline (A8-A10): training data from the exact
kernels, the training loop, and the band-width margin choice.

The network only proposes the starting band of ``msa_lev_banded_batch``;
the band's certificate (accept d_k only when d_k <= k, else double k) keeps
every distance exact whatever the network predicts.  All arithmetic runs in
the library's kernels; this module only orders the calls.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api, synth


def training_set(ctx: api.Context, seed: int = 4, n_per_tree: int = 334,
                 root_lens=(1000, 2000, 3500, 5500, 8000, 10000), scales=(0.1, 0.3, 1.0)):
    """Exact distances on DNA simulated down Yule trees (the 2,000-sequence
    workload's recipe: per-branch substitution U(0.005, 0.05) x scale,
    indels 0.2x), all pairs of each tree.

    The grid of root lengths and rate scales spreads the training pairs over
    the lengths and divergences of the evaluation pairs (one tree of fixed
    length has few close relatives among its pairs, and 4-mer count
    differences shrink relative to length as sequences grow).  With the
    defaults, 18 trees of 334 leaves give 999,702 pairs.
    Returns ``(X bf16 [N, 256], y fp32 [N], info)`` on the device, with
    y = f(a, b) / max(m, n).
    """
    Xs, ys = [], []
    t0 = time.perf_counter()
    i = 0
    for L in root_lens:
        for sc in scales:
            ds = synth.tree_dna(seed=seed * 1000 + i, n=n_per_tree, root_len=L,
                                sub_lo=0.005 * sc, sub_hi=0.05 * sc)
            i += 1
            sq = api.upload_and_pack(ctx, ds)
            prof = api.kmer_profile(ctx, sq)
            pairs = torch.from_numpy(synth.all_pairs(ds.n)).cuda()
            Xs.append(api.pair_features(ctx, sq, prof, pairs))
            d = api.lev_batch(ctx, sq, pairs)
            lens = torch.from_numpy(np.diff(ds.offs)).cuda()
            mx = torch.maximum(lens[pairs[:, 0].long()], lens[pairs[:, 1].long()]).clamp(min=1)
            ys.append((d.double() / mx.double()).float())
    ctx.check()
    X, y = torch.cat(Xs), torch.cat(ys)
    return X, y, dict(pairs=int(y.numel()), trees=i, seconds=time.perf_counter() - t0)


def train(ctx: api.Context, X: torch.Tensor, y: torch.Tensor, epochs: float = 4.0, batch: int = 4096,
          lr: float = 1e-3, tau: float = 0.9, seed: int = 0, val_frac: float = 0.1):
    """Adam on the pinball loss, minibatches drawn by a seeded permutation.

    Returns ``(model, info)`` with the validation loss and the validation row
    indices (a held-out 10% that training never sees).
    """
    rng = np.random.default_rng(seed)
    N = y.numel()
    perm = rng.permutation(N)
    nval = int(N * val_frac)
    val_idx, tr_idx = perm[:nval], perm[nval:]
    model = api.BandModel(ctx, seed=seed)
    steps = max(1, int(epochs * len(tr_idx) / batch))
    t0 = time.perf_counter()
    order = rng.permutation(tr_idx)
    pos = 0
    idx_dev = torch.empty(batch, dtype=torch.int32, device="cuda")
    losses = []
    for s in range(steps):
        if pos + batch > len(order):
            order = rng.permutation(tr_idx)
            pos = 0
        idx_dev.copy_(torch.from_numpy(order[pos:pos + batch].astype(np.int32)))
        pos += batch
        loss = model.train_step(X, y, idx_dev, lr=lr, tau=tau)
        if s % 50 == 0 or s == steps - 1:
            losses.append(loss)
    ctx.check()
    t_train = time.perf_counter() - t0
    # validation loss: gradient-only steps over the held-out rows
    vl = []
    for c0 in range(0, nval, batch):
        vi = torch.from_numpy(val_idx[c0:c0 + batch].astype(np.int32)).cuda()
        vl.append(model.train_step(X, y, vi, lr=0.0, tau=tau).item() * vi.numel())
        model.read_grad()
    info = dict(steps=steps, batch=batch, seconds=t_train, train_loss=[float(v) for v in losses[-3:]],
                val_loss=sum(vl) / max(1, nval), val_idx=val_idx)
    return model, info


def calibrate(ctx: api.Context, model: api.BandModel, seqs: api.DeviceSeqs, prof: torch.Tensor,
              pairs: torch.Tensor, tau: float = 0.95):
    """Fits the network's band calibration (``msa_band_calibrate``) on
    held-out pairs: the network's outputs beside the exact full-DP distances.

    The network is trained on pairs from simulated trees; on another
    population its output is not the tau-quantile it was trained for (on the
    divergent-pair evaluation recipe it runs high by 0.1 and more in y where
    most of the band cost lies), and one global margin cannot fix a bias
    that depends on yhat.  Returns the knots."""
    yhat, _ = model.predict_band(seqs, prof, pairs, gamma=0.0, margin=0)
    d = api.lev_batch(ctx, seqs, pairs)
    lens = seqs.offs[1:] - seqs.offs[:-1]
    mx = torch.maximum(lens[pairs[:, 0].long()], lens[pairs[:, 1].long()]).clamp(min=1)
    y = (d.double() / mx.double()).float()
    model.calibrate(yhat, y, tau=tau)
    ctx.check()
    return model.calibration()


def pick_gamma(ctx: api.Context, model: api.BandModel, seqs: api.DeviceSeqs, prof: torch.Tensor,
               pairs: torch.Tensor, candidates=(-0.15, -0.1, -0.05, 0.0, 0.05, 0.1, 0.2, 0.35), margin: int = 8,
               reps: int = 5, tolerance: float = 0.02):
    """The band margin gamma for the fastest certified banded run on a
    validation batch (median of ``reps`` runs timed with CUDA events; all
    candidates are exact).  Margins within ``tolerance`` of the fastest time
    count as equally fast (the timing batch and the batches the band serves
    differ by about that much), and the narrowest of them is taken: it
    computes the fewest cells.  Returns
    ``(gamma, ms)``."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for g in candidates:
        _, k = model.predict_band(seqs, prof, pairs, gamma=g, margin=margin)
        api.lev_banded_batch(ctx, seqs, pairs, k)
        ts = []
        for _ in range(reps):
            ev0.record()
            api.lev_banded_batch(ctx, seqs, pairs, k)
            ev1.record()
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        times.append(float(np.median(ts)))
    best_t = min(times)
    g, t = min(((g, t) for g, t in zip(candidates, times) if t <= best_t * (1.0 + tolerance)), key=lambda x: x[0])
    return g, t


def pick_band(ctx: api.Context, model: api.BandModel, cal_set, gamma_set, taus=(0.95, 0.99, 1.0),
              candidates=(-0.05, -0.025, 0.0, 0.025, 0.05, 0.1, 0.15, 0.25), margin: int = 8):
    """Calibration quantile tau and margin gamma together: for each tau the
    calibration is fitted on ``cal_set`` and gamma picked by timing on
    ``gamma_set`` (each a ``(seqs, prof, pairs)`` of held-out pairs; the
    timing set should be as large as the batches the band is for: a failed
    band's retry runs after the first pass, and a long pair's retry is a
    fixed latency that weighs more, and favours wider bands, in a smaller
    batch); the model is left calibrated with the best tau.  Returns
    ``(tau, gamma, ms)``; tau None is the network without calibration, when
    that is fastest."""
    best = (None, *pick_gamma(ctx, model, *gamma_set, candidates=candidates, margin=margin))
    for tau in taus:
        calibrate(ctx, model, *cal_set, tau=tau)
        g, t = pick_gamma(ctx, model, *gamma_set, candidates=candidates, margin=margin)
        if t < best[2]:
            best = (tau, g, t)
    if best[0] is None:
        model.calibrate(None, None)
    else:
        calibrate(ctx, model, *cal_set, tau=best[0])
    return best
