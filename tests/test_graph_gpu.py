"""The batch entry points enqueue only kernels, memsets and event waits on
the caller's stream (no host read-back, no allocation), so they can be
captured into a CUDA graph and replayed; the replayed results equal the
oracle's."""
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
    c = api.Context(0, workspace_bytes=1 << 28)
    yield c
    c.close()


def _capture(fn):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                      # warm-up outside the capture (tuning state, lazy attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def test_lev_batch_graph_replay(ctx):
    ds = synth.tree_dna(seed=9, n=48, root_len=700)
    pairs_np = synth.all_pairs(ds.n)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs_np)
    seqs = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(pairs_np).cuda()
    out = torch.full((len(pairs_np),), -1, dtype=torch.int32, device="cuda")
    g = _capture(lambda: api.lev_batch(ctx, seqs, pairs, out))
    for _ in range(2):
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_lev_batch_graph_sees_new_inputs(ctx):
    """A replay reads the buffers at replay time: new sequences written into
    the captured arena (same offsets) give the new distances."""
    a = synth.tree_dna(seed=10, n=32, root_len=500)
    b = synth.SeqSet.from_list([bytes(reversed(a.seq(i))) for i in range(a.n)])
    pairs_np = synth.all_pairs(a.n)
    seqs = api.upload_and_pack(ctx, a)
    pairs = torch.from_numpy(pairs_np).cuda()
    out = torch.empty(len(pairs_np), dtype=torch.int32, device="cuda")
    g = _capture(lambda: (api.pack(ctx, seqs), api.lev_batch(ctx, seqs, pairs, out)))
    seqs.ascii[:b.arena.size].copy_(torch.from_numpy(b.arena))
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.lev_pairs(b.arena, b.offs, pairs_np))


def test_banded_graph_replay(ctx):
    ds = synth.divergent_pairs(seed=41, n_pairs=96, len_lo=300, len_hi=3000)
    pairs_np = np.stack([np.arange(0, ds.n, 2), np.arange(1, ds.n, 2)], axis=1).astype(np.int32)
    ref = oracle.lev_pairs(ds.arena, ds.offs, pairs_np)
    seqs = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(pairs_np).cuda()
    k0 = torch.from_numpy((ref // 3).astype(np.int32)).cuda()     # too narrow: forces doubling rounds
    out = torch.empty(len(ref), dtype=torch.int32, device="cuda")
    k_used = torch.empty_like(out)
    g = _capture(lambda: api.lev_banded_batch(ctx, seqs, pairs, k0, out, k_used))
    out.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    ctx.check()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    assert np.all(k_used.cpu().numpy() >= ref)
