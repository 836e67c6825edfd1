"""msa_lev_batch_noalloc: the batched Levenshtein distance for callers that
cannot allocate device memory, checked against msa_lev_batch.

Who needs it: code that runs under another framework's memory budget (a
caching allocator that has reserved the free device memory), plug-ins that
must not allocate after start-up, and loops that cannot afford the implicit
synchronisation of an allocation.  The entry point takes no context and keeps
its scratch in a fixed device array inside the library, so these tests call
it through the C ABI exactly as such a caller would, twice in a row (the
array keeps the previous call's contents, which must not leak into the next
result).  This file is named to run last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_15458_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu

MSA_EINVAL = 1


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_15458_gb300 import build
    build.build()
    c = api.Context(0, workspace_bytes=256 << 20)
    yield c
    c.close()


def _noalloc(seqs, pairs: torch.Tensor) -> torch.Tensor:
    out = torch.full((pairs.shape[0],), -7, dtype=torch.int32, device="cuda")
    rc = _lib.lib().msa_lev_batch_noalloc(ctypes.byref(seqs.c), pairs.data_ptr(), pairs.shape[0], out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("alphabet", ["dna", "protein"])
def test_noalloc_matches_lev_batch_two_calls(ctx, alphabet):
    if alphabet == "dna":
        ds = synth.tree_dna(seed=13, n=300, root_len=800)
    else:
        ds = synth.protein_families(seed=3, n_fam=6, per_fam=40)[0]
    seqs = api.upload_and_pack(ctx, ds)
    calls = [torch.from_numpy(synth.all_pairs(ds.n)).cuda(),            # one-to-many: lane kernels
             torch.from_numpy(synth.random_pairs(14, ds.n, 5000)).cuda()]  # few targets per query: slot and warp kernels
    for pairs in calls:
        ref = api.lev_batch(ctx, seqs, pairs)
        ctx.check()
        got = _noalloc(seqs, pairs)
        assert torch.equal(got, ref)


def test_noalloc_long_queries_and_repeat(ctx):
    rng = np.random.default_rng(15)
    seqs_list = [rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes() for L in (0, 31, 65, 2049, 5000)]
    ds = synth.SeqSet.from_list(seqs_list)
    seqs = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(np.array([[i, j] for i in range(ds.n) for j in range(ds.n)], np.int32)).cuda()
    ref = api.lev_batch(ctx, seqs, pairs)
    ctx.check()
    first = _noalloc(seqs, pairs)
    second = _noalloc(seqs, pairs)
    assert torch.equal(first, ref) and torch.equal(second, ref)


def test_noalloc_rejects_sizes_beyond_its_maximum(ctx):
    ds = synth.small_dna(seed=1, n=4)
    seqs = api.upload_and_pack(ctx, ds)
    dummy = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc = _lib.lib().msa_lev_batch_noalloc(ctypes.byref(seqs.c), dummy.data_ptr(), (1 << 18) + 1, dummy.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
    assert rc == MSA_EINVAL
