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

import oracle
from paper_2601_15458_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu

MSA_EINVAL = 1
MSA_EUNSUPPORTED = 5


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


def _call_raw(c, pairs_ptr, P, out_ptr):
    return _lib.lib().msa_lev_batch_noalloc(ctypes.byref(c) if c is not None else None, pairs_ptr, P, out_ptr,
                                            torch.cuda.current_stream().cuda_stream)


def _variant(seqs, **kw):
    """A copy of the set's C descriptor with some fields replaced."""
    c = _lib.SeqSetC()
    ctypes.pointer(c)[0] = seqs.c
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("case,code", [
    ("too_many_pairs", MSA_EINVAL), ("too_many_seqs", MSA_EINVAL), ("no_seqs", MSA_EINVAL),
    ("null_pairs", MSA_EINVAL), ("null_out", MSA_EINVAL), ("null_set", MSA_EINVAL), ("null_offs", MSA_EINVAL),
    ("bad_alphabet", MSA_EINVAL), ("negative_max_len", MSA_EINVAL), ("max_len_beyond_kernels", MSA_EUNSUPPORTED),
    ("negative_P", MSA_EINVAL)])
def test_noalloc_rejects_bad_calls_before_enqueueing(ctx, case, code):
    """Every rejection happens on the host: d_out keeps its sentinel, so
    nothing was enqueued."""
    ds = synth.small_dna(seed=1, n=4)
    seqs = api.upload_and_pack(ctx, ds)
    pairs = torch.tensor([[0, 1], [2, 3]], dtype=torch.int32, device="cuda")
    out = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    c, pp, P, op = seqs.c, pairs.data_ptr(), 2, out.data_ptr()
    if case == "too_many_pairs":
        P = (1 << 18) + 1
    elif case == "too_many_seqs":
        c = _variant(seqs, n_seqs=(1 << 16) + 1)
    elif case == "no_seqs":
        c = _variant(seqs, n_seqs=0)
    elif case == "null_pairs":
        pp = None
    elif case == "null_out":
        op = None
    elif case == "null_set":
        c = None
    elif case == "null_offs":
        c = _variant(seqs, offs=None)
    elif case == "bad_alphabet":
        c = _variant(seqs, alphabet=7)
    elif case == "negative_max_len":
        c = _variant(seqs, max_len=-1)
    elif case == "max_len_beyond_kernels":
        c = _variant(seqs, max_len=16385)
    elif case == "negative_P":
        P = -1
    assert _call_raw(c, pp, P, op) == code
    torch.cuda.synchronize()
    assert out.tolist() == [-7, -7]


def test_noalloc_bad_index_and_overlong_query_give_minus_one(ctx):
    """No context means no error word: a pair with an index outside the set,
    or whose first sequence is longer than the set's max_len (here a
    17,000-residue sequence described with max_len 16,384, the most the
    kernels hold), comes back as -1; every other pair is exact."""
    rng = np.random.default_rng(16)
    rows = [rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes() for L in (300, 17000, 450, 40)]
    ds = synth.SeqSet.from_list(rows)
    seqs = api.upload_and_pack(ctx, ds)
    ctx.check()
    c = _variant(seqs, max_len=16384)
    pairs_np = np.array([[0, 2], [0, 4], [-1, 2], [1, 0], [3, 1], [2, 3], [4, 4]], np.int32)
    pairs = torch.from_numpy(pairs_np).cuda()
    for _ in range(2):
        out = torch.full((len(pairs_np),), -7, dtype=torch.int32, device="cuda")
        assert _call_raw(c, pairs.data_ptr(), len(pairs_np), out.data_ptr()) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ok = [0, 4, 5]
        ref = oracle.lev_pairs(ds.arena, ds.offs, pairs_np[ok])
        np.testing.assert_array_equal(got[ok], ref)
        assert list(got[[1, 2, 3, 6]]) == [-1, -1, -1, -1]


def test_noalloc_allocates_nothing(ctx):
    """After a first call (which does the one-time set-up), further calls
    leave the device's free memory exactly as it was and match
    msa_lev_batch."""
    ds = synth.tree_dna(seed=17, n=200, root_len=600)
    seqs = api.upload_and_pack(ctx, ds)
    pairs = torch.from_numpy(synth.all_pairs(ds.n)).cuda()
    ref = api.lev_batch(ctx, seqs, pairs)
    ctx.check()
    outs = [torch.full((pairs.shape[0],), -7, dtype=torch.int32, device="cuda") for _ in range(4)]
    assert _call_raw(seqs.c, pairs.data_ptr(), pairs.shape[0], outs[0].data_ptr()) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs[1:]:
        assert _call_raw(seqs.c, pairs.data_ptr(), pairs.shape[0], out.data_ptr()) == 0
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    for out in outs:
        assert torch.equal(out, ref)
