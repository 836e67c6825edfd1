"""Guide tree (Alg. 1, A11) and bottom-up merge (section "Merging", A12)
on the GPU against the oracle: identical trees, identical MSAs."""
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


def _gpu_nodes(tree):
    order = tree.order.cpu().numpy()
    out = []
    for k in range(tree.n_nodes):
        out.append(dict(members=sorted(int(x) for x in order[tree.lo[k]:tree.hi[k]]), center=int(tree.center[k]),
                        left=int(tree.left[k]), right=int(tree.right[k]), parent=int(tree.parent[k])))
    return out


def _check_same_tree(gpu, ref):
    assert len(gpu) == len(ref)
    for g, r in zip(gpu, ref):
        assert g == r


def _full(ctx, ds, gap_open=None):
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    pos, width, score = api.merge_tree(ctx, sq, tree, gap_open=gap_open)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0]))
    ctx.check()
    return sq, tree, width, score, rows.cpu().numpy()


def test_line_metric_tree(ctx):
    ds = synth.SeqSet.from_list([b"A" * k for k in range(1, 8)])
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    ctx.check()
    _check_same_tree(_gpu_nodes(tree), oracle.partition(ds.seqs()))


@pytest.mark.parametrize("maker", [lambda: synth.small_dna(seed=1),
                                   lambda: synth.protein_families(seed=3, n_fam=3, per_fam=30)[0]])
def test_tree_and_msa_match_oracle(ctx, maker):
    ds = maker()
    seqs = ds.seqs()
    sq, tree, width, score, rows = _full(ctx, ds)
    ref_nodes = oracle.partition(seqs)
    _check_same_tree(_gpu_nodes(tree), ref_nodes)
    ref_rows, ref_order, merges = oracle.merge_tree(seqs, ref_nodes)
    assert list(tree.order.cpu().numpy()) == ref_order
    assert [r.tobytes() for r in rows] == ref_rows
    for k, (sc, _) in merges.items():
        assert score[k] == sc
    assert width[0] == len(ref_rows[0])


def test_larger_tree_sampled_nodes(ctx):
    """A 1,500-sequence 16S-like set: invariants everywhere, and Alg. 1 redone
    by the oracle on sampled clusters (including sampled-medoid ones)."""
    ds = synth.gg16s_dna(seed=5, n=1500)
    seqs = ds.seqs()
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    ctx.check()
    nodes = _gpu_nodes(tree)
    assert tree.n_nodes == 2 * ds.n - 1
    leaves = [nd for nd in nodes if nd["left"] < 0]
    assert sorted(nd["members"][0] for nd in leaves) == list(range(ds.n))
    rng = np.random.default_rng(0)
    internal = [k for k, nd in enumerate(nodes) if nd["left"] >= 0]
    big = [k for k in internal if len(nodes[k]["members"]) > 256][:2]
    small = list(rng.choice([k for k in internal if 2 <= len(nodes[k]["members"]) <= 40], 6, replace=False))
    for k in big + small:
        nd = nodes[k]
        mem = nd["members"]
        # one application of Alg. 1 to the cluster (the oracle's batched step)
        step = oracle.partition_levels([seqs[x] for x in mem], max_levels=1)
        assert nd["center"] == mem[step[0]["center"]]
        assert nodes[nd["left"]]["members"] == [mem[i] for i in step[1]["members"]]
        assert nodes[nd["right"]]["members"] == [mem[i] for i in step[2]["members"]]
    # merge: rows de-gap to their sequences, equal widths
    pos, width, score = api.merge_tree(ctx, sq, tree)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0])).cpu().numpy()
    ctx.check()
    order = tree.order.cpu().numpy()
    for r in rng.choice(ds.n, 50, replace=False):
        assert rows[r].tobytes().replace(b"-", b"") == seqs[order[r]]
    assert not np.any(np.all(rows == ord("-"), axis=0))


def test_small_cluster_matrices_any_pool_size(ctx):
    """Clusters of at most 256 members read their distances from matrices
    kept in the workspace, as many as the pool (a quarter of the free
    workspace) holds; the others compute them.  Workspaces from one that
    holds few matrices to one that holds all give the same tree, and that
    tree matches the oracle's step on sampled clusters."""
    ds = synth.gg16s_dna(seed=7, n=700)
    seqs = ds.seqs()
    trees = []
    for ws in (2 << 20, 5 << 19, 3 << 20, 1 << 30):
        c = api.Context(0, workspace_bytes=ws)
        try:
            sq = api.upload_and_pack(c, ds)
            tree = api.clam_partition(c, sq)
            c.check()
            trees.append(_gpu_nodes(tree))
        except api.MsaError:
            pass                              # a level needs more than this workspace
        finally:
            c.close()
    assert len(trees) >= 2
    for t in trees[1:]:
        _check_same_tree(t, trees[0])
    nodes = trees[0]
    rng = np.random.default_rng(1)
    internal = [k for k, nd in enumerate(nodes) if nd["left"] >= 0]
    for k in [internal[0]] + list(rng.choice([k for k in internal if 2 <= len(nodes[k]["members"]) <= 64], 6,
                                            replace=False)):
        nd = nodes[k]
        mem = nd["members"]
        step = oracle.partition_levels([seqs[x] for x in mem], max_levels=1)
        assert nd["center"] == mem[step[0]["center"]]
        assert nodes[nd["left"]]["members"] == [mem[i] for i in step[1]["members"]]


def test_protein_families_tree_and_merges_full_size(ctx):
    """The 10,000-protein workload (100 families, 10-40% mutation): Alg. 1
    over all members and all 9,999 guide-tree merges, against the oracle
    run end to end on the same sequences (its level-batched partition and
    merge): every node and centre, every merge cost, and every row of the
    root MSA -- which fixes each merge's edit script, since a node's columns
    are the root columns its members' residues occupy."""
    members, _ = synth.protein_families(seed=3)
    assert members.n == 10000
    seqs = members.seqs()
    sq, tree, width, score, rows = _full(ctx, members)
    assert tree.n_nodes == 2 * members.n - 1
    ref_nodes = oracle.partition_levels(seqs)
    _check_same_tree(_gpu_nodes(tree), ref_nodes)
    ref_rows, ref_order, merges = oracle.merge_tree_levels(seqs, ref_nodes)
    assert list(tree.order.cpu().numpy()) == ref_order
    assert len(merges) == 9999
    for k, (sc, _) in merges.items():
        assert score[k] == sc
    assert width[0] == len(ref_rows[0])
    assert [r.tobytes() for r in rows] == ref_rows


@pytest.mark.parametrize("gamma", [0.2, -0.9])
def test_banded_partition_same_tree(ctx, gamma):
    """Alg. 1 with every distance batch from the network's band and the
    certified banded DP: the same tree as the full DP, whatever the network
    (an untrained one here; gamma = -0.9 starts almost every band too narrow,
    so the retries decide)."""
    model = api.BandModel(ctx, seed=0)
    ds = synth.small_dna(seed=1)
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq, band=model, gamma=gamma, margin=0)
    ctx.check()
    _check_same_tree(_gpu_nodes(tree), oracle.partition(ds.seqs()))
    ds = synth.gg16s_dna(seed=5, n=1500)
    sq = api.upload_and_pack(ctx, ds)
    full = api.clam_partition(ctx, sq)
    banded = api.clam_partition(ctx, sq, band=model, gamma=gamma, margin=0)
    ctx.check()
    _check_same_tree(_gpu_nodes(banded), _gpu_nodes(full))


def test_banded_partition_rejects_protein(ctx):
    model = api.BandModel(ctx, seed=0)
    members, _ = synth.protein_families(seed=3, n_fam=2, per_fam=5)
    sq = api.upload_and_pack(ctx, members)
    prof = torch.zeros((members.n, 256), dtype=torch.int16, device="cuda")
    with pytest.raises(api.MsaError):
        api.clam_partition(ctx, sq, band=model, prof=prof)


def _metrics_check(ctx, ds, sample):
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    pos, width, score = api.merge_tree(ctx, sq, tree)
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0]))
    ctx.check()
    got = api.msa_metrics(ctx, sq, tree, rows, sample=sample, seed=3)
    order = tree.order.cpu().numpy()
    host_rows = rows.cpu().numpy()
    pick = got["sample"]
    seqs = ds.seqs()
    pct, p, dist, n = oracle.msa_metrics([host_rows[r].tobytes() for r in pick], [seqs[order[r]] for r in pick])
    assert (got["gaps"], got["compared"], got["mismatched"], got["pairs"]) == \
        (n["gaps"], n["compared"], n["mismatched"], n["pairs"])
    assert got["pct_gaps"] == pytest.approx(pct, rel=1e-12, abs=1e-12)
    assert got["p_score"] == pytest.approx(p, rel=1e-12, abs=1e-12)
    assert got["distortion"] == pytest.approx(dist, rel=1e-12)
    assert got["distortion"] >= 1.0
    return got


def test_msa_metrics_small_all_rows(ctx):
    _metrics_check(ctx, synth.small_dna(seed=1), None)


def test_msa_metrics_16s_sample(ctx):
    """A seeded 130-row sample of a 1,500-sequence 16S-like MSA (two 64-row
    tiles and a ragged one in the Hamming kernel)."""
    _metrics_check(ctx, synth.gg16s_dna(seed=5, n=1500), 130)


def test_msa_metrics_protein(ctx):
    members, _ = synth.protein_families(seed=3, n_fam=3, per_fam=30)
    _metrics_check(ctx, members, None)



@pytest.mark.parametrize("maker", [lambda: synth.small_dna(seed=1),
                                   lambda: synth.protein_families(seed=3, n_fam=3, per_fam=30)[0]])
def test_affine_merge_matches_oracle(ctx, maker):
    """The merge with affine gaps (open 10, extend 1): identical MSA rows and
    per-merge scores to the oracle's post-order merge."""
    ds = maker()
    seqs = ds.seqs()
    sq, tree, width, score, rows = _full(ctx, ds, gap_open=10)
    ref_nodes = oracle.partition(seqs)
    ref_rows, ref_order, merges = oracle.merge_tree(seqs, ref_nodes, gap=1, gap_open=10)
    assert list(tree.order.cpu().numpy()) == ref_order
    assert [r.tobytes() for r in rows] == ref_rows
    for k, (sc, _) in merges.items():
        assert score[k] == sc


def test_blosum62_merge_matches_oracle(ctx):
    """The paper's protein setting (section "Implementation"): merges with
    BLOSUM62 substitution costs and affine gaps (open 10, extend 1), the gap
    of a centre row read as BLOSUM62's '*'; identical MSA rows and per-merge
    costs to the oracle's post-order merge."""
    ds = synth.protein_families(seed=3, n_fam=3, per_fam=30)[0]
    seqs = ds.seqs()
    sq = api.upload_and_pack(ctx, ds)
    tree = api.clam_partition(ctx, sq)
    pos, width, score = api.merge_tree(ctx, sq, tree, gap=1, gap_open=10, sub=api.blosum62_table())
    rows = api.msa_rows(ctx, sq, tree, pos, int(width[0])).cpu().numpy()
    ctx.check()
    ref_nodes = oracle.partition(seqs)
    ref_rows, ref_order, merges = oracle.merge_tree(seqs, ref_nodes, gap=1, gap_open=10, sub=oracle.blosum62_costs())
    assert list(tree.order.cpu().numpy()) == ref_order
    assert [r.tobytes() for r in rows] == ref_rows
    for k, (sc, _) in merges.items():
        assert score[k] == sc
