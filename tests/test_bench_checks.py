"""The oracle checks bench.py runs on the GPU's guide tree and merges,
exercised on the CPU against the oracle's own tree and MSA: they report no
mismatch there and catch planted ones."""
import types

import numpy as np
import torch

import bench
import oracle
from paper_2601_15458_gb300 import synth


def _as_gpu_outputs(ds):
    """The oracle's tree and merge in the shape the library returns them:
    BFS node arrays, the member order, per-residue root columns, node widths
    and merge costs."""
    seqs = ds.seqs()
    nodes = oracle.partition(seqs)
    rows, order, merges = oracle.merge_tree(seqs, nodes)
    n = len(nodes)
    tree = types.SimpleNamespace(n_nodes=n, lo=np.zeros(n, np.int32), hi=np.zeros(n, np.int32),
                                 center=np.array([nd["center"] for nd in nodes], np.int32),
                                 left=np.array([nd["left"] for nd in nodes], np.int32),
                                 right=np.array([nd["right"] for nd in nodes], np.int32),
                                 order=torch.tensor(order, dtype=torch.int32))
    tree.hi[0] = len(seqs)
    for k in range(n):            # parents come first in BFS order
        if tree.left[k] >= 0:
            nl = len(nodes[tree.left[k]]["members"])
            tree.lo[tree.left[k]], tree.hi[tree.left[k]] = tree.lo[k], tree.lo[k] + nl
            tree.lo[tree.right[k]], tree.hi[tree.right[k]] = tree.lo[k] + nl, tree.hi[k]
    pos = np.zeros(int(ds.offs[-1]), np.int32)
    for r, s in enumerate(order):
        cols = np.nonzero(np.frombuffer(rows[r], np.uint8) != ord("-"))[0]
        pos[ds.offs[s]:ds.offs[s + 1]] = cols
    width = np.array([len(bench._cols_of(tree, np.array(order), k, ds.offs, pos)) for k in range(n)], np.int32)
    score = np.full(n, -1, np.int32)
    for k, (sc, _) in merges.items():
        score[k] = sc
    return tree, pos, width, score, rows, order


def test_stepwise_merge_check_clean_and_planted():
    ds = synth.small_dna(seed=1, n=24)
    tree, pos, width, score, rows, order = _as_gpu_outputs(ds)
    internal = [k for k in range(tree.n_nodes) if tree.left[k] >= 0]
    r = bench.stepwise_merge_check(ds, tree, pos, width, score, internal)
    assert r["merges"] == len(internal) == ds.n - 1
    assert r["score_mismatches"] == r["script_mismatches"] == r["width_mismatches"] == 0
    bad = score.copy()
    bad[internal[3]] += 1
    assert bench.stepwise_merge_check(ds, tree, pos, width, bad, internal)["score_mismatches"] == 1
    # move the root's last column of one sequence: its merge script changes
    moved = pos.copy()
    s = int(order[0])
    moved[ds.offs[s + 1] - 1] += 1
    r = bench.stepwise_merge_check(ds, tree, moved, width, score, [0])
    assert r["script_mismatches"] + r["width_mismatches"] >= 1


def test_cluster_checks_and_rows():
    ds = synth.small_dna(seed=1, n=24)
    tree, pos, width, score, rows, order = _as_gpu_outputs(ds)
    internal = [k for k in range(tree.n_nodes) if tree.left[k] >= 0]
    assert bench.cluster_checks(ds.seqs(), tree, internal)["mismatches"] == 0
    tree.center[internal[2]] = tree.left[internal[2]]        # not a sequence of the cluster's medoid
    assert bench.cluster_checks(ds.seqs(), tree, internal)["mismatches"] >= 1
    R = np.frombuffer(b"".join(rows), np.uint8).reshape(len(rows), -1)
    assert bench.rows_match_sequences(R, order, ds)
    assert not bench.rows_match_sequences(R, order[::-1], ds)


def test_distance_invariants():
    offs = np.array([0, 3, 5, 5], np.int64)
    pairs = np.array([[0, 1], [0, 2], [1, 2]], np.int32)
    assert bench.distance_invariants(np.array([1, 3, 2]), pairs, offs) == 0
    assert bench.distance_invariants(np.array([0, 2, 3]), pairs, offs) == 3
