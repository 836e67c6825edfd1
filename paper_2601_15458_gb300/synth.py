"""Seeded synthetic sequence generators shaped like the paper's workloads.

The paper's datasets (Greengenes 16S DNA, lengths 1,111-2,368 with median
about 1,375; PDB proteins 30-1,000 with median 224; Pfam with median 236-255
and a long tail; Table 1) are not available here, so these generators stand in
for them.  This module holds none of the method's arithmetic: it only draws
random sequences.  Both the CUDA path and the CPU oracle consume what it
returns, so it is the one module they share.

Every generator is deterministic in its seed (numpy PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DNA = b"ACGT"
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"


@dataclass
class SeqSet:
    """Ragged sequences in one ASCII arena: sequence s is arena[offs[s]:offs[s+1]]."""
    arena: np.ndarray            # uint8
    offs: np.ndarray             # int64 [n + 1]
    alphabet: str = "dna"        # "dna" | "protein"
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.offs) - 1

    @property
    def lens(self) -> np.ndarray:
        return np.diff(self.offs)

    def seq(self, i: int) -> bytes:
        return self.arena[self.offs[i]:self.offs[i + 1]].tobytes()

    def seqs(self) -> list:
        return [self.seq(i) for i in range(self.n)]

    @staticmethod
    def from_list(seqs, alphabet="dna", extra=None) -> "SeqSet":
        lens = np.array([len(s) for s in seqs], dtype=np.int64)
        offs = np.zeros(len(seqs) + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        arena = np.frombuffer(b"".join(bytes(s) for s in seqs), dtype=np.uint8).copy()
        if arena.size == 0:
            arena = np.zeros(0, dtype=np.uint8)
        return SeqSet(arena, offs, alphabet, dict(extra or {}))


# ---------------------------------------------------------------------------
# mutation model
# ---------------------------------------------------------------------------

def _codes(seq: np.ndarray, alphabet: bytes) -> np.ndarray:
    lut = np.full(256, 255, dtype=np.uint8)
    lut[np.frombuffer(alphabet, dtype=np.uint8)] = np.arange(len(alphabet), dtype=np.uint8)
    return lut[seq]


def random_seq(rng, length: int, probs: np.ndarray) -> np.ndarray:
    """``length`` symbol codes drawn i.i.d. from ``probs``."""
    if np.all(probs == probs[0]):
        return rng.integers(0, len(probs), size=length).astype(np.uint8)
    return rng.choice(len(probs), size=length, p=probs).astype(np.uint8)


def mutate(rng, seq: np.ndarray, sub_rate: float, indel_rate: float, probs: np.ndarray) -> np.ndarray:
    """Per-site substitutions and indel events on a code array.

    Each site is substituted with probability ``sub_rate`` by a symbol drawn
    from the background ``probs`` conditioned on differing from the current
    one.  Independently, an indel event starts at a site with probability
    ``indel_rate``; it is an insertion or a deletion with probability 1/2
    each, of length Geometric(p=0.5) on {1, 2, ...}.  A deletion at site i of
    length L removes sites i .. i+L-1 (overlapping deletions remove their
    union); an insertion at site i puts L background symbols before site i
    (several at one site are concatenated, the site itself may be deleted).
    """
    out = seq.copy()
    n = len(out)
    if n == 0:
        return out
    sub = rng.random(n) < sub_rate
    idx = np.nonzero(sub)[0]
    if len(idx):
        cur = out[idx]
        new = random_seq(rng, len(idx), probs)
        bad = new == cur
        while bad.any():
            new[bad] = random_seq(rng, int(bad.sum()), probs)
            bad = new == cur
        out[idx] = new
    ev = np.nonzero(rng.random(n) < indel_rate)[0]
    if len(ev) == 0:
        return out
    ins = rng.random(len(ev)) < 0.5
    lengths = rng.geometric(0.5, size=len(ev)).astype(np.int64)
    # deletions: coverage by a difference array
    cover = np.zeros(n + 1, np.int64)
    dpos, dlen = ev[~ins], lengths[~ins]
    np.add.at(cover, dpos, 1)
    np.add.at(cover, np.minimum(dpos + dlen, n), -1)
    keep = (np.cumsum(cover[:n]) == 0).astype(np.int64)
    # insertions: symbols placed before their site
    ins_at = np.zeros(n, np.int64)
    np.add.at(ins_at, ev[ins], lengths[ins])
    contrib = ins_at + keep
    start = np.cumsum(contrib) - contrib
    total = int(contrib.sum())
    res = np.empty(total, np.uint8)
    kept = np.nonzero(keep)[0]
    res[start[kept] + ins_at[kept]] = out[kept]
    tot_ins = int(ins_at.sum())
    if tot_ins:
        sites = np.nonzero(ins_at)[0]
        reps = ins_at[sites]
        base = np.repeat(start[sites], reps)
        within = np.arange(tot_ins) - np.repeat(np.cumsum(reps) - reps, reps)
        res[base + within] = random_seq(rng, tot_ins, probs)
    return res


def yule_tree(rng, n_leaves: int):
    """Random binary tree by the Yule process: split a uniformly chosen leaf.

    Returns ``parent`` (int array over nodes, -1 for the root) and the list
    of leaf node ids in creation order.  Node 0 is the root.
    """
    parent = [-1]
    leaves = [0]
    while len(leaves) < n_leaves:
        k = int(rng.integers(len(leaves)))
        v = leaves[k]
        a, b = len(parent), len(parent) + 1
        parent += [v, v]
        leaves[k] = a
        leaves.append(b)
    return np.array(parent, dtype=np.int64), leaves


def _simulate_tree(rng, n_leaves, root, branch_rates, probs, accept=None, max_redraw=200):
    """Sequences at the leaves of a Yule tree, mutating down every branch.

    ``branch_rates(rng) -> (sub_rate, indel_rate)`` is drawn per branch.  A
    leaf whose sequence fails ``accept`` or duplicates an earlier leaf has its
    last branch re-simulated.
    """
    parent, leaves = yule_tree(rng, n_leaves)
    children = [[] for _ in range(len(parent))]
    for v in range(1, len(parent)):
        children[parent[v]].append(v)
    seqs = {0: root}
    stack = [0]
    while stack:
        v = stack.pop()
        for c in children[v]:
            seqs[c] = mutate(rng, seqs[v], *branch_rates(rng), probs)
            stack.append(c)
    out = []
    seen = set()
    for v in leaves:
        s = seqs[v]
        tries = 0
        while (accept is not None and not accept(s)) or s.tobytes() in seen:
            tries += 1
            if tries > max_redraw:
                raise RuntimeError("could not draw an acceptable leaf")
            s = mutate(rng, seqs[parent[v]], *branch_rates(rng), probs)
        seen.add(s.tobytes())
        out.append(s)
    return out, parent, leaves


def _to_seqset(code_seqs, alphabet_bytes, name, extra=None) -> SeqSet:
    table = np.frombuffer(alphabet_bytes, dtype=np.uint8)
    return SeqSet.from_list([table[s].tobytes() for s in code_seqs],
                            "dna" if alphabet_bytes == DNA else "protein", extra)


def _dedup(rng, seqs, redraw):
    seen = set()
    out = []
    for s in seqs:
        while s.tobytes() in seen:
            s = redraw()
        seen.add(s.tobytes())
        out.append(s)
    return out


UNIFORM4 = np.full(4, 0.25)

# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def small_dna(seed: int = 1, n: int = 64, root_len: int = 150,
              sub_rate: float = 0.05, indel_rate: float = 0.01) -> SeqSet:
    """64 DNA sequences: each leaf = uniform root of length 150 with 5%
    per-site substitution and 1% per-site indel events (lengths ~130-170)."""
    rng = np.random.default_rng(seed)
    root = random_seq(rng, root_len, UNIFORM4)
    seqs = [mutate(rng, root, sub_rate, indel_rate, UNIFORM4) for _ in range(n)]
    seqs = _dedup(rng, seqs, lambda: mutate(rng, root, sub_rate, indel_rate, UNIFORM4))
    return _to_seqset(seqs, DNA, "small_dna")


def tree_dna(seed: int = 2, n: int = 2000, root_len: int = 1500,
             sub_lo: float = 0.005, sub_hi: float = 0.05, indel_frac: float = 0.2,
             accept_len=None) -> SeqSet:
    """DNA simulated down a Yule tree from a uniform root.

    Per branch the substitution rate is U(sub_lo, sub_hi) and the indel rate
    ``indel_frac`` times that.  With the defaults: 2,000 sequences of lengths
    about 1,200-1,800.  ``accept_len=(lo, hi)`` re-simulates any leaf whose
    length falls outside [lo, hi].
    """
    rng = np.random.default_rng(seed)
    root = random_seq(rng, root_len, UNIFORM4)

    def rates(r):
        s = float(r.uniform(sub_lo, sub_hi))
        return s, s * indel_frac

    accept = None
    if accept_len is not None:
        lo, hi = accept_len
        accept = lambda s: lo <= len(s) <= hi  # noqa: E731
    seqs, _, _ = _simulate_tree(rng, n, root, rates, UNIFORM4, accept)
    return _to_seqset(seqs, DNA, "tree_dna")


def gg16s_dna(seed: int = 5, n: int = 50000) -> SeqSet:
    """16S-like DNA: Yule tree of ``n`` leaves, root length 1,500, per-branch
    substitution U(0.002, 0.03), indels 0.1x that; leaves kept only with
    length in [1,400, 1,600] (re-simulated otherwise)."""
    return tree_dna(seed=seed, n=n, root_len=1500, sub_lo=0.002, sub_hi=0.03,
                    indel_frac=0.1, accept_len=(1400, 1600))


def protein_families(seed: int = 3, n_fam: int = 100, per_fam: int = 100,
                     median: float = 300.0, sigma: float = 0.6, clip=(50, 1000)):
    """Protein families: background ~ Dirichlet(1^20); family roots of
    log-normal length (median 300, sigma 0.6, clipped to [50, 1000]); each
    member mutated from its root at a rate U(0.10, 0.40) of which 80% are
    substitutions and 20% indel events; member lengths clipped to [50, 1000].

    Returns ``(members, roots)``: 10,000 member sequences and the 100 family
    roots as a separate set.
    """
    rng = np.random.default_rng(seed)
    probs = rng.dirichlet(np.ones(20))
    roots = []
    for _ in range(n_fam):
        L = int(np.clip(round(median * np.exp(sigma * rng.standard_normal())), *clip))
        roots.append(random_seq(rng, L, probs))
    roots = _dedup(rng, roots, lambda: random_seq(rng, int(median), probs))
    members = []
    fam = []
    seen = set()
    for f, root in enumerate(roots):
        for _ in range(per_fam):
            while True:
                rate = float(rng.uniform(0.10, 0.40))
                s = mutate(rng, root, 0.8 * rate, 0.2 * rate, probs)
                if clip[0] <= len(s) <= clip[1] and s.tobytes() not in seen:
                    break
            seen.add(s.tobytes())
            members.append(s)
            fam.append(f)
    extra = dict(family=np.array(fam, dtype=np.int32), background=probs)
    return (_to_seqset(members, PROTEIN, "protein_families", extra),
            _to_seqset(roots, PROTEIN, "protein_roots", dict(background=probs)))


_C_LIB = None


def _c_lib():
    """The compiled pair generator (``synth_c/synth_pairs.c``), built with gcc on first use."""
    global _C_LIB
    if _C_LIB is None:
        import ctypes
        import os
        import subprocess
        here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_c")
        src, so = os.path.join(here, "synth_pairs.c"), os.path.join(here, "libsynth_pairs.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src, "-o", tmp])
            os.replace(tmp, so)
        L = ctypes.CDLL(so)
        L.synth_divergent_pairs.restype = ctypes.c_int32
        L.synth_divergent_pairs.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32]
        L.synth_compact_pairs.restype = None
        L.synth_compact_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p]
        _C_LIB = L
    return _C_LIB


def divergent_pairs(seed: int = 40, n_pairs: int = 100000, len_lo: int = 1000,
                    len_hi: int = 10000, div_lo: float = 0.01, div_hi: float = 0.30,
                    indel_share: float = 0.2, threads: int | None = None) -> SeqSet:
    """Independent DNA pairs: a uniform root of length U{len_lo..len_hi} and a
    partner mutated from it at divergence delta ~ U(div_lo, div_hi): per root
    site an indel event with probability indel_share * delta (insertion or
    deletion, Geometric(1/2) length), else a substitution with probability
    delta.  Sequence 2p is the root of pair p, sequence 2p+1 its partner.
    Generated by ``synth_c/synth_pairs.c`` (one SplitMix64 stream per pair)."""
    import os
    L = _c_lib()
    slab = 3 * len_hi + 64
    buf = np.empty(n_pairs * slab, np.uint8)
    lens = np.zeros(2 * n_pairs, np.int32)
    nt = threads or min(32, os.cpu_count() or 1)
    rc = L.synth_divergent_pairs(seed, n_pairs, len_lo, len_hi, div_lo, div_hi, indel_share,
                                 buf.ctypes.data, slab, lens.ctypes.data, nt)
    if rc != 0:
        raise RuntimeError("divergent_pairs: a partner overflowed its slab")
    lens64 = lens.astype(np.int64)
    offs = np.zeros(2 * n_pairs + 1, np.int64)
    np.cumsum(lens64, out=offs[1:])
    codes = np.empty(int(offs[-1]), np.uint8)
    L.synth_compact_pairs(buf.ctypes.data, slab, lens.ctypes.data, n_pairs, offs.ctypes.data, codes.ctypes.data)
    return SeqSet(codes, offs, "dna")


# ---------------------------------------------------------------------------
# pair lists
# ---------------------------------------------------------------------------

def all_pairs(n: int) -> np.ndarray:
    """All unordered pairs (i, j), i < j, as int32 [n(n-1)/2, 2], grouped by i."""
    i, j = np.triu_indices(n, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


def all_pairs_balanced(n: int) -> np.ndarray:
    """All unordered pairs, each listed once, grouped by a first index that
    owns about (n-1)/2 of them: i pairs with i+1..i+h (mod n), h = (n-1)//2,
    and for even n the first n/2 rows also take i + n/2."""
    h = (n - 1) // 2
    rows = []
    for i in range(n):
        js = [(i + d) % n for d in range(1, h + 1)]
        if n % 2 == 0 and i < n // 2:
            js.append(i + n // 2)
        rows.append(np.stack([np.full(len(js), i), np.array(js)], axis=1))
    return np.concatenate(rows).astype(np.int32) if rows else np.zeros((0, 2), np.int32)


def random_pairs(seed: int, n: int, P: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=(P, 2)).astype(np.int32)
