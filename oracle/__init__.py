"""Plain CPU oracle for the batched alignment DP of MuSAlS (arXiv 2601.15458).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and imports nothing from it.
Every function takes raw byte strings (ASCII residues, ``-`` for a gap) and
computes the plain definition of what the GPU path computes:

* :func:`lev` / :func:`lev_pairs` -- the Levenshtein distance ``f`` of
  Alg. 1 (section "Clustering"), full-matrix Wagner-Fischer (``oracle.c``).
* :func:`nw` / :func:`nw_pairs` -- Needleman-Wunsch (section "Merging",
  step 2) as a minimum-cost DP with a flat cost model and the traceback
  preference diagonal > up > left (``oracle.c``).
* :func:`nw_affine` -- the same with affine gap costs (Gotoh), the cost model
  of the paper's experiments, with flat substitution costs or a table
  (:func:`blosum62_costs`: BLOSUM62, which the paper names for proteins).
* :func:`brute_alignments` -- every alignment of two short strings, used to
  pin the functions above.
* :func:`nw_anchored` -- NW split at unique k-mer anchors, linear or affine
  gaps, flat costs or a table (the paper's future work for long pairs; this
  project's definition).
* :func:`kmer_counts`, :func:`pair_feature` -- 4-mer count profiles and the
  pair feature of the learned band proposer (no counterpart in the paper; the
  definition is this project's).
* :func:`mlp_forward`, :func:`mlp_backward`, :func:`adam_step` -- the band
  proposer network 256->128->64->1 in float64 on bf16-rounded operands.
* :func:`band_policy`, :func:`band_calibrate` -- the starting band from the
  network's output and its per-bin quantile calibration (this project's).
* :func:`partition` -- Alg. 1 ``Partition`` with the readings listed in the
  design notes (medoid sample rule, tie-breaks).
* :func:`merge_tree` -- the post-order merge of section "Merging".
* :func:`partition_levels`, :func:`merge_tree_levels` -- the same two with
  the distances / alignments of one tree level gathered into one batch, for
  sets too large for the per-pair versions (pinned to them in the tests).
* :func:`msa_metrics` -- the alignment quality metrics of section
  "Evaluation": percentage of gaps, p-score, distance distortion.

Functions that no independent fact pins say "parity unpinned" in their
docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``liboracle.so`` (host code only)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.oracle_lev.restype = ctypes.c_int32
            L.oracle_lev.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64]
            L.oracle_nw.restype = ctypes.c_int32
            L.oracle_nw.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    i32p, u8p, i64p]
            L.oracle_nw_affine.restype = ctypes.c_int32
            L.oracle_nw_affine.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           i32p, u8p, i64p]
            L.oracle_nw_affine_sub.restype = ctypes.c_int32
            L.oracle_nw_affine_sub.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i32p,
                                               ctypes.c_int32, ctypes.c_int32, i32p, u8p, i64p]
            L.oracle_lev_pairs.restype = ctypes.c_int32
            L.oracle_lev_pairs.argtypes = [u8p, i64p, i32p, ctypes.c_int64, i32p, ctypes.c_int32]
            L.oracle_nw_pairs.restype = ctypes.c_int32
            L.oracle_nw_pairs.argtypes = [u8p, i64p, i32p, ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          i32p, u8p, i64p, i64p, ctypes.c_int32]
            _lib = L
    return _lib


def _ptr(arr: np.ndarray, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _as_u8(s) -> np.ndarray:
    if isinstance(s, np.ndarray):
        return np.ascontiguousarray(s, dtype=np.uint8)
    return np.frombuffer(bytes(s), dtype=np.uint8).copy()


def cpu_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# Levenshtein and Needleman-Wunsch (C, full matrix)
# ---------------------------------------------------------------------------

def lev(a, b) -> int:
    """Unit-cost edit distance f(a, b) of Alg. 1, full-matrix Wagner-Fischer."""
    A, B = _as_u8(a), _as_u8(b)
    d = _load().oracle_lev(_ptr(A, ctypes.c_uint8), len(A), _ptr(B, ctypes.c_uint8), len(B))
    if d < 0:
        raise MemoryError("oracle_lev: matrix allocation failed")
    return int(d)


def nw(a, b, match: int = 0, mismatch: int = 1, gap: int = 1):
    """Minimum-cost global alignment (section "Merging", step 2).

    Returns ``(score, ops)`` with ``ops`` a bytes string over ``M X D I``
    in forward order; ``D`` consumes a residue of ``a`` against a gap, ``I``
    consumes a residue of ``b`` against a gap.
    """
    A, B = _as_u8(a), _as_u8(b)
    ops = np.zeros(len(A) + len(B) + 1, dtype=np.uint8)
    score = ctypes.c_int32(0)
    L = ctypes.c_int64(0)
    rc = _load().oracle_nw(_ptr(A, ctypes.c_uint8), len(A), _ptr(B, ctypes.c_uint8), len(B),
                           match, mismatch, gap, ctypes.byref(score),
                           _ptr(ops, ctypes.c_uint8), ctypes.byref(L))
    if rc != 0:
        raise MemoryError("oracle_nw: matrix allocation failed")
    return int(score.value), bytes(ops[: L.value])


def nw_affine(a, b, match: int = 0, mismatch: int = 1, gap_open: int = 10, gap_ext: int = 1, sub=None):
    """Needleman-Wunsch with affine gap costs (the paper's merges use affine
    gaps, open = 10 x extend; section "Implementation"): a run of L gap
    positions costs ``gap_open + L * gap_ext``.  Gotoh's three matrices and
    the traceback of ``oracle.c`` (diagonal, then up, then left; a gap run
    closes where opening it attains, else it extends), which with
    ``gap_open = 0`` is :func:`nw`'s traceback.  With ``sub`` (a 256 x 256
    integer array over byte values) a substitution costs ``sub[a_i, b_j]``
    instead of match / mismatch (``M`` / ``X`` still label identity).
    Returns ``(score, ops)``.
    """
    A, B = _as_u8(a), _as_u8(b)
    ops = np.zeros(len(A) + len(B) + 1, dtype=np.uint8)
    score = ctypes.c_int32(0)
    L = ctypes.c_int64(0)
    if sub is not None:
        T = np.ascontiguousarray(sub, dtype=np.int32)
        assert T.shape == (256, 256)
        rc = _load().oracle_nw_affine_sub(_ptr(A, ctypes.c_uint8), len(A), _ptr(B, ctypes.c_uint8), len(B),
                                          _ptr(T, ctypes.c_int32), gap_open, gap_ext, ctypes.byref(score),
                                          _ptr(ops, ctypes.c_uint8), ctypes.byref(L))
        if rc != 0:
            raise MemoryError("oracle_nw_affine_sub: allocation failed")
        return int(score.value), ops[:L.value].tobytes()
    rc = _load().oracle_nw_affine(_ptr(A, ctypes.c_uint8), len(A), _ptr(B, ctypes.c_uint8), len(B),
                                  match, mismatch, gap_open, gap_ext, ctypes.byref(score),
                                  _ptr(ops, ctypes.c_uint8), ctypes.byref(L))
    if rc != 0:
        raise MemoryError("oracle_nw_affine: allocation failed")
    return int(score.value), ops[:L.value].tobytes()


def rescore_affine(a, b, ops, match=0, mismatch=1, gap_open=10, gap_ext=1, sub=None):
    """Cost of an alignment under affine gaps: substitutions (match /
    mismatch, or ``sub[a_i, b_j]``) plus, for every maximal run of D (or of
    I) of length L, gap_open + L * gap_ext."""
    a, b = bytes(a), bytes(b)
    i = j = 0
    cost = 0
    prev = None
    for op in bytes(ops):
        if op in (ord("M"), ord("X")):
            cost += int(sub[a[i], b[j]]) if sub is not None else (match if a[i] == b[j] else mismatch)
            i += 1
            j += 1
        elif op == ord("D"):
            cost += gap_ext + (gap_open if prev != op else 0)
            i += 1
        else:
            cost += gap_ext + (gap_open if prev != op else 0)
            j += 1
        prev = op
    assert i == len(a) and j == len(b)
    return cost


def lev_pairs(arena: np.ndarray, offs: np.ndarray, pairs: np.ndarray, nthreads: int | None = None) -> np.ndarray:
    """``f`` over a pair list ``pairs[P, 2]`` of indices into the sequence arena."""
    arena = np.ascontiguousarray(arena, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(pairs), dtype=np.int32)
    if len(pairs) == 0:
        return out
    rc = _load().oracle_lev_pairs(_ptr(arena, ctypes.c_uint8), _ptr(offs, ctypes.c_int64),
                                  _ptr(pairs, ctypes.c_int32), len(pairs),
                                  _ptr(out, ctypes.c_int32), nthreads or cpu_threads())
    if rc != 0:
        raise MemoryError("oracle_lev_pairs: allocation failed")
    return out


def nw_pairs(arena, offs, pairs, match=0, mismatch=1, gap=1, nthreads=None):
    """NW over a pair list. Returns ``(score[P], ops_bytes, ops_off[P+1], ops_len[P])``."""
    arena = np.ascontiguousarray(arena, dtype=np.uint8)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    lens = np.diff(offs)
    cap = lens[pairs[:, 0]] + lens[pairs[:, 1]] if len(pairs) else np.zeros(0, np.int64)
    ops_off = np.zeros(len(pairs) + 1, dtype=np.int64)
    np.cumsum(cap, out=ops_off[1:])
    ops = np.zeros(max(int(ops_off[-1]), 1), dtype=np.uint8)
    score = np.zeros(len(pairs), dtype=np.int32)
    ops_len = np.zeros(len(pairs), dtype=np.int64)
    if len(pairs):
        rc = _load().oracle_nw_pairs(_ptr(arena, ctypes.c_uint8), _ptr(offs, ctypes.c_int64),
                                     _ptr(pairs, ctypes.c_int32), len(pairs), match, mismatch, gap,
                                     _ptr(score, ctypes.c_int32), _ptr(ops, ctypes.c_uint8),
                                     _ptr(ops_off, ctypes.c_int64), _ptr(ops_len, ctypes.c_int64),
                                     nthreads or cpu_threads())
        if rc != 0:
            raise MemoryError("oracle_nw_pairs: allocation failed")
    return score, ops, ops_off, ops_len


def rescore(a, b, ops, match=0, mismatch=1, gap=1):
    """Cost of an edit script, and the two gapped rows it spells.

    Raises ``ValueError`` if the script does not consume exactly ``a`` and ``b``.
    """
    a, b = bytes(a), bytes(b)
    i = j = 0
    cost = 0
    ra, rb = bytearray(), bytearray()
    for o in bytes(ops):
        if o in (ord("M"), ord("X")):
            if i >= len(a) or j >= len(b):
                raise ValueError("script overruns the sequences")
            eq = a[i] == b[j]
            if (o == ord("M")) != eq:
                raise ValueError("M/X label disagrees with the symbols")
            cost += match if eq else mismatch
            ra.append(a[i]); rb.append(b[j]); i += 1; j += 1
        elif o == ord("D"):
            if i >= len(a):
                raise ValueError("script overruns a")
            cost += gap
            ra.append(a[i]); rb.append(ord("-")); i += 1
        elif o == ord("I"):
            if j >= len(b):
                raise ValueError("script overruns b")
            cost += gap
            ra.append(ord("-")); rb.append(b[j]); j += 1
        else:
            raise ValueError(f"unknown op {o!r}")
    if i != len(a) or j != len(b):
        raise ValueError("script does not consume both sequences")
    return cost, bytes(ra), bytes(rb)


# ---------------------------------------------------------------------------
# Brute force over all alignments (pure Python, tiny inputs only)
# ---------------------------------------------------------------------------

def brute_alignments(a, b):
    """Yield every alignment of ``a`` and ``b`` as an op string over M/X/D/I.

    The number of alignments is the Delannoy number D(m, n); keep m, n <= 6.
    """
    a, b = bytes(a), bytes(b)
    out = []

    def rec(i, j, acc):
        if i == len(a) and j == len(b):
            out.append(bytes(acc))
            return
        if i < len(a) and j < len(b):
            acc.append(ord("M") if a[i] == b[j] else ord("X"))
            rec(i + 1, j + 1, acc)
            acc.pop()
        if i < len(a):
            acc.append(ord("D"))
            rec(i + 1, j, acc)
            acc.pop()
        if j < len(b):
            acc.append(ord("I"))
            rec(i, j + 1, acc)
            acc.pop()

    rec(0, 0, bytearray())
    return out


def brute_best(a, b, match=0, mismatch=1, gap=1):
    """Minimum cost over all alignments, and the optimal alignment whose
    reversed op string is least under diagonal < up < left.

    The greedy traceback that prefers diagonal, then up, then left, walking
    back from (m, n), picks exactly that alignment: every move that attains
    D[i][j] can be completed into an optimal alignment.
    """
    rank = {ord("M"): 0, ord("X"): 0, ord("D"): 1, ord("I"): 2}
    best = None
    best_key = None
    for ops in brute_alignments(a, b):
        c, _, _ = rescore(a, b, ops, match, mismatch, gap)
        key = (c, [rank[o] for o in reversed(ops)])
        if best_key is None or key < best_key:
            best_key, best = key, ops
    return best_key[0], best


# ---------------------------------------------------------------------------
# Learned band proposer: features and network (float64 on bf16 operands)
# ---------------------------------------------------------------------------

DNA = b"ACGT"


def kmer_counts(seq, k: int = 4) -> np.ndarray:
    """Counts of every DNA k-mer (4**k bins) over the len-k+1 windows of ``seq``.

    The k-mer with symbols s_0..s_{k-1} (A=0, C=1, G=2, T=3) has bin
    sum_t s_t * 4**(k-1-t).  Windows containing another byte are skipped.
    """
    seq = bytes(seq)
    idx = {c: v for v, c in enumerate(DNA)}
    out = np.zeros(4 ** k, dtype=np.int64)
    for s in range(len(seq) - k + 1):
        v = 0
        ok = True
        for t in range(k):
            c = idx.get(seq[s + t])
            if c is None:
                ok = False
                break
            v = v * 4 + c
        if ok:
            out[v] += 1
    return out


def pair_feature(ca: np.ndarray, cb: np.ndarray, la: int, lb: int) -> np.ndarray:
    """Pair feature (c_a - c_b)^2 / ((len_a + len_b) / 2), rounded to bf16 (as float64).

    The square and the division are taken in float32, the precision of the
    GPU feature kernel, and the result rounded to bf16.  It is this project's
    definition (the paper has no learned component), pinned by closed forms
    in the tests.
    """
    diff = np.abs(ca.astype(np.int64) - cb.astype(np.int64)).astype(np.float32)
    den = np.float32((la + lb) * 0.5)
    if den == 0:
        den = np.float32(1.0)
    return bf16_round((diff * diff) / den)


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bf16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(x) -> np.ndarray:
    """bf16 bit patterns (uint16) of ``x`` after :func:`bf16_round`."""
    r = bf16_round(x).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def mlp_forward(params: dict, X: np.ndarray):
    """Forward pass y = W3 relu(W2 relu(W1 x + b1) + b2) + b3.

    ``params`` holds float64 arrays W1[256,128], b1[128], W2[128,64], b2[64],
    W3[64,1], b3[1]; the weights and ``X`` are rounded to bf16 first, the
    hidden activations are rounded to bf16 after ReLU, biases are used as
    given; all arithmetic is float64.  Returns ``(y, cache)``.
    """
    W1, W2, W3 = (bf16_round(params[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(params[k], dtype=np.float64) for k in ("b1", "b2", "b3"))
    X = bf16_round(X)
    z1 = X @ W1 + b1
    h1 = bf16_round(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + b2
    h2 = bf16_round(np.maximum(z2, 0.0))
    y = (h2 @ W3)[:, 0] + b3[0]
    cache = dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, W3=W3)
    return y, cache


def pinball_loss(yhat: np.ndarray, y: np.ndarray, tau: float = 0.9):
    """Mean quantile (pinball) loss and its derivative with respect to yhat.

    rho(r) = tau * r for r = y - yhat > 0, (tau - 1) * r otherwise; the
    derivative at r <= 0 is taken as (1 - tau) / B.
    """
    r = y - yhat
    B = len(y)
    loss = np.mean(np.where(r > 0, tau * r, (tau - 1.0) * r))
    dy = np.where(r > 0, -tau, 1.0 - tau) / B
    return float(loss), dy


def mlp_backward(cache: dict, dy: np.ndarray) -> dict:
    """Gradients of the loss with respect to every parameter, given dL/dy."""
    X, z1, h1, z2, h2 = (cache[k] for k in ("X", "z1", "h1", "z2", "h2"))
    W2, W3 = cache["W2"], cache["W3"]
    dy = dy.reshape(-1, 1)
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = dy.sum(axis=0)
    dh2 = (dy @ W3.T) * (z2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (z1 > 0)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return g


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) on float64 master copies."""
    out = {}
    for k in params:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        out[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return out, m, v


# Band policy and its calibration.  The band proposer turns the network's
# output into a Ukkonen band; these functions are this project's definition
# of that step, pinned in the tests by numpy's inverted-CDF quantile, the
# exact reduction of identity knots to the plain policy, the map's values at
# and halfway between knots, monotonicity and hand-worked bands.

CAL_KNOTS = 33          # knots at yhat = 0, 1/32, ..., 1
CAL_MIN_PAIRS = 16      # a bin with fewer held-out pairs keeps the identity


def band_calibrate(yhat, y, tau: float = 0.95) -> np.ndarray:
    """Knots of the monotone map c(yhat): knot i is the tau-quantile (the
    smallest value v with #{y <= v} >= ceil(tau * n), the inverted-CDF
    quantile) of the true y = f / max(m, n), clamped to [0, 1], over the
    held-out pairs whose yhat rounds to i / 32; a bin with fewer than
    CAL_MIN_PAIRS pairs keeps the identity i / 32; then a running maximum
    makes the map non-decreasing.  All in float32 as the kernel does."""
    yh = np.asarray(yhat, np.float32)
    yv = np.fmin(np.fmax(np.asarray(y, np.float32), np.float32(0)), np.float32(1))
    x = np.fmin(np.fmax(yh * np.float32(32) + np.float32(0.5), np.float32(0)), np.float32(32))
    b = x.astype(np.int64)
    knots = np.empty(CAL_KNOTS, np.float32)
    for i in range(CAL_KNOTS):
        v = np.sort(yv[b == i])
        if len(v) < CAL_MIN_PAIRS:
            knots[i] = np.float32(i) / np.float32(32)
        else:
            r = int(np.ceil(np.float64(np.float32(tau)) * len(v)))
            knots[i] = v[min(max(r, 1), len(v)) - 1]
    return np.maximum.accumulate(knots).astype(np.float32)


def band_calibrated(knots: np.ndarray, yhat) -> np.ndarray:
    """c(yhat): linear interpolation of the knots at clamp(yhat, 0, 1) * 32,
    every operation rounded to float32."""
    yh = np.fmin(np.fmax(np.asarray(yhat, np.float32), np.float32(0)), np.float32(1))
    x = (yh * np.float32(32)).astype(np.float32)
    i = np.minimum(x.astype(np.int64), CAL_KNOTS - 2)
    f = (x - i.astype(np.float32)).astype(np.float32)
    k0, k1 = knots[i], knots[i + 1]
    return (k0 + (f * (k1 - k0)).astype(np.float32)).astype(np.float32)


def band_policy(yhat, la, lb, gamma: float, margin: int, knots=None) -> np.ndarray:
    """Starting band k = max(|m - n|, ceil((1 + gamma) * c * max(m, n)) +
    margin) with c = max(yhat, 0), or c(yhat) of the calibration knots; the
    products in float32 left to right."""
    yh = np.asarray(yhat, np.float32)
    c = np.fmax(yh, np.float32(0)) if knots is None else band_calibrated(knots, yh)
    mx = np.maximum(la, lb).astype(np.float32)
    kf = np.ceil(((np.float32(1) + np.float32(gamma)) * c).astype(np.float32) * mx).astype(np.int64)
    return np.maximum(np.abs(np.asarray(la, np.int64) - lb), kf + margin)


# ---------------------------------------------------------------------------
# k-mer anchored splitting of long alignments (the paper's future work for
# length scaling, section "Discussion and Future Work"; the definition below is this
# project's, the paper gives none)
# ---------------------------------------------------------------------------

def kmer_anchors(a, b, k):
    """Anchors of a pair: every (i, j) where the k-mer a[i:i+k] occurs
    exactly once in a, exactly once in b, and b[j:j+k] is that k-mer; sorted
    by i."""
    a, b = bytes(a), bytes(b)
    ca, cb, pa, pb = {}, {}, {}, {}
    for i in range(len(a) - k + 1):
        w = a[i:i + k]
        ca[w] = ca.get(w, 0) + 1
        pa[w] = i
    for j in range(len(b) - k + 1):
        w = b[j:j + k]
        cb[w] = cb.get(w, 0) + 1
        pb[w] = j
    return sorted((pa[w], pb[w]) for w in ca if ca[w] == 1 and cb.get(w, 0) == 1)


def anchor_chain(anchors):
    """The longest chain of anchors increasing in both i and j, by patience
    sorting over the anchors in i order: each anchor replaces the first
    chain tail whose j is >= its own (binary search) and links to the tail
    before it; the chain is read back from the last tail."""
    tails, tail_idx, prev = [], [], [-1] * len(anchors)
    for t, (_, j) in enumerate(anchors):
        lo, hi = 0, len(tails)
        while lo < hi:
            mid = (lo + hi) // 2
            if tails[mid] < j:
                lo = mid + 1
            else:
                hi = mid
        if lo == len(tails):
            tails.append(j)
            tail_idx.append(t)
        else:
            tails[lo] = j
            tail_idx[lo] = t
        prev[t] = tail_idx[lo - 1] if lo > 0 else -1
    chain = []
    t = tail_idx[-1] if tail_idx else -1
    while t >= 0:
        chain.append(anchors[t])
        t = prev[t]
    return chain[::-1]


def anchor_blocks(chain, k):
    """Matched blocks from a chain, left to right: an anchor on the current
    block's diagonal that starts inside or right after it extends the block
    to its own end; an anchor that starts at or after the block's end in both
    sequences starts a new block; any other anchor is dropped.  Returns
    (start_a, start_b, length) per block."""
    blocks = []
    for i, j in chain:
        if blocks:
            sa, sb, ln = blocks[-1]
            if j - i == sb - sa and i <= sa + ln:
                blocks[-1] = (sa, sb, max(ln, i + k - sa))
                continue
            if i < sa + ln or j < sb + ln:
                continue
        blocks.append((i, j, k))
    return blocks


def nw_anchored(a, b, k=12, match=0, mismatch=1, gap=1, gap_open=None, sub=None):
    """Needleman-Wunsch split at k-mer anchors: the blocks of
    :func:`anchor_blocks` (over :func:`anchor_chain` of
    :func:`kmer_anchors`) are aligned as runs of matches, the segments
    between them (and before the first, after the last) by :func:`nw`, or,
    with ``gap_open``, by :func:`nw_affine` with gap extension ``gap`` (and
    ``sub``, a 256 x 256 cost table over byte values, when given).  A block
    residue costs ``match``, or ``sub[x, x]`` with a table.  Returns
    ``(score, ops)``; the score is an upper bound of the optimal cost, equal
    to it whenever an optimal alignment passes through every block.  Without
    anchors this is the plain alignment."""
    a, b = bytes(a), bytes(b)
    blocks = anchor_blocks(anchor_chain(kmer_anchors(a, b, k)), k)
    score, ops = 0, bytearray()
    ia = ib = 0
    for sa, sb, ln in blocks + [(len(a), len(b), 0)]:
        if gap_open is None:
            sc, op = nw(a[ia:sa], b[ib:sb], match, mismatch, gap)
        else:
            sc, op = nw_affine(a[ia:sa], b[ib:sb], match, mismatch, gap_open, gap, sub)
        block = a[sa:sa + ln]
        score += sc + (sum(int(sub[x, x]) for x in block) if sub is not None else ln * match)
        ops += op + b"M" * ln
        ia, ib = sa + ln, sb + ln
    return score, bytes(ops)


# ---------------------------------------------------------------------------
# BLOSUM62 costs for protein merges
# ---------------------------------------------------------------------------

def blosum62_scores() -> dict:
    """BLOSUM62 (Henikoff & Henikoff 1992) as {(x, y): score} over the 20
    residue letters, read from ``blosum62.txt``."""
    rows = [ln.split() for ln in open(os.path.join(_HERE, "blosum62.txt")) if ln.strip() and not ln.startswith("#")]
    cols = rows[0]
    return {(r[0], c): int(v) for r in rows[1:] for c, v in zip(cols, r[1:])}


def blosum62_costs(gap: int = ord("-")) -> np.ndarray:
    """256 x 256 cost table over byte values for minimising NW: cost = -score
    for two residues; the gap symbol of a gapped centre row is read as
    BLOSUM62's stop row '*' (score -4 against any residue, 1 against itself,
    so cost 4 and -1); other bytes cost 0 (never used)."""
    T = np.zeros((256, 256), np.int32)
    for (x, y), v in blosum62_scores().items():
        T[ord(x), ord(y)] = -v
    for x in "ARNDCQEGHILKMFPSTWYV":
        T[ord(x), gap] = T[gap, ord(x)] = 4
    T[gap, gap] = -1
    return T


# ---------------------------------------------------------------------------
# Alg. 1 Partition and the post-order merge
# ---------------------------------------------------------------------------

MEDOID_SAMPLE = 256


def medoid_candidates(members):
    """Members over which the geometric median is taken (section "Clustering").

    All of C when |C| <= 256, else the 256 members at positions
    floor(k |C| / 256), k = 0..255, of C sorted by global index (the paper
    allows "a smaller subset" without fixing it; this is the reading taken).
    """
    members = sorted(members)
    if len(members) <= MEDOID_SAMPLE:
        return members
    n = len(members)
    return [members[(k * n) // MEDOID_SAMPLE] for k in range(MEDOID_SAMPLE)]


def _default_dist(seqs):
    cache = {}

    def dist(x, y):
        key = (x, y) if x < y else (y, x)
        if key not in cache:
            cache[key] = lev(seqs[key[0]], seqs[key[1]])
        return cache[key]
    return dist


def partition_step(members, dist):
    """One application of Alg. 1 to the cluster ``members`` (|C| > 1).

    Returns ``(c, l, r, L, R)``: the centre (geometric median over
    :func:`medoid_candidates`), the two poles and the two children (sorted).
    """
    C = sorted(members)
    S = medoid_candidates(C)
    sums = [(sum(dist(x, y) for y in S), x) for x in S]
    c = min(sums)[1]
    l = min((-dist(c, x), x) for x in C)[1]
    r = min((-dist(l, x), x) for x in C)[1]
    Lm = [x for x in C if dist(l, x) <= dist(r, x)]
    Rm = [x for x in C if dist(r, x) < dist(l, x)]
    return c, l, r, Lm, Rm


def partition(seqs, dist=None):
    """Alg. 1 ``Partition`` applied from the root until every leaf is a singleton.

    ``seqs`` is a list of distinct byte strings.  Returns the tree as a list of
    nodes in breadth-first order; node k is a dict with ``members`` (sorted
    global indices), ``center``, ``left``, ``right`` (node ids or -1) and
    ``parent``.  Ties: the geometric median and both poles take the smallest
    global index among equal values; ``f(l, x) == f(r, x)`` goes to L exactly
    as Alg. 1 states.
    """
    if dist is None:
        dist = _default_dist(seqs)
    nodes = [dict(members=sorted(range(len(seqs))), center=-1, left=-1, right=-1, parent=-1)]
    q = 0
    while q < len(nodes):
        node = nodes[q]
        C = node["members"]
        if len(C) == 1:
            node["center"] = C[0]
        else:
            c, l, r, Lm, Rm = partition_step(C, dist)
            node["center"] = c
            assert Lm and Rm, "de-duplicated input guarantees both children are non-empty"
            for side, mem in (("left", Lm), ("right", Rm)):
                node[side] = len(nodes)
                nodes.append(dict(members=mem, center=-1, left=-1, right=-1, parent=q))
        q += 1
    return nodes


def merge_tree(seqs, nodes, match=0, mismatch=1, gap=1, gap_open=None, sub=None):
    """Post-order merge of section "Merging" over the tree from :func:`partition`.

    With ``gap_open`` the centers are aligned by :func:`nw_affine` (a run of L
    gaps costs ``gap_open + L * gap``) instead of :func:`nw`, and with ``sub``
    too, substitutions cost ``sub[x, y]`` (e.g. :func:`blosum62_costs`).

    A leaf is the one-row MSA of its sequence.  At an internal node the two
    children's centers, as gapped rows of the children's MSAs, are aligned by
    :func:`nw` with ``-`` an ordinary symbol; every ``I`` op inserts an all-gap
    column into the left child's rows, every ``D`` op into the right child's;
    the parent's rows are the left child's rows followed by the right
    child's.  Returns ``(rows, order, merges)``: the root MSA rows (bytes), the
    sequence index of each row, and per internal node the NW ``(score, ops)``.
    """
    msa = {}
    merges = {}

    def center_row(k):
        rows, order = msa[k]
        return rows[order.index(nodes[k]["center"])]

    # children come after parents in BFS order, so reverse order is a valid post-order
    for k in range(len(nodes) - 1, -1, -1):
        nd = nodes[k]
        if nd["left"] < 0:
            s = nd["members"][0]
            msa[k] = ([bytes(seqs[s])], [s])
            continue
        L, R = nd["left"], nd["right"]
        if gap_open is None:
            score, ops = nw(center_row(L), center_row(R), match, mismatch, gap)
        else:
            score, ops = nw_affine(center_row(L), center_row(R), match, mismatch, gap_open, gap, sub=sub)
        merges[k] = (score, ops)
        rowsL, ordL = msa.pop(L)
        rowsR, ordR = msa.pop(R)
        newL = [bytearray() for _ in rowsL]
        newR = [bytearray() for _ in rowsR]
        i = j = 0
        for o in ops:
            if o in (ord("M"), ord("X"), ord("D")):
                for t, r in enumerate(rowsL):
                    newL[t].append(r[i])
                i += 1
            else:
                for t in range(len(rowsL)):
                    newL[t].append(ord("-"))
            if o in (ord("M"), ord("X"), ord("I")):
                for t, r in enumerate(rowsR):
                    newR[t].append(r[j])
                j += 1
            else:
                for t in range(len(rowsR)):
                    newR[t].append(ord("-"))
        msa[k] = ([bytes(r) for r in newL] + [bytes(r) for r in newR], ordL + ordR)
    rows, order = msa[0]
    return rows, order, merges


def _arena_of(seqs):
    lens = np.array([len(x) for x in seqs], np.int64)
    offs = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    arena = np.frombuffer(b"".join(bytes(x) for x in seqs) + b"\0", np.uint8).copy()
    return arena, offs


def partition_levels(seqs, nthreads=None, max_levels=None):
    """The tree of :func:`partition`, with the distances of all clusters of
    one tree level computed together.

    Alg. 1 is applied to every cluster exactly as :func:`partition_step`
    does (same medoid candidates, sums, poles, split and tie rules), and the
    nodes are numbered in the same breadth-first order; only the Levenshtein
    distances of each step are gathered over the clusters of a level and
    handed to :func:`lev_pairs` as one batch (clusters of one level are
    disjoint, so no step waits on another cluster's).  Used where the plain
    per-pair version would take hours (10,000 sequences); tests pin it to
    :func:`partition` on small sets.  With ``max_levels`` only that many
    levels are split (``max_levels=1``: one application of Alg. 1 to the
    whole set, the batched form of :func:`partition_step`).
    """
    arena, offs = _arena_of(seqs)

    def batch(pairs):
        if not pairs:
            return np.zeros(0, np.int32)
        return lev_pairs(arena, offs, np.array(pairs, np.int32), nthreads)

    nodes = [dict(members=sorted(range(len(seqs))), center=-1, left=-1, right=-1, parent=-1)]
    level = [0]
    depth = 0
    while level and (max_levels is None or depth < max_levels):
        depth += 1
        work = []
        for q in level:
            C = nodes[q]["members"]
            if len(C) == 1:
                nodes[q]["center"] = C[0]
            else:
                work.append(q)
        # geometric median over the candidates: sums of f over all pairs of S
        med_pairs, spans = [], []
        for q in work:
            S = medoid_candidates(nodes[q]["members"])
            start = len(med_pairs)
            med_pairs += [(S[i], S[j]) for i in range(len(S)) for j in range(i + 1, len(S))]
            spans.append((S, start))
        dm = batch(med_pairs)
        center = {}
        for q, (S, start) in zip(work, spans):
            sums = {x: 0 for x in S}
            for t, (x, y) in enumerate(med_pairs[start:start + len(S) * (len(S) - 1) // 2]):
                sums[x] += int(dm[start + t])
                sums[y] += int(dm[start + t])
            center[q] = min((sums[x], x) for x in S)[1]

        def far(frm):
            pairs = [(frm[q], x) for q in work for x in nodes[q]["members"]]
            d = batch(pairs)
            out, o = {}, 0
            for q in work:
                C = nodes[q]["members"]
                out[q] = d[o:o + len(C)]
                o += len(C)
            return out

        dc = far(center)
        pole_l = {q: min((-int(dc[q][i]), x) for i, x in enumerate(nodes[q]["members"]))[1] for q in work}
        dl = far(pole_l)
        pole_r = {q: min((-int(dl[q][i]), x) for i, x in enumerate(nodes[q]["members"]))[1] for q in work}
        dr = far(pole_r)
        nxt = []
        for q in level:
            node = nodes[q]
            if q not in center:
                continue
            node["center"] = center[q]
            C = node["members"]
            Lm = [x for i, x in enumerate(C) if dl[q][i] <= dr[q][i]]
            Rm = [x for i, x in enumerate(C) if dr[q][i] < dl[q][i]]
            assert Lm and Rm, "de-duplicated input guarantees both children are non-empty"
            for side, mem in (("left", Lm), ("right", Rm)):
                node[side] = len(nodes)
                nxt.append(len(nodes))
                nodes.append(dict(members=mem, center=-1, left=-1, right=-1, parent=q))
        level = nxt
    return nodes


def merge_tree_levels(seqs, nodes, match=0, mismatch=1, gap=1, nthreads=None):
    """The merge of :func:`merge_tree`, with the center alignments of all
    nodes of one height computed as one :func:`nw_pairs` batch and the MSAs
    held as 2-D byte arrays.

    A node's height is 1 + the larger of its children's (leaves 0); merges of
    one height touch disjoint subtrees whose children are all finished, so
    the result is the post-order result.  Each merge is the step of section
    "Merging" as :func:`merge_tree` takes it: align the children's center
    rows (``-`` an ordinary symbol), put an all-gap column into the left
    rows for every ``I`` and into the right rows for every ``D``, left rows
    over right rows.  Returns ``(rows, order, merges)`` like
    :func:`merge_tree`.  Tests pin it to :func:`merge_tree` on small sets.
    """
    gapb = ord("-")
    height = [0] * len(nodes)
    for k in range(len(nodes) - 1, -1, -1):
        if nodes[k]["left"] >= 0:
            height[k] = 1 + max(height[nodes[k]["left"]], height[nodes[k]["right"]])
    msa = {}
    for k, nd in enumerate(nodes):
        if nd["left"] < 0:
            s = nd["members"][0]
            msa[k] = (np.frombuffer(bytes(seqs[s]), np.uint8).reshape(1, -1).copy(), [s])
    merges = {}
    for h in range(1, max(height) + 1 if nodes else 1):
        ks = [k for k in range(len(nodes)) if height[k] == h]
        rows = []
        for k in ks:
            for child in (nodes[k]["left"], nodes[k]["right"]):
                block, order = msa[child]
                rows.append(block[order.index(nodes[child]["center"])].tobytes())
        arena, offs = _arena_of(rows)
        pairs = np.arange(2 * len(ks), dtype=np.int32).reshape(-1, 2)
        score, ops, ops_off, ops_len = nw_pairs(arena, offs, pairs, match, mismatch, gap, nthreads)
        for t, k in enumerate(ks):
            op = ops[ops_off[t]:ops_off[t] + ops_len[t]]
            merges[k] = (int(score[t]), op.tobytes())
            bl, ol = msa.pop(nodes[k]["left"])
            br, orr = msa.pop(nodes[k]["right"])
            take_l = np.isin(op, (ord("M"), ord("X"), ord("D")))
            take_r = np.isin(op, (ord("M"), ord("X"), ord("I")))
            newl = np.full((bl.shape[0], len(op)), gapb, np.uint8)
            newr = np.full((br.shape[0], len(op)), gapb, np.uint8)
            newl[:, take_l] = bl
            newr[:, take_r] = br
            msa[k] = (np.concatenate([newl, newr]), ol + orr)
    rows, order = msa[0]
    return [r.tobytes() for r in rows], order, merges


# ---------------------------------------------------------------------------
# alignment quality (section "Evaluation")
# ---------------------------------------------------------------------------

def msa_metrics(rows, seqs, gap: int = ord("-")):
    """The three metrics of section "Evaluation" over aligned ``rows`` (equal
    length byte strings) whose unaligned sequences are ``seqs``:

    * percentage of gaps: per row, gap bytes / row length, averaged over the
      rows, x 100;
    * p-score: over every unordered pair of rows and every column where
      neither row has a gap, the share of columns whose bytes differ, x 100
      (one ratio over all such pairs of units);
    * distance distortion: over every unordered pair of rows, the Hamming
      distance of the aligned rows (columns whose bytes differ; a gap-gap
      column is equal) divided by the Levenshtein distance of the unaligned
      sequences, averaged over the pairs (pairs of identical sequences, whose
      ratio is undefined, are left out; the paper's inputs are de-duplicated).

    Returns ``(pct_gaps, p_score, distortion, counts)`` with the integer
    totals behind them.  Plain loops over pairs and columns.
    """
    R = len(rows)
    W = len(rows[0]) if R else 0
    M = np.frombuffer(b"".join(bytes(r) for r in rows), np.uint8).reshape(R, W) if R else np.zeros((0, 0), np.uint8)
    gaps = int((M == gap).sum())
    pct = 100.0 * float(np.mean((M == gap).sum(1) / W)) if R and W else 0.0
    compared = mismatched = 0
    ratio_sum = 0.0
    pairs = 0
    for i in range(R):
        for j in range(i + 1, R):
            a, b = M[i], M[j]
            both = (a != gap) & (b != gap)
            compared += int(both.sum())
            mismatched += int((both & (a != b)).sum())
            h = int((a != b).sum())
            f = lev(seqs[i], seqs[j])
            if f == 0:               # identical sequences have no ratio: left out
                continue
            ratio_sum += h / f
            pairs += 1
    p = 100.0 * mismatched / compared if compared else 0.0
    dist = ratio_sum / pairs if pairs else 0.0
    return pct, p, dist, dict(gaps=gaps, compared=compared, mismatched=mismatched, pairs=pairs)
