"""CPU model of the anchored NW's warp-batched chain passes (the device's
anchor_chain_kernel): windows of 32 positions or chain anchors taken in one
step when they follow the common case, anchor by anchor otherwise.  The
model must give the chain and blocks of the oracle's definitions
(anchor_chain, anchor_blocks) on random anchor sets: related pairs (long
increasing runs), crossing and repeated segments (the one-at-a-time
paths), and windows that break at every lane."""
import numpy as np

import oracle

W = 32


def _forward(aj):
    """Patience levels by windows: a window whose anchors all exceed the
    last tail and increase is appended at once."""
    m = len(aj)
    level = [-1] * m
    tails, last_j, last_i = [], -1, -1
    for w0 in range(0, m, W):
        win = list(range(w0, min(w0 + W, m)))
        js = [aj[i] for i in win]
        run, fast = last_j, True
        for j in js:
            if j < 0:
                continue
            if j <= run:
                fast = False
            run = max(run, j)
        if fast:
            for i in win:
                if aj[i] >= 0:
                    tails.append(aj[i])
                    level[i] = len(tails) - 1
                    last_j, last_i = aj[i], i
            continue
        for i in win:
            j = aj[i]
            if j < 0:
                continue
            lo = len(tails)
            if j < last_j:
                lo = next(t for t in range(len(tails)) if tails[t] >= j)
            if lo == len(tails):
                tails.append(j)
            else:
                tails[lo] = j
            level[i] = lo
            if lo == len(tails) - 1:
                last_j, last_i = j, i
    return level, len(tails), last_i


def _backward(aj, level, length, last_i):
    """The chain back to front by windows of 32 positions (highest first)."""
    chain, want = [], length - 1
    top = last_i
    while top >= 0 and want >= 0:
        lanes = [top - l for l in range(W) if top - l >= 0]
        anchors = [p for p in lanes if aj[p] >= 0]
        if anchors and all(level[p] == want - r for r, p in enumerate(anchors)):
            chain += [(p, aj[p]) for p in anchors]
            want -= len(anchors)
        else:
            cur = top + 1
            while want >= 0:
                hit = [p for p in lanes if p < cur and aj[p] >= 0 and level[p] == want]
                if not hit:
                    break
                p = hit[0]
                chain.append((p, aj[p]))
                want -= 1
                cur = p
        top -= W
    return chain[::-1]


def _blocks(chain, k):
    """Blocks by windows of 32 chain anchors: a run on the open block's
    diagonal, each inside or right after the block as extended, in one step;
    the anchor that ends the run alone."""
    blocks, b = [], None
    for w0 in range(0, len(chain), W):
        win = chain[w0:w0 + W]
        start = 0
        while start < len(win):
            f = len(win)
            for l in range(start, len(win)):
                i, j = win[l]
                if b is None:
                    f = l
                    break
                end_before = b[0] + b[2] if l == start else max(b[0] + b[2], win[l - 1][0] + k)
                if not (j - i == b[1] - b[0] and i <= end_before):
                    f = l
                    break
            if f > start:
                nl = max(b[2], win[f - 1][0] + k - b[0])
                b = (b[0], b[1], nl)
            if f >= len(win):
                break
            i, j = win[f]
            start = f + 1
            if b is not None:
                if i < b[0] + b[2] or j < b[1] + b[2]:
                    continue
                blocks.append(b)
            b = (i, j, k)
    if b is not None:
        blocks.append(b)
    return blocks


def _check(a, b, k):
    anchors = oracle.kmer_anchors(a, b, k)
    aj = [-1] * len(a)
    for i, j in anchors:
        aj[i] = j
    level, length, last_i = _forward(aj)
    chain = _backward(aj, level, length, last_i)
    assert chain == oracle.anchor_chain(anchors)
    assert _blocks(chain, k) == oracle.anchor_blocks(chain, k)


def _mutate(rng, a, rate):
    out = bytearray()
    for x in a:
        u = rng.random()
        if u < rate / 3:
            out.append(b"ACGT"[int(rng.integers(0, 4))])
        elif u < 2 * rate / 3:
            out += bytes([x, b"ACGT"[int(rng.integers(0, 4))]])
        elif u >= rate:
            out.append(x)
    return bytes(out)


def test_model_related_pairs():
    rng = np.random.default_rng(5)
    for L, rate in ((200, 0.0), (900, 0.02), (1500, 0.1), (700, 0.3)):
        a = bytes(rng.choice(list(b"ACGT"), size=L).astype(np.uint8))
        _check(a, _mutate(rng, a, rate), 8)


def test_model_crossing_and_repeats():
    rng = np.random.default_rng(6)
    parts = [bytes(rng.choice(list(b"ACGT"), size=300).astype(np.uint8)) for _ in range(4)]
    _check(parts[0] + parts[1] + parts[2], parts[2] + parts[1] + parts[0], 10)   # crossing blocks
    unit = bytes(rng.choice(list(b"ACGT"), size=40).astype(np.uint8))
    _check(parts[0] + unit * 5 + parts[1], _mutate(rng, parts[0], 0.05) + unit * 3 + parts[1], 12)
    for k in (4, 6):                                                             # short k: few anchors
        _check(parts[3], _mutate(rng, parts[3], 0.1), k)


def test_model_every_lane_breaks():
    """Anchors whose j alternates so no window is in order, and a chain of
    single-anchor blocks spaced so every window ends runs at every lane."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        a = bytes(rng.choice(list(b"ACGT"), size=int(rng.integers(50, 400))).astype(np.uint8))
        b = bytearray(a)
        for p in range(0, len(b), int(rng.integers(3, 15))):
            b[p] = b"ACGT"[(b"ACGT".index(b[p]) + 1) % 4]
        _check(a, bytes(b), int(rng.integers(2, 7)))
