"""Rounding-choice enumeration for comparing the band network's forward
pass (fp32 sums on the GPU) with the float64 oracle: a hidden value that
lies, within the fp32 summation error, on a bf16 rounding boundary may be
rounded to either neighbour, and each choice gives a valid output."""
import numpy as np

import oracle


def _bf16_pair(a):
    """The two bf16 values around each (float32-rounded) positive value."""
    u = a.astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    lo = u.view(np.float32).astype(np.float64)
    hi = (u + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    return lo, hi


def _near_ties(pre, bound):
    """Units whose ReLU output lies within `bound` of a bf16 rounding
    boundary: there fp32 accumulation may round to either neighbour."""
    a = np.maximum(pre, 0.0)
    lo, hi = _bf16_pair(a)
    return np.nonzero((a > 0) & (np.abs(a - 0.5 * (lo + hi)) <= bound))[0]


def forward_candidates(op, x, cap=4):
    """Oracle outputs of one row for every rounding choice of its near-tie
    hidden units (the oracle's own choice included)."""
    W1, W2, W3 = (oracle.bf16_round(op[k]) for k in ("W1", "W2", "W3"))
    x = oracle.bf16_round(x)
    z1 = x @ W1 + op["b1"]
    # fp32 sums of 256 exact bf16 products: error far below 1e-4 of the sum of magnitudes
    t1 = _near_ties(z1, 1e-4 * (np.abs(x) @ np.abs(W1) + np.abs(op["b1"])))[:cap]
    out = []
    for c1 in range(1 << len(t1)):
        h1 = oracle.bf16_round(np.maximum(z1, 0.0))
        for b, u in enumerate(t1):
            lo, hi = _bf16_pair(np.array([max(z1[u], 0.0)]))
            h1[u] = hi[0] if (c1 >> b) & 1 else lo[0]
        z2 = h1 @ W2 + op["b2"]
        t2 = _near_ties(z2, 1e-4 * (np.abs(h1) @ np.abs(W2) + np.abs(op["b2"])))[:cap]
        for c2 in range(1 << len(t2)):
            h2 = oracle.bf16_round(np.maximum(z2, 0.0))
            for b, u in enumerate(t2):
                lo, hi = _bf16_pair(np.array([max(z2[u], 0.0)]))
                h2[u] = hi[0] if (c2 >> b) & 1 else lo[0]
            out.append(float(h2 @ W3[:, 0] + op["b3"][0]))
    return out, len(t1) + len(t2)
