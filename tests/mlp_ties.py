"""Rounding-choice enumeration for comparing the band network's forward
pass with the float64 oracle.

The kernel sums 256 (or 128) exact bf16 products in fp32 on the tensor
cores, the oracle in float64.  The two sums differ by far less than
`window` (a few fp32 rounding steps of the summed magnitudes); a hidden
value within that distance of a bf16 rounding boundary may therefore be
rounded to either neighbour, and both outputs are correct results of the
same arithmetic.  forward_candidates() lists the oracle outputs of a row
for every such choice."""
import numpy as np

import oracle

WINDOW = 1e-6          # relative to the sum of |products| + |bias|; fp32 sums of 256 exact products stay within ~1e-7


def _bf16_pair(a):
    """The two bf16 values around each (float32-rounded) non-negative value."""
    u = np.asarray(a, np.float64).astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    lo = u.view(np.float32).astype(np.float64)
    hi = (u + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    return lo, hi


def _near_ties(pre, bound):
    """Units whose ReLU output lies within `bound` of a bf16 rounding boundary."""
    a = np.maximum(pre, 0.0)
    lo, hi = _bf16_pair(a)
    return np.nonzero((a > 0) & (np.abs(a - 0.5 * (lo + hi)) <= bound))[0]


def _layer(z, bound, cap):
    """bf16(relu(z)) for every rounding choice of the near-tie units."""
    base = oracle.bf16_round(np.maximum(z, 0.0))
    ties = _near_ties(z, bound)[:cap]
    outs = []
    for c in range(1 << len(ties)):
        h = base.copy()
        for b, u in enumerate(ties):
            lo, hi = _bf16_pair(np.array([max(z[u], 0.0)]))
            h[u] = hi[0] if (c >> b) & 1 else lo[0]
        outs.append(h)
    return outs, len(ties)


def forward_candidates(op, x, window=WINDOW, cap=8):
    """Oracle outputs of one row for every rounding choice of its near-tie
    hidden units (the oracle's own choice among them), and the number of
    near-tie units met.  `op` holds float64 parameters in the oracle's
    layout (W1 [256, 128], ..., W3 [64, 1])."""
    W1, W2, W3 = (oracle.bf16_round(op[k]) for k in ("W1", "W2", "W3"))
    x = oracle.bf16_round(x)
    z1 = x @ W1 + op["b1"]
    h1s, t1 = _layer(z1, window * (np.abs(x) @ np.abs(W1) + np.abs(op["b1"])), cap)
    out, t2max = [], 0
    for h1 in h1s:
        z2 = h1 @ W2 + op["b2"]
        h2s, t2 = _layer(z2, window * (np.abs(h1) @ np.abs(W2) + np.abs(op["b2"])), cap)
        t2max = max(t2max, t2)
        out += [float(h2 @ W3[:, 0] + op["b3"][0]) for h2 in h2s]
    return out, t1 + t2max
