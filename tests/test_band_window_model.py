"""The one-lane band window, as a CPU bit model, against the oracle.

The one-lane banded kernel keeps a window of W 32-row words that moves down
one word at 32-column boundaries (w0 = floor((j - dhi) / 32) for columns
j + 1 .. j + 32, with 32 W >= k + 63), carries the value T of the row above
the window with +1 per column, and starts every entering word at +1 per row.
This model runs those steps with Python integers as the bit vectors; the
certificate must hold for every band: the result is never below f, and it is
f whenever the band is at least f (so accepting d <= k is exact)."""
import random

import oracle

M32 = 0xFFFFFFFF


def _popc(x):
    return bin(x & M32).count("1")


def _column(eq, Pv, Mv):
    # one column over the window, row above +1 (Ph in = 1, carry in = 0)
    cy, php = 0, 1 << 31
    for w in range(len(Pv)):
        u = eq[w] & Pv[w]
        t = u + Pv[w] + cy
        s, cy = t & M32, t >> 32
        mhs = (s ^ u ^ Pv[w]) & M32
        ph = (Mv[w] | ~(s | Pv[w] | eq[w])) & M32
        phs = ((ph << 1) | (php >> 31)) & M32
        php = ph
        xv = eq[w] | Mv[w]
        Pv[w] = (mhs | ~(xv | phs)) & M32
        Mv[w] = phs & xv


def window_band(a, b, k):
    if len(a) < len(b):
        a, b = b, a
    m, n = len(a), len(b)
    if n == 0:
        return m
    k = min(max(k, m - n), m)
    dhi = (n - m + k) >> 1
    W = (k + 63 + 31) // 32

    def eq_word(word, c):
        return sum(1 << r for r in range(32) if 32 * word + r < m and a[32 * word + r] == c)

    Pv, Mv, w0, T = [M32] * W, [0] * W, 0, 0
    for j in range(1, n + 1):
        J = j - 1
        if J and J % 32 == 0:
            w0n = max(0, (J - dhi) // 32)
            assert w0n in (w0, w0 + 1)
            if w0n > w0:
                T += _popc(Pv[0]) - _popc(Mv[0])
                Pv, Mv, w0 = Pv[1:] + [M32], Mv[1:] + [0], w0n
        _column([eq_word(w0 + w, b[j - 1]) for w in range(W)], Pv, Mv)
        T += 1
    assert 32 * w0 < m <= 32 * (w0 + W)        # row m is inside the window at column n
    d = T
    for w in range(W):
        rem = m - 32 * (w0 + w)
        mk = M32 if rem >= 32 else (0 if rem <= 0 else (1 << rem) - 1)
        d += _popc(Pv[w] & mk) - _popc(Mv[w] & mk)
    return d


def _mutated(rng, L):
    a = bytes(rng.choice(b"ACGT") for _ in range(L))
    b = bytearray(a)
    for _ in range(rng.randint(0, L // 3 + 1)):
        p = rng.randrange(len(b) + 1)
        r = rng.random()
        if r < 0.5 and b:
            b[min(p, len(b) - 1)] = rng.choice(b"ACGT")
        elif r < 0.75:
            b.insert(p, rng.choice(b"ACGT"))
        elif b:
            del b[min(p, len(b) - 1)]
    return a, bytes(b)


def test_window_certificate_on_random_pairs():
    rng = random.Random(1)
    for _ in range(120):
        a, b = _mutated(rng, rng.randint(1, 200))
        if rng.random() < 0.3:
            a, b = b, a
        f = oracle.lev(a, b)
        lo = abs(len(a) - len(b))
        for k in sorted({0, max(0, f - 2), f, f + 5, 2 * f + 1, rng.randint(0, 150)}):
            d = window_band(a, b, k)
            assert d >= f
            if max(k, lo) >= f:
                assert d == f
