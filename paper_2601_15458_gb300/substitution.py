"""Substitution costs for the affine Needleman-Wunsch entry points.

The paper's protein merges score substitutions with BLOSUM62 (section
"Implementation"), a table it names but does not print.  The library
minimises a cost, so a score s becomes the cost -s.  The table below is
BLOSUM62 (Henikoff & Henikoff 1992, "Amino acid substitution matrices from
protein blocks", PNAS 89:10915) in the library's protein code order
(ACDEFGHIKLMNPQRSTVWY = codes 0..19); code 20 is the gap of a gapped centre
row, read as BLOSUM62's stop symbol '*' (score -4 against a residue, 1
against itself).
"""
from __future__ import annotations

PROTEIN_ORDER = "ACDEFGHIKLMNPQRSTVWY"

# scores, rows and columns in PROTEIN_ORDER
_BLOSUM62 = """
A  4  0 -2 -1 -2  0 -2 -1 -1 -1 -1 -2 -1 -1 -1  1  0  0 -3 -2
C  0  9 -3 -4 -2 -3 -3 -1 -3 -1 -1 -3 -3 -3 -3 -1 -1 -1 -2 -2
D -2 -3  6  2 -3 -1 -1 -3 -1 -4 -3  1 -1  0 -2  0 -1 -3 -4 -3
E -1 -4  2  5 -3 -2  0 -3  1 -3 -2  0 -1  2  0  0 -1 -2 -3 -2
F -2 -2 -3 -3  6 -3 -1  0 -3  0  0 -3 -4 -3 -3 -2 -2 -1  1  3
G  0 -3 -1 -2 -3  6 -2 -4 -2 -4 -3  0 -2 -2 -2  0 -2 -3 -2 -3
H -2 -3 -1  0 -1 -2  8 -3 -1 -3 -2  1 -2  0  0 -1 -2 -3 -2  2
I -1 -1 -3 -3  0 -4 -3  4 -3  2  1 -3 -3 -3 -3 -2 -1  3 -3 -1
K -1 -3 -1  1 -3 -2 -1 -3  5 -2 -1  0 -1  1  2  0 -1 -2 -3 -2
L -1 -1 -4 -3  0 -4 -3  2 -2  4  2 -3 -3 -2 -2 -2 -1  1 -2 -1
M -1 -1 -3 -2  0 -3 -2  1 -1  2  5 -2 -2  0 -1 -1 -1  1 -1 -1
N -2 -3  1  0 -3  0  1 -3  0 -3 -2  6 -2  0  0  1  0 -3 -4 -2
P -1 -3 -1 -1 -4 -2 -2 -3 -1 -3 -2 -2  7 -1 -2 -1 -1 -2 -4 -3
Q -1 -3  0  2 -3 -2  0 -3  1 -2  0  0 -1  5  1  0 -1 -2 -2 -1
R -1 -3 -2  0 -3 -2  0 -3  2 -2 -1  0 -2  1  5 -1 -1 -3 -3 -2
S  1 -1  0  0 -2  0 -1 -2  0 -2 -1  1 -1  0 -1  4  1 -2 -3 -2
T  0 -1 -1 -1 -2 -2 -2 -1 -1 -1 -1  0 -1 -1 -1  1  5  0 -2 -2
V  0 -1 -3 -2 -1 -3 -3  3 -2  1  1 -3 -2 -2 -3 -2  0  4 -3 -1
W -3 -2 -4 -3  1 -2 -2 -3 -3 -2 -1 -4 -4 -2 -3 -3 -2 -3 11  2
Y -2 -2 -3 -2  3 -3  2 -1 -2 -1 -1 -2 -3 -1 -2 -2 -2 -1  2  7
"""

GAP_VS_RESIDUE = 4     # -(score of '*' against a residue)
GAP_VS_GAP = -1        # -(score of '*' against itself)


def blosum62_costs_by_code() -> list:
    """21 x 21 costs (-score) over the protein codes 0..19 and the gap code 20."""
    rows = [ln.split() for ln in _BLOSUM62.strip().splitlines()]
    assert "".join(r[0] for r in rows) == PROTEIN_ORDER
    n = len(PROTEIN_ORDER)
    T = [[GAP_VS_RESIDUE] * (n + 1) for _ in range(n + 1)]
    for i, r in enumerate(rows):
        for j, v in enumerate(r[1:]):
            T[i][j] = -int(v)
    T[n][n] = GAP_VS_GAP
    return T
