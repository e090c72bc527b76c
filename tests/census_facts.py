"""Facts about the 16 triad classes, written from the class definitions (Holland-Leinhardt
M-A-N labels), used to pin census results by weighted sums.

Class order (0-based): 003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D 120U 120C
210 300.  Per class: mutual / asymmetric / null dyads, out-2-stars (a vertex with arcs to
both others), in-2-stars, directed 2-paths x->y->z with x != z, and whether all three
pairs are connected (an undirected triangle).
"""
import numpy as np

NAMES = ("003", "012", "102", "021D", "021U", "021C", "111D", "111U",
         "030T", "030C", "201", "120D", "120U", "120C", "210", "300")

#               003 012 102 21D 21U 21C 11D 11U 30T 30C 201 20D 20U 20C 210 300
M = np.array([0, 0, 1, 0, 0, 0, 1, 1, 0, 0, 2, 1, 1, 1, 2, 3], dtype=object)
A = np.array([0, 1, 0, 2, 2, 2, 1, 1, 3, 3, 0, 2, 2, 2, 1, 0], dtype=object)
N = np.array([3, 2, 2, 1, 1, 1, 1, 1, 0, 0, 1, 0, 0, 0, 0, 0], dtype=object)
OUT2 = np.array([0, 0, 0, 1, 0, 0, 0, 1, 1, 0, 1, 1, 2, 1, 2, 3], dtype=object)
IN2 = np.array([0, 0, 0, 0, 1, 0, 1, 0, 1, 0, 1, 2, 1, 1, 2, 3], dtype=object)
PATHS = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1, 3, 2, 2, 2, 3, 4, 6], dtype=object)
TRI = np.array([0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 0, 1, 1, 1, 1, 1], dtype=object)

# Reversing every arc swaps these classes and fixes the others.
REVERSE = {3: 4, 4: 3, 6: 7, 7: 6, 11: 12, 12: 11}
# Complementing the digraph (arc present iff absent) swaps these classes.
COMPLEMENT = {0: 15, 15: 0, 1: 14, 14: 1, 2: 10, 10: 2, 3: 12, 12: 3, 4: 11, 11: 4, 5: 13, 13: 5}

# Number of labelled 6-bit tricodes in each class: 3!/|Aut(class)|.
ORBIT = [1, 6, 3, 3, 3, 6, 6, 6, 6, 2, 3, 3, 3, 6, 6, 1]


def choose2(x):
    return x * (x - 1) // 2


def choose3(x):
    return x * (x - 1) * (x - 2) // 6 if x >= 3 else 0


def check_invariants(n, census, inv, triangles=True):
    """Assert every weighted-sum identity between a census and the O(m) statistics (the
    triangle identity only when the statistics counted triangles)."""
    c = np.array(census, dtype=object)
    assert sum(census) == choose3(n)
    assert int((c * M).sum()) == inv["M"] * (n - 2)
    assert int((c * A).sum()) == inv["A"] * (n - 2)
    assert int((c * N).sum()) == inv["N"] * (n - 2)
    assert int((c * OUT2).sum()) == inv["out2"]
    assert int((c * IN2).sum()) == inv["in2"]
    assert int((c * PATHS).sum()) == inv["paths"]
    if triangles:
        assert int((c * TRI).sum()) == inv["triangles"]


def permute_classes(census, mapping):
    out = list(census)
    for a, b in mapping.items():
        out[b] = census[a]
    return out
