"""The matrix form of the census (paper Sec. 4 names Moody's matrix census as the dense
alternative to the Fig. 5 method, without formulas): each of the 16 class counts as sums of
elementwise products of 0/1 dyad matrices with matrix products of them.  With A the arcs,
M = A o A^T the mutual dyads, S = A - M the one-way arcs (S[i,j] = 1 for i -> j only) and N the
null dyads (i != j, no arc either way):

  003 = sum(N o NN) / 6     012 = sum(S o NN)        102 = sum(M o NN) / 2
  021D = sum(N o S^T S) / 2 021U = sum(N o S S^T) / 2 021C = sum(N o SS)
  111D = sum(S o NM)        111U = sum(S^T o NM)      030T = sum(S o SS)
  030C = sum(S^T o SS) / 3  201 = sum(N o MM) / 2     120D = sum(M o S^T S) / 2
  120U = sum(M o S S^T) / 2 120C = sum(M o SS)        210 = sum(S o MM)
  300 = sum(M o MM) / 6

Each is a labelled count of the class's arc pattern divided by the pattern's symmetries.  This
CPU test pins the formula set, written here in plain numpy, to the oracle's census; the GPU
kernel of tc_census_matrix evaluates the same sums on bit-packed matrices and is compared with
the oracle in tests/test_matrix_gpu.py."""
import numpy as np
import pytest

import graphgen
import oracle


def matrix_census(n, s, d):
    A = np.zeros((n, n), dtype=np.int64)
    keep = s != d
    A[s[keep], d[keep]] = 1
    M = A * A.T
    S = A - M
    N = 1 - np.maximum(A, A.T)
    np.fill_diagonal(N, 0)
    NN, StS, SSt, SS, NM, MM = N @ N, S.T @ S, S @ S.T, S @ S, N @ M, M @ M
    tot = lambda Z, P: int((Z * P).sum())
    c = [tot(N, NN) // 6, tot(S, NN), tot(M, NN) // 2, tot(N, StS) // 2, tot(N, SSt) // 2, tot(N, SS),
         tot(S, NM), tot(S.T, NM), tot(S, SS), tot(S.T, SS) // 3, tot(N, MM) // 2, tot(M, StS) // 2,
         tot(M, SSt) // 2, tot(M, SS), tot(S, MM), tot(M, MM) // 6]
    return c


@pytest.mark.parametrize("seed", range(8))
def test_formulas_equal_the_oracle_on_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 70))
    n, s, d = graphgen.gnp(n, float(rng.choice([0.05, 0.2, 0.5, 0.9])), seed)
    assert matrix_census(n, s, d) == oracle.census_bm(n, s, d)


def test_formulas_on_every_three_vertex_digraph():
    ordered = [(a, b) for a in range(3) for b in range(3) if a != b]
    for mask in range(64):
        pairs = [ordered[i] for i in range(6) if mask >> i & 1]
        s = np.array([p[0] for p in pairs], np.uint32)
        d = np.array([p[1] for p in pairs], np.uint32)
        assert matrix_census(3, s, d) == oracle.census_brute(3, s, d), mask


def test_formulas_on_workload_graphs():
    for (n, s, d) in (graphgen.rmat(9, 16, 0.15, 1), graphgen.chung_lu(400, 8.0, 2.1, 0.1, 4, 2)):
        assert matrix_census(n, s, d) == oracle.census_bm(n, s, d)
