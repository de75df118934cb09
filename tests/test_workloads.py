"""The seeded generators produce what their recipes state."""
import numpy as np

import workloads


def _canonical(B):
    for i in range(B.d):
        c = B.col[B.rowptr[i]:B.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)  # sorted, no duplicates


def test_sparse_random_spd_recipe():
    B = workloads.sparse_random_spd(500, 3, 1)
    _canonical(B)
    A = B.dense()
    assert np.allclose(A, A.T)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    g_hi = np.max(np.diag(A) + off)
    assert abs(g_hi - 0.99) < 1e-12
    assert np.allclose(np.diag(A) - off, np.diag(A) - off)  # diagonal = (R + 1) * scale
    scale = 0.99 / np.max(2 * off / (0.99 / g_hi) + 1)
    assert np.all(np.diag(A) > off)


def test_gmrf_grid_closed_form():
    for N, rho in [(5, -0.22), (8, 0.2), (3, 0.0)]:
        G = workloads.gmrf_grid(N, rho)
        _canonical(G)
        c = np.cos(np.pi * np.arange(1, N + 1) / (N + 1))
        exact = np.sum(np.log(1 - rho * 2 * (c[:, None] + c[None, :])))
        assert abs(np.linalg.slogdet(G.dense())[1] - exact) < 1e-10


def test_block_diag_assembly():
    mats = [workloads.sparse_random_spd(d, 3, d) for d in (1, 7, 40)]
    br, S = workloads.block_diag(mats)
    assert list(br) == [0, 1, 8, 48]
    D = S.dense()
    for b, m in enumerate(mats):
        assert np.array_equal(D[br[b]:br[b + 1], br[b]:br[b + 1]], m.dense())
    assert np.count_nonzero(D) == sum(np.count_nonzero(m.dense()) for m in mats)


def test_wendland_and_apex_graph():
    K, pts = workloads.wendland(400, 0.1, 0.1, 3)
    _canonical(K)
    A = K.dense()
    assert np.allclose(A, A.T) and np.allclose(np.diag(A), 1.1)
    assert np.linalg.eigvalsh(A)[0] >= 0.1 - 1e-9  # Wendland kernel is positive semidefinite in 2-D
    L = workloads.apex_graph(300, 700, 2)
    A = L.dense()
    assert np.allclose(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert ev[0] >= 1 - 1e-9 and ev[-1] <= 2 * np.max(np.diag(A)) - 1 + 1e-9


def test_wendland_cell_order_is_a_permutation():
    """order="cell" renumbers the same points: K_cell = P K_random P^T."""
    Kr, pr = workloads.wendland(500, 0.08, 0.1, 4)
    Kc, pc = workloads.wendland(500, 0.08, 0.1, 4, order="cell")
    _canonical(Kc)
    # the permutation that maps random-order points to cell-order points
    key_r = {tuple(p): i for i, p in enumerate(pr)}
    perm = np.array([key_r[tuple(p)] for p in pc])
    assert sorted(perm.tolist()) == list(range(500))
    np.testing.assert_array_equal(Kc.dense(), Kr.dense()[np.ix_(perm, perm)])
    # neighbours are closer in index after the renumbering
    def mean_span(K):
        rows = np.repeat(np.arange(K.d), np.diff(K.rowptr))
        return np.mean(np.abs(rows - K.col))
    assert mean_span(Kc) < 0.5 * mean_span(Kr)


def test_nonsymmetric_dominant_recipe():
    C = workloads.nonsymmetric_dominant(300, 3, 5)
    _canonical(C)
    A = C.dense()
    R = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    S = np.abs(A).sum(axis=0) - np.abs(np.diag(A))
    assert np.allclose(np.diag(A), np.maximum(R, S) + 1)
