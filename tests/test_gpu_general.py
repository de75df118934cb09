"""Algorithm 2 on the GPU: log|det C| = 1/2 logdet(C^T C) for general
non-singular C, applied as C then C^T (device transpose), against the oracle;
and the spanning-tree application (Sec. 3.3)."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import moment_tol, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def gen_interval(C):
    """[alpha beta, ||C||_1 ||C||_inf] from the oracle's own bounds."""
    al, be = oracle.dominance_margins(C.rowptr, C.col, C.val)
    return al * be, oracle.sigma_max_bound(C.rowptr, C.col, C.val) ** 2


@pytest.mark.parametrize("d,M,n", [(50, 8, 10), (777, 32, 40), (3001, 64, 25)])
def test_general_matches_oracle(torch, d, M, n):
    from paper_1503_06394_gb300 import CsrLogdet

    C = workloads.nonsymmetric_dominant(d, 3, d)
    c32, c64 = C.stored("f32")
    Cs = workloads.Csr(C.rowptr, C.col, c64)
    a, b = gen_interval(Cs)
    m = CsrLogdet(C.rowptr, C.col, c32, kind="general")
    ga, gb = m.auto_interval(0)
    assert abs(ga - a) <= 1e-9 * a and abs(gb - b) <= 1e-9 * b
    r = m.estimate(n, M, 3, moments=True)
    ref = oracle.estimate(C.rowptr, C.col, c64, a, b, n, M, seed=3, kind=1)
    assert np.all(np.abs(r["t"] - ref["t"]) <= moment_tol(d, n))
    assert abs(r["logdet"] - ref["gamma"] / 2) <= 1e-5 * abs(ref["gamma"] / 2)
    # the same numbers through the literal Algorithm 2 (sigma_min^2 = a, sigma_max^2 = b)
    V = oracle.rademacher(3, d, np.arange(M))
    g2 = oracle.alg2_literal(C.rowptr, C.col, c64, np.sqrt(a), np.sqrt(b), n, V)
    assert abs(r["logdet"] - g2) <= 1e-5 * abs(g2)
    m.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
def test_general_kernel_variants(torch, variant):
    """Algorithm 2's two products per step (C x, then C^T y with the recurrence)
    with every inner-loop variant, including the ring's plain-product form."""
    from paper_1503_06394_gb300 import CsrLogdet

    d, M, n = 1500, 32, 20
    C = workloads.nonsymmetric_dominant(d, 3, 11)
    c32, c64 = C.stored("f32")
    a, b = gen_interval(workloads.Csr(C.rowptr, C.col, c64))
    m = CsrLogdet(C.rowptr, C.col, c32, kind="general")
    m.set_kernel_variant(variant)
    m.set_interval(a, b)
    r = m.estimate(n, M, 5, moments=True)
    m.close()
    ref = oracle.estimate(C.rowptr, C.col, c64, a, b, n, M, seed=5, kind=1)
    assert np.all(np.abs(r["t"] - ref["t"]) <= moment_tol(d, n))
    assert abs(r["logdet"] - ref["gamma"] / 2) <= 1e-5 * abs(ref["gamma"] / 2)


def test_general_vs_exact_with_high_degree(torch):
    """Against numpy's log|det C|: statistical (M = 256) within 5 stderr."""
    from paper_1503_06394_gb300 import CsrLogdet

    C = workloads.nonsymmetric_dominant(1500, 3, 4)
    c32, c64 = C.stored("f32")
    m = CsrLogdet(C.rowptr, C.col, c32, kind="general")
    m.auto_interval(0)
    r = m.estimate(80, 256, 0)
    exact = np.linalg.slogdet(workloads.Csr(C.rowptr, C.col, c64).dense())[1]
    assert abs(r["logdet"] - exact) <= 5 * r["stderr"] + 1e-6 * abs(exact)
    m.close()


@pytest.mark.parametrize("nv,edges", [(400, 800), (2000, 6000)])
def test_spanning_trees_apex_graph(torch, nv, edges):
    """tau(G) = det L(i*) for a graph with an apex vertex i* (Kirchhoff); the
    eigenvalues of L(i*) lie in [1, 2 Delta_max - 1] (Sec. 3.3), so Algorithm 2
    runs with sigma_min = 1, sigma_max = 2 Delta_max - 1 (the reduced Laplacian
    is symmetric positive definite, so the SPD path on [1, 2 Delta_max - 1]
    gives log tau as well)."""
    from paper_1503_06394_gb300 import CsrLogdet

    L = workloads.apex_graph(nv, edges, 11)
    l32, l64 = L.stored("f32")
    A = workloads.Csr(L.rowptr, L.col, l64).dense()
    ev = np.linalg.eigvalsh(A)
    rows = np.repeat(np.arange(L.d), np.diff(L.rowptr))
    deg_max = float(np.max(A.diagonal()))  # degree within G (the apex edge included)
    assert ev[0] >= 1 - 1e-9 and ev[-1] <= 2 * deg_max - 1 + 1e-9
    exact = oracle.logdet_cholesky(A)  # log tau(G)
    m = CsrLogdet(L.rowptr, L.col, l32, kind="general")
    m.set_interval(1.0, (2 * deg_max - 1) ** 2)
    rg = m.estimate(120, 128, 1)
    m.close()
    m = CsrLogdet(L.rowptr, L.col, l32)
    m.set_interval(1.0, 2 * deg_max - 1)
    rs = m.estimate(60, 128, 1)
    m.close()
    for r in (rg, rs):
        assert abs(r["logdet"] - exact) <= 5 * r["stderr"] + 1e-3 * abs(exact), (r, exact)


def test_paper_generator_alg2_matches_oracle(torch):
    """The paper's own timing setting (Sec. 5.1) at d = 1e4: its sparse random
    generator (five U[-1,1] picks per row, mirrored, diagonal = absolute row
    sum + 1e-3), Algorithm 2 with sigma_min = 1e-3 and sigma_max = ||C||_1,
    n = 15, m = 10.  Every moment against the oracle on the same probes, the
    estimate within 1e-5 of the oracle and of the literal Algorithm 2; the
    error against numpy's log|det C| is printed (n = 15 is the paper's low
    degree, so that error is the method's, not the kernel's)."""
    from paper_1503_06394_gb300 import CsrLogdet

    d, n, M = 10_000, 15, 10
    C = workloads.paper_sparse_random(d, 1006)
    c32, c64 = C.stored("f32")
    smax = float(np.max(np.add.reduceat(np.abs(c64), C.rowptr[:-1])))  # ||C||_1 (C is symmetric)
    a, b = 1e-3 ** 2, smax ** 2
    m = CsrLogdet(C.rowptr, C.col, c32, kind="general")
    m.set_interval(a, b)
    r = m.estimate(n, M, 0, moments=True)
    m.close()
    ref = oracle.estimate(C.rowptr, C.col, c64, a, b, n, M, seed=0, kind=1)
    dt = np.abs(r["t"] - ref["t"])
    assert np.all(dt <= moment_tol(d, n)), dt.max()
    assert abs(r["logdet"] - ref["gamma"] / 2) <= 1e-5 * abs(ref["gamma"] / 2)
    V = oracle.rademacher(0, d, np.arange(M))
    g2 = oracle.alg2_literal(C.rowptr, C.col, c64, 1e-3, smax, n, V)
    assert abs(r["logdet"] - g2) <= 1e-5 * abs(g2)
    exact = float(np.linalg.slogdet(C.dense())[1])
    print("paper generator d=%d: gpu %.4f oracle %.4f exact %.4f rel err vs exact %.3e" % (
        d, r["logdet"], ref["gamma"] / 2, exact, abs(r["logdet"] - exact) / abs(exact)))


@pytest.mark.parametrize("kind", ["general", "spd"])
def test_spanning_trees_apex_graph_matches_oracle(torch, kind):
    """Spanning-tree counts (Sec. 3.3) with identical probes: the reduced
    Laplacian L(i*) of a graph with an apex vertex, Algorithm 2 on
    [1, (2 Delta_max - 1)^2] (kind 'general') or Algorithm 1 on
    [1, 2 Delta_max - 1] (kind 'spd'); every moment and the estimate of
    log tau(G) against the oracle."""
    from paper_1503_06394_gb300 import CsrLogdet

    L = workloads.apex_graph(2000, 6000, 11)
    l32, l64 = L.stored("f32")
    rows = np.repeat(np.arange(L.d), np.diff(L.rowptr))
    deg_max = float(np.max(l64[L.col == rows]))
    n, M = (120, 64) if kind == "general" else (60, 64)
    a, b = (1.0, (2 * deg_max - 1) ** 2) if kind == "general" else (1.0, 2 * deg_max - 1)
    m = CsrLogdet(L.rowptr, L.col, l32, kind=kind)
    m.set_interval(a, b)
    r = m.estimate(n, M, 1, moments=True)
    m.close()
    ref = oracle.estimate(L.rowptr, L.col, l64, a, b, n, M, seed=1, kind=1 if kind == "general" else 0)
    tol = moment_tol(L.d, n)
    dt = np.abs(r["t"] - ref["t"])
    assert np.all(dt <= tol), (dt / tol).max()
    want = ref["gamma"] / 2 if kind == "general" else ref["gamma"]
    assert abs(r["logdet"] - want) <= 1e-5 * abs(want)
    print("apex graph %s: max |dt|/tol %.3g" % (kind, (dt / tol).max()))
