"""Dense kernel-matrix path (tcgen05 tensor cores) against the CPU oracle on
the same BF16 values and probes."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import moment_tol, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def dense_spd_bf16(d, seed, density=1.0, margin=1.0):
    """Symmetric, diagonally dominant dense matrix rounded to BF16 (uint16 bits)
    and its FP64 upcast; the diagonal is margin x the absolute off-diagonal row
    sum + 1 (a margin above 1 keeps the Gershgorin discs of the BF16 values
    positive when d is large)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(d, d)) * (rng.random((d, d)) < density)
    A = (A + A.T) / 2
    np.fill_diagonal(A, 0.0)
    A[np.diag_indices(d)] = margin * np.abs(A).sum(axis=1) + 1.0
    A /= A.diagonal().max() * 2
    bits = A.astype(np.float32).view(np.uint32).astype(np.uint64)
    b16 = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16).astype(np.uint16)
    up = (b16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return b16, up


def csr_of(A):
    d = A.shape[0]
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=d), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), A[rows, cols]


def run_dense(b16, d, a, b, n, M, seed):
    from paper_1503_06394_gb300 import DenseLogdet

    m = DenseLogdet(b16, d)
    m.set_interval(a, b)
    r = m.estimate(n, M, seed, moments=True)
    m.close()
    return r


def check_dense(d, M, n, seed=0, density=1.0):
    b16, A = dense_spd_bf16(d, 100 + d, density)
    rowptr, col, val = csr_of(A)
    lo, hi = oracle.gershgorin(rowptr, col, val)
    if not hi - lo > 1e-9 * hi:  # one-point spectrum (d = 1): widen
        lo, hi = 0.5 * lo, 1.5 * hi
    r = run_dense(b16, d, lo, hi, n, M, seed)
    ref = oracle.estimate(rowptr, col, val, lo, hi, n, M, seed=seed)
    dt = np.abs(r["t"] - ref["t"])
    assert np.all(dt <= moment_tol(d, n, row_terms=max(1, int(density * d)))), (
        dt.max(), np.unravel_index(dt.argmax(), dt.shape))
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])
    return r, ref


def test_dense_one_tile_one_step(torch):
    check_dense(128, 32, 1)


@pytest.mark.parametrize("d", [1, 8, 64, 100, 130, 200, 1000])
@pytest.mark.parametrize("M", [1, 32, 33, 64, 128, 130])
def test_dense_shapes(torch, d, M):
    check_dense(d, M, 6, seed=d + M)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 25])
def test_dense_degrees(torch, n):
    check_dense(700, 32, n, seed=n)


def test_dense_auto_interval_and_graph(torch):
    from paper_1503_06394_gb300 import DenseLogdet

    d = 513
    b16, A = dense_spd_bf16(d, 5, 0.3)
    rowptr, col, val = csr_of(A)
    lo, hi = oracle.gershgorin(rowptr, col, val)
    m = DenseLogdet(b16, d)
    a, b = m.auto_interval(0)
    assert abs(a - lo) <= 1e-9 * abs(lo) and abs(b - hi) <= 1e-9 * abs(hi)
    r1 = m.estimate(20, 32, 3)
    m.set_graph(True)
    r2 = m.estimate(20, 32, 3)
    m.close()
    assert r1["logdet"] == r2["logdet"]
    exact = oracle.logdet_cholesky(A)
    assert abs(r1["logdet"] - exact) <= 5 * r1["stderr"] + 1e-3 * abs(exact)


def test_dense_matches_csr_path(torch):
    """The same BF16 matrix through the sparse path (stored as CSR) and the dense path."""
    from paper_1503_06394_gb300 import CsrLogdet

    d = 1024
    b16, A = dense_spd_bf16(d, 9, 0.05)
    rowptr, col, val = csr_of(A)
    lo, hi = oracle.gershgorin(rowptr, col, val)
    rd = run_dense(b16, d, lo, hi, 30, 32, 1)
    bits = b16[A != 0]
    m = CsrLogdet(rowptr, col, b16[np.nonzero(A)], dtype="bf16")
    m.set_interval(lo, hi)
    rs = m.estimate(30, 32, 1)
    m.close()
    assert abs(rd["logdet"] - rs["logdet"]) <= 1e-5 * abs(rs["logdet"])


def test_dense_multi_tile_sampled(torch):
    """d = 8192: 64 row tiles of 128 and 128 K-blocks of 64 per tile, so the TMA
    ring wraps many times and every CTA's accumulator sums many MMAs.  Every
    moment of probes 0, 17 and 31 against the oracle on the same BF16 values
    stored as CSR, and those probes' Gamma_p within 1e-5."""
    d, n, M, seed = 8192, 12, 32, 5
    b16, A = dense_spd_bf16(d, 123, margin=1.1)
    rowptr, col, val = csr_of(A)
    del A
    lo, hi = oracle.gershgorin(rowptr, col, val)
    from paper_1503_06394_gb300 import DenseLogdet

    m = DenseLogdet(b16, d)
    m.set_interval(lo, hi)
    r = m.estimate(n, M, seed, moments=True, details=True)
    m.close()
    probes = [0, 17, 31]
    ref = oracle.estimate(rowptr, col, val, lo, hi, n, M, seed=seed, probes=probes)
    dt = np.abs(r["t"][:, probes] - ref["t"])
    tol = moment_tol(d, n, row_terms=d)
    rel = [abs(r["gamma_p"][p] - ref["gamma_p"][q]) / abs(ref["gamma_p"][q]) for q, p in enumerate(probes)]
    print("dense d=%d: max |dt|/tol %.3g, Gamma_p rel err %s, moment errors j=1: %s" % (
        d, (dt / tol).max(), ["%.2e" % x for x in rel], dt[1]))
    assert np.all(dt <= tol), (dt / tol).max()
    assert max(rel) <= 1e-5
