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


def check_dense(d, M, n, seed=0, density=1.0, margin=1.0):
    b16, A = dense_spd_bf16(d, 100 + d, density, margin)
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


def test_dense_launch_config_reports_stream_k(torch):
    """cld_launch_config on a dense handle reports the stream-K step's launch:
    a persistent grid of at most two CTAs per SM at 32 probes (one at 64),
    never more CTAs than (tile, K block) units, 192 threads each.  d = 1000:
    8 row tiles x 16 K blocks = 128 units, so 128 CTAs; d = 2048: 512 units,
    so two (one) CTAs per SM."""
    from paper_1503_06394_gb300 import DenseLogdet

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for d, M, want in ((1000, 32, 128), (2048, 32, min(512, 2 * sms)), (2048, 64, min(512, sms))):
        b16, _ = dense_spd_bf16(d, 7)
        m = DenseLogdet(b16, d)
        got = m.launch_config(M)
        m.close()
        assert tuple(got) == (32 if M <= 32 else 64, 1, want, 192), (d, M, got)


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


@pytest.mark.parametrize("M", [64, 128])
def test_dense_pieces_reuse_tmem(torch, M):
    """d = 2000 at 64 and 128 probes (one CTA per SM): 16 row tiles of 32
    K blocks over 152 stream-K CTAs, so CTAs hold two pieces of adjacent
    tiles and the accumulator sets are reused (one set at 128 probes: the
    second piece's MMAs wait for the first piece's epilogue).  Every moment
    against the oracle on the same BF16 values."""
    check_dense(2000, M, 6, seed=M, margin=1.1)


def test_dense_more_tiles_than_ctas(torch):
    """d = 40960: 320 row tiles of 640 K blocks over 304 stream-K CTAs, so some
    CTAs hold the end of one tile, a whole tile and the start of a third, and
    each accumulator set serves several pieces.  The Kac-Murdock-Szego matrix
    0.5^|i-k| (exact in BF16) against its closed-form logdet within 4
    standard errors, and two estimates bit-identical (a tile's pieces are added
    in piece order, whichever CTA finishes it)."""
    from paper_1503_06394_gb300 import DenseLogdet

    d, n, M, rho = 40960, 30, 32, 0.5
    free, _ = torch.cuda.mem_get_info()
    if free < 8e9:
        pytest.skip("needs about 8 GB of free device memory")
    Ab = torch.empty((d, d), dtype=torch.bfloat16, device="cuda")
    cols = torch.arange(d, device="cuda", dtype=torch.float32)
    for r0 in range(0, d, 2048):
        rows = torch.arange(r0, min(d, r0 + 2048), device="cuda", dtype=torch.float32)
        Ab[r0:r0 + rows.numel()] = torch.pow(rho, (rows[:, None] - cols[None, :]).abs()).to(torch.bfloat16)
    m = DenseLogdet(Ab, d)
    m.set_interval((1 - rho) / (1 + rho), (1 + rho) / (1 - rho))
    r1 = m.estimate(n, M, 3, moments=True)
    r2 = m.estimate(n, M, 3, moments=True)
    m.close()
    del Ab
    torch.cuda.empty_cache()
    exact = oracle.kms_logdet(d, rho)
    assert abs(r1["logdet"] - exact) <= 4 * r1["stderr"], (r1["logdet"], exact, r1["stderr"])
    assert r1["logdet"] == r2["logdet"] and np.array_equal(r1["t"], r2["t"])
