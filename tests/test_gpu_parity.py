"""GPU parity: libcld (through the C ABI) against the CPU FP64 oracle on
identical probes.  Tolerance: the estimate within 1e-5 relative (FP32 and FP64
storage) or 2e-3 (BF16 storage, against the oracle on the original values);
moments within the FP32-recurrence bound of gpu_common.moment_tol."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import moment_tol, require_gpu, rows_per_lane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def run_gpu(B, dtype, a, b, n, M, seed=0, moments=True, variant=None):
    from paper_1503_06394_gb300 import CsrLogdet

    stored, _ = B.stored(dtype)
    m = CsrLogdet(B.rowptr, B.col, stored, dtype=dtype)
    if variant is not None:
        m.set_kernel_variant(variant)
    m.set_interval(a, b)
    r = m.estimate(n, M, seed, moments=moments, details=True)
    r["rows_per_lane"] = rows_per_lane(m, M)
    m.close()
    return r


def check(B, dtype, n, M, seed=0, probes=None, interval=None, tol_gamma=1e-5, variant=None):
    _, v64 = B.stored(dtype)
    a, b = interval if interval is not None else oracle.gershgorin(B.rowptr, B.col, v64)
    if not b - a > 1e-9 * abs(b):  # one-point spectrum (d = 1): widen
        a, b = 0.5 * a, 1.5 * b
    r = run_gpu(B, dtype, a, b, n, M, seed, variant=variant)
    ref = oracle.estimate(B.rowptr, B.col, v64, a, b, n, M, seed=seed, probes=probes)
    cols = np.arange(M) if probes is None else np.asarray(probes)
    dt = np.abs(r["t"][:, cols] - ref["t"])
    tol = moment_tol(B.d, n, rows_per_lane=r["rows_per_lane"])
    assert np.all(dt <= tol), "moment mismatch: max |dt|/tol %g at %s" % (
        (dt / tol).max(), np.unravel_index((dt / tol).argmax(), dt.shape))
    r["tol_ratio"] = float((dt / tol).max())
    if probes is None:
        assert abs(r["logdet"] - ref["gamma"]) <= tol_gamma * abs(ref["gamma"]) + 1e-9
        np.testing.assert_allclose(r["c"], ref["c"], rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(r["gamma_p"], ref["gamma_p"], rtol=1e-5, atol=1e-6 * B.d)
        assert abs(r["stderr"] - ref["stderr"]) <= 1e-3 * ref["stderr"] + 1e-9 if M > 1 else True
    return r, ref


@pytest.mark.parametrize("d", [1, 31, 32, 33, 1000, 2048])
@pytest.mark.parametrize("M", [1, 16, 30, 64])
def test_parity_shapes(torch, d, M):
    B = workloads.sparse_random_spd(d, 3, 100 + d)
    check(B, "f32", 12, M, seed=d + M)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("M", [3, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_parity_kernel_variants(torch, variant, M, dtype):
    """Every inner-loop variant at every panel width (4..128 probes), on rows of
    1 to ~50 entries, including a final grid-stride round that only some row
    groups of a warp take."""
    rng = np.random.default_rng(M)
    d = 4099
    deg = rng.integers(0, 25, size=d)
    rows = np.repeat(np.arange(d), deg)
    cols = rng.integers(0, d, size=rows.size)
    keep = rows != cols
    Bo = workloads._coo_to_csr(d, rows[keep], cols[keep], rng.standard_normal(int(keep.sum())), "v")
    B = workloads._with_diagonal(d, Bo, np.zeros(d), "v")
    A = workloads.Csr(B.rowptr, B.col, B.val)
    # symmetrise: (A + A^T) with a dominant diagonal
    sym = workloads._coo_to_csr(d, np.concatenate([np.repeat(np.arange(d), np.diff(A.rowptr)), A.col]),
                                np.concatenate([A.col, np.repeat(np.arange(d), np.diff(A.rowptr))]),
                                np.concatenate([A.val, A.val]), "sym")
    rs = workloads._abs_row_sums(d, sym)
    S = workloads._with_diagonal(d, sym, rs + 1.0, "sym")
    S.val = S.val / (2 * rs.max() + 1.0)
    check(S, dtype, 9, M, seed=M + variant, variant=variant)


@pytest.mark.parametrize("variant", [3, 4, 6, 7])
@pytest.mark.parametrize("M", [16, 64])
def test_parity_ring_variants_grid(torch, variant, M):
    """The shared-memory ring variants, the staged tiles and the gather windows
    on a 64 x 64 five-point grid (every row inside the staged chunk, neighbour rows shared
    between groups) against the oracle."""
    B = workloads.grid_gmrf(64, 0.1)
    r, ref = check(B, "f32", 20, M, seed=M + variant, interval=(0.1, 8.1), variant=variant)
    print("grid 64x64 variant %d M %d: max|dt|/tol %.3g" % (variant, M, r["tol_ratio"]))


@pytest.mark.parametrize("variant", [3, 4])
def test_ring_variants_first_use_in_graph(torch, variant):
    """FP64 values with a ring variant are used by no other test, so their
    kernels meet the shared-memory opt-in first on the way into a CUDA graph
    capture; the replays equal the plain launches and the oracle."""
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.sparse_random_spd(3000, 3, 77)
    _, v64 = B.stored("f64")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    m = CsrLogdet(B.rowptr, B.col, v64, dtype="f64")
    m.set_kernel_variant(variant)
    m.set_interval(a, b)
    m.set_graph(True)
    graph = [m.estimate(15, 24, s)["logdet"] for s in (0, 1, 0)]
    m.set_graph(False)
    plain = [m.estimate(15, 24, s)["logdet"] for s in (0, 1)]
    m.close()
    assert graph == [plain[0], plain[1], plain[0]]
    ref = oracle.estimate(B.rowptr, B.col, v64, a, b, 15, 24, seed=1)
    assert abs(plain[1] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_parity_low_degree(torch, n):
    B = workloads.sparse_random_spd(777, 3, 5)
    check(B, "f32", n, 20, seed=9)


@pytest.mark.parametrize("M", [4, 8, 128, 130, 300])
def test_parity_panels(torch, M):
    """M up to 128 is one panel (padded to a power of two); beyond, panels of 128."""
    B = workloads.sparse_random_spd(600, 3, 11)
    check(B, "f32", 10, M, seed=3)


def test_parity_ragged_rows(torch):
    """Rows with 1 to ~70 stored entries: the first 1000 rows hold only their
    diagonal, the rest pick 0..29 partners among themselves (mirrored), so the
    4-entry unrolled gather loop sees every tail length."""
    rng = np.random.default_rng(0)
    d, lo = 3000, 1000
    deg = rng.integers(0, 30, size=d - lo)
    rows = np.repeat(np.arange(lo, d), deg)
    cols = rng.integers(lo, d, size=rows.size)
    off = rows != cols
    rows, cols = rows[off], cols[off]
    vals = rng.standard_normal(rows.size)
    Bo = workloads._coo_to_csr(d, np.concatenate([rows, cols]), np.concatenate([cols, rows]),
                               np.concatenate([vals, vals]), "ragged")
    R = workloads._abs_row_sums(d, Bo)
    B = workloads._with_diagonal(d, Bo, R + 0.5, "ragged")
    lens = np.diff(B.rowptr)
    assert lens.min() == 1 and lens.max() > 40 and len(set((lens % 4).tolist())) == 4
    check(B, "f32", 15, 32, seed=4)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_config0_full(torch, dtype):
    """Sparse random SPD, d=2048, n=30, M=30, probe seed 0; error vs Cholesky reported."""
    cfg = workloads.CONFIGS[0]
    B = workloads.make(cfg)
    r, ref = check(B, dtype, cfg["n"], cfg["M"], seed=cfg["probe_seed"])
    _, v64 = B.stored(dtype)
    exact = oracle.logdet_cholesky(workloads.Csr(B.rowptr, B.col, v64).dense())
    rel_exact = abs(r["logdet"] - exact) / abs(exact)
    print("config0 %s: gpu=%.6f oracle=%.6f exact=%.6f rel_vs_oracle=%.2e rel_vs_exact=%.2e stderr=%.3f" % (
        dtype, r["logdet"], ref["gamma"], exact, abs(r["logdet"] - ref["gamma"]) / abs(ref["gamma"]),
        rel_exact, r["stderr"]))
    assert abs(r["logdet"] - exact) <= 5 * r["stderr"] + 1e-3 * abs(exact)


def test_bf16_storage(torch):
    """BF16 values: parity with the oracle on the BF16 values, and within 2e-3
    of the oracle on the original FP64 values."""
    B = workloads.sparse_random_spd(4000, 3, 21)
    n, M = 30, 32
    _, v16 = B.stored("bf16")
    lo, hi = oracle.gershgorin(B.rowptr, B.col, B.val)
    lo16, hi16 = oracle.gershgorin(B.rowptr, B.col, v16)
    a, b = 0.98 * min(lo, lo16), 1.0
    r, _ = check(B, "bf16", n, M, interval=(a, b))
    ref64 = oracle.estimate(B.rowptr, B.col, B.val, a, b, n, M, seed=0)
    assert abs(r["logdet"] - ref64["gamma"]) <= 2e-3 * abs(ref64["gamma"])


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("M", [8, 32, 128])
def test_bf16_values_at_either_word_half(torch, variant, M):
    """BF16 value arrays that start on a 4-byte boundary or 2 bytes past one,
    with an odd and an even entry count.  The wide lanes (variant 5) read a
    BF16 value as the 4-byte word that holds it (16-bit loads for the rows that
    hold the array's first or last entry), the other variants 16 bits at a
    time; either way the results must not depend on where the array starts:
    bit-identical across the two starts, and equal to the oracle on the stored
    values.  (Variants 6 and 7 stage only 16-byte aligned arrays: the array 2
    bytes past the boundary runs variant 5, whose w_j are the same but whose
    moment sums run in another order, so there the two starts agree to 1e-5.)"""
    from paper_1503_06394_gb300 import CsrLogdet

    for d, seed in ((1001, 3), (1000, 4)):  # symmetric pattern + diagonal: nnz has the parity of d
        B = workloads.sparse_random_spd(d, 3, seed)
        assert B.nnz % 2 == d % 2
        v16, v64 = B.stored("bf16")
        a, b = oracle.gershgorin(B.rowptr, B.col, v64)
        check(B, "bf16", 9, M, seed=M, interval=(a, b), variant=variant)
        t16 = torch.from_numpy(v16.view(np.int16)).cuda().view(torch.bfloat16)
        runs = []
        for off in (0, 1):
            buf = torch.zeros(B.nnz + 2, dtype=torch.bfloat16, device="cuda")
            buf[off:off + B.nnz] = t16
            vals = buf[off:off + B.nnz]
            assert vals.data_ptr() % 4 == 2 * off
            m = CsrLogdet(B.rowptr, B.col, vals, dtype="bf16")
            m.set_kernel_variant(variant)
            m.set_interval(a, b)
            runs.append(m.estimate(9, M, M, moments=True))
            m.close()
        if variant >= 6:
            assert abs(runs[0]["logdet"] - runs[1]["logdet"]) <= 1e-5 * abs(runs[1]["logdet"])
        else:
            assert runs[0]["logdet"] == runs[1]["logdet"]
            assert np.array_equal(runs[0]["t"], runs[1]["t"])


def test_config1_full_sampled(torch):
    """GMRF 1000x1000 grid (d=1e6), n=50, M=64: all moments of probes 0, 37 and 63
    against the oracle; the estimate against the closed form within 5 stderr."""
    cfg = workloads.CONFIGS[1]
    B = workloads.make(cfg)
    a, b = cfg["kappa2"], cfg["kappa2"] + 8.0
    r, ref = check(B, "f32", cfg["n"], cfg["M"], seed=0, probes=[0, 37, 63], interval=(a, b))
    exact = oracle.grid_laplacian_logdet(cfg["N"], cfg["kappa2"])
    print("config1: gpu=%.3f exact=%.3f rel=%.2e stderr=%.3f max|dt|/tol %.3g" % (
        r["logdet"], exact, abs(r["logdet"] - exact) / exact, r["stderr"], r["tol_ratio"]))
    assert abs(r["logdet"] - exact) <= 5 * r["stderr"]
    # the sampled probes' estimates equal the GPU's per-probe estimates
    for q, p in enumerate([0, 37, 63]):
        assert abs(r["gamma_p"][p] - ref["gamma_p"][q]) <= 1e-5 * abs(ref["gamma_p"][q])


CONFIG2_PROBES = [0, 13, 31]


@pytest.fixture(scope="module")
def config2():
    """Config 2 (sparse random SPD, d = 1e7, 5 picks per row), one interval that
    encloses the Gershgorin discs of the FP64, FP32 and BF16 values alike, and
    the oracle on the original FP64 values for the sampled probes."""
    cfg = workloads.CONFIGS[2]
    B = workloads.make(cfg)
    ends = [oracle.gershgorin(B.rowptr, B.col, B.stored(dt)[1]) for dt in ("f64", "f32", "bf16")]
    a, b = min(e[0] for e in ends), max(e[1] for e in ends)
    ref64 = oracle.estimate(B.rowptr, B.col, B.val, a, b, cfg["n"], cfg["M"], seed=cfg["probe_seed"],
                            probes=CONFIG2_PROBES)
    return cfg, B, (a, b), ref64


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_config2_full_sampled(torch, config2, dtype):
    """Config 2 at full size (d = 1e7, about 1.1e8 stored entries, n = 100,
    M = 32, probe seed 0) with the autotuned inner loop the benchmark times:
    every moment t[j, p] of probes 0, 13 and 31 against the oracle on the
    stored values (FP32 or BF16, upcast exactly), and those probes' Gamma_p
    within 1e-5.  Each precision's error against the oracle on the original
    FP64 values is printed; BF16 storage is gated at 2e-3 there."""
    from paper_1503_06394_gb300 import CsrLogdet

    cfg, B, (a, b), ref64 = config2
    n, M = cfg["n"], cfg["M"]
    stored, v64 = B.stored(dtype)
    m = CsrLogdet(B.rowptr, B.col, stored, dtype=dtype)
    m.set_interval(a, b)
    variant, _ = m.autotune(n, M)
    r = m.estimate(n, M, cfg["probe_seed"], moments=True, details=True)
    L = rows_per_lane(m, M)
    m.close()
    ref = oracle.estimate(B.rowptr, B.col, v64, a, b, n, M, seed=cfg["probe_seed"], probes=CONFIG2_PROBES)
    dt = np.abs(r["t"][:, CONFIG2_PROBES] - ref["t"])
    tol = moment_tol(B.d, n, rows_per_lane=L)
    assert np.all(dt <= tol), "moment mismatch: max |dt|/tol %g at %s" % (
        (dt / tol).max(), np.unravel_index((dt / tol).argmax(), dt.shape))
    worst = 0.0
    for q, p in enumerate(CONFIG2_PROBES):
        rel = abs(r["gamma_p"][p] - ref["gamma_p"][q]) / abs(ref["gamma_p"][q])
        rel64 = abs(r["gamma_p"][p] - ref64["gamma_p"][q]) / abs(ref64["gamma_p"][q])
        worst = max(worst, rel64)
        assert rel <= 1e-5, (p, rel)
        assert rel64 <= (2e-3 if dtype == "bf16" else 1e-5), (p, rel64)
    print("config2 %s variant %d, %d rows per lane: max |dt| %.3g (max |dt|/tol %.3f); Gamma_p rel err vs oracle on stored values "
          "<= 1e-5; vs FP64 oracle on original values %.2e; logdet %.4f stderr %.4f" % (
              dtype, variant, L, dt.max(), (dt / tol).max(), worst, r["logdet"], r["stderr"]))


def test_degenerate_inputs(torch):
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    # empty matrix: log det of a 0 x 0 matrix is 0
    m = CsrLogdet(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    m.set_interval(0.5, 1.0)
    assert m.estimate(5, 3)["logdet"] == 0.0
    m.close()
    # 1 x 1: exact for any probes: sum_j c_j T_j(mu) = p_n(lambda)
    m = CsrLogdet(np.array([0, 1], np.int64), np.array([0], np.int32), np.array([0.3], np.float32))
    m.set_interval(0.1, 1.0)
    r = m.estimate(40, 4)
    assert abs(r["logdet"] - np.log(np.float32(0.3))) < 1e-5
    m.close()
    B = workloads.sparse_random_spd(100, 3, 1)
    v32, _ = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    for a, b in [(0.0, 1.0), (-1.0, 1.0), (0.5, 0.5), (0.9, 0.1), (np.nan, 1.0), (0.1, np.inf)]:
        with pytest.raises(CldError) as e:
            m.set_interval(a, b)
        assert e.value.status == Bd.CLD_ERR_INTERVAL
    with pytest.raises(CldError) as e:
        m.estimate(10, 4)  # no interval yet
    assert e.value.status == Bd.CLD_ERR_INTERVAL
    m.set_interval(0.01, 1.0)
    for n, M in [(-1, 4), (5, 0)]:
        with pytest.raises(CldError) as e:
            m.estimate(n, M)
        assert e.value.status == Bd.CLD_ERR_INVALID
    # interval that misses the top of the spectrum -> CLD_ERR_SPECTRUM
    lo, hi = oracle.gershgorin(B.rowptr, B.col, B.val)
    m.set_interval(lo, 0.4 * hi)
    with pytest.raises(CldError) as e:
        m.estimate(60, 8)
    assert e.value.status == Bd.CLD_ERR_SPECTRUM
    m.close()


@pytest.mark.parametrize("d", [1, 50])
def test_auto_interval_one_point_spectrum(torch, d):
    """A diagonal matrix with equal entries: Gershgorin gives [beta, beta]; the
    automatic interval is widened by 0.1 % on each side and the estimate is
    d log beta (every probe sees the same diagonal)."""
    from paper_1503_06394_gb300 import CsrLogdet

    beta = np.float32(0.37)
    rowptr = np.arange(d + 1, dtype=np.int64)
    col = np.arange(d, dtype=np.int32)
    val = np.full(d, beta, dtype=np.float32)
    m = CsrLogdet(rowptr, col, val)
    a, b = m.auto_interval(0)
    assert np.isclose(a, float(beta) * (1 - 1e-3), rtol=1e-12) and np.isclose(b, float(beta) * (1 + 1e-3), rtol=1e-12)
    r = m.estimate(12, 8, 0)
    m.close()
    exact = d * np.log(float(beta))
    assert abs(r["logdet"] - exact) <= 1e-6 * abs(exact)
    ref = oracle.estimate(rowptr, col, val.astype(np.float64), a, b, 12, 8, seed=0)
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-6 * abs(ref["gamma"])


def test_malformed_csr_rejected(torch):
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    B = workloads.sparse_random_spd(50, 3, 2)
    v32, _ = B.stored("f32")
    bad_col = B.col.copy()
    bad_col[7] = 50
    bad_val = v32.copy()
    bad_val[3] = np.nan
    bad_ptr = B.rowptr.copy()
    bad_ptr[10], bad_ptr[11] = bad_ptr[11], bad_ptr[10]
    for rp, c, v in [(B.rowptr, bad_col, v32), (B.rowptr, B.col, bad_val), (bad_ptr, B.col, v32)]:
        m = CsrLogdet(rp, c, v)
        with pytest.raises(CldError) as e:
            m.reserve(5, 4)
        assert e.value.status == Bd.CLD_ERR_INVALID
        m.close()


def test_gershgorin_and_lanczos_interval(torch):
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.sparse_random_spd(2048, 3, 1000)
    v32, v64 = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    a, b = m.auto_interval(0)
    lo, hi = oracle.gershgorin(B.rowptr, B.col, v64)
    assert abs(a - lo) <= 1e-12 * abs(lo) and abs(b - hi) <= 1e-12 * abs(hi)
    a2, b2 = m.auto_interval(40)
    ev = np.linalg.eigvalsh(workloads.Csr(B.rowptr, B.col, v64).dense())
    assert a2 == a and ev[-1] <= b2 <= b
    assert b2 < 0.8 * b  # Lanczos tightens the Gershgorin end (0.99 -> ~0.62)
    r = m.estimate(30, 30, 0)
    ref = oracle.estimate(B.rowptr, B.col, v64, a2, b2, 30, 30, seed=0)
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])
    m.close()


def test_host_entry_matches_device_entry(torch):
    from paper_1503_06394_gb300 import logdet_host

    B = workloads.sparse_random_spd(5000, 3, 8)
    v32, v64 = B.stored("f32")
    lo, hi = oracle.gershgorin(B.rowptr, B.col, v64)
    r = run_gpu(B, "f32", lo, hi, 25, 32, seed=5, moments=False)
    g, se = logdet_host(B.rowptr, B.col, v32, lo, hi, 25, 32, seed=5)
    assert g == r["logdet"] and se == r["stderr"]


def test_profiling_counts_launches(torch):
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.sparse_random_spd(20000, 3, 8)
    v32, v64 = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.auto_interval(0)
    m.set_profiling(True)
    m.estimate(20, 32, 0)
    ms, steps, total = m.last_timing()
    assert ms > 0 and steps == 18 and total == 20 + 4
    m.close()


def test_autotune_keeps_parity(torch):
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.sparse_random_spd(30000, 5, 77)
    v32, v64 = B.stored("f32")
    lo, hi = oracle.gershgorin(B.rowptr, B.col, v64)
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_interval(lo, hi)
    variant, ms = m.autotune(20, 32)
    assert variant in range(8) and ms > 0
    r = m.estimate(20, 32, 1)
    ref = oracle.estimate(B.rowptr, B.col, v64, lo, hi, 20, 32, seed=1)
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])
    m.close()


def split_length_matrix(d, seed, long_from):
    """SPD matrix whose rows below `long_from` hold about 7 stored entries and
    the rest about 40 (mirrored picks, dominant diagonal, scaled into (0, 1)),
    so the staged kernel meets tiles that fit its stage and tiles that do not."""
    rng = np.random.default_rng(seed)
    picks = np.where(np.arange(d) < long_from, 3, 20)
    rows = np.repeat(np.arange(d), picks)
    cols = (rows + rng.integers(1, d, size=rows.size)) % d
    vals = rng.standard_normal(rows.size)
    Bo = workloads._coo_to_csr(d, np.concatenate([rows, cols]), np.concatenate([cols, rows]),
                               np.concatenate([vals, vals]), "split")
    R = workloads._abs_row_sums(d, Bo)
    B = workloads._with_diagonal(d, Bo, R + 1.0, "split")
    B.val = B.val / (2 * R.max() + 1.0)
    return B


@pytest.mark.parametrize("M", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("d", [7, 1000, 5003])
def test_parity_staged_tiles(torch, M, dtype, d):
    """Variant 6 (tiles staged by bulk copies) against the oracle: tiles whose
    entries fit the stage and tiles that read them from global memory, a
    ragged last tile, fewer rows than one tile, every panel width and value
    type; the estimate within rounding of variant 5's."""
    B = split_length_matrix(d, 50 + d, d // 2)
    r6, ref = check(B, dtype, 12, M, seed=M, variant=6)
    r5, _ = check(B, dtype, 12, M, seed=M, variant=5)
    assert abs(r6["logdet"] - r5["logdet"]) <= 1e-6 * abs(r5["logdet"])


def windowed_matrices():
    """Matrices for the gather windows (variant 7): a five-point grid whose
    tiles reach three row ranges (ragged last tiles at every panel width); a
    Wendland covariance of points numbered by cell (three rows of cells per
    tile); the grid with a long-range pair in every 25th row, so tiles that
    need more than four ranges (no window: global gathers) sit between
    windowed ones."""
    G = workloads.grid_gmrf(70, 0.1)
    W, _ = workloads.wendland(8000, 0.022, 0.1, 31, order="cell")
    d = G.d
    rng = np.random.default_rng(5)
    rows = np.arange(0, d, 25)
    far = (rows + d // 2 + rng.integers(0, 100, size=rows.size)) % d
    rr = np.repeat(np.arange(d), np.diff(G.rowptr))
    Bo = workloads._coo_to_csr(d, np.concatenate([rr, rows, far]), np.concatenate([G.col, far, rows]),
                               np.concatenate([G.val, np.full(rows.size, -0.5), np.full(rows.size, -0.5)]), "gridfar")
    R = workloads._abs_row_sums(d, Bo)
    rrb = np.repeat(np.arange(d), np.diff(Bo.rowptr))
    Bo.val = np.where(Bo.col == rrb, R[rrb] + 0.1, Bo.val)
    # Wendland: the kernel is positive semidefinite, so sigma^2 = 0.1 bounds
    # the spectrum below; the largest absolute row sum bounds it above
    wb = float(np.max(np.add.reduceat(np.abs(W.val), W.rowptr[:-1])))
    return {"grid": (G, (0.1, 8.1)), "wendland": (W, (0.1, wb)), "gridfar": (Bo, None)}


_WINDOWED = {}


@pytest.mark.parametrize("M", [16, 32, 64, 128])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("kind", ["grid", "wendland", "gridfar"])
def test_parity_gather_windows(torch, kind, dtype, M):
    """Variant 7 (gathers from staged windows of w_j) against the oracle on
    the three window matrices at every panel width of 16 or more probes and
    every value type (FP64 at 16 probes has no window room and runs variant 6),
    and within rounding of variant 6's estimate: the same w_j, moment sums in
    another CTA order."""
    if not _WINDOWED:
        _WINDOWED.update(windowed_matrices())
    B, interval = _WINDOWED[kind]
    r7, ref = check(B, dtype, 12, M, seed=M + 1, interval=interval, variant=7)
    r6, _ = check(B, dtype, 12, M, seed=M + 1, interval=interval, variant=6)
    assert abs(r7["logdet"] - r6["logdet"]) <= 1e-9 * abs(r6["logdet"])
    np.testing.assert_allclose(r7["t"], r6["t"], rtol=1e-9, atol=1e-9 * B.d)


def test_gather_windows_wide_span_falls_back(torch):
    """d > 65536 random SPD matrix: every tile's columns span more rows than the
    plan's bitmap covers, so no tile is windowed and variant 7 runs the staged
    path throughout; the result is the oracle's."""
    B = workloads.sparse_random_spd(100_000, 3, 41)
    r7, ref = check(B, "f32", 8, 32, seed=4, variant=7)
    r6, _ = check(B, "f32", 8, 32, seed=4, variant=6)
    assert abs(r7["logdet"] - r6["logdet"]) <= 1e-9 * abs(r6["logdet"])


def test_gather_windows_replan_per_panel(torch):
    """The window plan depends on the panel width (tiles of 2048 / P rows): one
    handle estimated at M = 32, then 64, then 32 again through the same CUDA
    graph, each equal to a fresh handle's estimate at that M."""
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.grid_gmrf(60, 0.1)
    v32, v64 = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_kernel_variant(7)
    m.set_interval(0.1, 8.1)
    m.set_graph(True)
    runs = [m.estimate(10, M, 3, moments=True) for M in (32, 64, 32)]
    m.close()
    for M, r in zip((32, 64, 32), runs):
        ref = oracle.estimate(B.rowptr, B.col, v64, 0.1, 8.1, 10, M, seed=3)
        assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])
        dt = np.abs(r["t"] - ref["t"])
        assert np.all(dt <= moment_tol(B.d, 10))
    assert runs[0]["logdet"] == runs[2]["logdet"]


def test_gather_windows_wait_runs_out(torch):
    """The bounded waits of variant 7: a withheld tile makes the consumers'
    waits run out (CLD_ERR_TIMEOUT), and the handle then gives the oracle's
    result."""
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    B = workloads.grid_gmrf(60, 0.1)
    v32, v64 = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_kernel_variant(7)
    m.set_interval(0.1, 8.1)
    Bd.cld_debug_withhold_tile(m.h, 5)
    with pytest.raises(CldError) as e:
        m.estimate(3, 32, 0)
    assert e.value.status == Bd.CLD_ERR_TIMEOUT
    Bd.cld_debug_withhold_tile(m.h, 0)
    r = m.estimate(6, 32, 0)
    m.close()
    ref = oracle.estimate(B.rowptr, B.col, v64, 0.1, 8.1, 6, 32, seed=0)
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])


def test_staged_wait_runs_out(torch):
    """The bounded waits of variant 6: with one row tile withheld (its stage is
    never filled: an arrival that nothing makes), the consumers' waits run
    out, cld_estimate returns CLD_ERR_TIMEOUT, and the same handle then gives
    the oracle's result once the tile is no longer withheld."""
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    B = workloads.sparse_random_spd(3000, 3, 12)
    v32, v64 = B.stored("f32")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_kernel_variant(6)
    m.set_interval(a, b)
    Bd.cld_debug_withhold_tile(m.h, 3)  # the third tile of 64 rows (M = 32)
    with pytest.raises(CldError) as e:
        m.estimate(2, 32, 0)  # two staged launches, each waiting about 2 s
    assert e.value.status == Bd.CLD_ERR_TIMEOUT
    Bd.cld_debug_withhold_tile(m.h, 0)
    r = m.estimate(6, 32, 0)
    m.close()
    ref = oracle.estimate(B.rowptr, B.col, v64, a, b, 6, 32, seed=0)
    assert abs(r["logdet"] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])
