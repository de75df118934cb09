"""Batched estimates (many matrices of uneven size in one pass per step):
each block against the single-matrix path with seed + b and against the
oracle; intervals per block; CUDA-graph replay; tile sizes; variants."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import moment_tol, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def spd_mats(sizes, seed):
    return [workloads.sparse_random_spd(int(d), 3, seed + i) for i, d in enumerate(sizes)]


def intervals(mats, general=False):
    a, b = [], []
    for m in mats:
        _, v64 = m.stored("f32")
        if general:
            al, be = oracle.dominance_margins(m.rowptr, m.col, v64)
            lo, hi = al * be, oracle.sigma_max_bound(m.rowptr, m.col, v64) ** 2
        else:
            lo, hi = oracle.gershgorin(m.rowptr, m.col, v64)
        if not hi - lo > 1e-9 * hi:
            lo, hi = 0.5 * lo, 1.5 * hi
        a.append(lo)
        b.append(hi)
    return np.array(a), np.array(b)


SIZES = [1, 2, 31, 32, 33, 300, 1024, 1025, 4000, 7, 2047, 5000, 13, 600]


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_batch_spd_matches_single_and_oracle(torch, variant):
    from paper_1503_06394_gb300 import CsrBatchLogdet, CsrLogdet

    mats = spd_mats(SIZES, 40)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats)
    n, M, seed = 20, 16, 9
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    bt.set_kernel_variant(variant)
    bt.set_intervals(a, b)
    r = bt.estimate(n, M, seed)
    bt.close()
    for k, m in enumerate(mats):
        v32, v64 = m.stored("f32")
        one = CsrLogdet(m.rowptr, m.col, v32)
        one.set_interval(a[k], b[k])
        g1 = one.estimate(n, M, seed + k)["logdet"]
        one.close()
        ref = oracle.estimate(m.rowptr, m.col, v64, a[k], b[k], n, M, seed=seed + k)
        # same probes; only the FP32 per-thread moment sums see another row order
        assert abs(r["logdet"][k] - g1) <= 1e-6 * abs(g1) + 1e-9, (k, r["logdet"][k], g1)
        assert abs(r["logdet"][k] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"]) + 1e-9
        if M > 1 and m.d > 1:
            assert abs(r["stderr"][k] - ref["stderr"]) <= 1e-3 * ref["stderr"] + 1e-9


@pytest.mark.parametrize("variant", [0, 5, 6])
def test_batch_general_matches_oracle(torch, variant):
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = [workloads.nonsymmetric_dominant(int(d), 3, 70 + i) for i, d in enumerate([3, 64, 500, 2500, 1200, 90])]
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32, kind="general")
    bt.set_kernel_variant(variant)
    a, b = bt.auto_intervals()
    ea, eb = intervals(mats, general=True)
    np.testing.assert_allclose(a, ea, rtol=1e-9)
    np.testing.assert_allclose(b, eb, rtol=1e-9)
    n, M = 30, 8
    r = bt.estimate(n, M, 5)
    bt.close()
    for k, m in enumerate(mats):
        _, v64 = m.stored("f32")
        ref = oracle.estimate(m.rowptr, m.col, v64, a[k], b[k], n, M, seed=5 + k, kind=1)
        assert abs(r["logdet"][k] - ref["gamma"] / 2) <= 1e-5 * abs(ref["gamma"] / 2), k


def test_batch_auto_intervals_match_oracle(torch):
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([10, 700, 3000, 40], 3)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    a, b = bt.auto_intervals()
    ea, eb = intervals(mats)
    np.testing.assert_allclose(a, ea, rtol=1e-12)
    np.testing.assert_allclose(b, eb, rtol=1e-12)
    bt.close()


def test_graph_replay_is_identical(torch):
    from paper_1503_06394_gb300 import CsrBatchLogdet, CsrLogdet

    mats = spd_mats([500, 2000, 64], 8)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats)
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    bt.set_intervals(a, b)
    plain = [bt.estimate(15, 16, s)["logdet"] for s in (0, 1)]
    bt.set_graph(True)
    graph = [bt.estimate(15, 16, s)["logdet"] for s in (0, 1, 0)]
    bt.close()
    np.testing.assert_array_equal(plain[0], graph[0])
    np.testing.assert_array_equal(plain[1], graph[1])
    np.testing.assert_array_equal(plain[0], graph[2])
    m = mats[1]
    v32, _ = m.stored("f32")
    one = CsrLogdet(m.rowptr, m.col, v32)
    one.set_interval(a[1], b[1])
    p = one.estimate(30, 32, 4, moments=True)
    one.set_graph(True)
    g = one.estimate(30, 32, 4, moments=True)
    g2 = one.estimate(30, 32, 5, moments=True)
    one.set_graph(False)
    p2 = one.estimate(30, 32, 5, moments=True)
    one.close()
    assert p["logdet"] == g["logdet"] and np.array_equal(p["t"], g["t"])
    assert p2["logdet"] == g2["logdet"]


def test_batch_tile_rows(torch):
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([3000, 900, 5000], 21)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats)
    res = []
    for rows in (256, 1024, 4096):
        bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
        bt.set_tile_rows(rows)
        bt.set_intervals(a, b)
        res.append(bt.estimate(20, 32, 2)["logdet"])
        bt.close()
    for r in res[1:]:
        np.testing.assert_allclose(r, res[0], rtol=1e-6)  # FP32 per-thread sums follow the tiling


def test_batch_autotune_picks_tiles(torch):
    """The batch autotuner times every variant at tile sizes 256 ... 4096, keeps
    a (variant, tile size) pair, leaves that tile size installed, and the
    estimate after it still matches the oracle block by block."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([3000, 900, 5000, 257], 23)
    br, S = workloads.block_diag(mats)
    s32, s64 = S.stored("f32")
    a, b = intervals(mats)
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    bt.set_intervals(a, b)
    v, ms = bt.autotune(20, 32)
    assert v in range(7) and ms > 0
    assert bt.tile_rows in (256, 512, 1024, 2048, 4096)
    got = bt.estimate(20, 32, 9)["logdet"]
    bt.close()
    for i, m in enumerate(mats):
        _, m64 = m.stored("f32")
        ref = oracle.estimate(m.rowptr, m.col, m64, a[i], b[i], 20, 32, seed=9 + i)
        assert abs(got[i] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])


@pytest.mark.parametrize("variant", [0, 5, 6])
def test_batch_two_panels(torch, variant):
    """M = 140 probes: two panels (128 + 12), each block against the oracle."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([700, 40, 1500], 51)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats)
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    bt.set_kernel_variant(variant)
    bt.set_intervals(a, b)
    got = bt.estimate(12, 140, 6)["logdet"]
    bt.close()
    for i, m in enumerate(mats):
        _, m64 = m.stored("f32")
        ref = oracle.estimate(m.rowptr, m.col, m64, a[i], b[i], 12, 140, seed=6 + i)
        assert abs(got[i] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"])


@pytest.mark.parametrize("variant", [0, 4, 5, 6])
def test_batch_bf16_values_at_either_word_half(torch, variant):
    """BF16 batches, the value array starting on a 4-byte boundary or 2 bytes
    past one (odd entry count): the wide tile kernel reads the values as the
    4-byte words that hold them, the others 16 bits at a time; every block
    matches the oracle on the stored values and the two starts agree bit for
    bit (variant 6 stages 16-byte aligned arrays only: 2 bytes past the
    boundary it runs the wide kernel, whose moment sums run in another order,
    so there the two starts agree to 1e-6)."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([1, 301, 2048, 77, 1500], 61)
    br, S = workloads.block_diag(mats)
    assert S.nnz % 2 == 1
    s16, _ = S.stored("bf16")
    a, b = [], []
    for m in mats:
        _, m64 = m.stored("bf16")
        lo, hi = oracle.gershgorin(m.rowptr, m.col, m64)
        if not hi - lo > 1e-9 * hi:
            lo, hi = 0.5 * lo, 1.5 * hi
        a.append(lo)
        b.append(hi)
    n, M, seed = 15, 16, 4
    t16 = torch.from_numpy(s16.view(np.int16)).cuda().view(torch.bfloat16)
    got = []
    for off in (0, 1):
        buf = torch.zeros(S.nnz + 2, dtype=torch.bfloat16, device="cuda")
        buf[off:off + S.nnz] = t16
        bt = CsrBatchLogdet(br, S.rowptr, S.col, buf[off:off + S.nnz], dtype="bf16")
        bt.set_kernel_variant(variant)
        bt.set_intervals(np.array(a), np.array(b))
        got.append(bt.estimate(n, M, seed)["logdet"])
        bt.close()
    if variant == 6:
        np.testing.assert_allclose(got[0], got[1], rtol=1e-6)
    else:
        np.testing.assert_array_equal(got[0], got[1])
    for k, m in enumerate(mats):
        _, m64 = m.stored("bf16")
        ref = oracle.estimate(m.rowptr, m.col, m64, a[k], b[k], n, M, seed=seed + k)
        assert abs(got[0][k] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"]) + 1e-9, k


def test_batch_empty_and_single_row_blocks(torch):
    """Blocks of 0 and 1 rows among ordinary ones, with automatic intervals:
    an empty block gets [1, 2] and estimates exactly 0; a 1 x 1 block's
    one-point spectrum [beta, beta] is widened by 0.1 % on each side and its
    estimate is log beta; every block matches the oracle on the returned
    interval."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    sizes = [1, 0, 5, 0, 300, 1]
    mats = spd_mats(sizes, 31)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    a, b = bt.auto_intervals()
    got = bt.estimate(20, 8, 3)["logdet"]
    bt.close()
    for i, m in enumerate(mats):
        if m.d == 0:
            assert (a[i], b[i]) == (1.0, 2.0) and got[i] == 0.0
            continue
        _, m64 = m.stored("f32")
        if m.d == 1:
            beta = m64[0]
            assert np.isclose(a[i], beta * (1 - 1e-3), rtol=1e-12) and np.isclose(b[i], beta * (1 + 1e-3), rtol=1e-12)
            assert abs(got[i] - np.log(beta)) <= 1e-6 * abs(np.log(beta)) + 1e-9
        ref = oracle.estimate(m.rowptr, m.col, m64, a[i], b[i], 20, 8, seed=3 + i)
        assert abs(got[i] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"]) + 1e-9


def test_batch_rejects_off_block_columns(torch):
    from paper_1503_06394_gb300 import CldError, CsrBatchLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    mats = spd_mats([100, 100], 1)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    col = S.col.copy()
    col[5] = 150  # row of block 0 pointing into block 1
    bt = CsrBatchLogdet(br, S.rowptr, col, s32)
    with pytest.raises(CldError) as e:
        bt.reserve(5, 4)
    assert e.value.status == Bd.CLD_ERR_INVALID
    bt.close()


@pytest.mark.parametrize("kind", ["spd", "general"])
def test_batch_profiling_counts_steps(torch, kind):
    """Profiling events bracket the general degree steps of a batched estimate
    with plain launches (not in graph mode); the results are unchanged."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([300, 4000, 1025], 70) if kind == "spd" else \
        [workloads.nonsymmetric_dominant(d, 3, 70 + i) for i, d in enumerate([300, 4000, 1025])]
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats, general=kind == "general")
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32, kind=kind)
    bt.set_intervals(a, b)
    plain = bt.estimate(20, 16, 3)
    bt.set_profiling(True)
    prof = bt.estimate(20, 16, 3)
    ms, steps, total = bt.last_timing()
    assert ms > 0 and steps == 18 and total > steps
    assert np.array_equal(plain["logdet"], prof["logdet"])
    bt.set_graph(True)
    bt.estimate(20, 16, 3)
    ms, steps, _ = bt.last_timing()
    assert ms == 0 and steps == 0
    bt.close()


@pytest.mark.parametrize("tile_rows", [256, 1024, 4096])
@pytest.mark.parametrize("M", [8, 16, 32, 64, 128])
def test_batch_staged_tiles(torch, tile_rows, M):
    """The staged batch kernel (variant 6): queue tiles cut into sub-tiles of
    2048 / P rows, blocks starting at rows that are not multiples of 4 (the
    copies start up to 3 rows early), blocks shorter than a sub-tile, every
    panel width; each block against the oracle."""
    from paper_1503_06394_gb300 import CsrBatchLogdet

    mats = spd_mats([1, 5, 130, 1027, 3001, 77, 600], 90 + M)
    br, S = workloads.block_diag(mats)
    s32, _ = S.stored("f32")
    a, b = intervals(mats)
    bt = CsrBatchLogdet(br, S.rowptr, S.col, s32)
    bt.set_kernel_variant(6)
    bt.set_tile_rows(tile_rows)
    bt.set_intervals(a, b)
    n = 12
    got = bt.estimate(n, M, 3)
    bt.close()
    for k, m in enumerate(mats):
        _, m64 = m.stored("f32")
        ref = oracle.estimate(m.rowptr, m.col, m64, a[k], b[k], n, M, seed=3 + k)
        assert abs(got["logdet"][k] - ref["gamma"]) <= 1e-5 * abs(ref["gamma"]) + 1e-9, k
