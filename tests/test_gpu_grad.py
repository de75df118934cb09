"""GPU adjoint (cld_grad / autograd) against the CPU oracle.

* elementwise dGamma/dval against the oracle adjoint on identical probes;
* directional derivatives against central finite differences of the FP64
  oracle estimate (same probes, same interval);
* kernel hyper-parameters (Wendland length scale and nugget) through
  torch.autograd against finite differences and against tr(K^-1 dK/dtheta)
  from a dense inverse (statistical: estimator noise).
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def gpu_grad(B, vals, a, b, n, M, seed, dtype="f32", variant=None):
    from paper_1503_06394_gb300 import CsrLogdet

    m = CsrLogdet(B.rowptr, B.col, vals, dtype=dtype)
    if variant is not None:
        m.set_kernel_variant(variant)
    m.set_interval(a, b)
    g, G = m.grad(n, M, seed)
    r = m.estimate(n, M, seed)
    m.close()
    return g, G.cpu().numpy().astype(np.float64), r["logdet"]


def wendland_small(d=2048, seed=5, sigma2=0.1, order="random"):
    ell = 0.002 * np.sqrt(1e6 / d)  # same expected neighbour count as the d = 1e6 workload
    P, _ = workloads.wendland_pattern(d, ell, seed, order)
    rows = np.repeat(np.arange(d), np.diff(P.rowptr))
    diag = rows == P.col
    return P, diag, ell, sigma2


@pytest.mark.parametrize("kind", ["random", "wendland"])
@pytest.mark.parametrize("n,M", [(1, 4), (2, 8), (7, 16), (30, 32), (20, 64), (5, 128), (6, 3), (8, 140)])
def test_grad_matches_oracle_adjoint(torch, kind, n, M):
    if kind == "random":
        B = workloads.sparse_random_spd(1500, 3, 31)
        v32, v64 = B.stored("f32")
        a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    else:
        P, diag, ell, s2 = wendland_small(1024)
        val = workloads.wendland_values(P.val, diag, ell, s2)
        B = workloads.Csr(P.rowptr, P.col, val)
        v32, v64 = B.stored("f32")
        a, b = s2, s2 + float(np.max(np.add.reduceat(np.abs(v64), B.rowptr[:-1])))
    g, G, est = gpu_grad(B, v32, a, b, n, M, seed=n + M)
    V = oracle.rademacher(n + M, B.d, np.arange(M))
    Gref = oracle.grad(B.rowptr, B.col, v64, a, b, n, V)
    scale = np.max(np.abs(Gref))
    assert np.max(np.abs(G - Gref)) <= 2e-5 * scale + 1e-7, np.max(np.abs(G - Gref)) / scale
    assert g == est  # cld_grad's Gamma is the forward estimate


@pytest.mark.parametrize("variant", [None, 6, 7])
@pytest.mark.parametrize("n,K", [(2, 2), (3, 2), (9, 2), (9, 4), (30, 6), (30, 29), (30, 40), (60, 11)])
def test_grad_checkpointed_equals_store_all(torch, n, K, variant):
    """The checkpointed reverse pass (pairs every K steps, segments recomputed)
    gives bit-identical gradients and estimate to keeping every w_j, with a
    smaller workspace when n is large (default inner loop, the staged tiles of
    variant 6 in both passes, and variant 7's gather windows in the forward
    steps and their recomputed segments)."""
    from paper_1503_06394_gb300 import CsrLogdet

    P, diag, ell, s2 = wendland_small(1024)
    val = workloads.wendland_values(P.val, diag, ell, s2)
    B = workloads.Csr(P.rowptr, P.col, val)
    v32, v64 = B.stored("f32")
    a, b = s2, s2 + float(np.max(np.add.reduceat(np.abs(v64), B.rowptr[:-1])))
    out = {}
    for k in (0, K):
        m = CsrLogdet(B.rowptr, B.col, v32)
        if variant is not None:
            m.set_kernel_variant(variant)
        m.set_interval(a, b)
        m.set_grad_checkpoint(k)
        ws = m.reserve(n, 32, 1)
        g, G = m.grad(n, 32, 3)
        out[k] = (g, G.cpu().numpy(), ws)
        m.close()
    assert out[K][0] == out[0][0]
    assert np.array_equal(out[K][1], out[0][1])
    nseg = -(-(n - 1) // K)
    if 2 * (nseg - 1) + K < n:
        assert out[K][2] < out[0][2]


def test_grad_checkpoint_rejects_bad_interval(torch):
    from paper_1503_06394_gb300 import CldError, CsrLogdet

    B = workloads.sparse_random_spd(100, 3, 1)
    v32, _ = B.stored("f32")
    m = CsrLogdet(B.rowptr, B.col, v32)
    for k in (1, -2):
        with pytest.raises(CldError):
            m.set_grad_checkpoint(k)
    m.close()


@pytest.mark.parametrize("variant", [5, 6, 7])
@pytest.mark.parametrize("kind", ["random", "wendland", "wendland_cell"])
@pytest.mark.parametrize("n,M", [(2, 8), (7, 16), (30, 32), (20, 64), (5, 128), (8, 140), (6, 12)])
def test_grad_wide_lanes_matches_oracle_adjoint(torch, kind, n, M, variant):
    """With the forward's wide lanes (variant 5), staged tiles (variant 6) or
    gather windows (variant 7) the reverse pass runs its wide or staged form
    (8 probes per lane, P >= 8; 1 lane per row at P = 8)."""
    if kind == "random":
        B = workloads.sparse_random_spd(1500, 3, 31)
        v32, v64 = B.stored("f32")
        a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    else:
        # cell order: tiles reach three rows of cells (variant 7's windows)
        P, diag, ell, s2 = wendland_small(4096 if kind == "wendland_cell" else 1024,
                                          order="cell" if kind == "wendland_cell" else "random")
        val = workloads.wendland_values(P.val, diag, ell, s2)
        B = workloads.Csr(P.rowptr, P.col, val)
        v32, v64 = B.stored("f32")
        a, b = s2, s2 + float(np.max(np.add.reduceat(np.abs(v64), B.rowptr[:-1])))
    g, G, est = gpu_grad(B, v32, a, b, n, M, seed=n + M, variant=variant)
    V = oracle.rademacher(n + M, B.d, np.arange(M))
    Gref = oracle.grad(B.rowptr, B.col, v64, a, b, n, V)
    scale = np.max(np.abs(Gref))
    assert np.max(np.abs(G - Gref)) <= 2e-5 * scale + 1e-7, np.max(np.abs(G - Gref)) / scale
    assert g == est


@pytest.mark.parametrize("variant", [0, 5, 6])
@pytest.mark.parametrize("M", [8, 32])
def test_grad_bf16_values_at_either_word_half(torch, variant, M):
    """The wide reverse step (taken when the forward runs variant 5) reads
    BF16 values as the 4-byte words that hold them, the narrow one 16 bits at
    a time: either way the gradient of a BF16-valued matrix is the same bit for
    bit whether the value array starts on a 4-byte boundary or 2 bytes past one
    (odd entry count, so the last entry sits alone in its word), and matches
    the oracle adjoint on the stored values.  (Variant 6 stages only 16-byte
    aligned arrays; 2 bytes past the boundary both passes take the wide form,
    whose gradient is the same bit for bit but whose forward moments are
    summed in another order, so there the estimates agree to 1e-12.)"""
    from paper_1503_06394_gb300 import CsrLogdet

    B = workloads.sparse_random_spd(1201, 3, 41)
    assert B.nnz % 2 == 1
    v16, v64 = B.stored("bf16")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    n = 12
    t16 = torch.from_numpy(v16.view(np.int16)).cuda().view(torch.bfloat16)
    Gs = []
    for off in (0, 1):
        buf = torch.zeros(B.nnz + 2, dtype=torch.bfloat16, device="cuda")
        buf[off:off + B.nnz] = t16
        m = CsrLogdet(B.rowptr, B.col, buf[off:off + B.nnz], dtype="bf16")
        m.set_kernel_variant(variant)
        m.set_interval(a, b)
        g, G = m.grad(n, M, 7)
        Gs.append((g, G.cpu().numpy().astype(np.float64)))
        m.close()
    if variant == 6:
        assert abs(Gs[0][0] - Gs[1][0]) <= 1e-12 * abs(Gs[1][0])
    else:
        assert Gs[0][0] == Gs[1][0]
    assert np.array_equal(Gs[0][1], Gs[1][1])
    V = oracle.rademacher(7, B.d, np.arange(M))
    Gref = oracle.grad(B.rowptr, B.col, v64, a, b, n, V)
    scale = np.max(np.abs(Gref))
    assert np.max(np.abs(Gs[0][1] - Gref)) <= 2e-5 * scale + 1e-7


def test_grad_directional_finite_differences(torch):
    """sum_k G_k dir_k against (Gamma(val + h dir) - Gamma(val - h dir)) / 2h of
    the FP64 oracle on the same probes and interval."""
    B = workloads.sparse_random_spd(800, 3, 9)
    v32, v64 = B.stored("f32")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    a, b = 0.8 * a, 1.05 * b  # room for the perturbed spectrum
    n, M, seed = 25, 16, 2
    _, G, _ = gpu_grad(B, v32, a, b, n, M, seed)
    V = oracle.rademacher(seed, B.d, np.arange(M))
    c = oracle.cheb_coeffs(n, a, b)
    rng = np.random.default_rng(0)
    rows = np.repeat(np.arange(B.d), np.diff(B.rowptr))
    for trial in range(3):
        # symmetric perturbation keeps the matrix symmetric: the same value on (r,k) and (k,r)
        key = np.minimum(rows, B.col) * B.d + np.maximum(rows, B.col)
        _, inv = np.unique(key, return_inverse=True)
        dirv = rng.standard_normal(inv.max() + 1)[inv] * 1e-2
        h = 1e-3
        gp = oracle.finalize(c, oracle.moments(B.rowptr, B.col, v64 + h * dirv, a, b, n, V))[1]
        gm = oracle.finalize(c, oracle.moments(B.rowptr, B.col, v64 - h * dirv, a, b, n, V))[1]
        fd = (gp - gm) / (2 * h)
        assert abs(np.dot(G, dirv) - fd) <= 1e-4 * max(1.0, abs(fd)), (np.dot(G, dirv), fd)


def test_grad_edge_cases(torch):
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    B = workloads.sparse_random_spd(300, 3, 3)
    v32, v64 = B.stored("f32")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    g, G, est = gpu_grad(B, v32, a, b, 0, 8, 0)
    assert np.all(G == 0) and abs(g - est) == 0
    # a structurally nonsymmetric pattern is refused
    C = workloads.nonsymmetric_dominant(200, 3, 1)
    c32, _ = C.stored("f32")
    m = CsrLogdet(C.rowptr, C.col, c32)
    m.set_interval(0.5, 20.0)
    with pytest.raises(CldError) as e:
        m.grad(5, 4, 0)
    assert e.value.status == Bd.CLD_ERR_INVALID
    m.close()
    m = CsrLogdet(C.rowptr, C.col, c32, kind="general")
    m.set_interval(0.5, 20.0)
    with pytest.raises(CldError) as e:
        m.grad(5, 4, 0)
    assert e.value.status == Bd.CLD_ERR_UNSUPPORTED
    m.close()


def _wendland_torch(torch, P, diag, ell_t, s2_t):
    dist = torch.as_tensor(P.val, dtype=torch.float64, device="cuda")
    dg = torch.as_tensor(diag, device="cuda")
    r = dist / ell_t
    off = (1 - r) ** 4 * (4 * r + 1)
    return torch.where(dg, 1.0 + s2_t, off).float()


def test_autograd_hyperparameters_vs_finite_differences(torch):
    from paper_1503_06394_gb300 import autograd_logdet

    P, diag, ell0, s20 = wendland_small(2048)
    n, M, seed = 40, 32, 3
    ell = torch.tensor(ell0, dtype=torch.float64, device="cuda", requires_grad=True)
    s2 = torch.tensor(s20, dtype=torch.float64, device="cuda", requires_grad=True)
    vals = _wendland_torch(torch, P, diag, ell, s2)
    rs = float(np.max(np.add.reduceat(np.abs(vals.detach().cpu().numpy().astype(np.float64)), P.rowptr[:-1])))
    iv = (0.5 * s20, 1.1 * (s20 + rs))
    rp = torch.as_tensor(P.rowptr, device="cuda")
    cl = torch.as_tensor(P.col, device="cuda")
    g = autograd_logdet(vals, rp, cl, n, M, seed, iv)
    g.backward()
    # FD of the FP64 oracle on the same probes and interval (values rounded to FP32 as stored)
    V = oracle.rademacher(seed, P.d, np.arange(M))
    c = oracle.cheb_coeffs(n, *iv)

    def gam(e, s):
        v = workloads.wendland_values(P.val, diag, e, s)
        return oracle.finalize(c, oracle.moments(P.rowptr, P.col, v, iv[0], iv[1], n, V))[1]

    he, hs = 1e-4 * ell0, 1e-3
    fd_ell = (gam(ell0 + he, s20) - gam(ell0 - he, s20)) / (2 * he)
    fd_s2 = (gam(ell0, s20 + hs) - gam(ell0, s20 - hs)) / (2 * hs)
    assert abs(ell.grad.item() - fd_ell) <= 2e-3 * abs(fd_ell), (ell.grad.item(), fd_ell)
    assert abs(s2.grad.item() - fd_s2) <= 2e-3 * abs(fd_s2), (s2.grad.item(), fd_s2)


def test_autograd_hyperparameters_vs_cholesky_trace(torch):
    """E[grad] = d/dtheta tr p_n(At) ~ tr(K^-1 dK/dtheta) (dense inverse of the
    d = 2048 instance); the estimator is random, so compare the mean over 8
    independent probe seeds within 5 standard errors."""
    from paper_1503_06394_gb300 import autograd_logdet

    P, diag, ell0, s20 = wendland_small(2048)
    rows = np.repeat(np.arange(P.d), np.diff(P.rowptr))
    K = workloads.Csr(P.rowptr, P.col, workloads.wendland_values(P.val, diag, ell0, s20)).dense()
    Kinv = np.linalg.inv(K)
    r = P.val / ell0
    dK = np.where(diag, 0.0, 20.0 * r ** 2 * (1 - r) ** 3 / ell0)
    exact_ell = float(np.sum(Kinv[P.col, rows] * dK))
    exact_s2 = float(np.trace(Kinv))
    rs = float(np.max(K.sum(axis=1)))
    iv = (0.9 * s20, 1.05 * (s20 + rs))
    rp = torch.as_tensor(P.rowptr, device="cuda")
    cl = torch.as_tensor(P.col, device="cuda")
    ge, gs = [], []
    for seed in range(8):
        ell = torch.tensor(ell0, dtype=torch.float64, device="cuda", requires_grad=True)
        s2 = torch.tensor(s20, dtype=torch.float64, device="cuda", requires_grad=True)
        g = autograd_logdet(_wendland_torch(torch, P, diag, ell, s2), rp, cl, 80, 64, 100 + seed, iv)
        g.backward()
        ge.append(ell.grad.item())
        gs.append(s2.grad.item())
    for est, exact in ((ge, exact_ell), (gs, exact_s2)):
        mean, se = np.mean(est), np.std(est, ddof=1) / np.sqrt(len(est))
        print("grad mean %.4f +- %.4f exact %.4f" % (mean, se, exact))
        assert abs(mean - exact) <= 5 * se + 1e-3 * abs(exact)


def test_grad_config3_full_sampled(torch):
    """Config 3 at full size (1e6 Wendland points, n = 60): the gradient for 4
    probes against the oracle adjoint on the same probes, on a sample of 20,000
    stored entries (and the max over all entries within the same bound)."""
    cfg = workloads.CONFIGS[3]
    K = workloads.make(cfg)
    v32, v64 = K.stored("f32")
    a = cfg["sigma2"]
    b = float(np.max(np.add.reduceat(np.abs(v64), K.rowptr[:-1])))
    n, M, seed = cfg["n"], 4, 7
    g, G, est = gpu_grad(K, v32, a, b, n, M, seed)
    V = oracle.rademacher(seed, K.d, np.arange(M))
    Gref = oracle.grad(K.rowptr, K.col, v64, a, b, n, V)
    scale = np.max(np.abs(Gref))
    idx = np.random.default_rng(0).choice(K.nnz, 20000, replace=False)
    assert np.max(np.abs(G[idx] - Gref[idx])) <= 2e-5 * scale
    assert np.max(np.abs(G - Gref)) <= 2e-5 * scale


def test_grad_staged_wait_runs_out(torch):
    """cld_grad with the staged tiles of variant 6 and one row tile withheld:
    the bounded waits run out and the call returns CLD_ERR_TIMEOUT; with no
    tile withheld the same handle gives the oracle adjoint."""
    from paper_1503_06394_gb300 import CldError, CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    B = workloads.sparse_random_spd(1500, 3, 31)
    v32, v64 = B.stored("f32")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_kernel_variant(6)
    m.set_interval(a, b)
    Bd.cld_debug_withhold_tile(m.h, 2)
    with pytest.raises(CldError) as e:
        m.grad(2, 32, 4)
    assert e.value.status == Bd.CLD_ERR_TIMEOUT
    Bd.cld_debug_withhold_tile(m.h, 0)
    g, G = m.grad(6, 32, 4)
    m.close()
    V = oracle.rademacher(4, B.d, np.arange(32))
    Gref = oracle.grad(B.rowptr, B.col, v64, a, b, 6, V)
    scale = np.max(np.abs(Gref))
    assert np.max(np.abs(G.cpu().numpy() - Gref)) <= 2e-5 * scale + 1e-7
