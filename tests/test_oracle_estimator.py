"""Pins for the oracle's estimator (Algorithms 1 and 2, Sec. 2.2, Sec. 3).

Each check compares the oracle against something other than itself:
spectral calculus through numpy's dense eigensolver, exhaustive enumeration of
all Rademacher vectors, numpy's slogdet, the closed-form grid spectrum, or
finite differences.
"""
import itertools
import json
import os

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_from_dense(A):
    d = A.shape[0]
    rows, cols = np.nonzero(A)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=d), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), A[rows, cols].astype(np.float64)


def spectral_moments(X, a, b, n, V):
    """v^T T_j(At) v by spectral calculus: At = Q diag(mu) Q^T, T_j(At) = Q diag(T_j(mu)) Q^T."""
    d = X.shape[0]
    At = (2.0 * X - (a + b) * np.eye(d)) / (b - a)
    mu, Q = np.linalg.eigh(At)
    P = Q.T @ V  # d x M
    t = np.empty((n + 1, V.shape[1]))
    for j in range(n + 1):
        e = np.zeros(j + 1)
        e[j] = 1.0
        t[j] = np.sum(npc.chebval(mu, e)[:, None] * P * P, axis=0)
    return t


def random_spd(d, seed, lo=0.2, hi=0.9):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return (Q * rng.uniform(lo, hi, d)) @ Q.T


def test_diagonal_matrix_exact_for_any_probes(oracle_mod):
    """For diagonal B, v_i^2 = 1 makes every probe give sum_i T_j(mu_i) exactly."""
    d, n, M = 300, 25, 7
    lam = np.random.default_rng(1).uniform(0.05, 0.95, d)
    rowptr, col = np.arange(d + 1, dtype=np.int64), np.arange(d, dtype=np.int32)
    a, b = 0.04, 0.96
    V = oracle_mod.rademacher(11, d, np.arange(M))
    t = oracle_mod.moments(rowptr, col, lam, a, b, n, V)
    mu = (2 * lam - a - b) / (b - a)
    for j in range(n + 1):
        e = np.zeros(j + 1)
        e[j] = 1
        np.testing.assert_allclose(t[j], np.sum(npc.chebval(mu, e)), rtol=1e-12, atol=1e-10)
    # and Gamma is within d times the Sec. 4.1 bound of sum log(lam)
    c = oracle_mod.cheb_coeffs(n, a, b)
    _, g = oracle_mod.finalize(c, t)
    delta = a  # [a, b] = [delta, 1-delta]
    assert abs(g - np.sum(np.log(lam))) <= d * oracle_mod.chebyshev_error_bound(delta, n)


def test_moments_match_spectral_calculus_nonsymmetric_CtC(oracle_mod):
    """kind=1 applies C^T C (not C C^T, which has the same trace but other moments)."""
    d, n = 40, 12
    rng = np.random.default_rng(5)
    C = np.eye(d) * 3 + rng.standard_normal((d, d)) * (rng.random((d, d)) < 0.15)
    rowptr, col, val = csr_from_dense(C)
    X = C.T @ C
    ev = np.linalg.eigvalsh(X)
    a, b = ev[0] * 0.9, ev[-1] * 1.1
    V = oracle_mod.rademacher(2, d, np.arange(5))
    t = oracle_mod.moments(rowptr, col, val, a, b, n, V, kind=1)
    np.testing.assert_allclose(t, spectral_moments(X, a, b, n, V), rtol=1e-9, atol=1e-9)
    t_wrong = spectral_moments(C @ C.T, a, b, n, V)
    assert np.max(np.abs(t - t_wrong)) > 1e-3


def test_moments_match_spectral_calculus_symmetric(oracle_mod):
    d, n = 60, 20
    A = random_spd(d, 3)
    A[np.abs(A) < 0.02] = 0.0
    A = (A + A.T) / 2
    rowptr, col, val = csr_from_dense(A)
    ev = np.linalg.eigvalsh(A)
    a, b = ev[0] - 0.01, ev[-1] + 0.01
    V = np.random.default_rng(4).standard_normal((d, 6))
    t = oracle_mod.moments(rowptr, col, val, a, b, n, V)
    np.testing.assert_allclose(t, spectral_moments(A, a, b, n, V), rtol=1e-9, atol=1e-9)


def test_bruteforce_all_sign_vectors_equals_trace(oracle_mod):
    """Averaging over all 2^d Rademacher vectors gives tr T_j(At) exactly (Sec. 2.2:
    E[z^T A z] = tr A), and the spread of z^T A z is 2(||A||_F^2 - sum A_ii^2)."""
    d, n = 10, 9
    A = random_spd(d, 7, 0.1, 0.9)
    rowptr, col, val = csr_from_dense(A)
    a, b = 0.05, 0.95
    V = np.array(list(itertools.product([1.0, -1.0], repeat=d))).T  # d x 2^d
    t = oracle_mod.moments(rowptr, col, val, a, b, n, V)
    mu = np.linalg.eigvalsh((2 * A - (a + b) * np.eye(d)) / (b - a))
    for j in range(n + 1):
        e = np.zeros(j + 1)
        e[j] = 1
        assert abs(t[j].mean() - np.sum(npc.chebval(mu, e))) < 1e-10
    # variance reading of Sec. 2.2 for the matrix T_2(At)
    At = (2 * A - (a + b) * np.eye(d)) / (b - a)
    T2 = 2 * At @ At - np.eye(d)
    var_formula = 2 * (np.sum(T2 * T2) - np.sum(np.diag(T2) ** 2))
    assert abs(t[2].var() - var_formula) < 1e-9 * max(1.0, var_formula)


def test_basis_probes_give_exact_trace(oracle_mod):
    B = workloads.sparse_random_spd(128, 3, 42)
    A = B.dense()
    ev = np.linalg.eigvalsh(A)
    a, b = 0.9 * ev[0], 1.05 * ev[-1]
    n = 40
    t = oracle_mod.moments(B.rowptr, B.col, B.val, a, b, n, np.eye(B.d))
    mu = (2 * ev - a - b) / (b - a)
    for j in range(n + 1):
        e = np.zeros(j + 1)
        e[j] = 1
        assert abs(t[j].sum() - np.sum(npc.chebval(mu, e))) < 1e-9
    c = oracle_mod.cheb_coeffs(n, a, b)
    _, g = oracle_mod.finalize(c, t)
    assert abs(g * B.d - np.sum(np.log(ev))) < 1e-6 * abs(np.sum(np.log(ev)))


@pytest.mark.parametrize("delta,n", [(0.1, 4), (0.1, 10), (0.2, 6), (0.05, 20)])
def test_lemma1_trace_bound(oracle_mod, delta, n):
    """Lemma 1 (Sec. 4.1): for spec(B) in [delta, 1-delta],
    |log det B - tr p_n(B)| <= d * (the per-eigenvalue bound).  tr p_n(B) is
    the estimator's deterministic part, taken exactly with the d basis vectors
    as probes; log det B comes from the eigenvalues numpy draws."""
    d = 96
    X = random_spd(d, 17 + n, lo=delta, hi=1.0 - delta)
    ev = np.linalg.eigvalsh(X)
    rowptr, col, val = csr_from_dense(X)
    t = oracle_mod.moments(rowptr, col, val, delta, 1.0 - delta, n, np.eye(d))
    _, g = oracle_mod.finalize(oracle_mod.cheb_coeffs(n, delta, 1.0 - delta), t)
    err = abs(np.sum(np.log(ev)) - g * d)
    assert err <= d * oracle_mod.chebyshev_error_bound(delta, n)


def test_lemma2_every_probe_estimate_negative(oracle_mod):
    """Lemma 2 at the matrix level: once n meets the lemma's condition, p_n < 0
    on [delta, 1-delta], so p_n(B) is negative definite for spec(B) there and
    every probe's Gamma_p = v^T p_n(B) v is negative, whatever the signs."""
    delta = 0.1
    n = next(k for k in range(1, 200) if oracle_mod.chebyshev_error_bound(delta, k) <= np.log(1 / (1 - delta)))
    X = random_spd(80, 5, lo=delta, hi=1.0 - delta)
    rowptr, col, val = csr_from_dense(X)
    r = oracle_mod.estimate(rowptr, col, val, delta, 1.0 - delta, n, 64, seed=11)
    assert np.all(r["gamma_p"] < 0)


def test_spectrum_invariant(oracle_mod):
    """|t_{j,p}| <= ||v||^2 = d whenever the spectrum lies in [a, b]."""
    B = workloads.sparse_random_spd(500, 3, 9)
    lo, hi = oracle_mod.gershgorin(B.rowptr, B.col, B.val)
    r = oracle_mod.estimate(B.rowptr, B.col, B.val, lo, hi, 60, 8, seed=3)
    assert np.max(np.abs(r["t"])) <= B.d * (1 + 1e-12)
    assert np.all(r["t"][0] == B.d)
    # an interval that misses the top of the spectrum makes the moments blow up
    r_bad = oracle_mod.estimate(B.rowptr, B.col, B.val, lo, 0.5 * hi, 60, 8, seed=3)
    assert np.max(np.abs(r_bad["t"])) > B.d


def test_cholesky_matches_numpy(oracle_mod):
    for d, seed in [(1, 0), (5, 1), (200, 2)]:
        A = random_spd(d, seed, 0.01, 10.0)
        s, ld = np.linalg.slogdet(A)
        assert s > 0 and abs(oracle_mod.logdet_cholesky(A) - ld) < 1e-10 * max(1, abs(ld))
    with pytest.raises(ValueError):
        oracle_mod.logdet_cholesky(-np.eye(3))


def test_gershgorin_encloses_spectrum(oracle_mod):
    B = workloads.sparse_random_spd(400, 3, 13)
    lo, hi = oracle_mod.gershgorin(B.rowptr, B.col, B.val)
    ev = np.linalg.eigvalsh(B.dense())
    assert lo <= ev[0] and ev[-1] <= hi
    assert abs(hi - 0.99) < 1e-12 and lo > 0  # the generator's scaling


def test_sigma_max_bound(oracle_mod):
    C = workloads.nonsymmetric_dominant(300, 3, 4)
    s = np.linalg.svd(C.dense(), compute_uv=False)
    assert s[0] <= oracle_mod.sigma_max_bound(C.rowptr, C.col, C.val)
    assert s[-1] >= 1.0 - 1e-12  # Varah: diagonal dominance by 1 in rows and columns


def test_dominance_margins_bound_sigma_min(oracle_mod):
    """Sec. 3.2 via Varah: sigma_min(C)^2 >= alpha * beta for row/column dominant C."""
    for seed in range(3):
        C = workloads.nonsymmetric_dominant(200, 3, seed)
        al, be = oracle_mod.dominance_margins(C.rowptr, C.col, C.val)
        A = C.dense()
        s = np.linalg.svd(A, compute_uv=False)
        assert al >= 1.0 - 1e-12 and be >= 1.0 - 1e-12
        assert s[-1] ** 2 >= al * be * (1 - 1e-12)
        R = np.sum(np.abs(A), axis=1) - np.abs(np.diag(A))
        S = np.sum(np.abs(A), axis=0) - np.abs(np.diag(A))
        assert abs(al - np.min(np.abs(np.diag(A)) - R)) < 1e-12
        assert abs(be - np.min(np.abs(np.diag(A)) - S)) < 1e-12


def test_grid_closed_form(oracle_mod):
    for N in (1, 2, 6, 9):
        G = workloads.grid_gmrf(N, 0.1)
        assert G.nnz == 5 * N * N - 4 * N
        ld = np.linalg.slogdet(G.dense())[1]
        assert abs(oracle_mod.grid_laplacian_logdet(N, 0.1) - ld) < 1e-10 * max(1, abs(ld))
    g = json.load(open(os.path.join(GOLDEN, "grid_gmrf_logdet.json")))
    assert abs(oracle_mod.grid_laplacian_logdet(g["N"], g["kappa2"]) - g["logdet"]) < 1e-6


def test_kms_closed_form(oracle_mod):
    """log det of rho^|i-k| against numpy's slogdet, and its spectrum inside
    [(1 - |rho|)/(1 + |rho|), (1 + |rho|)/(1 - |rho|)] (the interval the dense
    benchmark gives the estimator)."""
    for d in (1, 2, 5, 64, 300):
        for rho in (0.5, -0.3, 0.9, 0.0):
            i = np.arange(d)
            A = rho ** np.abs(i[:, None] - i[None, :]).astype(np.float64)
            ld = np.linalg.slogdet(A)[1]
            assert abs(oracle_mod.kms_logdet(d, rho) - ld) < 1e-10 * max(1.0, abs(ld)), (d, rho)
            ev = np.linalg.eigvalsh(A)
            r = abs(rho)
            assert ev[0] >= (1 - r) / (1 + r) * (1 - 1e-12) and ev[-1] <= (1 + r) / (1 - r) * (1 + 1e-12)


def test_alg1_literal_equals_interval_form(oracle_mod):
    """Algorithm 1 as printed (recurrence on (I-2B)/(1-2 delta), coefficients of
    log(1-((1-2 delta)x+1)/2)) equals the [delta, 1-delta] interval form."""
    B = workloads.sparse_random_spd(300, 3, 21)
    lo, hi = oracle_mod.gershgorin(B.rowptr, B.col, B.val)
    delta = min(lo, 1 - hi) * 0.999
    for n in (0, 1, 2, 15):
        V = oracle_mod.rademacher(4, B.d, np.arange(9))
        g_lit = oracle_mod.alg1_literal(B.rowptr, B.col, B.val, delta, n, V)
        t = oracle_mod.moments(B.rowptr, B.col, B.val, delta, 1 - delta, n, V)
        _, g = oracle_mod.finalize(oracle_mod.cheb_coeffs(n, delta, 1 - delta), t)
        assert abs(g_lit - g) <= 1e-11 * abs(g)


def test_alg2_literal_equals_interval_form_and_truth(oracle_mod):
    """Algorithm 2 = half the interval-form estimate of logdet(C^T C) on
    [sigma_min^2, sigma_max^2]; with all basis probes and a high degree it meets
    numpy's log|det C|."""
    C = workloads.nonsymmetric_dominant(120, 3, 8)
    smax = oracle_mod.sigma_max_bound(C.rowptr, C.col, C.val)
    smin = 1.0
    n = 80
    V = oracle_mod.rademacher(1, C.d, np.arange(10))
    g2 = oracle_mod.alg2_literal(C.rowptr, C.col, C.val, smin, smax, n, V)
    t = oracle_mod.moments(C.rowptr, C.col, C.val, smin ** 2, smax ** 2, n, V, kind=1)
    _, g = oracle_mod.finalize(oracle_mod.cheb_coeffs(n, smin ** 2, smax ** 2), t)
    assert abs(g2 - g / 2) <= 1e-10 * abs(g2)
    I = np.eye(C.d)
    g2_exact = oracle_mod.alg2_literal(C.rowptr, C.col, C.val, smin, smax, n, I) * 1.0
    # V = I averages over d probes; alg2 divides by m = d, so scale back
    ld = np.linalg.slogdet(C.dense())[1]
    tr_est = (2 * g2_exact - C.d * np.log(smin ** 2 + smax ** 2)) * C.d / 2 + C.d * np.log(smin ** 2 + smax ** 2) / 2
    assert abs(tr_est - ld) < 1e-4 * abs(ld)


def test_config0_estimate_vs_cholesky(oracle_mod):
    """Config-0 workload: the estimate lies within 5 stderr (+ truncation) of the
    exact Cholesky value; the relative error is in the paper's regime."""
    B = workloads.make(workloads.CONFIGS[0])
    _, v64 = B.stored("f32")
    lo, hi = oracle_mod.gershgorin(B.rowptr, B.col, v64)
    r = oracle_mod.estimate(B.rowptr, B.col, v64, lo, hi, 30, 30, seed=0)
    exact = oracle_mod.logdet_cholesky(workloads.Csr(B.rowptr, B.col, v64).dense())
    assert abs(r["gamma"] - exact) <= 5 * r["stderr"] + 1e-3 * abs(exact)
    assert abs(r["gamma"] - exact) / abs(exact) < 5e-3


def test_gradient_matches_finite_differences(oracle_mod):
    """The estimate is a polynomial in the stored values: central differences
    with the same probes match the adjoint gradient."""
    B = workloads.sparse_random_spd(60, 3, 5)
    lo, hi = oracle_mod.gershgorin(B.rowptr, B.col, B.val)
    n, M = 12, 4
    V = oracle_mod.rademacher(0, B.d, np.arange(M))
    G = oracle_mod.grad(B.rowptr, B.col, B.val, lo, hi, n, V)
    c = oracle_mod.cheb_coeffs(n, lo, hi)

    def gamma(val):
        return oracle_mod.finalize(c, oracle_mod.moments(B.rowptr, B.col, val, lo, hi, n, V))[1]

    h = 1e-5
    for k in np.random.default_rng(0).choice(B.nnz, 25, replace=False):
        vp, vm = B.val.copy(), B.val.copy()
        vp[k] += h
        vm[k] -= h
        fd = (gamma(vp) - gamma(vm)) / (2 * h)
        assert abs(fd - G[k]) <= 1e-6 * max(1.0, abs(fd))


def test_gradient_mean_is_inverse_transpose(oracle_mod):
    """With all basis vectors as probes the estimate is tr p_n(At)/d; as n grows its
    gradient tends to d log det B / dB_rk = (B^{-1})_{kr}."""
    B = workloads.sparse_random_spd(50, 3, 6)
    A = B.dense()
    ev = np.linalg.eigvalsh(A)
    a, b = 0.95 * ev[0], 1.02 * ev[-1]
    G = oracle_mod.grad(B.rowptr, B.col, B.val, a, b, 60, np.eye(B.d)) * B.d
    Ainv = np.linalg.inv(A)
    rows = np.repeat(np.arange(B.d), np.diff(B.rowptr))
    np.testing.assert_allclose(G, Ainv[B.col, rows], rtol=0, atol=1e-8)
