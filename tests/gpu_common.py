"""Helpers for the GPU parity tests: build once, compare with the oracle."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    return torch


def rows_per_lane(m, M):
    """Rows one lane of the handle's step kernel visits (grid-stride), from its
    launch configuration: the length of the lane's FP32 moment sum."""
    _, lpr, ctas, threads = m.launch_config(M)
    groups = max(1, ctas * threads // max(1, lpr))
    return max(1, -(-m.d // groups))


def moment_tol(d, n, row_terms=16, rows_per_lane=1):
    """|t_gpu - t_oracle| bound for FP32 recurrence vectors against the FP64 oracle.

    Each step rounds w_{j+1} entries to FP32 (relative 2^-24 of terms bounded
    by a small multiple of the row's absolute sum); the three-term recurrence
    propagates a perturbation introduced at step i by U_{j-i}, |U_k| <= k+1 on
    [-1,1], and the v^T(.) sum of d such errors grows like sqrt(d) for random
    signs.  The bound allows 64 (j+1)^2 eps32 sqrt(d) plus a 1e-9 d floor.

    ``row_terms``: stored entries per row.  A row's product rounds a sum of
    that many terms, whose random rounding grows like sqrt(terms); the bound
    scales by sqrt(row_terms / 16) beyond 16 (dense rows: row_terms = d).

    ``rows_per_lane``: each lane sums v_i w_j[i] over the L rows it visits in
    FP32 before the FP64 reduction.  With |w_j|_1 <= sqrt(d) |w_j|_2 <= d
    (T_j(At) has spectral norm <= 1 on an enclosing interval) the terms have
    mean magnitude at most 1; a sum of L such terms that share a sign (as
    v_i w_1[i] ~ At_ii does) carries a rounding error of about
    eps32 L^1.5 / sqrt(3), and the d / L lane sums add these at random, so the
    total is about eps32 L sqrt(d) / sqrt(3).  The bound allows 8 eps32 L sqrt(d).

    The same bound holds on the grid Laplacian, whose few distinct, exactly
    representable values could have made the FP32 roundings share a sign: at
    d = 1e6 (n = 50, M = 64) the largest moment error measured on GB300 is 0.3
    of it, on a 64 x 64 grid 0.07."""
    eps = 2.0 ** -24
    j = np.arange(n + 1)[:, None]
    acc = 8.0 * eps * rows_per_lane * np.sqrt(max(d, 1)) if rows_per_lane > 1 else 0.0
    grow = np.sqrt(max(1.0, row_terms / 16.0))
    return 64.0 * (j + 1) ** 2 * eps * np.sqrt(max(d, 1)) * grow + 1e-9 * max(d, 1) + acc
