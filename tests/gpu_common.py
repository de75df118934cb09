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


def moment_tol(d, n, structured=False, row_terms=16):
    """|t_gpu - t_oracle| bound for FP32 recurrence vectors against the FP64 oracle.

    Each step rounds w_{j+1} entries to FP32 (relative 2^-24 of terms bounded
    by a small multiple of the row's absolute sum); the three-term recurrence
    propagates a perturbation introduced at step i by U_{j-i}, |U_k| <= k+1 on
    [-1,1], and the v^T(.) sum of d such errors grows like sqrt(d) for random
    signs.  The bound allows 64 (j+1)^2 eps32 sqrt(d) plus a 1e-9 d floor.

    ``row_terms``: stored entries per row.  A row's product rounds a sum of
    that many terms, whose random rounding grows like sqrt(terms); the bound
    scales by sqrt(row_terms / 16) beyond 16 (dense rows: row_terms = d).

    ``structured=True`` drops the random-sign assumption: on matrices with a
    few distinct exactly-representable values (the grid Laplacian) the
    entries of w_j take few distinct values and their FP32 roundings share a
    sign, so the errors add up linearly: (j+1)^2 eps32 d."""
    eps = 2.0 ** -24
    j = np.arange(n + 1)[:, None]
    if structured:
        return (j + 1) ** 2 * eps * max(d, 1) + 1e-9 * max(d, 1)
    grow = np.sqrt(max(1.0, row_terms / 16.0))
    return 64.0 * (j + 1) ** 2 * eps * np.sqrt(max(d, 1)) * grow + 1e-9 * max(d, 1)
