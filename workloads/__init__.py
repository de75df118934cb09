"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module builds matrices only.  It holds none of the estimator's arithmetic
(no coefficients, no recurrence, no spectral bounds used by the method): both
the GPU library and the CPU oracle receive the same arrays from here and
compute everything else on their own.

Every generator is deterministic for a given seed (numpy ``default_rng``,
PCG64, platform independent) and returns a ``Csr`` with int64 row pointers,
int32 column indices sorted within each row, duplicates summed, and FP64
values.  ``Csr.stored(dtype)`` gives the values as the GPU stores them (FP32 by
round-to-nearest-even from FP64; BF16 by round-to-nearest-even from that FP32)
together with their exact FP64 upcast, which is what the oracle is fed.

Recipes
-------
* ``sparse_random_spd(d, picks, seed)``: each row i picks ``picks`` columns
  j != i uniformly at random with N(0,1) values; each pick is mirrored to
  (j, i); duplicate (i, j) entries are summed; the diagonal is the absolute
  off-diagonal row sum + 1; the whole matrix is then scaled by 0.99 / g_hi with
  g_hi = max_i (B_ii + R_i), R_i the absolute off-diagonal row sum, so that the
  Gershgorin discs lie inside (0, 0.99].  picks=3 at d=2048 gives about 6
  off-diagonals per row; picks=5 at d=1e7 gives about 10 (about 1.1e8 stored
  entries with the diagonal).
* ``paper_sparse_random(d, seed)``: the paper's own sparse random generator
  (Sec. 5.1): five off-diagonal picks per row with values uniform in [-1, 1],
  mirrored, diagonal = absolute row sum + 1e-3, no scaling.
* ``grid_gmrf(N, kappa2)``: kappa^2 I + L with L the 5-point Dirichlet
  Laplacian on an N x N grid in natural row-major order (diagonal 4 + kappa^2,
  neighbours -1); nnz = 5 N^2 - 4 N.
* ``nonsymmetric_dominant(d, picks, seed)``: general non-singular C with
  ``picks`` N(0,1) off-diagonals per row at uniform columns and diagonal
  max(row abs-sum, column abs-sum) + 1.
* ``wendland(npts, ell, sigma2, seed, order)``: compactly supported Wendland
  kernel matrix K_ik = (1 - r)^4_+ (4 r + 1), r = |x_i - x_k| / ell, on uniform
  points in the unit square, plus sigma2 on the diagonal; points numbered as
  drawn (order="random") or by cell of side ell (order="cell", neighbours at
  nearby indices; a symmetric permutation of the same matrix).
* ``apex_graph(nv, extra_edges, seed)``: a simple graph with an apex vertex
  joined to every other vertex plus random extra edges; returns the reduced
  Laplacian L(i*) with the apex row and column removed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Csr:
    rowptr: np.ndarray  # int64, d+1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    name: str = ""

    @property
    def d(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def stored(self, dtype: str = "f32"):
        """(stored array, FP64 upcast of the stored values) for dtype f32/bf16/f64."""
        if dtype == "f64":
            v = np.ascontiguousarray(self.val, dtype=np.float64)
            return v, v
        v32 = self.val.astype(np.float32)  # round to nearest even
        if dtype == "f32":
            return v32, v32.astype(np.float64)
        if dtype == "bf16":
            bits = v32.view(np.uint32).astype(np.uint64)
            rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
            b16 = rounded.astype(np.uint16)
            up = (b16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
            return b16, up
        raise ValueError("dtype must be f32, bf16 or f64")

    def dense(self) -> np.ndarray:
        A = np.zeros((self.d, self.d), dtype=np.float64)
        rows = np.repeat(np.arange(self.d), np.diff(self.rowptr))
        np.add.at(A, (rows, self.col), self.val)
        return A


def _coo_to_csr(d: int, rows, cols, vals, name: str) -> Csr:
    """Sort (row, col) and sum duplicates (scipy's linear-time conversion when it
    is importable, else a plain numpy sort; both give the same arrays)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    if rows.size == 0:
        return Csr(np.zeros(d + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                   np.zeros(0, dtype=np.float64), name)
    try:
        import scipy.sparse as sp
    except ImportError:  # pragma: no cover - scipy is present on every target
        sp = None
    if sp is not None and d < 2**31 - 1:
        m = sp.coo_matrix((vals, (rows, cols)), shape=(d, d)).tocsr()
        m.sum_duplicates()
        m.sort_indices()
        return Csr(m.indptr.astype(np.int64), m.indices.astype(np.int32),
                   np.ascontiguousarray(m.data, dtype=np.float64), name)
    key = rows * np.int64(d) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    first = np.ones(key.shape[0], dtype=bool)
    first[1:] = key[1:] != key[:-1]
    starts = np.flatnonzero(first)
    sv = np.add.reduceat(vals, starts)
    uk = key[starts]
    r = uk // d
    c = (uk % d).astype(np.int32)
    counts = np.bincount(r, minlength=d)
    rowptr = np.zeros(d + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return Csr(rowptr, c, sv, name)


def _symmetric_picks(d: int, picks: int, rng, values: str):
    if d < 2 or picks <= 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros(0)
    rows = np.repeat(np.arange(d, dtype=np.int64), picks)
    cols = (rows + rng.integers(1, d, size=rows.shape[0], dtype=np.int64)) % d
    if values == "normal":
        v = rng.standard_normal(rows.shape[0])
    else:
        v = rng.uniform(-1.0, 1.0, size=rows.shape[0])
    return np.concatenate([rows, cols]), np.concatenate([cols, rows]), np.concatenate([v, v])


def _with_diagonal(d: int, off: Csr, diag: np.ndarray, name: str) -> Csr:
    rows = np.repeat(np.arange(d, dtype=np.int64), np.diff(off.rowptr))
    r = np.concatenate([rows, np.arange(d, dtype=np.int64)])
    c = np.concatenate([off.col.astype(np.int64), np.arange(d, dtype=np.int64)])
    v = np.concatenate([off.val, diag])
    return _coo_to_csr(d, r, c, v, name)


def _abs_row_sums(d: int, m: Csr) -> np.ndarray:
    rows = np.repeat(np.arange(d, dtype=np.int64), np.diff(m.rowptr))
    return np.bincount(rows, weights=np.abs(m.val), minlength=d)


def sparse_random_spd(d: int, picks: int, seed: int) -> Csr:
    rng = np.random.default_rng(seed)
    r, c, v = _symmetric_picks(d, picks, rng, "normal")
    off = _coo_to_csr(d, r, c, v, "off")
    R = _abs_row_sums(d, off)
    B = _with_diagonal(d, off, R + 1.0, "sparse_random_spd(d=%d,picks=%d,seed=%d)" % (d, picks, seed))
    g_hi = float(np.max(2.0 * R + 1.0)) if d > 0 else 1.0
    B.val *= 0.99 / g_hi
    return B


def paper_sparse_random(d: int, seed: int, picks: int = 5) -> Csr:
    rng = np.random.default_rng(seed)
    r, c, v = _symmetric_picks(d, picks, rng, "uniform")
    off = _coo_to_csr(d, r, c, v, "off")
    R = _abs_row_sums(d, off)
    return _with_diagonal(d, off, R + 1e-3, "paper_sparse_random(d=%d,seed=%d)" % (d, seed))


def grid_gmrf(N: int, kappa2: float) -> Csr:
    d = N * N
    idx = np.arange(d, dtype=np.int64)
    r, c = idx // N, idx % N
    rows, cols, vals = [idx], [idx], [np.full(d, 4.0 + kappa2)]
    for dr, dc in ((-1, 0), (0, -1), (0, 1), (1, 0)):
        ok = (r + dr >= 0) & (r + dr < N) & (c + dc >= 0) & (c + dc < N)
        rows.append(idx[ok])
        cols.append(idx[ok] + dr * N + dc)
        vals.append(np.full(int(ok.sum()), -1.0))
    return _coo_to_csr(d, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals),
                       "grid_gmrf(N=%d,kappa2=%g)" % (N, kappa2))


def gmrf_grid(N: int, rho: float) -> Csr:
    """Precision J = I - rho A of the 4-neighbour GMRF on an N x N grid (Sec.
    5.2): unit diagonal, -rho between grid neighbours (partial correlation
    rho), natural row-major order; SPD for |rho| < 1/4."""
    G = grid_gmrf(N, 0.0)  # pattern: diagonal 4, neighbours -1
    rows = np.repeat(np.arange(G.d), np.diff(G.rowptr))
    G.val = np.where(G.col == rows, 1.0, rho)
    G.name = "gmrf_grid(N=%d,rho=%g)" % (N, rho)
    return G


def nonsymmetric_dominant(d: int, picks: int, seed: int) -> Csr:
    rng = np.random.default_rng(seed)
    if d < 2 or picks <= 0:
        off = _coo_to_csr(d, [], [], [], "off")
    else:
        rows = np.repeat(np.arange(d, dtype=np.int64), picks)
        cols = (rows + rng.integers(1, d, size=rows.shape[0], dtype=np.int64)) % d
        off = _coo_to_csr(d, rows, cols, rng.standard_normal(rows.shape[0]), "off")
    R = _abs_row_sums(d, off)
    Cs = np.bincount(off.col.astype(np.int64), weights=np.abs(off.val), minlength=d)
    return _with_diagonal(d, off, np.maximum(R, Cs) + 1.0,
                          "nonsymmetric_dominant(d=%d,picks=%d,seed=%d)" % (d, picks, seed))


def wendland_pattern(npts: int, ell: float, seed: int, order: str = "random"):
    """(Csr of distances with the diagonal stored as 0, points npts x 2): all
    pairs of uniform points in the unit square closer than ell, plus the
    diagonal, sorted rows.  Values are the pair distances.  order="random"
    numbers the points as drawn; order="cell" numbers them by cell of side
    ell (row-major), so neighbours get nearby indices (the same matrix up to
    a symmetric permutation: the same logdet)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((npts, 2))
    # cell list with cells of side >= ell: neighbours lie in the 3 x 3 block
    ncell = max(1, int(np.floor(1.0 / ell)))
    cx = np.minimum((pts[:, 0] * ncell).astype(np.int64), ncell - 1)
    cy = np.minimum((pts[:, 1] * ncell).astype(np.int64), ncell - 1)
    cell = cx * ncell + cy
    if order == "cell":
        perm = np.argsort(cell, kind="stable")
        pts, cx, cy, cell = pts[perm], cx[perm], cy[perm], cell[perm]
    elif order != "random":
        raise ValueError("order must be 'random' or 'cell'")
    order = np.argsort(cell, kind="stable")
    starts = np.searchsorted(cell[order], np.arange(ncell * ncell + 1))
    rows_l, cols_l, dist_l = [], [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            nx, ny = cx + ox, cy + oy
            ok = (nx >= 0) & (nx < ncell) & (ny >= 0) & (ny < ncell)
            src = np.flatnonzero(ok)
            nb = nx[src] * ncell + ny[src]
            lo, hi = starts[nb], starts[nb + 1]
            cnt = hi - lo
            rep = np.repeat(src, cnt)
            offs = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
            tgt = order[np.repeat(lo, cnt) + offs]
            dist = np.sqrt(((pts[rep] - pts[tgt]) ** 2).sum(axis=1))
            keep = (dist < ell) & (rep != tgt)
            rows_l.append(rep[keep])
            cols_l.append(tgt[keep])
            dist_l.append(dist[keep])
    rows_l.append(np.arange(npts))
    cols_l.append(np.arange(npts))
    dist_l.append(np.zeros(npts))
    # a stored 0 distance on the diagonal must survive the duplicate summation
    P = _coo_to_csr(npts, np.concatenate(rows_l), np.concatenate(cols_l), np.concatenate(dist_l) + 1.0,
                    "wendland_pattern(n=%d,ell=%g,seed=%d)" % (npts, ell, seed))
    P.val -= 1.0
    return P, pts


def wendland_values(dist: np.ndarray, is_diag: np.ndarray, ell: float, sigma2: float) -> np.ndarray:
    """K_rk = (1 - r)^4 (4 r + 1), r = dist / ell, off the diagonal; 1 + sigma2 on it."""
    r = dist / ell
    return np.where(is_diag, 1.0 + sigma2, (1.0 - r) ** 4 * (4.0 * r + 1.0))


def wendland(npts: int, ell: float, sigma2: float, seed: int, order: str = "random") -> tuple[Csr, np.ndarray]:
    """(K + sigma2 I as Csr, points npts x 2); `order` as in wendland_pattern."""
    P, pts = wendland_pattern(npts, ell, seed, order)
    rows = np.repeat(np.arange(npts), np.diff(P.rowptr))
    vals = wendland_values(P.val, rows == P.col, ell, sigma2)
    return Csr(P.rowptr, P.col, vals, "wendland(n=%d,ell=%g,sigma2=%g,seed=%d)" % (npts, ell, sigma2, seed)), pts


def apex_graph(nv: int, extra_edges: int, seed: int) -> Csr:
    """Reduced Laplacian L(i*) of a simple graph on nv vertices whose vertex 0 is
    joined to all others, plus ``extra_edges`` random edges among vertices 1..nv-1."""
    rng = np.random.default_rng(seed)
    m = nv - 1
    if m < 1:
        return _coo_to_csr(0, [], [], [], "apex")
    if m >= 2 and extra_edges > 0:
        u = rng.integers(0, m, size=extra_edges, dtype=np.int64)
        w = (u + rng.integers(1, m, size=extra_edges, dtype=np.int64)) % m
        a, b = np.minimum(u, w), np.maximum(u, w)
        key = np.unique(a * m + b)  # simple graph: no repeated edges
        a, b = key // m, key % m
    else:
        a = b = np.zeros(0, dtype=np.int64)
    deg = np.ones(m) + np.bincount(a, minlength=m) + np.bincount(b, minlength=m)
    rows = np.concatenate([a, b, np.arange(m)])
    cols = np.concatenate([b, a, np.arange(m)])
    vals = np.concatenate([-np.ones(a.shape[0]), -np.ones(b.shape[0]), deg])
    return _coo_to_csr(m, rows, cols, vals, "apex_graph(nv=%d,edges=%d,seed=%d)" % (nv, extra_edges, seed))


def batch_mixed(count: int, dmin: float, dmax: float, seed: int, picks: int = 3):
    """``count`` matrices with d log-uniform in [dmin, dmax]: the first half
    sparse random SPD (as ``sparse_random_spd``), the second half general
    non-singular (as ``nonsymmetric_dominant``).  Returns (spd list, general list)."""
    rng = np.random.default_rng(seed)
    ds = np.exp(rng.uniform(np.log(dmin), np.log(dmax), size=count)).astype(np.int64)
    seeds = rng.integers(0, 2**31, size=count)
    half = count // 2
    spd = [sparse_random_spd(int(ds[i]), picks, int(seeds[i])) for i in range(half)]
    gen = [nonsymmetric_dominant(int(ds[i]), picks, int(seeds[i])) for i in range(half, count)]
    return spd, gen


def block_diag(mats):
    """(blk_rows, Csr) of the block-diagonal matrix with global indices."""
    ds = np.array([m.d for m in mats], dtype=np.int64)
    blk_rows = np.zeros(len(mats) + 1, dtype=np.int64)
    np.cumsum(ds, out=blk_rows[1:])
    nnzs = np.array([m.nnz for m in mats], dtype=np.int64)
    noff = np.zeros(len(mats) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=noff[1:])
    rowptr = np.zeros(int(blk_rows[-1]) + 1, dtype=np.int64)
    col = np.empty(int(noff[-1]), dtype=np.int32)
    val = np.empty(int(noff[-1]), dtype=np.float64)
    for b, m in enumerate(mats):
        rowptr[blk_rows[b] + 1:blk_rows[b + 1] + 1] = m.rowptr[1:] + noff[b]
        col[noff[b]:noff[b + 1]] = m.col + blk_rows[b]
        val[noff[b]:noff[b + 1]] = m.val
    return blk_rows, Csr(rowptr, col, val, "block_diag(%d)" % len(mats))


def paper_sparse_random_device(d: int, seed: int, torch, device="cuda", picks: int = 5):
    """The recipe of ``paper_sparse_random`` built with torch on the device,
    for sizes whose numpy construction takes minutes (the benchmark's
    d = 3e7 timing of Sec. 5.1).  Same distribution, another random stream
    (torch's Philox on the device), so not the same matrix as the numpy
    generator at equal seed.  Returns (rowptr int64, col int32, val float64)
    CUDA tensors with sorted rows and duplicates summed."""
    g = torch.Generator(device=device).manual_seed(seed)
    rows = torch.arange(d, device=device, dtype=torch.int64).repeat_interleave(picks)
    cols = (rows + torch.randint(1, d, rows.shape, device=device, generator=g, dtype=torch.int64)) % d
    v = torch.rand(rows.shape, device=device, generator=g, dtype=torch.float64) * 2.0 - 1.0
    diag = torch.arange(d, device=device, dtype=torch.int64)
    key = torch.cat([rows * d + cols, cols * d + rows, diag * d + diag])
    val = torch.cat([v, v, torch.zeros(d, device=device, dtype=torch.float64)])
    del rows, cols, v
    key, order = torch.sort(key)
    val = val[order]
    del order
    uk, inv = torch.unique_consecutive(key, return_inverse=True)
    del key
    sv = torch.zeros(uk.shape, device=device, dtype=torch.float64).index_add_(0, inv, val)
    del inv, val
    r = uk // d
    c = uk % d
    del uk
    is_diag = r == c
    absum = torch.zeros(d, device=device, dtype=torch.float64).index_add_(0, r, torch.where(is_diag, 0.0, sv.abs()))
    sv = torch.where(is_diag, absum[r] + 1e-3, sv)
    rowptr = torch.zeros(d + 1, device=device, dtype=torch.int64)
    rowptr[1:] = torch.cumsum(torch.bincount(r, minlength=d), 0)
    return rowptr, c.to(torch.int32), sv


def grid_pattern_device(N: int, torch, device="cuda"):
    """The 5-point pattern of ``grid_gmrf`` on an N x N grid in natural
    row-major order, built on the device: (rowptr int64, col int32,
    is_diag bool) CUDA tensors."""
    d = N * N
    i = torch.arange(d, device=device, dtype=torch.int64)
    r, c = i // N, i % N
    cand = torch.stack([i - N, i - 1, i, i + 1, i + N], dim=1)
    ok = torch.stack([r > 0, c > 0, torch.ones_like(r, dtype=torch.bool), c < N - 1, r < N - 1], dim=1)
    dg = torch.zeros_like(ok)
    dg[:, 2] = True
    rowptr = torch.zeros(d + 1, device=device, dtype=torch.int64)
    rowptr[1:] = torch.cumsum(ok.sum(dim=1), 0)
    return rowptr, cand[ok].to(torch.int32), dg[ok]


# Named workloads of the benchmark and the parity tests.
CONFIGS = {
    0: dict(kind="sparse_random_spd", d=2048, picks=3, seed=1000, n=30, M=30, probe_seed=0),
    1: dict(kind="grid_gmrf", N=1000, kappa2=0.1, n=50, M=64, probe_seed=0),
    2: dict(kind="sparse_random_spd", d=10_000_000, picks=5, seed=1002, n=100, M=32, probe_seed=0),
    3: dict(kind="wendland", npts=1_000_000, ell=0.002, sigma2=0.1, seed=1003, n=60, M=32, probe_seed=0),
    4: dict(kind="batch", count=512, dmin=1e3, dmax=2e5, seed=1004, n=40, M=16, probe_seed=0),
}


def make(cfg: dict) -> Csr:
    if cfg["kind"] == "wendland":
        return wendland(cfg["npts"], cfg["ell"], cfg["sigma2"], cfg["seed"], cfg.get("order", "random"))[0]
    if cfg["kind"] == "sparse_random_spd":
        return sparse_random_spd(cfg["d"], cfg["picks"], cfg["seed"])
    if cfg["kind"] == "grid_gmrf":
        return grid_gmrf(cfg["N"], cfg["kappa2"])
    raise ValueError(cfg["kind"])
