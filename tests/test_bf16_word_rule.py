"""Host-side model of how the wide-lane kernels read BF16 values: each value
is taken from the aligned 4-byte word that holds it (the upper half on a
little-endian machine when the value sits 2 bytes past a word boundary),
except in rows that hold the array's first or last entry, which read 16 bits.

Checked here for every entry of CSR arrays with empty rows, both word halves
for the array start and odd and even entry counts: the word read outside
the edge rows never leaves the array's bytes, and the half it selects is
the entry itself."""
import numpy as np
import pytest


def word_rule(base, e, nnz, k0, k1):
    """(bytes read [lo, hi), value bits as float32 bits or None for a 16-bit read)."""
    a = base + 2 * e
    if k0 == 0 or k1 == nnz:  # edge row: 16-bit load
        return (a, a + 2), None
    w = a & ~3
    return (w, w + 4), a


@pytest.mark.parametrize("base", [512, 514])
@pytest.mark.parametrize("nnz_parity", [0, 1])
def test_word_reads_stay_in_the_array_and_pick_the_entry(base, nnz_parity):
    rng = np.random.default_rng(base + nnz_parity)
    for trial in range(50):
        d = int(rng.integers(1, 40))
        deg = rng.integers(0, 6, size=d)
        deg[rng.random(d) < 0.3] = 0  # empty rows, at the ends too
        nnz = int(deg.sum())
        if nnz % 2 != nnz_parity:
            deg[int(rng.integers(0, d))] += 1
            nnz += 1
        if nnz == 0:
            continue
        rowptr = np.concatenate([[0], np.cumsum(deg)])
        vals = rng.integers(0, 1 << 16, size=nnz, dtype=np.uint16)
        mem = np.zeros(base + 2 * nnz + 8, dtype=np.uint8)
        mem[base:base + 2 * nnz] = vals.view(np.uint8)  # little-endian storage
        for r in range(d):
            k0, k1 = int(rowptr[r]), int(rowptr[r + 1])
            for e in range(k0, k1):
                (lo, hi), a = word_rule(base, e, nnz, k0, k1)
                assert base <= lo and hi <= base + 2 * nnz, (trial, r, e)
                if a is None:
                    continue
                w = int(mem[lo:hi].view("<u4")[0])
                bits = (w & 0xFFFF0000) if (a & 2) else ((w << 16) & 0xFFFFFFFF)
                assert bits == int(vals[e]) << 16, (trial, e)


def test_edge_rows_are_needed():
    """Without the edge rule the first entry (array 2 bytes past a boundary)
    or the last (array ending 2 bytes past one) would read outside."""
    nnz = 5
    for base, e in ((514, 0), (512, nnz - 1)):
        a = base + 2 * e
        w = a & ~3
        assert w < base or w + 4 > base + 2 * nnz
