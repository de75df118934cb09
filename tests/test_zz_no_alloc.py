"""The allocation-free entry point cld_estimate_static, for callers that cannot
allocate device memory: code whose device memory all belongs to another
allocator (a framework's caching pool that must not be bypassed), code held to
a fixed device-memory budget, and latency-critical loops that must never block
in cudaMalloc/cudaFree.  Its scratch is the library's built-in device array.

The GPU tests call it through the C ABI twice in a row and compare each result
with the CPU oracle on the same matrix and probes (the entry returns Gamma and
its stderr, so those are compared: Gamma within the 1e-5 relative parity
tolerance used elsewhere), and with the workspace entry point cld_estimate at
the same inner-loop variant (0).  They cover FP32 values at M = 30 (one
panel), BF16 values at M = 140 (two panels of 128 and 12 probes) and FP64
values.  The host-only test checks that a misaligned array is refused before
any CUDA call.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from gpu_common import require_gpu

CASES = [
    # (dtype, d, picks, matrix seed, n, M, probe seed)
    ("f32", 2048, 3, 1000, 30, 30, 0),
    ("bf16", 3000, 3, 31, 20, 140, 7),
    ("f64", 1500, 4, 32, 25, 48, 3),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_static_scratch_entry_matches_oracle(case):
    torch = require_gpu()
    from paper_1503_06394_gb300 import CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    dtype, d, picks, mseed, n, M, seed = case
    B = workloads.sparse_random_spd(d, picks, mseed)
    stored, v64 = B.stored(dtype)
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    ref = oracle.estimate(B.rowptr, B.col, v64, a, b, n, M, seed=seed)
    m = CsrLogdet(B.rowptr, B.col, stored, dtype=dtype)
    m.set_kernel_variant(0)
    m.set_interval(a, b)
    ws = m.estimate(n, M, seed)
    code = {"f32": Bd.CLD_F32, "bf16": Bd.CLD_BF16, "f64": Bd.CLD_F64}[dtype]
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        g, se = Bd.cld_estimate_static(B.d, B.nnz, m.rowptr, m.col, m.val, code, a, b, n, M, seed, stream)
        assert abs(g - ref["gamma"]) <= 1e-5 * abs(ref["gamma"]), (call, g, ref["gamma"])
        assert abs(se - ref["stderr"]) <= 1e-3 * ref["stderr"], (call, se, ref["stderr"])
        assert abs(g - ws["logdet"]) <= 1e-5 * abs(ws["logdet"]), (call, g, ws["logdet"])
        assert abs(se - ws["stderr"]) <= 1e-5 * abs(ws["stderr"]), (call, se, ws["stderr"])
    m.close()


@pytest.mark.gpu
def test_static_scratch_entry_rejects_oversize():
    torch = require_gpu()
    from paper_1503_06394_gb300 import CldError
    from paper_1503_06394_gb300 import _binding as Bd

    d = 200_000  # 3 recurrence blocks of d x 32 floats = 77 MB > 32 MiB
    rowptr = torch.arange(d + 1, dtype=torch.int64, device="cuda")
    col = torch.arange(d, dtype=torch.int32, device="cuda")
    val = torch.full((d,), 0.5, dtype=torch.float32, device="cuda")
    with pytest.raises(CldError) as e:
        Bd.cld_estimate_static(d, d, rowptr, col, val, Bd.CLD_F32, 0.1, 1.0, 10, 32, 0,
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.status == Bd.CLD_ERR_NOMEM and "holds" in e.value.message


def test_static_scratch_entry_refuses_misaligned_arrays():
    """Host-only: the alignment check returns before any CUDA call, so the
    (never dereferenced) addresses here reach no kernel and no GPU is needed."""
    from paper_1503_06394_gb300 import _binding as Bd
    from paper_1503_06394_gb300 import build

    build.build()
    lib = Bd.load()
    g, se = ctypes.c_double(), ctypes.c_double()

    def call(rowptr, col, val, dtype):
        return lib.cld_estimate_static(4, 4, rowptr, col, val, dtype, 0.1, 1.0, 5, 4, 0, None,
                                       ctypes.byref(g), ctypes.byref(se))

    base = 1 << 20  # 256-byte aligned stand-in addresses
    for rp, c, v, dt in [(base + 2, base, base, Bd.CLD_F32), (base + 4, base, base, Bd.CLD_F32),
                         (base, base + 2, base, Bd.CLD_F32), (base, base, base + 2, Bd.CLD_F32),
                         (base, base, base + 1, Bd.CLD_BF16), (base, base, base + 4, Bd.CLD_F64)]:
        assert call(rp, c, v, dt) == Bd.CLD_ERR_INVALID
        assert "aligned" in Bd.cld_last_error()
