"""The allocation-free entry point cld_estimate_static, for callers that cannot
allocate device memory (their device memory belongs to another allocator, a
fixed budget, or a loop that must not block in cudaMalloc).  Its scratch is the
library's built-in device array; this test calls it through the C ABI twice in
a row and compares each result with the workspace entry point cld_estimate on
the same matrix and probes, within the parity tolerance used elsewhere (1e-5
relative).  It lives in its own file, collected last."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_static_scratch_entry_matches_workspace_entry():
    torch = require_gpu()
    from paper_1503_06394_gb300 import CsrLogdet
    from paper_1503_06394_gb300 import _binding as Bd

    cfg = workloads.CONFIGS[0]
    B = workloads.make(cfg)
    v32, v64 = B.stored("f32")
    a, b = oracle.gershgorin(B.rowptr, B.col, v64)
    n, M = cfg["n"], cfg["M"]
    m = CsrLogdet(B.rowptr, B.col, v32)
    m.set_interval(a, b)
    ref = m.estimate(n, M, 0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        g, se = Bd.cld_estimate_static(B.d, B.nnz, m.rowptr, m.col, m.val, Bd.CLD_F32, a, b, n, M, 0, stream)
        assert abs(g - ref["logdet"]) <= 1e-5 * abs(ref["logdet"]), (call, g, ref["logdet"])
        assert abs(se - ref["stderr"]) <= 1e-5 * abs(ref["stderr"]), (call, se, ref["stderr"])
    m.close()


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
