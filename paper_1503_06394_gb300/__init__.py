"""GB300 (sm_103a) stochastic Chebyshev log-determinants.

Implements the Chebyshev-Hutchinson estimator of Han, Malioutov and Shin,
"Large-scale Log-determinant Computation through Stochastic Chebyshev
Expansions" (arXiv 1503.06394) on one GPU.  The compute lives in libcld.so
(hand-written CUDA behind the C ABI of include/cld.h); this package is its
thin Python binding:

* ``paper_1503_06394_gb300._binding`` -- one ctypes function per ABI entry
  point, same names (``cld_create_csr``, ``cld_estimate``, ...);
* ``CsrLogdet`` / ``logdet`` -- convenience wrappers that hold the device
  arrays and the workspace as torch tensors (PyTorch supplies device memory
  and streams only);
* ``autograd.CldLogdet`` -- a torch.autograd.Function whose backward is the
  library's adjoint kernel (cld_grad).
"""
from ._binding import *  # noqa: F401,F403
from ._binding import CldError, load  # noqa: F401
from .api import CsrBatchLogdet, CsrLogdet, DenseLogdet, logdet, logdet_host  # noqa: F401


def autograd_logdet(values, rowptr, col, n, M, seed=0, interval=(None, None)):
    """torch.autograd-aware estimate (see autograd.py); imports torch lazily."""
    from .autograd import logdet as _ad

    return _ad(values, rowptr, col, n, M, seed, interval)
