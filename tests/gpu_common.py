"""Shared helpers of the GPU parity tests: the library context, device
tensors from numpy, and the tolerances derived from the rounding analysis."""
import numpy as np

U = 2.0 ** -53
# updates the library runs after the stopping rule first holds (ls_default_opts)
DEFAULT_EXTRA = 3


def gamma(k):
    return k * U / (1 - k * U)


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2311_04362_gb300 as ls
    from paper_2311_04362_gb300 import build
    build.build()
    return torch, ls


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def padded_rowmajor(A, lda):
    m, n = A.shape
    P = np.zeros((m, lda))
    P[:, :n] = A
    return P
