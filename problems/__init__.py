"""Seeded synthetic least-squares problems shaped like the paper's experiments.

Shared by the tests, ``bench.py`` and ``__graft_entry__.smoke()``.  This module
holds none of the solver's arithmetic (no sketching, no solver QR, no
iteration): it only draws inputs.

Construction (Sec. 1.1.1 of the paper): ``A = U diag(sigma) V^T`` with ``U``
an ``m x n`` orthonormalised Gaussian (Haar after the sign fix), ``V`` an
``n x n`` orthonormalised Gaussian, ``sigma_k = kappa^{-k/(n-1)}`` (log-spaced
from 1 to 1/kappa, so ``||A|| = 1``), ``x = w/||w||`` for Gaussian ``w``,
``r = beta (I - U U^T) g / ||(I - U U^T) g||`` for Gaussian ``g`` (projected
twice), and ``b = A x + r``.
"""
from __future__ import annotations

import numpy as np


def _haar_columns(G):
    Q, Rg = np.linalg.qr(G)
    s = np.sign(np.diag(Rg))
    s[s == 0] = 1.0
    return Q * s


def sigmas(n: int, kappa: float) -> np.ndarray:
    if n == 1:
        return np.ones(1)
    return kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))


def make_problem(m: int, n: int, kappa: float, resnorm: float, seed: int):
    """numpy problem: returns dict with A (C-contiguous m x n), b, x, r, U, sigma."""
    rng = np.random.default_rng(seed)
    U = _haar_columns(rng.standard_normal((m, n)))
    V = _haar_columns(rng.standard_normal((n, n)))
    sig = sigmas(n, kappa)
    A = np.ascontiguousarray((U * sig) @ V.T)
    w = rng.standard_normal(n)
    x = w / np.linalg.norm(w)
    g = rng.standard_normal(m)
    r = g - U @ (U.T @ g)
    r = r - U @ (U.T @ r)
    nr = np.linalg.norm(r)
    r = r * (resnorm / nr) if nr > 0 else r
    b = A @ x + r
    return {"A": A, "b": b, "x": x, "r": r, "U": U, "V": V, "sigma": sig,
            "kappa": kappa, "resnorm": resnorm, "m": m, "n": n, "seed": seed}


def make_problem_torch(m: int, n: int, kappa: float, resnorm: float, seed: int, device="cuda"):
    """Same construction drawn with torch on ``device`` (for problems too large
    for host numpy); returns torch float64 tensors A (m x n row-major), b, x."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    G = torch.randn(m, n, dtype=torch.float64, device=device, generator=gen)
    Q, Rg = torch.linalg.qr(G, mode="reduced")
    del G
    s = torch.sign(torch.diagonal(Rg))
    s[s == 0] = 1.0
    Q.mul_(s)
    H = torch.randn(n, n, dtype=torch.float64, device=device, generator=gen)
    V, Rv = torch.linalg.qr(H)
    sv = torch.sign(torch.diagonal(Rv))
    sv[sv == 0] = 1.0
    V = V * sv
    sig = torch.as_tensor(sigmas(n, kappa), dtype=torch.float64, device=device)
    w = torch.randn(n, dtype=torch.float64, device=device, generator=gen)
    x = w / torch.linalg.norm(w)
    g = torch.randn(m, dtype=torch.float64, device=device, generator=gen)
    r = g - Q @ (Q.T @ g)
    r = r - Q @ (Q.T @ r)
    r = r * (resnorm / torch.linalg.norm(r))
    A = (Q * sig) @ V.T
    del Q
    A = A.contiguous()
    b = A @ x + r
    return {"A": A, "b": b, "x": x, "r": r, "sigma": sig, "kappa": kappa,
            "resnorm": resnorm, "m": m, "n": n, "seed": seed}


# The paper-shaped configurations (Sec. 1.1.1; Sec. 3.3: d = 20 n, zeta = 8).
SMALL = dict(m=4000, n=50, kappa=1e10, resnorm=1e-6, d=1000, zeta=8, seed=0, q=100)
LARGE = dict(m=2_000_000, n=1000, kappa=1e8, resnorm=1e-4, d=20_000, zeta=8, seed=0, q=100)
