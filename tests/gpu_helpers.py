"""Shared helpers of the GPU tests (no compute of the method here: only data
movement and the residual written out entry by entry on the host)."""
import numpy as np


def sampled_residual(A, B_flat_host, X_dev, shape, nrhs, count=2000, seed=123):
    """Backward error of X at `count` random entries.

    r_i = b_i - sum_j sum_k a_{j, i_j k} x_{i with i_j -> k}   (Eq. (sylvesterND))
    eta = max_i |r_i| / (sum_j ||A_j||_inf ||X||_inf + ||B||_inf)

    X stays on the device; only the fibres through the sampled entries are
    gathered (torch indexing is data movement, the arithmetic is numpy here).
    """
    import torch
    rng = np.random.default_rng(seed)
    N = len(shape)
    S = np.ones(N, dtype=np.int64)
    for j in range(1, N):
        S[j] = S[j - 1] * shape[j - 1]
    ntot = int(np.prod(shape, dtype=np.int64))
    ii = np.stack([rng.integers(0, shape[j], size=count) for j in range(N)], axis=1)
    rhs = rng.integers(0, nrhs, size=count)
    lin = (ii * S).sum(axis=1) + rhs * ntot
    acc = np.zeros(count, dtype=np.complex128)
    for j in range(N):
        nj = shape[j]
        ks = np.arange(nj)
        idx = lin[:, None] + (ks[None, :] - ii[:, j:j + 1]) * S[j]
        xs = X_dev[torch.as_tensor(idx.reshape(-1), device=X_dev.device)].cpu().numpy()
        xs = xs.reshape(count, nj)
        acc += np.einsum("ck,ck->c", A[j][ii[:, j], :], xs)
    r = B_flat_host[lin] - acc
    xn = float(X_dev.abs().max().item())
    bn = float(np.abs(B_flat_host).max())
    an = sum(float(np.abs(a).sum(axis=1).max()) for a in A)
    return float(np.abs(r).max()) / (an * xn + bn)
