"""Seeded synthetic dependence matrices and initial factors.

This module is the one piece shared by the FP64 oracle and the CUDA path: it
draws the inputs, and holds none of the solver's arithmetic (no gradient, no
objective, no update rule).  Every matrix is symmetric, entrywise in [0, 1]
and has a unit diagonal, like the two input types of the paper (absolute
Pearson correlation, Sec. 3.1; unit-diagonal empirical TPDM, Sec. 3.4 and
Appendix "Benchmark Data Generation").  Rows are permuted before the
dependence matrix is formed, as the paper's generator does, so block
structure is not visible in storage order.

Random draws use numpy's PCG64 ``Generator`` (stream-stable across machines);
the n x n Gram/correlation products run through torch in float64 on the
requested device (CPU for small n, the GPU for the large fixtures), in row
chunks so that no n x n float64 intermediate is held for large n.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Instance", "corr_planted", "tpdm_groups", "corr_factor", "planted_exact",
    "init_uniform", "init_scaled", "batch_specs",
]


@dataclass
class Instance:
    """One generated dependence matrix plus its metadata.

    ``S`` is either a numpy float64 array (``materialize='numpy'``) or a torch
    tensor of ``dtype`` on ``device``; ``perm`` maps storage row -> original
    row; ``labels`` is the planted group of each storage row.
    """
    S: object
    n: int
    kind: str
    seed: int
    perm: np.ndarray
    labels: np.ndarray
    meta: dict = field(default_factory=dict)


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _torch():
    import torch
    return torch


def _gram_abs_unitdiag(Y: np.ndarray, scale: float, device: str, out_dtype,
                       absolute: bool, chunk: int = 8192, ld: int | None = None,
                       block_fn=None, compute_dtype=None):
    """S = D^-1/2 |scale * Y Y^T| D^-1/2, filled chunk pair by chunk pair.

    ``Y`` is n x T (float64).  Only chunk pairs (r, c) with c >= r are
    computed; each is written to (r, c) and, transposed, to (c, r), so the
    stored matrix is exactly symmetric.  Returns a torch tensor n x ld
    (columns past n zero) of ``out_dtype`` on ``device`` and the float64 sum
    of squares of the float64 values before the final cast.

    With ``block_fn`` nothing is stored: each chunk pair (c >= r) is passed
    as ``block_fn(r0, r1, c0, c1, blk)`` (the caller stores it and, for
    c0 != r0, its transpose) and the first return value is None.
    ``compute_dtype`` (default float64) is the precision of the products.
    """
    torch = _torch()
    n = Y.shape[0]
    ld = n if ld is None else ld
    cdt = compute_dtype or torch.float64
    Yt = torch.from_numpy(np.ascontiguousarray(Y)).to(device=device, dtype=torch.float64)
    d = (Yt * Yt).sum(dim=1) * scale
    rs = torch.rsqrt(d).to(cdt)
    Yt = Yt.to(cdt)
    out = torch.zeros((n, ld), dtype=out_dtype, device=device) if block_fn is None else None
    norm2 = 0.0
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        for c0 in range(r0, n, chunk):
            c1 = min(n, c0 + chunk)
            blk = (Yt[r0:r1] @ Yt[c0:c1].T) * scale
            if absolute:
                blk = blk.abs()
            blk = blk * rs[r0:r1, None] * rs[None, c0:c1]
            blk.clamp_(0.0, 1.0)
            if c0 == r0:
                lower = torch.tril(blk, -1)
                blk = lower + lower.T
                blk.fill_diagonal_(1.0)
            w = 1.0 if c0 == r0 else 2.0
            norm2 += w * float((blk.double() * blk.double()).sum())
            if block_fn is not None:
                block_fn(r0, r1, c0, c1, blk)
                continue
            out[r0:r1, c0:c1] = blk.to(out_dtype)
            if c0 != r0:
                out[c0:c1, r0:r1] = blk.T.to(out_dtype)
    return out, norm2


def _finish(S_t, n, kind, seed, perm, labels, meta, materialize):
    if materialize == "numpy":
        S = S_t[:, :n].double().cpu().numpy() if S_t.shape[1] != n else S_t.double().cpu().numpy()
    else:
        S = S_t
    return Instance(S=S, n=n, kind=kind, seed=seed, perm=perm, labels=labels, meta=meta)


def corr_planted(n: int = 512, groups: int = 8, T: int = 2000, lo: float = 0.3,
                 hi: float = 0.9, seed: int = 0, device: str = "cpu",
                 dtype=None, materialize: str = "numpy", ld: int | None = None) -> Instance:
    """Absolute Pearson correlation of a planted one-factor-per-group model.

    x_i = a_i z_{g(i)} + e_i over T samples, a_i ~ U[lo, hi], z, e iid N(0, 1);
    ``groups`` groups of (about) n/groups rows, rows permuted, S = |corr(x)|.
    At n=512, groups=8, T=2000 this is the n=512 k=8 correlation workload.
    """
    torch = _torch()
    rng = _rng(seed, 1)
    labels0 = np.repeat(np.arange(groups), int(math.ceil(n / groups)))[:n]
    a = rng.uniform(lo, hi, size=n)
    z = rng.standard_normal((groups, T))
    e = rng.standard_normal((n, T))
    perm = rng.permutation(n)
    labels = labels0[perm]
    X = a[perm, None] * z[labels] + e[perm]
    Xc = X - X.mean(axis=1, keepdims=True)
    S_t, norm2 = _gram_abs_unitdiag(Xc, 1.0 / T, device, dtype or torch.float64, True, ld=ld)
    return _finish(S_t, n, "corr", seed, perm, labels, {"T": T, "groups": groups, "normS2_f64": norm2}, materialize)


def tpdm_groups(n: int = 20000, groups: int = 32, T: int = 5000, overlap: float = 0.03,
                q: float = 0.05, lo: float = 0.2, hi: float = 1.0, common: tuple | None = None,
                seed: int = 0, device: str = "cpu", dtype=None, materialize: str = "numpy",
                ld: int | None = None, block_fn=None, compute_dtype=None) -> Instance:
    """Unit-diagonal empirical TPDM of a Pareto(2) factor model.

    A (n x groups, non-negative): each row loads U[lo, hi] on its own group
    and, with probability ``overlap``, U[lo, hi] on one other random group;
    ``common=(clo, chi)`` adds a common column with loadings U[clo, chi] on
    every row (the near-dominant common factor).  Rows are L2-normalised and
    permuted.  x_t = A z_t with z_j iid Pareto(alpha=2) (z = U^-1/2).  The
    top ``q`` fraction of samples by radius R = ||x||_2 are kept; with
    Omega the n_exc x n matrix of their angular parts x/R, the estimator is
    (n / n_exc) Omega^T Omega normalised to unit diagonal (Sec. 3.4).
    """
    torch = _torch()
    rng = _rng(seed, 2)
    base = np.repeat(np.arange(groups), int(math.ceil(n / groups)))[:n]
    ncol = groups + (1 if common is not None else 0)
    A = np.zeros((n, ncol))
    A[np.arange(n), base] = rng.uniform(lo, hi, size=n)
    extra = rng.random(n) < overlap
    other = (base + 1 + rng.integers(0, groups - 1, size=n)) % groups
    A[np.nonzero(extra)[0], other[extra]] = rng.uniform(lo, hi, size=int(extra.sum()))
    if common is not None:
        A[:, groups] = rng.uniform(common[0], common[1], size=n)
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    perm = rng.permutation(n)
    A = A[perm]
    labels = base[perm]
    n_exc = max(1, int(math.floor(q * T)))
    # draw the factor samples in chunks, keep only the radii first
    Z = rng.random((ncol, T)) ** -0.5
    At = torch.from_numpy(A).to(device=device, dtype=torch.float64)
    Zt = torch.from_numpy(Z).to(device=device, dtype=torch.float64)
    R2 = torch.zeros(T, dtype=torch.float64, device=device)
    for c0 in range(0, T, 2048):
        Xc = At @ Zt[:, c0:c0 + 2048]
        R2[c0:c0 + 2048] = (Xc * Xc).sum(dim=0)
    keep = torch.argsort(R2, descending=True, stable=True)[:n_exc]
    Xk = At @ Zt[:, keep]                      # n x n_exc
    W = Xk / torch.sqrt(R2[keep])[None, :]     # angular parts, columns = Omega rows
    S_t, norm2 = _gram_abs_unitdiag(W.cpu().numpy() if device == "cpu" else W.double().cpu().numpy(),
                                    n / n_exc, device, dtype or torch.float64, False, ld=ld,
                                    block_fn=block_fn, compute_dtype=compute_dtype)
    meta = {"T": T, "groups": groups, "n_exc": n_exc, "normS2_f64": norm2}
    if block_fn is not None:
        return Instance(S=None, n=n, kind="tpdm", seed=seed, perm=perm, labels=labels, meta=meta)
    return _finish(S_t, n, "tpdm", seed, perm, labels, meta, materialize)


def corr_factor(n: int = 100000, T: int = 500, sectors: int = 49, density: float = 0.1,
                market: tuple = (0.4, 0.8), sector_hi: float = 0.5, seed: int = 0,
                device: str = "cpu", dtype=None, materialize: str = "numpy",
                ld: int | None = None) -> Instance:
    """|Pearson correlation| of a 50-factor model with a dominant market factor.

    x = A z + e: market loadings U[market], ``sectors`` sector factors with
    loadings U[0, sector_hi] at ``density``, unit-variance Gaussian
    idiosyncratic noise, T samples, rows permuted, no shrinkage.
    """
    torch = _torch()
    rng = _rng(seed, 3)
    A = np.zeros((n, sectors + 1))
    A[:, 0] = rng.uniform(market[0], market[1], size=n)
    mask = rng.random((n, sectors)) < density
    A[:, 1:] = np.where(mask, rng.uniform(0.0, sector_hi, size=(n, sectors)), 0.0)
    perm = rng.permutation(n)
    A = A[perm]
    labels = np.argmax(A[:, 1:], axis=1)
    z = rng.standard_normal((sectors + 1, T))
    e = rng.standard_normal((n, T))
    X = A @ z + e
    Xc = X - X.mean(axis=1, keepdims=True)
    S_t, norm2 = _gram_abs_unitdiag(Xc, 1.0 / T, device, dtype or torch.float64, True, ld=ld)
    return _finish(S_t, n, "corr", seed, perm, labels, {"T": T, "normS2_f64": norm2}, materialize)


def planted_exact(n: int, k: int, density: float = 0.5, seed: int = 0):
    """A sparse non-negative H0 (n x k, float64) with S = H0 H0^T.

    Under the noiseless alpha=2 factor model the population TPDM is exactly
    a Gram matrix A A^T (Sec. 3.3), so S = H0 H0^T with H0 >= 0 is an exact
    SymNMF instance: f(H0) = 0.  Every row gets at least one non-zero.
    """
    rng = _rng(seed, 4)
    H0 = np.where(rng.random((n, k)) < density, rng.uniform(0.1, 1.0, size=(n, k)), 0.0)
    empty = ~(H0 > 0).any(axis=1)
    H0[np.nonzero(empty)[0], rng.integers(0, k, size=int(empty.sum()))] = rng.uniform(0.1, 1.0, size=int(empty.sum()))
    return H0, H0 @ H0.T


def init_uniform(n: int, k: int, hi: float = 0.1, seed: int = 0, stream: int = 0) -> np.ndarray:
    """H0 ~ U[0, hi] entrywise (float64), seeded by (seed, stream)."""
    return _rng(seed, 100 + int(stream)).uniform(0.0, hi, size=(n, k))


def init_scaled(mean_S: float, n: int, k: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    """H0 ~ U[0, sqrt(mean(S)/k)] (Sec. 4.4, "Initialization and seeds")."""
    return init_uniform(n, k, math.sqrt(mean_S / k), seed, stream)


def batch_specs(count: int = 64, nmin: int = 2000, nmax: int = 30000):
    """Per-instance (n, k, kind, seed) of the 64-instance batching workload.

    n ~ U{nmin..nmax} drawn from the instance seed, k = [8,16,32,64][i mod 4],
    even instances correlation, odd instances TPDM.
    """
    out = []
    for i in range(count):
        n = int(_rng(i, 5).integers(nmin, nmax + 1))
        out.append({"n": n, "k": [8, 16, 32, 64][i % 4], "kind": "corr" if i % 2 == 0 else "tpdm", "seed": i})
    return out
