"""Plain FP64 CPU oracle for the dependence matrices that are the solver's
input (Sec. 3: correlation matrices; the TPDM estimator; the appendix on
the synthetic matrices).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA path.

Both inputs are unit-diagonal normalisations of a Gram matrix of n
variables over T observations, Y in R^{T x n}:
* absolute Pearson correlation: Y = the observations with each column
  centred; C_ij = Cov(X_i, X_j) / (sigma_i sigma_j) = G_ij / sqrt(G_ii G_jj)
  with G = Y^T Y (the 1/(T-1) factors cancel); S = |C|;
* TPDM: Y = Omega, the angular components of the exceedances (rows on the
  unit sphere); Sigma~ = (n / n_exc) Omega^T Omega and the input is its
  unit-diagonal normalisation D^-1/2 Sigma~ D^-1/2, D = diag(Sigma~), in
  which the factor n / n_exc cancels.
So one routine covers both: S_ij = |G_ij| / sqrt(G_ii G_jj), G = Y^T Y,
with the columns of Y centred first for the correlation.
"""
from __future__ import annotations

import numpy as np


def centred(Y):
    """Columns of Y minus their means."""
    Y = np.asarray(Y, dtype=np.float64)
    return Y - Y.mean(axis=0, keepdims=True)


def gram(Y):
    """G = Y^T Y (n x n)."""
    Y = np.asarray(Y, dtype=np.float64)
    return Y.T @ Y


def unit_diagonal_abs(G):
    """|G_ij| / sqrt(G_ii G_jj); the diagonal is 1."""
    G = np.asarray(G, dtype=np.float64)
    d = np.sqrt(np.diag(G))
    S = np.abs(G) / np.outer(d, d)
    np.fill_diagonal(S, 1.0)
    return S


def abs_correlation(X):
    """S = |C|, C the Pearson sample correlation of the columns of X (T x n)."""
    return unit_diagonal_abs(gram(centred(X)))


def tpdm(Omega, n_scale=True):
    """Unit-diagonal TPDM from the n_exc x n matrix of exceedance angles;
    n_scale applies the (n / n_exc) factor before normalising (it cancels)."""
    Omega = np.asarray(Omega, dtype=np.float64)
    n_exc, n = Omega.shape
    G = gram(Omega)
    if n_scale:
        G = (n / n_exc) * G
    return unit_diagonal_abs(G)


def dependence(Y, center):
    """The routine both matrices reduce to (see the module docstring)."""
    return unit_diagonal_abs(gram(centred(Y) if center else Y))
