"""Plain FP64 CPU oracle for spherical K-means (Lloyd) on the rows of S.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA path.

What it computes (Sec. 6, "Clustering alternatives", spherical K-means and
its theorem; the algorithm is Lloyd's, as in Dhillon & Modha 2001 and
Hornik et al. 2012, which the paper cites):

* the observations are the rows s_i of S, normalised: x_i = s_i / ||s_i||;
* the centroid of cluster k is the normalised sum of its members,
  c_k = sum_{i in C_k} x_i,  c~_k = c_k / ||c_k||;
* the assignment step gives each row the cluster of largest cosine
  <x_i, c~_k>; the objective is S_K = sum_i (1 - <x_i, c~_{L(i)}>);
* one Lloyd iteration takes labels L_t to the centroids of L_t, then to the
  new labels L_{t+1}; J_t = sum_i (1 - max_k <x_i, c~_k>) is the objective
  of L_{t+1} against the centroids of L_t.

Readings where the paper is silent (also listed in the design notes):
* the run starts from caller-given labels (the paper's seeds do not say how
  it initialises);
* ties in the argmax go to the lowest cluster index;
* a cluster with no members (or a zero sum) has c~_k = 0, so every cosine
  with it is 0;
* the run stops after iteration t when no label changed, or when t >= 1 and
  the relative drop of the objective is at most tol,
  J_{t-1} - J_t <= tol * J_{t-1}  (tol = 1e-4, the paper's criterion);
* rows with ||s_i|| = 0 are not valid input (S has a unit diagonal).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def row_norms(S):
    """||s_i|| for every row of S, FP64."""
    S = np.asarray(S, dtype=np.float64)
    return np.sqrt(np.sum(S * S, axis=1))


def normalized_rows(S):
    """x_i = s_i / ||s_i|| (Sec. 6, spherical K-means)."""
    S = np.asarray(S, dtype=np.float64)
    return S / row_norms(S)[:, None]


def centroid_sums(S, labels, K):
    """c_k = sum of the normalised rows with label k, as the columns of an
    n x K matrix (S is symmetric, so rows and columns coincide)."""
    X = normalized_rows(S)
    n = X.shape[0]
    C = np.zeros((n, K))
    for k in range(K):
        members = np.flatnonzero(np.asarray(labels) == k)
        if members.size:
            C[:, k] = X[members].sum(axis=0)
    return C


def cosines(S, C):
    """<x_i, c~_k> for every row i and cluster k; c~_k = 0 where ||c_k|| = 0."""
    X = normalized_rows(S)
    norms = np.sqrt(np.sum(C * C, axis=0))
    Cn = np.zeros_like(C)
    nz = norms > 0
    Cn[:, nz] = C[:, nz] / norms[nz]
    return X @ Cn


def first_argmax(scores):
    """Index of the largest entry per row, lowest index on ties."""
    return np.argmax(scores, axis=1).astype(np.int64)


def lloyd_step(S, labels, K):
    """One Lloyd iteration: centroids of ``labels``, then the assignment.
    Returns (new labels, J, cosines)."""
    C = centroid_sums(S, labels, K)
    cos = cosines(S, C)
    new = first_argmax(cos)
    J = float(np.sum(1.0 - cos[np.arange(cos.shape[0]), new]))
    return new, J, cos


def objective(S, labels, K):
    """S_K = sum_i (1 - <x_i, c~_{L(i)}>) with the centroids of ``labels``."""
    cos = cosines(S, centroid_sums(S, labels, K))
    lab = np.asarray(labels)
    return float(np.sum(1.0 - cos[np.arange(cos.shape[0]), lab]))


@dataclass
class Run:
    labels: np.ndarray
    J: list = field(default_factory=list)        # J_t per iteration
    changed: list = field(default_factory=list)  # labels changed in iteration t
    converged: bool = False


def spkmeans(S, labels0, K, max_iter=100, tol=1e-4):
    """Lloyd iterations from ``labels0`` until the stopping reading above."""
    lab = np.asarray(labels0, dtype=np.int64).copy()
    run = Run(labels=lab)
    for t in range(max_iter):
        new, J, _ = lloyd_step(S, lab, K)
        ch = int(np.sum(new != lab))
        run.J.append(J)
        run.changed.append(ch)
        lab = new
        if ch == 0 or (t >= 1 and run.J[t - 1] - J <= tol * run.J[t - 1]):
            run.converged = True
            break
    run.labels = lab
    return run
