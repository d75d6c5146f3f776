"""Pins of the dependence-matrix oracle (Sec. 3; appendix on the synthetic
matrices) against library routines and the mathematics."""
import numpy as np

from oracle import dependence_oracle as D


def test_abs_correlation_equals_numpy_corrcoef():
    rng = np.random.default_rng(0)
    for T, n in ((50, 7), (400, 33), (31, 60)):
        X = rng.standard_normal((T, n)) @ rng.uniform(0.0, 1.0, size=(n, n)) + 3.0
        ref = np.abs(np.corrcoef(X, rowvar=False))
        np.fill_diagonal(ref, 1.0)
        assert np.max(np.abs(D.abs_correlation(X) - ref)) < 1e-12


def test_correlation_invariances():
    """Shifting or positively scaling a variable, or reordering the
    observations, leaves |C| unchanged; a negative scale too (absolute value)."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((200, 12))
    S = D.abs_correlation(X)
    a = rng.uniform(-3.0, 3.0, size=12)
    b = rng.uniform(-5.0, 5.0, size=12)
    assert np.max(np.abs(D.abs_correlation(X * a + b) - S)) < 1e-12
    assert np.max(np.abs(D.abs_correlation(X[rng.permutation(200)]) - S)) < 1e-12


def test_unit_diagonal_symmetric_bounded_psd():
    """S is symmetric, unit-diagonal, in [0, 1]; the signed normalised Gram
    is positive semidefinite (Sec. 3)."""
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((80, 40))
    S = D.dependence(Y, center=True)
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == 1.0)
    assert np.all(S >= 0.0) and np.all(S <= 1.0 + 1e-15)
    G = D.gram(D.centred(Y))
    d = np.sqrt(np.diag(G))
    assert np.min(np.linalg.eigvalsh(G / np.outer(d, d))) > -1e-12


def test_tpdm_explicit_loops_and_rank():
    """The TPDM by explicit sums over the exceedances; rank <= n_exc
    (Sec. 3, empirical TPDM); the n / n_exc factor cancels."""
    rng = np.random.default_rng(3)
    n, n_exc = 9, 5
    W = rng.uniform(0.0, 1.0, size=(n_exc, n))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    S = D.tpdm(W)
    for i in range(n):
        for j in range(n):
            gij = sum(W[t, i] * W[t, j] for t in range(n_exc)) * n / n_exc
            gii = sum(W[t, i] ** 2 for t in range(n_exc)) * n / n_exc
            gjj = sum(W[t, j] ** 2 for t in range(n_exc)) * n / n_exc
            ref = 1.0 if i == j else abs(gij) / np.sqrt(gii * gjj)
            assert abs(S[i, j] - ref) < 1e-14
    assert np.max(np.abs(D.tpdm(W, n_scale=False) - S)) < 1e-14
    sgn = D.gram(W) / np.sqrt(np.outer(np.diag(D.gram(W)), np.diag(D.gram(W))))
    ev = np.linalg.eigvalsh(sgn)
    assert np.sum(ev > 1e-10) <= n_exc


def test_dependence_without_centring_is_cosine_similarity():
    """center=False gives the absolute cosine similarity of the columns."""
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((30, 6))
    S = D.dependence(Y, center=False)
    for i in range(6):
        for j in range(6):
            c = abs(Y[:, i] @ Y[:, j]) / (np.linalg.norm(Y[:, i]) * np.linalg.norm(Y[:, j]))
            assert abs(S[i, j] - (1.0 if i == j else c)) < 1e-14
