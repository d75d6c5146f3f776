"""Pins of the spherical K-means oracle against what the paper and the
mathematics fix (Sec. 6 and its theorem on spherical K-means)."""
import itertools

import numpy as np
import pytest

from oracle import spkmeans_oracle as K


def _sym_unit(n, rng, lo=0.0, hi=1.0):
    A = rng.uniform(lo, hi, size=(n, n))
    S = (A + A.T) / 2.0
    np.fill_diagonal(S, 1.0)
    return S


def _labels_all_used(n, Kc, rng):
    lab = rng.integers(0, Kc, size=n)
    lab[:Kc] = np.arange(Kc)
    return rng.permutation(lab)


def test_objective_equals_theorem_form():
    """Theorem (Sec. 6): with the normalised-sum centroids,
    S_K = n - sum_k ||s_k||, s_k = sum of the member rows x_i."""
    rng = np.random.default_rng(0)
    for trial in range(10):
        n, Kc = int(rng.integers(5, 40)), int(rng.integers(2, 6))
        S = _sym_unit(n, rng)
        lab = _labels_all_used(n, Kc, rng)
        total = 0.0
        for k in range(Kc):
            s_k = np.zeros(n)
            for i in range(n):
                if lab[i] == k:
                    s_k += S[i] / np.sqrt(S[i] @ S[i])
            total += np.sqrt(s_k @ s_k)
        assert abs(K.objective(S, lab, Kc) - (n - total)) < 1e-12 * n


def test_lloyd_objective_never_increases():
    """J_{t+1} <= S_K(L_{t+1}) <= J_t: each Lloyd half-step can only lower
    the objective."""
    rng = np.random.default_rng(1)
    for trial in range(8):
        n, Kc = 60, int(rng.integers(2, 7))
        S = _sym_unit(n, rng)
        run = K.spkmeans(S, _labels_all_used(n, Kc, rng), Kc, max_iter=30, tol=0.0)
        J = np.array(run.J)
        assert np.all(np.diff(J) <= 1e-12 * n)
        lab = _labels_all_used(n, Kc, rng)
        for _ in range(5):
            new, Jt, _ = K.lloyd_step(S, lab, Kc)
            assert K.objective(S, new, Kc) <= Jt + 1e-12 * n
            assert Jt <= K.objective(S, lab, Kc) + 1e-12 * n
            lab = new


def test_brute_force_optimum_is_a_lloyd_fixed_point():
    """On 8 rows and 2 clusters the best of all 2^8 labelings (brute force on
    the theorem's form) is left unchanged by a Lloyd step."""
    rng = np.random.default_rng(2)
    for trial in range(4):
        n, Kc = 8, 2
        S = _sym_unit(n, rng, 0.0, 1.0)
        X = S / np.sqrt(np.sum(S * S, axis=1))[:, None]
        best, best_lab = -1.0, None
        for bits in itertools.product(range(Kc), repeat=n):
            lab = np.array(bits)
            if len(set(bits)) < Kc:
                continue
            v = sum(np.linalg.norm(X[lab == k].sum(axis=0)) for k in range(Kc))
            if v > best:
                best, best_lab = v, lab
        new, J, _ = K.lloyd_step(S, best_lab, Kc)
        assert np.array_equal(new, best_lab)
        assert abs(J - (n - best)) < 1e-12 * n


def test_planted_blocks_recovered():
    """Block-diagonal S (no similarity across blocks): from the true labels
    with 15% of them flipped, Lloyd returns the true partition."""
    rng = np.random.default_rng(3)
    Kc, m = 5, 30
    n = Kc * m
    S = np.zeros((n, n))
    for b in range(Kc):
        B = rng.uniform(0.5, 1.0, size=(m, m))
        S[b * m:(b + 1) * m, b * m:(b + 1) * m] = (B + B.T) / 2.0
    np.fill_diagonal(S, 1.0)
    perm = rng.permutation(n)
    S = S[np.ix_(perm, perm)]
    truth = (np.arange(n) // m)[perm]
    lab = truth.copy()
    flip = rng.choice(n, size=int(0.15 * n), replace=False)
    lab[flip] = (lab[flip] + 1 + rng.integers(0, Kc - 1, size=flip.size)) % Kc
    run = K.spkmeans(S, lab, Kc)
    assert run.converged
    assert np.array_equal(run.labels, truth)
    total = sum(np.linalg.norm(K.normalized_rows(S)[truth == k].sum(axis=0)) for k in range(Kc))
    assert abs(run.J[-1] - (n - total)) < 1e-10 * n


def test_scale_and_permutation_invariance():
    rng = np.random.default_rng(4)
    n, Kc = 50, 4
    S = _sym_unit(n, rng)
    lab = _labels_all_used(n, Kc, rng)
    new, J, _ = K.lloyd_step(S, lab, Kc)
    new2, J2, _ = K.lloyd_step(3.7 * S, lab, Kc)
    assert np.array_equal(new, new2) and abs(J - J2) < 1e-12 * n
    p = rng.permutation(n)
    new3, J3, _ = K.lloyd_step(S[np.ix_(p, p)], lab[p], Kc)
    assert np.array_equal(new3, new[p]) and abs(J - J3) < 1e-12 * n


def test_singleton_and_empty_clusters():
    """A row alone in its cluster has cosine 1 with it; an empty cluster has
    a zero centroid, hence cosine 0 with every row; ties go to the lowest
    index."""
    rng = np.random.default_rng(5)
    n, Kc = 20, 4
    S = _sym_unit(n, rng, 0.1, 1.0)
    lab = np.zeros(n, dtype=np.int64)
    lab[7] = 1            # singleton
    # cluster 2 and 3 empty
    cos = K.cosines(S, K.centroid_sums(S, lab, Kc))
    assert abs(cos[7, 1] - 1.0) < 1e-14
    assert np.all(cos[:, 2] == 0.0) and np.all(cos[:, 3] == 0.0)
    assert np.all(cos >= -1.0 - 1e-14) and np.all(cos <= 1.0 + 1e-14)
    assert list(K.first_argmax(np.array([[0.3, 0.7, 0.7], [0.0, 0.0, 0.0]]))) == [1, 0]


def test_stop_rule():
    """A fixed point stops after one iteration (no label changed); with
    tol = 1 the run stops at iteration 1 unless the objective rose."""
    rng = np.random.default_rng(6)
    n, Kc = 40, 3
    S = _sym_unit(n, rng)
    lab = _labels_all_used(n, Kc, rng)
    for _ in range(50):
        new, _, _ = K.lloyd_step(S, lab, Kc)
        if np.array_equal(new, lab):
            break
        lab = new
    run = K.spkmeans(S, lab, Kc)
    assert run.converged and len(run.J) == 1 and run.changed == [0]
    run = K.spkmeans(S, _labels_all_used(n, Kc, rng), Kc, tol=1.0)
    assert run.converged and len(run.J) <= 2
