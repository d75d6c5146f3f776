"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, brute force on a tiny input, a value the paper prints,
or a published test vector.  No GPU is used.
"""
import math
import os

import numpy as np
import pytest

import gen
from oracle import symnmf_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_problem(n=40, k=4, seed=0):
    inst = gen.tpdm_groups(n=n, groups=k, T=800, q=0.1, seed=seed)
    H0 = gen.init_scaled(float(inst.S.mean()), n, k, seed=seed)
    return inst.S, H0


# ---------------------------------------------------------------- objective
def test_trace_identity_equals_explicit_objective():
    """Eq. 2 equals Eq. 1 (expanded Frobenius norm) to rounding."""
    for n, k in [(7, 1), (64, 5), (300, 8)]:
        inst = gen.corr_planted(n=n, groups=max(1, k), T=400, seed=n)
        H = gen.init_uniform(n, k, 0.3, seed=n)
        fe = O.objective_explicit(inst.S, H)
        ft = O.objective_trace(inst.S, H)
        assert abs(fe - ft) <= 1e-12 * max(1.0, fe, float(np.sum(inst.S ** 2)))


def test_objective_by_brute_force_sum():
    """Eq. 1 against a pure-Python double loop over all entries."""
    rng = np.random.default_rng(3)
    n, k = 6, 2
    X = rng.random((n, n))
    S = (X + X.T) / 2
    H = rng.random((n, k))
    tot = 0.0
    for i in range(n):
        for j in range(n):
            r = S[i, j] - sum(H[i, c] * H[j, c] for c in range(k))
            tot += r * r
    assert abs(O.objective_explicit(S, H) - tot) < 1e-12
    assert abs(O.objective_trace(S, H) - tot) < 1e-12


# ----------------------------------------------------------------- gradient
def test_gradient_matches_central_finite_differences():
    """grad f = 4(H H^T H - S H) against central differences of Eq. 1."""
    rng = np.random.default_rng(1)
    n, k = 12, 3
    X = rng.random((n, n))
    S = (X + X.T) / 2
    H = rng.random((n, k))
    G = O.gradient(S, H)
    h = 1e-6
    fd = np.zeros_like(H)
    for i in range(n):
        for c in range(k):
            Hp, Hm = H.copy(), H.copy()
            Hp[i, c] += h
            Hm[i, c] -= h
            fd[i, c] = (O.objective_explicit(S, Hp) - O.objective_explicit(S, Hm)) / (2 * h)
    assert np.linalg.norm(G - fd) / np.linalg.norm(fd) < 1e-7


def test_gradient_euler_identity():
    """f = q + r with q = -2 tr(H^T S H) of degree 2 and r = ||H^T H||^2 of
    degree 4; Euler's theorem gives <grad f, H> = 2q + 4r."""
    S, H = _small_problem(50, 5, seed=2)
    G = O.gradient(S, H)
    q = -2.0 * np.einsum("ic,ij,jc->", H, S, H)
    r = np.einsum("ic,id,jc,jd->", H, H, H, H)
    lhs = float(np.sum(G * H))
    assert abs(lhs - (2 * q + 4 * r)) <= 1e-11 * abs(2 * q) + 1e-11 * abs(4 * r)


def test_gradient_is_row_local_formula():
    """Row i of the gradient depends on S only through row i of S."""
    S, H = _small_problem(30, 3, seed=4)
    G = O.gradient(S, H)
    S2 = S.copy()
    S2[5, :] = 0.0
    S2[:, 5] = S[:, 5]  # keep column 5 (it feeds other rows)
    G2 = O.gradient(S2, H)
    changed = np.nonzero(np.abs(G - G2).max(axis=1) > 0)[0]
    assert list(changed) == [5]


# ----------------------------------------------------- planted exact, zero
def test_planted_exact_factorisation():
    """S = H0 H0^T with H0 >= 0 (Sec. 3.3: the noiseless TPDM is A A^T):
    f(H0) = 0, grad f(H0) = 0, KKT holds, and AdaGrad from a perturbed H0
    drives E to <= 1e-10."""
    H0, S = gen.planted_exact(60, 4, seed=1)
    normS2 = float(np.sum(S * S))
    assert abs(O.objective_trace(S, H0)) <= 1e-12 * normS2
    G = O.gradient(S, H0)
    assert np.abs(G).max() <= 1e-12 * np.abs(S @ H0).max()
    assert O.kkt_norm(H0, G) <= 1e-13
    Hs = H0 + np.random.default_rng(0).uniform(0, 0.05, H0.shape)
    hp = O.HParams.paper(O.ADAGRAD)
    hp.eta = 0.05
    hp.tau_g = 1e-14         # run on past the default gate
    s = O.Solver(S, Hs, hp)
    s.run(1500)
    assert O.objective_explicit(S, s.H) / normS2 <= 1e-10


def test_zero_is_a_fixed_point_of_every_method():
    """grad f(0) = 0, so H = 0 never moves; E(0) = 1 fails the loss gate."""
    S, _ = _small_problem(64, 4, seed=5)
    Z = np.zeros((64, 4))
    assert np.all(O.gradient(S, Z) == 0)
    assert O.objective_trace(S, Z) / float(np.sum(S * S)) == 1.0
    for m in range(5):
        hp = O.HParams.paper(m)
        hp.block_rows = 16
        s = O.Solver(S, Z, hp)
        recs = s.run(30)
        assert np.all(s.H == 0)
        assert recs[0].E == 1.0 and not any(r.converged for r in recs)


def test_rank_one_closed_form():
    """k = 1 and S = h h^T with h > 0: the unique non-negative optimum is h."""
    rng = np.random.default_rng(7)
    h = rng.uniform(0.2, 1.0, size=(25, 1))
    S = h @ h.T
    hp = O.HParams.paper(O.ADAGRAD)
    hp.eta = 0.1
    hp.tau_g = 1e-14
    s = O.Solver(S, np.full((25, 1), 0.5), hp)
    s.run(4000)
    assert np.max(np.abs(s.H - h)) < 1e-6


# ------------------------------------------------------- first-step forms
def test_first_adagrad_step_closed_form():
    """With G_0 = 0, G_1 = g0^2 and H_1 = [H0 - eta g0 / (|g0| + eps)]_+."""
    S, H0 = _small_problem(40, 4, seed=8)
    hp = O.HParams.paper(O.ADAGRAD)
    s = O.Solver(S, H0, hp)
    s.step()
    g0 = O.gradient(S, H0)
    expect = np.maximum(H0 - hp.eta * g0 / (np.abs(g0) + hp.eps), 0.0)
    assert np.allclose(s.H, expect, rtol=1e-14, atol=1e-15)


def test_first_rmsprop_step_closed_form():
    """v_1 = (1-a) g0^2, m_1 = eta g0 / (sqrt(1-a)|g0| + eps), H_1 = [H0 - m_1]_+."""
    S, H0 = _small_problem(40, 4, seed=9)
    hp = O.HParams.paper(O.RMSPROP)
    s = O.Solver(S, H0, hp)
    s.step()
    g0 = O.gradient(S, H0)
    m1 = hp.eta * g0 / (math.sqrt(1 - hp.alpha) * np.abs(g0) + hp.eps)
    assert np.allclose(s.H, np.maximum(H0 - m1, 0.0), rtol=1e-13, atol=1e-15)


def _gradient_by_loops(S, H):
    """g_ic = 4 (sum_d H_id (H^T H)_dc - sum_j S_ij H_jc), entry by entry."""
    n, k = H.shape
    gram = [[sum(H[j, c] * H[j, d] for j in range(n)) for d in range(k)] for c in range(k)]
    g = np.zeros_like(H)
    for i in range(n):
        for c in range(k):
            hg = sum(H[i, d] * gram[d][c] for d in range(k))
            sh = sum(S[i, j] * H[j, c] for j in range(n))
            g[i, c] = 4 * (hg - sh)
    return g


def test_rmsprop_three_steps_by_hand():
    """RMSprop (appendix, Family 3) written out entry by entry for three
    steps, so the momentum carry mu * m_{t-1} and the EMA of g^2 are both
    exercised (m_0 = v_0 = 0 hides them in the first step):
        v_t = a v_{t-1} + (1 - a) g_t^2
        m_t = mu m_{t-1} + eta g_t / (sqrt(v_t) + eps)
        H_{t+1} = [H_t - m_t]_+"""
    S, H0 = _small_problem(16, 2, seed=19)
    hp = O.HParams.paper(O.RMSPROP)
    hp.eta = 0.02                 # small enough that no entry is clamped to 0
    s = O.Solver(S, H0, hp)
    H = H0.copy()
    v = np.zeros_like(H)
    m = np.zeros_like(H)
    n, k = H.shape
    for step in range(3):
        s.step()
        g = _gradient_by_loops(S, H)
        for i in range(n):
            for c in range(k):
                v[i, c] = hp.alpha * v[i, c] + (1.0 - hp.alpha) * g[i, c] ** 2
                m[i, c] = hp.mu * m[i, c] + hp.eta * g[i, c] / (math.sqrt(v[i, c]) + hp.eps)
                H[i, c] = max(H[i, c] - m[i, c], 0.0)
        assert np.allclose(s.A, v, rtol=1e-12, atol=1e-15), step
        assert np.allclose(s.M, m, rtol=1e-12, atol=1e-15), step
        assert np.allclose(s.H, H, rtol=1e-12, atol=1e-15), step
    # the carried momentum is a real part of step 3 (not a vanishing term)
    assert np.max(np.abs(hp.mu * m)) > 1e-3 * np.max(np.abs(H))
    assert np.all(H > 0)


def test_second_adagrad_step_by_hand():
    """Two steps written out with plain loops over entries."""
    S, H0 = _small_problem(20, 2, seed=10)
    hp = O.HParams.paper(O.ADAGRAD)
    hp.eta = 0.3
    s = O.Solver(S, H0, hp)
    s.step()
    s.step()
    H = H0.copy()
    A = np.zeros_like(H)
    for _ in range(2):
        g = np.zeros_like(H)
        n, k = H.shape
        for i in range(n):
            for c in range(k):
                hg = sum(H[i, d] * sum(H[j, d] * H[j, c] for j in range(n)) for d in range(k))
                sh = sum(S[i, j] * H[j, c] for j in range(n))
                g[i, c] = 4 * (hg - sh)
        A = A + g * g
        H = np.maximum(H - hp.eta * g / (np.sqrt(A) + hp.eps), 0.0)
    assert np.allclose(s.H, H, rtol=1e-12, atol=1e-14)


# ------------------------------------------------ paper-stated equivalences
def test_row_gradient_with_all_rows_is_the_full_gradient():
    """Row-Stochastic with |I| = n is full-batch (Sec. 5.1)."""
    S, H0 = _small_problem(70, 3, seed=11)
    hp = O.HParams.paper(O.ROW_SVRG)
    hp.row_frac, hp.block_rows = 1.0, 16
    s = O.Solver(S, H0, hp)
    g = s.row_gradient(t=3)
    assert len(s.last_I) == 70
    assert np.allclose(g, O.gradient(S, H0), rtol=1e-13, atol=1e-13)


def test_block_gradient_at_phi_one_is_the_full_gradient():
    """With I = J = [n]: 2 R H + 2 R^T H = 4(H H^T H - S H), so the block
    step at phi = 1 is full-batch AdaGrad (Sec. 5.1)."""
    S, H0 = _small_problem(70, 3, seed=12)
    hp = O.HParams.paper(O.BLOCK_SVRG)
    hp.block_rows = 16
    s = O.Solver(S, H0, hp)
    s.ctrl.phi = 1.0
    g = s.block_gradient(t=5)
    assert len(s.last_I) == 70 and len(s.last_J) == 70
    assert np.allclose(g, O.gradient(S, H0), rtol=1e-12, atol=1e-12)


def test_block_gradient_pieces_by_loops():
    """g_i = 2 sum_{j in J} (h_i.h_j - S_ij) h_j for i in I, plus the J side,
    snapshot elsewhere; the entry-wise form of the appendix formula."""
    S, H0 = _small_problem(48, 2, seed=13)
    hp = O.HParams.paper(O.BLOCK_SVRG)
    hp.block_rows = 8
    s = O.Solver(S, H0, hp)
    s.ctrl.phi = 0.3
    s.mu = np.random.default_rng(0).random(H0.shape)
    g = s.block_gradient(t=7)
    I, J = set(s.last_I.tolist()), set(s.last_J.tolist())
    assert I != J
    exp = s.mu.copy()
    for i in range(48):
        if i in I or i in J:
            exp[i] = 0.0
        if i in I:
            for j in J:
                exp[i] += 2 * (H0[i] @ H0[j] - S[i, j]) * H0[j]
        if i in J:
            for j in I:
                exp[i] += 2 * (H0[j] @ H0[i] - S[j, i]) * H0[j]
    assert np.allclose(g, exp, rtol=1e-12, atol=1e-12)


def test_row_gradient_partial_fraction_by_loops():
    """Row-Stochastic SVRG at |I| < n (Sec. 5.1; appendix): sampled rows get
    the exact row gradient 4 (h_i (H^T H) - S_i H), every other row keeps
    the snapshot mu_i.  The row set is a union of whole blocks, drawn as
    ceil(frac n) rows rounded up to blocks."""
    S, H0 = _small_problem(48, 2, seed=20)
    hp = O.HParams.paper(O.ROW_SVRG)
    hp.row_frac, hp.block_rows = 0.4, 8
    s = O.Solver(S, H0, hp)
    s.mu = np.random.default_rng(1).random(H0.shape) - 0.5
    g = s.row_gradient(t=7)
    I = set(s.last_I.tolist())
    # ceil(0.4 * 48) = 20 rows -> 3 blocks of 8 = 24 rows, whole blocks
    assert len(I) == 24 and s.last_J is None
    assert all({b * 8 + r for r in range(8)} <= I for b in {i // 8 for i in I})
    full = _gradient_by_loops(S, H0)
    for i in range(48):
        want = full[i] if i in I else s.mu[i]
        assert np.allclose(g[i], want, rtol=1e-12, atol=1e-13), i
    # the two parts really differ, so a wrong branch cannot pass by accident
    assert min(np.abs(full[i] - s.mu[i]).max() for i in range(48)) > 1e-6


def test_full_pass_schedule_and_snapshot_refresh():
    """Stochastic methods take a full pass at t % s == 0 or t % delta == 0
    (and Block-SVRG whenever phi = 1); that pass evaluates f, E and the KKT
    norm at H_t and refreshes the snapshot mu = grad f(H_t).  Sampled
    iterations leave mu unchanged and report no objective."""
    S, H0 = _small_problem(48, 2, seed=21)
    for method, extra in [(O.ROW_SVRG, {"row_frac": 0.5}), (O.BLOCK_SVRG, {"phi0": 0.25})]:
        hp = O.HParams.paper(method)
        hp.eta, hp.block_rows, hp.snapshot_period, hp.check_interval = 0.05, 8, 3, 10
        hp.tau_g = 1e-12                   # no convergence, phi never grows here
        for a, b in extra.items():
            setattr(hp, a, b)
        s = O.Solver(S, H0, hp)
        normS2 = float(np.sum(S * S))
        for t in range(32):
            H_t, mu_prev = s.H.copy(), s.mu.copy()
            rec = s.step()
            assert rec.t == t
            assert rec.full == (t % 3 == 0 or t % 10 == 0), (method, t)
            if rec.full:
                assert np.allclose(s.mu, _gradient_by_loops(S, H_t), rtol=1e-12, atol=1e-13)
                f = float(np.sum((S - H_t @ H_t.T) ** 2))
                assert math.isclose(rec.E, f / normS2, rel_tol=1e-10)
            else:
                assert np.array_equal(s.mu, mu_prev)
                assert rec.E != rec.E          # NaN: no objective on a sampled step
        assert s.ctrl.phi == hp.phi0 if method == O.BLOCK_SVRG else True
    # Block-SVRG at phi = 1 is full at every iteration
    hp = O.HParams.paper(O.BLOCK_SVRG)
    hp.phi0, hp.snapshot_period = 1.0, 3
    s = O.Solver(S, H0, hp)
    assert all(s.step().full for _ in range(7))


def test_stochastic_methods_at_full_fraction_equal_adagrad():
    """Row-SVRG at |I|/n = 1 and Block-SVRG at phi0 = 1 run AdaGrad."""
    S, H0 = _small_problem(64, 4, seed=14)
    base = O.Solver(S, H0, O.HParams.paper(O.ADAGRAD))
    base.run(40)
    for m, kw in [(O.ROW_SVRG, {"row_frac": 1.0}), (O.BLOCK_SVRG, {"phi0": 1.0})]:
        hp = O.HParams.paper(m)
        for a, b in kw.items():
            setattr(hp, a, b)
        s = O.Solver(S, H0, hp)
        s.run(40)
        assert np.array_equal(s.H, base.H)


def test_piecewise_without_reset_is_adagrad():
    """Piecewise equals AdaGrad while no reset fires (Sec. 5.1)."""
    S, H0 = _small_problem(64, 4, seed=15)
    hp_a = O.HParams.paper(O.ADAGRAD)
    hp_a.eta = 1.0
    a = O.Solver(S, H0, hp_a)
    a.run(120)
    hp_p = O.HParams.paper(O.PIECEWISE)
    hp_p.c_r = 1e30          # margin gate never passes
    p = O.Solver(S, H0, hp_p)
    p.run(120)
    assert p.ctrl.resets == 0
    assert np.array_equal(p.H, a.H)


# ------------------------------------------------------------- symmetries
def test_column_permutation_equivariance():
    """(H Pi)(H Pi)^T = H H^T (Sec. 2): the solve from H0 Pi is the solve
    from H0 with columns permuted."""
    S, H0 = _small_problem(50, 5, seed=16)
    pi = np.array([3, 0, 4, 1, 2])
    for m in (O.ADAGRAD, O.RMSPROP):
        a = O.Solver(S, H0, O.HParams.paper(m))
        a.run(60)
        b = O.Solver(S, H0[:, pi], O.HParams.paper(m))
        b.run(60)
        assert np.allclose(b.H, a.H[:, pi], rtol=1e-9, atol=1e-12)


def test_row_permutation_equivariance():
    """Relabelling the variables (P S P^T, P H0) relabels the solution."""
    S, H0 = _small_problem(50, 3, seed=17)
    p = np.random.default_rng(5).permutation(50)
    a = O.Solver(S, H0, O.HParams.paper(O.ADAGRAD))
    a.run(60)
    b = O.Solver(S[np.ix_(p, p)], H0[p], O.HParams.paper(O.ADAGRAD))
    b.run(60)
    assert np.allclose(b.H, a.H[p], rtol=1e-9, atol=1e-12)


# ------------------------------------------------------ stopping rule (AND)
def test_tau_g_scaled_values_printed_in_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tau_g_scaled.txt")) if l[0] != "#"]
    for n, v in rows:
        assert math.isclose(O.tau_g_default(int(n)), float(v), rel_tol=1e-12)


def test_stopping_rule_truth_table():
    hp = O.HParams()
    n = 10000
    c = O.Ctrl(E0=1.0, E_prev=0.05, have_prev=True)
    # all three criteria hold
    assert O.stopping_rule(c, hp, n, 100, 0.05, 5e-5)[0]
    # loss gate fails
    c2 = O.Ctrl(E0=1.0, E_prev=0.2, have_prev=True)
    assert not O.stopping_rule(c2, hp, n, 100, 0.2, 5e-5)[0]
    # KKT fails
    assert not O.stopping_rule(c, hp, n, 100, 0.05, 2e-4)[0]
    # still descending: (E_prev - E)/E0 = 1e-3 >= 1e-5
    c3 = O.Ctrl(E0=1.0, E_prev=0.051, have_prev=True)
    assert not O.stopping_rule(c3, hp, n, 100, 0.05, 5e-5)[0]
    # warm-up suppresses stagnation before t = 50
    assert not O.stopping_rule(c, hp, n, 40, 0.05, 5e-5)[1]
    assert O.stopping_rule(c, hp, n, 50, 0.05, 5e-5)[1]
    # no previous check -> no stagnation
    assert not O.stopping_rule(O.Ctrl(E0=1.0), hp, n, 100, 0.05, 5e-5)[1]


def test_kkt_at_convergence():
    """At a converged AdaGrad solve the KKT conditions of Eq. 5 hold to the
    gate: H >= 0, grad >= -tol on the boundary, |H * grad| small."""
    inst = gen.tpdm_groups(n=128, groups=4, T=2000, q=0.05, seed=3)
    H0 = gen.init_scaled(float(inst.S.mean()), 128, 4, seed=3)
    hp = O.HParams.paper(O.ADAGRAD)
    s = O.Solver(inst.S, H0, hp)
    recs = s.run(5000)
    assert recs[-1].converged
    G = O.gradient(inst.S, s.H)
    tau = O.tau_g_default(128) * 128 * 4
    assert np.all(s.H >= 0)
    assert np.all(G[s.H == 0] >= -tau)
    assert np.linalg.norm(s.H * G) <= tau * np.abs(s.H).max()
    assert O.kkt_norm(s.H, G) < O.tau_g_default(128)


def test_projected_gradient_cases():
    H = np.array([[0.0, 0.0, 1.0, 2.0]])
    G = np.array([[-3.0, 4.0, -5.0, 6.0]])
    assert np.array_equal(O.projected_gradient(H, G), [[-3.0, 0.0, -5.0, 6.0]])


# ---------------------------------------- piecewise and adaptgrow control
def _stagnating_solver(method, **kw):
    S, H0 = _small_problem(64, 4, seed=18)
    hp = O.HParams.paper(method)
    hp.eta = 1e-7            # E barely moves: every post-warm-up check stagnates
    hp.tau_g = 1e-9
    for a, b in kw.items():
        setattr(hp, a, b)
    return O.Solver(S, H0, hp)


def test_piecewise_reset_formula_and_self_termination():
    s = _stagnating_solver(O.PIECEWISE, c=10.0, c_r=10.0)
    reset_at = None
    while s.ctrl.t <= 50:
        rec = s.step()
        if rec.reset:
            reset_at = rec.t
            g = s.g
            med = O.lower_median(g * g)
            assert np.array_equal(s.A, np.maximum(10.0 * g * g, 10.0 * med))
    assert reset_at == 50 and s.ctrl.resets == 1 and s.ctrl.cooldown
    # cooldown lasts until sum(G) doubles; afterwards the next stagnating
    # check finds no loss reduction and disables resets for good
    post = s.ctrl.sumA_post
    for _ in range(400):
        s.step()
        if not s.ctrl.cooldown:
            break
    assert float(np.sum(s.A)) >= 2 * post or not s.ctrl.cooldown
    for _ in range(200):
        s.step()
    assert s.ctrl.resets == 1 and not s.ctrl.resets_enabled


def test_adaptgrow_doubles_phi_after_three_stagnating_checks():
    s = _stagnating_solver(O.BLOCK_SVRG, phi0=0.25, block_rows=8, snapshot_period=3)
    phis = {}
    for _ in range(101):
        rec = s.step()
        if rec.check:
            phis[rec.t] = s.ctrl.phi
    # checks 50, 60, 70 stagnate -> grow at 70; 80, 90, 100 -> grow at 100
    assert phis[60] == 0.25 and phis[70] == 0.5 and phis[90] == 0.5 and phis[100] == 1.0


# ------------------------------------------------------------- sampling
def test_splitmix64_published_vectors():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt")) if l[0] != "#"]
    assert O.splitmix64_sequence(0, 4) == vals


def test_sample_blocks_valid_and_uniform():
    nb, m = 10, 3
    counts = np.zeros(nb)
    for t in range(3000):
        b = O.sample_blocks(42, t, 1, nb, m)
        assert len(b) == m and len(set(b)) == m and b == sorted(b)
        assert all(0 <= x < nb for x in b)
        counts[b] += 1
    expect = 3000 * m / nb
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    assert chi2 < 30.0          # 9 dof; p ~ 4e-4
    assert O.sample_blocks(42, 5, 1, nb, nb) == list(range(nb))


def test_sample_count_rounds_up_to_blocks():
    assert O.sample_count(0.5, 1000, 128) == 4          # 500 rows -> 4 blocks
    assert O.sample_count(math.sqrt(0.75), 300000, 4096) == 64
    assert O.sample_count(1.0, 1000, 128) == 8


# ------------------------------------------------------- column matching
def test_hungarian_equals_brute_force():
    rng = np.random.default_rng(9)
    for k in range(1, 8):
        for _ in range(5):
            C = rng.random((k, k))
            perm = O.hungarian(C)
            best_perm, best = O.brute_force_assignment(C)
            assert abs(sum(C[i, perm[i]] for i in range(k)) - best) < 1e-12


def test_match_columns_recovers_permutation():
    rng = np.random.default_rng(10)
    H = rng.random((30, 6))
    pi = rng.permutation(6)
    assert np.array_equal(O.match_columns(H[:, pi], H), H)
    assert O.factor_error(H[:, pi], H) == 0.0


def test_lower_median():
    assert O.lower_median([3.0, 1.0, 2.0]) == 2.0
    assert O.lower_median([4.0, 1.0, 3.0, 2.0]) == 2.0
    x = np.random.default_rng(0).random(1001)
    assert O.lower_median(x) == float(np.median(x))


# ------------------------------------------------------------ FP8 storage
def test_e4m3_round_matches_torch_float8():
    """The E4M3 rounding against torch's float8_e4m3fn conversion (a library
    routine) on values spread over every binade and the subnormals."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(0, 448, 20000), 2.0 ** rng.uniform(-12, 8.8, 20000),
                        np.arange(0, 449, 0.0625)])
    x = x[x <= 448.0]
    ours = O.e4m3_round(x)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).double().numpy()
    x32 = torch.tensor(x, dtype=torch.float32).double().numpy()
    ours32 = O.e4m3_round(x32)
    assert np.array_equal(ours32, ref)


def test_e4m3_grid_facts():
    """Format facts: 448 is the largest value, 2^-9 the smallest subnormal,
    ties go to the even mantissa."""
    assert O.e4m3_round(448.0) == 448.0
    assert O.e4m3_round(2.0 ** -9) == 2.0 ** -9
    assert O.e4m3_round(2.0 ** -10) == 0.0          # tie between 0 and 2^-9 -> even (0)
    assert O.e4m3_round(1.0625) == 1.0              # tie -> even mantissa
    assert O.e4m3_round(1.1875) == 1.25
    grid = np.concatenate([[0.0], 2.0 ** np.linspace(-10, np.log2(448.0), 400001)])
    assert len(np.unique(O.e4m3_round(grid))) == 127   # 2^7 codes minus NaN, incl. 0


def test_tile_scale_power_of_two_bound():
    for amax in [1e-7, 0.3, 1.0, 448.0 / 1024, 448.0 / 1024 * 1.0000001, 7.0]:
        sc = O.tile_scale(amax)
        assert math.log2(sc) == round(math.log2(sc))
        assert amax / sc <= 448.0 and amax / sc > 224.0
    assert O.tile_scale(0.0) == 1.0


def test_quantize_dequantize_error_bound():
    """Relative error of each quantised entry is at most 2^-4 (3 mantissa
    bits, round to nearest) in the normal range of its tile."""
    inst = gen.tpdm_groups(n=300, groups=6, T=1200, q=0.05, seed=4)
    q, sc = O.quantize_fp8(inst.S)
    D = O.dequantize_fp8(q, sc)
    big = inst.S > 1e-2
    assert np.all(np.abs(D[big] - inst.S[big]) <= 2.0 ** -4 * inst.S[big])
    assert np.all(np.abs(q) <= 448.0)


def test_gradient_rows_is_the_full_gradient_restricted():
    inst = gen.tpdm_groups(n=260, groups=5, T=1100, q=0.05, seed=9)
    H = gen.init_scaled(float(inst.S.mean()), 260, 6, seed=9)
    rows = np.array([0, 7, 128, 259])
    G = O.gradient(inst.S, H)
    np.testing.assert_allclose(O.gradient_rows(inst.S[rows], H, rows), G[rows], rtol=1e-13, atol=1e-12)


def test_hparams_match_the_printed_anchors():
    """Golden values: tests/golden/hparams_anchors.txt (appendix, Family 3;
    Sec. 5.1 for Piecewise AdaGrad; Sec. 5.1 and the Phase-2 configuration
    table for ADMM's penalty)."""
    names = {"adagrad": O.ADAGRAD, "rmsprop": O.RMSPROP, "piecewise": O.PIECEWISE,
             "admm": O.ADMM}
    path = os.path.join(os.path.dirname(__file__), "golden", "hparams_anchors.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 7
    for method, param, value in rows:
        assert getattr(O.HParams.paper(names[method]), param) == float(value)


def test_blocks_to_rows_example():
    assert list(O.blocks_to_rows([0, 2], 4, 10)) == [0, 1, 2, 3, 8, 9]
    assert list(O.blocks_to_rows([1], 4, 10)) == [4, 5, 6, 7]
    assert len(O.blocks_to_rows([], 4, 10)) == 0


def test_comparison_helpers():
    # ||(3,4) - (0,0)|| / ||(0,0)|| falls back to the absolute norm 5
    assert O.rel_err([3.0, 4.0], [0.0, 0.0]) == 5.0
    assert abs(O.rel_err([1.0, 1.0], [1.0, 2.0]) - 1.0 / math.sqrt(5.0)) < 1e-15
    rng = np.random.default_rng(3)
    H = rng.random((20, 4))
    assert O.factor_error(H[:, [2, 0, 3, 1]], H) < 1e-15
    A = np.array([[0.0, 1.0], [2.0, 0.0]])
    B = np.array([[0.0, 0.0], [2.0, 3.0]])
    assert O.boundary_disagreement(A, B) == 2


# ------------------------------------------------------------ ADMM (Family 6)
def test_admm_planted_solution_is_a_fixed_point():
    """At S = W0 W0^T with U = 0: S W0 = W0 G, so the H-update returns W0,
    W = [W0]_+ = W0 and U stays 0."""
    W0, S = gen.planted_exact(60, 4, seed=2)
    s = O.Solver(S, W0, O.HParams.paper(O.ADMM))
    s.step()
    np.testing.assert_allclose(s.H, W0, rtol=0, atol=1e-10)
    assert np.max(np.abs(s.A)) < 1e-10


def test_admm_h_update_is_the_least_squares_minimiser():
    """The H-update minimises ||S - H W^T||^2 + (rho/2) ||H - W + U||^2
    (Appendix, Family 6): checked against numpy's least-squares solver on
    the stacked system, row by row."""
    inst = gen.tpdm_groups(n=90, groups=3, T=600, q=0.05, seed=8)
    rng = np.random.default_rng(4)
    W = rng.random((90, 3))
    U = -0.1 * rng.random((90, 3))
    hp = O.HParams.paper(O.ADMM)
    hp.rho = 7.0
    s = O.Solver(inst.S, W, hp)
    s.A = U.copy()
    s.step()
    # row i: min_h ||S_i - W h||^2 + (rho/2) ||h - (W_i - U_i)||^2
    A = np.vstack([W, np.sqrt(hp.rho / 2.0) * np.eye(3)])
    Hn = np.array([np.linalg.lstsq(A, np.concatenate([inst.S[i], np.sqrt(hp.rho / 2.0) * (W[i] - U[i])]),
                                   rcond=None)[0] for i in range(90)])
    Wn = np.maximum(Hn + U, 0.0)
    np.testing.assert_allclose(s.H, Wn, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(s.A, U + Hn - Wn, rtol=1e-10, atol=1e-12)


def test_admm_dual_stays_non_positive_and_w_non_negative():
    """U' = U + H - [H + U]_+ = min(H + U, 0) <= 0, and W >= 0, at every step."""
    inst = gen.corr_planted(n=120, groups=4, T=800, seed=6)
    s = O.Solver(inst.S, gen.init_uniform(120, 4, 0.1, seed=6), O.HParams.paper(O.ADMM))
    for _ in range(15):
        s.step()
        assert np.all(s.A <= 0.0) and np.all(s.H >= 0.0)
