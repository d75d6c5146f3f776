"""Property-based pins of the oracles over random small inputs: identities
that hold for every input, so a dropped term, a wrong sign or a transposed
operand anywhere in them fails for most draws."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle import dependence_oracle as D  # noqa: E402
from oracle import spkmeans_oracle as K  # noqa: E402
from oracle import symnmf_oracle as O  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None)


def _sym(rng, n):
    A = rng.uniform(0.0, 1.0, size=(n, n))
    S = (A + A.T) / 2.0
    np.fill_diagonal(S, 1.0)
    return S


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(2, 24), k=st.integers(1, 6))
def test_trace_form_equals_explicit_objective(seed, n, k):
    """Eq. 2 (trace form) equals Eq. 1 (explicit) for any S and H."""
    rng = np.random.default_rng(seed)
    S = _sym(rng, n)
    H = rng.uniform(0.0, 1.0, size=(n, k))
    f1 = O.objective_explicit(S, H)
    f2 = O.objective_trace(S, H)
    assert abs(f1 - f2) <= 1e-10 * max(1.0, f1)


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(2, 16), k=st.integers(1, 4))
def test_gradient_is_the_directional_derivative(seed, n, k):
    """<grad f, D> equals the derivative of f along D (central difference)."""
    rng = np.random.default_rng(seed)
    S = _sym(rng, n)
    H = rng.uniform(0.1, 1.0, size=(n, k))
    Dd = rng.standard_normal((n, k))
    eps = 1e-6
    fd = (O.objective_explicit(S, H + eps * Dd) - O.objective_explicit(S, H - eps * Dd)) / (2 * eps)
    g = float(np.sum(O.gradient(S, H) * Dd))
    assert abs(fd - g) <= 1e-5 * max(1.0, abs(g))


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(3, 20), k=st.integers(1, 4),
       rho=st.floats(0.5, 1000.0))
def test_admm_planted_fixed_point(seed, n, k, rho):
    """S = W W^T, U = 0: one ADMM iteration (appendix, Family 6) returns W."""
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.0, 1.0, size=(n, k))
    hp = O.HParams.paper(O.ADMM)
    hp.rho = rho
    s = O.Solver(W @ W.T, W, hp)
    s.step()
    assert np.max(np.abs(s.H - W)) <= 1e-8 * max(1.0, float(W.max()))
    assert np.max(np.abs(s.A)) <= 1e-8


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(4, 30), K_=st.integers(2, 5))
def test_spkmeans_objective_theorem_and_step_bounds(seed, n, K_):
    """S_K = n - sum_k ||s_k|| (Sec. 6 theorem) and J_t lies between the
    objectives of the labels before and after the step."""
    rng = np.random.default_rng(seed)
    S = _sym(rng, n)
    lab = rng.integers(0, K_, size=n)
    X = K.normalized_rows(S)
    theo = n - sum(np.linalg.norm(X[lab == c].sum(axis=0)) for c in range(K_))
    assert abs(K.objective(S, lab, K_) - theo) <= 1e-10 * n
    new, J, _ = K.lloyd_step(S, lab, K_)
    assert K.objective(S, new, K_) <= J + 1e-10 * n <= K.objective(S, lab, K_) + 2e-10 * n


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), T=st.integers(3, 40), n=st.integers(2, 12))
def test_dependence_is_a_cosine_matrix(seed, T, n):
    """The centred dependence matrix equals |corrcoef|, and without centring
    it equals the absolute cosine similarity of the columns."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((T, n)) + rng.uniform(-2, 2, size=n)
    ref = np.abs(np.corrcoef(Y, rowvar=False))
    np.fill_diagonal(ref, 1.0)
    assert np.max(np.abs(D.dependence(Y, True) - ref)) <= 1e-10
    Yn = Y / np.linalg.norm(Y, axis=0)
    cosm = np.abs(Yn.T @ Yn)
    np.fill_diagonal(cosm, 1.0)
    assert np.max(np.abs(D.dependence(Y, False) - cosm)) <= 1e-10


@SETTINGS
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(1, 300))
def test_quantizer_error_bound(seed, n):
    """Per-tile power-of-two E4M3 storage: every entry within half an E4M3
    step of its value (relative 2^-4 for normal codes, absolute 2^-10 of
    the tile scale for subnormal ones)."""
    rng = np.random.default_rng(seed)
    S = rng.uniform(0.0, 1.0, size=(n, n)) * rng.choice([1e-3, 1.0, 50.0])
    q, sc = O.quantize_fp8(S)
    R = O.dequantize_fp8(q, sc)
    scale = np.repeat(np.repeat(sc, 128, 0), 128, 1)[:n, :n]
    err = np.abs(R - S)
    assert np.all(err <= np.maximum(2.0 ** -4 * S, 2.0 ** -10 * scale) * (1 + 1e-12))
