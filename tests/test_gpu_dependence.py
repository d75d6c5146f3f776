"""The dependence-matrix builder (Sec. 3) on the GPU against the FP64 oracle.

G = Y^T Y runs on the tensor cores as hi hi + lo hi + hi lo over tf32
pieces of the FP32 centred values (the dropped lo lo term is below 2^-21
relative), accumulated in FP32 over K = 3 T' terms; S_ij = |G_ij| /
sqrt(G_ii G_jj) with FP64 column norms.  Each S_ij is a cosine, so its
error is bounded by the relative error of G_ij against sqrt(G_ii G_jj):
2^-21 from the pieces plus the FP32 accumulation, a few units of 2^-24
times the number of chained MMAs K / 8 in the worst case.  The tests hold
FP32 output to TOL(T) = 2^-21 + 4 (3 T' / 8) 2^-24, BF16 to that plus half
a bf16 step (2^-9 for values up to 1), and FP8 codes to the oracle's
quantiser applied to the oracle's S, allowing one-step differences only
where the two S values straddle a rounding boundary (ties of the round to
nearest even, mostly).  ||S||^2 is summed in
FP32 over runs of 32 values and in FP64 across them, so it is held to
32 * 2^-24 relative."""
import numpy as np
import pytest
import torch

from oracle import dependence_oracle as D
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NRM_REL = 32 * 2.0 ** -24


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def tol(T):
    Tp = (T + 31) // 32 * 32
    return 2.0 ** -21 + 4.0 * (3 * Tp / 8) * 2.0 ** -24


def _data(T, n, center, seed):
    rng = np.random.default_rng(seed)
    if center:
        k = max(2, n // 40)
        A = rng.uniform(0.0, 1.0, size=(n, k)) * (rng.random((n, k)) < 0.3)
        Y = rng.standard_normal((T, k)) @ A.T + rng.standard_normal((T, n)) + 0.5
    else:
        Y = rng.pareto(2.0, size=(T, n)) + 0.01
        Y /= np.linalg.norm(Y, axis=1, keepdims=True)
    return Y.astype(np.float32)


def _build(L, Y, n, center, out, lds=None):
    T = Y.shape[0]
    es = {L.F32: 4, L.BF16: 2, L.FP8E4M3: 1}[out]
    lds = lds or (n + 16 // es - 1) // (16 // es) * (16 // es)
    dt = {L.F32: torch.float32, L.BF16: torch.bfloat16, L.FP8E4M3: torch.uint8}[out]
    S = torch.zeros(n, lds, dtype=dt, device=DEV)
    nt = (n + 127) // 128
    sc = torch.zeros(nt, nt, dtype=torch.float32, device=DEV) if out == L.FP8E4M3 else None
    nrm = torch.zeros(1, dtype=torch.float64, device=DEV)
    Yd = torch.tensor(Y, device=DEV)
    L.symnmf_build_dependence(Yd, T, n, n, center, out, S, lds, sc, nt if sc is not None else 0,
                              nrm)
    torch.cuda.synchronize()
    return S[:, :n], sc, float(nrm.item())


@pytest.mark.parametrize("T,n,center", [(5, 1, 1), (37, 100, 1), (257, 300, 1), (257, 300, 0),
                                        (64, 513, 0), (2000, 1000, 1), (250, 2100, 0)])
def test_dependence_fp32(L, T, n, center):
    Y = _data(T, n, center, seed=T + n)
    S, _, nrm = _build(L, Y, n, center, L.F32)
    ref = D.dependence(Y.astype(np.float64), bool(center))
    got = S.double().cpu().numpy()
    err = np.max(np.abs(got - ref))
    assert err <= tol(T), (err, tol(T))
    assert np.all(np.diag(got) == 1.0)
    assert np.all(got >= 0.0) and np.all(got <= 1.0)
    assert np.array_equal(got, got.T)
    assert abs(nrm - float(np.sum(got * got))) <= NRM_REL * nrm


def test_dependence_bf16(L):
    T, n = 300, 700
    Y = _data(T, n, 1, seed=1)
    S, _, nrm = _build(L, Y, n, 1, L.BF16)
    ref = D.dependence(Y.astype(np.float64), True)
    got = S.double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= tol(T) + 2.0 ** -9
    # round to nearest: every stored value is one of the two bf16 neighbours
    # of the FP32-accurate value, the nearer one unless it is a near tie
    lo = torch.tensor(ref - tol(T)).to(torch.bfloat16).double().numpy()
    hi = torch.tensor(ref + tol(T)).to(torch.bfloat16).double().numpy()
    assert np.all((got >= np.minimum(lo, hi)) & (got <= np.maximum(lo, hi)))
    assert abs(nrm - float(np.sum(got * got))) <= NRM_REL * nrm


def test_dependence_fp8_codes_and_scales(L):
    T, n = 400, 900
    Y = _data(T, n, 1, seed=2)
    S, sc, nrm = _build(L, Y, n, 1, L.FP8E4M3)
    ref = D.dependence(Y.astype(np.float64), True)
    q_ref, sc_ref = O.quantize_fp8(ref)
    assert np.array_equal(sc.double().cpu().numpy(), sc_ref)
    codes = S.cpu().view(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(codes, codes.T)
    mism = codes != q_ref
    if np.any(mism):
        # only where the exact value sits within the FP32-level error of a
        # rounding boundary: the code is then one of the E4M3 values that
        # the interval [S - TOL, S + TOL] rounds to
        scale = np.repeat(np.repeat(sc_ref, 128, 0), 128, 1)[:n, :n]
        x = ref / scale
        lo = O.e4m3_round(x - tol(T) / scale)
        hi = O.e4m3_round(x + tol(T) / scale)
        assert np.all((codes[mism] >= lo[mism]) & (codes[mism] <= hi[mism]))
        assert np.mean(mism) < 1e-3
    assert abs(nrm - float(np.sum(ref * ref))) <= 4 * tol(T) * float(np.sum(ref))


def test_dependence_feeds_the_solver(L):
    """The FP32 matrix built on the GPU is a valid solver input: the
    gradient through the handle matches the oracle's on the oracle's S to
    the builder's error."""
    T, n, k = 500, 640, 8
    Y = _data(T, n, 1, seed=3)
    S, _, nrm = _build(L, Y, n, 1, L.F32)
    ref = D.dependence(Y.astype(np.float64), True)
    S_c = S.contiguous()
    h = L.symnmf_create(S_c, n, k, L.F32)
    try:
        assert abs(L.symnmf_get_norm(h) - nrm) <= NRM_REL * nrm
        H0 = np.random.default_rng(0).uniform(0, 0.2, size=(n, k)).astype(np.float32)
        L.symnmf_set_H(h, torch.tensor(H0, device=DEV))
        G = torch.empty(n, k, device=DEV)
        L.symnmf_grad(h, G)
        torch.cuda.synchronize()
    finally:
        L.symnmf_destroy(h)
    H64 = H0.astype(np.float64)
    Gref = O.gradient(ref, H64)
    scale = 4.0 * (np.linalg.norm(ref @ H64) + np.linalg.norm(H64 @ (H64.T @ H64)))
    assert float(np.linalg.norm(G.double().cpu().numpy() - Gref)) / scale < 1e-5 + tol(T)


def test_dependence_invalid(L):
    n = 64
    Y = torch.zeros(10, n, device=DEV)
    S = torch.zeros(n, n, device=DEV)
    for args in ((Y, 10, n, n - 1, 1, L.F32, S, n), (Y, 1, n, n, 1, L.F32, S, n),
                 (Y, 10, n, n, 1, 7, S, n), (Y, 10, n, n, 1, L.F32, S, n - 1),
                 (Y, 10, n, n, 1, L.FP8E4M3, S, n)):
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_build_dependence(*args)
        assert e.value.status == L.ERR_INVALID
