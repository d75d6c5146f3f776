"""ADMM (appendix, Family 6) on the GPU against the FP64 oracle.

One iteration takes, with W the handle's H and U the scaled dual held in
the accumulator buffer,
    H  = (2 S W + rho (W - U)) (2 W^T W + rho I)^-1
    W' = [H + U]_+,   U' = U + H - W'.
The GPU forms (2 W^T W + rho I)^-1 in FP32 from the FP64 Gram (Gauss-Jordan
on a symmetric positive definite matrix whose condition number is at most
1 + 2 ||W||_2^2 / rho) and multiplies each right-hand-side row by it in the
step's epilogue.  Against the oracle the error of W' is that of S W (FP32
accumulation, 1e-5 relative as for the other methods) plus the inverse's
FP32 rounding, so W' is held to 1e-5 relative; U' = min(H + U, 0) carries the
absolute error of H + U, so it is measured against ||W'|| + ||U'||.
"""
import numpy as np
import pytest
import torch

import gen
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
REL = 1e-5
OBJ_ABS = 1e-6


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _get(L, h, n, k, which=None):
    out = torch.empty(n, k, dtype=torch.float32, device=DEV)
    if which is None:
        L.symnmf_get_H(h, out)
    else:
        L.symnmf_get_buffer(h, which, out)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def _problem(n, k, seed, dtype=torch.float32, kind="tpdm"):
    if kind == "tpdm":
        inst = gen.tpdm_groups(n=n, groups=max(2, min(k, 32)), T=max(400, 4 * n), q=0.05,
                               seed=seed)
    else:
        inst = gen.corr_planted(n=n, groups=max(2, k), T=1000, seed=seed)
    S_t = _dev(inst.S, dtype)
    S64 = S_t.double().cpu().numpy()
    H0 = _f32(gen.init_scaled(float(S64.mean()), n, k, seed=seed))
    return S_t, S64, H0


def _errors(W, U, s):
    eW = O.rel_err(W, s.H)
    eU = float(np.linalg.norm(U - s.A)) / (np.linalg.norm(s.H) + np.linalg.norm(s.A))
    return eW, eU


def _teacher_step(L, S_t, S64, H0, n, k, rho, t0, impl=None, lds=None, dtype=None):
    hp = O.HParams.paper(O.ADMM)
    hp.rho = rho
    s = O.Solver(S64, H0, hp)
    for _ in range(t0):
        s.step()
    s.H, s.A = _f32(s.H), _f32(s.A)
    dt = L.F32 if dtype is None else dtype
    h = L.symnmf_create(S_t, n, k, dt) if lds is None else L.symnmf_create_ld(S_t, n, lds, k, dt)
    try:
        if impl is not None:
            L.symnmf_set_impl(h, impl)
        L.symnmf_set_H(h, _dev(s.H))
        L.symnmf_set_buffer(h, L.BUF_ACC, _dev(s.A))
        c = L.symnmf_get_ctrl(h)
        c.t, c.E0, c.E_prev, c.have_prev = s.ctrl.t, s.ctrl.E0, s.ctrl.E_prev, int(s.ctrl.have_prev)
        L.symnmf_set_ctrl(h, c)
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADMM, rho=rho), 1)
        used = L.symnmf_get_impl(h)
        W_t = s.H.copy()
        s.step()
        W = _get(L, h, n, k)
        U = _get(L, h, n, k, L.BUF_ACC)
        g = _get(L, h, n, k, L.BUF_GRAD)
        rec = L.symnmf_get_trace(h)[-1]
    finally:
        L.symnmf_destroy(h)
    return s, W_t, W, U, g, rec, used


@pytest.mark.parametrize("n,k", [(129, 5), (700, 8), (1028, 32), (2000, 64)])
@pytest.mark.parametrize("rho", [500.0, 5.0])
def test_admm_teacher_forced_step_fp32(L, n, k, rho):
    """One step from the oracle's state after 6 ADMM iterations: W', U', the
    gradient at W and the record agree.  Rows of S whose pitch is a multiple
    of 16 bytes take the fused tensor-core step, the others (n = 129) the
    SIMT product with the stand-alone epilogue."""
    S_t, S64, H0 = _problem(n, k, seed=n)
    s, W_t, W, U, g, rec, used = _teacher_step(L, S_t, S64, H0, n, k, rho, 6)
    assert used == (2 if (4 * n) % 16 == 0 else 1)
    eW, eU = _errors(W, U, s)
    assert eW < REL and eU < REL, (eW, eU)
    scale = 4.0 * (np.linalg.norm(S64 @ W_t) + np.linalg.norm(W_t @ (W_t.T @ W_t)))
    assert float(np.linalg.norm(g - s.g)) / scale < REL
    r = s.records[-1]
    assert abs(rec.E - r.E) < OBJ_ABS
    # kkt = ||proj grad|| / (n k): its error is the gradient's, relative to
    # the size of the gradient's two terms
    assert abs(rec.kkt - r.kkt) <= REL * scale / (n * k) + 1e-6 * r.kkt
    # sumA = sum U': each entry carries the error of H + U
    assert abs(rec.sumA - float(np.sum(s.A))) <= REL * float(np.sum(np.abs(s.A)) + np.sum(s.H))


def test_admm_teacher_forced_step_simt(L):
    """The same step through the SIMT product and the stand-alone epilogue."""
    n, k = 1028, 32
    S_t, S64, H0 = _problem(n, k, seed=7)
    s, _, W, U, _, _, used = _teacher_step(L, S_t, S64, H0, n, k, 500.0, 4, impl=1)
    assert used == 1
    eW, eU = _errors(W, U, s)
    assert eW < REL and eU < REL, (eW, eU)


def test_admm_teacher_forced_step_bf16(L):
    """BF16 storage of S: the oracle multiplies the same (widened) S."""
    n, k = 1032, 32
    S_t, S64, H0 = _problem(n, k, seed=9, dtype=torch.bfloat16)
    s, _, W, U, _, _, used = _teacher_step(L, S_t, S64, H0, n, k, 500.0, 3, dtype=L.BF16)
    assert used == 2
    eW, eU = _errors(W, U, s)
    assert eW < REL and eU < REL, (eW, eU)


def test_admm_complementarity_is_exact(L):
    """W' = [x]_+ and U' = x - W' for one FP32 x: every entry has W' >= 0,
    U' <= 0 and W' U' = 0 exactly, after any number of steps."""
    n, k = 900, 16
    S_t, S64, H0 = _problem(n, k, seed=2)
    h = L.symnmf_create(S_t, n, k, L.F32)
    try:
        L.symnmf_set_H(h, _dev(H0))
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADMM, rho=20.0), 37)
        W = _get(L, h, n, k)
        U = _get(L, h, n, k, L.BUF_ACC)
    finally:
        L.symnmf_destroy(h)
    assert np.all(W >= 0) and np.all(U <= 0)
    assert np.all(W * U == 0)
    assert np.any(U < 0)


def test_admm_planted_fixed_point(L):
    """S = W* W*^T with U = 0 is a fixed point of the ADMM map: H = W* (the
    right-hand side equals W* (2 W*^T W* + rho I)), so W' = W*, U' = 0."""
    n, k = 640, 8
    rng = np.random.default_rng(5)
    Ws = _f32(rng.uniform(0.0, 1.0, size=(n, k)))
    S = Ws @ Ws.T
    S_t = _dev(S)
    h = L.symnmf_create(S_t, n, k, L.F32)
    try:
        L.symnmf_set_H(h, _dev(Ws))
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADMM), 10)
        W = _get(L, h, n, k)
        U = _get(L, h, n, k, L.BUF_ACC)
    finally:
        L.symnmf_destroy(h)
    assert O.rel_err(W, Ws) < 1e-5
    assert np.linalg.norm(U) <= 1e-5 * np.linalg.norm(Ws)


def test_admm_free_running_n512(L):
    """300 ADMM iterations on the n = 512, k = 8 planted correlation workload
    from H0 ~ U[0, 0.1] (seed 0): the E trajectory and the final W."""
    inst = gen.corr_planted(n=512, groups=8, T=2000, seed=0)
    S_t = _dev(inst.S)
    S64 = S_t.double().cpu().numpy()
    H0 = _f32(gen.init_uniform(512, 8, 0.1, seed=0))
    for rho in (500.0, 20.0):
        hp = O.HParams.paper(O.ADMM)
        hp.rho = rho
        s = O.Solver(S64, H0, hp)
        s.run(300)
        h = L.symnmf_create(S_t, 512, 8, L.F32)
        try:
            L.symnmf_set_H(h, _dev(H0))
            L.symnmf_step(h, L.symnmf_hparams_default(L.ADMM, rho=rho), 300)
            tr = L.symnmf_get_trace(h)
            W = _get(L, h, 512, 8)
        finally:
            L.symnmf_destroy(h)
        assert len(tr) == len(s.records) == 300
        Eg = np.array([r.E for r in tr])
        Er = np.array([r.E for r in s.records])
        assert np.max(np.abs(Eg - Er)) < OBJ_ABS, (rho, np.max(np.abs(Eg - Er)))
        assert O.rel_err(W, s.H) < 1e-4, (rho, O.rel_err(W, s.H))
        assert Er[-1] < Er[0]


def test_admm_invalid_rho(L):
    n, k = 200, 4
    S_t, _, H0 = _problem(n, k, seed=1)
    h = L.symnmf_create(S_t, n, k, L.F32)
    try:
        L.symnmf_set_H(h, _dev(H0))
        for rho in (0.0, -1.0, float("nan")):
            with pytest.raises(Exception):
                L.symnmf_step(h, L.symnmf_hparams_default(L.ADMM, rho=rho), 1)
    finally:
        L.symnmf_destroy(h)
