"""Tensor-core (tcgen05) product paths against the FP64 oracle on the same
(dequantised) matrix, and against the SIMT path.  BF16-stored S uses
kind::f16; FP32-stored S uses the error-compensated 3xTF32 kernel.

H enters the MMA as bf16 hi + bf16 lo (about 16 significant bits, relative
representation error <= 2^-17 per entry, unbiased rounding), products are
exact in FP32 and accumulated in FP32, so the gradient's relative error
against the oracle on the same S stays below 1e-5."""
import numpy as np
import pytest
import torch

import gen
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
REL = 1e-5


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _bf16_problem(n, k, seed, lds=None, dtype=torch.bfloat16):
    inst = gen.tpdm_groups(n=n, groups=max(2, min(k, 32)), T=max(400, 4 * n), q=0.05, seed=seed)
    lds = n if lds is None else lds
    S_pad = torch.zeros(n, lds, dtype=dtype, device=DEV)
    S_pad[:, :n] = torch.tensor(inst.S, dtype=dtype, device=DEV)
    S64 = S_pad[:, :n].double().cpu().numpy()
    H0 = torch.tensor(gen.init_scaled(float(S64.mean()), n, k, seed=seed), dtype=torch.float32,
                      device=DEV)
    return S_pad, S64, H0, H0.double().cpu().numpy()


def _grad(L, h, n, k):
    G = torch.empty(n, k, dtype=torch.float32, device=DEV)
    L.symnmf_grad(h, G)
    torch.cuda.synchronize()
    return G.double().cpu().numpy()


@pytest.mark.parametrize("storage", ["bf16", "f32"])
@pytest.mark.parametrize("n,k", [(8, 1), (64, 8), (100, 5), (128, 16), (129, 32), (1000, 64),
                                 (1031, 33), (4097, 8), (5000, 32)])
def test_tc_gradient_matches_oracle_and_simt(L, n, k, storage):
    lds = (n + 7) // 8 * 8            # row pitch a multiple of 16 bytes
    tdt, ldt = (torch.bfloat16, L.BF16) if storage == "bf16" else (torch.float32, L.F32)
    S, S64, H0, H64 = _bf16_problem(n, k, seed=n, lds=lds, dtype=tdt)
    h = L.symnmf_create_ld(S, n, lds, k, ldt)
    try:
        assert L.symnmf_get_impl(h) == 2
        L.symnmf_set_H(h, H0)
        g_tc = _grad(L, h, n, k)
        f_tc, _ = L.symnmf_objective(h)
        L.symnmf_set_impl(h, 1)
        g_simt = _grad(L, h, n, k)
    finally:
        L.symnmf_destroy(h)
    ref = O.gradient(S64, H64)
    assert O.rel_err(g_tc, ref) < REL
    assert O.rel_err(g_tc, g_simt) < REL
    normS2 = float(np.sum(S64 * S64))
    assert abs(f_tc - O.objective_trace(S64, H64)) <= 1e-6 * normS2


def test_unaligned_pitch_falls_back_to_simt(L):
    n, k = 101, 4
    S, S64, H0, H64 = _bf16_problem(n, k, seed=1)     # pitch 202 bytes
    h = L.symnmf_create(S, n, k, L.BF16)
    try:
        assert L.symnmf_get_impl(h) == 1
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_set_impl(h, 2)
        assert e.value.status == L.ERR_UNSUPPORTED
        L.symnmf_set_H(h, H0)
        assert O.rel_err(_grad(L, h, n, k), O.gradient(S64, H64)) < REL
    finally:
        L.symnmf_destroy(h)


@pytest.mark.parametrize("storage", ["bf16", "f32"])
@pytest.mark.parametrize("method", [3, 4])
def test_tc_sampled_lists_teacher_forced(L, method, storage):
    """Row-SVRG (row list) and Block-SVRG (row and column lists) through
    the tensor-core product: one sampled step from the same state."""
    n, k = 1500, 16
    lds = 1504                        # 16-byte row pitch
    tdt, ldt = (torch.bfloat16, L.BF16) if storage == "bf16" else (torch.float32, L.F32)
    S, S64, H0, H64 = _bf16_problem(n, k, seed=21, lds=lds, dtype=tdt)
    hp = O.HParams.paper(method)
    hp.eta, hp.snapshot_period, hp.phi0 = 0.05, 4, 0.3
    s = O.Solver(S64, H64, hp)
    for _ in range(5):
        s.step()
    for name in ("H", "A", "M", "mu"):
        setattr(s, name, getattr(s, name).astype(np.float32).astype(np.float64))
    h = L.symnmf_create_ld(S, n, lds, k, ldt)
    try:
        assert L.symnmf_get_impl(h) == 2
        L.symnmf_set_H(h, torch.tensor(s.H, dtype=torch.float32, device=DEV))
        for b, arr in ((L.BUF_ACC, s.A), (L.BUF_SNAPSHOT, s.mu)):
            L.symnmf_set_buffer(h, b, torch.tensor(arr, dtype=torch.float32, device=DEV))
        c = L.symnmf_get_ctrl(h)
        c.t, c.phi, c.E0, c.E_prev, c.have_prev = s.ctrl.t, s.ctrl.phi, s.ctrl.E0, s.ctrl.E_prev, 1
        L.symnmf_set_ctrl(h, c)
        L.symnmf_step(h, L.symnmf_hparams_default(method, eta=0.05, snapshot_period=4, phi0=0.3), 1)
        H_t = s.H.copy()
        s.step()
        assert not s.records[-1].full
        out = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_get_buffer(h, L.BUF_GRAD, out)
        g = out.double().cpu().numpy()
        L.symnmf_get_H(h, out)
        Hn = out.double().cpu().numpy()
    finally:
        L.symnmf_destroy(h)
    assert O.rel_err(Hn, s.H) < REL
    # the gradient against the size of its terms (it cancels as H converges)
    scale = 4.0 * (np.linalg.norm(S64 @ H_t) + np.linalg.norm(H_t @ (H_t.T @ H_t)))
    assert float(np.linalg.norm(g - s.g)) / scale < REL


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_tc_free_running_matches_oracle(L, storage):
    n, k = 2000, 16
    tdt, ldt = (torch.bfloat16, L.BF16) if storage == "bf16" else (torch.float32, L.F32)
    S, S64, H0, H64 = _bf16_problem(n, k, seed=4, dtype=tdt)
    hp = O.HParams.paper(O.ADAGRAD)
    hp.eta = 0.1
    s = O.Solver(S64, H64, hp)
    s.run(200)
    h = L.symnmf_create(S, n, k, ldt)
    try:
        assert L.symnmf_get_impl(h) == 2
        L.symnmf_set_H(h, H0)
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADAGRAD, eta=0.1), 200)
        tr = L.symnmf_get_trace(h)
        out = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_get_H(h, out)
        Hg = out.double().cpu().numpy()
    finally:
        L.symnmf_destroy(h)
    Eg = np.array([r.E for r in tr])
    Er = np.array([r.E for r in s.records])
    # the trace form's error is bounded relative to ||S||^2 (Sec. 2.1), so E
    # is compared in absolute terms
    assert np.max(np.abs(Eg - Er)) < 5e-6
    assert O.rel_err(Hg, s.H) < 1e-3
