"""FP8 E4M3 storage of S: the quantiser against the oracle's (codes and
scales bit-exact), and the kind::f8f6f4 tensor-core step against the FP64
oracle on the dequantised S.

On the tensor core H enters as two E4M3 pieces per entry at a power-of-two
factor d per 128-row tile, H ~ d (hi + lo), lo the E4M3 value of the
remainder: each piece keeps 3 stored mantissa bits with round to nearest,
so the representation error is at most 2^-8 of the entry, plus 2^-10 d
where the remainder falls below E4M3's normal range (2^-10 d is below
5e-6 of the tile's largest entry).  Against the oracle fed the same two-piece H
(formed here with the oracle's E4M3 rounding) the gradient agrees to FP32
accumulation error (1e-5); against the exact H it stays inside the 2^-8
bound.  Teacher-forced steps use an H that the two-piece form represents
exactly, so they compare at 1e-5 too."""
import numpy as np
import pytest
import torch

import gen
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
REL = 1e-5
PIECE_BOUND = 2.0 ** -8


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _codes_to_f64(q):
    return q.cpu().view(torch.float8_e4m3fn).double().numpy()


def _quantize(L, S, n, src_dtype, ldq=None):
    ldq = (n + 15) // 16 * 16 if ldq is None else ldq
    nt = (n + 127) // 128
    q = torch.zeros(n, ldq, dtype=torch.uint8, device=DEV)
    sc = torch.zeros(nt, nt, dtype=torch.float32, device=DEV)
    ss = torch.zeros(nt, nt, dtype=torch.float64, device=DEV)
    L.symnmf_quantize_fp8(S, src_dtype, n, n, S.stride(0), q, ldq, sc, nt, ss)
    torch.cuda.synchronize()
    return q, sc, ss, ldq


def _problem(n, k, seed):
    inst = gen.tpdm_groups(n=n, groups=max(2, min(k, 32)), T=max(400, 4 * n), q=0.05, seed=seed)
    S32 = torch.tensor(inst.S, dtype=torch.float32, device=DEV)
    return inst, S32


def two_piece(H, tile=128):
    """H as the tensor core sees it: per 128-row tile, d = the smallest power
    of two with max / d <= 448, hi = e4m3(H / d), lo = e4m3(H / d - hi)."""
    out = np.zeros_like(H)
    for r0 in range(0, H.shape[0], tile):
        blk = H[r0:r0 + tile]
        d = O.tile_scale(float(blk.max()) if blk.size else 0.0)
        x = blk / d
        hi = O.e4m3_round(x)
        lo = O.e4m3_round(x - hi)
        out[r0:r0 + tile] = d * (hi + lo)
    return out


def snap(H):
    """An H that the two-piece form represents exactly (fixed point)."""
    for _ in range(6):
        Hn = two_piece(H)
        if np.array_equal(Hn, H):
            return H
        H = Hn
    raise AssertionError("two-piece snapping did not settle")


def _grad(L, h, n, k):
    G = torch.empty(n, k, dtype=torch.float32, device=DEV)
    L.symnmf_grad(h, G)
    torch.cuda.synchronize()
    return G.double().cpu().numpy()


# ------------------------------------------------------------- quantiser
@pytest.mark.parametrize("n", [1, 100, 128, 300, 1031])
@pytest.mark.parametrize("src", ["f32", "bf16"])
def test_quantize_matches_oracle(L, n, src):
    inst, S32 = _problem(n, 8, seed=n)
    tdt, ldt = (torch.float32, L.F32) if src == "f32" else (torch.bfloat16, L.BF16)
    S = S32.to(tdt)
    q, sc, ss, _ = _quantize(L, S, n, ldt)
    S64 = S.double().cpu().numpy()
    q_ref, sc_ref = O.quantize_fp8(S64)
    assert np.array_equal(_codes_to_f64(q)[:, :n], q_ref)
    assert np.array_equal(sc.double().cpu().numpy(), sc_ref)
    nt = (n + 127) // 128
    ss_ref = np.array([[np.sum(S64[a * 128:(a + 1) * 128, b * 128:(b + 1) * 128] ** 2)
                        for b in range(nt)] for a in range(nt)])
    np.testing.assert_allclose(ss.cpu().numpy(), ss_ref, rtol=1e-13, atol=0)


def test_quantize_bands_equal_one_call(L):
    n = 700
    _, S = _problem(n, 8, seed=3)
    q1, sc1, _, ldq = _quantize(L, S, n, L.F32)
    nt = (n + 127) // 128
    q2 = torch.zeros_like(q1)
    sc2 = torch.zeros_like(sc1)
    for r0, r1 in ((0, 256), (256, 640), (640, n)):
        L.symnmf_quantize_fp8(S[r0:r1], L.F32, r1 - r0, n, n, q2[r0:r1], ldq, sc2[r0 // 128:],
                              nt, None)
    torch.cuda.synchronize()
    assert torch.equal(q1, q2) and torch.equal(sc1, sc2)


def test_quantize_zero_tile_and_invalid(L):
    n = 200
    S = torch.zeros(n, n, dtype=torch.float32, device=DEV)
    S[150:, 150:] = 0.5
    q, sc, ss, ldq = _quantize(L, S, n, L.F32)
    s = sc.cpu().numpy()
    assert s[0, 0] == 1.0 and s[0, 1] == 1.0 and s[1, 1] == 2.0 ** -9
    assert int(q[:128, :128].sum()) == 0
    with pytest.raises(L.SymNMFError):
        L.symnmf_quantize_fp8(S, L.FP8E4M3, n, n, n, q, ldq, sc, 2, None)
    with pytest.raises(L.SymNMFError):
        L.symnmf_quantize_fp8(S, L.F32, n, n, n - 1, q, ldq, sc, 2, None)
    with pytest.raises(L.SymNMFError):
        L.symnmf_quantize_fp8(S, L.F32, n, n, n, q, ldq, sc, 1, None)


# --------------------------------------------------------- FP8 solver step
def _fp8_handle(L, n, k, seed):
    inst, S32 = _problem(n, k, seed)
    q, sc, ss, ldq = _quantize(L, S32, n, L.F32)
    q_ref, sc_ref = O.quantize_fp8(S32.double().cpu().numpy())
    S64 = O.dequantize_fp8(q_ref, sc_ref)
    h = L.symnmf_create_ld(q, n, ldq, k, L.FP8E4M3)
    L.symnmf_set_tile_scales(h, sc, sc.shape[1])
    return h, (q, sc), S64


@pytest.mark.parametrize("n,k", [(8, 1), (100, 5), (128, 16), (129, 32), (1000, 64), (1031, 33),
                                 (4097, 8), (5000, 32)])
def test_fp8_gradient_matches_oracle(L, n, k):
    h, keep, S64 = _fp8_handle(L, n, k, seed=n)
    H64 = gen.init_scaled(float(S64.mean()), n, k, seed=n).astype(np.float32).astype(np.float64)
    try:
        assert L.symnmf_get_impl(h) == 2
        L.symnmf_set_H(h, torch.tensor(H64, dtype=torch.float32, device=DEV))
        g_tc = _grad(L, h, n, k)
        f_tc, _ = L.symnmf_objective(h)
        normS2 = L.symnmf_get_norm(h)
        L.symnmf_set_impl(h, 1)
        g_simt = _grad(L, h, n, k)
    finally:
        L.symnmf_destroy(h)
    np.testing.assert_allclose(normS2, np.sum(S64 * S64), rtol=1e-12)
    Hp = two_piece(H64)
    # the product sees the two-piece H; H Gram uses the FP32 H
    g_emul = 4.0 * (H64 @ (H64.T @ H64) - S64 @ Hp)
    scale = 4.0 * (np.linalg.norm(S64 @ H64) + np.linalg.norm(H64 @ (H64.T @ H64)))
    assert np.linalg.norm(g_tc - g_emul) / scale < REL
    assert np.linalg.norm(g_tc - O.gradient(S64, H64)) / scale < PIECE_BOUND
    assert np.linalg.norm(g_simt - O.gradient(S64, H64)) / scale < REL
    f_emul = normS2 - 2.0 * np.sum(H64 * (S64 @ Hp)) + np.sum((H64.T @ H64) ** 2)
    assert abs(f_tc - f_emul) <= 1e-6 * normS2


@pytest.mark.parametrize("method", [0, 1, 3, 4, 5])
def test_fp8_teacher_forced_step(L, method):
    """One step from an oracle state whose H the two-piece form holds
    exactly: full-batch AdaGrad / RMSprop / ADMM through the fused kernel,
    Row-SVRG and Block-SVRG through the sampled row / column lists."""
    n, k = 1500, 16
    h, keep, S64 = _fp8_handle(L, n, k, seed=21)
    hp = O.HParams.paper(method)
    hp.eta, hp.snapshot_period, hp.phi0 = 0.05, 4, 0.3
    H0 = gen.init_scaled(float(S64.mean()), n, k, seed=21)
    s = O.Solver(S64, snap(H0.astype(np.float32).astype(np.float64)), hp)
    for _ in range(5):
        s.step()
    s.H = snap(s.H.astype(np.float32).astype(np.float64))
    for name in ("A", "M", "mu"):
        setattr(s, name, getattr(s, name).astype(np.float32).astype(np.float64))
    try:
        assert L.symnmf_get_impl(h) == 2
        L.symnmf_set_H(h, torch.tensor(s.H, dtype=torch.float32, device=DEV))
        for b, arr in ((L.BUF_ACC, s.A), (L.BUF_MOM, s.M), (L.BUF_SNAPSHOT, s.mu)):
            L.symnmf_set_buffer(h, b, torch.tensor(arr, dtype=torch.float32, device=DEV))
        c = L.symnmf_get_ctrl(h)
        c.t, c.phi, c.E0, c.E_prev, c.have_prev = s.ctrl.t, s.ctrl.phi, s.ctrl.E0, s.ctrl.E_prev, 1
        L.symnmf_set_ctrl(h, c)
        L.symnmf_step(h, L.symnmf_hparams_default(method, eta=0.05, snapshot_period=4, phi0=0.3), 1)
        H_t = s.H.copy()
        s.step()
        out = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_get_buffer(h, L.BUF_GRAD, out)
        g = out.double().cpu().numpy()
        L.symnmf_get_H(h, out)
        Hn = out.double().cpu().numpy()
    finally:
        L.symnmf_destroy(h)
    if method in (3, 4):
        assert not s.records[-1].full
    assert O.rel_err(Hn, s.H) < REL
    scale = 4.0 * (np.linalg.norm(S64 @ H_t) + np.linalg.norm(H_t @ (H_t.T @ H_t)))
    assert float(np.linalg.norm(g - s.g)) / scale < REL


def test_fp8_free_running_close_to_oracle(L):
    """200 AdaGrad iterations: the trajectory through the two-piece H stays
    close to the oracle's exact-H trajectory on the same (dequantised) S."""
    n, k = 2000, 16
    h, keep, S64 = _fp8_handle(L, n, k, seed=4)
    H0 = gen.init_scaled(float(S64.mean()), n, k, seed=4).astype(np.float32).astype(np.float64)
    hp = O.HParams.paper(O.ADAGRAD)
    hp.eta = 0.1
    s = O.Solver(S64, H0, hp)
    s.run(200)
    try:
        L.symnmf_set_H(h, torch.tensor(H0, dtype=torch.float32, device=DEV))
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADAGRAD, eta=0.1), 200)
        tr = L.symnmf_get_trace(h)
        out = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_get_H(h, out)
        Hg = out.double().cpu().numpy()
    finally:
        L.symnmf_destroy(h)
    Eg = np.array([r.E for r in tr])
    Er = np.array([r.E for r in s.records])
    print("fp8 free-running: max |dE| %.3g, H rel %.3g" % (np.max(np.abs(Eg - Er)),
                                                           O.rel_err(Hg, s.H)))
    assert np.max(np.abs(Eg - Er)) < 1e-3
    assert O.rel_err(Hg, s.H) < 2e-2
