"""Rolling windows (Sec. 8 names streaming SymNMF over rolling windows as
the next step): symnmf_set_matrix rebinds a handle to the next window's S
and keeps H as the warm start, with the solver state fresh.  The oracle
takes the same warm start (the GPU's H after the previous window) on the
same stored S, so the window's trajectory is compared like a cold run."""
import numpy as np
import pytest
import torch

from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
OBJ_ABS = 1e-6


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _window_stream(n, T, steps, stride, seed):
    rng = np.random.default_rng(seed)
    k = max(2, n // 64)
    A = rng.uniform(0.0, 1.0, size=(n, k)) * (rng.random((n, k)) < 0.3)
    A[:, 0] = rng.uniform(0.4, 0.8, size=n)
    Tt = T + (steps - 1) * stride
    return (rng.standard_normal((Tt, k)) @ A.T + rng.standard_normal((Tt, n))).astype(np.float32)


def _build(L, Y, n, lds):
    S = torch.empty(n, lds, dtype=torch.float32, device=DEV)
    L.symnmf_build_dependence(torch.tensor(Y, device=DEV), Y.shape[0], n, n, 1, L.F32, S, lds)
    return S


def test_set_matrix_matches_a_fresh_handle(L):
    """After set_matrix the gradient and objective are those of a new handle
    on the new S with the same H (bit for bit: the same kernels run)."""
    n, k, T = 700, 8, 200
    Y = _window_stream(n, T, 2, 50, seed=1)
    lds = (n + 3) // 4 * 4
    S1, S2 = _build(L, Y[:T], n, lds), _build(L, Y[50:50 + T], n, lds)
    H0 = torch.rand(n, k, device=DEV, generator=torch.Generator(DEV).manual_seed(0)) * 0.2
    h = L.symnmf_create_ld(S1, n, lds, k, L.F32)
    h2 = L.symnmf_create_ld(S2, n, lds, k, L.F32)
    try:
        L.symnmf_set_H(h, H0)
        L.symnmf_step(h, L.symnmf_hparams_default(L.ADAGRAD, eta=0.1), 7)
        H = torch.empty(n, k, device=DEV)
        L.symnmf_get_H(h, H)
        L.symnmf_set_matrix(h, S2, lds)
        L.symnmf_set_H(h2, H)
        G1, G2 = torch.empty(n, k, device=DEV), torch.empty(n, k, device=DEV)
        L.symnmf_grad(h, G1)
        L.symnmf_grad(h2, G2)
        f1, _ = L.symnmf_objective(h)
        f2, _ = L.symnmf_objective(h2)
        torch.cuda.synchronize()
        assert torch.equal(G1, G2) and f1 == f2
        assert L.symnmf_get_norm(h) == L.symnmf_get_norm(h2)
        A = torch.empty(n, k, device=DEV)
        L.symnmf_get_buffer(h, L.BUF_ACC, A)
        torch.cuda.synchronize()
        assert float(A.abs().max()) == 0.0
        assert L.symnmf_get_ctrl(h).t == 0 and len(L.symnmf_get_trace(h)) == 0
    finally:
        L.symnmf_destroy(h)
        L.symnmf_destroy(h2)


def test_warm_started_window_matches_oracle(L):
    """Window 1: 80 AdaGrad iterations; window 2 (stride 40): 80 more from
    the warm start; the second window's E trajectory and final H match the
    oracle run from the same warm start on the same stored S."""
    n, k, T = 640, 8, 300
    Y = _window_stream(n, T, 2, 40, seed=2)
    lds = n
    S1, S2 = _build(L, Y[:T], n, lds), _build(L, Y[40:40 + T], n, lds)
    H0 = np.random.default_rng(3).uniform(0.0, 0.1, size=(n, k)).astype(np.float32)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=0.1)
    h = L.symnmf_create(S1, n, k, L.F32)
    try:
        L.symnmf_set_H(h, torch.tensor(H0, device=DEV))
        L.symnmf_step(h, hp, 80)
        Hw = torch.empty(n, k, device=DEV)
        L.symnmf_get_H(h, Hw)
        L.symnmf_set_matrix(h, S2, lds)
        L.symnmf_step(h, hp, 80)
        tr = L.symnmf_get_trace(h)
        Hg = torch.empty(n, k, device=DEV)
        L.symnmf_get_H(h, Hg)
        torch.cuda.synchronize()
    finally:
        L.symnmf_destroy(h)
    ohp = O.HParams.paper(O.ADAGRAD)
    ohp.eta = 0.1
    s = O.Solver(S2.double().cpu().numpy(), Hw.double().cpu().numpy(), ohp)
    s.run(80)
    assert len(tr) == 80 and tr[0].t == 0
    Eg = np.array([r.E for r in tr])
    Er = np.array([r.E for r in s.records])
    assert np.max(np.abs(Eg - Er)) < OBJ_ABS
    assert O.rel_err(Hg.double().cpu().numpy(), s.H) < 1e-4


def test_set_matrix_invalid(L):
    n, k = 300, 4
    S = torch.eye(n, device=DEV)
    h = L.symnmf_create(S, n, k, L.F32)
    try:
        for args in ((None, n), (S, n - 1)):
            with pytest.raises(L.SymNMFError) as e:
                L.symnmf_set_matrix(h, *args)
            assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_set_matrix_fp8_takes_the_new_scales(L):
    """FP8 storage: the rebound handle's ||S||^2 is that of a fresh handle
    on the new codes and scales."""
    from oracle import symnmf_oracle as O
    n, k, T = 512, 8, 200
    Y = _window_stream(n, T, 2, 60, seed=4)
    nt = (n + 127) // 128
    qs = []
    for w in range(2):
        S = _build(L, Y[w * 60:w * 60 + T], n, n).double().cpu().numpy()
        q_ref, sc_ref = O.quantize_fp8(S)
        q = torch.tensor(q_ref, dtype=torch.float32).to(torch.float8_e4m3fn).view(torch.uint8).to(DEV)
        qs.append((q, torch.tensor(sc_ref, dtype=torch.float32, device=DEV)))
    h = L.symnmf_create(qs[0][0], n, k, L.FP8E4M3)
    h2 = L.symnmf_create(qs[1][0], n, k, L.FP8E4M3)
    try:
        L.symnmf_set_tile_scales(h, qs[0][1], nt)
        L.symnmf_set_tile_scales(h2, qs[1][1], nt)
        L.symnmf_set_matrix(h, qs[1][0], n, qs[1][1], nt)
        assert L.symnmf_get_norm(h) == L.symnmf_get_norm(h2)
        with pytest.raises(L.SymNMFError):
            L.symnmf_set_matrix(h, qs[0][0], n)   # FP8 without scales
    finally:
        L.symnmf_destroy(h)
        L.symnmf_destroy(h2)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_window_update_matches_the_oracles(L, storage):
    """symnmf_window_update builds the next window's |corr| into the buffer
    the handle reads, rebinds it with H kept and ||S||^2 from the build:
    S matches the dependence oracle (Sec. 3) within the build's bound, the
    norm is that of the stored matrix, and the warm-started window's E
    trajectory and final H match the solver oracle run from the same warm
    start on the same stored S (Sec. 8)."""
    from oracle import dependence_oracle as D
    n, k, T, stride, iters = 640, 8, 300, 40, 60
    Tp = (T + 31) // 32 * 32
    tolS = 2.0 ** -21 + 4.0 * (3 * Tp / 8) * 2.0 ** -24
    Y = _window_stream(n, T, 2, stride, seed=5)
    code, dt = {"f32": (L.F32, torch.float32), "bf16": (L.BF16, torch.bfloat16)}[storage]
    S = torch.empty(n, n, dtype=dt, device=DEV)
    L.symnmf_build_dependence(torch.tensor(Y[:T], device=DEV), T, n, n, 1, code, S, n)
    H0 = np.random.default_rng(6).uniform(0.0, 0.1, size=(n, k)).astype(np.float32)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=0.1)
    h = L.symnmf_create(S, n, k, code)
    try:
        L.symnmf_set_H(h, torch.tensor(H0, device=DEV))
        L.symnmf_step(h, hp, iters)
        Hw = torch.empty(n, k, device=DEV)
        L.symnmf_get_H(h, Hw)
        Y2 = torch.tensor(Y[stride:stride + T], device=DEV)
        L.symnmf_window_update(h, Y2, T, n, 1, S, n)
        nrm = L.symnmf_get_norm(h)
        S2 = S.double().cpu().numpy()
        L.symnmf_step(h, hp, iters)
        tr = L.symnmf_get_trace(h)
        Hg = torch.empty(n, k, device=DEV)
        L.symnmf_get_H(h, Hg)
        torch.cuda.synchronize()
    finally:
        L.symnmf_destroy(h)
    ref = D.dependence(Y[stride:stride + T].astype(np.float64), True)
    if storage == "f32":
        assert np.max(np.abs(S2 - ref)) <= tolS
    else:
        lo = torch.tensor(ref - tolS).to(torch.bfloat16).double().numpy()
        hi = torch.tensor(ref + tolS).to(torch.bfloat16).double().numpy()
        assert np.all((S2 >= np.minimum(lo, hi)) & (S2 <= np.maximum(lo, hi)))
    assert abs(nrm - float(np.sum(S2 * S2))) <= 1e-10 * nrm  # float-float runs, FP64 across
    ohp = O.HParams.paper(O.ADAGRAD)
    ohp.eta = 0.1
    s = O.Solver(S2, Hw.double().cpu().numpy(), ohp)
    s.run(iters)
    assert len(tr) == iters and tr[0].t == 0
    Eg = np.array([r.E for r in tr])
    Er = np.array([r.E for r in s.records])
    # E = 1 - (2 tr - ||H^T H||^2) / ||S||^2 carries twice the relative
    # error of tr, and the FP32 S H products carry up to 2^-20 of it (three
    # tf32 products, the dropped S_lo H_lo term); tr <= ||S||^2 from a warm
    # start near the previous window's solution
    assert np.max(np.abs(Eg - Er)) < 2.0 ** -19
    assert O.rel_err(Hg.double().cpu().numpy(), s.H) < 1e-4


def test_window_update_invalid(L):
    n, k, T = 256, 4, 50
    S = torch.eye(n, device=DEV)
    Y = torch.zeros(T, n, device=DEV)
    h = L.symnmf_create(S, n, k, L.F32)
    try:
        for args in ((None, T, n, 1, S, n), (Y, 1, n, 1, S, n), (Y, T, n - 1, 1, S, n),
                     (Y, T, n, 1, None, n), (Y, T, n, 1, S, n - 1)):
            with pytest.raises(L.SymNMFError) as e:
                L.symnmf_window_update(h, *args)
            assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)
