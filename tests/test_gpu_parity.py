"""GPU-vs-oracle parity through the C ABI.

Tolerances (FP32 path): the product S H is accumulated in FP32 over n terms
of non-negative values, so its relative error is a few units of 2^-24 times
a slowly growing factor; 1e-5 relative on the gradient (the target the
method's FP32 path is held to) leaves two orders of margin.  The objective is
checked as |f_gpu - f_ref| <= 1e-6 ||S||^2: the trace form cancels three
terms of size ~||S||^2 (Sec. 2.1, "Numerical consideration"), so the error
is bounded relative to ||S||^2, not to f.
"""
import math

import numpy as np
import pytest
import torch

import gen
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu

REL_FP32 = 1e-5
OBJ_ABS = 1e-6


def grad_err(g, g_ref, S, H):
    """Gradient error relative to the size of its two terms.

    g = 4 (H (H^T H) - S H) is a difference of two terms that nearly cancel
    as the solve converges, so an FP32 evaluation is accurate relative to
    4 ||S H|| + 4 ||H (H^T H)||, not to ||g|| (the measure used for the
    near-stationary case in the design notes)."""
    scale = 4.0 * (np.linalg.norm(S @ H) + np.linalg.norm(H @ (H.T @ H)))
    return float(np.linalg.norm(np.asarray(g) - np.asarray(g_ref))) / scale


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


DEV = "cuda:0"


def to_dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def dequant(St):
    return St.double().cpu().numpy()


class Handle:
    def __init__(self, L, S_t, n, k, dtype, lds=None):
        self.L = L
        self.S_t = S_t
        self.n, self.k = n, k
        self.h = L.symnmf_create(S_t, n, k, dtype) if lds is None else \
            L.symnmf_create_ld(S_t, n, lds, k, dtype)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.L.symnmf_destroy(self.h)

    def get(self, which=None):
        out = torch.empty(self.n, self.k, dtype=torch.float32, device=DEV)
        if which is None:
            self.L.symnmf_get_H(self.h, out)
        else:
            self.L.symnmf_get_buffer(self.h, which, out)
        torch.cuda.synchronize()
        return out.double().cpu().numpy()


def problem(n, k, kind="tpdm", seed=0, dtype=torch.float32):
    if kind == "tpdm":
        inst = gen.tpdm_groups(n=n, groups=max(2, k), T=max(400, 4 * n), q=0.05, seed=seed)
    else:
        inst = gen.corr_planted(n=n, groups=max(2, k), T=1000, seed=seed)
    S_t = to_dev(inst.S, dtype)
    S64 = dequant(S_t)
    H0 = gen.init_scaled(float(S64.mean()), n, k, seed=seed)
    H0_t = to_dev(H0)
    return S_t, S64, H0_t, H0_t.double().cpu().numpy()


@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (127, 8), (128, 8), (129, 5), (300, 16),
                                 (1000, 32), (2000, 64), (2500, 1)])
def test_grad_and_objective_fp32(L, n, k):
    S_t, S64, H0_t, H64 = problem(n, k, seed=n)
    with Handle(L, S_t, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        G = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_grad(hd.h, G)
        f, E = L.symnmf_objective(hd.h)
        torch.cuda.synchronize()
        Gref = O.gradient(S64, H64)
        assert O.rel_err(G.double().cpu().numpy(), Gref) < REL_FP32
        assert grad_err(G.double().cpu().numpy(), Gref, S64, H64) < 1e-6
        normS2 = float(np.sum(S64 * S64))
        assert abs(L.symnmf_get_norm(hd.h) - normS2) <= 1e-12 * normS2
        fref = O.objective_trace(S64, H64)
        assert abs(f - fref) <= OBJ_ABS * normS2
        assert abs(E - fref / normS2) <= OBJ_ABS


@pytest.mark.parametrize("n,k", [(300, 8), (1031, 32)])
def test_grad_bf16_storage(L, n, k):
    """BF16-stored S: the kernel error against the oracle on the same
    (dequantised) matrix is FP32-level."""
    S_t, S64, H0_t, H64 = problem(n, k, seed=3, dtype=torch.bfloat16)
    with Handle(L, S_t, n, k, L.BF16) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        G = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_grad(hd.h, G)
        torch.cuda.synchronize()
        assert O.rel_err(G.double().cpu().numpy(), O.gradient(S64, H64)) < REL_FP32


def _teacher_state(method, S64, H64, steps, hp):
    s = O.Solver(S64, H64, hp)
    for _ in range(steps):
        s.step()
    return s


def _load_state(L, hd, s):
    """Load the oracle state (rounded to FP32) into the handle."""
    L.symnmf_set_H(hd.h, to_dev(s.H))
    L.symnmf_set_buffer(hd.h, L.BUF_ACC, to_dev(s.A))
    L.symnmf_set_buffer(hd.h, L.BUF_MOM, to_dev(s.M))
    L.symnmf_set_buffer(hd.h, L.BUF_SNAPSHOT, to_dev(s.mu))
    c = L.symnmf_ctrl()
    oc = s.ctrl
    c.t, c.E0, c.E_prev, c.phi = oc.t, oc.E0, oc.E_prev, oc.phi
    c.sumA_post, c.E_at_reset = oc.sumA_post, oc.E_at_reset
    c.have_prev, c.stag_count, c.resets = int(oc.have_prev), oc.stag_count, oc.resets
    c.resets_enabled, c.cooldown, c.converged = int(oc.resets_enabled), int(oc.cooldown), 0
    L.symnmf_set_ctrl(hd.h, c)


def _rounded(s):
    """The oracle state rounded to FP32, as the GPU holds it."""
    for name in ("H", "A", "M", "mu"):
        setattr(s, name, getattr(s, name).astype(np.float32).astype(np.float64))
    return s


@pytest.mark.parametrize("method", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("t0", [0, 7, 13])
def test_teacher_forced_single_step(L, method, t0):
    """From the same (FP32-rounded) state at iteration t0 both sides take one
    step; H, G/v, m and the snapshot agree to 1e-5 relative."""
    n, k = 700, 8
    S_t, S64, H0_t, H64 = problem(n, k, seed=11)
    hp = O.HParams.paper(method)
    hp.eta = 0.05 if method != O.RMSPROP else 0.01
    hp.snapshot_period = 3
    hp.phi0 = 0.3
    s = _teacher_state(method, S64, H64, t0, hp)
    s = _rounded(s)
    with Handle(L, S_t, n, k, L.F32) as hd:
        _load_state(L, hd, s)
        lhp = L.symnmf_hparams_default(method, eta=hp.eta, snapshot_period=3, phi0=0.3)
        L.symnmf_step(hd.h, lhp, 1)
        H_t = s.H.copy()
        s.step()
        for which, ref in [(None, s.H), (L.BUF_ACC, s.A), (L.BUF_MOM, s.M), (L.BUF_SNAPSHOT, s.mu)]:
            got = hd.get(which)
            assert O.rel_err(got, ref) < REL_FP32, (which, O.rel_err(got, ref))
        eg = grad_err(hd.get(L.BUF_GRAD), s.g, S64, H_t)
        assert eg < REL_FP32, eg


def _block_lists(n, br, phi, t, seed):
    nb = -(-n // br)
    m = O.sample_count(np.sqrt(phi), n, br)
    return set(O.sample_blocks(seed, t, 1, nb, m)), set(O.sample_blocks(seed, t, 2, nb, m))


@pytest.mark.parametrize("case", ["disjoint", "equal", "overlap"])
@pytest.mark.parametrize("n,k,br,phi", [(700, 8, 128, 0.3), (1100, 16, 256, 0.15)])
def test_block_svrg_list_cases(L, case, n, k, br, phi):
    """Block-SVRG reads each sampled tile position once: (I u J) x K, I x
    (J \\ I) and J x (I \\ J) with K = I n J.  Seeds are picked with the
    oracle's sampler so that the step's I and J are disjoint (K empty),
    equal (only the K part) or overlap partly; one teacher-forced step is
    compared with the oracle."""
    t0 = 7
    for seed in range(5000):
        I, J = _block_lists(n, br, phi, t0, seed)
        kind = "disjoint" if not (I & J) else "equal" if I == J else "overlap"
        if kind == case:
            break
    else:
        pytest.fail("no seed gives case " + case)
    S_t, S64, H0_t, H64 = problem(n, k, seed=12)
    hp = O.HParams.paper(O.BLOCK_SVRG)
    hp.eta, hp.snapshot_period, hp.phi0, hp.block_rows, hp.seed = 0.05, 3, phi, br, seed
    s = _rounded(_teacher_state(O.BLOCK_SVRG, S64, H64, t0, hp))
    assert s.ctrl.t == t0 and not s.is_full(t0)
    with Handle(L, S_t, n, k, L.F32) as hd:
        _load_state(L, hd, s)
        lhp = L.symnmf_hparams_default(O.BLOCK_SVRG, eta=hp.eta, snapshot_period=3, phi0=phi,
                                       block_rows=br, seed=seed)
        L.symnmf_step(hd.h, lhp, 1)
        H_t = s.H.copy()
        s.step()
        for which, ref in [(None, s.H), (L.BUF_ACC, s.A), (L.BUF_SNAPSHOT, s.mu)]:
            got = hd.get(which)
            assert O.rel_err(got, ref) < REL_FP32, (which, O.rel_err(got, ref))
        eg = grad_err(hd.get(L.BUF_GRAD), s.g, S64, H_t)
        assert eg < REL_FP32, eg


@pytest.mark.parametrize("dt,pinned", [("f32", True), ("bf16", False)])
def test_solve_host_matches_the_device_calls(L, dt, pinned):
    """symnmf_solve_host from host buffers (pinned or pageable) gives the
    same H, bit for bit, as symnmf_set_H, symnmf_step and symnmf_get_H on a
    handle over the same S in device memory; it overwrites the device
    buffer its handle was created on and computes ||S||^2 from it."""
    n, k, iters = 700, 8, 30
    tdt, ldt = (torch.float32, L.F32) if dt == "f32" else (torch.bfloat16, L.BF16)
    S_t, _, H0_t, _ = problem(n, k, seed=14, dtype=tdt)
    hp = L.symnmf_hparams_default(L.ADAGRAD)
    with Handle(L, S_t, n, k, ldt) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        st_dev, stats_dev = L.symnmf_step(hd.h, hp, iters)
        H_dev = hd.get()
        norm_dev = L.symnmf_get_norm(hd.h)
    S_host, H0_host = S_t.cpu(), H0_t.cpu()
    H_out = torch.empty(n, k, dtype=torch.float32)
    if pinned:
        S_host, H0_host, H_out = S_host.pin_memory(), H0_host.pin_memory(), H_out.pin_memory()
    S_buf = torch.zeros_like(S_t)
    h = L.symnmf_create(S_buf, n, k, ldt)
    try:
        st, stats = L.symnmf_solve_host(h, S_host, n, H0_host, hp, iters, H_out)
        assert st == st_dev and stats.iter == stats_dev.iter
        assert torch.equal(S_buf, S_t)
        assert L.symnmf_get_norm(h) == norm_dev
        assert np.array_equal(H_out.numpy(), H_dev)
        for bad in (dict(S_host=None), dict(lds_host=n - 1), dict(iters=-1)):
            args = dict(S_host=S_host, lds_host=n, iters=iters)
            args.update(bad)
            with pytest.raises(L.SymNMFError) as e:
                L.symnmf_solve_host(h, args["S_host"], args["lds_host"], H0_host, hp,
                                    args["iters"], H_out)
            assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_solve_host_fp8_with_tile_scales(L):
    """FP8 storage: symnmf_solve_host also uploads the tile scales (host
    pitch nt) into the handle's scale buffer; H equals the device calls'
    bit for bit."""
    n, k, iters = 700, 16, 20
    ldq, nt = 704, (700 + 127) // 128
    S_t, _, H0_t, _ = problem(n, k, seed=15)
    q = torch.zeros(n, ldq, dtype=torch.uint8, device=DEV)
    sc = torch.zeros(nt, nt, dtype=torch.float32, device=DEV)
    L.symnmf_quantize_fp8(S_t, L.F32, n, n, n, q, ldq, sc, nt, None)
    hp = L.symnmf_hparams_default(L.ADAGRAD)
    with Handle(L, q, n, k, L.FP8E4M3, lds=ldq) as hd:
        L.symnmf_set_tile_scales(hd.h, sc, nt)
        L.symnmf_set_H(hd.h, H0_t)
        L.symnmf_step(hd.h, hp, iters)
        H_dev = hd.get()
    q_buf, sc_buf = torch.zeros_like(q), torch.ones_like(sc)
    h = L.symnmf_create_ld(q_buf, n, ldq, k, L.FP8E4M3)
    try:
        L.symnmf_set_tile_scales(h, sc_buf, nt)
        H_out = torch.empty(n, k, dtype=torch.float32).pin_memory()
        L.symnmf_solve_host(h, q.cpu().pin_memory(), ldq, H0_t.cpu().pin_memory(), hp, iters,
                            H_out, sc.cpu().pin_memory(), nt)
        assert torch.equal(q_buf, q) and torch.equal(sc_buf, sc)
        assert np.array_equal(H_out.numpy(), H_dev)
        with pytest.raises(L.SymNMFError) as e:   # FP8 without host scales
            L.symnmf_solve_host(h, q.cpu(), ldq, H0_t.cpu(), hp, iters, H_out)
        assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_free_running_adagrad_n512(L):
    """The n=512, k=8 planted correlation workload: 500 AdaGrad iterations
    from H0 ~ U[0, 0.1] (seed 0), eta = 2.0 and 0.1, against the oracle."""
    inst = gen.corr_planted(n=512, groups=8, T=2000, seed=0)
    S_t = to_dev(inst.S)
    S64 = dequant(S_t)
    H0_t = to_dev(gen.init_uniform(512, 8, 0.1, seed=0))
    H64 = H0_t.double().cpu().numpy()
    for eta in (2.0, 0.1):
        hp = O.HParams.paper(O.ADAGRAD)
        hp.eta = eta
        s = O.Solver(S64, H64, hp)
        s.run(500)
        with Handle(L, S_t, 512, 8, L.F32) as hd:
            L.symnmf_set_H(hd.h, H0_t)
            L.symnmf_step(hd.h, L.symnmf_hparams_default(O.ADAGRAD, eta=eta), 500)
            Hg = hd.get()
            tr = L.symnmf_get_trace(hd.h)
        assert len(tr) == len(s.records) == 500
        Eg = np.array([r.E for r in tr])
        Er = np.array([r.E for r in s.records])
        # E = f / ||S||^2 carries the trace form's error relative to ||S||^2
        assert np.max(np.abs(Eg - Er) / np.maximum(1.0, np.abs(Er))) < OBJ_ABS
        assert O.rel_err(Hg, s.H) < 1e-4
        assert O.boundary_disagreement(Hg, s.H) <= 2


def test_checkpoint_restore_is_bitwise(L):
    n, k = 600, 8
    S_t, S64, H0_t, _ = problem(n, k, seed=5)
    hp = L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD)
    with Handle(L, S_t, n, k, L.F32) as a, Handle(L, S_t, n, k, L.F32) as b:
        L.symnmf_set_H(a.h, H0_t)
        L.symnmf_step(a.h, hp, 80)
        L.symnmf_set_H(b.h, H0_t)
        L.symnmf_step(b.h, hp, 40)
        blob = L.symnmf_get_state(b.h)
        L.symnmf_set_H(b.h, torch.zeros_like(H0_t))
        L.symnmf_set_state(b.h, blob)
        L.symnmf_step(b.h, hp, 40)
        assert np.array_equal(a.get(), b.get())
        assert np.array_equal(a.get(L.BUF_ACC), b.get(L.BUF_ACC))


def test_runs_are_deterministic(L):
    n, k = 900, 16
    S_t, _, H0_t, _ = problem(n, k, seed=6)
    outs = []
    for _ in range(2):
        with Handle(L, S_t, n, k, L.F32) as hd:
            L.symnmf_set_H(hd.h, H0_t)
            L.symnmf_step(hd.h, L.symnmf_hparams_default(L.ADAGRAD), 30)
            outs.append((hd.get(), [r.f for r in L.symnmf_get_trace(hd.h)]))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


@pytest.mark.parametrize("method", [0, 1, 2, 3, 4])
def test_zero_factor_is_fixed_point(L, method):
    n, k = 256, 4
    S_t, _, _, _ = problem(n, k, seed=7)
    with Handle(L, S_t, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, torch.zeros(n, k, device=DEV))
        L.symnmf_step(hd.h, L.symnmf_hparams_default(method), 25)
        assert np.all(hd.get() == 0)
        assert L.symnmf_get_trace(hd.h)[0].E == 1.0


def test_planted_exact_converges(L):
    H0, S = gen.planted_exact(400, 6, seed=2)
    S_t = to_dev(S)
    Hs = H0 + np.random.default_rng(0).uniform(0, 0.05, H0.shape)
    with Handle(L, S_t, 400, 6, L.F32) as hd:
        L.symnmf_set_H(hd.h, to_dev(Hs))
        st, stats = L.symnmf_step(hd.h, L.symnmf_hparams_default(L.ADAGRAD, eta=0.05), 3000)
        assert st == L.CONVERGED and stats.E < 1e-3
        Hg = hd.get()
    assert O.objective_explicit(S, Hg) / float(np.sum(S * S)) < 1e-3


def test_converged_solve_matches_oracle(L):
    """A converging TPDM solve: the GPU stops at the same check as the
    oracle and the factors agree after optimal column matching."""
    n, k = 256, 4
    inst = gen.tpdm_groups(n=n, groups=k, T=2000, q=0.05, seed=3)
    S_t = to_dev(inst.S)
    S64 = dequant(S_t)
    H0_t = to_dev(gen.init_scaled(float(S64.mean()), n, k, seed=3))
    H64 = H0_t.double().cpu().numpy()
    for method in (O.ADAGRAD, O.RMSPROP, O.PIECEWISE):
        s = O.Solver(S64, H64, O.HParams.paper(method))
        s.run(4000)
        with Handle(L, S_t, n, k, L.F32) as hd:
            L.symnmf_set_H(hd.h, H0_t)
            st, stats = L.symnmf_step(hd.h, L.symnmf_hparams_default(method), 4000)
            Hg = hd.get()
        assert s.records[-1].converged and st == L.CONVERGED
        assert stats.iter == s.ctrl.t
        assert O.factor_error(Hg, s.H) < 1e-3


def test_invalid_calls(L):
    n, k = 64, 4
    S_t, _, H0_t, _ = problem(n, k, seed=8)
    with Handle(L, S_t, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        bad = L.symnmf_hparams_default(L.ADAGRAD, block_rows=100)
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_step(hd.h, bad, 1)
        assert e.value.status == L.ERR_INVALID
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_set_buffer(hd.h, L.BUF_GRAD, H0_t)
        assert e.value.status == L.ERR_INVALID
        L.symnmf_step(hd.h, L.symnmf_hparams_default(L.ADAGRAD), 2)   # still usable
    S8 = torch.zeros(128, 128, dtype=torch.uint8, device=DEV)
    h = L.symnmf_create(S8, 128, 4, L.FP8E4M3)
    try:
        L.symnmf_set_H(h, torch.zeros(128, 4, device=DEV))
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_step(h, L.symnmf_hparams_default(L.ADAGRAD), 1)
        assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_nonfinite_input_reported(L):
    n, k = 200, 4
    S_t, _, H0_t, _ = problem(n, k, seed=9)
    S_bad = S_t.clone()
    S_bad[3, 5] = float("nan")
    with Handle(L, S_bad, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_step(hd.h, L.symnmf_hparams_default(L.ADAGRAD), 5)
        assert e.value.status == L.ERR_NONFINITE
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_step(hd.h, L.symnmf_hparams_default(L.ADAGRAD), 1)
        assert e.value.status == L.ERR_STATE
        L.symnmf_set_H(hd.h, H0_t)      # clears the error state
        hd.S_t = S_bad


def test_full_size_sampled_rows_n20000(L):
    """n=20000, k=32 TPDM at full size: sampled gradient rows against the
    oracle's row formula g_i = 4 (h_i (H^T H) - S_i H)."""
    n, k = 20000, 32
    inst = gen.tpdm_groups(n=n, groups=32, T=5000, q=0.05, seed=0, device=DEV,
                           dtype=torch.float32, materialize="torch")
    S_t = inst.S
    H0_t = to_dev(gen.init_scaled(float(S_t.double().mean()), n, k, seed=0))
    H64 = H0_t.double().cpu().numpy()
    with Handle(L, S_t, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        G = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_grad(hd.h, G)
        torch.cuda.synchronize()
        rows = np.random.default_rng(0).choice(n, 64, replace=False)
        Srows = S_t[torch.tensor(rows, device=DEV)].double().cpu().numpy()
        gram = H64.T @ H64
        ref = 4.0 * (H64[rows] @ gram - Srows @ H64)
        got = G.double().cpu().numpy()[rows]
        assert O.rel_err(got, ref) < REL_FP32


def test_batch_step_caps_and_autotune(L):
    """symnmf_batch_step over handles on their own streams matches stepping
    each alone; a CTA cap changes only the stream-K split (FP32 sums in
    another order); the autotuner leaves caps in range and advances every
    solve by 4 x its trial iterations."""
    sizes = [(700, 8), (1000, 16), (1500, 32)]
    probs = [problem(n, k, seed=n) for n, k in sizes]
    hp = L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD)
    hs = []
    streams = []
    for (n, k), (S_t, _, H0_t, _) in zip(sizes, probs):
        st = torch.cuda.Stream()
        h = L.symnmf_create(S_t, n, k, L.F32)
        L.symnmf_set_stream(h, st)
        L.symnmf_set_H(h, H0_t)
        hs.append(h)
        streams.append(st)
    try:
        L.symnmf_set_ctas(hs[1], 7)
        assert L.symnmf_get_ctas(hs[1]) == 7
        L.symnmf_batch_step(hs, [hp] * 3, 30)
        for (n, k), (S_t, _, H0_t, _), h in zip(sizes, probs, hs):
            with Handle(L, S_t, n, k, L.F32) as solo:
                L.symnmf_set_H(solo.h, H0_t)
                L.symnmf_step(solo.h, hp, 30)
                ref = solo.get()
            out = torch.empty(n, k, dtype=torch.float32, device=DEV)
            L.symnmf_get_H(h, out)
            assert O.rel_err(out.double().cpu().numpy(), ref) < 1e-5
        caps = L.symnmf_batch_autotune(hs, [hp] * 3, 5)
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert all(1 <= c <= nsm for c in caps)
        for h, c in zip(hs, caps):
            assert L.symnmf_get_ctas(h) == c
            assert L.symnmf_get_ctrl(h).t == 30 + 4 * 5
    finally:
        for h in hs:
            L.symnmf_destroy(h)


def test_bounded_wait_times_out_and_the_context_survives(L):
    """A device wait on a barrier that nothing completes gives up after its
    limit (0.2 s) and reaches the host as SYMNMF_ERR_TIMEOUT; a solve on
    the same context afterwards is unaffected."""
    assert L.LIB.symnmf_selftest_wait_timeout(0.2) == L.ERR_TIMEOUT
    assert L.LIB.symnmf_selftest_wait_timeout(0.0) == L.ERR_INVALID
    n, k = 300, 4
    S_t, S64, H0_t, H64 = problem(n, k, seed=8)
    with Handle(L, S_t, n, k, L.F32) as hd:
        L.symnmf_set_H(hd.h, H0_t)
        G = torch.empty(n, k, dtype=torch.float32, device=DEV)
        L.symnmf_grad(hd.h, G)
        torch.cuda.synchronize()
        assert O.rel_err(G.double().cpu().numpy(), O.gradient(S64, H64)) < REL_FP32
