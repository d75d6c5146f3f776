"""Device Piecewise AdaGrad reset against the oracle (appendix, Family 3,
"Piecewise AdaGrad"; Sec. 5.1).

At a stagnating check with ||grad_proj||/(nk) > c_r tau_g the accumulator is
reset to G = max(c g^2, c median(g^2)), a cooldown runs until sum(G) has
doubled, and a reset that brought no loss reduction disables further ones.
The median is selected on the device (radix select over the FP32 bit
patterns of the n*k values g^2), so it is index work: given the device's own
gradient it must equal the lower median computed here bit for bit, and the
reset accumulator must equal c * max(g^2, median) in FP32 bit for bit.
Against the FP64 oracle the gradient, and so the median, the accumulator and
the factor, agree to the FP32 path's 1e-5.
"""
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


def to_dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def get(L, h, n, k, which=None):
    out = torch.empty(n, k, dtype=torch.float32, device=DEV)
    if which is None:
        L.symnmf_get_H(h, out)
    else:
        L.symnmf_get_buffer(h, which, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def lower_median_f32(g32):
    """Lower median of the FP32 squares g*g (numpy float32 multiply, round to
    nearest like the device), as the ((N-1)//2)-th smallest value."""
    sq = (g32 * g32).astype(np.float32).ravel()
    return np.partition(sq, (sq.size - 1) // 2)[(sq.size - 1) // 2]


def load(L, h, H, A, ctrl_fields):
    L.symnmf_set_H(h, to_dev(H))
    L.symnmf_set_buffer(h, L.BUF_ACC, to_dev(A))
    c = L.symnmf_ctrl()
    for name, v in ctrl_fields.items():
        setattr(c, name, v)
    L.symnmf_set_ctrl(h, c)


def forced_ctrl(t, E0, E_prev):
    """Controller state before check t: a previous check with E_prev, no
    reset yet, resets enabled, no cooldown."""
    return dict(t=t, E0=E0, E_prev=E_prev, phi=1.0, sumA_post=0.0, E_at_reset=float("nan"),
                have_prev=1, stag_count=0, resets=0, resets_enabled=1, cooldown=0, converged=0)


def check_reset_exact(L, h, n, k, c, A_pre, H_pre, eta, eps):
    """The reset and the update from the device's own gradient g (iteration
    t = the check): median, reset accumulator and sum(G) exact or to the
    order of a sum, and H_{t+1} = [H_t - eta g/(sqrt(A_pre + g^2) + eps)]_+."""
    rec = L.symnmf_get_trace(h)[-1]
    g = get(L, h, n, k, L.BUF_GRAD)
    med = lower_median_f32(g)
    assert rec.check == 1 and rec.reset == 1
    assert np.float32(rec.median_g2) == med            # bit-exact selection
    A = get(L, h, n, k, L.BUF_ACC)
    expect = np.float32(c) * np.maximum((g * g).astype(np.float32), med)
    assert np.array_equal(A, expect)                   # bit-exact reset
    ctrl = L.symnmf_get_ctrl(h)
    total = float(np.sum(A.astype(np.float64)))
    assert abs(ctrl.sumA_post - total) <= 1e-6 * total
    assert ctrl.resets == 1 and ctrl.cooldown == 1 and ctrl.resets_enabled == 1
    g64 = g.astype(np.float64)
    acc = A_pre.astype(np.float64) + g64 * g64
    Hn = np.maximum(H_pre - eta * g64 / (np.sqrt(acc) + eps), 0.0)
    assert O.rel_err(get(L, h, n, k), Hn) < 1e-6
    return rec, g, med, ctrl


@pytest.mark.parametrize("n,k,dt", [(700, 8, "f32"), (20000, 32, "bf16")])
def test_forced_reset_matches_oracle(L, n, k, dt):
    """Teacher-forced Piecewise state at check t = 50 whose stagnation gate
    fires (E at the previous check equal to E_50, KKT gate tau_g = 1e-9):
    both sides take iteration 50 and reset.  Compared with the oracle:
    the decisions, the median, sum(G) after the reset, G and H."""
    tdt = torch.float32 if dt == "f32" else torch.bfloat16
    lib_dt = L.F32 if dt == "f32" else L.BF16
    if n <= 4096:
        inst = gen.tpdm_groups(n=n, groups=k, T=4 * n, q=0.05, seed=11)
        S_t = to_dev(inst.S, tdt)
    else:
        S_t = gen.tpdm_groups(n=n, groups=k, T=5000, q=0.05, seed=11, device=DEV, dtype=tdt,
                              materialize="torch").S
    S64 = S_t.double().cpu().numpy()
    H0 = gen.init_scaled(float(S64.mean()), n, k, seed=11).astype(np.float32).astype(np.float64)
    hp = O.HParams.paper(O.PIECEWISE)
    hp.eta, hp.tau_g = 0.05, 1e-9
    s = O.Solver(S64, H0, hp)
    for _ in range(3):
        s.step()
    s.H = s.H.astype(np.float32).astype(np.float64)
    s.A = s.A.astype(np.float32).astype(np.float64)
    E0 = s.records[0].E
    E50 = O.objective_trace(S64, s.H, s.normS2) / s.normS2
    fields = forced_ctrl(50, E0, E50)
    for name in ("t", "E0", "E_prev", "have_prev", "resets", "resets_enabled", "cooldown"):
        setattr(s.ctrl, name, type(getattr(s.ctrl, name))(fields[name]))
    A_pre, H_pre = s.A.copy(), s.H.copy()
    orec = s.step()
    assert orec.reset and s.ctrl.resets == 1 and s.ctrl.cooldown
    h = L.symnmf_create(S_t, n, k, lib_dt)
    try:
        load(L, h, H_pre, A_pre, fields)
        L.symnmf_step(h, L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, eta=hp.eta, tau_g=hp.tau_g), 1)
        rec, g, med, ctrl = check_reset_exact(L, h, n, k, hp.c, A_pre, H_pre, hp.eta, hp.eps)
        assert rec.t == 50
        med_ref = O.lower_median(s.g * s.g)
        assert abs(rec.median_g2 - med_ref) <= 1e-4 * med_ref
        assert abs(ctrl.sumA_post - s.ctrl.sumA_post) <= REL * s.ctrl.sumA_post
        assert abs(ctrl.E_at_reset - s.ctrl.E_at_reset) <= 1e-6
        assert O.rel_err(get(L, h, n, k, L.BUF_ACC), s.A) < REL
        assert O.rel_err(get(L, h, n, k), s.H) < REL
    finally:
        L.symnmf_destroy(h)


def test_forced_reset_at_four_million_entries(L):
    """n = 62500, k = 64, BF16 S (n k = 4e6 values of g^2: the histogram
    passes of the selection stride over every block of the grid).  The full
    oracle does not fit here, so: the median, the reset accumulator and the
    update are checked bit-exactly (or to FP32 rounding) from the device's
    own gradient, the controller's decisions are replayed through the
    oracle's controller on the device's scalars, and the gradient itself is
    checked against the oracle's row formula on sampled rows."""
    n, k = 62500, 64
    S_t = gen.tpdm_groups(n=n, groups=k, T=4000, q=0.05, seed=5, device=DEV,
                          dtype=torch.bfloat16, materialize="torch").S
    meanS = float(torch.mean(S_t, dtype=torch.float64))
    H0 = gen.init_scaled(meanS, n, k, seed=5).astype(np.float32).astype(np.float64)
    A0 = (np.random.default_rng(5).uniform(0.5, 2.0, size=(n, k)) * 1e-3).astype(np.float32)
    hp = L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, eta=0.05, tau_g=1e-9)
    h = L.symnmf_create(S_t, n, k, L.BF16)
    try:
        L.symnmf_set_H(h, to_dev(H0))
        f0, E_h0 = L.symnmf_objective(h)
        load(L, h, H0, A0, forced_ctrl(50, 1.0, E_h0))
        L.symnmf_step(h, hp, 1)
        rec, g, med, ctrl = check_reset_exact(L, h, n, k, hp.c, A0, H0, hp.eta, hp.eps)
        # controller replay: the oracle's controller on the device's scalars
        oc = O.Ctrl(E0=1.0, E_prev=E_h0, have_prev=True)
        ohp = O.HParams.paper(O.PIECEWISE)
        ohp.eta, ohp.tau_g = 0.05, 1e-9
        out = O.controller_check(oc, ohp, n, 50, rec.E, rec.kkt, rec.sumA, lambda: float(med))
        assert out.reset and oc.resets == ctrl.resets and oc.cooldown == bool(ctrl.cooldown)
        assert oc.E_at_reset == ctrl.E_at_reset
        # the gradient on sampled rows against the oracle's row formula
        rows = np.sort(np.random.default_rng(1).choice(n, 48, replace=False))
        Srows = S_t[torch.tensor(rows, device=DEV)].double().cpu().numpy()
        ref = O.gradient_rows(Srows, H0, rows)
        assert O.rel_err(g[rows].astype(np.float64), ref) < REL
    finally:
        L.symnmf_destroy(h)


def test_free_running_reset_and_disable(L):
    """Piecewise AdaGrad free-running on the n=256, k=4 TPDM (seed 3) with
    eta = 1, c = 10 and the gradient-margin multiplier c_r = 1 (this small
    instance stagnates with ||grad_proj||/(nk) about 2 tau_g, below the
    c_r = 3 of the paper's range).  The oracle resets at iteration 520 (the
    reset's large step raises E) and disables resets at 530, when the
    stagnation gate fires again without a loss reduction.  The device must
    fire the same reset and disable at the same iterations, and its
    trajectory up to the reset must match."""
    n, k = 256, 4
    inst = gen.tpdm_groups(n=n, groups=k, T=1024, q=0.05, seed=3)
    S_t = to_dev(inst.S)
    S64 = S_t.double().cpu().numpy()
    H0_t = to_dev(gen.init_scaled(float(S64.mean()), n, k, seed=3))
    H64 = H0_t.double().cpu().numpy()
    hp = O.HParams.paper(O.PIECEWISE)
    hp.c_r = 1.0
    s = O.Solver(S64, H64, hp)
    s.run(530)
    assert [r.t for r in s.records if r.reset] == [520] and s.ctrl.resets_enabled
    lhp = L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, c_r=1.0)
    h = L.symnmf_create(S_t, n, k, L.F32)
    try:
        L.symnmf_set_H(h, H0_t)
        L.symnmf_step(h, lhp, 530)
        tr = L.symnmf_get_trace(h)
        assert [r.t for r in tr if r.reset] == [520]
        assert L.symnmf_get_ctrl(h).resets_enabled == 1
        rec520 = [r for r in tr if r.t == 520][0]
        Eg = np.array([r.E for r in tr if r.check and r.t <= 520])
        Er = np.array([r.E for r in s.records if r.check and r.t <= 520])
        assert np.max(np.abs(Eg - Er)) < 1e-6
        assert rec520.median_g2 == rec520.median_g2               # evaluated at the reset
        # iteration 530: stagnating again (E rose), no loss reduction -> disable
        s.step()
        L.symnmf_step(h, lhp, 1)
        c = L.symnmf_get_ctrl(h)
        assert not s.ctrl.resets_enabled and c.resets_enabled == 0 and c.resets == 1
        assert L.symnmf_get_trace(h)[-1].reset == 0
    finally:
        L.symnmf_destroy(h)


def test_joint_restarts_reset_on_their_own(L):
    """Three Piecewise restarts of the n=256, k=4 TPDM (seed 3; c_r = 1)
    concatenated in one handle of rank 12, from the starts of seeds 3, 7
    and 10.  Solved alone by the oracle, restart 0 resets at iteration 520,
    restart 1 at 480 and restart 2 never (within 530).  The joint handle
    must reset each restart at its own iteration, leave the others'
    accumulators alone, and disable a restart's resets when the oracle does."""
    n, kb, seeds = 256, 4, (3, 7, 10)
    R = len(seeds)
    inst = gen.tpdm_groups(n=n, groups=kb, T=1024, q=0.05, seed=3)
    S_t = to_dev(inst.S)
    S64 = S_t.double().cpu().numpy()
    H0 = np.concatenate([gen.init_scaled(float(S64.mean()), n, kb, seed=sd).astype(np.float32)
                         for sd in seeds], axis=1)
    hp = O.HParams.paper(O.PIECEWISE)
    hp.c_r = 1.0
    sols = [O.Solver(S64, H0[:, r * kb:(r + 1) * kb].astype(np.float64), hp) for r in range(R)]
    lhp = L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, c_r=1.0)
    h = L.symnmf_create(S_t, n, R * kb, L.F32)
    try:
        L.symnmf_set_restarts(h, R)
        L.symnmf_set_H(h, to_dev(H0))
        done = 0
        # A is compared where no reset's large step lies more than one
        # iteration back: after one the trajectories separate at the FP32
        # rounding level amplified (0.7% in A 40 iterations after 480)
        stages = ((481, [0, 1, 0], (0, 1, 2)), (521, [1, 1, 0], (0, 2)), (531, None, ()))
        for upto, resets, cmpA in stages:
            L.symnmf_step(h, lhp, upto - done)
            for s in sols:
                while s.ctrl.t < upto:
                    s.step()
            done = upto
            rs, en, cd, sp = L.symnmf_get_restart_ctrl(h, R)
            assert rs == [s.ctrl.resets for s in sols], (upto, rs)
            if resets is not None:
                assert rs == resets
            assert en == [int(s.ctrl.resets_enabled) for s in sols], (upto, en)
            assert cd == [int(s.ctrl.cooldown) for s in sols], (upto, cd)
            for r, s in enumerate(sols):
                if s.ctrl.resets:
                    assert abs(sp[r] - s.ctrl.sumA_post) <= 1e-3 * s.ctrl.sumA_post, (upto, r)
            A = get(L, h, n, R * kb, L.BUF_ACC).astype(np.float64)
            for r in cmpA:
                assert O.rel_err(A[:, r * kb:(r + 1) * kb], sols[r].A) < 1e-3, (upto, r)
        tr = L.symnmf_get_trace(h)
        assert [rec.t for rec in tr if rec.reset] == [480, 520]
        assert L.symnmf_get_ctrl(h).resets == 0          # the handle's own controller
    finally:
        L.symnmf_destroy(h)
