"""Restarts concatenated along N: one handle of rank R k with restarts = R
against R handles of rank k started from the matching column blocks.
With the block-diagonal Gram every column block sees exactly the
arithmetic of its own solve (the other blocks contribute exact zeros), so
the blocks of H agree with the separate runs; the concatenated record's E
is the mean of the separate E values."""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _get(L, h, n, k):
    out = torch.empty(n, k, device=DEV)
    L.symnmf_get_H(h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("method,iters", [(0, 40), (5, 15), (4, 24)])
def test_joint_restarts_match_separate_solves(L, method, iters):
    n, k, R = 704, 8, 4
    inst = gen.tpdm_groups(n=n, groups=8, T=3000, q=0.05, seed=1)
    S = torch.tensor(inst.S, dtype=torch.float32, device=DEV)
    rng = np.random.default_rng(2)
    H0 = rng.uniform(0.0, np.sqrt(float(inst.S.mean()) / k), size=(n, R * k)).astype(np.float32)
    over = dict(eta=0.1) if method != 5 else dict(rho=50.0)
    if method == 4:
        over.update(phi0=0.3, snapshot_period=3)
    hp = L.symnmf_hparams_default(method, **over)
    hj = L.symnmf_create(S, n, R * k, L.F32)
    hs = [L.symnmf_create(S, n, k, L.F32) for _ in range(R)]
    try:
        L.symnmf_set_restarts(hj, R)
        L.symnmf_set_H(hj, torch.tensor(H0, device=DEV))
        L.symnmf_step(hj, hp, iters)
        Hj = _get(L, hj, n, R * k)
        Ej = np.array([r.E for r in L.symnmf_get_trace(hj)])
        Es = []
        for r, h in enumerate(hs):
            L.symnmf_set_H(h, torch.tensor(np.ascontiguousarray(H0[:, r * k:(r + 1) * k]), device=DEV))
            L.symnmf_step(h, hp, iters)
            Hr = _get(L, h, n, k)
            blk = Hj[:, r * k:(r + 1) * k]
            assert np.max(np.abs(blk - Hr)) <= 1e-6 * max(1.0, float(np.abs(Hr).max())), r
            Es.append([rec.E for rec in L.symnmf_get_trace(h)])
    finally:
        L.symnmf_destroy(hj)
        for h in hs:
            L.symnmf_destroy(h)
    Em = np.mean(np.array(Es), axis=0)
    full = ~np.isnan(Ej)
    assert np.max(np.abs(Ej[full] - Em[full])) < 1e-6


def test_restarts_invalid(L):
    n = 256
    S = torch.eye(n, device=DEV)
    h = L.symnmf_create(S, n, 8, L.F32)
    try:
        for R in (0, 3, 16):
            with pytest.raises(L.SymNMFError) as e:
                L.symnmf_set_restarts(h, R)
            assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_joint_restarts_bf16_k64(L):
    """BF16 storage, four restarts of rank 16 in one rank-64 handle."""
    n, k, R = 1024, 16, 4
    inst = gen.tpdm_groups(n=n, groups=16, T=4000, q=0.05, seed=3)
    S = torch.tensor(inst.S, dtype=torch.bfloat16, device=DEV)
    H0 = np.random.default_rng(4).uniform(0.0, 0.05, size=(n, R * k)).astype(np.float32)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=0.1)
    hj = L.symnmf_create(S, n, R * k, L.BF16)
    h1 = L.symnmf_create(S, n, k, L.BF16)
    try:
        L.symnmf_set_restarts(hj, R)
        L.symnmf_set_H(hj, torch.tensor(H0, device=DEV))
        L.symnmf_step(hj, hp, 20)
        Hj = _get(L, hj, n, R * k)
        for r in (0, 3):
            L.symnmf_set_H(h1, torch.tensor(np.ascontiguousarray(H0[:, r * k:(r + 1) * k]), device=DEV))
            L.symnmf_step(h1, hp, 20)
            Hr = _get(L, h1, n, k)
            assert np.max(np.abs(Hj[:, r * k:(r + 1) * k] - Hr)) <= 1e-6 * max(1.0, float(np.abs(Hr).max()))
    finally:
        L.symnmf_destroy(hj)
        L.symnmf_destroy(h1)


def test_restart_checks_match_separate_records(L):
    """At each check every restart's E_r and KKT measure equal the records
    of its separate solve.  E_r is formed from the gradient the step wrote
    (f_r = ||S||^2 - ||Gram_rr||^2 + sum H_r .* g_r / 2), the separate record
    by the trace form; both carry the FP32 gradient's error, a few units of
    1e-6 relative to ||S||^2."""
    n, k, R = 704, 8, 4
    inst = gen.tpdm_groups(n=n, groups=8, T=3000, q=0.05, seed=5)
    S = torch.tensor(inst.S, dtype=torch.float32, device=DEV)
    H0 = np.random.default_rng(6).uniform(0.0, np.sqrt(float(inst.S.mean()) / k),
                                          size=(n, R * k)).astype(np.float32)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=0.1)
    hj = L.symnmf_create(S, n, R * k, L.F32)
    hs = [L.symnmf_create(S, n, k, L.F32) for _ in range(R)]
    try:
        L.symnmf_set_restarts(hj, R)
        L.symnmf_set_H(hj, torch.tensor(H0, device=DEV))
        got = []
        for steps in (1, 10, 10, 10):           # checks at t = 0, 10, 20, 30
            L.symnmf_step(hj, hp, steps)
            got.append(L.symnmf_get_restart_stats(hj, R))
        for r, h in enumerate(hs):
            L.symnmf_set_H(h, torch.tensor(np.ascontiguousarray(H0[:, r * k:(r + 1) * k]), device=DEV))
            L.symnmf_step(h, hp, 31)
            tr = L.symnmf_get_trace(h)
            for c, t in enumerate((0, 10, 20, 30)):
                E, kkt, cv = got[c]
                assert abs(E[r] - tr[t].E) < 5e-6, (r, t, E[r], tr[t].E)
                assert abs(kkt[r] - tr[t].kkt) <= 1e-4 * tr[t].kkt, (r, t, kkt[r], tr[t].kkt)
                assert cv[r] == 0
    finally:
        L.symnmf_destroy(hj)
        for h in hs:
            L.symnmf_destroy(h)


def test_joint_handle_stops_with_its_first_converged_restart(L):
    """Restart 0 starts next to an exact solution of S = W W^T, restart 1
    far from it: the concatenated handle stops at the check where restart 0's
    own solve stops, and reports which restart converged."""
    n, k = 400, 6
    W, S64 = gen.planted_exact(n, k, seed=2)
    S = torch.tensor(S64, dtype=torch.float32, device=DEV)
    rng = np.random.default_rng(0)
    H_near = (W + rng.uniform(0, 0.05, W.shape)).astype(np.float32)
    H_far = rng.uniform(0, 0.05, W.shape).astype(np.float32)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=0.05)
    h1 = L.symnmf_create(S, n, k, L.F32)
    hj = L.symnmf_create(S, n, 2 * k, L.F32)
    try:
        L.symnmf_set_H(h1, torch.tensor(H_near, device=DEV))
        st1, s1 = L.symnmf_step(h1, hp, 3000)
        assert st1 == L.CONVERGED
        L.symnmf_set_restarts(hj, 2)
        L.symnmf_set_H(hj, torch.tensor(np.concatenate([H_near, H_far], axis=1), device=DEV))
        stj, sj = L.symnmf_step(hj, hp, 3000)
        E, kkt, cv = L.symnmf_get_restart_stats(hj, 2)
    finally:
        L.symnmf_destroy(h1)
        L.symnmf_destroy(hj)
    assert stj == L.CONVERGED and cv == [1, 0]
    assert sj.iter == s1.iter
    assert E[0] < 1e-3


def test_batch_of_joint_handles_matches_the_oracle(L):
    """Three instances stepped together by symnmf_batch_step, each on its
    own handle and stream: k = 8 with four restarts concatenated (Piecewise
    AdaGrad), k = 32 with two (AdaGrad), k = 64 alone (RMSprop).  Every
    restart's column block is compared with the FP64 oracle solving that
    restart alone from the same start, and each handle's E trace with the
    mean of its restarts' oracle E."""
    from oracle import symnmf_oracle as O
    specs = [(384, 8, 4, O.PIECEWISE, 31), (520, 32, 2, O.ADAGRAD, 32), (300, 64, 1, O.RMSPROP, 33)]
    iters = 40
    hs, hps, refs, streams, mats = [], [], [], [], []   # the handles do not own S
    try:
        for n, k, R, method, seed in specs:
            inst = gen.tpdm_groups(n=n, groups=min(k, 16), T=2000, q=0.05, seed=seed)
            S = torch.tensor(inst.S, dtype=torch.float32, device=DEV)
            S64 = S.double().cpu().numpy()
            mats.append(S)
            rng = np.random.default_rng(seed)
            H0 = rng.uniform(0.0, np.sqrt(float(S64.mean()) / k), size=(n, R * k)).astype(np.float32)
            st = torch.cuda.Stream(DEV)
            h = L.symnmf_create(S, n, R * k, L.F32)
            hs.append(h)
            streams.append(st)
            L.symnmf_set_stream(h, st)
            if R > 1:
                L.symnmf_set_restarts(h, R)
            L.symnmf_set_H(h, torch.tensor(H0, device=DEV))
            hps.append(L.symnmf_hparams_default(method))
            sols = []
            for r in range(R):
                s = O.Solver(S64, H0[:, r * k:(r + 1) * k].astype(np.float64), O.HParams.paper(method))
                s.run(iters)
                sols.append(s)
            refs.append((n, k, R, sols))
        L.symnmf_batch_step(hs, hps, iters)
        torch.cuda.synchronize()
        for h, (n, k, R, sols) in zip(hs, refs):
            Hg = _get(L, h, n, R * k).astype(np.float64)
            for r, s in enumerate(sols):
                assert O.rel_err(Hg[:, r * k:(r + 1) * k], s.H) < 1e-4, (k, r)
            Eg = np.array([rec.E for rec in L.symnmf_get_trace(h)])
            Er = np.mean(np.array([[rec.E for rec in s.records] for s in sols]), axis=0)
            assert len(Eg) == len(Er) == iters
            full = ~np.isnan(Eg)
            assert full.any() and np.array_equal(full, ~np.isnan(Er))
            # E = 1 - (2 tr(H^T S H) - ||H^T H||^2) / ||S||^2 near a fit: both
            # terms are about ||S||^2 and carry the FP32 product's relative
            # error (up to about 1e-6 at k = 64), so E holds to a few 1e-6
            # (relative once E > 1, as after Piecewise's first large step)
            err = np.abs(Eg[full] - Er[full]) / np.maximum(1.0, np.abs(Er[full]))
            assert np.max(err) < 4e-6, (k, float(np.max(err)))
    finally:
        for h in hs:
            L.symnmf_destroy(h)
