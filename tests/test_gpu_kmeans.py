"""Spherical K-means (Lloyd on the rows of S, Sec. 6) on the GPU against the
FP64 oracle.

The labels are an argmax of cosines that the GPU forms from FP32 products
(error a few units of 1e-7 of a cosine for FP32 and BF16 storage, against
the oracle on the same stored S), so labels are compared exactly only where
the oracle's best cosine beats the runner-up by more than DELTA = 1e-5; at
closer calls the GPU's choice must be within DELTA of the best (both are
correct answers).  J = sum_i (1 - cos_i) then agrees to DELTA per row.
With BF16 storage the operands enter the product as bf16 hi/lo pairs
(about 16 bits) and the centroid sums pass through it twice, so DELTA is
1e-4 there."""
import numpy as np
import pytest
import torch

import gen
from oracle import spkmeans_oracle as K

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
DELTA = 1e-5


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _labels(n, Kc, seed):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, Kc, size=n)
    lab[:Kc] = np.arange(Kc)
    return rng.permutation(lab).astype(np.int32)


def _tpdm(n, Kc, seed, dtype=torch.float32):
    inst = gen.tpdm_groups(n=n, groups=max(2, min(Kc, 32)), T=max(400, 4 * n), q=0.05, seed=seed)
    S_t = torch.tensor(inst.S, dtype=dtype, device=DEV)
    return S_t, S_t.double().cpu().numpy()


def _run(L, h, lab0, n, max_iter, tol=1e-4):
    lin = torch.tensor(lab0, dtype=torch.int32, device=DEV)
    lout = torch.empty(n, dtype=torch.int32, device=DEV)
    st, Jt = L.symnmf_spkmeans(h, lin, lout, max_iter, tol)
    torch.cuda.synchronize()
    return lout.cpu().numpy().astype(np.int64), st, Jt


def _check_labels(got, S64, lab_in, Kc, delta=DELTA):
    ref, J, cos = K.lloyd_step(S64, lab_in, Kc)
    rows = np.arange(len(ref))
    best = cos[rows, ref]
    srt = np.sort(cos, axis=1)
    gap = srt[:, -1] - srt[:, -2] if Kc > 1 else np.full(len(ref), np.inf)
    clear = gap > delta
    assert np.array_equal(got[clear], ref[clear]), int(np.sum(got[clear] != ref[clear]))
    assert np.all(cos[rows, got] >= best - delta)
    return ref, J


@pytest.mark.parametrize("n,Kc,dt", [(129, 5, "f32"), (700, 8, "f32"), (1028, 32, "f32"),
                                     (2000, 64, "f32"), (1032, 16, "bf16")])
def test_kmeans_one_iteration(L, n, Kc, dt):
    """One Lloyd iteration from seeded labels: the labels (up to near-ties),
    J and the changed count.  n = 129 has an unaligned row pitch and takes
    the SIMT product; the others the tensor-core product."""
    S_t, S64 = _tpdm(n, Kc, seed=n, dtype=torch.float32 if dt == "f32" else torch.bfloat16)
    h = L.symnmf_create(S_t, n, Kc, L.F32 if dt == "f32" else L.BF16)
    try:
        impl = L.symnmf_get_impl(h)
        lab0 = _labels(n, Kc, seed=n + 1)
        got, st, Jt = _run(L, h, lab0, n, 1)
    finally:
        L.symnmf_destroy(h)
    assert impl == (2 if (n * (4 if dt == "f32" else 2)) % 16 == 0 else 1)
    delta = DELTA if dt == "f32" else 1e-4
    ref, J = _check_labels(got, S64, lab0, Kc, delta)
    assert st.iters == 1 and len(Jt) == 1
    assert abs(Jt[0] - J) <= delta * n, (Jt[0], J)
    assert abs(st.changed - int(np.sum(got != lab0))) == 0
    assert np.isnan(st.J_prev)


def test_kmeans_teacher_forced_trajectory(L):
    """Five iterations, each from the oracle's previous labels."""
    n, Kc = 1536, 16
    S_t, S64 = _tpdm(n, Kc, seed=3)
    lab = _labels(n, Kc, seed=4)
    h = L.symnmf_create(S_t, n, Kc, L.F32)
    try:
        for _ in range(5):
            got, st, Jt = _run(L, h, lab, n, 1)
            ref, J = _check_labels(got, S64, lab, Kc)
            assert abs(Jt[0] - J) <= DELTA * n
            lab = ref.astype(np.int32)
    finally:
        L.symnmf_destroy(h)


def test_kmeans_planted_run_to_convergence(L):
    """Planted groups with cross-group noise, 20% of the true labels
    flipped: both sides recover the partition, in the same number of
    iterations, with the same J trace."""
    rng = np.random.default_rng(8)
    Kc, m = 8, 160
    n = Kc * m
    S = rng.uniform(0.0, 0.3, size=(n, n))
    for b in range(Kc):
        S[b * m:(b + 1) * m, b * m:(b + 1) * m] += rng.uniform(0.3, 0.7, size=(m, m))
    S = (S + S.T) / 2.0
    np.fill_diagonal(S, 1.0)
    perm = rng.permutation(n)
    S = S[np.ix_(perm, perm)]
    truth = (np.arange(n) // m)[perm]
    lab0 = truth.copy()
    flip = rng.choice(n, size=n // 5, replace=False)
    lab0[flip] = rng.integers(0, Kc, size=flip.size)
    S_t = torch.tensor(S, dtype=torch.float32, device=DEV)
    S64 = S_t.double().cpu().numpy()
    run = K.spkmeans(S64, lab0, Kc)
    h = L.symnmf_create(S_t, n, Kc, L.F32)
    try:
        got, st, Jt = _run(L, h, lab0.astype(np.int32), n, 50)
    finally:
        L.symnmf_destroy(h)
    assert run.converged and st.converged
    assert np.array_equal(run.labels, truth) and np.array_equal(got, truth)
    assert st.iters == len(run.J)
    assert np.max(np.abs(np.array(Jt) - np.array(run.J))) <= DELTA * n


def test_kmeans_leaves_solver_state_and_is_deterministic(L):
    n, Kc = 900, 8
    S_t, _ = _tpdm(n, Kc, seed=5)
    H0 = torch.rand(n, Kc, device=DEV) * 0.1
    h = L.symnmf_create(S_t, n, Kc, L.F32)
    try:
        L.symnmf_set_H(h, H0)
        G0 = torch.empty(n, Kc, device=DEV)
        L.symnmf_grad(h, G0)
        f0, _ = L.symnmf_objective(h)
        lab0 = _labels(n, Kc, seed=6)
        a, sa, Ja = _run(L, h, lab0, n, 20)
        b, sb, Jb = _run(L, h, lab0, n, 20)
        G1 = torch.empty(n, Kc, device=DEV)
        L.symnmf_grad(h, G1)
        f1, _ = L.symnmf_objective(h)
        torch.cuda.synchronize()
    finally:
        L.symnmf_destroy(h)
    assert np.array_equal(a, b) and Ja == Jb and sa.iters == sb.iters
    assert torch.equal(G0, G1) and f0 == f1


def test_kmeans_invalid_arguments(L):
    n, Kc = 256, 4
    S_t, _ = _tpdm(n, Kc, seed=7)
    h = L.symnmf_create(S_t, n, Kc, L.F32)
    lab = torch.zeros(n, dtype=torch.int32, device=DEV)
    try:
        for mi, tol in ((0, 1e-4), (5, -1.0), (5, float("nan"))):
            with pytest.raises(L.SymNMFError) as e:
                L.symnmf_spkmeans(h, lab, lab, mi, tol)
            assert e.value.status == L.ERR_INVALID
    finally:
        L.symnmf_destroy(h)


def test_kmeans_fp8_storage(L):
    """FP8 storage: the operands enter the product as two E4M3 pieces
    (error up to 2^-8 of an entry), so labels are checked for validity:
    every label's oracle cosine (on the dequantised S) is within 2^-6 of
    the best, and J within 2^-6 per row."""
    from oracle import symnmf_oracle as O
    n, Kc = 1024, 16
    S_t, _ = _tpdm(n, Kc, seed=12)
    S64q = S_t.double().cpu().numpy()
    q_ref, sc_ref = O.quantize_fp8(S64q)
    nt = (n + 127) // 128
    q = torch.tensor(q_ref, dtype=torch.float32).to(torch.float8_e4m3fn).view(torch.uint8).to(DEV)
    sc = torch.tensor(sc_ref, dtype=torch.float32, device=DEV)
    S64 = O.dequantize_fp8(q_ref, sc_ref)
    h = L.symnmf_create(q, n, Kc, L.FP8E4M3)
    try:
        L.symnmf_set_tile_scales(h, sc, nt)
        lab0 = _labels(n, Kc, seed=13)
        got, st, Jt = _run(L, h, lab0, n, 1)
    finally:
        L.symnmf_destroy(h)
    ref, J, cos = K.lloyd_step(S64, lab0, Kc)
    rows = np.arange(n)
    assert np.all(cos[rows, got] >= cos[rows, ref] - 2.0 ** -6)
    assert abs(Jt[0] - J) <= 2.0 ** -6 * n
