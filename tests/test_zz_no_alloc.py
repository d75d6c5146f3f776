"""symnmf_objective_noalloc (objective with a fixed device scratch, no
allocation) against the handle-based symnmf_objective on the same S and H.

Both evaluate Eq. 2 with FP64 cross-tile sums; they differ in how S H is
formed (FP32 FMA here, the tensor-core or SIMT product there), so they
agree to the FP32 product error: |df| <= 1e-6 ||S||^2, the bound the
objective tests use.  Two calls in a row must give identical bits."""
import gc

import numpy as np
import pytest
import torch

import gen
from oracle import symnmf_oracle as O

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def _inputs(L, n, k, storage, seed, ldq=None):
    inst = gen.tpdm_groups(n=n, groups=max(2, min(k, 32)), T=max(400, 4 * n), q=0.05, seed=seed)
    S32 = torch.tensor(inst.S, dtype=torch.float32, device=DEV)
    H = torch.tensor(gen.init_scaled(float(inst.S.mean()), n, k, seed=seed), dtype=torch.float32,
                     device=DEV)
    if storage == "f32":
        return S32, n, L.F32, None, 0, H
    if storage == "bf16":
        return S32.to(torch.bfloat16), n, L.BF16, None, 0, H
    ldq = (n + 15) // 16 * 16 if ldq is None else ldq
    nt = (n + 127) // 128
    q = torch.zeros(n, ldq, dtype=torch.uint8, device=DEV)
    sc = torch.zeros(nt, nt, dtype=torch.float32, device=DEV)
    L.symnmf_quantize_fp8(S32, L.F32, n, n, n, q, ldq, sc, nt, None)
    return q, ldq, L.FP8E4M3, sc, nt, H


@pytest.mark.parametrize("storage,ldq", [("f32", None), ("bf16", None), ("fp8", None),
                                         ("fp8", "n+37")])
@pytest.mark.parametrize("n,k", [(1, 1), (300, 7), (1031, 33), (2048, 64)])
def test_noalloc_objective_matches_handle(L, n, k, storage, ldq):
    """FP8 also with a row pitch n + 37 bytes (not a multiple of 16), so the
    scale lookup of tile (i/128, j/128) is exercised away from the pitch."""
    S, lds, dt, sc, ldsc, H = _inputs(L, n, k, storage, seed=n + k,
                                      ldq=None if ldq is None else n + 37)
    h = L.symnmf_create_ld(S, n, lds, k, dt)
    try:
        if sc is not None:
            L.symnmf_set_tile_scales(h, sc, ldsc)
            # FP8 on the tensor core sees H in two E4M3 pieces (error 2^-8);
            # the SIMT product uses the FP32 H like this entry point
            L.symnmf_set_impl(h, 1)
        L.symnmf_set_H(h, H)
        f_ref, _ = L.symnmf_objective(h)
        normS2 = L.symnmf_get_norm(h)
    finally:
        L.symnmf_destroy(h)
    f = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
    for i in range(2):     # two calls in a row on the same stream
        L.symnmf_objective_noalloc(S, n, lds, dt, sc, ldsc, H, k, normS2, f[i:])
    torch.cuda.synchronize()
    f0, f1 = f.cpu().tolist()
    assert f0 == f1
    assert abs(f0 - f_ref) <= 1e-6 * normS2


def test_noalloc_objective_matches_oracle(L):
    n, k = 700, 12
    S, lds, dt, _, _, H = _inputs(L, n, k, "f32", seed=5)
    S64 = S.double().cpu().numpy()
    H64 = H.double().cpu().numpy()
    normS2 = float(np.sum(S64 * S64))
    f = torch.zeros(1, dtype=torch.float64, device=DEV)
    L.symnmf_objective_noalloc(S, n, lds, dt, None, 0, H, k, normS2, f)
    torch.cuda.synchronize()
    assert abs(float(f.item()) - O.objective_explicit(S64, H64)) <= 1e-6 * normS2


def test_noalloc_leaves_device_memory_untouched(L):
    """After the first call (the device's set-up) a call allocates nothing:
    torch's allocator and the device's free memory are the same before and
    after it."""
    S, lds, dt, sc, ldsc, H = _inputs(L, 1031, 33, "fp8", seed=3)
    f = torch.zeros(2, dtype=torch.float64, device=DEV)
    f1 = f[1:]
    L.symnmf_objective_noalloc(S, 1031, lds, dt, sc, ldsc, H, 33, 1.0, f)
    torch.cuda.synchronize()
    gc.collect()            # no Python temporary is freed between the readings
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
              torch.cuda.mem_get_info()[0])
    L.symnmf_objective_noalloc(S, 1031, lds, dt, sc, ldsc, H, 33, 1.0, f1)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
             torch.cuda.mem_get_info()[0])
    assert before == after
    assert f[0].item() == f[1].item()


def test_noalloc_rejects_beyond_scratch_and_bad_args(L):
    S = torch.zeros(16, 16, dtype=torch.float32, device=DEV)
    H = torch.zeros(16, 64, dtype=torch.float32, device=DEV)
    f = torch.zeros(1, dtype=torch.float64, device=DEV)
    # one 128-row tile past the limit at k = 64, with buffers of that size
    # (FP8 codes, tile scales and H), so the call could not read out of
    # bounds even if the host-side size check were wrong
    n_big = 65280 + 128
    nt = n_big // 128
    Sb = torch.zeros(n_big, n_big, dtype=torch.uint8, device=DEV)
    scb = torch.ones(nt, nt, dtype=torch.float32, device=DEV)
    Hb = torch.zeros(n_big, 64, dtype=torch.float32, device=DEV)
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_objective_noalloc(Sb, n_big, n_big, L.FP8E4M3, scb, nt, Hb, 64, 1.0, f)
    assert e.value.status == L.ERR_UNSUPPORTED and "scratch" in str(e.value)
    del Sb, scb, Hb
    for args in ((None, 16, 16, L.F32, None, 0, H, 4, 1.0, f),
                 (S, 16, 15, L.F32, None, 0, H, 4, 1.0, f),
                 (S, 16, 16, L.F32, None, 0, H, 65, 1.0, f),
                 (S, 16, 16, 7, None, 0, H, 4, 1.0, f),
                 (S, 16, 16, L.FP8E4M3, None, 0, H, 4, 1.0, f)):
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_objective_noalloc(*args)
        assert e.value.status == L.ERR_INVALID
    assert float(f.item()) == 0.0
