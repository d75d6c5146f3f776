"""C-ABI tests that need no GPU: the library loads, every symbol declared in
include/symnmf.h is exported, argument errors are reported before any CUDA
call, and the host-side pure functions (SplitMix64 sampling, controller)
agree with the oracle on the same inputs."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf
    return symnmf


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "symnmf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(symnmf_[A-Za-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 25
    for name in names:
        assert hasattr(L.LIB, name), name
    assert sorted(L.DECLARED) == names


def test_argument_errors_without_gpu(L):
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_create(None, 10, 4, L.F32)
    assert e.value.status == L.ERR_INVALID
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_create(4096, 0, 4, L.F32)
    assert e.value.status == L.ERR_INVALID
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_create(4096, 10, 65, L.F32)
    assert e.value.status == L.ERR_UNSUPPORTED
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_create(4096, 10, 0, L.F32)
    assert e.value.status == L.ERR_UNSUPPORTED
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_create(4096, 10, 4, 7)
    assert e.value.status == L.ERR_INVALID
    with pytest.raises(L.SymNMFError) as e:
        L.symnmf_hparams_default(9)
    assert e.value.status == L.ERR_INVALID


def test_next_row_argument_errors_without_gpu(L):
    """The dependence builder, K-means, rolling-window and restart entry
    points reject bad arguments before any CUDA call."""
    Y, S = 4096, 8192  # never dereferenced: validation fails first
    bad = [
        (None, 10, 64, 64, 1, L.F32, S, 64),        # null Y
        (Y, 10, 64, 63, 1, L.F32, S, 64),           # ldy < n
        (Y, 1, 64, 64, 1, L.F32, S, 64),            # T < 2 with centring
        (Y, 0, 64, 64, 0, L.F32, S, 64),            # T < 1
        (Y, 10, 64, 64, 1, 9, S, 64),               # unknown output type
        (Y, 10, 64, 64, 1, L.F32, S, 63),           # lds < n
        (Y, 10, 64, 64, 1, L.F32, S + 4, 64),       # S not 16-byte aligned
        (Y, 10, 65, 65, 1, L.F32, S, 65),           # FP32 pitch not a multiple of 16 bytes
        (Y, 10, 64, 64, 1, L.FP8E4M3, S, 64),       # FP8 without scales
    ]
    for args in bad:
        with pytest.raises(L.SymNMFError) as e:
            L.symnmf_build_dependence(*args)
        assert e.value.status == L.ERR_INVALID, args
    hp = L.symnmf_hparams_default(L.ADAGRAD)
    st = L.symnmf_stats()
    for fn, args in ((L.LIB.symnmf_spkmeans, (None, None, None, 1, 1e-4, None, None)),
                     (L.LIB.symnmf_set_matrix, (None, None, 64, None, 0)),
                     (L.LIB.symnmf_set_restarts, (None, 2)),
                     (L.LIB.symnmf_window_update, (None, None, 10, 64, 1, None, 64, None, 0)),
                     (L.LIB.symnmf_get_restart_ctrl, (None, 2, None, None, None, None)),
                     (L.LIB.symnmf_solve_host, (None, Y, 64, None, 0, 0.0, Y, ctypes.byref(hp), 1,
                                                Y, ctypes.byref(st)))):
        assert fn(*args) == L.ERR_INVALID


def test_status_strings(L):
    assert L.symnmf_status_string(L.OK) == "ok"
    assert L.symnmf_status_string(L.ERR_TIMEOUT) == "device wait timed out"


def test_hparams_default_match_oracle(L):
    from oracle import symnmf_oracle as O
    for m in range(6):
        hp = L.symnmf_hparams_default(m)
        ref = O.HParams.paper(m)
        for f in ("eta", "eps", "alpha", "mu", "c", "c_r", "row_frac", "phi0", "tau_E",
                  "tau_g", "tau_stag", "growth_kkt_mult", "check_interval", "warmup",
                  "snapshot_period", "block_rows", "method", "rho"):
            assert getattr(hp, f) == getattr(ref, f), (m, f)


def test_splitmix64_matches_published_vectors(L):
    vals = [int(l, 16) for l in open(os.path.join(ROOT, "tests", "golden", "splitmix64_state0.txt"))
            if l[0] != "#"]
    assert [L.symnmf_splitmix64(0, i) for i in range(4)] == vals


def test_sampling_matches_oracle(L):
    from oracle import symnmf_oracle as O
    rng = np.random.default_rng(0)
    for _ in range(300):
        seed = int(rng.integers(0, 2**63))
        t = int(rng.integers(0, 10**6))
        stream = int(rng.integers(0, 3))
        nb = int(rng.integers(1, 400))
        m = int(rng.integers(0, nb + 3))
        assert L.symnmf_sample_blocks(seed, t, stream, nb, m) == O.sample_blocks(seed, t, stream, nb, m)


def _ctrl_pair(L, O, method, n):
    hp = L.symnmf_hparams_default(method)
    hpo = O.HParams.paper(method)
    c = L.symnmf_ctrl()
    c.E0 = c.E_prev = c.E_at_reset = float("nan")
    c.phi = hpo.phi0 if method == O.BLOCK_SVRG else 1.0
    c.resets_enabled = 1
    co = O.Ctrl(phi=c.phi)
    return hp, hpo, c, co


@pytest.mark.parametrize("method", [0, 1, 2, 3, 4, 5])
def test_controller_replay_matches_oracle(L, method):
    """The same recorded scalar trace drives both controllers to identical
    decisions (converged / reset / grow) and identical stagnation ratios."""
    from oracle import symnmf_oracle as O
    rng = np.random.default_rng(100 + method)
    for trial in range(20):
        n = int(rng.choice([100, 1000, 20000]))
        hp, hpo, c, co = _ctrl_pair(L, O, method, n)
        E = 0.9
        sumA = 1.0
        for t in range(0, 600, 10):
            # a trace that descends, stalls, and sometimes jumps back
            r = rng.random()
            E = E * (0.5 if r < 0.2 else 1.0 - 1e-6 if r < 0.8 else 1.0 + 1e-3)
            kkt = float(10 ** rng.uniform(-6, -1))
            sumA *= float(rng.uniform(1.0, 3.0))
            med = float(10 ** rng.uniform(-12, -2))
            d = L.symnmf_controller_check(c, hp, n, t, E, kkt, sumA, med)
            out = O.controller_check(co, hpo, n, t, E, kkt, sumA, lambda: med)
            assert d["converged"] == out.converged
            assert d["reset"] == out.reset
            assert d["grow"] == out.grow
            assert (math.isnan(d["stag_ratio"]) and math.isnan(out.stag_ratio)) or \
                d["stag_ratio"] == out.stag_ratio
            if out.reset:
                co.sumA_post = c.sumA_post = sumA * 0.1
            assert c.phi == co.phi and c.resets == co.resets
            assert bool(c.cooldown) == co.cooldown and bool(c.resets_enabled) == co.resets_enabled
            if out.converged:
                break


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With the compiled library absent the binding raises ImportError: the
    product path has no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2607_24518_gb300"
    pkg.mkdir()
    src = os.path.join(ROOT, "paper_2607_24518_gb300")
    for f in ("__init__.py", "symnmf.py"):
        shutil.copy(os.path.join(src, f), pkg / f)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    import paper_2607_24518_gb300.symnmf\n"
            "except ImportError as e:\n"
            "    print('ImportError:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "not built" in r.stdout, r.stdout + r.stderr


def test_noalloc_size_check_on_the_host(L):
    """symnmf_objective_noalloc's argument and size check, run on the host
    with no CUDA call: the documented largest n per padded rank fit, one
    more 128-row tile does not, and the scratch bytes follow
    ceil(n/128) * 8 * 8 (256-byte aligned) + ceil(n/128) * 4 * kp^2."""
    limits = {8: 3355392, 16: 986880, 32: 258048, 64: 65280}
    for k, nmax in [(3, 3355392), (8, 3355392), (9, 986880), (16, 986880), (17, 258048),
                    (32, 258048), (33, 65280), (64, 65280)]:
        st, need = L.symnmf_objective_noalloc_check(nmax, nmax, L.F32, 0, 0, k)
        assert st == 0 and need <= L.NOALLOC_SCRATCH_BYTES, (k, nmax)
        assert need == L.noalloc_scratch_need(nmax, k)
        st, need = L.symnmf_objective_noalloc_check(nmax + 128, nmax + 128, L.F32, 0, 0, k)
        assert st == L.ERR_UNSUPPORTED and need > L.NOALLOC_SCRATCH_BYTES, (k, nmax)
    assert sorted(limits) == [8, 16, 32, 64]
    nt = -(-1031 // 128)
    assert L.symnmf_objective_noalloc_check(1031, 1068, L.FP8E4M3, 1, nt, 33) == \
        (0, (nt * 64 + 255) // 256 * 256 + nt * 4 * 64 * 64)
    assert L.symnmf_objective_noalloc_check(1, 1, L.BF16, 0, 0, 1)[0] == 0
    for args in [(0, 1, L.F32, 0, 0, 4), (16, 15, L.F32, 0, 0, 4), (16, 16, L.F32, 0, 0, 65),
                 (16, 16, L.F32, 0, 0, 0), (16, 16, 7, 0, 0, 4), (16, 16, L.FP8E4M3, 0, 1, 4),
                 (300, 300, L.FP8E4M3, 1, 2, 4)]:
        assert L.symnmf_objective_noalloc_check(*args)[0] == L.ERR_INVALID, args
