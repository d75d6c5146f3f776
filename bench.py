"""Benchmark of the fused SymNMF solver step on GB300.

A step is one full solver iteration over the whole matrix: the streamed
S H product, the fused gradient / optimizer / projection epilogue and the
fixed-order reductions (objective, KKT, Gram of the new iterate).  The
default workload is the n=20000, k=32 TPDM matrix stored in FP32 with
full-batch projected AdaGrad (eta=2.0); S (1.6 GB) is larger than L2, so
no flush is needed between iterations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--workload NAME]

Under torchrun each rank solves its own copy of the workload on its own
GPU (replicas only: the solve has no data-parallel exchange on one box);
the value is the sum of iterations over ranks divided by the slowest rank's
time.  ``--impl reference`` times the FP64 CPU oracle on the host cores.

Further workloads, one JSON line each:
  --workload NAME   the other n=20000 / n=1e5 step workloads (BF16, FP8,
                    RMSprop, ADMM, correlation)
  --time-to-tol     n=1e5 correlation, BF16 vs FP32 time to a relative
                    objective of 1e-3
  --large-fp8       n=3e5 k=64 TPDM in FP8, Block-SVRG AdaptGrow
  --batch           64 instances x 4 restarts, BF16, Piecewise AdaGrad
  --kmeans          spherical K-means on the n=20000 TPDM matrix, K=32
  --dependence      the |corr| build of n=1e5 variables over 500 observations
  --rolling         10 windows: fused GPU |corr| build + rebind, warm-started solves
  --rolling-batch   4 series of uneven n, 6 windows each, through the batched path
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused SH-step iters/s, HBM GB/s vs peak; time-to-tol at n=1e5 BF16 vs FP32"
UNIT = "iters/s"

WORKLOADS = {
    # name: (generator, n, k, dtype, method, eta (None: the method has none))
    "tpdm_n20000_k32_fp32_adagrad": ("tpdm", 20000, 32, "f32", 0, 2.0),
    "tpdm_n20000_k32_fp32_rmsprop": ("tpdm", 20000, 32, "f32", 1, 0.05),
    "tpdm_n20000_k32_bf16_adagrad": ("tpdm", 20000, 32, "bf16", 0, 2.0),
    "tpdm_n20000_k32_fp8_adagrad": ("tpdm", 20000, 32, "fp8", 0, 2.0),
    "tpdm_n20000_k32_fp32_admm": ("tpdm", 20000, 32, "f32", 5, None),  # rho 500
    "corr_n100000_k32_fp32_adagrad": ("corr", 100000, 32, "f32", 0, 2.0),
    "corr_n100000_k32_bf16_adagrad": ("corr", 100000, 32, "bf16", 0, 2.0),
}
METHOD = {0: "adagrad", 1: "rmsprop", 2: "piecewise_adagrad", 3: "row_svrg",
          4: "block_svrg_adaptgrow", 5: "admm"}
ESIZE = {"f32": 4, "bf16": 2, "fp8": 1}
# bytes per entry of the MMA copy of H (hi + lo pieces) for each storage type
BT_ESIZE = {"f32": 4, "bf16": 2, "fp8": 1}
KERNEL_SOURCES = ("k_prod_tc.cu", "tc_ptx.cuh", "epi_common.cuh", "symnmf_internal.h")


def alg_bytes_full_step(n, k, dt, method):
    """Algorithmic DRAM bytes of one full fused step: S once, plus the n x k
    state: H_t and G read, H_{t+1} and G written (ADMM: U in place of G;
    RMSprop adds m read and written; the gradient g is written only at
    check iterations and is not counted), the hi/lo MMA copy of H read once
    and written once (FP32 also its bf16 copy); FP8 adds the tile scales."""
    nt = -(-n // 128)
    b = n * n * ESIZE[dt]
    b += 16 * n * k + (8 * n * k if method == 1 else 0)
    b += 2 * (2 * k * n * BT_ESIZE[dt])
    if dt == "f32":
        b += 2 * (max(k, 16) * n * 2)  # bf16 copy of H for the S_lo H product
    if dt == "fp8":
        b += 4 * nt * nt
    return b


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2607_24518_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, or None when the kernel sources changed since the capture."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(p):
        return None
    cur = kernel_source_hash()
    for line in open(p):
        f = line.split()
        if len(f) == 3 and not line.startswith("#") and f[0] == workload and f[1] == cur:
            return float(f[2])
    return None
DEFAULT = "tpdm_n20000_k32_fp32_adagrad"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_config(name, world=1):
    """The config object of a workload's line, the same for both arms."""
    kind, n, k, dt, method, eta = WORKLOADS[name]
    return {"workload": name, "n": n, "k": k, "method": METHOD[method], "eta": eta,
            **({"rho": 500.0} if method == 5 else {}), "storage": dt,
            "l2": "S larger than L2 (no flush needed)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def make_input(name, device):
    import torch
    import gen
    kind, n, k, dt, method, eta = WORKLOADS[name]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "fp8": torch.float32}[dt]
    if kind == "tpdm":
        inst = gen.tpdm_groups(n=n, groups=32, T=5000, q=0.05, seed=0, device=device,
                               dtype=tdt, materialize="torch")
    else:
        inst = gen.corr_factor(n=n, T=500, seed=0, device=device, dtype=tdt, materialize="torch")
    S = inst.S
    mean = float(S.double().mean()) if n <= 30000 else float(S[:4096].double().mean())
    H0 = gen.init_scaled(mean, n, k, seed=0)
    return S, H0, inst


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(x.get("num_threads", 1)) for x in info)
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_rate(S64, H0, method, eta, budget_s=15.0, min_iters=2, max_iters=None):
    """Iterations/s of the FP64 oracle on the host cores (bounded sample)."""
    from oracle import symnmf_oracle as O
    hp = O.HParams.paper(method)
    if eta is not None:
        hp.eta = eta
    hp.tau_g = 1e-30
    s = O.Solver(S64, H0, hp)
    s.step()  # warm-up (first touch of S)
    t0 = time.perf_counter()
    it = 0
    while True:
        s.step()
        it += 1
        el = time.perf_counter() - t0
        if (it >= min_iters and el >= budget_s) or (max_iters and it >= max_iters):
            break
    return it / el, it, el


def oracle_rate_one_thread(name, budget_s=10.0):
    """The same oracle timing on one host thread: a child process with the
    BLAS thread counts set to 1 before numpy loads regenerates the workload
    on the CPU and times the oracle's iterations."""
    import subprocess
    kind, n, k, dt, method, eta = WORKLOADS[name]
    if kind != "tpdm" or dt != "f32":
        return None
    code = (
        "import sys, time, json\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import numpy as np, gen\n"
        "from oracle import symnmf_oracle as O\n"
        f"S = np.asarray(gen.tpdm_groups(n={n}, groups=32, T=5000, q=0.05, seed=0).S, dtype=np.float64)\n"
        f"H0 = gen.init_scaled(float(S.mean()), {n}, {k}, seed=0)\n"
        f"hp = O.HParams.paper({method})\n"
        + (f"hp.eta = {eta}\n" if eta is not None else "")
        + "hp.tau_g = 1e-30\n"
        "s = O.Solver(S, H0, hp)\n"
        "s.step()\n"
        "t0 = time.perf_counter(); it = 0\n"
        "while True:\n"
        "    s.step(); it += 1; el = time.perf_counter() - t0\n"
        f"    if it >= 2 and el >= {budget_s}: break\n"
        "print(json.dumps({'rate': it / el, 'iters': it, 'seconds': el}))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=600)
        d = json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, never fatal to the bench line
        return {"error": str(e)[:200]}
    return {"value": d["rate"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['iters']} FP64 oracle iterations of the same workload on one thread "
                      f"({d['seconds']:.1f} s; workload regenerated on the CPU)"}


def oracle_row_rate(S_rows, H, rows, n, budget_s=10.0):
    """Oracle iterations/s extrapolated from its gradient on a sample of
    rows of S: a full iteration costs n / len(rows) times as much (the
    update and the O(n k^2) terms are negligible at these sizes)."""
    from oracle import symnmf_oracle as O
    O.gradient_rows(S_rows, H, rows)
    t0 = time.perf_counter()
    it = 0
    while True:
        O.gradient_rows(S_rows, H, rows)
        it += 1
        el = time.perf_counter() - t0
        if it >= 2 and el >= budget_s:
            break
    per_iter = el / it * (n / len(rows))
    return {"value": 1.0 / per_iter, "unit": "iters/s (extrapolated)", "cores": cpu_threads(),
            "kind": "oracle",
            "sample": f"{it} FP64 oracle gradients of {len(rows)} rows of S ({el:.1f} s), "
                      f"extrapolated to a full iteration (x {n / len(rows):.0f})"}


def aggregate_ranks(ms, iters, world, device):
    """Replicas: the slowest rank's time and the iterations of all ranks
    (one value per rank; no data-path collective exists)."""
    if world <= 1:
        return ms, iters
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    it_t = torch.tensor([iters], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(it_t)
    return float(t.item()), int(it_t.item())


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2607_24518_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2607_24518_gb300 import symnmf as L

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    kind, n, k, dt, method, eta = WORKLOADS[args.workload]
    S, H0, inst = make_input(args.workload, dev)
    dtype = {"f32": L.F32, "bf16": L.BF16, "fp8": L.FP8E4M3}[dt]
    H0_t = torch.tensor(H0, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    scales = None
    if dt == "fp8":
        # per-tile E4M3 storage made by the library's quantiser; ||S||^2 of
        # the unquantised source from the quantiser's per-tile sums
        nt = -(-n // 128)
        q = torch.empty(n, n, dtype=torch.uint8, device=dev)
        scales = torch.empty(nt, nt, dtype=torch.float32, device=dev)
        ss = torch.empty(nt, nt, dtype=torch.float64, device=dev)
        L.symnmf_quantize_fp8(S, L.F32, n, n, n, q, n, scales, nt, ss)
        torch.cuda.synchronize()
        del S
        S = q
    h = L.symnmf_create(S, n, k, dtype)
    L.symnmf_set_stream(h, stream)
    if scales is not None:
        L.symnmf_set_tile_scales(h, scales, scales.shape[1])
    over = {} if eta is None else {"eta": eta}
    hp = L.symnmf_hparams_default(method, tau_g=1e-30, **over)  # never stop early: fixed work
    L.symnmf_set_H(h, H0_t)
    L.symnmf_step(h, hp, args.warmup)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    # timed region: no events between the kernels (an event would break
    # the overlap of each step with the previous iteration's reduction)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    status, st = L.symnmf_step(h, hp, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    iters = int(st.iter) - args.warmup
    # the same steps again with an event pair around every step kernel:
    # its average duration (roofline) and the kernels launched per step
    prof_steps = max(10, min(args.steps, 100))
    L.symnmf_set_profiling(h, True)
    L.symnmf_step(h, hp, prof_steps)
    torch.cuda.synchronize()
    prod_ms, prod_launches, prod_bytes, kernel_launches = L.symnmf_get_profile(h)
    L.symnmf_set_profiling(h, False)
    ck = clocks.stop() if clocks else None
    kernels_per_step = kernel_launches / max(1, prof_steps)
    ms, total_iters = aggregate_ranks(ms, iters, world, dev)
    impl = L.symnmf_get_impl(h)

    # end to end through the public API with host buffers: every e2e step
    # is one symnmf_solve_host call, which uploads S (and FP8 tile scales)
    # and H0 from pinned memory, computes ||S||^2, runs one check interval
    # (10 iterations) and reads H back
    e2e = None
    if rank == 0:
        S_host = S.cpu().pin_memory()
        H_host = H0_t.cpu().pin_memory()
        H_out = torch.empty_like(H_host).pin_memory()
        S_dev = torch.zeros_like(S)
        he = L.symnmf_create(S_dev, n, k, dtype)
        L.symnmf_set_stream(he, stream)
        sc_host, sc_dev, ld_sc = None, None, 0
        if scales is not None:
            sc_host = scales.cpu().pin_memory()
            sc_dev = torch.ones_like(scales)
            ld_sc = scales.shape[1]
            L.symnmf_set_tile_scales(he, sc_dev, ld_sc)
        # ||S||^2 as the caller knows it from building S (the timed handle's)
        norm_known = L.symnmf_get_norm(h)
        per = 10
        reps = max(2, min(5, args.steps // per))
        for rep in range(reps + 1):
            if rep == 1:
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
            L.symnmf_solve_host(he, S_host, S.stride(0), H_host, hp, per, H_out, sc_host, ld_sc,
                                normS2=norm_known)
        a1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a0.elapsed_time(a1)
        L.symnmf_destroy(he)
        h2d = S.numel() * S.element_size() + H0_t.numel() * 4
        if scales is not None:
            h2d += scales.numel() * 4
        e2e = {"value": reps * per / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d) // per,
               "d2h_bytes_per_step": int(H0_t.numel() * 4 + 8) // per,
               "call": "symnmf_solve_host (C-ABI, host buffers)",
               "note": "per 10-iteration solve: S and H0 uploaded from pinned host memory, "
                       "||S||^2 passed as the caller knows it from building S, H read back; "
                       "bytes shown per iteration"}
        del S_host
    L.symnmf_destroy(h)

    out = None
    if rank == 0:
        peak, src = peaks()
        per_launch_ms = prod_ms / max(1, prod_launches)
        # every timed iteration is a full step: one fused launch each
        per_launch_bytes = alg_bytes_full_step(n, k, dt, method)
        achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
        traffic = measured_traffic(args.workload) if impl == 2 else None
        cpu = None
        if args.cpu_baseline:
            if dt == "fp8":
                from oracle import symnmf_oracle as O
                S64 = O.dequantize_fp8(S.cpu().view(torch.float8_e4m3fn).double().numpy(),
                                       scales.double().cpu().numpy())
            else:
                S64 = S.double().cpu().numpy()
            rate, it, el = oracle_rate(S64, H0_t.double().cpu().numpy(), method, eta,
                                       budget_s=args.cpu_budget)
            del S64
            cpu = {"value": rate, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                   "sample": f"{it} FP64 oracle iterations of the same workload ({el:.1f} s, "
                             "numpy float64 on the host cores)"}
            one = oracle_rate_one_thread(args.workload, budget_s=min(args.cpu_budget, 10.0))
            if one is not None:
                cpu["one_thread"] = one
        out = {
            "metric": METRIC, "value": total_iters / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / max(1, iters),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16": "bf16", "fp8": "e4m3"}[dt]
                     + " storage, f32 accumulate, f64 reductions",
            "data": "synthetic (seeded TPDM / correlation generator)",
            "config": workload_config(args.workload, world),
            "product_impl": ["", "simt", "tcgen05"][impl],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                         "kernel": "fused step (S H product + epilogue)" if impl == 2 else "S H product",
                         "bytes_per_launch": per_launch_bytes, "s_bytes_per_launch":
                         prod_bytes / max(1, prod_launches), "ms_per_launch": per_launch_ms,
                         "frac_of_8TBps_nominal": achieved / 8000.0,
                         "kernel_source": kernel_source_hash()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "time_to_tol": None,
            "clocks": ck,
            "gpu_launches": int(round(kernels_per_step * iters)),
            "status": L.symnmf_status_string(status),
        }
        # the second half of the headline metric: time to a relative
        # objective of 1e-3 at n = 1e5, BF16 vs FP32 storage (about 40
        # GPU-seconds, after the timed region)
        if world == 1 and args.time_to_tol_line:
            del S
            torch.cuda.empty_cache()
            ttt, _ = time_to_tol_core(L, dev, args.ttt_n, args.ttt_cap)
            for key in ("reference_run", "runs", "generation_seconds"):
                ttt.pop(key, None)
            out["time_to_tol"] = ttt
    return out


def time_to_tol_core(L, dev, n, cap, tol=1e-3):
    """Time to a relative objective tolerance at n (correlation, k=32,
    full-batch AdaGrad), S stored FP32 vs BF16.  E* is the E of a long FP32
    run, stopped by the AND rule (Eq. 11) or at its iteration cap (reported
    as such); a run reaches tolerance at its first check with
    (E_t - E*) / E* <= tol.  The FP32 run to tolerance is the start of that
    same (deterministic) run, so its time is read at the first check within
    tolerance; the BF16 run is separate.  Each final H is also evaluated on
    the FP32 S."""
    import torch
    import gen
    k = 32
    t_gen = time.perf_counter()
    inst = gen.corr_factor(n=n, T=500, seed=0, device=dev, dtype=torch.float32, materialize="torch")
    S32 = inst.S
    Sbf = S32.to(torch.bfloat16)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    mean = float(S32[:4096].double().mean())
    H0 = torch.tensor(gen.init_scaled(mean, n, k, seed=0), dtype=torch.float32, device=dev)
    hp = L.symnmf_hparams_default(L.ADAGRAD)
    per = hp.check_interval

    def solve(S, dt, stop, cap):
        h = L.symnmf_create(S, n, k, dt)
        L.symnmf_set_H(h, H0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, E, conv = 0, float("nan"), False
        checks = []                       # (iteration, E, seconds) at every check
        while it < cap:
            status, st = L.symnmf_step(h, hp, per)
            it = int(st.iter)
            E = float(st.E)
            checks.append((int(st.last_check), E, time.perf_counter() - t0))
            if status == L.CONVERGED:
                conv = True
                break
            if stop is not None and st.last_check >= 0 and (E - stop) / stop <= tol:
                break
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        Hf = torch.empty(n, k, dtype=torch.float32, device=dev)
        L.symnmf_get_H(h, Hf)
        L.symnmf_destroy(h)
        return {"iters": it, "seconds": el, "E": E, "converged": conv}, Hf, checks

    ref, Href, checks = solve(S32, L.F32, None, cap)
    Estar = ref["E"]
    first = next(c for c in checks if (c[1] - Estar) / Estar <= tol)
    runs = {"fp32": {"iters": first[0] + 1, "seconds": first[2], "E": first[1],
                     "note": "the reference run's first check within tolerance"}}
    bf, Hbf, _ = solve(Sbf, L.BF16, Estar, cap)
    runs["bf16"] = bf
    h32 = L.symnmf_create(S32, n, k, L.F32)
    for name, Hf in (("reference", Href), ("bf16", Hbf)):
        L.symnmf_set_H(h32, Hf)
        (ref if name == "reference" else bf)["E_on_fp32_S"] = L.symnmf_objective(h32)[1]
    L.symnmf_destroy(h32)
    out = {"metric": "time-to-tol at n=%d BF16 vs FP32 (relative objective %g)" % (n, tol),
           "bf16_seconds": bf["seconds"], "fp32_seconds": first[2],
           "bf16_iters": bf["iters"], "fp32_iters": first[0] + 1,
           "speedup_bf16_vs_fp32": first[2] / bf["seconds"],
           "E_star": Estar,
           "E_star_rule": ("E of the FP32 run stopped by the AND rule at iteration %d" % ref["iters"]
                           if ref["converged"] else
                           "E of the FP32 run capped at %d iterations (the AND rule did not hold)" % cap),
           "config": {"workload": "corr_n%d_k32_adagrad_time_to_tol" % n, "n": n, "k": k,
                      "method": "adagrad", "eta": hp.eta, "tol": tol, "cap": cap},
           "reference_run": ref, "runs": runs, "generation_seconds": t_gen}
    del S32, Sbf, inst
    torch.cuda.empty_cache()
    return out, H0


def run_time_to_tol(args):
    """Stand-alone line of time_to_tol_core (n = --ttt-n, cap = --ttt-cap)."""
    import numpy as np
    import torch
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    core, H0 = time_to_tol_core(L, dev, args.ttt_n, args.ttt_cap)
    cpu = None
    if args.cpu_baseline:
        import gen
        inst = gen.corr_factor(n=args.ttt_n, T=500, seed=0, device=dev, dtype=torch.float32,
                               materialize="torch")
        rows = np.arange(1024)
        cpu = oracle_row_rate(inst.S[:1024].double().cpu().numpy(), H0.double().cpu().numpy(), rows,
                              args.ttt_n, budget_s=min(args.cpu_budget, 10.0))
    core.update({"value": core["bf16_seconds"], "unit": "s", "higher_is_better": False, "n_gpus": 1,
                 "data": "synthetic (seeded correlation generator)",
                 "dtype": "bf16 vs f32 storage, f32 accumulate, f64 reductions", "cpu_baseline": cpu})
    return core


def run_large_fp8(args):
    """n=3e5, k=64 TPDM with a near-dominant common factor, stored FP8 E4M3
    with one power-of-two scale per 128x128 tile (90 GB), Block-SVRG
    AdaptGrow (phi0 0.75, s 5, 4096-row blocks, eta 20).  The matrix is
    generated in 8192 x 8192 chunk pairs and quantised by the library's
    quantiser without ever being held in FP32.  After the timed iterations
    the gradient is checked on two sampled 128-row tiles against the FP64
    oracle (rows of S dequantised), and the tensor-core objective against
    the exact-FP32 SIMT product on the same handle."""
    import numpy as np
    import torch
    import gen
    from oracle import symnmf_oracle as O
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, k = args.large_n, 64
    nt = -(-n // 128)
    q = torch.empty(n, n, dtype=torch.uint8, device=dev)
    scales = torch.empty(nt, nt, dtype=torch.float32, device=dev)
    tsum = torch.empty(nt, nt, dtype=torch.float64, device=dev)
    acc = {"sum": 0.0}

    def store(r0, r1, c0, c1, blk):
        L.symnmf_quantize_fp8(blk, L.F32, r1 - r0, c1 - c0, blk.stride(0), q[r0:r1, c0:c1], n,
                              scales[r0 // 128:, c0 // 128:], nt, tsum[r0 // 128:, c0 // 128:])
        w = 1.0 if c0 == r0 else 2.0
        acc["sum"] += w * float(blk.double().sum())
        if c0 != r0:
            bt = blk.t().contiguous()
            L.symnmf_quantize_fp8(bt, L.F32, c1 - c0, r1 - r0, bt.stride(0), q[c0:c1, r0:r1], n,
                                  scales[c0 // 128:, r0 // 128:], nt, tsum[c0 // 128:, r0 // 128:])

    t_gen = time.perf_counter()
    inst = gen.tpdm_groups(n=n, groups=64, T=20000, q=0.05, common=(0.6, 1.0), seed=0,
                           device=dev, block_fn=store, compute_dtype=torch.float32)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    norm_src = float(tsum.sum())
    h = L.symnmf_create(q, n, k, L.FP8E4M3)
    L.symnmf_set_tile_scales(h, scales, nt)
    norm_q = L.symnmf_get_norm(h)
    H0 = torch.tensor(gen.init_scaled(acc["sum"] / (float(n) * n), n, k, seed=0), dtype=torch.float32,
                      device=dev)
    hp = L.symnmf_hparams_default(L.BLOCK_SVRG_ADAPTGROW, eta=20.0, phi0=0.75, snapshot_period=5,
                                  block_rows=4096, tau_g=1e-30)
    L.symnmf_set_H(h, H0)
    L.symnmf_step(h, hp, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    e0.record()
    status, st = L.symnmf_step(h, hp, args.steps)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    L.symnmf_set_profiling(h, True)
    L.symnmf_step(h, hp, 10)
    torch.cuda.synchronize()
    prod_ms, prod_launches, prod_bytes, kernels = L.symnmf_get_profile(h)
    L.symnmf_set_profiling(h, False)
    trace = L.symnmf_get_trace(h)
    full = [r for r in trace if r.full]
    # sampled-row gradient check against the FP64 oracle
    G = torch.empty(n, k, dtype=torch.float32, device=dev)
    L.symnmf_grad(h, G)
    Hc = torch.empty(n, k, dtype=torch.float32, device=dev)
    L.symnmf_get_H(h, Hc)
    torch.cuda.synchronize()
    H64 = Hc.double().cpu().numpy()
    rng = np.random.default_rng(1)
    tiles = rng.choice(nt - 1, size=2, replace=False)
    rows = np.concatenate([np.arange(t * 128, t * 128 + 128) for t in tiles])
    codes = q[torch.as_tensor(rows, device=dev)].cpu().view(torch.float8_e4m3fn).double().numpy()
    sc = scales.double().cpu().numpy()
    S_rows = codes * np.repeat(sc[rows // 128], 128, axis=1)[:, :n]
    g_ref = O.gradient_rows(S_rows, H64, rows)
    g_gpu = G.double().cpu().numpy()[rows]
    terms = 4.0 * (np.linalg.norm(S_rows @ H64) + np.linalg.norm(H64[rows] @ (H64.T @ H64)))
    grad_err = float(np.linalg.norm(g_gpu - g_ref) / terms)
    f_tc, _ = L.symnmf_objective(h)
    L.symnmf_set_impl(h, 1)
    f_simt, _ = L.symnmf_objective(h)
    L.symnmf_destroy(h)
    cpu = oracle_row_rate(S_rows, H64, rows, n, budget_s=min(args.cpu_budget, 10.0)) \
        if args.cpu_baseline else None
    if cpu:
        cpu["note"] = "a full-gradient iteration; a block step reads phi S (phi = 0.75)"
    iters = int(st.iter) - args.warmup
    return {"metric": "Block-SVRG AdaptGrow iters/s at n=3e5 FP8", "value": iters / (ms / 1e3),
            "unit": "iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / max(1, iters), "higher_is_better": True,
            "dtype": "e4m3 storage (per-tile power-of-two scales), f32 accumulate, f64 reductions",
            "data": "synthetic (seeded TPDM generator, common factor)",
            "config": {"workload": "tpdm_n%d_k64_fp8_blocksvrg" % n, "n": n, "k": k, "method":
                       "block_svrg_adaptgrow", "eta": 20.0, "phi0": 0.75, "snapshot_period": 5,
                       "block_rows": 4096, "S_bytes": n * n + 4 * nt * nt},
            "product_kernels": {"ms": prod_ms, "launches": prod_launches, "S_bytes": prod_bytes,
                                "achieved_GBps": prod_bytes / (prod_ms * 1e-3) / 1e9 if prod_ms else None,
                                "kernels_per_step": kernels / 10.0},
            "last_full_E": full[-1].E if full else None, "phi": float(st.phi),
            "normS2_source": norm_src, "normS2_stored": norm_q,
            "check": {"grad_rel_err_sampled_rows": grad_err, "rows": [int(t) for t in tiles],
                      "bound_two_piece_H": 2.0 ** -8,
                      "objective_tc_vs_fp32_simt_rel_normS2": abs(f_tc - f_simt) / norm_q},
            "cpu_baseline": cpu,
            "clocks": ck, "generation_seconds": t_gen, "status": L.symnmf_status_string(status)}


def run_batch(args):
    """Batching workload: 64 instances (n ~ U{2000..30000}, k in {8,16,32,64},
    even = correlation, odd = TPDM), BF16 S, 4 random restarts each, Piecewise
    AdaGrad (eta 1, c 10, c_r 10).  The restarts of an instance are
    concatenated along N, as many per handle as fit the rank-64 kernels
    (symnmf_set_restarts: one stream of S feeds them all): all four for
    k <= 16, two handles of two for k = 32, one handle per restart for
    k = 64; each handle runs on its own stream.  The library's autotuner picks the CTA caps
    (its trial iterations are part of the solves); then the batch runs to
    the AND rule.  Reports aggregate restart-iterations/s and per-instance
    time to tolerance (first handle of the instance to converge)."""
    import numpy as np
    import torch
    import gen
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs = gen.batch_specs(args.batch_count)
    t_gen = time.perf_counter()
    mats, handles, hps, owner, streams, mult = [], [], [], [], [], []
    for i, sp in enumerate(specs):
        n, k = sp["n"], sp["k"]
        ld = -(-n // 8) * 8  # 16-byte row pitch for the tensor-core path
        if sp["kind"] == "corr":
            inst = gen.corr_planted(n=n, groups=k, T=2000, seed=sp["seed"], device=dev,
                                    dtype=torch.bfloat16, materialize="torch", ld=ld)
        else:
            inst = gen.tpdm_groups(n=n, groups=k, T=5000, q=0.05, seed=sp["seed"], device=dev,
                                   dtype=torch.bfloat16, materialize="torch", ld=ld)
        S = inst.S
        mats.append(S)
        mean = float(S[: min(n, 4096), :n].double().mean())
        R = args.restarts
        # restarts per handle: the largest divisor g of R with g k <= 64
        g = max(d for d in range(1, R + 1) if R % d == 0 and d * k <= 64) if args.joint else 1
        if g > 1:
            for r0 in range(0, R, g):
                st = torch.cuda.Stream(device=dev)
                h = L.symnmf_create_ld(S, n, ld, g * k, L.BF16)
                L.symnmf_set_stream(h, st)
                L.symnmf_set_restarts(h, g)
                H0 = np.concatenate([gen.init_scaled(mean, n, k, seed=sp["seed"], stream=r)
                                     for r in range(r0, r0 + g)], axis=1)
                L.symnmf_set_H(h, torch.tensor(H0, dtype=torch.float32, device=dev))
                handles.append(h)
                streams.append(st)
                hps.append(L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, eta=1.0, c=10.0, c_r=10.0))
                owner.append(i)
                mult.append(g)
            continue
        for r in range(R):
            st = torch.cuda.Stream(device=dev)
            h = L.symnmf_create_ld(S, n, ld, k, L.BF16)
            L.symnmf_set_stream(h, st)
            H0 = torch.tensor(gen.init_scaled(mean, n, k, seed=sp["seed"], stream=r),
                              dtype=torch.float32, device=dev)
            L.symnmf_set_H(h, H0)
            handles.append(h)
            streams.append(st)
            hps.append(L.symnmf_hparams_default(L.PIECEWISE_ADAGRAD, eta=1.0, c=10.0, c_r=10.0))
            owner.append(i)
            mult.append(1)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    t0 = time.perf_counter()
    caps = L.symnmf_batch_autotune(handles, hps, args.tune_iters)
    conv_at = [None] * len(handles)
    iters_done = [0] * len(handles)
    while True:
        status, stats = L.symnmf_batch_step(handles, hps, 10)
        now = time.perf_counter() - t0
        live = 0
        for j, stt in enumerate(stats):
            iters_done[j] = int(stt.iter)
            if stt.converged and conv_at[j] is None:
                conv_at[j] = now
            if not stt.converged:
                live += 1
        if live == 0 or max(iters_done) >= args.batch_cap:
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    total_iters = sum(it * m for it, m in zip(iters_done, mult))
    # S bytes one round (an iteration of every handle) streams, and the
    # algorithmic figure (each instance's S once per round)
    s_round = sum(2 * specs[owner[j]]["n"] ** 2 for j in range(len(handles)))
    s_alg = sum(2 * sp["n"] ** 2 for sp in specs)
    per_inst = []
    for i, sp in enumerate(specs):
        js = [j for j in range(len(handles)) if owner[j] == i]
        times = [conv_at[j] for j in js if conv_at[j] is not None]
        per_inst.append({"n": sp["n"], "k": sp["k"], "kind": sp["kind"],
                         "converged_restarts": len(times),
                         "time_to_tol_s": min(times) if times else None,
                         "iters": [iters_done[j] for j in js]})
    for h in handles:
        L.symnmf_destroy(h)
    tt = [p["time_to_tol_s"] for p in per_inst if p["time_to_tol_s"] is not None]
    return {"metric": "batched solves: aggregate iters/s (64 instances x 4 restarts, BF16, Piecewise AdaGrad)",
            "value": total_iters / wall, "unit": "iters/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 storage, f32 accumulate, f64 reductions",
            "data": "synthetic (seeded correlation / TPDM generators, seeds 0-%d)" % (len(specs) - 1),
            "config": {"workload": "batch_%dx%d_bf16_piecewise" % (len(specs), args.restarts),
                       "instances": len(specs), "restarts": args.restarts,
                       "handles": len(handles), "restarts_along_n": bool(args.joint),
                       "sum_n2": int(sum(sp["n"] ** 2 for sp in specs)),
                       "autotune_iters_per_candidate": args.tune_iters, "iteration_cap": args.batch_cap},
            "wall_s": wall, "total_iters": total_iters,
            "s_bytes_per_round": s_round, "s_bytes_per_round_algorithmic": s_alg,
            "converged_handles": sum(1 for c in conv_at if c is not None),
            "instances_converged": len(tt),
            "time_to_tol_s": {"median": float(np.median(tt)) if tt else None,
                              "max": float(max(tt)) if tt else None},
            "cta_caps": {"min": min(caps), "max": max(caps), "distinct": len(set(caps))},
            "per_instance": per_inst, "generation_seconds": t_gen}


def run_kmeans(args):
    """Spherical K-means (Lloyd on the rows of S, Sec. 6) on the n=20000 TPDM
    matrix with K = 32 clusters: Lloyd iterations/s from the same seeded
    labels (fixed work per iteration: each timed call runs one iteration,
    two streamed passes of S, and returns its objective to the host), the
    product kernel's HBM fraction, and the FP64 oracle's rate on the host."""
    import numpy as np
    import torch
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    name = {"f32": "tpdm_n20000_k32_fp32_adagrad", "bf16": "tpdm_n20000_k32_bf16_adagrad"}[
        args.km_storage]
    kind, n, Kc, dt, _, _ = WORKLOADS[name]
    S, _, _ = make_input(name, dev)
    h = L.symnmf_create(S, n, Kc, {"f32": L.F32, "bf16": L.BF16}[dt])
    stream = torch.cuda.Stream(dev)
    L.symnmf_set_stream(h, stream)
    rng = np.random.default_rng(0)
    lab = rng.integers(0, Kc, size=n)
    lab[:Kc] = np.arange(Kc)
    lab0 = torch.tensor(rng.permutation(lab), dtype=torch.int32, device=dev)
    out_l = torch.empty(n, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        L.symnmf_spkmeans(h, lab0, out_l, 1, 1e-4, trace=False)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        L.symnmf_spkmeans(h, lab0, out_l, 1, 1e-4, trace=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    L.symnmf_set_profiling(h, True)
    prof = max(5, min(args.steps, 50))
    for _ in range(prof):
        L.symnmf_spkmeans(h, lab0, out_l, 1, 1e-4, trace=False)
    torch.cuda.synchronize()
    prod_ms, prod_launches, _, kernel_launches = L.symnmf_get_profile(h)
    L.symnmf_set_profiling(h, False)
    ck = clocks.stop()
    # a full run from the same labels: iterations to the paper's stop rule
    st, Jt = L.symnmf_spkmeans(h, lab0, out_l, 200, 1e-4)
    torch.cuda.synchronize()
    impl = L.symnmf_get_impl(h)
    L.symnmf_destroy(h)
    peak, src = peaks()
    per_launch_ms = prod_ms / max(1, prod_launches)
    pass_bytes = n * n * ESIZE[dt]
    achieved = pass_bytes / (per_launch_ms * 1e-3) / 1e9
    cpu = None
    if args.cpu_baseline:
        from oracle import spkmeans_oracle as KM
        S64 = S.double().cpu().numpy()
        labs = lab0.cpu().numpy().astype(np.int64)
        KM.lloyd_step(S64, labs, Kc)
        t0 = time.perf_counter()
        it = 0
        while True:
            KM.lloyd_step(S64, labs, Kc)
            it += 1
            el = time.perf_counter() - t0
            if it >= 2 and el >= args.cpu_budget:
                break
        cpu = {"value": it / el, "unit": "Lloyd iterations/s", "cores": cpu_threads(),
               "kind": "oracle", "sample": f"{it} FP64 oracle Lloyd iterations of the same "
                                           f"workload ({el:.1f} s)"}
        del S64
    return {
        "metric": "spherical K-means Lloyd iterations/s (two streamed passes of S each)",
        "value": args.steps / (ms / 1e3), "unit": "Lloyd iterations/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16"}[dt] + " storage, f32 accumulate, f64 norms and sums",
        "data": "synthetic (seeded TPDM generator, seeded initial labels)",
        "config": {"workload": f"spkmeans_tpdm_n{n}_K{Kc}_{dt}", "n": n, "K": Kc, "storage": dt,
                   "product_impl": ["", "simt", "tcgen05"][impl],
                   "l2": "S larger than L2 (no flush needed)",
                   "run_from_same_labels": {"iterations": st.iters, "converged": st.converged,
                                            "J": st.J}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": src,
                     "kernel": "product pass (S times an n x K operand)",
                     "bytes_per_launch": pass_bytes, "ms_per_launch": per_launch_ms},
        "cpu_baseline": cpu,
        "clocks": ck,
        "gpu_launches": int(kernel_launches / prof * args.steps),
        "status": "ok",
    }


def run_dependence(args):
    """The solver's input from data on the GPU (Sec. 3): the absolute
    Pearson correlation of n = 1e5 variables over T = 500 observations of
    the 50-factor model (market loadings U[0.4, 0.8], 49 sector factors
    U[0, 0.5] at 10% density, unit Gaussian noise; seed 0), written as FP32
    (40 GB), BF16 and FP8 E4M3 with tile scales.  One line: the FP32 build's
    time, its tf32 tensor throughput against the tensor peak (the kernel is
    tensor-bound: 3 tf32 products per value pair), the S bytes written per
    second, and the BF16 / FP8 times in the config."""
    import numpy as np
    import torch
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, T = args.dep_n, 500
    rng = np.random.default_rng(0)
    A = np.zeros((n, 50), dtype=np.float32)
    A[:, 0] = rng.uniform(0.4, 0.8, size=n)
    mask = rng.random((n, 49)) < 0.1
    A[:, 1:] = np.where(mask, rng.uniform(0.0, 0.5, size=(n, 49)), 0.0)
    Z = rng.standard_normal((T, 50)).astype(np.float32)
    Y = torch.tensor(Z @ A.T, device=dev) + torch.randn(T, n, device=dev,
                                                       generator=torch.Generator(dev).manual_seed(0))
    nt = (n + 127) // 128
    stream = torch.cuda.Stream(dev)
    times = {}
    nrm = torch.zeros(1, dtype=torch.float64, device=dev)
    clocks = None
    for out, es, tdt in ((L.F32, 4, torch.float32), (L.BF16, 2, torch.bfloat16),
                         (L.FP8E4M3, 1, torch.uint8)):
        lds = (n + 16 // es - 1) // (16 // es) * (16 // es)
        S = torch.empty(n, lds, dtype=tdt, device=dev)
        sc = torch.empty(nt, nt, dtype=torch.float32, device=dev) if out == L.FP8E4M3 else None
        L.symnmf_build_dependence(Y, T, n, n, 1, out, S, lds, sc, nt if sc is not None else 0,
                                  nrm, stream)
        if out == L.F32:
            clocks = Clocks(0)
            time.sleep(0.3)
        reps = 3
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            L.symnmf_build_dependence(Y, T, n, n, 1, out, S, lds, sc,
                                      nt if sc is not None else 0, nrm, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times[out] = e0.elapsed_time(e1) / reps
        if out == L.F32:
            ck = clocks.stop()
        del S, sc
        torch.cuda.empty_cache()
    Tp = (T + 31) // 32 * 32
    ms = times[L.F32]
    # executed tensor work: the 128 x 256 tiles on or above the diagonal,
    # 3 tf32 products over Tp each
    nib, njb = (n + 127) // 128, (n + 255) // 256
    tiles = sum(min(nib, 2 * jb + 2) for jb in range(njb))
    tf32_flops = 3 * 2.0 * tiles * 128 * 256 * Tp
    achieved = tf32_flops / (ms * 1e-3) / 1e12
    d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(d.get("bf16_tflops", 1900.0))
    peak = bf16 * (1.1 / 2.25)   # tf32 dense = bf16 dense x the nominal ratio
    cpu = None
    if args.cpu_baseline:
        from oracle import dependence_oracle as DO
        m = 4000
        Ys = Y[:, :m].double().cpu().numpy()
        t0 = time.perf_counter()
        it = 0
        while True:
            DO.dependence(Ys, True)
            it += 1
            el = time.perf_counter() - t0
            if el >= min(args.cpu_budget, 10.0) and it >= 1:
                break
        cpu = {"value": it * m * m / el / 1e9, "unit": "G entries of S per s",
               "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{it} FP64 oracle builds of a {m}-variable slice (T = {T}, {el:.1f} s)"}
    return {
        "metric": f"dependence matrix build: entries of S per second (|corr|, n = {n}, T = {T})",
        "value": n * n / (ms * 1e-3) / 1e9, "unit": "G entries of S per s", "n_gpus": 1,
        "steps": 3, "warmup": 1, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 in, tf32 hi/lo products, f32 out",
        "data": "synthetic (seeded 50-factor model)",
        "config": {"workload": f"abs_corr_n{n}_T{T}", "n": n, "T": T,
                   "ms_bf16_out": times[L.BF16], "ms_fp8_out": times[L.FP8E4M3],
                   "S_write_gbs_f32": n * n * 4 / (ms * 1e-3) / 1e9},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": "measured bf16 x nominal tf32/bf16 ratio (1.1 / 2.25)",
                     "kernel": "dep_gemm (3 tf32 products per pair, upper-triangle tiles)",
                     "flops_per_launch": tf32_flops, "tiles": tiles},
        "cpu_baseline": cpu,
        "clocks": ck,
        "gpu_launches": 3 * 4,
        "status": "ok",
    }


def run_rolling_batch(args):
    """Rolling windows of several series of uneven n through the batched
    path: 4 series (n = 5000, 10000, 15000, 20000 variables of the 50-factor
    model, k = 32), windows of T = 500 sliding by 100, 6 windows each.  Per
    round every handle moves to its next window with symnmf_window_update
    (fused GPU build of |corr| + rebind, H kept as the warm start), then
    symnmf_batch_step runs 100 AdaGrad iterations on all handles, each on
    its own stream, launching every handle's iterations before any check
    waits.  Reported: aggregate windows/s."""
    import numpy as np
    import torch
    import gen
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ns, k, T, stride, W, iters = [5000, 10000, 15000, 20000], 32, 500, 100, 6, 100
    Tt = T + (W - 1) * stride
    series = []
    for i, n in enumerate(ns):
        rng = np.random.default_rng(100 + i)
        A = np.zeros((n, 50), dtype=np.float32)
        A[:, 0] = rng.uniform(0.4, 0.8, size=n)
        mask = rng.random((n, 49)) < 0.1
        A[:, 1:] = np.where(mask, rng.uniform(0.0, 0.5, size=(n, 49)), 0.0)
        Z = rng.standard_normal((Tt, 50)).astype(np.float32)
        Y = torch.tensor(Z @ A.T, device=dev) + torch.randn(
            Tt, n, device=dev, generator=torch.Generator(dev).manual_seed(100 + i))
        S = torch.empty(n, n, dtype=torch.float32, device=dev)
        st = torch.cuda.Stream(dev)
        L.symnmf_build_dependence(Y[:T], T, n, n, 1, L.F32, S, n, None, 0, None, st)
        h = L.symnmf_create(S, n, k, L.F32)
        L.symnmf_set_stream(h, st)
        L.symnmf_set_H(h, torch.tensor(gen.init_scaled(0.1, n, k, seed=i), dtype=torch.float32,
                                       device=dev))
        series.append((n, Y, S, h))
    handles = [x[3] for x in series]
    hps = [L.symnmf_hparams_default(L.ADAGRAD, eta=2.0, tau_g=1e-30) for _ in handles]
    torch.cuda.synchronize()
    clocks = Clocks(0)
    time.sleep(0.3)
    t0 = time.perf_counter()
    Es = []
    for w in range(W):
        if w > 0:
            for n, Y, S, h in series:
                L.symnmf_window_update(h, Y[w * stride:w * stride + T], T, n, 1, S, n)
        L.symnmf_batch_step(handles, hps, iters)
        Es.append([L.symnmf_get_trace(h)[-1].E for h in handles])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    for h in handles:
        L.symnmf_destroy(h)
    return {
        "metric": "rolling windows of uneven n, batched: aggregate windows/s (GPU build of |corr| "
                  "+ 100 warm-started AdaGrad iterations per window)",
        "value": len(ns) * W / wall, "unit": "windows/s", "n_gpus": 1, "steps": W, "warmup": 0,
        "ms_per_step": 1e3 * wall / W, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded 50-factor model streams)",
        "config": {"workload": "rolling_batch_corr_n5k-20k_T500_stride100_k32", "ns": ns, "k": k,
                   "T": T, "stride": stride, "windows_per_series": W,
                   "iterations_per_window": iters, "handles": len(handles)},
        "mean_E_last_window": float(np.mean(Es[-1])), "clocks": ck, "status": "ok"}


def run_rolling(args):
    """Rolling windows (the paper's next step, Sec. 8): n = 20000 variables
    of the 50-factor model (as the n = 1e5 correlation workload), windows of
    T = 500 observations sliding by 100, 10 windows.  Per window one call,
    symnmf_window_update, builds the absolute correlation on the GPU (FP32,
    into the one S buffer the handle reads) and rebinds the handle with
    ||S||^2 from the build; AdaGrad (eta 2) then runs a fixed 100
    iterations, warm-started from the previous window's H, or cold from H0.
    Reported: windows/s warm (build + solve), and the mean E after the 100
    iterations, warm against cold."""
    import numpy as np
    import torch
    import gen
    from paper_2607_24518_gb300 import build
    build.build()
    from paper_2607_24518_gb300 import symnmf as L
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, k, T, stride, W, iters = 20000, 32, 500, 100, 10, 100
    rng = np.random.default_rng(0)
    A = np.zeros((n, 50), dtype=np.float32)
    A[:, 0] = rng.uniform(0.4, 0.8, size=n)
    mask = rng.random((n, 49)) < 0.1
    A[:, 1:] = np.where(mask, rng.uniform(0.0, 0.5, size=(n, 49)), 0.0)
    Tt = T + (W - 1) * stride
    Z = rng.standard_normal((Tt, 50)).astype(np.float32)
    Y = torch.tensor(Z @ A.T, device=dev) + torch.randn(Tt, n, device=dev,
                                                        generator=torch.Generator(dev).manual_seed(0))
    S = torch.empty(n, n, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    hp = L.symnmf_hparams_default(L.ADAGRAD, eta=2.0, tau_g=1e-30)
    H0 = torch.tensor(gen.init_scaled(0.1, n, k, seed=0), dtype=torch.float32, device=dev)
    res = {}
    clocks = None
    for mode in ("cold", "warm"):
        h = None
        Es = []
        torch.cuda.synchronize()
        if mode == "warm":
            clocks = Clocks(0)
            time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for w in range(W):
            Yw = Y[w * stride:w * stride + T]
            if h is None:
                L.symnmf_build_dependence(Yw, T, n, n, 1, L.F32, S, n, None, 0, None, stream)
                h = L.symnmf_create(S, n, k, L.F32)
                L.symnmf_set_stream(h, stream)
                L.symnmf_set_H(h, H0)
            else:
                L.symnmf_window_update(h, Yw, T, n, 1, S, n)
                if mode == "cold":
                    L.symnmf_set_H(h, H0)
            _, st = L.symnmf_step(h, hp, iters)
            Es.append(L.symnmf_get_trace(h)[-1].E)
        e1.record(stream)
        torch.cuda.synchronize()
        res[mode] = (e0.elapsed_time(e1), Es)
        L.symnmf_destroy(h)
    ck = clocks.stop()
    ms_w, E_w = res["warm"]
    ms_c, E_c = res["cold"]
    return {
        "metric": "rolling-window SymNMF: windows/s (GPU build of |corr| + 100 warm-started "
                  "AdaGrad iterations per window)",
        "value": W / (ms_w / 1e3), "unit": "windows/s", "n_gpus": 1, "steps": W, "warmup": 0,
        "ms_per_step": ms_w / W, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded 50-factor model stream)",
        "config": {"workload": f"rolling_corr_n{n}_T{T}_stride{stride}_k{k}", "n": n, "k": k,
                   "T": T, "stride": stride, "windows": W, "iterations_per_window": iters,
                   "mean_E_warm": float(np.mean(E_w[1:])), "mean_E_cold": float(np.mean(E_c[1:])),
                   "E_warm": E_w, "E_cold": E_c, "windows_per_s_cold": W / (ms_c / 1e3)},
        "roofline": None, "cpu_baseline": None, "clocks": ck, "status": "ok",
    }


def run_reference(args, rank):
    """The FP64 CPU oracle on the same workload, bounded per step."""
    if rank != 0:
        return None
    import torch
    import numpy as np
    kind, n, k, dt, method, eta = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    S, H0, inst = make_input(args.workload, dev)
    S64 = S.double().cpu().numpy()
    H0_64 = torch.tensor(H0, dtype=torch.float32).double().numpy()
    del S
    from oracle import symnmf_oracle as O
    if dt == "fp8":
        S64 = O.dequantize_fp8(*O.quantize_fp8(S64))
    hp = O.HParams.paper(method)
    if eta is not None:
        hp.eta = eta
    hp.tau_g = 1e-30
    s = O.Solver(S64, H0_64, hp)
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    el = time.perf_counter() - t0
    v = args.steps / el
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded TPDM / correlation generator)",
            "config": workload_config(args.workload),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed FP64 oracle iterations after {args.warmup} warm-up"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--time-to-tol", dest="time_to_tol", action="store_true",
                    help="time to relative objective 1e-3 at n=1e5, BF16 vs FP32 (own JSON line)")
    ap.add_argument("--no-time-to-tol", dest="time_to_tol_line", action="store_false",
                    help="leave the time-to-tolerance object out of the default line")
    ap.add_argument("--ttt-n", dest="ttt_n", type=int, default=100000)
    ap.add_argument("--ttt-cap", dest="ttt_cap", type=int, default=4000)
    ap.add_argument("--large-fp8", dest="large_fp8", action="store_true",
                    help="n=3e5 k=64 FP8 Block-SVRG AdaptGrow (own JSON line)")
    ap.add_argument("--large-n", dest="large_n", type=int, default=300000)
    ap.add_argument("--batch", action="store_true",
                    help="64 instances x 4 restarts, BF16, Piecewise AdaGrad (own JSON line)")
    ap.add_argument("--batch-count", dest="batch_count", type=int, default=64)
    ap.add_argument("--restarts", type=int, default=4)
    ap.add_argument("--separate-restarts", dest="joint", action="store_false",
                    help="one handle per restart even where 4 k <= 64")
    ap.add_argument("--tune-iters", dest="tune_iters", type=int, default=10)
    ap.add_argument("--batch-cap", dest="batch_cap", type=int, default=3000)
    ap.add_argument("--rolling-batch", dest="rolling_batch", action="store_true",
                    help="rolling windows of 4 series of uneven n through the batched path "
                         "(own JSON line)")
    ap.add_argument("--rolling", action="store_true",
                    help="rolling windows: GPU |corr| build + warm-started solves (own JSON line)")
    ap.add_argument("--dependence", action="store_true",
                    help="dependence matrix build, |corr| n=1e5 T=500 (own JSON line)")
    ap.add_argument("--dep-n", dest="dep_n", type=int, default=100000)
    ap.add_argument("--kmeans", action="store_true",
                    help="spherical K-means on the n=20000 TPDM matrix, K=32 (own JSON line)")
    ap.add_argument("--km-storage", dest="km_storage", default="f32", choices=["f32", "bf16"])
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.time_to_tol:
        print(json.dumps(run_time_to_tol(args)), flush=True)
        return
    if args.large_fp8:
        print(json.dumps(run_large_fp8(args)), flush=True)
        return
    if args.batch:
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.kmeans:
        print(json.dumps(run_kmeans(args)), flush=True)
        return
    if args.dependence:
        print(json.dumps(run_dependence(args)), flush=True)
        return
    if args.rolling:
        print(json.dumps(run_rolling(args)), flush=True)
        return
    if args.rolling_batch:
        print(json.dumps(run_rolling_batch(args)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_native(args, rank, world, local_rank)
    if out:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
