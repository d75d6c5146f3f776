"""Plain FP64 CPU oracle for the SymNMF solver hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this module.  It shares no code
with the CUDA path (no kernels, headers, helpers or constants); the only
common dependency is the seeded input generator module ``gen``, which holds
none of the method's arithmetic.

Every quantity is computed in float64 with numpy, written as the paper
states it, with a library matmul as the only primitive and no blocking,
fusion or reordering:

* objective      f(H) = ||S - H H^T||_F^2                      (Sec. 2, Eq. 1)
* trace form     ||S||^2 - 2 tr(H^T S H) + ||H^T H||^2          (Sec. 2.1, Eq. 2)
* gradient       grad f = 4 (H (H^T H) - S H)                  (Sec. 2.1)
* projected gradient / KKT                                      (Sec. 4.1, Eqs. 5-6)
* AND stopping rule, tau_g(n), stagnation with warm-up          (Sec. 4.1, Eqs. 7-11)
* AdaGrad, RMSprop, Piecewise AdaGrad updates                   (Appendix, Family 3)
* ADMM (H least-squares update, W = [H + U]_+, dual U)           (Appendix, Family 6)
* Row-Stochastic SVRG, Block-SVRG AdaptGrow                     (Sec. 5.1; Appendix, Family 3)
* SplitMix64 counter-based sampling of row blocks (Steele, Lea & Flood,
  OOPSLA 2014), partial Fisher-Yates selection
* optimal column matching (Kuhn-Munkres / Hungarian method) for the
  permutation ambiguity of Sec. 2 ("Identifiability").

Readings where the paper is silent (each also listed in the design notes):
epsilon of AdaGrad 1e-10 and of RMSprop 1e-8; the accumulator is updated
before the step and starts at zero; f_t, E_t and the KKT norm of iteration t
are evaluated at H_t (before the update); checks happen at t % delta == 0,
and stagnation compares E_t with E at the previous check, suppressed while
t < warmup; Piecewise "measurable loss reduction" means
E_t < E_at_previous_reset - tau * E_0, its median is the lower median of the
n*k values g_t^2, and the cooldown ends at the first check where sum(G) is at
least twice its post-reset value; stochastic methods take a full pass (that
also refreshes the snapshot mu) whenever t % s == 0 or t % delta == 0;
AdaptGrow doubles phi after 3 consecutive stagnating checks whose KKT norm is
above growth_kkt_mult * tau_g; I and J are drawn independently (streams 1
and 2), each as whole blocks of ``block_rows`` rows; the block gradient has
no reweighting (factor 2, sums over I and J, Appendix "Block-SVRG").
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field, replace

import numpy as np

ADAGRAD, RMSPROP, PIECEWISE, ROW_SVRG, BLOCK_SVRG, ADMM = 0, 1, 2, 3, 4, 5
METHOD_NAMES = {ADAGRAD: "adagrad", RMSPROP: "rmsprop", PIECEWISE: "piecewise",
                ROW_SVRG: "row_svrg", BLOCK_SVRG: "block_svrg", ADMM: "admm"}

# --------------------------------------------------------------------------
# objective, gradient, projected gradient (Sec. 2, 2.1, 4.1)
# --------------------------------------------------------------------------


def objective_explicit(S, H):
    """f(H) = ||S - H H^T||_F^2 with the n x n residual formed (Eq. 1)."""
    R = S - H @ H.T
    return float(np.sum(R * R))


def objective_trace(S, H, normS2=None):
    """||S||_F^2 - 2 tr(H^T S H) + ||H^T H||_F^2 (Eq. 2); no n x n temporary."""
    if normS2 is None:
        normS2 = float(np.sum(S * S))
    SH = S @ H
    tr = float(np.sum(H * SH))          # tr(H^T S H) = sum_ij H_ij (SH)_ij
    gram = H.T @ H
    return normS2 - 2.0 * tr + float(np.sum(gram * gram))


def gradient(S, H):
    """grad_H f = 4 (H (H^T H) - S H), formed right to left (Sec. 2.1)."""
    return 4.0 * (H @ (H.T @ H) - S @ H)


def gradient_rows(S_rows, H, rows):
    """Rows `rows` of grad_H f = 4 (H (H^T H) - S H) (Sec. 2.1), from the
    matching rows of S only (for checks at sizes where S does not fit)."""
    S_rows = np.asarray(S_rows, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    rows = np.asarray(rows)
    return 4.0 * (H[rows] @ (H.T @ H) - S_rows @ H)


def projected_gradient(H, G):
    """Projected gradient of Eq. 6: G where H > 0, min(0, G) where H == 0."""
    return np.where(H > 0, G, np.minimum(0.0, G))


def kkt_norm(H, G):
    """||grad_proj f||_F / (n k), the per-element KKT measure of Eq. 8."""
    n, k = H.shape
    return float(np.linalg.norm(projected_gradient(H, G))) / (n * k)


def tau_g_default(n):
    """Scaled KKT threshold of Eq. 9: 1e-4 * max(1, 1e4 / n)."""
    return 1e-4 * max(1.0, 1e4 / n)


def lower_median(x):
    """Lower median of a flat array: the ((N-1) // 2)-th smallest value."""
    v = np.sort(np.asarray(x, dtype=np.float64).ravel())
    return float(v[(v.size - 1) // 2])


# --------------------------------------------------------------------------
# counter-based sampling (SplitMix64; partial Fisher-Yates)
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z):
    """The SplitMix64 output function (Steele, Lea & Flood 2014)."""
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_sequence(state, count):
    """First ``count`` outputs of SplitMix64 started at ``state``."""
    out = []
    for _ in range(count):
        state = (state + _GAMMA) & _M64
        out.append(splitmix64_mix(state))
    return out


def sample_state(seed, t, stream):
    """Start state for the draws of iteration t on a stream:
    seed*gamma + t*0xBF58476D1CE4E5B9 + stream*0x94D049BB133111EB mod 2^64."""
    return (seed * _GAMMA + t * 0xBF58476D1CE4E5B9 + stream * 0x94D049BB133111EB) & _M64


def sample_blocks(seed, t, stream, nb, m):
    """m distinct block indices out of nb, sorted ascending.

    Draw d (0-based) is the (d+1)-th SplitMix64 output u_d from
    ``sample_state``; step d of a partial Fisher-Yates shuffle of 0..nb-1
    swaps position d with position d + (u_d mod (nb - d)).
    """
    m = min(m, nb)
    perm = list(range(nb))
    us = splitmix64_sequence(sample_state(seed, t, stream), m)
    for d in range(m):
        j = d + us[d] % (nb - d)
        perm[d], perm[j] = perm[j], perm[d]
    return sorted(perm[:m])


def blocks_to_rows(blocks, block_rows, n):
    rows = [np.arange(b * block_rows, min(n, (b + 1) * block_rows)) for b in blocks]
    return np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)


def sample_count(frac, n, block_rows):
    """Number of blocks covering ceil(frac * n) rows, rounded up to whole blocks."""
    nb = -(-n // block_rows)
    rows = math.ceil(frac * n)
    return min(nb, -(-rows // block_rows))


# --------------------------------------------------------------------------
# hyper-parameters and the stopping rule
# --------------------------------------------------------------------------


@dataclass
class HParams:
    method: int = ADAGRAD
    eta: float = 2.0
    eps: float = 1e-10
    alpha: float = 0.99
    mu: float = 0.5
    c: float = 10.0
    c_r: float = 10.0
    row_frac: float = 0.5
    phi0: float = 0.5
    snapshot_period: int = 10
    block_rows: int = 128
    check_interval: int = 10
    warmup: int = 50
    tau_E: float = 0.1
    tau_g: float = 0.0          # <= 0: the scaled default of Eq. 9
    tau_stag: float = 1e-5
    growth_kkt_mult: float = 3.0
    seed: int = 0
    rho: float = 500.0          # ADMM penalty

    @staticmethod
    def paper(method):
        """Phase-1 anchors of the Appendix (Family 3) and Sec. 5.1."""
        if method == ADAGRAD:
            return HParams(method=ADAGRAD, eta=2.0, eps=1e-10)
        if method == RMSPROP:
            return HParams(method=RMSPROP, eta=0.05, mu=0.5, alpha=0.99, eps=1e-8)
        if method == PIECEWISE:
            return HParams(method=PIECEWISE, eta=1.0, c=10.0, c_r=10.0, eps=1e-10)
        if method == ROW_SVRG:
            return HParams(method=ROW_SVRG, eta=2.0, row_frac=0.5, snapshot_period=10, eps=1e-10)
        if method == BLOCK_SVRG:
            return HParams(method=BLOCK_SVRG, eta=2.0, phi0=0.5, snapshot_period=2, eps=1e-10)
        if method == ADMM:
            return HParams(method=ADMM, rho=500.0)
        raise ValueError(method)


@dataclass
class Ctrl:
    """Scalar controller state carried between iterations."""
    t: int = 0
    E0: float = float("nan")
    E_prev: float = float("nan")     # E at the previous check
    have_prev: bool = False
    phi: float = 1.0
    stag_count: int = 0
    resets: int = 0
    resets_enabled: bool = True
    cooldown: bool = False
    sumA_post: float = 0.0
    E_at_reset: float = float("nan")
    converged: bool = False


@dataclass
class CheckResult:
    converged: bool
    stagnating: bool
    stag_ratio: float
    reset: bool = False
    grow: bool = False


def stopping_rule(ctrl: Ctrl, hp: HParams, n: int, t: int, E: float, kkt: float):
    """Criteria 1-3 of Sec. 4.1 (Eqs. 7, 8/9, 10) combined by Eq. 11.

    Criterion 3 compares E_t with E at the previous check and is suppressed
    (never satisfied) while t < warmup.  Returns (converged, stagnating,
    ratio); E_0 must already be set.
    """
    tau_g = hp.tau_g if hp.tau_g > 0 else tau_g_default(n)
    ratio = (ctrl.E_prev - E) / ctrl.E0 if ctrl.have_prev else float("nan")
    stagnating = bool(ctrl.have_prev and t >= hp.warmup and ratio < hp.tau_stag)
    converged = bool(E < hp.tau_E and kkt < tau_g and stagnating)
    return converged, stagnating, ratio


def controller_check(c: Ctrl, hp: HParams, n: int, t: int, E: float, kkt: float,
                     sumA: float, median_fn) -> CheckResult:
    """Scalar decisions at a check iteration t (t % delta == 0).

    E_0 is taken at the first check.  The AND rule of Eq. 11 decides
    convergence.  Piecewise AdaGrad (Sec. 5.1; appendix): the cooldown
    after a reset lasts until sum(G) reaches twice its post-reset value;
    a reset fires on stagnation while ||grad_proj||/(nk) > c_r tau_g and
    median(g_t^2) > eps, unless the previous reset brought no measurable
    loss reduction (E_t >= E_at_reset - tau E_0), which disables resets for
    good.  AdaptGrow: phi <- min(2 phi, 1) after 3 consecutive stagnating
    checks while ||grad_proj||/(nk) > growth_kkt_mult tau_g.  The caller
    applies the reset to G and sets c.sumA_post.
    """
    if t == 0 or not (c.E0 == c.E0):
        c.E0 = E
    conv, stag, ratio = stopping_rule(c, hp, n, t, E, kkt)
    out = CheckResult(converged=conv, stagnating=stag, stag_ratio=ratio)
    if conv:
        c.converged = True
        return out
    tau_g = hp.tau_g if hp.tau_g > 0 else tau_g_default(n)
    if hp.method == PIECEWISE:
        if c.cooldown and sumA >= 2.0 * c.sumA_post:
            c.cooldown = False
        if not c.cooldown and c.resets_enabled and stag and kkt > hp.c_r * tau_g:
            med = median_fn()
            if med > hp.eps:
                if c.resets > 0 and not (E < c.E_at_reset - hp.tau_stag * c.E0):
                    c.resets_enabled = False
                else:
                    out.reset = True
                    c.cooldown = True
                    c.E_at_reset = E
                    c.resets += 1
    if hp.method == BLOCK_SVRG:
        c.stag_count = c.stag_count + 1 if stag else 0
        if c.stag_count >= 3 and kkt > hp.growth_kkt_mult * tau_g and c.phi < 1.0:
            c.phi = min(2.0 * c.phi, 1.0)
            c.stag_count = 0
            out.grow = True
    c.E_prev, c.have_prev = E, True
    return out


# --------------------------------------------------------------------------
# the solver
# --------------------------------------------------------------------------


@dataclass
class Record:
    t: int
    full: bool
    f: float = float("nan")
    E: float = float("nan")
    kkt: float = float("nan")
    check: bool = False
    stag_ratio: float = float("nan")
    phi: float = 1.0
    reset: bool = False
    converged: bool = False


class Solver:
    """One SymNMF solve in float64, iteration by iteration.

    ``S`` (n x n, symmetric, float64) and ``H0`` (n x k, >= 0) are inputs;
    ``normS2`` overrides ||S||_F^2 when the objective should refer to a
    different S than the one multiplied (a quantised copy).
    """

    def __init__(self, S, H0, hp: HParams, normS2=None):
        self.S = np.asarray(S, dtype=np.float64)
        self.n, self.k = H0.shape
        self.hp = hp
        self.H = np.array(H0, dtype=np.float64)
        self.A = np.zeros_like(self.H)       # AdaGrad accumulator G_t / RMSprop v_t
        self.M = np.zeros_like(self.H)       # RMSprop momentum m_t
        self.mu = np.zeros_like(self.H)      # SVRG snapshot
        self.g = np.zeros_like(self.H)       # gradient used by the last update
        self.normS2 = float(np.sum(self.S * self.S)) if normS2 is None else float(normS2)
        self.ctrl = Ctrl(phi=hp.phi0 if hp.method == BLOCK_SVRG else 1.0)
        self.records: list[Record] = []
        self.last_I = self.last_J = None

    # ---- the kind of iteration t --------------------------------------
    def is_full(self, t):
        hp = self.hp
        if hp.method == ROW_SVRG:
            return hp.row_frac >= 1.0 or t % hp.snapshot_period == 0 or t % hp.check_interval == 0
        if hp.method == BLOCK_SVRG:
            return self.ctrl.phi >= 1.0 or t % hp.snapshot_period == 0 or t % hp.check_interval == 0
        return True

    # ---- gradients -----------------------------------------------------
    def full_gradient(self):
        return gradient(self.S, self.H)

    def row_gradient(self, t):
        """Row-Stochastic SVRG: fresh exact rows on I, snapshot mu elsewhere
        (Sec. 5.1; Appendix, Row-Stochastic AdaGrad / SVRG)."""
        hp = self.hp
        m = sample_count(hp.row_frac, self.n, hp.block_rows)
        nb = -(-self.n // hp.block_rows)
        I = blocks_to_rows(sample_blocks(hp.seed, t, 0, nb, m), hp.block_rows, self.n)
        self.last_I, self.last_J = I, None
        H = self.H
        g = self.mu.copy()
        g[I] = 4.0 * (H[I] @ (H.T @ H) - self.S[I, :] @ H)
        return g

    def block_gradient(self, t):
        """Block-SVRG AdaptGrow block estimate (Sec. 5.1; Appendix):
        R_IJ = H_I H_J^T - S_IJ, g_I += 2 R_IJ H_J, g_J += 2 R_IJ^T H_I,
        snapshot mu on rows outside I u J."""
        hp = self.hp
        nb = -(-self.n // hp.block_rows)
        m = sample_count(math.sqrt(self.ctrl.phi), self.n, hp.block_rows)
        I = blocks_to_rows(sample_blocks(hp.seed, t, 1, nb, m), hp.block_rows, self.n)
        J = blocks_to_rows(sample_blocks(hp.seed, t, 2, nb, m), hp.block_rows, self.n)
        self.last_I, self.last_J = I, J
        H = self.H
        R = H[I] @ H[J].T - self.S[np.ix_(I, J)]
        g = self.mu.copy()
        g[I] = 0.0
        g[J] = 0.0
        g[I] += 2.0 * (R @ H[J])
        g[J] += 2.0 * (R.T @ H[I])
        return g

    # ---- updates (Appendix, Families 3 and 6) -----------------------------
    def apply_update(self, g):
        hp = self.hp
        if hp.method == ADMM:
            # Appendix, Family 6, Eqs. admm_H / admm_W / admm_U: W = self.H
            # (the feasible factor the objective and the check track), the
            # scaled dual U = self.A
            W, U = self.H, self.A
            rhs = 2.0 * (self.S @ W) + hp.rho * (W - U)
            Mk = 2.0 * (W.T @ W) + hp.rho * np.eye(self.k)
            Hn = np.linalg.solve(Mk, rhs.T).T          # rhs Mk^-1 (Mk symmetric)
            Wn = np.maximum(Hn + U, 0.0)
            self.A = U + Hn - Wn
            self.H = Wn
        elif hp.method == RMSPROP:
            self.A = hp.alpha * self.A + (1.0 - hp.alpha) * g * g
            self.M = hp.mu * self.M + hp.eta * g / (np.sqrt(self.A) + hp.eps)
            self.H = np.maximum(self.H - self.M, 0.0)
        else:
            self.A = self.A + g * g
            self.H = np.maximum(self.H - hp.eta * g / (np.sqrt(self.A) + hp.eps), 0.0)

    # ---- one iteration ---------------------------------------------------
    def step(self):
        hp, c = self.hp, self.ctrl
        t = c.t
        full = self.is_full(t)
        rec = Record(t=t, full=full, phi=c.phi)
        if full:
            g = self.full_gradient()
            rec.f = objective_trace(self.S, self.H, self.normS2)
            rec.E = rec.f / self.normS2
            rec.kkt = kkt_norm(self.H, g)
            if hp.method in (ROW_SVRG, BLOCK_SVRG):
                self.mu = g.copy()
            self.last_I = self.last_J = None
        elif hp.method == ROW_SVRG:
            g = self.row_gradient(t)
        else:
            g = self.block_gradient(t)
        H_t = self.H.copy()
        self.g = g
        self.apply_update(g)
        if t % hp.check_interval == 0:
            rec.check = True
            self._check(rec, g, H_t)
        self.records.append(rec)
        if rec.converged:
            self.H = H_t            # the certified iterate is H_t
            return rec
        c.t = t + 1
        return rec

    def _check(self, rec, g, H_t):
        out = controller_check(self.ctrl, self.hp, self.n, rec.t, rec.E, rec.kkt,
                               float(np.sum(self.A)), lambda: lower_median(g * g))
        rec.stag_ratio = out.stag_ratio
        rec.converged = out.converged
        if out.reset:
            # G_i <- max(c g_i^2, c median(g^2)) (appendix, Piecewise AdaGrad)
            med = lower_median(g * g)
            self.A = np.maximum(self.hp.c * g * g, self.hp.c * med)
            self.ctrl.sumA_post = float(np.sum(self.A))
            rec.reset = True

    def run(self, iters):
        for _ in range(iters):
            rec = self.step()
            if rec.converged:
                break
        return self.records


# --------------------------------------------------------------------------
# FP8 E4M3 storage of S (OCP 8-bit floating point, E4M3: bias 7, 3 mantissa
# bits, largest finite 448, subnormal step 2^-9)
# --------------------------------------------------------------------------
E4M3_MAX = 448.0


def e4m3_round(x):
    """Round |x| <= 448 to the nearest E4M3 value, ties to even mantissa."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    m, E = np.frexp(a)                      # a = m 2^E, m in [0.5, 1)
    e = np.maximum(E - 1, -6)               # binade exponent, subnormals share 2^-6
    step = np.ldexp(1.0, e - 3)             # 3 mantissa bits
    q = np.round(a / step) * step           # numpy rounds half to even
    q = np.minimum(q, E4M3_MAX)
    return np.where(a == 0, 0.0, np.sign(x) * q)


def tile_scale(amax):
    """Power-of-two scale 2^ceil(log2(amax / 448)) of a tile (1 for amax = 0)."""
    if amax <= 0:
        return 1.0
    m, E = math.frexp(amax / E4M3_MAX)
    e = E - 1 if m == 0.5 else E
    return math.ldexp(1.0, e)


def quantize_fp8(S, tile=128):
    """Per-tile power-of-two scaled E4M3 storage: returns (q, scales) with
    S ~ scales[i // tile, j // tile] * q[i, j]."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    nt = -(-n // tile)
    q = np.zeros_like(S)
    scales = np.ones((nt, nt))
    for a in range(nt):
        for b in range(nt):
            blk = S[a * tile:(a + 1) * tile, b * tile:(b + 1) * tile]
            sc = tile_scale(float(np.max(np.abs(blk))) if blk.size else 0.0)
            scales[a, b] = sc
            q[a * tile:(a + 1) * tile, b * tile:(b + 1) * tile] = e4m3_round(blk / sc)
    return q, scales


def dequantize_fp8(q, scales, tile=128):
    n = q.shape[0]
    return q * np.kron(scales, np.ones((tile, tile)))[:n, :n]


# --------------------------------------------------------------------------
# comparison helpers: column matching and error metrics
# --------------------------------------------------------------------------


def hungarian(C):
    """Minimum-cost perfect assignment of a square cost matrix.

    Kuhn-Munkres with potentials (shortest augmenting paths), O(k^3).
    Returns perm with perm[row] = assigned column.
    """
    C = np.asarray(C, dtype=np.float64)
    k = C.shape[0]
    INF = float("inf")
    u = [0.0] * (k + 1)
    v = [0.0] * (k + 1)
    p = [0] * (k + 1)       # p[j]: row matched to column j (1-based), 0 = free
    way = [0] * (k + 1)
    for i in range(1, k + 1):
        p[0] = i
        j0 = 0
        minv = [INF] * (k + 1)
        used = [False] * (k + 1)
        while True:
            used[j0] = True
            i0 = p[j0]
            delta, j1 = INF, 0
            for j in range(1, k + 1):
                if not used[j]:
                    cur = C[i0 - 1, j - 1] - u[i0] - v[j]
                    if cur < minv[j]:
                        minv[j], way[j] = cur, j0
                    if minv[j] < delta:
                        delta, j1 = minv[j], j
            for j in range(k + 1):
                if used[j]:
                    u[p[j]] += delta
                    v[j] -= delta
                else:
                    minv[j] -= delta
            j0 = j1
            if p[j0] == 0:
                break
        while True:
            j1 = way[j0]
            p[j0] = p[j1]
            j0 = j1
            if j0 == 0:
                break
    perm = np.zeros(k, dtype=np.int64)
    for j in range(1, k + 1):
        perm[p[j] - 1] = j - 1
    return perm


def brute_force_assignment(C):
    """Exhaustive minimum-cost assignment (k! permutations; tiny k only)."""
    k = C.shape[0]
    best, arg = float("inf"), None
    for p in itertools.permutations(range(k)):
        s = sum(C[i, p[i]] for i in range(k))
        if s < best:
            best, arg = s, p
    return np.array(arg), best


def match_columns(H, H_ref):
    """Permute the columns of H to best match H_ref (Sec. 2, identifiability).

    Cost C_ab = ||H[:, a] - H_ref[:, b]||^2; returns H[:, pi] aligned to H_ref.
    """
    H = np.asarray(H, dtype=np.float64)
    H_ref = np.asarray(H_ref, dtype=np.float64)
    C = ((H[:, :, None] - H_ref[:, None, :]) ** 2).sum(axis=0)
    perm = hungarian(C)                 # column a of H -> column perm[a] of H_ref
    out = np.empty_like(H)
    out[:, perm] = H
    return out


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (den if den > 0 else 1.0)


def factor_error(H, H_ref):
    """||H Pi - H_ref||_F / ||H_ref||_F after optimal column matching."""
    return rel_err(match_columns(H, H_ref), H_ref)


def boundary_disagreement(H, H_ref):
    return int(np.sum((np.asarray(H) == 0) != (np.asarray(H_ref) == 0)))
