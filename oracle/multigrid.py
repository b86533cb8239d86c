"""Adaptive multigrid for CP (Sections 4, 5 and 6.1), float64.

Contents, in the paper's order:
* geometric coarsening of one mode (Section 4.3),
* weighted least-squares interpolation weights (Section 4.4, Eqs. LSQinterp and
  interpweights),
* B = P^T P, its Cholesky factor L, P-hat = P L^{-T}, R-hat = P-hat^T, and the
  coarse tensor Z x_{n in I_c} R-hat^(n) (Section 4.1, Eq. ctensor_transformed),
* CP-AMG-mult, the setup V-cycle (Algorithm 1, Eqs. coarseapprox_new, CGC_new),
* CP-FAS, the solve V-cycle (Algorithm 2, Eqs. FASop, FASrhs, FASCGC),
* FMG-CP-FAS (Algorithm 3),
* the setup/solve driver with its stagnation rules (Section 6.1, Eq. stagnation).

Readings of points the paper leaves open (all listed in the design notes):
* coarsening: 0-based fine point i is coarse when i is even (the paper's odd
  1-based points), coarse label i/2; an odd fine point i interpolates from
  coarse labels (i-1)/2 and (i+1)/2, or only (i-1)/2 when i+1 = I_n.
* LS weights: w = ||A_t^(n)||_F^2 / ||G^(n)||_F^2 with G evaluated for that block
  on the current level tensor at the block's current (relaxed) factors.  A gradient
  at the rounding level of the arithmetic, ||G^(n)|| <= 1e-12 ||A^(n) Gamma^(n)||,
  counts as zero (after an ALS iteration the last-updated mode's gradient is zero in
  exact arithmetic, and its float value is noise); a zero gradient, or a ratio
  above 1e30, gives w = 1e30, so such blocks weigh equally.
* singular LS normal equations: if the 2x2 normal matrix has condition number
  above 1e12 (or is zero), the row gets weights (1/2, 1/2); a one-point stencil
  with a zero normal equation gets weight 1.
* the non-coarsened modes (n not in I_c) in the FAS right-hand side use
  Eq. FASrhs with R-hat = I, i.e. F_c = H_c(A~_c) + F - H(A), which keeps the
  exact solution a fixed point of the cycle.
* sorting/normalization: setup relaxations normalize after every ALS iteration
  and sort at the end of each relaxation call; CP-FAS normalizes and sorts after
  every BNGS iteration on the top level of the V-cycle only.
* the solve-phase stagnation test applies from the sixth solve cycle on; the
  rebuild is a "down-sweep": TFMs relaxed nu1 times and operators rebuilt on
  every level, the boot factors restricted but never relaxed or prolongated.
* the fine-level TFMs persist across setup cycles; coarse TFMs are restricted
  anew on every cycle.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .tensor import as64, ttm_modes, gradient, fas_operator, g_value, gamma, mttkrp
from .als import als, bngs_sweep

W_CAP = 1e30
COND_MAX = 1e12
G_ZERO_REL = 1e-12


@dataclasses.dataclass
class Options:
    """Parameters of Table tab:params and Section 6.1."""
    nu1_setup: int = 5
    nu2_setup: int = 5
    nuc_setup: int = 100
    n_t: int = 2
    nu1: int = 1
    nu2: int = 1
    nuc: int = 50
    gs_sweeps: int = 10
    tol: float = 1e-10
    max_cycles: int = 500
    max_setup_cycles: int = 5
    stag_eps: float = 0.1
    stag_check_after: int = 3        # setup: Eq. stagnation checked from this cycle on
    solve_stag_after: int = 5        # solve: test g_new >= g_old after this many cycles
    coarsest: tuple = ()             # I_{n,coarsest} per mode
    als_fallback: bool = False       # not in the paper: see mg_fas_solve
    max_als_iters: int = 10000       # ALS cap of Section 6.1


@dataclasses.dataclass
class Level:
    Z: np.ndarray                    # the level tensor (the input tensor on level 0)
    Ic: list                         # Ic[n] True when mode n is coarsened below this level
    P: list                          # P^(n) (I_n x I_{n,c}) or None
    Phat: list                       # P-hat^(n) = P L^{-T} or None
    Rhat: list                       # R-hat^(n) = P-hat^T or None

    @property
    def dims(self):
        return self.Z.shape


# ---------------------------------------------------------------- Section 4.3
def coarse_size(I):
    """Number of coarse points of a mode of size I (odd 1-based points are coarse)."""
    return (I + 1) // 2


def stencil(i, I):
    """Coarse labels that fine point i (0-based, odd) interpolates from."""
    s = [(i - 1) // 2]
    if i + 1 < I:
        s.append((i + 1) // 2)
    return s


# ---------------------------------------------------------------- Section 4.4
def block_weight(Z, block, n):
    """Eq. interpweights: ||A_t^(n)||^2 / ||G^(n)||^2 for one block of factor matrices, with
    G^(n) = A^(n) Gamma^(n) - Z_(n) Phi^(n) (Eq. gradEqn) treated as zero below the
    rounding level G_ZERO_REL * ||A^(n) Gamma^(n)||."""
    a2 = float(np.sum(block[n] * block[n]))
    AG = block[n] @ gamma(block, n)
    G = AG - mttkrp(Z, block, n)
    g2 = float(np.sum(G * G))
    ag2 = float(np.sum(AG * AG))
    if g2 <= (G_ZERO_REL ** 2) * ag2 or a2 / g2 > W_CAP:
        return W_CAP
    return a2 / g2


def interpolation(U, w, I):
    """P for one mode: identity rows on coarse points, and for each fine point the
    weighted least-squares fit of Eq. LSQinterp solved by normal equations.
    U is I x n_f (the vectors to fit), w the n_f weights."""
    Ic = coarse_size(I)
    P = np.zeros((I, Ic))
    for j in range(Ic):
        P[2 * j, j] = 1.0
    Uc = U[0::2, :]                 # injection: coarse label j is fine point 2j
    for i in range(1, I, 2):
        s = stencil(i, I)
        X = Uc[s, :].T              # n_f x |s|
        y = U[i, :]
        NE = X.T @ (w[:, None] * X)
        rhs = X.T @ (w * y)
        if len(s) == 1:
            P[i, s[0]] = rhs[0] / NE[0, 0] if NE[0, 0] > 0 else 1.0
        else:
            ev = np.linalg.eigvalsh(NE)
            if ev[-1] <= 0 or ev[0] <= ev[-1] / COND_MAX:
                P[i, s] = 0.5
            else:
                P[i, s] = np.linalg.solve(NE, rhs)
    return P


def transform(P):
    """B = P^T P, B = L L^T, P-hat = P L^{-T}, R-hat = P-hat^T (Section 4.1, Algorithm 1)."""
    B = P.T @ P
    L = np.linalg.cholesky(B)
    Rhat = np.linalg.solve(L, P.T)       # L^{-1} P^T
    return Rhat.T, Rhat


def build_operators(Z, A, tfms, Ic, first_cycle):
    """Interpolation operators and their Cholesky transforms (Algorithm 1) for every n in I_c."""
    N = Z.ndim
    P, Phat, Rhat = [None] * N, [None] * N, [None] * N
    for n in range(N):
        if not Ic[n]:
            continue
        cols, wts = [], []
        for T in tfms:
            cols.append(T[n])
            wts.append(np.full(T[n].shape[1], block_weight(Z, T, n)))
        if not first_cycle:
            cols.append(A[n])
            wts.append(np.full(A[n].shape[1], block_weight(Z, A, n)))
        U = np.hstack(cols)
        w = np.concatenate(wts)
        P[n] = interpolation(U, w, Z.shape[n])
        Phat[n], Rhat[n] = transform(P[n])
    return P, Phat, Rhat


def restrict_factors(A, Rhat, Ic):
    """Eq. coarseapprox_new."""
    return [Rhat[n] @ A[n] if Ic[n] else A[n].copy() for n in range(len(A))]


def coarse_tensor(Z, Rhat, Ic):
    """Eq. ctensor_transformed over the coarsened modes only: Z x_{n in I_c} R-hat^(n)."""
    return ttm_modes(Z, Rhat, [n for n in range(Z.ndim) if Ic[n]])


# ---------------------------------------------------------------- Algorithm 1
def cp_amg_mult(Z, A, tfms, opts, first_cycle, levels, relax_boot=True, upsweep=True):
    """One CP-AMG-mult V-cycle from the level whose tensor is Z.

    Appends every level visited to ``levels`` (fine to coarse).  Returns
    (updated BFMs, updated TFMs of this level).  With ``relax_boot=False,
    upsweep=False`` it is the down-sweep used to rebuild the operators."""
    Z = as64(Z)
    N = Z.ndim
    Ic = [Z.shape[n] > opts.coarsest[n] for n in range(N)]
    if any(Ic):
        tfms = [als(Z, T, opts.nu1_setup)[0] for T in tfms]                 # pre-relax TFMs
        if relax_boot:
            A = als(Z, A, opts.nu1_setup)[0]
        P, Phat, Rhat = build_operators(Z, A, tfms, Ic, first_cycle)        # P, B, L, P-hat
        levels.append(Level(Z=Z, Ic=Ic, P=P, Phat=Phat, Rhat=Rhat))
        Ac = restrict_factors(A, Rhat, Ic)                                    # coarse BFMs
        tfms_c = [restrict_factors(T, Rhat, Ic) for T in tfms]
        Zc = coarse_tensor(Z, Rhat, Ic)                                       # coarse tensor
        Ahat_c, _ = cp_amg_mult(Zc, Ac, tfms_c, opts, first_cycle, levels,  # recursion
                                relax_boot, upsweep)
        if upsweep:
            A = [Phat[n] @ Ahat_c[n] if Ic[n] else Ahat_c[n] for n in range(N)]  # CGC
            A = als(Z, A, opts.nu2_setup)[0]                                  # post-relax
    else:
        levels.append(Level(Z=Z, Ic=Ic, P=[None] * N, Phat=[None] * N, Rhat=[None] * N))
        if upsweep:
            A = als(Z, A, opts.nuc_setup)[0]                                  # coarsest
    return A, tfms


def down_sweep(Z, A, tfms, opts):
    """Rebuild the operators by the downward half of CP-AMG-mult, boot factors frozen
    (Section 6.1).  Returns (levels, updated fine-level TFMs)."""
    levels = []
    _, tfms = cp_amg_mult(Z, A, tfms, opts, first_cycle=False, levels=levels,
                          relax_boot=False, upsweep=False)
    return levels, tfms


# ---------------------------------------------------------------- Algorithm 2
def fas_rhs(levels, lvl, F, A, At):
    """The coarse right-hand side of Algorithm 2 (Eq. FASrhs): F_c = H_c(A~_c) + R-hat (F - H(A))."""
    L, Lc = levels[lvl], levels[lvl + 1]
    N = len(A)
    Fc = []
    for n in range(N):
        r = fas_operator(L.Z, A, n)
        if F is not None:
            r = F[n] - r
        else:
            r = -r
        hc = fas_operator(Lc.Z, At, n)
        Fc.append(hc + (L.Rhat[n] @ r if L.Ic[n] else r))
    return Fc


def cp_fas(levels, lvl, F, A, opts, top=0):
    """One CP-FAS V-cycle on level ``lvl`` for H({A}) = F (Algorithm 2).
    ``F=None`` means F = 0.  Normalization/sorting happen only on level ``top``."""
    L = levels[lvl]
    Z = L.Z
    finest = lvl == top
    if lvl < len(levels) - 1:
        for _ in range(opts.nu1):                                             # pre-relax
            A = bngs_sweep(Z, A, F, opts.gs_sweeps, finest)
        At = restrict_factors(A, L.Rhat, L.Ic)                                # coarse guess
        Fc = fas_rhs(levels, lvl, F, A, At)                                   # coarse RHS
        Ac = cp_fas(levels, lvl + 1, Fc, At, opts, top)                       # recursion
        A = [A[n] + (L.Phat[n] @ (Ac[n] - At[n]) if L.Ic[n] else Ac[n] - At[n])  # CGC
             for n in range(len(A))]
        for _ in range(opts.nu2):                                             # post-relax
            A = bngs_sweep(Z, A, F, opts.gs_sweeps, finest)
    else:
        for _ in range(opts.nuc):                                             # coarsest
            A = bngs_sweep(Z, A, F, opts.gs_sweeps, finest)
    return A


# ---------------------------------------------------------------- Algorithm 3
def fmg_cp_fas(levels, A_coarsest, nu, opts):
    """FMG-CP-FAS: nu ALS iterations on the coarsest level from the given start, then
    prolongate and run one CP-FAS cycle with F = 0 on each finer level."""
    Lc = len(levels) - 1
    A = als(levels[Lc].Z, A_coarsest, nu)[0]                                  # coarsest ALS
    for lvl in range(Lc - 1, -1, -1):                                         # nested iteration
        L = levels[lvl]
        A = [L.Phat[n] @ A[n] if L.Ic[n] else A[n] for n in range(len(A))]
        A = cp_fas(levels, lvl, None, A, opts, top=lvl)
    return A


# ---------------------------------------------------------------- Section 6.1
@dataclasses.dataclass
class Result:
    A: list
    tfms: list
    levels: list
    setup_cycles: int
    solve_cycles: int
    g_history: list
    restarted: bool = False
    converged: bool = False


def mg_setup(Z, A, tfms, opts):
    """Setup phase: CP-AMG-mult cycles until Eq. stagnation holds (checked from the third
    cycle on), g < tol, or ``max_setup_cycles`` cycles."""
    Z = as64(Z)
    hist = []
    levels = []
    g_prev = None
    cycles = 0
    for cycle in range(1, opts.max_setup_cycles + 1):
        levels = []
        A, tfms = cp_amg_mult(Z, A, tfms, opts, first_cycle=(cycle == 1), levels=levels)
        cycles = cycle
        g = g_value(Z, A)
        hist.append(g)
        if g < opts.tol:
            break
        if cycle >= opts.stag_check_after and g > (1.0 - opts.stag_eps) * g_prev:
            break
        g_prev = g
    return Result(A=A, tfms=tfms, levels=levels, setup_cycles=cycles, solve_cycles=0,
                  g_history=hist, converged=bool(hist and hist[-1] < opts.tol))


def mg_fas_solve(Z, levels, A, tfms, opts, cycles_done=0):
    """Solve phase: CP-FAS V-cycles until g < tol or the cycle cap, with the one-time
    stagnation rebuild of Section 6.1.

    ``opts.als_fallback`` (an addition, not in the paper): when stagnation is seen
    again after the rebuild, the new iterate is discarded and plain ALS iterations
    (normalized, g checked after each) continue from the previous iterate until
    g < tol or ``max_als_iters``; the components are then sorted."""
    Z = as64(Z)
    g_old = g_value(Z, A)
    hist = []
    solve = 0
    restarted = False
    als_iters = 0
    while g_old >= opts.tol and cycles_done + solve < opts.max_cycles:
        A_new = cp_fas(levels, 0, None, A, opts)
        solve += 1
        g_new = g_value(Z, A_new)
        hist.append(g_new)
        if solve > opts.solve_stag_after and g_new >= g_old:
            if not restarted:
                restarted = True
                levels, tfms = down_sweep(Z, A, tfms, opts)
                continue
            if opts.als_fallback:
                A, als_iters = als(Z, A, opts.max_als_iters, tol=opts.tol, g_fn=g_value)
                g_old = g_value(Z, A)
                hist.append(g_old)
                break
        A, g_old = A_new, g_new
    r = Result(A=A, tfms=tfms, levels=levels, setup_cycles=0, solve_cycles=solve,
               g_history=hist, restarted=restarted, converged=g_old < opts.tol)
    r.als_iters = als_iters
    return r


def multilevel(Z, A0, tfms, opts):
    """'Multilevel' solver of Section 6.1: setup phase then solve phase."""
    s = mg_setup(Z, A0, tfms, opts)
    r = mg_fas_solve(Z, s.levels, s.A, s.tfms, opts, cycles_done=s.setup_cycles)
    r.setup_cycles = s.setup_cycles
    r.g_history = s.g_history + r.g_history
    return r


def multilevel_fmg(Z, A0, tfms, A_coarsest0, nu, opts):
    """'Multilevel + FMG' (Section 6.1): setup cycles, one FMG-CP-FAS cycle for new boot
    factors, one down-sweep rebuild of the operators, then solve cycles."""
    s = mg_setup(Z, A0, tfms, opts)
    A = fmg_cp_fas(s.levels, A_coarsest0, nu, opts)
    levels, tfms2 = down_sweep(Z, A, s.tfms, opts)
    r = mg_fas_solve(Z, levels, A, tfms2, opts, cycles_done=s.setup_cycles + 1)
    r.setup_cycles = s.setup_cycles + 1
    r.g_history = s.g_history + r.g_history
    return r
