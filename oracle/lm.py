"""Oracle: Levenberg-Marquardt minimiser for the per-antenna pointing offsets.

Test infrastructure only (see ``oracle/__init__``).

Paper basis: Sec. 2.2 updates a_n = a_{n-1} + f(d chi^2 / d a*) and leaves f
to the minimiser, pointing to Jacobian-based methods (Numerical Recipes);
Algorithm 1 leaves Terminate() and f() to the minimiser as well.  The reading
taken here is Levenberg-Marquardt with Marquardt's diagonal damping:

    (H_a + lam diag(H_a)) delta_a = -g_a

solved over all 2 N_ant parameters at once from the full Gauss-Newton matrix
(``solve_full``: per-antenna 2x2 diagonal blocks plus one 2x2 cross block per
baseline), or per antenna a from its diagonal block alone (``solve_block``,
all antennas updated from the same iteration, i.e. Jacobi).  Because the
pointing ramp depends on l_i + l_j, dV/dl_i and dV/dl_j are nearly equal on
every baseline and the block (Jacobi) form double-counts the common mode; it
needs the paper's loop gain (Eq. SelfCal's gamma): its step is scaled by
``block_gain`` = 0.5, which cancels the doubled common mode.  It converges
far more slowly than the full solve and is kept as an option.  A trial is accepted when it lowers chi^2
(lam /= 10), else rejected (lam *= 10).  Stop when the largest step is below
``step_tol`` (rad), when an accepted step lowers chi^2 by a relative amount
below ``chi2_rtol``, when lam exceeds ``lam_max``, when a rejected step was
already below 10 ``step_tol`` (the minimum is then found to within that, and
raising lam would only shrink the step to the tolerance), or after
``max_iter`` iterations.  Every iteration costs exactly one evaluation at the
trial point.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)


@dataclasses.dataclass
class Options:
    max_iter: int = 50
    lam0: float = 1e-3
    lam_max: float = 1e10
    lam_min: float = 1e-12
    step_tol: float = 1e-4 * ARCSEC
    chi2_rtol: float = 1e-10
    block_gain: float = 0.5       # loop gain of the per-antenna (block) step


@dataclasses.dataclass
class Report:
    n_iter: int
    n_eval: int
    reason: str
    chi2: float
    lam: float
    chi2_history: list


def block_step(g: np.ndarray, H: np.ndarray, lam: float) -> np.ndarray:
    """delta [n_ant][2] from the damped 2x2 blocks; a singular block gives 0."""
    a = H[:, 0] * (1.0 + lam)
    b = H[:, 1]
    d = H[:, 2] * (1.0 + lam)
    det = a * d - b * b
    ok = (det > 0.0) & (a > 0.0)
    delta = np.zeros_like(g)
    safe = np.where(ok, det, 1.0)
    delta[:, 0] = np.where(ok, -(d * g[:, 0] - b * g[:, 1]) / safe, 0.0)
    delta[:, 1] = np.where(ok, -(-b * g[:, 0] + a * g[:, 1]) / safe, 0.0)
    return delta


def full_step(g: np.ndarray, H: np.ndarray, lam: float) -> np.ndarray:
    Hd = H + lam * np.diag(np.diag(H))
    return -np.linalg.solve(Hd, g)


def _solve(evaluate, step, lm0, opts: Options):
    lm = np.array(lm0, dtype=np.float64, copy=True)
    chi2, g, H = evaluate(lm)
    lam = opts.lam0
    hist = [chi2]
    n_eval = 1
    reason = "max_iter"
    it = 0
    for it in range(1, opts.max_iter + 1):
        delta = step(g, H, lam).reshape(lm.shape)
        if np.max(np.abs(delta)) < opts.step_tol:
            reason = "step"
            break
        trial = lm + delta
        chi2_t, g_t, H_t = evaluate(trial)
        n_eval += 1
        if chi2_t < chi2:
            rel = (chi2 - chi2_t) / chi2 if chi2 > 0 else 0.0
            lm, chi2, g, H = trial, chi2_t, g_t, H_t
            lam = max(lam / 10.0, opts.lam_min)
            hist.append(chi2)
            if rel < opts.chi2_rtol:
                reason = "chi2"
                break
        else:
            lam *= 10.0
            if lam > opts.lam_max:
                reason = "lambda"
                break
            # a rejected step already below ten times the tolerance ends the
            # solve: raising lam would only shrink it to the tolerance
            if math.isfinite(chi2_t) and np.max(np.abs(delta)) < 10.0 * opts.step_tol:
                reason = "step"
                break
    return lm, Report(n_iter=it, n_eval=n_eval, reason=reason, chi2=chi2, lam=lam, chi2_history=hist)


def solve_block(evaluate, lm0, opts: Options = Options()):
    """``evaluate(lm) -> (chi2, g[n][2], H[n][3], ...)``; returns (lm, Report)."""
    def step(g, H, lam):
        return opts.block_gain * block_step(g, H, lam)
    return _solve(lambda p: evaluate(p)[:3], step, lm0, opts)


def solve_full(evaluate_full, lm0, opts: Options = Options()):
    """``evaluate_full(lm) -> (chi2, g[2n], H[2n][2n])``; returns (lm, Report)."""
    def step(g, H, lam):
        return full_step(g, H, lam)
    return _solve(evaluate_full, step, lm0, opts)
