"""Transition-point search from the Gu-Wen ratio X (Sec. III D, eq. X).

X = (Tr A)^2 / Tr(A^2) of the coarse tensor counts the degenerate ground states: about 2
in the Z2-ordered phase (large beta), about 1 in the disordered phase.  The search
evaluates X after a fixed number of coarse-graining steps on a grid of couplings, one
batched instance per coupling (all steps in the library's kernels), keeps the grid
interval where X crosses the level 1.5, and refines it with a finer grid.  The estimate
is the linear interpolation of the crossing inside the last interval, with the interval
itself as its resolution (the error bars of the paper's T_c-versus-D figure are the
resolution of such a search).

`refine` is host logic only (it takes any evaluator); `tc_scan` binds it to the batched
library calls.
"""
from __future__ import annotations

import numpy as np


def bracket_crossing(betas, X, level: float = 1.5):
    """(i, i+1): the first adjacent pair of couplings with X[i] < level <= X[i+1]
    (disordered below, ordered above), or None when X does not cross upward."""
    X = np.asarray(X, dtype=np.float64)
    for i in range(len(X) - 1):
        if X[i] < level <= X[i + 1]:
            return i, i + 1
    return None


def refine(evaluate, beta_lo: float, beta_hi: float, points: int = 8, rounds: int = 2,
           level: float = 1.5) -> dict:
    """Search [beta_lo, beta_hi] for the crossing of X = level.

    evaluate(betas) returns X at each coupling.  Each round evaluates `points` evenly
    spaced couplings in the current interval (ends included) and keeps the sub-interval
    that holds the crossing.  Returns beta_c (None if X does not cross in the first
    grid), the final interval and every evaluated (betas, X) round."""
    if points < 2 or rounds < 1 or not beta_hi > beta_lo:
        raise ValueError("need points >= 2, rounds >= 1 and beta_hi > beta_lo")
    lo, hi = float(beta_lo), float(beta_hi)
    history = []
    beta_c = None
    for _ in range(rounds):
        betas = np.linspace(lo, hi, points)
        X = np.asarray(evaluate(betas), dtype=np.float64)
        history.append((betas, X))
        br = bracket_crossing(betas, X, level)
        if br is None:
            if beta_c is None:
                return {"beta_c": None, "interval": (lo, hi), "history": history}
            break                        # keep the previous round's estimate
        i, j = br
        lo, hi = float(betas[i]), float(betas[j])
        beta_c = lo + (level - X[i]) / (X[j] - X[i]) * (hi - lo)
    return {"beta_c": beta_c, "interval": (lo, hi), "history": history}


def tc_scan(beta_lo: float, beta_hi: float, D: int, nsteps: int, points: int = 8,
            rounds: int = 2, lanes: int = 4, precision: int = 0, model: int = 0,
            h: float = 0.0, level: float = 1.5) -> dict:
    """T_c of the 4D model `model` (0 Ising, q >= 3 the Z_q clock model) at bond
    dimension D from X after `nsteps` steps (lattice of 2^nsteps sites), on the GPU.
    Returns the refine() result plus T_c = 1/beta_c and the T interval."""
    from . import _lib as L

    def evaluate(betas):
        n = len(betas)
        L.trg_batch_create([model] * n, list(betas), [h] * n, [D] * n, lanes=min(lanes, n),
                           precision=precision)
        try:
            L.trg_batch_step(nsteps)
            return L.trg_batch_gu_wen(n)
        finally:
            L.trg_batch_free()

    out = refine(evaluate, beta_lo, beta_hi, points, rounds, level)
    bc = out["beta_c"]
    out["T_c"] = None if bc is None else 1.0 / bc
    out["T_interval"] = (1.0 / out["interval"][1], 1.0 / out["interval"][0])
    return out
