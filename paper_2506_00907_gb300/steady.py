"""Steady runs in two storage precisions (not part of the paper's method: it
changes how long the method runs, not its arithmetic).

A batch of cases first steps with 16-bit storage (stochastic rounding, so the
mean field follows the exact dynamics while each value carries zero-mean
rounding noise), each case until its residual stops falling, which is where the
noise takes over; the state is then converted on the GPU to FP32 storage and
every case runs on to the residual `tol`.  Cases leave the launch
(lbm_set_active) as soon as they are done in either phase.  Every step, check
and freeze is one call of the C ABI; this module only decides when to switch.
"""
import math

import numpy as np


def residuals(out):
    """Per-case relative residual sqrt(sum|dphi|^2 / sum|phi|^2) of a check
    record (slots 6 and 7)."""
    den = np.where(out[:, 7] > 0, out[:, 7], 1.0)
    return np.where(out[:, 7] > 0, np.sqrt(out[:, 6] / den), 0.0)


def run_to_plateau(sol, max_steps, interval=100, window=20, ratio=0.9, tol=0.0):
    """Step every case of `sol` until its residual (over `interval` steps)
    levels off, or is below `tol`, or max_steps are done: levelled off means
    that the mean residual of the last `window` checks is above `ratio` times
    the mean of the `window` checks before them (means over windows longer
    than the period of the slow oscillation a warm start's residual shows,
    about 1200 steps in the MHD pipes); each case is frozen when it stops,
    and all cases the call froze are resumed before it returns.
    Every case of `sol` is taken to be active on entry.  Returns (time
    steps of the batch, last residual of each case)."""
    n = sol.check().shape[0]
    hist = [[] for _ in range(n)]
    active = [True] * n
    done = 0
    last = np.full(n, math.inf)
    try:
        while done < max_steps and any(active):
            k = min(interval, max_steps - done)
            sol.step(k)
            done += k
            res = residuals(sol.check())
            for i in range(n):
                if not active[i]:
                    continue
                last[i] = res[i]
                hist[i].append(res[i])
                h = hist[i]
                if res[i] < tol or (len(h) >= 2 * window and
                                    sum(h[-window:]) > ratio * sum(h[-2 * window:-window])):
                    sol.set_active(i, False)
                    active[i] = False
    finally:
        for i in range(n):
            if not active[i]:
                sol.set_active(i, True)
    return done, last


def two_precision_steady(lo, hi, tol, max_steps, interval=100, window=20, ratio=0.9):
    """`lo` (16-bit storage, the start state already written) runs to its
    plateau; `hi` (FP32 storage, same cases and walls) takes its state and
    runs each case to the residual `tol`.  Returns a record of both phases."""
    k_lo, r_lo = run_to_plateau(lo, max_steps, interval, window, ratio, tol)
    hi.convert_from(lo)
    k_hi, r_hi = hi.run_each_to_steady(max(0, max_steps - k_lo), interval, tol)
    return {"lo_steps": int(k_lo), "lo_residual": [float(v) for v in r_lo], "hi_steps": int(k_hi),
            "hi_residual": float(r_hi)}
