"""Empirical choice of the Ewald splitting parameter on the GPU.

The paper (Sec. III, Eqs. TRDF-Topt) picks the real-space cutoff r_c, and
with it alpha = M/r_c and K = 2 alpha M, to balance the real-space cost
(~ pairs x images) against the reciprocal cost (~ pairs x k-vectors), using
per-term times fitted on its CPU.  On GB300 the per-image term (erfc, exp,
rsqrt) and the per-k term (two FMAs for the phase, six for the tensor) have
different relative costs, so the balance point moves.  This module measures
it: it times bd_build_D for a few alpha factors f (alpha = f sqrt(pi)/L, with
r_c and n2max re-derived for the same accuracy M) and returns the fastest.
The sum is alpha-independent up to the truncation error set by M, so every
candidate is an equally valid D.
"""
from __future__ import annotations

import math

import torch

from . import binding
from .inputs import SQRT_PI


def params_for_alpha(p: dict, f: float, M: float) -> dict:
    q = dict(p)
    L = q["L"]
    alpha = f * SQRT_PI / L
    q["alpha"] = alpha
    q["rc"] = M / alpha
    kc = 2.0 * alpha * M
    q["kc"] = kc
    q["n2max"] = int(math.floor((kc * L / (2.0 * math.pi)) ** 2 + 1e-9))
    return q


def tune_alpha(p: dict, R: torch.Tensor, precision: str = "fp64", M: float | None = None,
               factors=(1.0, 1.25, 1.5, 1.75, 2.0, 2.5), reps: int = 2):
    """Time bd_build_D for each alpha factor; returns (best_factor, {f: ms})."""
    if M is None:
        M = p["rc"] * p["alpha"]
    times = {}
    for f in factors:
        q = params_for_alpha(p, f, M)
        plan = binding.Plan(q, precision, max_rhs=1, max_cheb=2)
        D = plan.alloc_D()
        plan.build_D(R, D)                       # warm up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.build_D(R, D)
        e1.record()
        torch.cuda.synchronize()
        times[f] = e0.elapsed_time(e1) / reps
        del D
        plan.close()
    best = min(times, key=times.get)
    return best, times
