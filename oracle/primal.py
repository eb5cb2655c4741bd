"""Oracle: primal recovery, i.e. a feasible dispatch and an upper bound from a dual
point, in plain FP64 numpy.

Test infrastructure only (see the package docstring).

The paper certifies its lower bounds against optima from a commercial solver; it
builds no primal point. This module is the recovery the library implements for a gap
without a stored optimum. Every step is elementary, and any point it returns is
feasible, so its cost is an upper bound on gamma* (weak duality, Section 3,
Remarks 1-2: every dual value is at most every feasible cost).

Steps, at a dual point (lambda, mu_hi, mu_lo):

1. Minimiser. Bus prices nu = lambda 1 + H_a^T (mu_hi - mu_lo). p_j(delta) is the
   closed-form minimiser of cost_j(p) + (nu_bus(j) + delta) p over [pmin_j, pmax_j]
   (eq. (6) / eq. (16), as in dcopf.inner_min), for a uniform price shift delta.
2. Balance. P(delta) = sum_j p_j(delta) does not increase with delta. Bisection on
   delta brackets the demand D between two adjacent shifts, P(lo) >= D >= P(hi). The
   balanced dispatch is the convex combination
   p_bal = p(hi) + phi (p(lo) - p(hi)) with phi = (D - P(hi)) / (P(lo) - P(hi)).
   It lies in the box, and its sum is D.
3. Reference. p_ref is a dispatch of the caller. The default is the proportional
   dispatch pmin + theta (pmax - pmin). It must meet the box and the balance (to
   tol, the balance relative to max(1, D)) and the flow limits (to tol); otherwise
   there is no bound (status 2).
4. Line repair. The feasible set is convex. So p_ub = (1 - t) p_bal + t p_ref is
   feasible for the smallest t in [0, 1] that pulls every violated flow of p_bal back
   to its limit: for f_l(p_bal) > fmax_l, t >= (f_l(p_bal) - fmax_l) /
   (f_l(p_bal) - f_l(p_ref)), and likewise below fmin_l.
5. Bound. ub = cost(p_ub). The flows of p_ub are recomputed, and their largest
   violation (rounding only) is returned.

A caller may instead pass a candidate dispatch p_cand in the box (for example the
weighted mean of the minimisers over a solve, dcopf.solve's mean_dispatch). It then
replaces steps 1-2 and is balanced by moving it towards a corner of the box: towards
pmax when its total is below the demand, towards pmin when above,
p_bal = p_cand + phi (corner - p_cand), with phi in [0, 1] chosen to meet the demand.
"""
from __future__ import annotations

import numpy as np

from .dcopf import Net, inner_min


def _marginal(net: Net, p):
    """d cost_j / dp at p ($/h per p.u.)."""
    return net.c * net.S + 2.0 * net.a * net.S * net.S * p


def balanced_minimiser(net: Net, nu_gen, demand, max_steps=2000):
    """Steps 1-2: the box minimiser at prices nu_gen + delta, balanced to ``demand`` by
    bisection on the uniform shift delta and a convex combination of the two
    bracketing dispatches. Returns (p_bal, delta_lo, delta_hi), or None when the
    demand is outside [sum pmin, sum pmax]."""
    if demand > net.pmax.sum() or demand < net.pmin.sum():
        return None
    nu_gen = np.asarray(nu_gen, dtype=np.float64)
    # all units at pmax for delta <= lo, all at pmin for delta >= hi
    lo = float(np.min(-_marginal(net, net.pmax) - nu_gen)) - 1.0
    hi = float(np.max(-_marginal(net, net.pmin) - nu_gen)) + 1.0

    def disp(delta):
        return inner_min(net, nu_gen + delta)[0]

    for _ in range(max_steps):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if disp(mid).sum() >= demand:
            lo = mid
        else:
            hi = mid
    p_lo, p_hi = disp(lo), disp(hi)
    P_lo, P_hi = p_lo.sum(), p_hi.sum()
    phi = (demand - P_hi) / (P_lo - P_hi) if P_lo > P_hi else 0.0
    phi = min(1.0, max(0.0, phi))
    return p_hi + phi * (p_lo - p_hi), lo, hi


def balance_candidate(net: Net, p_cand, demand):
    """A box dispatch moved towards pmax (total below the demand) or pmin (above) until
    its total meets the demand; None when the demand is outside the box totals."""
    if demand > net.pmax.sum() or demand < net.pmin.sum():
        return None
    p = np.clip(np.asarray(p_cand, dtype=np.float64), net.pmin, net.pmax)
    s = p.sum()
    if s < demand:
        room = net.pmax.sum() - s
        phi = (demand - s) / room if room > 0 else 0.0
        return p + min(1.0, phi) * (net.pmax - p)
    room = s - net.pmin.sum()
    phi = (s - demand) / room if room > 0 else 0.0
    return p - min(1.0, phi) * (p - net.pmin)


def proportional_dispatch(net: Net, demand):
    """pmin + theta (pmax - pmin) with the theta that meets the demand."""
    span = net.pmax.sum() - net.pmin.sum()
    theta = (demand - net.pmin.sum()) / span if span > 0 else 0.0
    return net.pmin + theta * (net.pmax - net.pmin)


def violation(net: Net, f):
    """Largest flow-limit violation (0 when feasible)."""
    return float(max(0.0, np.max(f - net.fmax, initial=0.0), np.max(net.fmin - f, initial=0.0)))


def recover(net: Net, loads, lam, mu_hi, mu_lo, p_ref=None, tol=1e-9, p_cand=None):
    """Steps 1-5 (steps 1-2 replaced by balance_candidate when p_cand is given).
    Returns a dict with ub ($/h, inf without a bound), p (the dispatch), t (the weight
    of the reference), status (0 bound, 1 demand outside the box, 2 reference
    infeasible) and maxviol (largest flow violation of p)."""
    loads = np.asarray(loads, dtype=np.float64)
    D = float(loads.sum())
    out = dict(ub=np.inf, p=None, t=np.nan, status=1, maxviol=np.nan)
    if p_cand is None:
        eta = np.asarray(mu_hi, dtype=np.float64) - np.asarray(mu_lo, dtype=np.float64)
        nu_gen = lam + net.prices(eta)[net.gen_bus]
        bal = balanced_minimiser(net, nu_gen, D)
        if bal is None:
            return out
        p_bal = bal[0]
    else:
        p_bal = balance_candidate(net, p_cand, D)
        if p_bal is None:
            return out
    p_ref = proportional_dispatch(net, D) if p_ref is None else np.asarray(p_ref, dtype=np.float64)

    def flows(p):
        return net.flows(net.gen_injection(p) - loads)

    if (np.any(p_ref < net.pmin - tol) or np.any(p_ref > net.pmax + tol)
            or abs(p_ref.sum() - D) > tol * max(1.0, D)):
        out.update(status=2)
        return out
    f_bal, f_ref = flows(p_bal), flows(p_ref)
    if violation(net, f_ref) > tol:
        out.update(status=2)
        return out
    t = 0.0
    for fb, fr, hi, lo in zip(f_bal, f_ref, net.fmax, net.fmin):
        if fb > hi:
            t = max(t, (fb - hi) / (fb - fr) if fr < fb else 1.0)
        if fb < lo:
            t = max(t, (lo - fb) / (fr - fb) if fr > fb else 1.0)
    t = min(1.0, t)
    p = (1.0 - t) * p_bal + t * p_ref
    out.update(ub=net.cost(p), p=p, t=t, status=0, maxviol=violation(net, flows(p)))
    return out
