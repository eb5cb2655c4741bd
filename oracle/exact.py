"""Oracle: exact optimum of the DCOPF primal (problem (1)) for gap measurement.

Test infrastructure only (see the package docstring).

``ipm`` solves the LP/QP in the generator outputs p with a textbook Mehrotra
predictor-corrector primal-dual interior point method (dense normal equations),
then certifies its answer with a sandwich: the cost of its primal point (feasible to
``feas_tol``) bounds gamma* from above, the dual function (weak duality, Section 3,
eq. (5) and Remarks 1-2) at its projected multipliers bounds it from below.

``vertex_enumeration`` solves tiny LPs by brute force over basic solutions.
"""
from __future__ import annotations

import itertools
import numpy as np

from .dcopf import Net, dual_value_prices


def _problem(net: Net, loads):
    phi = net.ptdf_gen()
    fd = net.flows(np.asarray(loads, dtype=np.float64))            # H_a p_d
    # f = Phi p - fd;  rows: f <= fmax, fmin <= f, p <= pmax, pmin <= p
    h = np.concatenate([net.fmax + fd, -net.fmin - fd, net.pmax, -net.pmin])
    qd = 2.0 * net.a * net.S * net.S                               # diagonal of Q
    q = net.c * net.S
    D = float(np.sum(loads))
    return phi, fd, h, qd, q, D


def _G_mul(phi, p):
    fp = phi @ p
    return np.concatenate([fp, -fp, p, -p])


def _GT_mul(phi, v, nl, ng):
    return phi.T @ (v[:nl] - v[nl:2 * nl]) + v[2 * nl:2 * nl + ng] - v[2 * nl + ng:]


def ipm(net: Net, loads, max_iter=200, tol=1e-12, feas_tol=1e-9, verbose=False):
    """Solve min 1/2 p^T Q p + q^T p s.t. 1^T p = D, G p <= h (problem (1)).

    Returns dict(status, p, lam, mu_hi, mu_lo, ub, lb, rel_gap, iters) for the iterate
    with the tightest sandwich.  ``status`` is "optimal" when the sandwich
    (ub - lb)/|ub| <= 1e-9 holds with a primal point feasible to ``feas_tol``,
    "infeasible" when the iteration diverges, else "failed".
    """
    loads = np.asarray(loads, dtype=np.float64)
    phi, fd, h, qd, q, D = _problem(net, loads)
    nl, ng = net.n_line, net.n_gen
    m = 2 * nl + 2 * ng
    p = 0.5 * (net.pmin + net.pmax)
    if np.sum(net.pmax - net.pmin) > 0:
        t = (D - net.pmin.sum()) / (net.pmax - net.pmin).sum()
        p = net.pmin + np.clip(t, 0.05, 0.95) * (net.pmax - net.pmin)
    y = 0.0
    zscale = max(1.0, float(np.mean(np.abs(q))) if ng else 1.0)
    s = np.maximum(h - _G_mul(phi, p), 1e-1)
    z = np.full(m, zscale)
    status = "failed"
    it = 0
    best = None                    # (rel_gap, p, y, z) of the tightest feasible sandwich seen

    def sandwich(p, y, z):
        mh = np.maximum(z[:nl], 0.0)
        ml = np.maximum(z[nl:2 * nl], 0.0)
        f = phi @ p - fd
        viol = max(0.0, float(np.max(f - net.fmax, initial=0.0)),
                   float(np.max(net.fmin - f, initial=0.0)),
                   float(np.max(p - net.pmax, initial=0.0)),
                   float(np.max(net.pmin - p, initial=0.0)), abs(p.sum() - D))
        ub = net.cost(p)
        lb = dual_value_prices(net, loads, y, mh, ml)
        return (ub - lb) / max(1.0, abs(ub)), viol, ub, lb

    for it in range(1, max_iter + 1):
        rd = qd * p + q + y * np.ones(ng) + _GT_mul(phi, z, nl, ng)
        rp = p.sum() - D
        ri = _G_mul(phi, p) + s - h
        mu = float(np.dot(s, z) / m)
        nrm_d = np.linalg.norm(rd) / (1.0 + np.linalg.norm(q))
        nrm_p = (abs(rp) + np.linalg.norm(ri)) / (1.0 + np.linalg.norm(h) + abs(D))
        if verbose:
            print(it, nrm_d, nrm_p, mu)
        if not (np.all(np.isfinite(p)) and np.all(np.isfinite(z)) and np.isfinite(y)):
            status = "stalled"
            break
        if it >= 3:
            rel, viol, _, _ = sandwich(p, y, z)
            if viol <= feas_tol and (best is None or rel < best[0]):
                best = (rel, p.copy(), y, z.copy())
            if best is not None and best[0] <= 1e-12:
                status = "converged"
                break
        if nrm_d < tol and nrm_p < tol and mu < tol * (1.0 + abs(float(np.dot(q, p)))) / m:
            status = "converged"
            break
        if not np.isfinite(mu) or mu > 1e30 or np.linalg.norm(p) > 1e12:
            status = "infeasible"
            break
        w = z / np.maximum(s, 1e-300)
        if not np.all(np.isfinite(w)):
            status = "stalled"
            break
        K = (phi.T * (w[:nl] + w[nl:2 * nl])) @ phi
        K[np.diag_indices(ng)] += w[2 * nl:2 * nl + ng] + w[2 * nl + ng:] + qd
        try:
            Lc = np.linalg.cholesky(K)
        except np.linalg.LinAlgError:
            try:                        # regularise once; FP64 has run out of digits
                Lc = np.linalg.cholesky(K + np.eye(ng) * (1e-12 * np.trace(K) / ng))
            except np.linalg.LinAlgError:
                status = "stalled"
                break

        def ksolve(r):
            return np.linalg.solve(Lc.T, np.linalg.solve(Lc, r))

        ones = np.ones(ng)
        try:
            Kinv1 = ksolve(ones)
        except np.linalg.LinAlgError:
            status = "stalled"
            break
        s1k1 = float(ones @ Kinv1)

        def newton(rc):
            rhs = -rd - _GT_mul(phi, w * ri - rc / s, nl, ng)
            Kr = ksolve(rhs)
            dy = (float(ones @ Kr) + rp) / s1k1
            dp = Kr - Kinv1 * dy
            dz = w * (_G_mul(phi, dp) + ri) - rc / s
            ds = -(rc + s * dz) / z
            return dp, dy, ds, dz

        def maxstep(v, dv):
            neg = dv < 0
            return min(1.0, float(np.min(-v[neg] / dv[neg]))) if np.any(neg) else 1.0

        # predictor (affine scaling); a singular step means FP64 has run out of digits
        try:
            dp, dy, ds, dz = newton(s * z)
        except np.linalg.LinAlgError:
            status = "stalled"
            break
        a_aff = min(maxstep(s, ds), maxstep(z, dz))
        mu_aff = float(np.dot(s + a_aff * ds, z + a_aff * dz) / m)
        sigma = (mu_aff / mu) ** 3
        # corrector
        try:
            dp, dy, ds, dz = newton(s * z + ds * dz - sigma * mu)
        except np.linalg.LinAlgError:
            status = "stalled"
            break
        a = 0.99 * min(maxstep(s, ds), maxstep(z, dz))
        p = p + a * dp
        y = y + a * dy
        s = s + a * ds
        z = z + a * dz
    if status != "infeasible" and best is not None:
        _, p, y, z = best
    mu_hi = np.maximum(z[:nl], 0.0)
    mu_lo = np.maximum(z[nl:2 * nl], 0.0)
    rel, viol, ub, lb = sandwich(p, y, z)
    if status != "infeasible":
        status = "optimal" if (rel <= 1e-9 and viol <= feas_tol) else "failed"
    return dict(status=status, p=p, lam=float(y), mu_hi=mu_hi, mu_lo=mu_lo, ub=ub, lb=lb,
                rel_gap=rel, viol=viol, iters=it, gamma=0.5 * (ub + lb))


def vertex_enumeration(net: Net, loads, tol=1e-9):
    """Brute-force LP optimum of problem (1): every basic solution made of the power
    balance row and n_g - 1 active inequality rows, keeping the cheapest feasible one.
    Only for linear costs and tiny cases (n_g <= 5, n_l <= 8).  Returns (gamma, p)."""
    assert not net.qp
    loads = np.asarray(loads, dtype=np.float64)
    phi, fd, h, _, q, D = _problem(net, loads)
    nl, ng = net.n_line, net.n_gen
    G = np.vstack([phi, -phi, np.eye(ng), -np.eye(ng)])
    best, best_p = np.inf, None
    for rows in itertools.combinations(range(G.shape[0]), ng - 1):
        Ab = np.vstack([np.ones((1, ng)), G[list(rows)]])
        if abs(np.linalg.det(Ab)) < 1e-12:
            continue
        p = np.linalg.solve(Ab, np.concatenate([[D], h[list(rows)]]))
        if np.all(G @ p <= h + tol):
            val = float(q @ p)
            if val < best:
                best, best_p = val, p
    return best, best_p
