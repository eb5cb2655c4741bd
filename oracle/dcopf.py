"""Oracle: DCOPF dual function, supergradient and ascent rules in plain FP64 numpy.

Test infrastructure only (see the package docstring).

Notation (Section 2, problem (1)): n_b buses, n_l lines, n_g generators.  For an
injection vector y (generation minus load, p.u.) the line flows are f = H_a y with
H = Omega E (E^T Omega E)^{-1} the PTDF, E the reduced incidence matrix and H_a the
PTDF with a zero column for the slack bus.  The oracle never forms H: it applies
H_a and H_a^T by solving the reduced Laplacian E^T Omega E with a dense Cholesky.

Costs: generator j at output p (p.u.) costs a_j (S p)^2 + b_j S p in $/h, S = base MVA
(a_j = 0 for linear costs).  Multipliers: lambda (scalar) for the power balance,
mu_hi >= 0 for f <= flow_max and mu_lo >= 0 for flow_min <= f.
"""
from __future__ import annotations

import numpy as np


class Net:
    """A network in the oracle's own representation, built from plain arrays."""

    def __init__(self, n_bus, line_from, line_to, line_b, flow_max, flow_min, gen_bus,
                 pmin, pmax, cost_lin, cost_quad=None, base_mva=100.0, slack_bus=0):
        self.n_bus = int(n_bus)
        self.lf = np.asarray(line_from, dtype=np.int64)
        self.lt = np.asarray(line_to, dtype=np.int64)
        self.b = np.asarray(line_b, dtype=np.float64)
        self.fmax = np.asarray(flow_max, dtype=np.float64)
        self.fmin = (-self.fmax if flow_min is None
                     else np.asarray(flow_min, dtype=np.float64))
        self.gen_bus = np.asarray(gen_bus, dtype=np.int64)
        self.pmin = np.asarray(pmin, dtype=np.float64)
        self.pmax = np.asarray(pmax, dtype=np.float64)
        self.S = float(base_mva)
        self.c = np.asarray(cost_lin, dtype=np.float64)
        self.a = (np.zeros_like(self.c) if cost_quad is None
                  else np.asarray(cost_quad, dtype=np.float64))
        self.qp = cost_quad is not None
        self.slack = int(slack_bus)
        self.n_line = len(self.lf)
        self.n_gen = len(self.gen_bus)
        # Reduced incidence E (Section 2, below problem (1)): row l has +1 at the
        # from-bus and -1 at the to-bus; the slack column is removed.  E^T Omega E is
        # factorised once with SuperLU (scipy), a library primitive.
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        rows = np.repeat(np.arange(self.n_line), 2)
        cols = np.stack([self.lf, self.lt], 1).ravel()
        vals = np.tile(np.array([1.0, -1.0]), self.n_line)
        inc = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_line, self.n_bus))
        self.keep = np.array([i for i in range(self.n_bus) if i != self.slack], dtype=np.int64)
        self.E = inc[:, self.keep].tocsr()
        lap = (self.E.T @ sp.diags(self.b) @ self.E).tocsc()      # E^T Omega E
        self.lu = spl.splu(lap)

    @classmethod
    def from_dict(cls, d):
        return cls(**{k: d[k] for k in ("n_bus", "line_from", "line_to", "line_b",
                                        "flow_max", "flow_min", "gen_bus", "pmin",
                                        "pmax", "cost_lin", "cost_quad", "base_mva",
                                        "slack_bus")})

    # ------------------------------------------------------------ operators
    def _solve_lap(self, rhs):
        return self.lu.solve(np.asarray(rhs, dtype=np.float64))

    def flows(self, inj):
        """f = H_a y for a bus injection vector y (Section 2, constraint (1c)).

        ``inj`` may be [n_bus] or [n_bus, k] (k injections at once)."""
        inj = np.asarray(inj, dtype=np.float64)
        theta = self._solve_lap(inj[self.keep])
        ft = self.E @ theta
        return (self.b[:, None] * ft) if ft.ndim == 2 else self.b * ft

    def prices(self, eta):
        """z = H_a^T eta: bus prices of a line-multiplier vector; z_slack = 0."""
        zr = self._solve_lap(self.E.T @ (self.b * np.asarray(eta, dtype=np.float64)))
        z = np.zeros(self.n_bus)
        z[self.keep] = zr
        return z

    def gen_injection(self, p):
        y = np.zeros(self.n_bus)
        np.add.at(y, self.gen_bus, p)
        return y

    def ptdf_gen(self):
        """Phi = H_a G: the PTDF columns at each generator's bus (n_l x n_g)."""
        if self.n_gen == 0:
            return np.zeros((self.n_line, 0))
        e = np.zeros((self.n_bus, self.n_gen))
        e[self.gen_bus, np.arange(self.n_gen)] = 1.0
        return self.flows(e)

    # ------------------------------------------------------------ costs
    def cost(self, p):
        """Total generation cost in $/h (objective of problem (1), plus p^T M p for QPs)."""
        sp = self.S * np.asarray(p)
        return float(np.sum(self.a * sp * sp + self.c * sp))

    def gen_cost(self, p):
        sp = self.S * np.asarray(p)
        return self.a * sp * sp + self.c * sp


def inner_min(net: Net, nu):
    """Per-generator minimiser of cost_j(p) + nu_j p over [pmin_j, pmax_j].

    This is the closed-form inner minimisation of the Lagrangian (Section 3.1,
    eq. (6): over the l-infinity ball the minimum of a linear function is attained
    at a vertex, i.e. x = -sign(w); Section 3.2, eq. (16): for the quadratic cost the
    unconstrained stationary point clipped to the box).  A zero linear coefficient
    (LP tie, sign(0)) takes the box midpoint, x = 0 in normalised form.
    Returns (p_star, min_value_per_gen).
    """
    nu = np.asarray(nu, dtype=np.float64)
    lin = net.c * net.S + nu                       # d(cost + nu p)/dp at p = 0, $/h per p.u.
    if net.qp:
        quad = net.a * net.S * net.S               # coefficient of p^2
        p = np.clip(-lin / (2.0 * quad), net.pmin, net.pmax)
    else:
        p = np.where(lin > 0, net.pmin, np.where(lin < 0, net.pmax, 0.5 * (net.pmin + net.pmax)))
    vals = net.gen_cost(p) + nu * p
    return p, vals


def dual_parts(net: Net, loads, lam, mu_hi, mu_lo):
    """Shared pieces: eta = mu_hi - mu_lo, bus prices nu = lambda + H_a^T eta and the
    minimiser.  mu are used as given (callers project first)."""
    eta = np.asarray(mu_hi, dtype=np.float64) - np.asarray(mu_lo, dtype=np.float64)
    z = net.prices(eta)
    nu_bus = lam + z
    p, vals = inner_min(net, nu_bus[net.gen_bus])
    return eta, z, nu_bus, p, vals


def dual_value_lagrangian(net: Net, loads, lam, mu_hi, mu_lo):
    """Formula (i): the Lagrangian (eq. (3)) evaluated at the inner minimiser.

    g = sum_j cost_j(p*_j) + lambda (1^T p* - 1^T p_d) + mu_hi^T (f - f_max)
        + mu_lo^T (f_min - f),  with f = H_a (G p* - p_d).
    """
    loads = np.asarray(loads, dtype=np.float64)
    _, _, _, p, _ = dual_parts(net, loads, lam, mu_hi, mu_lo)
    f = net.flows(net.gen_injection(p) - loads)
    return (net.cost(p) + lam * (p.sum() - loads.sum())
            + float(np.dot(mu_hi, f - net.fmax)) + float(np.dot(mu_lo, net.fmin - f)))


def dual_value_prices(net: Net, loads, lam, mu_hi, mu_lo):
    """Formula (ii): adjoint-only form of the dual function G (eq. (4)).

    g = sum_j min_p [cost_j(p) + nu_bus(j) p] - nu^T p_d - mu_hi^T f_max + mu_lo^T f_min,
    nu = lambda 1 + H_a^T (mu_hi - mu_lo).
    """
    loads = np.asarray(loads, dtype=np.float64)
    _, _, nu_bus, _, vals = dual_parts(net, loads, lam, mu_hi, mu_lo)
    return (float(vals.sum()) - float(np.dot(nu_bus, loads))
            - float(np.dot(mu_hi, net.fmax)) + float(np.dot(mu_lo, net.fmin)))


def canonical(net: Net, loads):
    """The normalised canonical problem (eq. (2)) built by Appendix A1.

    x = M_sigma^{-1}(p - m_mu) lies in the unit l-infinity ball.  Returns a dict with
    the diagonal M, the linear term c, the single balance row A and its b, the flow
    rows C = [Phi M_sigma; -Phi M_sigma] and d, and the constant dropped by the
    substitution (ambiguity: eq. (6) and eq. (16) omit it; it is added back here so
    that the dual value bounds the generation cost itself).
    """
    loads = np.asarray(loads, dtype=np.float64)
    sig = 0.5 * (net.pmax - net.pmin)
    mid = 0.5 * (net.pmax + net.pmin)
    S = net.S
    M = net.a * S * S * sig * sig
    c = sig * (net.c * S + 2.0 * net.a * S * S * mid)
    const = float(np.sum(net.a * S * S * mid * mid + net.c * S * mid))
    phi = net.ptdf_gen()
    fd = net.flows(loads)                                 # H_a p_d
    f_mid = phi @ mid - fd                                # flows at the mid-box dispatch
    A = sig[None, :]
    b = np.array([loads.sum() - mid.sum()])
    C = np.vstack([phi * sig[None, :], -phi * sig[None, :]])
    d = np.concatenate([net.fmax - f_mid, f_mid - net.fmin])
    return dict(M=M, c=c, A=A, b=b, C=C, d=d, const=const, sigma=sig, mid=mid)


def dual_value_canonical_lp(can, lam, mu):
    """eq. (6): g_l = -||c + A^T lambda + C^T mu||_1 - lambda^T b - mu^T d (+ constant)."""
    w = can["c"] + can["A"].T @ np.atleast_1d(lam) + can["C"].T @ mu
    return float(-np.abs(w).sum() - np.dot(np.atleast_1d(lam), can["b"]) - np.dot(mu, can["d"])
                 + can["const"])


def dual_value_canonical_qp(can, lam, mu, s):
    """eq. (16): g_q = -||c + A^T lambda + C^T mu - sqrt(M) s||_1 - s^T s / 4
    - lambda^T b - mu^T d (+ constant), s free."""
    w = can["c"] + can["A"].T @ np.atleast_1d(lam) + can["C"].T @ mu - np.sqrt(can["M"]) * s
    return float(-np.abs(w).sum() - 0.25 * np.dot(s, s)
                 - np.dot(np.atleast_1d(lam), can["b"]) - np.dot(mu, can["d"]) + can["const"])


def supergradient(net: Net, loads, lam, mu_hi, mu_lo):
    """Supergradient of g at (lambda, mu): the primal residuals at the minimiser.

    d/d lambda = 1^T p* - 1^T p_d;  d/d mu_hi = f - f_max;  d/d mu_lo = f_min - f
    (Algorithm 1, gradient lines, with the sign reading A x* - b, C x* - d).
    """
    loads = np.asarray(loads, dtype=np.float64)
    _, _, _, p, _ = dual_parts(net, loads, lam, mu_hi, mu_lo)
    f = net.flows(net.gen_injection(p) - loads)
    return p.sum() - loads.sum(), f - net.fmax, net.fmin - f, p, f


def evaluate(net: Net, loads, lam, mu_hi, mu_lo):
    """Dual value (formula (i)) and supergradient in one call."""
    gl, ghi, glo, p, f = supergradient(net, loads, lam, mu_hi, mu_lo)
    val = (net.cost(p) + lam * gl + float(np.dot(mu_hi, ghi)) + float(np.dot(mu_lo, glo)))
    return val, gl, ghi, glo, p


def evaluate_qp_s(net: Net, can, loads, lam, mu_hi, mu_lo, s):
    """The QP dual of eq. (16) with s as a variable (Section 3.2, Remark 2), in the
    canonical form of eq. (2) built by Appendix A1 (``can = canonical(net, loads)``):

        g_q(lambda, mu, s) = -||c + A^T lambda + C^T mu - sqrt(M) s||_1 - s^T s / 4
                             - lambda^T b - mu^T d (+ the constant of the substitution).

    The inner minimiser over the unit box is x* = -sign(w), w = c + A^T lambda + C^T mu -
    sqrt(M) s (0 where w = 0), and the supergradient is (A x* - b, C x* - d,
    -sqrt(M) x* - s / 2).  Returns (value, g_lambda, g_mu_hi, g_mu_lo, g_s, p*) with the
    mu gradients split into the two flow-limit rows of C (f - f_max, f_min - f)."""
    mu = np.concatenate([np.asarray(mu_hi, dtype=np.float64), np.asarray(mu_lo, dtype=np.float64)])
    s = np.asarray(s, dtype=np.float64)
    sq = np.sqrt(can["M"])
    w = can["c"] + can["A"].T @ np.atleast_1d(lam) + can["C"].T @ mu - sq * s
    x = -np.sign(w)
    value = dual_value_canonical_qp(can, lam, mu, s)
    gl = float((can["A"] @ x - can["b"])[0])
    gmu = can["C"] @ x - can["d"]
    nl = net.n_line
    return value, gl, gmu[:nl], gmu[nl:], -sq * x - 0.5 * s, can["mid"] + can["sigma"] * x


def solve_qp_s(net: Net, loads, rule="adam", alpha=1.0, rho=0.9, beta1=0.9, beta2=0.999,
               eps=1e-8, decay=1.0, max_iters=1000, alpha_lambda=None, target=None, gap=1e-3,
               record=False):
    """Projected ascent on eq. (16)'s dual in (lambda, mu, s) (Section 3.2, Remark 2),
    with the rules of ``solve`` (Section 3.3): mu >= 0 projected after every step, lambda
    and s free, s with mu's step size alpha.  Starts from lambda = mu = s = 0.  The best
    point is the one with the largest g_q; ``best_closed`` is the closed-form dual value
    g(lambda, mu) = max_s g_q at that point (the bound a certificate of (lambda, mu)
    gives).  Stops when best_closed reaches target (1 - gap) if a target is given."""
    loads = np.asarray(loads, dtype=np.float64)
    can = canonical(net, loads)
    nl, ng = net.n_line, net.n_gen
    a_l = alpha if alpha_lambda is None else alpha_lambda
    th = dict(lam=np.zeros(1), mh=np.zeros(nl), ml=np.zeros(nl), s=np.zeros(ng))
    m1 = {k: np.zeros_like(v) for k, v in th.items()}
    m2 = {k: np.zeros_like(v) for k, v in th.items()}
    best, best_closed, best_pt, hist, pts = -np.inf, -np.inf, None, [], []
    it = 0
    for it in range(1, max_iters + 1):
        val, gl, gh, go, gs, _ = evaluate_qp_s(net, can, loads, th["lam"][0], th["mh"], th["ml"], th["s"])
        hist.append(val)
        if record:
            pts.append({k: v.copy() for k, v in th.items()})
        if val > best:
            best = val
            best_pt = {k: v.copy() for k, v in th.items()}
            best_closed = dual_value_prices(net, loads, th["lam"][0], th["mh"], th["ml"])
        if target is not None and best_closed >= target - gap * abs(target):
            break
        grads = dict(lam=np.array([gl]), mh=gh, ml=go, s=gs)
        scale = decay ** (it - 1)
        for k in th:
            a = (a_l if k == "lam" else alpha) * scale
            g = grads[k]
            if rule == "gdm":
                m1[k] = rho * m1[k] + a * g
                th[k] = th[k] + m1[k]
            elif rule == "adam":
                m1[k] = beta1 * m1[k] + (1 - beta1) * g
                m2[k] = beta2 * m2[k] + (1 - beta2) * g * g
                th[k] = th[k] + a * (m1[k] / (1 - beta1 ** it)) / (np.sqrt(m2[k] / (1 - beta2 ** it)) + eps)
            elif rule == "adagrad":
                m1[k] = m1[k] + g * g
                th[k] = th[k] + a * g / (np.sqrt(m1[k]) + eps)
            else:
                raise ValueError(rule)
        th["mh"] = np.maximum(th["mh"], 0.0)
        th["ml"] = np.maximum(th["ml"], 0.0)
    return dict(best=best, best_closed=best_closed, lam=best_pt["lam"][0], mu_hi=best_pt["mh"],
                mu_lo=best_pt["ml"], s=best_pt["s"], iters=it, history=np.array(hist), points=pts)


# ---------------------------------------------------------------- ascent rules

def solve(net: Net, loads, rule="gdm", alpha=1.0, rho=0.9, beta1=0.9, beta2=0.999,
          eps=1e-8, decay=1.0, max_iters=1000, target=None, gap=1e-3, tol=0.0,
          as_printed=False, lam0=0.0, mu_hi0=None, mu_lo0=None, alpha_lambda=None,
          record=False):
    """Projected gradient ascent on the dual (Section 3.3).

    rule="gdm": Algorithm 1 read as heavy-ball momentum: v <- rho v + alpha grad,
      theta <- theta + v (with ``as_printed`` the printed second "gradient update"
      theta <- theta + alpha grad is applied as well).
    rule="adam": Adam (Kingma and Ba), bias-corrected moments, ascent direction.
    rule="adagrad": AdaGrad, theta <- theta + alpha grad / (sqrt(sum grad^2) + eps).
    After every step mu <- max(mu, 0) (Algorithm 1, projection line).  The step size
    is multiplied by ``decay`` after every iteration (Section 4.1 step decay).
    ``alpha_lambda`` optionally gives lambda its own step size (default: alpha).
    Starts from lambda = mu = 0 and zero optimiser state (Algorithm 1, Require) unless
    a warm start is given.  ``mean_dispatch`` is the mean of the minimisers of every
    evaluation, the k-th weighted by k^2 (a candidate for the primal recovery in
    oracle/primal.py: averages of a dual method's minimisers approach the primal
    optimum, and the weights favour the late iterates).  Stops when the best value reaches target (1 - gap)
    (if target is given), when |g_{i+1} - g_i| < tol (Algorithm 1, stop test; tol > 0),
    or after max_iters evaluations.  Returns a dict with the best point and history
    (and, with ``record``, every evaluated point as (lambda, mu_hi, mu_lo)).
    """
    loads = np.asarray(loads, dtype=np.float64)
    nl = net.n_line
    lam = float(lam0)
    mh = np.zeros(nl) if mu_hi0 is None else np.maximum(np.asarray(mu_hi0, dtype=np.float64), 0)
    ml = np.zeros(nl) if mu_lo0 is None else np.maximum(np.asarray(mu_lo0, dtype=np.float64), 0)
    a_l = alpha if alpha_lambda is None else alpha_lambda
    st = dict(vl=0.0, vh=np.zeros(nl), vlo=np.zeros(nl),       # GDM velocity / Adam m / AdaGrad G
              sl=0.0, sh=np.zeros(nl), slo=np.zeros(nl))       # Adam v
    best = -np.inf
    best_pt = (lam, mh.copy(), ml.copy())
    hist = []
    pts = []
    prev = None
    it = 0
    stop = "max_iters"
    psum, wsum = np.zeros(net.n_gen), 0.0
    for it in range(1, max_iters + 1):
        val, gl, ghi, glo, p_it = evaluate(net, loads, lam, mh, ml)
        hist.append(val)
        psum += float(it) ** 2 * p_it       # mean of the minimisers, weight k^2
        wsum += float(it) ** 2
        if record:
            pts.append((lam, mh.copy(), ml.copy()))
        if val > best:
            best = val
            best_pt = (lam, mh.copy(), ml.copy())
        if target is not None and best >= target - gap * abs(target):
            stop = "target"
            break
        if tol > 0 and prev is not None and abs(val - prev) < tol:
            stop = "tol"
            break
        prev = val
        scale = decay ** (it - 1)
        al, am = a_l * scale, alpha * scale
        if rule == "gdm":
            st["vl"] = rho * st["vl"] + al * gl
            st["vh"] = rho * st["vh"] + am * ghi
            st["vlo"] = rho * st["vlo"] + am * glo
            lam = lam + st["vl"]
            mh = mh + st["vh"]
            ml = ml + st["vlo"]
            if as_printed:
                lam = lam + al * gl
                mh = mh + am * ghi
                ml = ml + am * glo
        elif rule == "adam":
            st["vl"] = beta1 * st["vl"] + (1 - beta1) * gl
            st["vh"] = beta1 * st["vh"] + (1 - beta1) * ghi
            st["vlo"] = beta1 * st["vlo"] + (1 - beta1) * glo
            st["sl"] = beta2 * st["sl"] + (1 - beta2) * gl * gl
            st["sh"] = beta2 * st["sh"] + (1 - beta2) * ghi * ghi
            st["slo"] = beta2 * st["slo"] + (1 - beta2) * glo * glo
            c1 = 1.0 - beta1 ** it
            c2 = 1.0 - beta2 ** it
            lam = lam + al * (st["vl"] / c1) / (np.sqrt(st["sl"] / c2) + eps)
            mh = mh + am * (st["vh"] / c1) / (np.sqrt(st["sh"] / c2) + eps)
            ml = ml + am * (st["vlo"] / c1) / (np.sqrt(st["slo"] / c2) + eps)
        elif rule == "adagrad":
            st["vl"] = st["vl"] + gl * gl
            st["vh"] = st["vh"] + ghi * ghi
            st["vlo"] = st["vlo"] + glo * glo
            lam = lam + al * gl / (np.sqrt(st["vl"]) + eps)
            mh = mh + am * ghi / (np.sqrt(st["vh"]) + eps)
            ml = ml + am * glo / (np.sqrt(st["vlo"]) + eps)
        else:
            raise ValueError(rule)
        mh = np.maximum(mh, 0.0)
        ml = np.maximum(ml, 0.0)
    return dict(best=best, lam=best_pt[0], mu_hi=best_pt[1], mu_lo=best_pt[2],
                iters=it, history=np.array(hist), stop=stop, points=pts,
                mean_dispatch=psum / wsum if wsum > 0 else psum)
