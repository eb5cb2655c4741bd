"""Seeded synthetic DCOPF workloads.

The paper measures on the IEEE/PGLib 2000-, 4601- and 10000-bus cases (Section 4,
Tables I-III and VII-IX).  Those files are not shipped here, so this module
generates networks of the same sizes and structure from a counter-free PCG64
stream: a geographically local random spanning tree plus extra edges between
nearby buses (real transmission grids are near-planar with small separators),
random orientations, susceptances U[5, 50] p.u., generators on distinct random
buses, linear or quadratic cost laws, load laws per workload, and line limits set
relative to the flows of a proportional base dispatch.

This module is shared by the oracle-side tests and the CUDA-side callers.  It
holds none of the dual method's arithmetic (no dual value, no inner minimiser,
no ascent step).  The one linear solve it performs is the DC power flow of the
proportional dispatch, used only to build inputs (placing the line limits, and keeping
warm-start scenarios that this dispatch makes feasible); it goes through a scipy
sparse LU and nothing else in the repository uses it.

Units: powers in p.u. on ``base_mva`` (100 MVA); linear cost coefficients in
$/MWh and quadratic ones in $/MW^2h, so that a generator producing ``p`` p.u.
costs ``a*(S*p)**2 + b*(S*p)`` $/h with ``S = base_mva``.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field
import numpy as np

BASE_MVA = 100.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Network:
    """Arrays describing one DCOPF network (Section 2, problem (1)).

    line_from/line_to: 0-based bus indices of each line; line_b: susceptance (p.u.);
    flow_max/flow_min: line limits (p.u.); gen_bus: bus of each generator;
    pmin/pmax (p.u.); cost_lin ($/MWh); cost_quad ($/MW^2h) or None for linear costs.
    """
    n_bus: int
    line_from: np.ndarray
    line_to: np.ndarray
    line_b: np.ndarray
    flow_max: np.ndarray
    flow_min: np.ndarray
    gen_bus: np.ndarray
    pmin: np.ndarray
    pmax: np.ndarray
    cost_lin: np.ndarray
    cost_quad: np.ndarray | None
    base_mva: float = BASE_MVA
    slack_bus: int = 0
    name: str = ""

    @property
    def n_line(self) -> int:
        return int(self.line_from.shape[0])

    @property
    def n_gen(self) -> int:
        return int(self.gen_bus.shape[0])

    @property
    def is_qp(self) -> bool:
        return self.cost_quad is not None

    def as_dict(self) -> dict:
        return dict(n_bus=self.n_bus, line_from=self.line_from, line_to=self.line_to,
                    line_b=self.line_b, flow_max=self.flow_max, flow_min=self.flow_min,
                    gen_bus=self.gen_bus, pmin=self.pmin, pmax=self.pmax,
                    cost_lin=self.cost_lin, cost_quad=self.cost_quad,
                    base_mva=self.base_mva, slack_bus=self.slack_bus)


@dataclass
class Workload:
    """A network plus a batch of instances: loads [B][n_bus] and outages [B] (-1 = none)."""
    net: Network
    loads: np.ndarray
    outage: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return int(self.loads.shape[0])


# ---------------------------------------------------------------- topology

def _geo_topology(rng, n_bus: int, n_line: int, k_tree: int = 3, k_extra: int = 8):
    """Random spanning tree (bus i joins one of its k nearest earlier buses) plus
    distinct extra edges from a uniform bus to one of its k nearest neighbours."""
    if n_line < n_bus - 1:
        raise ValueError("need at least n_bus-1 lines for a connected network")
    xy = rng.random((n_bus, 2))
    edges = []
    adj = [set() for _ in range(n_bus)]
    for i in range(1, n_bus):
        d2 = ((xy[:i] - xy[i]) ** 2).sum(1)
        k = min(k_tree, i)
        cand = np.argpartition(d2, k - 1)[:k] if i > k else np.arange(i)
        j = int(cand[rng.integers(len(cand))])
        edges.append((j, i))
        adj[i].add(j)
        adj[j].add(i)
    n_extra = n_line - (n_bus - 1)
    if n_extra > 0:
        from scipy.spatial import cKDTree
        kk = min(k_extra + 1, n_bus)
        _, nbr = cKDTree(xy).query(xy, k=kk)
        guard = 0
        while n_extra > 0:
            guard += 1
            if guard > 200 * n_line:
                raise RuntimeError("could not place extra edges")
            u = int(rng.integers(n_bus))
            v = int(nbr[u, 1 + rng.integers(kk - 1)])
            if v == u or v in adj[u]:
                continue
            edges.append((u, v))
            adj[u].add(v)
            adj[v].add(u)
            n_extra -= 1
    e = np.array(edges, dtype=np.int64)
    flip = rng.random(len(e)) < 0.5
    e[flip] = e[flip][:, ::-1]
    return e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), xy


def bridges(n_bus: int, line_from: np.ndarray, line_to: np.ndarray) -> np.ndarray:
    """Boolean mask of bridge lines (Tarjan low-link, iterative DFS)."""
    n_line = len(line_from)
    adj = [[] for _ in range(n_bus)]
    for l in range(n_line):
        adj[int(line_from[l])].append((int(line_to[l]), l))
        adj[int(line_to[l])].append((int(line_from[l]), l))
    disc = -np.ones(n_bus, dtype=np.int64)
    low = np.zeros(n_bus, dtype=np.int64)
    is_bridge = np.zeros(n_line, dtype=bool)
    t = 0
    for root in range(n_bus):
        if disc[root] >= 0:
            continue
        disc[root] = low[root] = t
        t += 1
        stack = [(root, -1, 0)]
        while stack:
            u, pl, it = stack[-1]
            if it < len(adj[u]):
                stack[-1] = (u, pl, it + 1)
                v, l = adj[u][it]
                if l == pl:
                    continue
                if disc[v] < 0:
                    disc[v] = low[v] = t
                    t += 1
                    stack.append((v, l, 0))
                else:
                    low[u] = min(low[u], disc[v])
            else:
                stack.pop()
                if stack:
                    p = stack[-1][0]
                    low[p] = min(low[p], low[u])
                    if low[u] > disc[p]:
                        is_bridge[pl] = True
    return is_bridge


def _laplacian_lu(n_bus, line_from, line_to, line_b, slack=0):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n_line = len(line_from)
    rows = np.repeat(np.arange(n_line), 2)
    cols = np.stack([line_from, line_to], 1).ravel()
    vals = np.tile(np.array([1.0, -1.0]), n_line)
    inc = sp.csr_matrix((vals, (rows, cols)), shape=(n_line, n_bus))
    lap = (inc.T @ sp.diags(line_b) @ inc).tocsc()
    keep = np.setdiff1d(np.arange(n_bus), [slack])
    return spl.splu(lap[keep][:, keep]), keep


def _dc_flows(n_bus, line_from, line_to, line_b, inj, slack=0, lu=None):
    """DC power flow of injection vectors (columns of ``inj``), used only to build
    inputs (line limits, feasible warm-start scenarios)."""
    if lu is None:
        lu, keep = _laplacian_lu(n_bus, line_from, line_to, line_b, slack)
    else:
        lu, keep = lu
    inj = np.asarray(inj, dtype=np.float64)
    theta = np.zeros((n_bus,) + inj.shape[1:])
    theta[keep] = lu.solve(np.ascontiguousarray(inj[keep]))
    return (line_b[:, None] if inj.ndim == 2 else line_b) * (theta[line_from] - theta[line_to])


def _proportional_injections(loads, gen_bus, pmax):
    """Columns: injections of the proportional dispatch p_j = pmax_j D / sum(pmax)."""
    L = np.atleast_2d(loads)
    inj = -L.T.copy()
    share = pmax / pmax.sum()
    for b in range(L.shape[0]):
        np.add.at(inj[:, b], gen_bus, share * L[b].sum())
    return inj


def _place_limits(rng, net_parts, loads_ref, frac_tight=0.10, outages=None):
    """Line limits relative to the proportional-dispatch flows.

    ``loads_ref`` is one load vector or a [k][n_bus] reference set; the flow of line l
    is taken as its largest |flow| over the reference instances (for an instance
    with an outaged line, the flows of the network without that line).  Limits are
    U[1.1, 1.5] times that envelope, 1.02 times for a random 10 % of lines, and at
    least 5 % of the median envelope.  Every reference instance is then feasible
    (its proportional dispatch satisfies every limit)."""
    n_bus, lf, lt, lb, gen_bus, pmax = net_parts
    L = np.atleast_2d(loads_ref)
    inj = _proportional_injections(L, gen_bus, pmax)
    lu = _laplacian_lu(n_bus, lf, lt, lb)
    env = np.abs(_dc_flows(n_bus, lf, lt, lb, inj, lu=lu)).max(1)
    if outages is not None:
        for b in np.flatnonzero(outages >= 0):
            k = int(outages[b])
            keep = np.arange(len(lf)) != k
            fk = _dc_flows(n_bus, lf[keep], lt[keep], lb[keep], inj[:, b])
            env[keep] = np.maximum(env[keep], np.abs(fk))
    factor = rng.uniform(1.1, 1.5, size=len(lf))
    tight = rng.random(len(lf)) < frac_tight
    factor[tight] = 1.02
    floor = 0.05 * np.median(env)
    fmax = np.maximum(factor * env, floor)
    return fmax, env


def make_network(seed: int, n_bus: int, n_line: int, n_gen: int, quadratic: bool,
                 load_law: str, load_frac: float, name: str = "", scenarios=None):
    """Build a network and its base load profile (returned as (Network, loads_base)).

    ``scenarios`` = (count, seed, outage_count, outage_seed) adds that workload's own
    scenario instances (per-bus multipliers U[0.85, 1.15] on the base profile, and
    line outages) to the reference set the limits are placed on."""
    rng = _rng(seed)
    lf, lt, _ = _geo_topology(rng, n_bus, n_line)
    lb = rng.uniform(5.0, 50.0, size=n_line)
    gen_bus = rng.choice(n_bus, size=n_gen, replace=False).astype(np.int32)
    pmin = np.zeros(n_gen)
    pmax = rng.uniform(0.5, 2.5, size=n_gen)
    if quadratic:
        cost_quad = rng.uniform(0.001, 0.05, size=n_gen)
        cost_lin = rng.uniform(10.0, 60.0, size=n_gen)
    else:
        cost_quad = None
        cost_lin = rng.uniform(10.0, 50.0, size=n_gen)
    if load_law == "uniform":
        loads = rng.uniform(0.0, 0.4, size=n_bus)
    elif load_law == "lognormal":
        loads = rng.lognormal(0.0, 0.5, size=n_bus)
    else:
        raise ValueError(load_law)
    loads *= load_frac * pmax.sum() / loads.sum()
    ref = loads[None, :]
    outs = None
    if scenarios is not None:
        count, sseed, n_out, oseed = scenarios
        sc = scenario_loads(loads, count, sseed)
        ref = np.vstack([ref, sc])
        if n_out:
            o = _outage_choice(n_bus, lf, lt, count, n_out, oseed)
            outs = np.concatenate([[-1], o])
    fmax, _ = _place_limits(rng, (n_bus, lf, lt, lb, gen_bus, pmax), ref, outages=outs)
    net = Network(n_bus=n_bus, line_from=lf, line_to=lt, line_b=lb, flow_max=fmax,
                  flow_min=-fmax, gen_bus=gen_bus, pmin=pmin, pmax=pmax,
                  cost_lin=cost_lin, cost_quad=cost_quad, name=name)
    return net, loads


# ---------------------------------------------------------------- workloads

CONFIG_NAMES = {
    0: "30-bus LP, 41 lines, 6 gens, single instance (FP64 plain method)",
    1: "2000-bus QP, 3200 lines, 540 gens, single instance (FP32 operators)",
    2: "4600-bus LP, 7200 lines, 410 gens, batch 1024 with 512 line outages",
    3: "10000-bus QP, 12700 lines, 2500 gens, batch 256 (BF16 split tensor cores)",
    4: "mixed 300/2000/4600-bus batch with learned warm start",
}


# scenario streams: (count, load seed, outage count, outage seed) per workload
SCENARIOS = {1: (256, 1001, 0, 0), 2: (1024, 2001, 512, 2002), 3: (256, 3001, 0, 0)}


@functools.lru_cache(maxsize=8)
def network_for(cfg: int):
    """The network of workload ``cfg`` and its base load profile (cached; treat the
    returned arrays as read-only)."""
    if cfg == 0:
        return make_network(1000, 30, 41, 6, False, "uniform", 0.60, "syn30")
    if cfg == 1:
        return make_network(1000 * 1, 2000, 3200, 540, True, "lognormal", 0.65, "syn2000",
                            scenarios=SCENARIOS[1])
    if cfg == 2:
        return make_network(1000 * 2, 4600, 7200, 410, False, "uniform", 0.60, "syn4600",
                            scenarios=SCENARIOS[2])
    if cfg == 3:
        return make_network(1000 * 3, 10000, 12700, 2500, True, "lognormal", 0.65, "syn10000",
                            scenarios=SCENARIOS[3])
    if cfg == 300:
        return make_network(1000 * 4 + 300, 300, 480, 81, True, "lognormal", 0.65, "syn300",
                            scenarios=(256, 4301, 0, 0))
    raise ValueError(cfg)


def scenario_loads(base_loads: np.ndarray, batch: int, seed: int, lo=0.85, hi=1.15):
    """Per-bus multipliers U[lo, hi] on a base profile, one row per instance."""
    rng = _rng(seed)
    return base_loads[None, :] * rng.uniform(lo, hi, size=(batch, base_loads.shape[0]))


def _outage_choice(n_bus, line_from, line_to, batch, n_out, seed):
    rng = _rng(seed)
    ok = np.flatnonzero(~bridges(n_bus, line_from, line_to))
    out = -np.ones(batch, dtype=np.int32)
    which = rng.choice(batch, size=n_out, replace=False)
    out[which] = rng.choice(ok, size=n_out, replace=True).astype(np.int32)
    return out


def outages_for(net: Network, batch: int, n_out: int, seed: int) -> np.ndarray:
    """-1 for intact instances; a uniform non-bridge line for ``n_out`` random instances."""
    return _outage_choice(net.n_bus, net.line_from, net.line_to, batch, n_out, seed)


def workload(cfg: int, batch: int | None = None) -> Workload:
    """Instances of workload ``cfg`` (the first ``batch`` of its scenario stream)."""
    net, base = network_for(cfg)
    if cfg == 0:
        b = 1 if batch is None else batch
        loads = np.repeat(base[None, :], b, 0)
        out = -np.ones(b, dtype=np.int32)
    elif cfg == 1:
        b = 1 if batch is None else batch
        loads = base[None, :] if b == 1 else scenario_loads(base, b, SCENARIOS[1][1])
        out = -np.ones(b, dtype=np.int32)
    elif cfg in (2, 3):
        count, sseed, n_out, oseed = SCENARIOS[cfg]
        b = count if batch is None else batch
        loads = scenario_loads(base, count, sseed)[:b]
        out = (_outage_choice(net.n_bus, net.line_from, net.line_to, count, n_out, oseed)[:b]
               if n_out else -np.ones(b, dtype=np.int32))
    else:
        raise ValueError(cfg)
    return Workload(net=net, loads=np.ascontiguousarray(loads), outage=out,
                    meta=dict(config=cfg, name=CONFIG_NAMES.get(cfg, "")))


# learned warm start on the 2000-bus network: (count, load seed) of the training set
# and of the held-out evaluation set
WARM_SETS = {"train": (50000, 4101), "heldout": (4096, 4102)}


def warm_loads(split: str, count: int | None = None) -> np.ndarray:
    """Load vectors of the warm-start sets on the 2000-bus network: per-bus multipliers
    U[0.85, 1.15] on the base profile, kept only when the proportional dispatch of the
    scenario meets every line limit (so every instance is feasible by construction).
    Candidates are drawn in fixed chunks, so a shorter ``count`` is a prefix."""
    n, seed = WARM_SETS[split]
    net, base = network_for(1)
    n = n if count is None else min(n, count)
    rng = _rng(seed)
    lu = _laplacian_lu(net.n_bus, net.line_from, net.line_to, net.line_b)
    out, have = np.empty((n, base.shape[0])), 0
    while have < n:
        cand = base[None, :] * rng.uniform(0.85, 1.15, size=(4096, base.shape[0]))
        inj = _proportional_injections(cand, net.gen_bus, net.pmax)
        f = _dc_flows(net.n_bus, net.line_from, net.line_to, net.line_b, inj, lu=lu)
        ok = np.flatnonzero(((f <= net.flow_max[:, None]) & (f >= net.flow_min[:, None])).all(0))
        take = ok[:n - have]
        out[have:have + len(take)] = cand[take]
        have += len(take)
    return out


def scenario_workload(seed: int, n_bus: int, n_line: int, n_gen: int, quadratic: bool,
                      batch: int, n_out: int) -> Workload:
    """A small network whose limits are placed on its own scenario set (multipliers
    U[0.85, 1.15] and ``n_out`` line outages), returned with that set."""
    sc = (batch, seed + 1, n_out, seed + 2)
    net, base = make_network(seed, n_bus, n_line, n_gen, quadratic,
                             "lognormal" if quadratic else "uniform", 0.6,
                             f"scen{n_bus}", scenarios=sc)
    loads = scenario_loads(base, batch, seed + 1)
    out = (_outage_choice(n_bus, net.line_from, net.line_to, batch, n_out, seed + 2) if n_out
           else -np.ones(batch, dtype=np.int32))
    return Workload(net=net, loads=np.ascontiguousarray(loads), outage=out,
                    meta=dict(config=None, name=net.name))


def tiny_network(seed: int, n_bus: int, n_line: int, n_gen: int, quadratic=False,
                 tight=0.3):
    """Small random networks for brute-force and property tests."""
    rng = _rng(seed)
    lf, lt, _ = _geo_topology(rng, n_bus, n_line, k_tree=2, k_extra=n_bus - 1)
    lb = rng.uniform(5.0, 50.0, size=n_line)
    gen_bus = rng.choice(n_bus, size=n_gen, replace=False).astype(np.int32)
    pmax = rng.uniform(0.5, 2.5, size=n_gen)
    pmin = np.zeros(n_gen)
    if quadratic:
        cq = rng.uniform(0.001, 0.05, size=n_gen)
        cl = rng.uniform(10.0, 60.0, size=n_gen)
    else:
        cq = None
        cl = rng.uniform(10.0, 50.0, size=n_gen)
    loads = rng.uniform(0.0, 0.4, size=n_bus)
    loads *= 0.6 * pmax.sum() / loads.sum()
    fmax, _ = _place_limits(rng, (n_bus, lf, lt, lb, gen_bus, pmax), loads, frac_tight=tight)
    net = Network(n_bus=n_bus, line_from=lf, line_to=lt, line_b=lb, flow_max=fmax,
                  flow_min=-fmax, gen_bus=gen_bus, pmin=pmin, pmax=pmax, cost_lin=cl,
                  cost_quad=cq, name=f"tiny{n_bus}")
    return net, loads
