"""Shared helpers of the GPU parity tests (seeded dual points, oracle wrappers)."""
import numpy as np

from oracle import dcopf, exact
from paper_2406_13191_gb300 import synth


def onet(net):
    return dcopf.Net.from_dict(net.as_dict())


def drop_line(net: synth.Network, k: int) -> dcopf.Net:
    """Oracle network with line k removed (the post-outage network, rebuilt)."""
    d = net.as_dict()
    keep = np.array([l for l in range(net.n_line) if l != k])
    for f in ("line_from", "line_to", "line_b", "flow_max", "flow_min"):
        d[f] = np.asarray(d[f])[keep]
    return dcopf.Net.from_dict(d)


def rand_point(rng, n_line, scale=300.0, density=0.3, lam_range=(1000.0, 5000.0)):
    lam = -rng.uniform(*lam_range)
    mh = rng.exponential(scale, n_line) * (rng.random(n_line) < density)
    ml = rng.exponential(scale, n_line) * (rng.random(n_line) < density)
    return lam, mh, ml


def near_tie(on: dcopf.Net, loads, lam, mh, ml, rel=1e-7):
    """True if some LP generator's reduced cost is within rel of zero (sign flips there
    are legitimate rounding differences)."""
    if on.qp:
        return False
    _, z, nu, _, _ = dcopf.dual_parts(on, loads, lam, mh, ml)
    k = on.c * on.S + nu[on.gen_bus]
    return bool(np.any(np.abs(k) < rel * (np.abs(on.c * on.S) + np.abs(nu[on.gen_bus]))))


def gamma(on, loads):
    r = exact.ipm(on, loads)
    assert r["status"] == "optimal", r["status"]
    return r["gamma"]
