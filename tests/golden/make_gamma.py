"""Writes tests/golden/gamma.json: exact optima gamma* of the benchmark instances.

Calls only the oracle (interior point with its weak-duality sandwich, and the
seeded generator for the inputs).  Run from the repository root:
    python tests/golden/make_gamma.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dcopf, exact  # noqa: E402
from paper_2406_13191_gb300 import synth  # noqa: E402


def main():
    out = {"_about": "gamma* = optimal DCOPF cost ($/h) of seeded synthetic instances, from the "
                     "oracle interior point method (sandwich (ub-lb)/|ub| <= 1e-9).  Keys: "
                     "config/instance index within synth.workload(config)."}
    jobs = [(0, 1), (1, 1)]
    for cfg, n in jobs:
        w = synth.workload(cfg, batch=n)
        on = dcopf.Net.from_dict(w.net.as_dict())
        for b in range(n):
            t = time.time()
            r = exact.ipm(on, w.loads[b])
            assert r["status"] == "optimal", (cfg, b, r["status"])
            out[f"{cfg}/{b}"] = dict(gamma=r["gamma"], ub=r["ub"], lb=r["lb"], rel_gap=r["rel_gap"])
            print(cfg, b, r["gamma"], r["rel_gap"], round(time.time() - t, 2))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gamma.json")
    json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main()
