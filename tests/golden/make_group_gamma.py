"""Writes tests/golden/group_gamma.json: exact optima gamma* of the mixed-size group
workload's instances that no other golden file holds: 1024 load scenarios of the
300-bus network (synth.scenario_loads(base, 1024, 4301)) and the first 256 scenarios
of the 2000-bus network (synth.workload(1, batch=256)).  The group's 4600-bus part is
the first 128 instances of the 4600-bus batch, in c2_gamma.json.

Calls only the oracle (interior point with its weak-duality sandwich) and the seeded
input generator; instances whose sandwich does not close are stored as null.
Run from the repository root (a few minutes on 8 cores):
    python tests/golden/make_group_gamma.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

_NETS = {}


def _net(cfg):
    from oracle import dcopf
    from paper_2406_13191_gb300 import synth
    if cfg not in _NETS:
        _NETS[cfg] = dcopf.Net.from_dict(synth.network_for(cfg)[0].as_dict())
    return _NETS[cfg]


def _one(args):
    key, i, cfg, loads = args
    from oracle import exact
    r = exact.ipm(_net(cfg), loads)
    return key, i, (r["gamma"] if r["status"] == "optimal" else None)


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from paper_2406_13191_gb300 import synth
    _, b300 = synth.network_for(300)
    jobs = [("300", i, 300, L) for i, L in enumerate(synth.scenario_loads(b300, 1024, 4301))]
    jobs += [("2000", i, 1, L) for i, L in enumerate(synth.workload(1, batch=256).loads)]
    out = {"300": [None] * 1024, "2000": [None] * 256}
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for k, (key, i, g) in enumerate(pool.imap_unordered(_one, jobs, chunksize=8)):
            out[key][i] = g
            if k % 256 == 0:
                print(k, round(time.time() - t0, 1), flush=True)
    out["_about"] = ("gamma* ($/h): '300' = synth.scenario_loads(network_for(300) base, 1024, 4301) "
                     "on the 300-bus network; '2000' = synth.workload(1, batch=256); oracle interior "
                     "point, sandwich (ub-lb)/|ub| <= 1e-9; null where it did not close.")
    json.dump(out, open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "group_gamma.json"), "w"))
    print("done", {k: sum(g is None for g in v) for k, v in out.items() if k != "_about"},
          round(time.time() - t0, 1))


if __name__ == "__main__":
    main()
