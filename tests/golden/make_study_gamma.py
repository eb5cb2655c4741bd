"""Writes tests/golden/study_gamma.json: exact optima gamma* of the instances the
optimiser study runs on (the first 512 training scenarios of the 2000-bus network,
and the first 256 instances of the 4600-bus batch, whose line outages are solved on
the network rebuilt without the line).

Calls only the oracle (interior point with its weak-duality sandwich) and the seeded
input generator; instances whose sandwich does not close are stored as null.
Run from the repository root:
    python tests/golden/make_study_gamma.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

_NETS = {}


def _net(cfg, drop):
    from oracle import dcopf
    from paper_2406_13191_gb300 import synth
    key = (cfg, drop)
    if key not in _NETS:
        net, _ = synth.network_for(cfg)
        d = net.as_dict()
        if drop >= 0:
            keep = np.array([l for l in range(net.n_line) if l != drop])
            for f in ("line_from", "line_to", "line_b", "flow_max", "flow_min"):
                d[f] = np.asarray(d[f])[keep]
        _NETS[key] = dcopf.Net.from_dict(d)
    return _NETS[key]


def _one(args):
    key, i, cfg, drop, loads = args
    from oracle import exact
    r = exact.ipm(_net(cfg, drop), loads)
    return key, i, (r["gamma"] if r["status"] == "optimal" else None)


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from paper_2406_13191_gb300 import synth
    jobs = [("2000", i, 1, -1, L) for i, L in enumerate(synth.warm_loads("train", 512))]
    w = synth.workload(2, batch=256)
    jobs += [("4600", i, 2, int(w.outage[i]), w.loads[i]) for i in range(256)]
    out = {"2000": [None] * 512, "4600": [None] * 256}
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for k, (key, i, g) in enumerate(pool.imap_unordered(_one, jobs, chunksize=4)):
            out[key][i] = g
            if k % 128 == 0:
                print(k, round(time.time() - t0, 1), flush=True)
    out["_about"] = ("gamma* ($/h): '2000' = synth.warm_loads('train', 512) on the 2000-bus "
                     "network; '4600' = synth.workload(2, batch=256) (outage instances on the "
                     "network without the line); oracle interior point, sandwich (ub-lb)/|ub| "
                     "<= 1e-9; null where it did not close.")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "study_gamma.json")
    json.dump(out, open(path, "w"))
    print("done", {k: sum(g is None for g in v) for k, v in out.items() if k != "_about"},
          round(time.time() - t0, 1))


if __name__ == "__main__":
    main()
