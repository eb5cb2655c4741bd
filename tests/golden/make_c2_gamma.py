"""Writes tests/golden/c2_gamma.json: exact optima gamma* of all 1024 instances of the
4600-bus LP batch (synth.workload(2)); an instance with a line outage is solved on the
network rebuilt without that line.

Calls only the oracle (interior point with its weak-duality sandwich) and the seeded
input generator; instances whose sandwich does not close are stored as null.
Run from the repository root (about 10 minutes on 8 cores):
    python tests/golden/make_c2_gamma.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N = 1024
_NETS = {}


def _net(drop):
    from oracle import dcopf
    from paper_2406_13191_gb300 import synth
    if drop not in _NETS:
        net, _ = synth.network_for(2)
        d = net.as_dict()
        if drop >= 0:
            keep = np.array([l for l in range(net.n_line) if l != drop])
            for f in ("line_from", "line_to", "line_b", "flow_max", "flow_min"):
                d[f] = np.asarray(d[f])[keep]
        if len(_NETS) > 4:
            _NETS.clear()
        _NETS[drop] = dcopf.Net.from_dict(d)
    return _NETS[drop]


def _one(args):
    i, drop, loads = args
    from oracle import exact
    r = exact.ipm(_net(drop), loads)
    return i, (r["gamma"] if r["status"] == "optimal" else None)


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from paper_2406_13191_gb300 import synth
    w = synth.workload(2, batch=N)
    jobs = [(i, int(w.outage[i]), w.loads[i]) for i in range(N)]
    gam = [None] * N
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for k, (i, g) in enumerate(pool.imap_unordered(_one, jobs, chunksize=4)):
            gam[i] = g
            if k % 64 == 0:
                print(k, round(time.time() - t0, 1), flush=True)
    out = {"_about": "gamma* ($/h) of the 1024 instances of synth.workload(2) (4600-bus LP, "
                     "512 with a line outage, solved on the network without the line); oracle "
                     "interior point, sandwich (ub-lb)/|ub| <= 1e-9; null where it did not close.",
           "gamma": gam}
    json.dump(out, open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_gamma.json"), "w"))
    print("done", sum(g is None for g in gam), round(time.time() - t0, 1))


if __name__ == "__main__":
    main()
