"""Writes tests/golden/warm_gamma.json: exact optima gamma* of the held-out load
scenarios of the 2000-bus network (the evaluation set of the learned warm start).

Calls only the oracle (interior point with its weak-duality sandwich) and the seeded
input generator.  Instances whose sandwich does not close are stored as null.
Run from the repository root (about half an hour on 8 cores):
    python tests/golden/make_warm_gamma.py [count]
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

_NET = None


def _init():
    global _NET
    from oracle import dcopf
    from paper_2406_13191_gb300 import synth
    net, _ = synth.network_for(1)
    _NET = dcopf.Net.from_dict(net.as_dict())


def _one(args):
    i, loads = args
    from oracle import exact
    r = exact.ipm(_NET, loads)
    return i, (r["gamma"] if r["status"] == "optimal" else None), r["rel_gap"]


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from paper_2406_13191_gb300 import synth
    count = int(sys.argv[1]) if len(sys.argv) > 1 else synth.WARM_SETS["heldout"][0]
    loads = synth.warm_loads("heldout", count)
    t0 = time.time()
    gam = [None] * count
    with mp.get_context("spawn").Pool(os.cpu_count(), initializer=_init) as pool:
        for k, (i, g, rg) in enumerate(pool.imap_unordered(_one, list(enumerate(loads)), chunksize=8)):
            gam[i] = g
            if k % 256 == 0:
                print(k, round(time.time() - t0, 1), flush=True)
    out = {"_about": "gamma* ($/h) of synth.warm_loads('heldout') instances on the 2000-bus "
                     "network, from the oracle interior point method (sandwich (ub-lb)/|ub| <= "
                     "1e-9); null where the sandwich did not close.",
           "gamma": gam}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warm_gamma.json")
    json.dump(out, open(path, "w"))
    print("done", sum(g is None for g in gam), "without optimum", round(time.time() - t0, 1))


if __name__ == "__main__":
    main()
