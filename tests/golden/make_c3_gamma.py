"""Writes tests/golden/c3_gamma.json: exact optima gamma* of all 256 instances of the
10000-bus QP batch (synth.workload(3)), the stopping targets of its to-gap solves.

Calls only the oracle (interior point with its weak-duality sandwich) and the seeded
input generator; instances whose sandwich does not close are stored as null.
Run from the repository root (about an hour on 8 cores):
    python tests/golden/make_c3_gamma.py [--resume]
With --resume, values already in the file (written by this script) are kept and only
the missing instances are solved.
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N = 256
_NET = None


def _init():
    global _NET
    from oracle import dcopf
    from paper_2406_13191_gb300 import synth
    net, _ = synth.network_for(3)
    _NET = dcopf.Net.from_dict(net.as_dict())


def _one(args):
    i, loads = args
    from oracle import exact
    r = exact.ipm(_NET, loads)
    return i, (r["gamma"] if r["status"] == "optimal" else None)


def main():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    from paper_2406_13191_gb300 import synth
    w = synth.workload(3, batch=N)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_gamma.json")
    gam = [None] * N
    if "--resume" in sys.argv and os.path.exists(path):
        old = json.load(open(path))["gamma"]
        gam[:len(old)] = old[:N]
    todo = [(i, w.loads[i]) for i in range(N) if gam[i] is None]
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count(), initializer=_init) as pool:
        for k, (i, g) in enumerate(pool.imap_unordered(_one, todo)):
            gam[i] = g
            print(k, round(time.time() - t0, 1), flush=True)
    out = {"_about": "gamma* ($/h) of the 256 instances of synth.workload(3) (10000-bus QP), "
                     "oracle interior point, sandwich (ub-lb)/|ub| <= 1e-9; null where it did "
                     "not close.", "gamma": gam}
    json.dump(out, open(path, "w"))
    print("done", sum(g is None for g in gam), round(time.time() - t0, 1))


if __name__ == "__main__":
    main()
