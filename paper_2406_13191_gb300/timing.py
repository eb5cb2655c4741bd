"""Timing utility for the library's paths on the seeded synthetic workloads.

    python -m paper_2406_13191_gb300.timing batched --config 2 --batch 1024 --iters 16 [--screen]
    python -m paper_2406_13191_gb300.timing certify --config 1 --batch 1
    python -m paper_2406_13191_gb300.timing fused --config 1 --repeat 3
    python -m paper_2406_13191_gb300.timing group --iters 400
    python -m paper_2406_13191_gb300.timing setup
    python -m paper_2406_13191_gb300.timing mlp --batch 512 --iters 50
    python -m paper_2406_13191_gb300.timing togap --config 2
    python -m paper_2406_13191_gb300.timing primal --batch 1024
    python -m paper_2406_13191_gb300.timing sparse

``batched`` runs the tensor-core batched solve (BF16 hi/lo split products) for a
fixed number of iterations and reports the time of the iteration kernels per batched
iteration (CUDA events recorded by the library on its stream).  ``certify`` times the
FP64 certificate and one FP64 evaluation.  ``fused`` times single-instance solves to
the certified 0.1 % gap with the fused persistent kernel (needs the stored optimum of
the 2000-bus instance, tests/golden/gamma.json).  ``group`` runs a mixed-size batch
(1024 instances of a 300-bus network, 256 of the 2000-bus one, 128 of the 4600-bus one
with line outages) for a fixed number of iterations, once network by network and once
as one group solve (one CUDA-graph launch per round over all three).  These are
measurements of the library, used for the kernel profiles; they are not the benchmark
line.  ``setup`` times the per-network work of each workload's network: handle creation
(validation, LDL^T factorisation, the FP64 Phi~ build and upload) and the first batched
FP32/BF16 operator preparation.  ``mlp`` times training steps of the warm-start
perceptron (2000 -> 512 -> 512 -> 3201, seeded random data) in both product modes.
``togap`` solves the 4600-bus batch (1024, half with an outage) or the 10000-bus batch
(256) to the certified 0.1 % gap against the oracle's optima (tests/golden/c2_gamma.json,
c3_gamma.json) in one batched tensor-core call, with the benchmark's settings.
``primal`` times the primal recovery (an upper bound from the dual point) after solves
of the 2000-bus instance and of held-out scenarios, and reports the gap it gives without
a stored optimum.  ``sparse`` times the sparse operator form (triangular solves, no
PTDF) against the PTDF paths.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import DcopfDual, solve_group, synth


def _seeded_point(rng, batch, n_line, density=0.1):
    lam = -rng.uniform(1000, 5000, batch)
    mh = rng.exponential(300.0, (batch, n_line)) * (rng.random((batch, n_line)) < density)
    return lam, mh, np.zeros_like(mh)


def batched(cfg, batch, iters, verbose=False, screen=False):
    """Time per batched iteration of a solve capped at `iters` iterations (no target), as
    the difference between solves of 2 x iters and iters iterations divided by iters:
    what stays the same in both (the setup, the rounds after the cap, the certificates)
    cancels."""
    w = synth.workload(cfg, batch=batch)
    g = DcopfDual(w.net, device=0, verbose=verbose)
    out = w.outage if (w.outage >= 0).any() else None
    kw = dict(rule="adam", alpha=4000.0 if w.net.is_qp else 1000.0, beta1=0.95, beta2=0.999,
              decay=0.997, path="batched", precision="bf16x3", screen=screen)
    g.solve(w.loads, outage=out, max_iters=iters, **kw)    # warm-up (graph capture, operands)
    g.solve(w.loads, outage=out, max_iters=2 * iters, **kw)
    res = {}
    for n in (iters, 2 * iters):
        g.set_timing(True)
        g.read_timing()
        g.read_kernel_timing()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = g.solve(w.loads, outage=out, max_iters=n, **kw)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms, launches, evals = g.read_timing()
        kt, ks = g.read_kernel_timing()
        res[n] = (wall, ms, evals, kt, ks, r)
    (w1, m1, e1, _, _, _), (w2, m2, e2, kt, ks, r) = res[iters], res[2 * iters]
    per_iter_us = 1e3 * (m2 - m1) / iters
    print(json.dumps(dict(mode="batched", config=cfg, batch=batch, iters=iters, screen=screen,
                          shapes=g.tensor_shapes(),
                          kernel_us={k: round(1e3 * v / max(1, ks), 2) for k, v in kt.items()},
                          kept_lines=int(g.screened_lines().sum()) if screen else w.net.n_line,
                          wall_ms=[1e3 * w1, 1e3 * w2], iteration_graphs_ms=[m1, m2],
                          us_per_batched_iteration=per_iter_us,
                          wall_us_per_batched_iteration=1e6 * (w2 - w1) / iters,
                          instance_iterations_per_s=batch / (per_iter_us * 1e-6),
                          status=np.bincount(r.status.cpu().numpy(), minlength=3).tolist())))


def certify(cfg, batch, repeat=10):
    w = synth.workload(cfg, batch=batch)
    g = DcopfDual(w.net, device=0)
    dev = torch.device("cuda", 0)
    loads = torch.tensor(w.loads, dtype=torch.float64, device=dev)
    lam, mh, ml = _seeded_point(np.random.default_rng(0), batch, w.net.n_line)
    lam, mh, ml = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (lam, mh, ml))
    out = torch.tensor(w.outage, device=dev) if (w.outage >= 0).any() else None

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeat):
            fn()
        e1.record()
        e1.synchronize()
        return 1e3 * e0.elapsed_time(e1) / repeat

    res = dict(mode="certify", config=cfg, batch=batch,
               certify_us=timed(lambda: g.certify(loads, lam, mh, ml, outage=out)),
               eval_fp64_us=timed(lambda: g.eval(loads, lam, mh, ml, outage=out, precision="fp64",
                                                 want_grad=False, want_dispatch=False)))
    print(json.dumps(res))


def fused(repeat, verbose=False):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    gam = json.load(open(os.path.join(root, "tests", "golden", "gamma.json")))["1/0"]["gamma"]
    net, base = synth.network_for(1)
    g = DcopfDual(net, device=0, verbose=verbose)
    kw = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000,
              path="fused")
    g.solve(base[None], target=[gam], **kw)
    g.set_timing(True)
    g.read_timing()
    for _ in range(repeat):
        r = g.solve(base[None], target=[gam], **kw)
    ms, launches, evals = g.read_timing()
    print(json.dumps(dict(mode="fused", repeat=repeat, status=int(r.status[0].item()),
                          iterations=int(r.iters[0].item()), fused_kernel_ms=ms,
                          us_per_iteration=1e3 * ms / max(1, evals))))


def group(iters, repeat=3):
    qp = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997)
    lp = dict(rule="adam", alpha=1000.0, beta1=0.95, beta2=0.999, decay=0.997)
    n300, b300 = synth.network_for(300)
    w1 = synth.workload(1, batch=256)
    w2 = synth.workload(2, batch=128)
    items = [(n300, synth.scenario_loads(b300, 1024, 4301), None, qp), (w1.net, w1.loads, None, qp),
             (w2.net, w2.loads, w2.outage, lp)]
    duals = [DcopfDual(n) for n, _, _, _ in items]
    common = dict(max_iters=iters, tol=0.0, precision="bf16x3", path="batched")

    def seq():
        return [d.solve(L, outage=o, **kw, **common) for d, (_, L, o, kw) in zip(duals, items)]

    def grp():
        return solve_group(duals, [L for _, L, _, _ in items], outage=[o for _, _, o, _ in items],
                           per_network=[kw for *_, kw in items], **common)

    res = dict(mode="group", iters=iters, networks=["300-bus QP x1024", "2000-bus QP x256",
                                                    "4600-bus LP x128 (64 outages)"])
    for name, fn in (("network_by_network", seq), ("group", grp)):
        fn()
        ts = []
        for _ in range(repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        res[f"{name}_ms"] = 1e3 * min(ts)
    res["identical_bounds"] = all(torch.equal(a.bound, b.bound) for a, b in zip(seq(), grp()))
    print(json.dumps(res))


def setup():
    res = {"mode": "setup"}
    for cfg in (0, 1, 2, 3):
        net, base = synth.network_for(cfg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = DcopfDual(net, device=0)
        t1 = time.perf_counter()
        g.eval(base[None], [0.0], np.zeros((1, net.n_line)), np.zeros((1, net.n_line)),
               precision="bf16x3")
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del g
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        gs = DcopfDual(net, device=0, operator_form="sparse")
        t4 = time.perf_counter()
        res[f"{net.n_bus}-bus"] = dict(n_line=net.n_line, n_gen=net.n_gen, create_s=t1 - t0,
                                       first_tensor_eval_s=t2 - t1,
                                       create_sparse_only_s=t4 - t3)
        del gs
    print(json.dumps(res))


def mlp(batch, steps):
    from . import warmstart
    rng = np.random.default_rng(0)
    X = torch.as_tensor(rng.uniform(0, 1, (4 * batch, 2000)), dtype=torch.float32, device="cuda")
    Y = torch.as_tensor(rng.normal(0, 1, (4 * batch, 3201)), dtype=torch.float32, device="cuda")
    res = {"mode": "mlp", "batch": batch, "steps": steps}
    for prec in ("bf16x3", "fp32"):
        m = warmstart.WarmStartMLP(2000, 3201, 512, max_batch=batch, precision=prec)
        m.set_params(warmstart.init_params(2000, 512, 3201, 1))
        idx = torch.as_tensor(rng.permutation(4 * batch)[:batch].astype(np.int32), device="cuda")
        for _ in range(3):
            m.train_step(idx, X, Y, 1e-4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = m.kernel_launches()
        e0.record()
        for _ in range(steps):
            m.train_step(idx, X, Y, 1e-4)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        flops = 3 * 2 * batch * m.num_params
        res[prec] = dict(ms_per_step=ms, tflops=flops / (ms * 1e-3) / 1e12,
                         launches_per_step=(m.kernel_launches() - l0) / steps)
        del m
    print(json.dumps(res))


def togap(cfg, repeat=2, screen=False, verbose=False):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if cfg == 2:   # the 4600-bus LP batch of 1024 (512 outages) and the bench's settings for it
        gam = json.load(open(os.path.join(root, "tests", "golden", "c2_gamma.json")))["gamma"]
        kw = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.99, decay=0.99, max_iters=1000)
    else:          # the 10000-bus QP batch of 256 and the bench's headline settings
        gam = json.load(open(os.path.join(root, "tests", "golden", "c3_gamma.json")))["gamma"]
        kw = dict(rule="adam", alpha=3000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)
    w = synth.workload(cfg, batch=len(gam))
    ok = np.array([x is not None for x in gam])
    T = np.array([x for x in gam if x is not None])
    L = torch.tensor(w.loads[ok], device="cuda")
    O = torch.tensor(w.outage[ok], device="cuda") if (w.outage >= 0).any() else None
    Td = torch.tensor(T, device="cuda")
    g = DcopfDual(w.net, device=0, verbose=verbose)
    kw = dict(kw, screen=screen)
    g.solve(L, outage=O, target=Td, path="batched", precision="bf16x3", **kw)
    best = None
    for _ in range(repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = g.solve(L, outage=O, target=Td, path="batched", precision="bf16x3", **kw)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    it = r.iters.cpu().numpy()
    st = r.status.cpu().numpy()
    b = r.bound.cpu().numpy()
    # one more solve with the library's timing hook: time in the iteration graphs against
    # the whole solve (the rest is certification of candidates and the per-round read-back)
    g.set_timing(True)
    g.read_timing()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.solve(L, outage=O, target=Td, path="batched", precision="bf16x3", **kw)
    torch.cuda.synchronize()
    wall = 1e3 * (time.perf_counter() - t0)
    it_ms, it_launches, _ = g.read_timing()
    g.set_timing(False)
    print(json.dumps(dict(mode="togap", config=cfg, instances=int(ok.sum()),
                          outages=int(0 if O is None else (O >= 0).sum().item()), settings=kw,
                          ms=best, iteration_graphs_ms=it_ms, timed_solve_wall_ms=wall,
                          instances_per_s=ok.sum() / (best * 1e-3),
                          mean_iters=float(it.mean()), p90_iters=float(np.percentile(it, 90)),
                          most_iters=int(it.max()), reached_gap=int((st == 0).sum()),
                          all_bounds_valid=bool(np.all(b <= T + 1e-9 * np.abs(T))))))


def primal(batch=1024, repeat=5):
    """Primal recovery after solves to the certified 0.1 % gap on the 2000-bus QP: the
    single instance at base loads (fused path) and ``batch`` held-out load scenarios
    (batched path).  Reports the time of dcopf_dual_primal_bound (CUDA events) and the
    gap it gives without a stored optimum, (upper - lower) / upper, next to the true
    gaps of both bounds against the oracle's gamma*."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    net, base = synth.network_for(1)
    g = DcopfDual(net, device=0)
    kw = dict(rule="adam", alpha=4000.0, beta1=0.95, beta2=0.999, decay=0.997, max_iters=4000)
    out = dict(mode="primal", network="synthetic 2000-bus QP")

    def timed(loads, r, mean=False):
        res = None
        ts = []
        for _ in range(repeat + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if mean:
                res = g.primal_bound(loads, p_cand=r.mean_dispatch)
            else:
                res = g.primal_bound(loads, r.lam, r.mu_hi, r.mu_lo)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return res, float(np.median(ts[1:]))

    def gaps(gam, lb, ub, st):
        ok = st == 0
        d = dict(bounded=int(ok.sum()), of=int(len(st)),
                 all_valid=bool(np.all(lb <= gam * (1 + 1e-12)) and np.all(ub[ok] >= gam[ok] * (1 - 1e-12))))
        if ok.any():
            for name, v in (("gap_without_oracle", (ub - lb) / ub), ("upper_gap", (ub - gam) / gam)):
                v = v[ok]
                d[name] = dict(median=float(np.median(v)), p90=float(np.percentile(v, 90)),
                               max=float(v.max()))
        return d

    gam1 = json.load(open(os.path.join(root, "tests", "golden", "gamma.json")))["1/0"]["gamma"]
    r = g.solve(base[None], target=[gam1], path="fused", mean_dispatch=True, **kw)
    for cand in ("dual_point", "mean_of_minimisers"):
        (ub, st, _, viol), ms = timed(base[None], r, mean=cand != "dual_point")
        out[f"single_from_{cand}"] = dict(
            ms=ms, lower=r.bound.item(), upper=ub.item(), status=int(st.item()),
            max_violation=viol.item(), iterations=int(r.iters.item()),
            **gaps(np.array([gam1]), r.bound.cpu().numpy(), ub.cpu().numpy(), st.cpu().numpy()))
    gam = np.array(json.load(open(os.path.join(root, "tests", "golden", "warm_gamma.json")))["gamma"][:batch])
    X = synth.warm_loads("heldout", batch)
    r = g.solve(X, target=gam, path="batched", precision="bf16x3", mean_dispatch=True, **kw)
    for cand in ("dual_point", "mean_of_minimisers"):
        (ub, st, _, viol), ms = timed(X, r, mean=cand != "dual_point")
        st_h = st.cpu().numpy()
        out[f"batch_from_{cand}"] = dict(
            instances=batch, ms=ms, per_instance_us=1e3 * ms / batch,
            reached_gap=int((r.status == 0).sum().item()),
            max_violation=float(np.nanmax(viol.cpu().numpy())),
            **gaps(gam, r.bound.cpu().numpy(), ub.cpu().numpy(), st_h))
    print(json.dumps(out))


def sparse(iters=100):
    """The sparse operator form (LDL^T solves, no PTDF) against the PTDF paths for a fixed
    number of FP64 iterations: the 2000-bus instance alone (sparse vs plain FP64 per-phase
    kernels) and the first 256 instances of the 4600-bus batch (half with an outage;
    sparse vs the tensor-core batched path).  Iteration-kernel time from the library's
    events."""
    out = dict(mode="sparse", iters=iters)
    kw = dict(rule="adam", alpha=1000.0, beta1=0.95, beta2=0.999, max_iters=iters)

    def run(g, loads, outage, path, precision):
        g.solve(loads, outage=outage, path=path, precision=precision, **kw)  # warm-up
        g.set_timing(True)
        g.read_timing()
        r = g.solve(loads, outage=outage, path=path, precision=precision, **kw)
        ms, launches, evals = g.read_timing()
        g.set_timing(False)
        return dict(ms=ms, us_per_instance_iteration=1e3 * ms / max(1, evals),
                    evaluations=evals, status_cap=int((r.status == 1).sum().item()))

    net, base = synth.network_for(1)
    g = DcopfDual(net, device=0)
    out["single_2000bus"] = {p: run(g, base[None], None, p, "fp64") for p in ("sparse", "plain")}
    w = synth.workload(2, batch=256)
    g = DcopfDual(w.net, device=0)
    L = torch.tensor(w.loads, device="cuda")
    O = torch.tensor(w.outage, device="cuda")
    out["batch_4600bus_256"] = dict(sparse=run(g, L, O, "sparse", "fp64"),
                                    batched_bf16x3=run(g, L, O, "batched", "bf16x3"))
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["batched", "certify", "fused", "group", "setup", "mlp", "togap",
                                     "primal", "sparse"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--iters", type=int, default=16)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--verbose", action="store_true", help="library setup and tuning messages")
    ap.add_argument("--screen", action="store_true", help="constraint screening (batched, togap)")
    a = ap.parse_args()
    if a.mode == "batched":
        batched(a.config, a.batch, a.iters, a.verbose, a.screen)
    elif a.mode == "certify":
        certify(a.config, a.batch)
    elif a.mode == "group":
        group(a.iters)
    elif a.mode == "setup":
        setup()
    elif a.mode == "mlp":
        mlp(a.batch, a.iters)
    elif a.mode == "togap":
        togap(a.config, screen=a.screen, verbose=a.verbose)
    elif a.mode == "primal":
        primal(a.batch)
    elif a.mode == "sparse":
        sparse(a.iters if a.iters != 16 else 100)
    else:
        fused(a.repeat, a.verbose)


if __name__ == "__main__":
    main()
