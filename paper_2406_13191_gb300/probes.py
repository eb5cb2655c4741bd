"""Measured limits of the GPU that bound this library's kernels (include/dcopf_probe.h).

    python -m paper_2406_13191_gb300.probes [--exchange-gens 540]

Prints one JSON object: streaming read bandwidth from L2 (32 and 64 MiB footprints)
and HBM (4 GiB), shared-memory read bandwidth, FP64 and FP32 FMA throughput and
dependent-FMA latency, the TMA tile feed of the tensor-core products from L2, and the
time of one loop of the fused solve's exchange for each cluster shape (no arithmetic:
the latency floor of one fused iteration).  Every figure is measured with CUDA events.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json

from . import _lib


def _call(fn, *args, n_out=1):
    outs = [C.c_double() for _ in range(n_out)]
    _lib.check(fn(*args, *[C.byref(o) for o in outs]), fn.__name__)
    return [o.value for o in outs] if n_out > 1 else outs[0].value


def run(exchange_gens: int = 540, loops: int = 2000) -> dict:
    import torch
    lib = _lib.load()
    torch.cuda.init()
    prop = torch.cuda.get_device_properties(torch.cuda.current_device())
    out = {"device": prop.name, "sm_count": prop.multi_processor_count,
           "l2_bytes": getattr(prop, "L2_cache_size", None)}
    out["l2_read_gbs_32MiB"] = _call(lib.dcopf_probe_read, 32 << 20, 50)
    out["l2_read_gbs_64MiB"] = _call(lib.dcopf_probe_read, 64 << 20, 25)
    out["hbm_read_gbs_4GiB"] = _call(lib.dcopf_probe_read, 4 << 30, 1)
    out["smem_read_gbs"] = _call(lib.dcopf_probe_smem)
    out["fp64_fma_tflops"], out["fp64_fma_chain_ns"] = _call(lib.dcopf_probe_fma, 1, n_out=2)
    out["fp32_fma_tflops"], out["fp32_fma_chain_ns"] = _call(lib.dcopf_probe_fma, 0, n_out=2)
    out["tma_feed_gbs_64MiB"] = _call(lib.dcopf_probe_tma_feed, 64 << 20)
    out["tma_feed_gbs_256MiB"] = _call(lib.dcopf_probe_tma_feed, 256 << 20)
    ex = {}
    sms = prop.multi_processor_count
    for c in (2, 4, 8):
        for div in (1, 2, 4):
            g = max(c, sms // div // c * c)
            key = f"{g // c}x{c}"
            if key in ex:
                continue
            ex[key] = _call(lib.dcopf_probe_exchange, c, g, exchange_gens, loops)
    if sms >= 144:   # the fused solve's shape on the 2000-bus network: 36 clusters of 4
        ex["36x4"] = _call(lib.dcopf_probe_exchange, 4, 144, exchange_gens, loops)
    out["exchange_us_per_loop"] = ex
    out["exchange_n_gen"] = exchange_gens
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--exchange-gens", type=int, default=540)
    ap.add_argument("--loops", type=int, default=2000)
    a = ap.parse_args()
    print(json.dumps(run(a.exchange_gens, a.loops)))


if __name__ == "__main__":
    main()
