"""C ABI checks that need no GPU: the library builds and loads, exports every
function the headers in include/ declare, and rejects invalid networks on the host
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2406_13191_gb300 import _lib, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dcopf_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = _lib.load()
    names = header_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(_lib.EXPORTS)
    assert b"sm_103a" in lib.dcopf_version()
    for code in range(7):
        assert lib.dcopf_status_string(code)


def test_default_params():
    lib = _lib.load()
    p = _lib.SolveParams()
    lib.dcopf_solve_params_default(C.byref(p))
    assert p.rule == 1 and p.precision == 1 and p.max_iters == 5000 and p.gap == 1e-3
    assert p.alpha == 1000.0 and p.beta2 == 0.999 and p.decay == 1.0


def _desc(d, keep):
    def arr(v, dt):
        if v is None:
            return None
        a = np.ascontiguousarray(np.asarray(v, dtype=dt))
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int32 if dt == np.int32 else C.c_double))
    desc = _lib.NetworkDesc()
    desc.n_bus = d["n_bus"]
    desc.n_line = len(d["line_from"])
    desc.n_gen = len(d["gen_bus"])
    desc.slack_bus = d.get("slack_bus", 0)
    desc.line_from = arr(d["line_from"], np.int32)
    desc.line_to = arr(d["line_to"], np.int32)
    desc.line_b = arr(d["line_b"], np.float64)
    desc.flow_max = arr(d["flow_max"], np.float64)
    desc.flow_min = arr(d.get("flow_min"), np.float64)
    desc.gen_bus = arr(d["gen_bus"], np.int32)
    desc.pmin = arr(d["pmin"], np.float64)
    desc.pmax = arr(d["pmax"], np.float64)
    desc.cost_lin = arr(d["cost_lin"], np.float64)
    desc.cost_quad = arr(d.get("cost_quad"), np.float64)
    desc.base_mva = d.get("base_mva", 100.0)
    return desc


def _create(d):
    lib = _lib.load()
    keep = []
    desc = _desc(d, keep)
    h = C.c_void_p()
    code = lib.dcopf_dual_create(C.byref(desc), None, C.byref(h))
    if code == 0:
        lib.dcopf_dual_destroy(h)
    return code


def _good():
    net, _ = synth.tiny_network(3, 8, 11, 3)
    return net.as_dict()


@pytest.mark.parametrize("mutate,expect", [
    (lambda d: d.update(n_bus=0), 1),
    (lambda d: d.update(slack_bus=99), 1),
    (lambda d: d["line_b"].__setitem__(0, -1.0), 2),
    (lambda d: d["line_b"].__setitem__(0, np.nan), 1),
    (lambda d: d["pmin"].__setitem__(0, 5.0), 2),
    (lambda d: d["line_to"].__setitem__(0, 999), 1),
    (lambda d: d["gen_bus"].__setitem__(0, -2), 1),
    (lambda d: d.update(line_from=np.array(d["line_from"][:2]), line_to=np.array(d["line_to"][:2]),
                        line_b=np.array(d["line_b"][:2]), flow_max=np.array(d["flow_max"][:2]),
                        flow_min=np.array(d["flow_min"][:2])), 2),   # islanded
    (lambda d: d.update(base_mva=0.0), 1),
    (lambda d: d.update(n_bus=1, line_from=np.zeros(0, np.int32), line_to=np.zeros(0, np.int32),
                        line_b=np.zeros(0), flow_max=np.zeros(0), flow_min=np.zeros(0),
                        gen_bus=np.zeros(len(d["gen_bus"]), np.int32)), 6),   # no lines
])
def test_host_validation(mutate, expect):
    d = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in _good().items()}
    mutate(d)
    assert _create(d) == expect


def test_valid_network_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _create(_good()) == 3


@pytest.mark.parametrize("B,n", [(1, 41), (2, 5), (3, 7), (64, 3)])
def test_packed_result_views(B, n):
    """The binding's solve results are views of one FP64 buffer laid out
    [bound | lambda | iters | status | mu_hi | mu_lo], the int32 counts and statuses two
    per FP64 slot: the views tile the buffer without overlap, and writes through each
    view land where the layout says."""
    import torch
    from paper_2406_13191_gb300.dual import _packed_size, _packed_views
    flat = torch.zeros(_packed_size(B, n), dtype=torch.float64)
    lam, mh, ml, bound, iters, status = _packed_views(flat, B, n)
    assert lam.shape == (B,) and bound.shape == (B,) and mh.shape == (B, n) and ml.shape == (B, n)
    assert iters.shape == (B,) and status.shape == (B,)
    assert iters.dtype == torch.int32 and status.dtype == torch.int32
    bound.fill_(1.0); lam.fill_(2.0); mh.fill_(3.0); ml.fill_(4.0)
    iters.copy_(torch.arange(B, dtype=torch.int32) + 7)
    status.copy_(torch.arange(B, dtype=torch.int32) % 3)
    h = (B + 1) // 2
    assert torch.all(flat[:B] == 1.0) and torch.all(flat[B:2 * B] == 2.0)
    o = 2 * B + 2 * h
    assert torch.all(flat[o:o + B * n] == 3.0) and torch.all(flat[o + B * n:] == 4.0)
    ints = flat[2 * B:o].view(torch.int32)
    assert torch.equal(ints[:B], torch.arange(B, dtype=torch.int32) + 7)
    assert torch.equal(ints[2 * h:2 * h + B], torch.arange(B, dtype=torch.int32) % 3)
