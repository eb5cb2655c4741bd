"""Python binding of the C ABI: torch tensors in, torch tensors out.

Every numeric step runs in libdcopfdual.so; this module only checks shapes, moves
arguments to contiguous float64/int32 CUDA tensors and passes raw pointers and the
current CUDA stream.  There is no CPU implementation: without the native library
or without a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


def _as_dev(x, dtype, device):
    if x is None:
        return None
    t = x if isinstance(x, torch.Tensor) else torch.as_tensor(np.asarray(x))
    # pinned host memory goes up asynchronously, ordered on the current stream before
    # the library call that reads it
    nb = t.device.type == "cpu" and t.dtype == dtype and t.is_pinned()
    return t.to(device=device, dtype=dtype, non_blocking=nb).contiguous()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _packed_views(flat: torch.Tensor, B: int, n: int):
    """(lam, mu_hi, mu_lo, bound, iters, status) as views of one flat FP64 buffer laid
    out [bound | lam | iters | status | mu_hi | mu_lo]; iters and status are int32
    views over ceil(B/2) FP64 slots each."""
    h = (B + 1) // 2
    o = 2 * B
    iters = flat[o:o + h].view(torch.int32)[:B]
    status = flat[o + h:o + 2 * h].view(torch.int32)[:B]
    o += 2 * h
    return (flat[B:2 * B], flat[o:o + B * n].view(B, n), flat[o + B * n:o + 2 * B * n].view(B, n),
            flat[:B], iters, status)


def _packed_size(B: int, n: int) -> int:
    return 2 * B + 2 * ((B + 1) // 2) + 2 * B * n


@dataclass
class SolveResult:
    lam: torch.Tensor          # [B] best iterate, lambda
    mu_hi: torch.Tensor        # [B][n_line]
    mu_lo: torch.Tensor        # [B][n_line]
    bound: torch.Tensor        # [B] certified FP64 lower bound
    iters: torch.Tensor        # [B] iterations taken
    status: torch.Tensor       # [B] 0 target reached, 1 cap/tol, 2 infeasible suspected
    mean_dispatch: torch.Tensor | None = None  # [B][n_gen] k^2-weighted mean of the minimisers
    flat: torch.Tensor | None = None  # the device buffer the six results are views of

    def to_host(self, into: "SolveResult | None" = None) -> "SolveResult":
        """The results in host memory with one device-to-host transfer, ordered after
        the work already on the current stream.  Results made by ``new_result`` (or by
        ``solve`` without ``out=``) are views of one device buffer, which is copied as it
        is: into ``into`` when given (a result from ``new_host_result``, whose buffer is
        pinned, so that the copy runs at the host link's rate; it is reused, and the call
        returns once the copy is in), else by one blocking copy into new host memory
        (for small results faster on a Grace host than an asynchronous copy followed by
        a stream synchronisation).  Results that are not such views are packed on the
        device first (iteration counts and statuses travel exactly as FP64)."""
        B, n = self.mu_hi.shape
        if self.flat is not None:
            if into is not None:
                if into.flat is None or into.flat.shape != self.flat.shape or into.flat.device.type != "cpu":
                    raise ValueError("into= is not a host result of this batch")
                into.flat.copy_(self.flat, non_blocking=into.flat.is_pinned())
                torch.cuda.current_stream(self.flat.device).synchronize()
                return into
            host = self.flat.cpu()
            return SolveResult(*_packed_views(host, B, n), flat=host)
        if into is not None:
            raise ValueError("into= needs results that are views of one device buffer (new_result)")
        packed = torch.cat([self.bound, self.lam, self.iters.double(), self.status.double(),
                            self.mu_hi.reshape(-1), self.mu_lo.reshape(-1)]).cpu()
        o = 4 * B
        return SolveResult(packed[B:2 * B], packed[o:o + B * n].reshape(B, n),
                           packed[o + B * n:].reshape(B, n), packed[:B],
                           packed[2 * B:3 * B].int(), packed[3 * B:4 * B].int())


class DcopfDual:
    """One network on one GPU (``dcopf_dual_create``).

    ``net`` is a ``synth.Network`` or any object/dict with its fields (n_bus,
    line_from, line_to, line_b, flow_max, flow_min, gen_bus, pmin, pmax, cost_lin,
    cost_quad, base_mva, slack_bus)."""

    def __init__(self, net, device: int | None = None, verbose: bool = False,
                 operator_form: str = "ptdf"):
        """``operator_form``: "ptdf" (the PTDF Phi~ and the sparse factor, every call) or
        "sparse" (the sparse factor only, no PTDF: path="sparse" solves and certificates)."""
        self.lib = _lib.load()
        d = net.as_dict() if hasattr(net, "as_dict") else dict(net)
        self._keep = []

        def arr(v, dt):
            if v is None:
                return None
            a = np.ascontiguousarray(np.asarray(v, dtype=dt))
            self._keep.append(a)
            ct = C.c_int32 if dt == np.int32 else C.c_double
            return a.ctypes.data_as(C.POINTER(ct))

        desc = _lib.NetworkDesc()
        desc.n_bus = int(d["n_bus"])
        desc.n_line = len(d["line_from"])
        desc.n_gen = len(d["gen_bus"])
        desc.slack_bus = int(d.get("slack_bus", 0))
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
        desc.base_mva = float(d.get("base_mva", 100.0))
        opt = _lib.Options()
        opt.device = -1 if device is None else int(device)
        opt.verbose = 1 if verbose else 0
        opt.operator_form = {"ptdf": 0, "sparse": 1}[operator_form]
        h = C.c_void_p()
        _lib.check(self.lib.dcopf_dual_create(C.byref(desc), C.byref(opt), C.byref(h)),
                   "dcopf_dual_create")
        self._keep = []
        self.h = h
        self.n_bus, self.n_line, self.n_gen = desc.n_bus, desc.n_line, desc.n_gen
        self.is_qp = desc.cost_quad is not None and bool(desc.cost_quad)
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", int(device))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dcopf_dual_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _batch_inputs(self, loads, outage):
        loads = _as_dev(loads, torch.float64, self.device)
        if loads.dim() == 1:
            loads = loads[None]
        if loads.shape[1] != self.n_bus:
            raise ValueError("loads must be [batch][n_bus]")
        out = _as_dev(outage, torch.int32, self.device)
        if out is not None and out.numel() != loads.shape[0]:
            raise ValueError("outage must be [batch]")
        return loads, out

    def bridge_mask(self) -> np.ndarray:
        m = np.zeros(self.n_line, dtype=np.uint8)
        _lib.check(self.lib.dcopf_dual_info(self.h, None, None, None, None,
                                            m.ctypes.data_as(C.POINTER(C.c_uint8))),
                   "dcopf_dual_info")
        return m.astype(bool)

    def kernel_launches(self) -> int:
        return int(self.lib.dcopf_dual_kernel_launches(self.h))

    def set_timing(self, enable: bool = True) -> None:
        _lib.check(self.lib.dcopf_dual_set_timing(self.h, 1 if enable else 0), "set_timing")

    def read_timing(self):
        """(iteration-kernel milliseconds, their launches, evaluations), then reset."""
        ms = C.c_double()
        nl = C.c_int64()
        ne = C.c_int64()
        _lib.check(self.lib.dcopf_dual_read_timing(self.h, C.byref(ms), C.byref(nl), C.byref(ne)),
                   "read_timing")
        return ms.value, nl.value, ne.value

    def screened_lines(self) -> np.ndarray:
        """``dcopf_dual_screened_lines``: boolean [n_line], True for the lines the last
        screened solve iterated on (all False before any screened solve)."""
        m = np.zeros(self.n_line, dtype=np.uint8)
        n = C.c_int32()
        _lib.check(self.lib.dcopf_dual_screened_lines(self.h, C.byref(n), m.ctypes.data_as(C.POINTER(C.c_uint8))),
                   "dcopf_dual_screened_lines")
        return m.astype(bool)

    KERNELS = ("adjoint", "minimiser", "forward", "step", "value")

    def read_kernel_timing(self):
        """``dcopf_dual_read_kernel_timing``: {kernel: summed ms} over the sampled
        iterations of batched solves, and the sample count; then reset."""
        ms = (C.c_double * 5)()
        n = C.c_int64()
        _lib.check(self.lib.dcopf_dual_read_kernel_timing(self.h, ms, C.byref(n)),
                   "dcopf_dual_read_kernel_timing")
        return dict(zip(self.KERNELS, list(ms))), n.value

    def tensor_shapes(self) -> dict:
        """``dcopf_dual_tensor_shapes``: the product shapes of the last batched solve."""
        v = (C.c_int32 * 7)()
        _lib.check(self.lib.dcopf_dual_tensor_shapes(self.h, v), "dcopf_dual_tensor_shapes")
        tiles = ("single 128x128", "pairs 256x256", "pairs 256x192", "pairs 256x160", "pairs 256x144",
                 "2 pairs 256x256", "2 pairs 256x192", "2 pairs 256x160", "2 pairs 256x144")
        return {"batch": v[0], "lines": v[1], "adjoint": tiles[v[2]], "adjoint_split_k": v[3],
                "forward": tiles[v[4]], "branches": v[5], "first_group": v[6],
                "code": f"{v[2]},{v[3]},{v[4]},{v[5]}"}

    def workspace_limit(self, limit_bytes: int | None = None) -> int:
        """``dcopf_dual_workspace_limit``: sets the workspace budget in bytes (0 = none;
        None leaves it unchanged) and returns the bytes the workspaces hold now."""
        used = C.c_int64()
        _lib.check(self.lib.dcopf_dual_workspace_limit(
            self.h, -1 if limit_bytes is None else int(limit_bytes), C.byref(used)),
            "dcopf_dual_workspace_limit")
        return used.value

    def selftest_fused_timeout(self, loads, timeout_ns: int) -> int:
        """``dcopf_selftest_fused_timeout``: the status code of a fused solve whose
        inter-cluster wait cannot complete (DCOPF_ERR_TIMEOUT = 5 expected)."""
        ld = _as_dev(loads, torch.float64, self.device).reshape(self.n_bus)
        return int(self.lib.dcopf_selftest_fused_timeout(self.h, _ptr(ld), int(timeout_ns),
                                                         self._stream()))

    # ------------------------------------------------------------------ entry points
    def eval(self, loads, lam, mu_hi, mu_lo, outage=None, precision: str = "fp64",
             want_grad: bool = True, want_dispatch: bool = True):
        """``dcopf_dual_eval``: dual value, supergradient and minimiser at (lambda, mu)."""
        loads, out = self._batch_inputs(loads, outage)
        B = loads.shape[0]
        lam = _as_dev(lam, torch.float64, self.device).reshape(B)
        mh = _as_dev(mu_hi, torch.float64, self.device).reshape(B, self.n_line)
        ml = _as_dev(mu_lo, torch.float64, self.device).reshape(B, self.n_line)
        kw = dict(dtype=torch.float64, device=self.device)
        value = torch.empty(B, **kw)
        gl = torch.empty(B, **kw) if want_grad else None
        ghi = torch.empty(B, self.n_line, **kw) if want_grad else None
        glo = torch.empty(B, self.n_line, **kw) if want_grad else None
        disp = torch.empty(B, self.n_gen, **kw) if want_dispatch else None
        _lib.check(self.lib.dcopf_dual_eval(self.h, B, _ptr(loads), _ptr(out), _ptr(lam), _ptr(mh),
                                            _ptr(ml), _lib.PRECISION[precision], _ptr(value),
                                            _ptr(gl), _ptr(ghi), _ptr(glo), _ptr(disp),
                                            self._stream()), "dcopf_dual_eval")
        return dict(value=value, g_lambda=gl, g_mu_hi=ghi, g_mu_lo=glo, dispatch=disp)

    def certify(self, loads, lam, mu_hi, mu_lo, outage=None):
        """``dcopf_dual_certify_bound``: certified FP64 bound and its rounding allowance."""
        loads, out = self._batch_inputs(loads, outage)
        B = loads.shape[0]
        lam = _as_dev(lam, torch.float64, self.device).reshape(B)
        mh = _as_dev(mu_hi, torch.float64, self.device).reshape(B, self.n_line)
        ml = _as_dev(mu_lo, torch.float64, self.device).reshape(B, self.n_line)
        bound = torch.empty(B, dtype=torch.float64, device=self.device)
        err = torch.empty(B, dtype=torch.float64, device=self.device)
        _lib.check(self.lib.dcopf_dual_certify_bound(self.h, B, _ptr(loads), _ptr(out), _ptr(lam),
                                                     _ptr(mh), _ptr(ml), _ptr(bound), _ptr(err),
                                                     self._stream()), "dcopf_dual_certify_bound")
        return bound, err

    def primal_bound(self, loads, lam=None, mu_hi=None, mu_lo=None, outage=None, p_ref=None,
                     p_cand=None):
        """``dcopf_dual_primal_bound``: a feasible dispatch recovered from the dual point (or
        from the candidate ``p_cand``, e.g. a solve's mean_dispatch) and its cost, an
        upper bound on gamma*.  Returns (upper, status, dispatch, max_violation); upper
        is +inf and the dispatch NaN where status != 0 (1: demand outside the generator
        box, 2: the reference dispatch is infeasible)."""
        loads, out = self._batch_inputs(loads, outage)
        B = loads.shape[0]

        def opt(x, shape):
            return None if x is None else _as_dev(x, torch.float64, self.device).reshape(shape)
        lam, mh, ml = opt(lam, (B,)), opt(mu_hi, (B, self.n_line)), opt(mu_lo, (B, self.n_line))
        pr, pc = opt(p_ref, (B, self.n_gen)), opt(p_cand, (B, self.n_gen))
        upper = torch.empty(B, dtype=torch.float64, device=self.device)
        status = torch.empty(B, dtype=torch.int32, device=self.device)
        disp = torch.empty(B, self.n_gen, dtype=torch.float64, device=self.device)
        viol = torch.empty(B, dtype=torch.float64, device=self.device)
        _lib.check(self.lib.dcopf_dual_primal_bound(self.h, B, _ptr(loads), _ptr(out), _ptr(lam),
                                                    _ptr(mh), _ptr(ml), _ptr(pc), _ptr(pr), _ptr(upper),
                                                    _ptr(status), _ptr(disp), _ptr(viol),
                                                    self._stream()), "dcopf_dual_primal_bound")
        return upper, status, disp, viol

    def _params(self, rule, precision, path, max_iters, alpha, alpha_lambda, rho, beta1, beta2, eps,
                decay, gap, tol, as_printed, check_every, screen=False, qp_dual="closed", warm=False):
        p = _lib.SolveParams()
        self.lib.dcopf_solve_params_default(C.byref(p))
        p.rule = _lib.RULE[rule]
        p.precision = _lib.PRECISION[precision]
        p.path = _lib.PATH[path]
        p.max_iters = int(max_iters)
        p.warm_start = 1 if warm else 0
        p.as_printed = 1 if as_printed else 0
        p.check_every = int(check_every)
        p.screen_lines = 1 if screen else 0
        p.qp_dual_s = {"closed": 0, "s": 1}[qp_dual]
        p.alpha, p.alpha_lambda, p.rho = float(alpha), float(alpha_lambda), float(rho)
        p.beta1, p.beta2, p.eps, p.decay = float(beta1), float(beta2), float(eps), float(decay)
        p.gap, p.tol = float(gap), float(tol)
        return p

    def new_result(self, batch: int) -> SolveResult:
        """Output tensors for ``solve(..., out=...)`` (reusable across calls): views of
        one device buffer, so that ``to_host`` is a single copy."""
        flat = torch.empty(_packed_size(batch, self.n_line), dtype=torch.float64, device=self.device)
        return SolveResult(*_packed_views(flat, batch, self.n_line), flat=flat)

    def new_host_result(self, batch: int) -> SolveResult:
        """A pinned host buffer laid out like ``new_result``'s, for ``to_host(into=...)``
        (reusable across calls)."""
        flat = torch.empty(_packed_size(batch, self.n_line), dtype=torch.float64).pin_memory()
        return SolveResult(*_packed_views(flat, batch, self.n_line), flat=flat)

    def _solve_arrays(self, loads, outage, target, warm, res=None):
        loads, out = self._batch_inputs(loads, outage)
        B = loads.shape[0]
        tgt = _as_dev(target, torch.float64, self.device)
        if tgt is not None:
            tgt = tgt.reshape(B)
        if res is not None:
            if res.lam.shape != (B,) or res.mu_hi.shape != (B, self.n_line) or res.lam.device != self.device:
                raise ValueError("out= does not match the batch")
        else:  # cold start: the library initialises the state and only writes these
            res = self.new_result(B)
        if warm is not None:
            res.lam.copy_(_as_dev(warm[0], torch.float64, self.device).reshape(B))
            res.mu_hi.copy_(_as_dev(warm[1], torch.float64, self.device).reshape(B, self.n_line))
            res.mu_lo.copy_(_as_dev(warm[2], torch.float64, self.device).reshape(B, self.n_line))
        return loads, out, tgt, res

    def solve(self, loads, outage=None, rule="adam", precision="fp32", path="auto",
              max_iters=5000, alpha=1000.0, alpha_lambda=0.0, rho=0.9, beta1=0.9, beta2=0.999,
              eps=1e-8, decay=1.0, gap=1e-3, tol=0.0, target=None, warm=None,
              as_printed=False, check_every=1, out: SolveResult | None = None,
              mean_dispatch: bool = False, screen: bool = False, qp_dual: str = "closed") -> SolveResult:
        """``dcopf_dual_solve_batch``.  ``target`` ([B] optimal costs) enables the
        certified-gap stop; ``warm`` = (lambda, mu_hi, mu_lo) warm start; ``out`` (from
        ``new_result``) receives the results instead of new tensors; ``mean_dispatch``
        also returns the k^2-weighted mean of the minimisers (a primal candidate); ``screen``
        turns on constraint screening (batched tensor-core solves without outages);
        ``qp_dual="s"`` ascends on eq. (16) with s as a variable (plain path, QP)."""
        loads, outg, tgt, r = self._solve_arrays(loads, outage, target, warm, out)
        p = self._params(rule, precision, path, max_iters, alpha, alpha_lambda, rho, beta1, beta2,
                         eps, decay, gap, tol, as_printed, check_every, screen=screen,
                         qp_dual=qp_dual, warm=warm is not None)
        p.target_value = None if tgt is None else tgt.data_ptr()
        if mean_dispatch:
            if r.mean_dispatch is None or r.mean_dispatch.shape != (r.lam.shape[0], self.n_gen):
                r.mean_dispatch = torch.empty(r.lam.shape[0], self.n_gen, dtype=torch.float64,
                                              device=self.device)
            p.mean_dispatch = r.mean_dispatch.data_ptr()
        _lib.check(self.lib.dcopf_dual_solve_batch(self.h, r.lam.shape[0], _ptr(loads), _ptr(outg),
                                                   C.byref(p), _ptr(r.lam), _ptr(r.mu_hi),
                                                   _ptr(r.mu_lo), _ptr(r.bound), _ptr(r.iters),
                                                   _ptr(r.status), self._stream()),
                   "dcopf_dual_solve_batch")
        return r


_SOLVE_DEFAULTS = dict(rule="adam", precision="bf16x3", path="batched", max_iters=5000,
                      alpha=1000.0, alpha_lambda=0.0, rho=0.9, beta1=0.9, beta2=0.999, eps=1e-8,
                      decay=1.0, gap=1e-3, tol=0.0, as_printed=False, check_every=1, screen=False,
                      qp_dual="closed")


def solve_group(duals, loads, outage=None, target=None, warm=None, per_network=None,
                **settings) -> list[SolveResult]:
    """``dcopf_dual_solve_group``: batched solves of several networks (one ``DcopfDual``
    each, distinct, on one device) advanced together, each round one CUDA-graph launch
    over all of them.  ``loads``, ``outage``, ``target``, ``warm`` are per-network lists
    (``None`` entries allowed); ``settings`` are the shared ascent settings (the keywords
    of ``DcopfDual.solve``) and ``per_network`` an optional list of dicts overriding
    them for one network."""
    n = len(duals)
    outage = outage or [None] * n
    target = target or [None] * n
    warm = warm or [None] * n
    per_network = per_network or [None] * n
    base = dict(_SOLVE_DEFAULTS, **settings)
    keep, items, res = [], (_lib.GroupItem * n)(), []
    for i, d in enumerate(duals):
        ld, out, tgt, r = d._solve_arrays(loads[i], outage[i], target[i], warm[i])
        keep += [ld, out, tgt]
        it = items[i]
        it.net = d.h.value
        it.batch = r.lam.shape[0]
        it.loads, it.outage = ld.data_ptr(), (None if out is None else out.data_ptr())
        it.target_value = None if tgt is None else tgt.data_ptr()
        it.lambda_, it.mu_hi, it.mu_lo = r.lam.data_ptr(), r.mu_hi.data_ptr(), r.mu_lo.data_ptr()
        it.best_bound, it.iters, it.inst_status = (r.bound.data_ptr(), r.iters.data_ptr(),
                                                   r.status.data_ptr())
        if per_network[i]:
            pi = d._params(**dict(base, **per_network[i]), warm=warm[i] is not None)
            keep.append(pi)
            it.params = C.cast(C.pointer(pi), C.c_void_p)
        res.append(r)
    d0 = duals[0]
    if any((w is None) != (warm[0] is None) for w in warm):
        raise ValueError("give a warm start for every network or for none")
    p = d0._params(**base, warm=warm[0] is not None)
    _lib.check(d0.lib.dcopf_dual_solve_group(n, items, C.byref(p), d0._stream()),
               "dcopf_dual_solve_group")
    return res
