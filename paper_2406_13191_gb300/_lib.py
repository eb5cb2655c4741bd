"""ctypes view of include/dcopf_dual.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdcopfdual.so")

# The exported C symbols, in the order include/dcopf_dual.h declares them.
EXPORTS = ("dcopf_version", "dcopf_status_string", "dcopf_solve_params_default",
           "dcopf_dual_create", "dcopf_dual_destroy", "dcopf_dual_info", "dcopf_dual_eval",
           "dcopf_dual_certify_bound", "dcopf_dual_primal_bound", "dcopf_dual_solve_batch",
           "dcopf_dual_kernel_launches",
           "dcopf_dual_device_error", "dcopf_dual_set_timing", "dcopf_dual_read_timing",
           "dcopf_dual_screened_lines", "dcopf_dual_read_kernel_timing", "dcopf_dual_tensor_shapes",
           "dcopf_dual_workspace_limit", "dcopf_selftest_bounded_wait",
           "dcopf_selftest_fused_timeout", "dcopf_dual_eval_noalloc", "dcopf_dual_solve_group",
           "dcopf_mlp_create", "dcopf_mlp_destroy", "dcopf_mlp_num_params", "dcopf_mlp_set_params",
           "dcopf_mlp_get_params", "dcopf_mlp_set_normalization", "dcopf_mlp_forward",
           "dcopf_mlp_loss_grad", "dcopf_mlp_train_step", "dcopf_mlp_warm_start",
           "dcopf_mlp_device_error", "dcopf_mlp_kernel_launches",
           "dcopf_probe_read", "dcopf_probe_smem", "dcopf_probe_fma", "dcopf_probe_tma_feed",
           "dcopf_probe_exchange")

STATUS = {0: "DCOPF_OK", 1: "DCOPF_ERR_INVALID_ARG", 2: "DCOPF_ERR_NETWORK", 3: "DCOPF_ERR_CUDA",
          4: "DCOPF_ERR_OOM", 5: "DCOPF_ERR_TIMEOUT", 6: "DCOPF_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16x3": 2}
RULE = {"gdm": 0, "adam": 1, "adagrad": 2}
PATH = {"auto": 0, "plain": 1, "fused": 2, "batched": 3, "sparse": 4}

P = C.c_void_p
I32P = C.POINTER(C.c_int32)
F64P = C.POINTER(C.c_double)


class NetworkDesc(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_line", C.c_int32), ("n_gen", C.c_int32),
                ("slack_bus", C.c_int32), ("line_from", I32P), ("line_to", I32P),
                ("line_b", F64P), ("flow_max", F64P), ("flow_min", F64P), ("gen_bus", I32P),
                ("pmin", F64P), ("pmax", F64P), ("cost_lin", F64P), ("cost_quad", F64P),
                ("base_mva", C.c_double)]


class Options(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_batch", C.c_int32), ("verbose", C.c_int32),
                ("operator_form", C.c_int32)]


class SolveParams(C.Structure):
    _fields_ = [("rule", C.c_int32), ("precision", C.c_int32), ("path", C.c_int32),
                ("max_iters", C.c_int32), ("warm_start", C.c_int32), ("as_printed", C.c_int32),
                ("check_every", C.c_int32), ("screen_lines", C.c_int32), ("alpha", C.c_double),
                ("alpha_lambda", C.c_double), ("rho", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("decay", C.c_double),
                ("gap", C.c_double), ("tol", C.c_double), ("target_value", P),
                ("mean_dispatch", P), ("qp_dual_s", C.c_int32), ("reserved", C.c_int32)]


class GroupItem(C.Structure):
    _fields_ = [("net", P), ("batch", C.c_int32), ("reserved", C.c_int32), ("params", P), ("loads", P),
                ("outage", P), ("target_value", P), ("lambda_", P), ("mu_hi", P), ("mu_lo", P),
                ("best_bound", P), ("iters", P), ("inst_status", P)]


class MlpDesc(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("n_hidden", C.c_int32), ("n_out", C.c_int32),
                ("max_batch", C.c_int32), ("precision", C.c_int32)]


class AdamParams(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


class DcopfError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


_lib = None


def load(build_if_missing: bool = True) -> C.CDLL:
    """Loads libdcopfdual.so (building it with nvcc if it is missing or stale).  Raises if the
    native library cannot be loaded: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and os.path.isdir(os.path.join(HERE, "csrc")):
        from . import build as _build
        _build.build()          # no-op when the library is newer than its sources
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"native library missing: {LIB_PATH}")
    lib = C.CDLL(LIB_PATH)
    lib.dcopf_version.restype = C.c_char_p
    lib.dcopf_status_string.restype = C.c_char_p
    lib.dcopf_status_string.argtypes = [C.c_int]
    lib.dcopf_solve_params_default.argtypes = [C.POINTER(SolveParams)]
    lib.dcopf_solve_params_default.restype = None
    lib.dcopf_dual_create.argtypes = [C.POINTER(NetworkDesc), C.POINTER(Options), C.POINTER(P)]
    lib.dcopf_dual_destroy.argtypes = [P]
    lib.dcopf_dual_info.argtypes = [P, I32P, I32P, I32P, I32P, C.POINTER(C.c_uint8)]
    lib.dcopf_dual_eval.argtypes = [P, C.c_int32, P, P, P, P, P, C.c_int32, P, P, P, P, P, P]
    lib.dcopf_dual_certify_bound.argtypes = [P, C.c_int32, P, P, P, P, P, P, P, P]
    lib.dcopf_dual_solve_batch.argtypes = [P, C.c_int32, P, P, C.POINTER(SolveParams), P, P, P, P,
                                           P, P, P]
    lib.dcopf_dual_kernel_launches.argtypes = [P]
    lib.dcopf_dual_kernel_launches.restype = C.c_int64
    lib.dcopf_dual_device_error.argtypes = [P]
    lib.dcopf_dual_set_timing.argtypes = [P, C.c_int32]
    lib.dcopf_selftest_bounded_wait.argtypes = [P, C.c_int64, P]
    lib.dcopf_selftest_fused_timeout.argtypes = [P, P, C.c_int64, P]
    lib.dcopf_dual_workspace_limit.argtypes = [P, C.c_int64, C.POINTER(C.c_int64)]
    lib.dcopf_dual_read_kernel_timing.argtypes = [P, F64P, C.POINTER(C.c_int64)]
    lib.dcopf_dual_tensor_shapes.argtypes = [P, I32P]
    lib.dcopf_dual_screened_lines.argtypes = [P, I32P, C.POINTER(C.c_uint8)]
    lib.dcopf_dual_eval_noalloc.argtypes = [P, C.c_int32, P, P, P, P, P, C.c_int32, P, P, P, P,
                                            P, P]
    lib.dcopf_dual_read_timing.argtypes = [P, F64P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.dcopf_dual_solve_group.argtypes = [C.c_int32, C.POINTER(GroupItem), C.POINTER(SolveParams), P]
    lib.dcopf_dual_solve_group.restype = C.c_int
    lib.dcopf_mlp_create.argtypes = [C.POINTER(MlpDesc), C.POINTER(P)]
    lib.dcopf_mlp_destroy.argtypes = [P]
    lib.dcopf_mlp_num_params.argtypes = [P]
    lib.dcopf_mlp_num_params.restype = C.c_int64
    lib.dcopf_mlp_set_params.argtypes = [P, P, P]
    lib.dcopf_mlp_get_params.argtypes = [P, P, P]
    lib.dcopf_mlp_set_normalization.argtypes = [P, P, P, P, P, P]
    lib.dcopf_mlp_forward.argtypes = [P, C.c_int32, P, P, P]
    lib.dcopf_mlp_loss_grad.argtypes = [P, C.c_int32, P, C.c_int64, P, P, P, P, P]
    lib.dcopf_mlp_train_step.argtypes = [P, C.c_int32, P, C.c_int64, P, P,
                                         C.POINTER(AdamParams), P, P]
    lib.dcopf_mlp_warm_start.argtypes = [P, C.c_int32, P, P, P, P, P]
    lib.dcopf_mlp_device_error.argtypes = [P]
    lib.dcopf_probe_read.argtypes = [C.c_int64, C.c_int32, F64P]
    lib.dcopf_probe_smem.argtypes = [F64P]
    lib.dcopf_probe_fma.argtypes = [C.c_int32, F64P, F64P]
    lib.dcopf_probe_tma_feed.argtypes = [C.c_int64, F64P]
    lib.dcopf_probe_exchange.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, F64P]
    for name in ("dcopf_probe_read", "dcopf_probe_smem", "dcopf_probe_fma", "dcopf_probe_tma_feed",
                 "dcopf_probe_exchange"):
        getattr(lib, name).restype = C.c_int
    lib.dcopf_mlp_kernel_launches.argtypes = [P]
    lib.dcopf_mlp_kernel_launches.restype = C.c_int64
    for name in ("dcopf_mlp_create", "dcopf_mlp_destroy", "dcopf_mlp_set_params",
                 "dcopf_mlp_get_params", "dcopf_mlp_set_normalization", "dcopf_mlp_forward",
                 "dcopf_mlp_loss_grad", "dcopf_mlp_train_step", "dcopf_mlp_warm_start",
                 "dcopf_mlp_device_error"):
        getattr(lib, name).restype = C.c_int
    for name in ("dcopf_dual_create", "dcopf_dual_destroy", "dcopf_dual_info", "dcopf_dual_eval",
                 "dcopf_dual_certify_bound", "dcopf_dual_solve_batch", "dcopf_dual_device_error",
                 "dcopf_dual_set_timing", "dcopf_dual_read_timing",
                 "dcopf_selftest_bounded_wait", "dcopf_dual_eval_noalloc", "dcopf_dual_solve_group",
                 "dcopf_selftest_fused_timeout", "dcopf_dual_workspace_limit",
                 "dcopf_dual_read_kernel_timing", "dcopf_dual_screened_lines",
                 "dcopf_dual_tensor_shapes",
           "dcopf_mlp_create", "dcopf_mlp_destroy", "dcopf_mlp_num_params", "dcopf_mlp_set_params",
           "dcopf_mlp_get_params", "dcopf_mlp_set_normalization", "dcopf_mlp_forward",
           "dcopf_mlp_loss_grad", "dcopf_mlp_train_step", "dcopf_mlp_warm_start",
           "dcopf_mlp_device_error", "dcopf_mlp_kernel_launches"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != 0:
        raise DcopfError(code, where)
