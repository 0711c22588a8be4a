"""ctypes view of the C ABI in include/bcrown.h (argument marshalling only).

The shared library is built in-tree by ``paper_2103_06624_gb300.build_native``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbcrown.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNIMPLEMENTED = 0, -1, -2, -3, -4, -5, -6
LAYER_FC, LAYER_CONV = 0, 1
FP32, BF16, CERTIFY = 0, 1, 2
ALPHA_ADAPTIVE, ALPHA_FIXED = 0, 1
MAX_SPLITS = 64

EXPORTS = ["bcrown_load_net", "bcrown_free_net", "bcrown_net_info", "bcrown_root_bounds", "bcrown_bound",
           "bcrown_bound_grad", "bcrown_optimize", "bcrown_batch_split", "bcrown_neuron_codes",
           "bcrown_status", "bcrown_last_error", "bcrown_profile", "bcrown_profile_read",
           "bcrown_kernel_launches", "bcrown_bound_static", "bcrown_peak_probe", "bcrown_bound_xstar",
           "bcrown_forward", "bcrown_path_supported", "bcrown_set_launch", "bcrown_get_launch",
           "bcrown_autotune", "bcrown_joint_sizes", "bcrown_joint_init_alpha", "bcrown_bound_joint",
           "bcrown_bound_joint_grad", "bcrown_optimize_joint", "bcrown_workspace"]
FREEZE_ALPHA, FREEZE_BETA = 1, 2
PATH_DEFAULT, PATH_FUSED, PATH_LAYER_EPI, PATH_LAYER_GATHER, PATH_LAYER_IM2COL = range(5)
PATH_NAMES = {PATH_FUSED: "fused", PATH_LAYER_EPI: "layer_epi", PATH_LAYER_GATHER: "layer_gather",
              PATH_LAYER_IM2COL: "layer_im2col"}
PROF_CONTRACT, PROF_RELAX, PROF_CONCRETIZE, PROF_ADJOINT, PROF_ADAM, PROF_FUSED, PROF_LAYER_GEMM = range(7)


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int), ("in_c", C.c_int), ("in_h", C.c_int), ("in_w", C.c_int),
                ("out_c", C.c_int), ("out_h", C.c_int), ("out_w", C.c_int), ("k", C.c_int),
                ("stride", C.c_int), ("pad", C.c_int), ("W", C.c_void_p), ("b", C.c_void_p)]


class Domain(C.Structure):
    _fields_ = [("n_props", C.c_int), ("x_lo", C.c_void_p), ("x_hi", C.c_void_p),
                ("l", C.c_void_p), ("u", C.c_void_p)]


class Batch(C.Structure):
    _fields_ = [("B", C.c_int), ("prop_of", C.c_void_p), ("split_off", C.c_void_p),
                ("split_cnt", C.c_void_p), ("split_layer", C.c_void_p), ("split_idx", C.c_void_p),
                ("split_sign", C.c_void_p), ("alpha_off", C.c_void_p), ("n_alpha", C.c_int64),
                ("n_beta", C.c_int64)]


class OptCfg(C.Structure):
    _fields_ = [("iters", C.c_int), ("lr_alpha", C.c_float), ("lr_beta", C.c_float), ("decay", C.c_float),
                ("adam_beta1", C.c_float), ("adam_beta2", C.c_float), ("adam_eps", C.c_float),
                ("precision", C.c_int), ("certify", C.c_int), ("freeze", C.c_int)]


class OptState(C.Structure):
    _fields_ = [("alpha_cur", C.c_void_p), ("beta_cur", C.c_void_p), ("m_alpha", C.c_void_p),
                ("v_alpha", C.c_void_p), ("m_beta", C.c_void_p), ("v_beta", C.c_void_p),
                ("best_lb", C.c_void_p), ("t", C.c_int)]


class LaunchCfg(C.Structure):
    _fields_ = [("path", C.c_int), ("grid_per_sm", C.c_int)]


class BcrownError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bcrown error {code}: {msg}")
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load libbcrown.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbcrown.so not built at {path}; run paper_2103_06624_gb300.build_native.build()")
    lib = C.CDLL(path)
    vp, i32, f32 = C.c_void_p, C.c_int, C.c_float
    sig = {
        "bcrown_load_net": ([C.POINTER(Layer), i32, vp, i32, C.POINTER(vp)], i32),
        "bcrown_free_net": ([vp], None),
        "bcrown_net_info": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], i32),
        "bcrown_root_bounds": ([vp, i32, vp, vp, i32, f32, i32, vp, vp, vp, vp], i32),
        "bcrown_bound": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, i32, vp, vp], i32),
        "bcrown_bound_grad": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, i32, vp, vp, vp, vp], i32),
        "bcrown_optimize": ([vp, C.POINTER(Domain), C.POINTER(Batch), C.POINTER(OptCfg), vp, vp, vp,
                             C.POINTER(OptState), vp], i32),
        "bcrown_batch_split": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, vp, vp,
                                vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "bcrown_neuron_codes": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp], i32),
        "bcrown_status": ([vp, vp], i32),
        "bcrown_last_error": ([], C.c_char_p),
        "bcrown_profile": ([vp, i32], i32),
        "bcrown_profile_read": ([vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], i32),
        "bcrown_kernel_launches": ([], C.c_longlong),
        "bcrown_bound_static": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, vp, vp], i32),
        "bcrown_peak_probe": ([i32, i32, C.POINTER(C.c_double), vp], i32),
        "bcrown_bound_xstar": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, vp, vp, vp], i32),
        "bcrown_forward": ([vp, i32, vp, vp, vp], i32),
        "bcrown_path_supported": ([vp, i32], i32),
        "bcrown_set_launch": ([vp, C.POINTER(LaunchCfg)], i32),
        "bcrown_get_launch": ([vp, i32, C.POINTER(LaunchCfg)], i32),
        "bcrown_autotune": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, i32, C.POINTER(LaunchCfg),
                             C.POINTER(C.c_double), i32, C.POINTER(i32), C.POINTER(LaunchCfg), vp], i32),
        "bcrown_workspace": ([vp, C.c_int64, C.POINTER(vp), C.POINTER(C.c_int64)], i32),
        "bcrown_joint_sizes": ([vp, C.POINTER(Domain), C.POINTER(Batch), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64), vp], i32),
        "bcrown_joint_init_alpha": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, C.c_int64, vp], i32),
        "bcrown_bound_joint": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, vp, C.c_int64, vp, C.c_int64,
                                vp, vp, vp, vp], i32),
        "bcrown_bound_joint_grad": ([vp, C.POINTER(Domain), C.POINTER(Batch), vp, vp, vp, C.c_int64, vp,
                                     C.c_int64, vp, vp, vp, vp, vp, vp], i32),
        "bcrown_optimize_joint": ([vp, C.POINTER(Domain), C.POINTER(Batch), C.POINTER(OptCfg), vp, vp, vp,
                                   C.c_int64, vp, C.c_int64, vp, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(code):
    if code != OK:
        msg = load().bcrown_last_error().decode(errors="replace")
        raise BcrownError(code, msg)
    return code
