"""ctypes binding of ``libefunc.so`` (include/efunc.h): argument marshalling only.

Every entry point of the header is declared here with its C signature.  The
library is built in-tree on first use (nvcc) and fails loudly if it cannot be
built or loaded: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

c_int32, c_int64, c_float, c_double = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
c_size_t, c_void_p, c_char_p = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p
P_float = ctypes.POINTER(ctypes.c_float)

STATUS = {0: "EFUNC_OK", 1: "EFUNC_ERR_ARG", 2: "EFUNC_ERR_CUDA", 3: "EFUNC_ERR_WORKSPACE",
          4: "EFUNC_ERR_NONFINITE", 5: "EFUNC_ERR_UNSUPPORTED", 6: "EFUNC_ERR_IO", 7: "EFUNC_ERR_TIMEOUT"}
LOSS_L1, LOSS_MSE = 0, 1


class Grid(ctypes.Structure):
    _fields_ = [("R", c_int32), ("W", c_int32), ("log_beta0", c_float)]


class Adam(ctypes.Structure):
    _fields_ = [("lr", c_double), ("beta1", c_double), ("beta2", c_double), ("eps", c_double),
                ("weight_decay", c_double), ("decoupled", c_int32)]


class Variant(ctypes.Structure):
    _fields_ = [("sets", c_int32), ("degree", c_int32), ("learn_scale", c_int32)]


class CheckpointInfo(ctypes.Structure):
    _fields_ = [("R", c_int32), ("W", c_int32), ("log_beta0", c_float), ("channels", c_int32), ("n", c_int64),
                ("step", c_int64), ("seed", ctypes.c_uint64), ("loss", c_int32), ("adam", Adam)]


class Shape(ctypes.Structure):
    _fields_ = [("R", c_int32), ("log_beta0", c_float), ("J", c_int64)]


class Tuning(ctypes.Structure):
    _fields_ = [("chunk", c_int32), ("lanes2_max", c_int32), ("lanes4_max", c_int32), ("sort_blocks", c_int32),
                ("group_max", c_int32)]


KEYS_GRID, KEYS_OFFSET, KEYS_BOTH = 1, 2, 3

# name -> (restype, argtypes); the order follows include/efunc.h
SIGNATURES = {
    "efunc_param_count": (c_int64, [c_int32]),
    "efunc_default_log_beta0": (c_float, [c_int32]),
    "efunc_status_str": (c_char_p, [c_int32]),
    "efunc_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), c_int64]),
    "efunc_eval_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), c_int64]),
    "efunc_fit_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), c_int64]),
    "efunc_cell_sort": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                  c_void_p, c_size_t, c_void_p]),
    "efunc_forward": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_backward": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_backward_grad": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_eval_loss": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_size_t,
                                  c_void_p]),
    "efunc_f64_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), c_int64]),
    "efunc_forward_f64": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_backward_f64": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_adam_step": (c_int32, [ctypes.POINTER(Adam), c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                  c_void_p]),
    "efunc_fit": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Adam), c_int32, c_float, c_void_p, c_void_p,
                            c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64, c_void_p, c_void_p, c_size_t,
                            c_void_p]),
    "efunc_checkpoint_save": (c_int32, [c_char_p, ctypes.POINTER(CheckpointInfo), c_void_p, c_void_p, c_void_p]),
    "efunc_checkpoint_info_read": (c_int32, [c_char_p, ctypes.POINTER(CheckpointInfo)]),
    "efunc_checkpoint_load": (c_int32, [c_char_p, ctypes.POINTER(CheckpointInfo), c_void_p, c_void_p, c_void_p,
                                        c_int64]),
    "efunc_last_cuda_error": (c_int32, []),
    "efunc_cuda_error_name": (ctypes.c_char_p, [c_int32]),
    "efunc_fit_graph": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Adam), c_int32, c_float, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64, c_void_p, c_void_p,
                                  c_size_t, c_void_p]),
    "efunc_forward_noalloc": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_void_p]),
    "efunc_mean_shift_init": (c_int32, [ctypes.POINTER(Grid), c_void_p, c_int64, c_float, c_void_p, c_void_p]),
    "efunc_variant_channels": (c_int32, [ctypes.POINTER(Variant)]),
    "efunc_variant_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), ctypes.POINTER(Variant), c_int64]),
    "efunc_variant_forward": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Variant), c_void_p, c_void_p, c_int64,
                                        c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_variant_backward": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Variant), c_void_p, c_void_p, c_int64,
                                         c_int32, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_variant_fit": (c_int32, [ctypes.POINTER(Grid), ctypes.POINTER(Variant), ctypes.POINTER(Adam), c_int32,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64,
                                    c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_cosine_workspace_bytes": (c_size_t, [ctypes.POINTER(Grid), c_int32, c_int64]),
    "efunc_cosine_forward": (c_int32, [ctypes.POINTER(Grid), c_int32, c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                                       c_void_p, c_size_t, c_void_p]),
    "efunc_cosine_backward": (c_int32, [ctypes.POINTER(Grid), c_int32, c_void_p, c_void_p, c_int64, c_int32,
                                        c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_cosine_fit": (c_int32, [ctypes.POINTER(Grid), c_int32, ctypes.POINTER(Adam), c_int32, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64, c_void_p, c_void_p,
                                   c_size_t, c_void_p]),
    "efunc_default_tuning": (None, [ctypes.POINTER(Tuning)]),
    "efunc_batched_param_count": (c_int64, [ctypes.POINTER(Shape), c_int32]),
    "efunc_batched_query_count": (c_int64, [ctypes.POINTER(Shape), c_int32]),
    "efunc_batched_workspace_bytes": (c_size_t, [ctypes.POINTER(Shape), c_int32]),
    "efunc_fit_batched": (c_int32, [ctypes.POINTER(Shape), c_int32, ctypes.POINTER(Adam), c_int32, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_int32, c_int32, c_int64, c_void_p, ctypes.POINTER(Tuning),
                                    c_int32, c_void_p, c_size_t, c_void_p]),
    "efunc_eval_batched": (c_int32, [ctypes.POINTER(Shape), c_int32, c_void_p, c_void_p, c_void_p,
                                     ctypes.POINTER(Tuning), c_void_p, c_size_t, c_void_p]),
    "efunc_tune_batched": (c_int32, [ctypes.POINTER(Shape), c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_int32, c_int32, ctypes.POINTER(Tuning), ctypes.POINTER(c_double), c_void_p,
                                     c_size_t, c_void_p]),
    "efunc_encoder_weight_count": (c_int64, []),
    "efunc_encoder_workspace_bytes": (c_size_t, [c_int32]),
    "efunc_encoder_forward": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
    "efunc_encoder_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                           c_void_p, c_size_t, c_void_p]),
    "efunc_encoder_status": (c_int32, [c_void_p]),
    "efunc_conv3d_bf16": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p, c_int32,
                                    c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "efunc_conv3d_wgrad_bf16": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32, c_int32, c_void_p,
                                          c_void_p, c_void_p]),
    "efunc_profile_enable": (None, [c_int32]),
    "efunc_profile_read": (c_int32, [c_char_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "efunc_profile_reset": (None, []),
    "efunc_launch_count": (c_int64, []),
    "efunc_debug_bounds": (c_int32, [ctypes.POINTER(c_int32)]),
}

_lock = threading.Lock()
_lib = None


def debug_bounds_requested() -> bool:
    """EFUNC_DEBUG_BOUNDS=1 selects the bounds-checking build of the library."""
    return os.environ.get("EFUNC_DEBUG_BOUNDS", "0") not in ("", "0")


def load(build: bool = True) -> ctypes.CDLL:
    """Build (if needed) and load the library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            debug = debug_bounds_requested()
            path = _build.lib_path(debug)
            if build and not _build.up_to_date(debug):
                _build.build(debug=debug)
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing and could not be built")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class EfuncError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = load()
        msg = lib.efunc_status_str(code).decode()
        self.cuda_error = None
        if code == 2:   # EFUNC_ERR_CUDA: name the CUDA error behind it
            self.cuda_error = int(lib.efunc_last_cuda_error())
            msg += ": " + (lib.efunc_cuda_error_name(self.cuda_error) or b"?").decode()
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({msg})")
        self.code = code


def check(fn: str, code: int) -> None:
    if code != 0:
        raise EfuncError(fn, code)
