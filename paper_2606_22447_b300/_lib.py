"""ctypes binding of libvcs (include/vcs.h).

Argument marshalling only: every step of the emulation runs in the library's
CUDA kernels.  The library is loaded from this package's directory; if it is
missing the import of this module fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvcs.so")

VCS_OK, VCS_ERR_ARG, VCS_ERR_ROM_SIZE, VCS_ERR_MAPPER = 0, 1, 2, 3
VCS_ERR_CUDA, VCS_ERR_OOM, VCS_ERR_WATCHDOG, VCS_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "VCS_OK", 1: "VCS_ERR_ARG", 2: "VCS_ERR_ROM_SIZE", 3: "VCS_ERR_MAPPER",
                4: "VCS_ERR_CUDA", 5: "VCS_ERR_OOM", 6: "VCS_ERR_WATCHDOG", 7: "VCS_ERR_STATE"}
ENV_WATCHDOG, ENV_JAMMED, ENV_DONE = 1, 2, 4


class VcsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class LossWeights(C.Structure):
    _fields_ = [("ram", C.c_void_p), ("screen", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("alpha", C.c_float), ("ystart", C.c_int32), ("boot_noop_frames", C.c_int32),
                ("boot_reset_frames", C.c_int32),
                ("envs_per_block", C.c_int32), ("segment_frames", C.c_int32),
                ("sched_policy", C.c_int32), ("sched_window", C.c_int32), ("steps_per_launch", C.c_int32),
                ("threads_per_env", C.c_int32), ("position_sampler", C.c_int32),
                ("step_instructions", C.c_int32), ("tape_budget_mb", C.c_int32), ("full_tia", C.c_int32),
                ("graphics_bits", C.c_int32), ("inline_render", C.c_int32),
                ("sweep_mode", C.c_int32)]


class Tune(C.Structure):
    _fields_ = [("envs_per_block", C.c_int32), ("threads_per_env", C.c_int32), ("sched_policy", C.c_int32),
                ("sched_window", C.c_int32),
                ("steps_per_launch", C.c_int32), ("ms_per_step", C.c_float), ("n_trials", C.c_int32)]


vp = C.c_void_p
i32 = C.c_int32
u8p = C.POINTER(C.c_uint8)

# name -> (restype, argtypes)
SIGNATURES = {
    "vcs_config_default": (C.c_int, [C.POINTER(Config)]),
    "vcs_create_batch": (C.c_int, [C.POINTER(u8p), C.POINTER(C.c_uint32), u8p, i32,
                                   C.POINTER(C.c_int32), i32, C.POINTER(Config), C.POINTER(vp)]),
    "vcs_destroy": (C.c_int, [vp]),
    "vcs_rom_stride": (C.c_int, [vp, C.POINTER(i32)]),
    "vcs_full_divergence": (C.c_int, [vp, C.c_float, C.c_float, vp, i32, vp, vp, vp, vp]),
    "vcs_last_error": (C.c_char_p, [vp]),
    "vcs_time_kernels": (C.c_int, [vp, i32]),
    "vcs_kernel_times": (C.c_int, [vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(i32),
                                   C.POINTER(C.c_double)]),
    "vcs_batch_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "vcs_set_episodes": (C.c_int, [vp, C.POINTER(C.c_uint32), i32]),
    "vcs_reset": (C.c_int, [vp, vp, vp]),
    "vcs_step": (C.c_int, [vp, vp, i32, vp, vp, vp, vp]),
    "vcs_rollout": (C.c_int, [vp, vp, i32, i32, vp, vp, vp, vp]),
    "vcs_step_host": (C.c_int, [vp, vp, i32, vp, vp, vp]),
    "vcs_sync": (C.c_int, [vp, vp]),
    "vcs_state_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
    "vcs_save_state": (C.c_int, [vp, vp, vp]),
    "vcs_load_state": (C.c_int, [vp, vp, vp]),
    "vcs_soft_rollout": (C.c_int, [vp, C.c_float, vp, vp, vp, i32, i32, vp, vp, C.POINTER(vp), vp]),
    "vcs_soft_step": (C.c_int, [vp, C.c_float, vp, i32, i32, vp, vp, C.POINTER(vp), vp]),
    "vcs_backward": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "vcs_tape_free": (C.c_int, [vp]),
    "vcs_backward_static": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "vcs_cart_ram": (C.c_int, [vp, vp, vp]),
    "vcs_detect_mapper": (C.c_int, [u8p, C.c_uint32, u8p]),
    "vcs_autotune": (C.c_int, [vp, i32, i32, vp, vp, vp, C.POINTER(Tune), vp]),
    "vcs_graph_create": (C.c_int, [vp, vp, i32, i32, vp, vp, vp, C.POINTER(vp)]),
    "vcs_graph_launch": (C.c_int, [vp, vp]),
    "vcs_graph_destroy": (C.c_int, [vp]),
    "vcs_digest": (C.c_int, [vp, vp, vp, i32, vp, vp]),
    "vcs_autotune_cache_clear": (C.c_int, []),
    "vcs_rollout_host": (C.c_int, [vp, vp, i32, i32, vp, vp, vp, vp]),
    "vcs_int_peak": (C.c_int, [C.POINTER(C.c_double), vp]),
    "vcs_set_start_noops": (C.c_int, [vp, u8p, i32]),
}

_lib = None


def load() -> C.CDLL:
    """Load libvcs.so from the package directory (raises if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libvcs.so is not built ({LIB_PATH}); run paper_2606_22447_b300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(status: int, handle=None):
    if status != VCS_OK:
        msg = load().vcs_last_error(handle)
        raise VcsError(status, msg.decode() if msg else "")
