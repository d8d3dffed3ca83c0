"""B300-native batched Atari VCS emulation (hard and SOFT-STE modes).

The emulation itself runs in libvcs.so (CUDA for sm_103a, C ABI declared in
include/vcs.h).  This package holds the thin Python binding over that ABI,
the PyTorch-facing wrappers (device memory and streams only) and the seeded
synthetic-input generator.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import ENV_DONE, ENV_JAMMED, ENV_WATCHDOG, Config, VcsError
from .synth import (MAPPER_2K, MAPPER_4K, MAPPER_E0, MAPPER_F4, MAPPER_F4SC, MAPPER_F6, MAPPER_F6SC, MAPPER_F8, MAPPER_FE,
                    MAPPER_F8SC, MAPPER_SIZE)

SCREEN_H, SCREEN_W, RAM_BYTES = 210, 160, 128

__all__ = ["Batch", "Tape", "Graph", "Config", "VcsError", "default_config", "autotune_cache_clear", "detect_mapper",
           "MAPPER_2K", "MAPPER_4K", "MAPPER_F8", "MAPPER_F6", "MAPPER_F4", "MAPPER_F8SC", "MAPPER_F6SC", "MAPPER_F4SC",
           "MAPPER_E0", "MAPPER_FE", "MAPPER_SIZE", "ENV_WATCHDOG", "ENV_JAMMED", "ENV_DONE"]


def default_config(**overrides) -> Config:
    cfg = Config()
    _lib.check(_lib.load().vcs_config_default(C.byref(cfg)))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def autotune_cache_clear():
    """Forget the process's cached autotuning results."""
    _lib.check(_lib.load().vcs_autotune_cache_clear(), None)


def int_peak(stream=None) -> float:
    """Measured integer operations per second of the current GPU."""
    v = C.c_double()
    _lib.check(_lib.load().vcs_int_peak(C.byref(v), _stream(stream)), None)
    return v.value


def _ptr(t):
    """Device address of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def detect_mapper(rom: bytes) -> int:
    """The cartridge format of an image (vcs_detect_mapper): one of the
    MAPPER_* codes, from its size and content."""
    buf = np.frombuffer(bytes(rom), dtype=np.uint8).copy()
    out = C.c_uint8()
    _lib.check(_lib.load().vcs_detect_mapper(buf.ctypes.data_as(_lib.u8p), len(buf), C.byref(out)), None)
    return int(out.value)


class Batch:
    """A batch of n_envs VCS machines over a list of cartridges.

    roms: list of bytes; mappers: list of MAPPER_* codes; env_cart: int array
    [n_envs] giving each env's cart.  Device buffers passed to the methods are
    torch CUDA tensors owned by the caller.
    """

    def __init__(self, roms, mappers, env_cart, config: Config | None = None):
        L = _lib.load()
        self.n_carts = len(roms)
        self._roms = [np.frombuffer(bytes(r), dtype=np.uint8).copy() for r in roms]
        ptrs = (_lib.u8p * self.n_carts)(*[r.ctypes.data_as(_lib.u8p) for r in self._roms])
        sizes = (C.c_uint32 * self.n_carts)(*[len(r) for r in self._roms])
        maps = np.ascontiguousarray(mappers, dtype=np.uint8)
        ec = np.ascontiguousarray(env_cart, dtype=np.int32)
        self.n_envs = int(ec.shape[0])
        self.mappers = [int(m) for m in maps]
        self.env_cart = ec.copy()
        h = C.c_void_p()
        cfg = config if config is not None else default_config()
        st = L.vcs_create_batch(ptrs, sizes, maps.ctypes.data_as(_lib.u8p), self.n_carts,
                                ec.ctypes.data_as(C.POINTER(C.c_int32)), self.n_envs, C.byref(cfg), C.byref(h))
        _lib.check(st, None)
        self.h = h
        self.config = cfg
        epb = C.c_int32()
        L.vcs_batch_info(self.h, None, None, C.byref(epb))
        self.envs_per_block = epb.value
        rs = C.c_int32()
        L.vcs_rom_stride(self.h, C.byref(rs))
        self.rom_stride = rs.value   # floats per cart row of the soft API's ROM tensors

    def close(self):
        if getattr(self, "h", None):
            _lib.load().vcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        _lib.check(st, self.h)

    def set_start_noops(self, counts):
        """NOOP frames starting each episode: uint8 [n_envs][n_per_env]."""
        c = np.ascontiguousarray(counts, dtype=np.uint8)
        n = 0 if c.size == 0 else int(c.shape[1])
        self._check(_lib.load().vcs_set_start_noops(self.h, c.ctypes.data_as(_lib.u8p), n))

    def reset(self, env_mask=None, stream=None):
        self._check(_lib.load().vcs_reset(self.h, _ptr(env_mask), _stream(stream)))

    def set_episodes(self, ep_len):
        ep = np.ascontiguousarray(ep_len, dtype=np.uint32)
        n_ep = 0 if ep.size == 0 else int(ep.shape[1])
        self._check(_lib.load().vcs_set_episodes(self.h, ep.ctypes.data_as(C.POINTER(C.c_uint32)), n_ep))

    def step(self, actions, frame_skip: int, ram_out=None, screen_out=None, status_out=None, stream=None):
        self._check(_lib.load().vcs_step(self.h, _ptr(actions), frame_skip, _ptr(ram_out), _ptr(screen_out),
                                         _ptr(status_out), _stream(stream)))

    def rollout(self, actions, frame_skip: int, ram_out=None, screen_out=None, status_out=None, stream=None):
        n_steps = int(actions.shape[0])
        self._check(_lib.load().vcs_rollout(self.h, _ptr(actions), n_steps, frame_skip, _ptr(ram_out),
                                            _ptr(screen_out), _ptr(status_out), _stream(stream)))

    def step_host(self, actions: np.ndarray, frame_skip: int, ram_out=None, screen_out=None, stream=None):
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        p = lambda x: None if x is None else C.c_void_p(x.ctypes.data)
        self._check(_lib.load().vcs_step_host(self.h, C.c_void_p(a.ctypes.data), frame_skip, p(ram_out),
                                              p(screen_out), _stream(stream)))

    def rollout_host(self, actions: np.ndarray, frame_skip: int, ram_out=None, screen_out=None, status_out=None,
                     stream=None):
        """Pipelined rollout through host (numpy) buffers: actions uint8
        [n_steps][n_envs]; outputs [n_steps][n_envs][...] filled on return."""
        a = np.ascontiguousarray(actions, dtype=np.uint8)
        p = lambda x: None if x is None else C.c_void_p(x.ctypes.data)
        for x in (ram_out, screen_out, status_out):
            if x is not None and not (x.flags["C_CONTIGUOUS"] and x.dtype == np.uint8):
                raise ValueError("host outputs must be C-contiguous uint8 arrays")
        self._check(_lib.load().vcs_rollout_host(self.h, C.c_void_p(a.ctypes.data), int(a.shape[0]), frame_skip,
                                                 p(ram_out), p(screen_out), p(status_out), _stream(stream)))

    def time_kernels(self, on: bool = True):
        """Record CUDA events around each step-launch's kernels (the step
        kernel and the raster kernel) from now on, or stop."""
        self._check(_lib.load().vcs_time_kernels(self.h, 1 if on else 0))

    def kernel_times(self) -> dict:
        """Summed milliseconds of the step and raster kernels since
        time_kernels(True), the launches timed and the raster log entries
        they drew."""
        s, r, n, k = C.c_float(), C.c_float(), C.c_int32(), C.c_double()
        self._check(_lib.load().vcs_kernel_times(self.h, C.byref(s), C.byref(r), C.byref(n), C.byref(k)))
        return {"step_ms": s.value, "raster_ms": r.value, "launches": n.value, "log_entries": k.value}

    def sync(self, stream=None):
        self._check(_lib.load().vcs_sync(self.h, _stream(stream)))

    def state_bytes(self) -> int:
        n = C.c_size_t()
        self._check(_lib.load().vcs_state_bytes(self.h, C.byref(n)))
        return n.value

    def save_state(self, stream=None) -> np.ndarray:
        blob = np.zeros(self.state_bytes(), np.uint8)
        self._check(_lib.load().vcs_save_state(self.h, C.c_void_p(blob.ctypes.data), _stream(stream)))
        return blob

    def soft_rollout(self, tau: float, u, frame_skip: int, rom_f32=None, ram0=None, ram_out=None,
                     screen_out=None, stream=None) -> "Tape":
        """SOFT-STE forward over u [n_steps][n_envs][5] (float CUDA tensor);
        returns the tape for backward().  Outputs are filled in place."""
        h = C.c_void_p()
        n_steps = int(u.shape[0])
        self._check(_lib.load().vcs_soft_rollout(self.h, float(tau), _ptr(rom_f32), _ptr(ram0), _ptr(u), n_steps,
                                                 frame_skip, _ptr(ram_out), _ptr(screen_out), C.byref(h),
                                                 _stream(stream)))
        return Tape(self, h, n_steps)

    def soft_step(self, tau: float, u, frame_skip: int, ram_out=None, screen_out=None, stream=None) -> "Tape":
        """vcs_soft_step: SOFT-STE forward over u [n_steps][n_envs][5] from
        the batch's own ROMs and current RAM; returns the tape."""
        h = C.c_void_p()
        n_steps = int(u.shape[0])
        self._check(_lib.load().vcs_soft_step(self.h, float(tau), _ptr(u), n_steps, frame_skip, _ptr(ram_out),
                                              _ptr(screen_out), C.byref(h), _stream(stream)))
        return Tape(self, h, n_steps)

    def autotune(self, frame_skip: int, n_steps: int, actions=None, ram_out=None, screen_out=None,
                 stream=None) -> dict:
        """Time launch geometries on the current state (restored after each
        trial) and keep the fastest; returns the choice."""
        t = _lib.Tune()
        self._check(_lib.load().vcs_autotune(self.h, frame_skip, n_steps, _ptr(actions), _ptr(ram_out),
                                             _ptr(screen_out), C.byref(t), _stream(stream)))
        self.envs_per_block = t.envs_per_block
        return {"envs_per_block": t.envs_per_block, "threads_per_env": t.threads_per_env,
                "sched_policy": t.sched_policy,
                "sched_window": t.sched_window, "steps_per_launch": t.steps_per_launch,
                "ms_per_step": t.ms_per_step, "n_trials": t.n_trials}

    def digest(self, ram, screen=None, out=None, stream=None):
        """uint64 digests [n_steps][n_envs] of rollout outputs (device
        tensors laid out as rollout() writes them); returns a torch int64
        tensor holding the 64-bit patterns."""
        import torch
        n_steps = int(ram.shape[0])
        if out is None:
            out = torch.empty((n_steps, self.n_envs), dtype=torch.int64, device=ram.device)
        self._check(_lib.load().vcs_digest(self.h, _ptr(ram), _ptr(screen), n_steps, _ptr(out), _stream(stream)))
        return out

    def cart_ram(self, out=None, stream=None):
        """The Superchip RAM of every env (vcs_cart_ram): a torch uint8 CUDA
        tensor [n_envs][128], zero for envs of other carts."""
        import torch
        if out is None:
            out = torch.empty((self.n_envs, 128), dtype=torch.uint8, device="cuda")
        self._check(_lib.load().vcs_cart_ram(self.h, _ptr(out), _stream(stream)))
        return out

    def full_divergence(self, T: float, alpha: float, n_instr: int, actions=None, counts=True, ram=True,
                        stream=None):
        """The fully relaxed forward study (vcs_full_divergence): returns
        (n_div int32 [n_envs], counts uint32 [n_envs][4] or None, the FULL
        machine's RAM uint8 [n_envs][128] or None) as torch CUDA tensors."""
        import torch
        n_div = torch.empty(self.n_envs, dtype=torch.int32, device="cuda")
        cnt = torch.empty((self.n_envs, 4), dtype=torch.int32, device="cuda") if counts else None
        rf = torch.empty((self.n_envs, 128), dtype=torch.uint8, device="cuda") if ram else None
        self._check(_lib.load().vcs_full_divergence(self.h, float(T), float(alpha), _ptr(actions), int(n_instr),
                                                    _ptr(n_div), _ptr(cnt), _ptr(rf), _stream(stream)))
        return n_div, cnt, rf

    def graph(self, actions, frame_skip: int, ram_out=None, screen_out=None, status_out=None) -> "Graph":
        """Capture one rollout over these fixed buffers as a CUDA graph."""
        h = C.c_void_p()
        n_steps = int(actions.shape[0])
        self._check(_lib.load().vcs_graph_create(self.h, _ptr(actions), n_steps, frame_skip, _ptr(ram_out),
                                                 _ptr(screen_out), _ptr(status_out), C.byref(h)))
        return Graph(self, h, (actions, ram_out, screen_out, status_out))

    def load_state(self, blob: np.ndarray, stream=None):
        b = np.ascontiguousarray(blob, dtype=np.uint8)
        if b.size != self.state_bytes():
            raise ValueError("state blob size mismatch")
        self._check(_lib.load().vcs_load_state(self.h, C.c_void_p(b.ctypes.data), _stream(stream)))


class Tape:
    """Checkpoints of one soft rollout; backward() may be called repeatedly."""

    def __init__(self, batch: Batch, handle, n_steps: int):
        self.batch = batch
        self.h = handle
        self.n_steps = n_steps

    def backward(self, grad_ram=None, grad_screen=None, w_ram=None, w_screen=None, grad_rom=None,
                 grad_ram0=None, grad_u=None, grad_rom_per_cart=None, grad_cart_ram0=None, stream=None):
        w = None
        if w_ram is not None or w_screen is not None:
            w = _lib.LossWeights(_ptr(w_ram), _ptr(w_screen))
        st = _lib.load().vcs_backward(self.h, _ptr(grad_ram), _ptr(grad_screen), C.byref(w) if w else None,
                                      _ptr(grad_rom), _ptr(grad_ram0), _ptr(grad_cart_ram0), _ptr(grad_u),
                                      _ptr(grad_rom_per_cart), _stream(stream))
        _lib.check(st, self.batch.h)

    def free(self):
        if getattr(self, "h", None):
            _lib.load().vcs_tape_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Graph:
    """A captured rollout; launch() replays it on the buffers given at capture."""

    def __init__(self, batch: Batch, handle, buffers):
        self.batch = batch
        self.h = handle
        self._buffers = buffers   # keep the captured tensors alive

    def launch(self, stream=None):
        _lib.check(_lib.load().vcs_graph_launch(self.h, _stream(stream)), self.batch.h)

    def destroy(self):
        if getattr(self, "h", None):
            _lib.load().vcs_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
