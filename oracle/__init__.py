"""Python access to the CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain C emulator (vcs_oracle.c) built into liboracle.so.
Only tests/, the package smoke check and the benchmark's CPU-baseline leg
use it; the product path never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vcs_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

SCREEN = 210 * 160


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (idempotent)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "vcs_oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Counters(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "instructions", "cycles", "frames", "tia_writes", "ram_reads", "ram_writes",
        "rom_reads", "pixels", "watchdog", "relaxed_reads", "relaxed_reads_exact", "branches",
        "branches_exact")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, u8p, u32p, dp = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint32), C.POINTER(C.c_double)
        L.ovcs_new.restype = vp
        L.ovcs_new.argtypes = [u8p, C.c_uint32, C.c_int, C.c_int]
        L.ovcs_free.argtypes = [vp]
        L.ovcs_reset.argtypes = [vp]
        L.ovcs_step.restype = C.c_int
        L.ovcs_step.argtypes = [vp, C.c_int, C.c_int, u8p, u8p]
        L.ovcs_get_counters.argtypes = [vp, C.POINTER(Counters)]
        L.ovcs_get_state.argtypes = [vp, u32p]
        L.ovcs_get_ram.argtypes = [vp, u8p]
        L.ovcs_get_cart_ram.argtypes = [vp, u8p]
        L.ovcs_trace.restype = C.c_int
        L.ovcs_trace.argtypes = [vp, C.c_int, C.c_int, u32p]
        L.ovcs_set_regs.argtypes = [vp] + [C.c_int] * 6
        L.ovcs_set_ram.argtypes = [vp, u8p]
        L.ovcs_exec_one.restype = C.c_int
        L.ovcs_exec_one.argtypes = [vp]
        L.ovcs_peek.restype = C.c_uint8
        L.ovcs_peek.argtypes = [vp, C.c_uint16]
        L.ovcs_bank.restype = C.c_int
        L.ovcs_bank.argtypes = [vp]
        L.ovcs_soft_rollout.restype = vp
        L.ovcs_soft_rollout.argtypes = [vp, dp, C.c_int, C.c_int, C.c_double, C.c_double,
                                        dp, dp, dp, dp]
        L.ogrf_free.argtypes = [vp]
        L.ogrf_reverse.argtypes = [vp, dp, dp, dp]
        L.ogrf_tangent.restype = C.c_double
        L.ogrf_tangent.argtypes = [vp, dp, dp, dp]
        L.ogrf_eval.restype = C.c_double
        L.ogrf_eval.argtypes = [vp, dp, dp, dp]
        L.ogrf_nodes.restype = C.c_int64
        L.ogrf_nodes.argtypes = [vp]
        L.ovcs_set_switches.argtypes = [vp, C.c_uint8]
        L.ovcs_set_sampler.argtypes = [vp, C.c_int]
        L.ovcs_set_graphics.argtypes = [vp, C.c_int]
        L.ovcs_set_full_tia.argtypes = [vp, C.c_int]
        L.ovcs_set_step_instructions.argtypes = [vp, C.c_int]
        L.ovcs_set_full.argtypes = [vp, C.c_int, C.c_double, C.c_double]
        L.ovcs_digest.restype = C.c_uint64
        L.ovcs_digest.argtypes = [u8p, u8p]
        L.ovcs_relaxed_read.restype = C.c_double
        L.ovcs_relaxed_read.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, dp]
        L.ovcs_gate_slope.restype = C.c_double
        L.ovcs_gate_slope.argtypes = [C.c_double, C.c_double]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def _dp(a):
    return _p(a, C.c_double)


class SoftGraph:
    """FP64 deviation graph of one soft rollout (frozen switches)."""

    def __init__(self, handle, rom_size: int, n_steps: int):
        self.h = handle
        self.rom_size = rom_size
        self.n_steps = n_steps

    def __del__(self):
        if getattr(self, "h", None):
            lib().ogrf_free(self.h)
            self.h = None

    @property
    def n_nodes(self) -> int:
        return lib().ogrf_nodes(self.h)

    def reverse(self, cart_ram: bool = False):
        """(grad ROM, grad initial RAM [128], grad inputs [n_steps][5]), and
        with cart_ram the gradient of the initial Superchip RAM [128] too."""
        g_rom = np.zeros(self.rom_size)
        g_ram0 = np.zeros(256)
        g_u = np.zeros((self.n_steps, 5))
        lib().ogrf_reverse(self.h, _dp(g_rom), _dp(g_ram0), _dp(g_u))
        if cart_ram:
            return g_rom, g_ram0[:128], g_u, g_ram0[128:]
        return g_rom, g_ram0[:128], g_u

    def _args(self, d_rom, d_ram0, d_u):
        """d_ram0: 128 RIOT cells, or 256 (then the Superchip's RAM)."""
        f = lambda a, n: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(n)
        if d_ram0 is not None:
            d = np.zeros(256)
            r = np.asarray(d_ram0, dtype=np.float64).reshape(-1)
            d[:len(r)] = r
            d_ram0 = d
        return (f(d_rom, self.rom_size), f(d_ram0, 256), f(d_u, self.n_steps * 5))

    def tangent(self, d_rom=None, d_ram0=None, d_u=None) -> float:
        a = self._args(d_rom, d_ram0, d_u)
        return lib().ogrf_tangent(self.h, *[_dp(x) for x in a])

    def eval(self, d_rom=None, d_ram0=None, d_u=None) -> float:
        a = self._args(d_rom, d_ram0, d_u)
        return lib().ogrf_eval(self.h, *[_dp(x) for x in a])


class Oracle:
    """One emulated VCS (hard mode, optional soft rollouts)."""

    def __init__(self, rom: bytes, mapper: int, ystart: int = 34, full_tia: bool = False):
        self.rom = np.frombuffer(bytes(rom), dtype=np.uint8).copy()
        self.mapper = mapper
        self.h = lib().ovcs_new(_p(self.rom, C.c_uint8), len(self.rom), mapper, ystart)
        if not self.h:
            raise ValueError("bad ROM size for mapper")
        lib().ovcs_set_full_tia(self.h, 1 if full_tia else 0)

    def __del__(self):
        if getattr(self, "h", None):
            lib().ovcs_free(self.h)
            self.h = None

    def reset(self):
        lib().ovcs_reset(self.h)

    def boot(self, noop_frames: int, reset_frames: int, extra_noops: int = 0):
        """The paper's boot protocol after a power-on (supplement, settings
        table): NOOP frames, frames with the console RESET switch held, then
        the episode's extra NOOP frames."""
        for _ in range(noop_frames):
            self.step(0, 1)
        lib().ovcs_set_switches(self.h, 0x0A)
        for _ in range(reset_frames):
            self.step(0, 1)
        lib().ovcs_set_switches(self.h, 0x0B)
        for _ in range(extra_noops):
            self.step(0, 1)

    def set_sampler(self, on: bool):
        """Switch the differentiable position sampler (Section 3) on or off for
        the soft rollouts that follow."""
        lib().ovcs_set_sampler(self.h, 1 if on else 0)

    def set_graphics(self, on: bool):
        """Switch the graphics-bit surrogate (Section 3.1's stored-switch
        paragraph) on or off for the soft rollouts that follow."""
        lib().ovcs_set_graphics(self.h, 1 if on else 0)

    def set_step_instructions(self, n: int):
        """Make every following step run n instruction slots (n > 0) instead
        of frame_skip frames (n = 0)."""
        lib().ovcs_set_step_instructions(self.h, int(n))

    def set_full(self, mode: int, T: float = 0.0, alpha: float = 6.0):
        """Fully relaxed casts: 2 = FULL (executed), 1 = probe (counted
        only), 0 = off."""
        lib().ovcs_set_full(self.h, int(mode), float(T), float(alpha))

    def step(self, action: int, frame_skip: int = 1):
        ram = np.zeros(128, np.uint8)
        scr = np.zeros((210, 160), np.uint8)
        st = lib().ovcs_step(self.h, int(action), frame_skip, _p(ram, C.c_uint8), _p(scr, C.c_uint8))
        return ram, scr, st

    def rollout(self, acts, frame_skip: int = 1, screens: bool = True):
        n = len(acts)
        rams = np.zeros((n, 128), np.uint8)
        scrs = np.zeros((n, 210, 160), np.uint8) if screens else None
        status = np.zeros(n, np.int32)
        for t, a in enumerate(acts):
            r, s, st = self.step(int(a), frame_skip)
            rams[t] = r
            if screens:
                scrs[t] = s
            status[t] = st
        return rams, scrs, status

    def counters(self) -> dict:
        c = Counters()
        lib().ovcs_get_counters(self.h, C.byref(c))
        return {n: getattr(c, n) for n, _ in Counters._fields_}

    def state(self) -> np.ndarray:
        o = np.zeros(64, np.uint32)
        lib().ovcs_get_state(self.h, _p(o, C.c_uint32))
        return o

    def ram(self) -> np.ndarray:
        o = np.zeros(128, np.uint8)
        lib().ovcs_get_ram(self.h, _p(o, C.c_uint8))
        return o

    def cart_ram(self) -> np.ndarray:
        """The Superchip's 128 bytes of cartridge RAM (zero for other carts)."""
        o = np.zeros(128, np.uint8)
        lib().ovcs_get_cart_ram(self.h, _p(o, C.c_uint8))
        return o

    def trace(self, action: int, n: int) -> np.ndarray:
        o = np.zeros((n, 10), np.uint32)
        lib().ovcs_trace(self.h, int(action), n, _p(o, C.c_uint32))
        return o

    def set_regs(self, A=0, X=0, Y=0, SP=0xFF, P=0x30, PC=0xF000):
        lib().ovcs_set_regs(self.h, A, X, Y, SP, P, PC)

    def set_ram(self, ram):
        r = np.ascontiguousarray(ram, dtype=np.uint8)
        lib().ovcs_set_ram(self.h, _p(r, C.c_uint8))

    def exec_one(self) -> int:
        return lib().ovcs_exec_one(self.h)

    def peek(self, addr: int) -> int:
        return lib().ovcs_peek(self.h, addr)

    def bank(self) -> int:
        return lib().ovcs_bank(self.h)

    def soft_rollout(self, u, frame_skip: int, tau: float, alpha: float = 6.0,
                     grad_ram=None, grad_screen=None, outputs: bool = True):
        u = np.ascontiguousarray(u, dtype=np.float64)
        n = u.shape[0]
        gr = None if grad_ram is None else np.ascontiguousarray(grad_ram, dtype=np.float64)
        gs = None if grad_screen is None else np.ascontiguousarray(grad_screen, dtype=np.float64)
        ram_out = np.zeros((n, 128)) if outputs else None
        scr_out = np.zeros((n, 210, 160)) if outputs else None
        h = lib().ovcs_soft_rollout(self.h, _dp(u), n, frame_skip, float(tau), float(alpha),
                                    _dp(gr), _dp(gs), _dp(ram_out), _dp(scr_out))
        return SoftGraph(h, len(self.rom), n), ram_out, scr_out


def digest(ram, screen=None) -> int:
    """64-bit digest of one env-step's RAM [128] and screen [210][160]
    (uint8 arrays; screen optional), as defined in vcs_oracle.h."""
    r = np.ascontiguousarray(ram, dtype=np.uint8)
    if screen is None:
        return int(lib().ovcs_digest(_p(r, C.c_uint8), None))
    sc = np.ascontiguousarray(screen, dtype=np.uint8)
    return int(lib().ovcs_digest(_p(r, C.c_uint8), _p(sc, C.c_uint8)))


def relaxed_read(r, a0: int, a: float, tau: float):
    r = np.ascontiguousarray(r, dtype=np.float64)
    d = C.c_double()
    v = lib().ovcs_relaxed_read(_dp(r), len(r), int(a0), float(a), float(tau), C.byref(d))
    return v, d.value


def gate_slope(alpha: float, z: float) -> float:
    return lib().ovcs_gate_slope(float(alpha), float(z))
