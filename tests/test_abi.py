"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/vcs.h, and rejects bad arguments before touching the
device (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2606_22447_b300 import _lib, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vcs_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "vcs_create_batch" in names and "vcs_step" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # the binding covers every declared entry point
    assert names <= set(_lib.SIGNATURES), names - set(_lib.SIGNATURES)


def test_config_defaults(lib):
    cfg = _lib.Config()
    assert lib.vcs_config_default(C.byref(cfg)) == 0
    assert cfg.alpha == 6.0 and cfg.ystart == 34 and cfg.boot_noop_frames == 0
    assert cfg.segment_frames == 64
    assert cfg.full_tia == 0 and cfg.position_sampler == 0 and cfg.step_instructions == 0
    assert cfg.inline_render == 0   # deferred rasterisation
    assert cfg.sweep_mode == 0      # the sweep chosen by batch size


def test_binding_config_matches_header():
    """The ctypes Config lists the header's vcs_config fields in order."""
    src = open(os.path.join(ROOT, "include", "vcs.h")).read()
    body = re.search(r"typedef struct vcs_config \{(.*?)\} vcs_config;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:float|int32_t)\s+(\w+)\s*;", body)
    assert fields == [f for f, _ in _lib.Config._fields_]


def _create(lib, roms, sizes, mappers, env_cart, n_carts=None, cfg=None):
    n_carts = len(roms) if n_carts is None else n_carts
    keep = [np.frombuffer(r, np.uint8).copy() if r is not None else None for r in roms]
    ptrs = (_lib.u8p * max(1, len(roms)))(*[k.ctypes.data_as(_lib.u8p) if k is not None else None for k in keep])
    sz = (C.c_uint32 * max(1, len(sizes)))(*sizes)
    mp = np.array(mappers, np.uint8)
    ec = np.array(env_cart, np.int32)
    h = C.c_void_p()
    st = lib.vcs_create_batch(ptrs, sz, mp.ctypes.data_as(_lib.u8p), n_carts,
                              ec.ctypes.data_as(C.POINTER(C.c_int32)), len(env_cart), cfg, C.byref(h))
    return st, h, lib.vcs_last_error(None).decode()


def test_argument_errors_before_device_work(lib):
    rom4 = synth.generate_cart(1, 0, synth.MAPPER_4K)
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_4K], [0, 1])
    assert st == _lib.VCS_ERR_ARG and "out of range" in msg and not h.value
    st, h, msg = _create(lib, [rom4], [4096], [200], [0])
    assert st == _lib.VCS_ERR_MAPPER and not h.value
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_2K], [0])
    assert st == _lib.VCS_ERR_ROM_SIZE and "want 2048" in msg
    st, h, msg = _create(lib, [None], [4096], [synth.MAPPER_4K], [0])
    assert st == _lib.VCS_ERR_ARG
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_4K], [])
    assert st == _lib.VCS_ERR_ARG
    cfg = _lib.Config()
    lib.vcs_config_default(C.byref(cfg))
    cfg.envs_per_block = 48
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_4K], [0], cfg=C.byref(cfg))
    assert st == _lib.VCS_ERR_ARG and "envs_per_block" in msg
    lib.vcs_config_default(C.byref(cfg))
    cfg.inline_render = 2
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_4K], [0], cfg=C.byref(cfg))
    assert st == _lib.VCS_ERR_ARG and "inline_render" in msg
    lib.vcs_config_default(C.byref(cfg))
    cfg.sweep_mode = 3
    st, h, msg = _create(lib, [rom4], [4096], [synth.MAPPER_4K], [0], cfg=C.byref(cfg))
    assert st == _lib.VCS_ERR_ARG and "sweep_mode" in msg
    assert lib.vcs_step(None, None, 1, None, None, None, None) == _lib.VCS_ERR_ARG
    tape = C.c_void_p()
    assert lib.vcs_soft_step(None, 0.1, None, 1, 1, None, None, C.byref(tape), None) == _lib.VCS_ERR_ARG
    assert lib.vcs_destroy(None) == _lib.VCS_ERR_ARG
    assert lib.vcs_time_kernels(None, 1) == _lib.VCS_ERR_ARG
    f, i, d = C.c_float(), C.c_int32(), C.c_double()
    assert lib.vcs_kernel_times(None, C.byref(f), C.byref(f), C.byref(i), C.byref(d)) == _lib.VCS_ERR_ARG


def test_detect_mapper(lib):
    """Content-based detection (host only): every generated format is
    recognised from its image; an 8 KB image with E0-hotspot accesses is E0
    unless it also touches the F8 hotspots; one without either and with a
    JSR into $D000-$DFFF is FE; Superchip filler in every bank picks the SC
    variant; other sizes are refused."""
    from paper_2606_22447_b300 import detect_mapper
    all_mappers = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8, synth.MAPPER_F6, synth.MAPPER_F4,
                   synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC, synth.MAPPER_E0, synth.MAPPER_FE]
    for seed in (31, 32):
        for m, rom in zip(all_mappers, synth.config_carts(seed, all_mappers)):
            assert detect_mapper(rom) == m, (seed, m)
    f8 = bytearray(synth.generate_cart(33, 0, synth.MAPPER_F8))
    f8[0x200:0x203] = bytes((0xAD, 0xE5, 0xFF))       # LDA $FFE5: an E0 hotspot mirror, in a cart
    assert detect_mapper(bytes(f8)) == synth.MAPPER_F8  # that also switches through $1FF8-9
    e0 = bytearray(synth.generate_cart(33, 0, synth.MAPPER_E0))
    e0[0x300:0x303] = bytes((0x2C, 0xF9, 0x1F))       # BIT $1FF9: an F8 hotspot
    assert detect_mapper(bytes(e0)) == synth.MAPPER_F8
    blank = bytearray(range(256)) * 32                  # no hotspot access, no Superchip filler
    assert detect_mapper(bytes(blank)) == synth.MAPPER_F8
    fe = bytearray(blank)
    fe[0x100:0x103] = bytes((0x20, 0x00, 0xD4))        # JSR $D400: a call into FE's second bank
    assert detect_mapper(bytes(fe)) == synth.MAPPER_FE
    fe[0x300:0x303] = bytes((0x2C, 0xF8, 0x1F))        # BIT $1FF8: an F8 hotspot
    assert detect_mapper(bytes(fe)) == synth.MAPPER_F8
    blank[0x1000:0x1003] = bytes((0x8D, 0xF3, 0x3F))  # STA $3FF3 -> $1FF3
    assert detect_mapper(bytes(blank)) == synth.MAPPER_E0
    sc = bytearray(synth.generate_cart(34, 0, synth.MAPPER_F6))
    for b in range(0, len(sc), 4096):
        sc[b:b + 256] = bytes(range(128)) * 2
    assert detect_mapper(bytes(sc)) == synth.MAPPER_F6SC
    sc[4096 + 200] ^= 1                                 # one bank without the repeat
    assert detect_mapper(bytes(sc)) == synth.MAPPER_F6
    out = C.c_uint8()
    buf = np.zeros(3000, np.uint8)
    assert lib.vcs_detect_mapper(buf.ctypes.data_as(_lib.u8p), 3000, C.byref(out)) == _lib.VCS_ERR_ROM_SIZE
    assert lib.vcs_detect_mapper(None, 4096, C.byref(out)) == _lib.VCS_ERR_ARG
