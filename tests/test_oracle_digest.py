"""The oracle's output digest against its definition (sum mod 2^64 of the
splitmix64 finaliser of (word index << 32) | word over the little-endian
32-bit words of RAM then screen), evaluated here with numpy, plus the
properties a parity digest needs (position sensitivity, RAM-only form)."""
import numpy as np

import oracle

M1, M2 = np.uint64(0xBF58476D1CE4E5B9), np.uint64(0x94D049BB133111EB)


def _fin(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def _digest_np(ram, screen=None):
    b = ram if screen is None else np.concatenate([ram, screen.ravel()])
    w = b.view("<u4").astype(np.uint64)
    i = np.arange(len(w), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(_fin((i << np.uint64(32)) | w), dtype=np.uint64))


def test_digest_definition_random_outputs():
    rng = np.random.default_rng(7)
    for _ in range(5):
        ram = rng.integers(0, 256, 128, dtype=np.uint8)
        scr = rng.integers(0, 256, (210, 160), dtype=np.uint8)
        assert oracle.digest(ram, scr) == _digest_np(ram, scr)
        assert oracle.digest(ram) == _digest_np(ram)


def test_digest_finaliser_known_value_and_sensitivity():
    # splitmix64's first output for seed 0 is the finaliser of 0x9E3779B97F4A7C15
    assert int(_fin(np.uint64(0x9E3779B97F4A7C15))) == 0xE220A8397B1DCDAF
    ram = np.zeros(128, np.uint8)
    scr = np.zeros((210, 160), np.uint8)
    d0 = oracle.digest(ram, scr)
    scr[0, 0] = 1
    d1 = oracle.digest(ram, scr)
    scr[0, 0], scr[0, 4] = 0, 1   # the same byte value in another word
    d2 = oracle.digest(ram, scr)
    assert len({d0, d1, d2}) == 3
