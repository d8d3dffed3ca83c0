"""Digests of RAM and screens (parity at scale, where full outputs are too
large to compare): the GPU digest kernel against the oracle's digest of the
oracle's own outputs, on a small mixed batch for every env and on the
4096-env bench workload for a seeded sample of envs."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import gpu_rollout, make_batch, oracle_rollout, torch_cuda

pytestmark = pytest.mark.gpu


def _oracle_digests(rom, mapper, acts, frame_skip, screens=True):
    r, s, _ = oracle_rollout(rom, mapper, acts, frame_skip, screens=screens)
    return np.array([oracle.digest(r[t], s[t] if screens else None) for t in range(len(acts))], dtype=np.uint64)


def test_digest_matches_oracle_small_mixed_batch():
    torch = torch_cuda()
    mappers = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]
    roms = synth.config_carts(909, mappers)
    ec = synth.env_cart_round_robin(40, 3, sort=False)
    acts = synth.actions(909, 40, 6)
    b = make_batch(roms, mappers, ec)
    ram = torch.empty((6, 40, 128), dtype=torch.uint8, device="cuda")
    scr = torch.empty((6, 40, 210, 160), dtype=torch.uint8, device="cuda")
    b.rollout(torch.from_numpy(acts).cuda(), 2, ram, scr)
    d_full = b.digest(ram, scr).cpu().numpy().view(np.uint64)
    d_ram = b.digest(ram).cpu().numpy().view(np.uint64)
    b.sync()
    for e in range(40):
        c = int(ec[e])
        want = _oracle_digests(roms[c], mappers[c], acts[:, e], 2)
        assert np.array_equal(d_full[:, e], want), f"env {e}"
        want_ram = _oracle_digests(roms[c], mappers[c], acts[:, e], 2, screens=False)
        assert np.array_equal(d_ram[:, e], want_ram), f"env {e} (RAM only)"
    # a single changed pixel changes the digest
    scr[3, 7, 100, 80] ^= 1
    assert b.digest(ram, scr).cpu().numpy().view(np.uint64)[3, 7] != d_full[3, 7]


def test_digest_bench_workload_4096_envs_sampled():
    """The bench workload (4096 envs of one 4 KB cart, frame-skip 4) for 48
    steps: every env's digest on the GPU, checked against the oracle on a
    seeded sample of envs."""
    torch = torch_cuda()
    n, steps, chunk = 4096, 48, 8
    rom = synth.generate_cart(2, 0, synth.MAPPER_4K)
    acts = synth.actions(2, n, steps)
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n, np.int32))
    ram = torch.empty((chunk, n, 128), dtype=torch.uint8, device="cuda")
    scr = torch.empty((chunk, n, 210, 160), dtype=torch.uint8, device="cuda")
    dig = []
    for t0 in range(0, steps, chunk):
        b.rollout(torch.from_numpy(np.ascontiguousarray(acts[t0:t0 + chunk])).cuda(), 4, ram, scr)
        dig.append(b.digest(ram, scr).cpu().numpy().view(np.uint64).copy())
    b.sync()
    dig = np.concatenate(dig)
    assert len(np.unique(dig[-1])) > 1, "envs with different actions should differ"
    sample = np.random.default_rng(2).choice(n, 24, replace=False)
    with ThreadPoolExecutor(8) as ex:
        wants = list(ex.map(lambda e: _oracle_digests(rom, synth.MAPPER_4K, acts[:, e], 4), sample))
    for e, want in zip(sample, wants):
        assert np.array_equal(dig[:, e], want), f"env {e}"
