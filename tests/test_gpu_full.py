"""The fully relaxed forward (FULL mode, Section 4's temperature-limit study)
on the GPU against the oracle: per env the first divergence from the hard
machine, the cast counts of the paper's cast-margin model and the FULL
machine's final RAM, bit-exact (integers decided by float32 casts that both
sides compute in the same order), on synthetic carts of all three mappers
and on the crafted boundary carts."""
import numpy as np
import pytest

import oracle
from paper_2606_22447_b300 import synth
from tests.gpu_util import gpu_rollout, make_batch, torch_cuda

pytestmark = pytest.mark.gpu

MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]
BANKED = [synth.MAPPER_F6, synth.MAPPER_F4, synth.MAPPER_F8]
SUPERCHIP = [synth.MAPPER_F8SC, synth.MAPPER_F6SC, synth.MAPPER_F4SC]
E0 = [synth.MAPPER_E0, synth.MAPPER_4K, synth.MAPPER_E0]
FE = [synth.MAPPER_FE, synth.MAPPER_F8, synth.MAPPER_FE]


def _oracle_study(rom, mapper, warm, action, T, alpha, n):
    """(first divergence, [reads, exact reads, branches, exact branches] on
    the hard trajectory, FULL machine's RAM after n slots)."""
    def start(mode):
        o = oracle.Oracle(rom, mapper)
        if len(warm):
            o.rollout(warm, 1, screens=False)
        o.set_full(mode, T, alpha)
        return o
    h, f, p = start(0), start(2), start(1)
    n_div = 0
    for k in range(1, n + 1):
        h.trace(action, 1)
        f.trace(action, 1)
        if not n_div and not (np.array_equal(h.state(), f.state()) and np.array_equal(h.ram(), f.ram()) and
                              np.array_equal(h.cart_ram(), f.cart_ram())):
            n_div = k
    p.trace(action, n)
    c = p.counters()
    return n_div, [c["relaxed_reads"], c["relaxed_reads_exact"], c["branches"], c["branches_exact"]], f.ram()


@pytest.mark.parametrize("T,alpha,warm,mappers", [(0.14, 6.0, 0, MAPPERS), (0.15, 6.0, 0, MAPPERS),
                                                  (0.2, 6.0, 2, MAPPERS), (0.14, 2.0, 0, MAPPERS),
                                                  (0.14, 3.0, 2, MAPPERS), (0.01, 20.0, 0, MAPPERS),
                                                  (1.0, 6.0, 0, MAPPERS), (0.15, 6.0, 2, BANKED),
                                                  (0.14, 2.0, 0, BANKED), (0.15, 6.0, 2, SUPERCHIP),
                                                  (0.14, 6.0, 0, SUPERCHIP), (0.15, 6.0, 2, E0),
                                                  (0.14, 3.0, 0, E0), (0.15, 6.0, 2, FE), (0.14, 3.0, 0, FE)])
def test_full_divergence_matches_oracle(T, alpha, warm, mappers):
    torch = torch_cuda()
    MAPPERS = mappers
    n_envs, n = 9, 3000
    roms = synth.config_carts(95, MAPPERS)
    ec = (np.arange(n_envs) % 3).astype(np.int32)
    b = make_batch(roms, MAPPERS, ec, envs_per_block=8)
    wa = synth.actions(96, n_envs, warm)
    if warm:
        gpu_rollout(b, wa, 1, screens=False)
    acts = synth.actions(97, n_envs, 1)[0]
    n_div, cnt, ram = b.full_divergence(T, alpha, n, actions=torch.from_numpy(acts).cuda())
    b.sync()
    n_div, cnt, ram = n_div.cpu().numpy(), cnt.cpu().numpy().view(np.uint32), ram.cpu().numpy()
    for e in range(n_envs):
        c = ec[e]
        o_div, o_cnt, o_ram = _oracle_study(roms[c], MAPPERS[c], wa[:, e], int(acts[e]), T, alpha, n)
        assert n_div[e] == o_div, f"env {e}: first divergence {n_div[e]} vs oracle {o_div}"
        assert list(cnt[e]) == o_cnt, f"env {e}: cast counts {list(cnt[e])} vs oracle {o_cnt}"
        assert np.array_equal(ram[e], o_ram), f"env {e}: FULL machine RAM differs"
    if T <= 0.01:
        assert np.all(n_div == 0)
    if T >= 0.15 or alpha <= 2.0:
        assert np.any(n_div > 0), "this setting must diverge somewhere"


def test_full_boundaries_on_crafted_carts():
    torch = torch_cuda()
    from tests.microrom import FULL_T_LOOP, full_branch_rom, full_temperature_rom
    from tests.test_oracle_full import _t_star
    t_star = _t_star()
    rom = full_temperature_rom()
    b = make_batch([rom], [synth.MAPPER_4K], [0])
    n_nops = FULL_T_LOOP - 0xF000
    for T, want in ((t_star - 1e-3, 0), (t_star + 1e-3, n_nops + 1), (0.17, n_nops + 1)):
        n_div, _, ram = b.full_divergence(T, 6.0, n_nops + 30)
        b.sync()
        assert int(n_div.cpu()[0]) == want, T
        if want:
            assert int(ram.cpu()[0, 0]) == 1
    for offset, taken in ((-3, True), (40, False), (100, True)):
        a_star = float(np.log(2 * abs(offset) - 1))
        b = make_batch([full_branch_rom(offset, taken)], [synth.MAPPER_4K], [0])
        for alpha, want in ((a_star - 0.05, 0x102), (a_star + 0.05, 0)):
            n_div, _, _ = b.full_divergence(0.05, alpha, 0x102 + 5)
            b.sync()
            assert int(n_div.cpu()[0]) == want, (offset, alpha)
