"""Launch geometry, autotuning and CUDA graphs change no result: outputs stay
bit-identical to one plain launch (and to the oracle), and the autotuner
leaves the batch in the state it found it."""
import numpy as np
import pytest

from paper_2606_22447_b300 import VcsError, autotune_cache_clear, synth
from paper_2606_22447_b300._lib import VCS_ERR_STATE
from tests.gpu_util import assert_env_equal, gpu_rollout, make_batch, oracle_rollout, torch_cuda

pytestmark = pytest.mark.gpu

MAPPERS = [synth.MAPPER_2K, synth.MAPPER_4K, synth.MAPPER_F8]


def _setup(n_envs, seed=808):
    roms = synth.config_carts(seed, MAPPERS)
    env_cart = synth.env_cart_round_robin(n_envs, len(MAPPERS), sort=False)
    return roms, env_cart


def test_autotune_keeps_state_and_results():
    torch = torch_cuda()
    roms, ec = _setup(45)
    acts = synth.actions(808, 45, 6)
    ref = make_batch(roms, MAPPERS, ec)
    ram1, scr1, st1 = gpu_rollout(ref, acts, 2)
    b = make_batch(roms, MAPPERS, ec)
    autotune_cache_clear()
    before = b.save_state()
    tune_acts = torch.from_numpy(np.ascontiguousarray(synth.actions(809, 45, 3))).cuda()
    choice = b.autotune(2, 3, actions=tune_acts)
    assert np.array_equal(b.save_state(), before), "autotune must restore the state"
    assert choice["envs_per_block"] in (8, 16, 32, 64, 128) and choice["n_trials"] >= 3
    assert choice["sched_policy"] in (0, 1) and choice["steps_per_launch"] in (0, 1, 4)
    ram2, scr2, st2 = gpu_rollout(b, acts, 2)
    assert np.array_equal(ram1, ram2) and np.array_equal(scr1, scr2) and np.array_equal(st1, st2)
    for e in (0, 1, 2, 44):
        c = int(ec[e])
        r, s, _ = oracle_rollout(roms[c], MAPPERS[c], acts[:, e], 2)
        assert_env_equal(e, ram2[:, e], r, "RAM")
        assert_env_equal(e, scr2[:, e], s, "screen")


@pytest.mark.parametrize("k", [1, 2, 4])
def test_steps_per_launch_split_equals_one_launch(k):
    roms, ec = _setup(21)
    acts = synth.actions(810, 21, 7)
    ep = synth.episode_lengths(810, 21, 4, mean_frames=6.0)
    outs = []
    for spl in (0, k):
        b = make_batch(roms, MAPPERS, ec, steps_per_launch=spl)
        b.set_episodes(ep)
        outs.append(gpu_rollout(b, acts, 2))
    for x, y in zip(outs[0], outs[1]):
        assert np.array_equal(x, y)
    assert np.any(outs[0][2] & 4), "the episode table should end some episodes inside the rollout"


def test_graph_replay_equals_rollout():
    torch = torch_cuda()
    roms, ec = _setup(30)
    n, steps = 30, 3
    rounds = [synth.actions(811 + i, n, steps) for i in range(3)]
    ref = make_batch(roms, MAPPERS, ec)
    want = [gpu_rollout(ref, a, 2) for a in rounds]

    b = make_batch(roms, MAPPERS, ec, steps_per_launch=2)
    a_buf = torch.zeros((steps, n), dtype=torch.uint8, device="cuda")
    ram = torch.zeros((steps, n, 128), dtype=torch.uint8, device="cuda")
    scr = torch.zeros((steps, n, 210, 160), dtype=torch.uint8, device="cuda")
    st = torch.zeros((steps, n), dtype=torch.uint8, device="cuda")
    g = b.graph(a_buf, 2, ram, scr, st)
    for a, (r1, s1, t1) in zip(rounds, want):
        a_buf.copy_(torch.from_numpy(np.ascontiguousarray(a)))
        g.launch()
        b.sync()
        assert np.array_equal(ram.cpu().numpy(), r1)
        assert np.array_equal(scr.cpu().numpy(), s1)
        assert np.array_equal(st.cpu().numpy(), t1)
    # a new geometry invalidates the graph: refused on the host, nothing launched
    autotune_cache_clear()   # the trials rebuild the block table
    b.autotune(2, 1)
    with pytest.raises(VcsError) as ei:
        g.launch()
    assert ei.value.status == VCS_ERR_STATE
    g.destroy()


def test_autotune_cache_per_shape():
    roms, ec = _setup(37)
    autotune_cache_clear()
    first = make_batch(roms, MAPPERS, ec).autotune(1, 1)
    assert first["n_trials"] > 0
    b = make_batch(roms, MAPPERS, ec)
    again = b.autotune(1, 1)
    assert again["n_trials"] == 0
    assert {k: again[k] for k in again if k not in ("n_trials",)} == {k: first[k] for k in first if k != "n_trials"}
    assert b.envs_per_block == first["envs_per_block"]
    other = make_batch(roms, MAPPERS, ec).autotune(3, 1)   # another frame-skip is another key
    assert other["n_trials"] > 0
    autotune_cache_clear()
    assert make_batch(roms, MAPPERS, ec).autotune(1, 1)["n_trials"] > 0


def test_int_peak_is_a_plausible_rate():
    """The roofline denominator: measured integer operations per second, within
    a factor of two of the SM count x 128 lanes x the clock."""
    import torch
    from paper_2606_22447_b300 import int_peak
    v = int_peak()
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2.032e9
    assert 0.5 * derived < v < 2.0 * derived
