"""Writes bench_counts.json: emulated instructions of the bench workloads,
counted by the oracle (the algorithmic work the roofline divides, and the
paper's throughput unit).  Calls only the oracle and the input generator.

    python tests/golden/make_bench_counts.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2606_22447_b300 import synth  # noqa: E402

SEED = 2            # the bench's seed
FRAME_SKIP = 4


def hard_instructions_per_env_step(steps=8):
    """The hard bench cart (seed 2, cart 0, 4 KB): one env's actions of the
    seeded stream, the oracle's instruction count per env-step."""
    rom = synth.generate_cart(SEED, 0, synth.MAPPER_4K)
    o = oracle.Oracle(rom, synth.MAPPER_4K)
    acts = synth.actions(SEED, 1, steps)
    for t in range(steps):
        o.step(int(acts[t, 0]), FRAME_SKIP)
    return o.counters()["instructions"] / steps


def instructions_per_frame(mappers, n_envs, frames=64):
    """A soft leg's cart mix: the oracle's count over the first `frames`
    frames of each cart with NOOP input, weighted by envs per cart."""
    roms = synth.config_carts(SEED, mappers)
    ec = synth.env_cart_round_robin(n_envs, len(mappers))
    per_cart = []
    for rom, mapper in zip(roms, mappers):
        o = oracle.Oracle(rom, mapper)
        for _ in range(frames):
            o.step(0, 1)
        per_cart.append(o.counters()["instructions"] / frames)
    w = np.bincount(ec, minlength=len(roms))
    return float(np.dot(per_cart, w) / w.sum())


def counts():
    return {
        "hard_4096x4k_instructions_per_env_step": hard_instructions_per_env_step(),
        "soft_short_1024x4k_instructions_per_frame": instructions_per_frame([synth.MAPPER_4K], 1024),
        "soft_long_4096xmix8_instructions_per_frame": instructions_per_frame(synth.MIX8, 4096),
        "recipe": "oracle counters; hard: 8 env-steps of env 0's seeded actions, frame-skip 4, "
                  "seed-2 4 KB cart; soft: first 64 frames of each cart with NOOP input, "
                  "weighted by envs per cart",
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "bench_counts.json"), "w") as f:
        json.dump(counts(), f, indent=1)
        f.write("\n")
    print(open(os.path.join(HERE, "bench_counts.json")).read())
