"""vcs_backward_static: the backward pass for callers that cannot let a
library allocate device memory (an application whose GPU memory belongs to
an allocator it does not control, or one held to a fixed device-memory
budget).  It must give the same gradients as vcs_backward, on two calls in a
row (the fixed scratch array keeps the previous call's contents), and reject
problems whose scratch does not fit the array with a clear error.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_22447_b300 import _lib, synth
from tests.gpu_util import gpu_rollout, make_batch, torch_cuda

pytestmark = pytest.mark.gpu


def _outputs(n_envs, n_steps, n_carts):
    torch = torch_cuda()
    return [torch.full((n_envs, 8192), 7.0, device="cuda"), torch.full((n_envs, 128), 7.0, device="cuda"),
            torch.full((n_envs, 128), 7.0, device="cuda"), torch.full((n_steps, n_envs, 5), 7.0, device="cuda"),
            torch.full((n_carts, 8192), 7.0, device="cuda")]


def _grads(entry, tape, gr, gs, out):
    """Run one backward entry point into the preallocated outputs; returns
    (the gradients, the device's free bytes before and after the call,
    both read with the GPU idle)."""
    torch = torch_cuda()
    p = lambda t: C.c_void_p(t.data_ptr())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = getattr(_lib.load(), entry)(tape.h, p(gr), p(gs), None, *[p(t) for t in out],
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, tape.batch.h)
    tape.batch.sync()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    return [t.cpu().numpy() for t in out], free0, free1


@pytest.mark.parametrize("full_tia", [0, 1])
def test_static_backward_matches_backward_on_two_calls(full_tia):
    """Plain, Superchip and E0 carts; with the whole TIA the carry also holds
    COLUP1's adjoint.  Both entry points run the same kernels on the same
    tape here (12 envs: one recompute geometry), so the gradients agree bit
    for bit; the second static call must not change the device's free
    memory (it allocates nothing; the first may load the library's module
    on this device)."""
    torch = torch_cuda()
    mappers = [synth.MAPPER_2K, synth.MAPPER_E0, synth.MAPPER_F8SC]
    n_envs, n_steps = 12, 5
    roms = synth.config_carts(71, mappers, full_tia=bool(full_tia))
    env_cart = (np.arange(n_envs) % 3).astype(np.int32)
    b = make_batch(roms, mappers, env_cart, segment_frames=2, full_tia=full_tia)
    gpu_rollout(b, synth.actions(72, n_envs, 2), 1, screens=False)
    u = torch.from_numpy(synth.action_inputs(synth.actions(71, n_envs, n_steps))).cuda()
    tape = b.soft_rollout(0.3, u, 1)
    gr = torch.from_numpy(synth.normal_f32(71, (n_steps, n_envs, 128), 1)).cuda()
    gs = torch.from_numpy(synth.normal_f32(71, (n_steps, n_envs, 210, 160), 2)).cuda()
    want, _, _ = _grads("vcs_backward", tape, gr, gs, _outputs(n_envs, n_steps, 3))
    assert np.abs(want[0]).max() > 0 and np.abs(want[4]).max() > 0 and np.abs(want[2]).max() > 0
    for call in range(2):
        got, free0, free1 = _grads("vcs_backward_static", tape, gr, gs, _outputs(n_envs, n_steps, 3))
        for g, w, name in zip(got, want, ("grad_rom", "grad_ram0", "grad_cart_ram0", "grad_u", "grad_rom_per_cart")):
            assert np.array_equal(g, w), f"call {call}: {name} differs from vcs_backward's"
        if call == 1:
            assert free1 == free0, f"the static backward changed the free device memory by {free0 - free1} bytes"


def test_static_backward_rejects_oversized_problems():
    torch = torch_cuda()
    rom = synth.generate_cart(73, 0, synth.MAPPER_4K)
    n_envs = 2048
    b = make_batch([rom], [synth.MAPPER_4K], np.zeros(n_envs, np.int32))
    u = torch.from_numpy(synth.action_inputs(synth.actions(73, n_envs, 8))).cuda()
    tape = b.soft_rollout(0.1, u, 1)
    b.sync()
    g = torch.empty((n_envs, 128), device="cuda")
    st = _lib.load().vcs_backward_static(tape.h, None, None, None, None, C.c_void_p(g.data_ptr()), None, None,
                                         None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.VCS_ERR_ARG
    assert "fixed" in _lib.load().vcs_last_error(b.h).decode()
