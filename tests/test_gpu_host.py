"""The host-buffer entry point (V and S in host memory, copies inside the library, calls
overlapped through double buffers) against the device-buffer path, through the C ABI."""
import pytest
import torch

from paper_1901_11095_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _device_result(Vh, p):
    S, _ = api.sal_saliency(Vh.to(DEV), p)
    return S.cpu()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_equals_device_call(pinned):
    shape = (23, 30, 71)
    Vh = torch.from_numpy(synth.make_volume(shape, seed=21))
    if pinned:
        Vh = Vh.pin_memory()
    p = api.params(L=7)
    stats = torch.empty(9, device=DEV, dtype=torch.float64)
    Sh = api.sal_saliency_host(Vh, p, stats=stats)
    torch.cuda.synchronize()
    ref = _device_result(Vh, p)
    assert torch.equal(Sh, ref)
    _, st_ref = api.sal_saliency(Vh.to(DEV), p, stats=torch.empty(9, device=DEV, dtype=torch.float64))
    assert torch.equal(stats, st_ref)


@pytest.mark.parametrize("bnd", ["reflect", "periodic"])
def test_host_call_in_pieces_equals_device_call(bnd):
    """T >= 64: V is copied in pieces of planes and the energies of each piece start once it
    and its halo are on the device; the result must match the whole-volume call exactly."""
    Vh = torch.from_numpy(synth.make_volume((150, 21, 45), seed=22)).pin_memory()
    p = api.params(L=7, boundary=bnd)
    Sh = api.sal_saliency_host(Vh, p)
    torch.cuda.synchronize()
    assert torch.equal(Sh, _device_result(Vh, p))


def test_overlapped_sequence_keeps_every_result():
    """Consecutive calls on one workspace with done events: each call's S must be its own
    volume's result although V and S buffers alternate and copies overlap kernels."""
    shapes = [(31, 40, 66)] * 5
    p = api.params(L=5)
    Vs = [torch.from_numpy(synth.make_volume(sh, seed=40 + i)).pin_memory() for i, sh in enumerate(shapes)]
    ws = torch.empty(api.sal_host_workspace_size(api.dims_of(Vs[0]), p), device=DEV, dtype=torch.uint8)
    outs, evs = [], []
    for V in Vs:
        ev = torch.cuda.Event()
        outs.append(api.sal_saliency_host(V, p, ws=ws, done_event=ev))
        evs.append(ev)
    for ev in evs:
        ev.synchronize()
    for V, S in zip(Vs, outs):
        assert torch.equal(S, _device_result(V, p))
    api.sal_host_release(ws)
    # the workspace can be used again after the release (state is recreated)
    S = api.sal_saliency_host(Vs[0], p, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(S, outs[0])
    api.sal_host_release(ws)


def test_host_call_tensor_core_precision():
    Vh = torch.from_numpy(synth.make_volume((20, 24, 40), seed=3)).pin_memory()
    p = api.params(L=7, precision="bf16")
    Sh = api.sal_saliency_host(Vh, p)
    torch.cuda.synchronize()
    assert torch.equal(Sh, _device_result(Vh, p))
