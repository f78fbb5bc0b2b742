"""The learned surrogate's kernels (forward, gradients, Adam), its training and its
inference with the per-block fallback, against the FP64 reference of its layers and the
plain method."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import _native as N
from paper_1901_11095_gb300 import api, surrogate, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _bf16(p):
    """Weights rounded to BF16 as the kernels read them (biases stay FP32)."""
    p = np.asarray(p, dtype=np.float32).copy()
    o = 0
    for l in range(len(surrogate.WIDTHS) - 1):
        nw = surrogate.WIDTHS[l + 1] * surrogate.WIDTHS[l] * 27
        p[o:o + nw] = torch.from_numpy(p[o:o + nw]).bfloat16().float().numpy()
        o += nw + surrogate.WIDTHS[l + 1]
    return p.astype(np.float64)


def _model(seed=3, scale=1.0):
    params = surrogate.init_params(seed)
    rng = np.random.default_rng(seed)
    params = params + 0.05 * rng.standard_normal(params.size).astype(np.float32)   # non-zero biases too
    params *= np.float32(scale)
    return surrogate.Surrogate(DEV, params=params), params


def test_forward_matches_reference():
    V = synth.make_volume((12, 14, 40), seed=1)
    model, params = _model()
    Vd = torch.from_numpy(V).to(DEV)
    rms = np.sqrt(np.mean(V.astype(np.float64) ** 2))
    ref = O.surrogate_forward(V[None].astype(np.float64) / rms, surrogate.WIDTHS, _bf16(params)) * rms
    got = model.forward(Vd, training=True).cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-4
    got_inf = model.forward(Vd, training=False).cpu().numpy()       # BF16 activations
    assert np.abs(got_inf - ref).max() / np.abs(ref).max() < 3e-2


@pytest.mark.parametrize("shape,bnd", [((12, 14, 40), "reflect"), ((9, 7, 300), "reflect"),
                                       ((5, 6, 128), "periodic"), ((8, 4, 129), "reflect"),
                                       ((6, 3, 257), "periodic"), ((10, 1, 1), "reflect")])
def test_tensor_core_inference_matches_cuda_cores_and_reference(shape, bnd):
    """Hidden layers as tcgen05 products (BF16 operands, FP32 accumulation) against the CUDA-core
    inference (same BF16 activations) and the FP64 reference; lines of 128 outputs along y,
    ragged at the end (40 and 300 = 2 x 128 + 44), lines whose halo meets both y faces, the
    extension row y = Y at every position of a line (Y = 128, 129, 257) and single-sample axes."""
    V = synth.make_volume(shape, seed=2)
    model, params = _model(seed=4)
    Vd = torch.from_numpy(V).to(DEV)
    rms = np.sqrt(np.mean(V.astype(np.float64) ** 2))
    ref = O.surrogate_forward(V[None].astype(np.float64) / rms, surrogate.WIDTHS, _bf16(params),
                              bnd=O.PERIODIC if bnd == "periodic" else O.REFLECT) * rms
    cc = model.forward(Vd, training=False, p=api.params(boundary=bnd)).cpu().numpy()
    api.sal_device_status()
    tc = model.forward(Vd, training=False, p=api.params(precision="bf16", boundary=bnd)).cpu().numpy()
    api.sal_device_status()
    assert np.isfinite(tc).all()
    assert np.abs(tc - cc).max() / np.abs(cc).max() < 1e-2
    assert np.abs(tc - ref).max() / np.abs(ref).max() < 3e-2


def test_tensor_core_inference_wait_runs_out_and_context_survives():
    V = torch.from_numpy(synth.make_volume((6, 5, 130), seed=5)).to(DEV)
    model, _ = _model(seed=6)
    p = api.params(precision="bf16")
    ref = model.forward(V, training=False, p=p).clone()
    api.sal_device_status()
    api.sal_test_stall_tensor_cores(True)
    try:
        model.forward(V, training=False, p=p)
        with pytest.raises(N.SalError) as ei:
            api.sal_device_status()
        assert ei.value.status == N.SAL_ERR_TIMEOUT
    finally:
        api.sal_test_stall_tensor_cores(False)
    api.sal_device_status()
    again = model.forward(V, training=False, p=p)
    api.sal_device_status()
    assert torch.equal(again, ref)


def test_backward_matches_reference():
    V = synth.make_volume((16, 17, 40), seed=2)
    model, params = _model(seed=4)
    Vd = torch.from_numpy(V).to(DEV)
    rng = np.random.default_rng(0)
    target = rng.standard_normal((3,) + V.shape).astype(np.float32)
    Td = torch.from_numpy(target).to(DEV)
    margin = surrogate.MARGIN
    p = api.params()
    ws = model._workspace(V.shape, True)
    s = torch.cuda.current_stream().cuda_stream
    N.check(N.lib().sal_surrogate_forward(Vd.data_ptr(), api.dims_of(Vd), ctypes.byref(p), model.params.data_ptr(),
                                          None, 1, ws.data_ptr(), ws.numel(), s))
    N.check(N.lib().sal_surrogate_backward(Vd.data_ptr(), api.dims_of(Vd), ctypes.byref(p), model.params.data_ptr(),
                                           Td.data_ptr(), margin, model.grads.data_ptr(), model.loss.data_ptr(),
                                           ws.data_ptr(), ws.numel(), s))
    g = model.grads.cpu().numpy().astype(np.float64)
    loss = float(model.loss.item())
    rms = np.sqrt(np.mean(V.astype(np.float64) ** 2))
    mask = np.zeros(V.shape)
    mask[margin:-margin, margin:-margin, margin:-margin] = 1.0
    cnt = mask.sum()
    ref_loss, ref_g = O.surrogate_loss_grad(V[None].astype(np.float64) / rms, surrogate.WIDTHS, _bf16(params),
                                            target.astype(np.float64) / rms, mask)
    assert np.isclose(loss, ref_loss / (3 * cnt), rtol=1e-4)
    ref_g /= 3 * cnt
    assert np.abs(g - ref_g).max() / np.abs(ref_g).max() < 1e-3


def test_adam_step():
    n = surrogate.param_count()
    rng = np.random.default_rng(5)
    w, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    m, v = rng.standard_normal(n).astype(np.float32) * 0.1, rng.uniform(0, 0.1, n).astype(np.float32)
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (w, g, m, v)]
    N.check(N.lib().sal_surrogate_adam_step(t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(), 3,
                                            ctypes.c_float(1e-2), ctypes.c_float(0.9), ctypes.c_float(0.999),
                                            ctypes.c_float(1e-8), None))
    m2 = 0.9 * m.astype(np.float64) + 0.1 * g
    v2 = 0.999 * v.astype(np.float64) + 0.001 * g.astype(np.float64) ** 2
    w2 = w - 1e-2 * (m2 / (1 - 0.9 ** 3)) / (np.sqrt(v2 / (1 - 0.999 ** 3)) + 1e-8)
    torch.cuda.synchronize()
    np.testing.assert_allclose(t[0].cpu().numpy(), w2, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t[2].cpu().numpy(), m2, rtol=1e-5, atol=1e-7)


def test_training_reduces_loss_and_checkpoint_roundtrip(tmp_path):
    vols = [torch.from_numpy(synth.make_volume((48, 48, 64), seed=100 + i)).to(DEV) for i in range(3)]
    p = api.params(L=7)
    labels = [api.sal_spectral_energy(V, p) for V in vols]
    model = surrogate.Surrogate(DEV, seed=0)
    hist = surrogate.train(model, vols, labels, steps=240, crop=32, lr=3e-3, lr_final=1e-3, seed=1, log_every=1)
    first = np.mean([l for _, l in hist[:20]])
    last = np.mean([l for _, l in hist[-20:]])
    assert last < 0.5 * first, (first, last)
    ck = tmp_path / "surr.npz"
    model.save(str(ck))
    other = surrogate.Surrogate(DEV, seed=9)
    other.load(str(ck))
    assert torch.equal(other.params, model.params) and other.step == model.step
    V = vols[0]
    assert torch.equal(other.forward(V), model.forward(V))


def test_inference_fallback_extremes():
    V = torch.from_numpy(synth.make_volume((40, 37, 70), seed=7)).to(DEV)
    api.sal_autotune_clear()
    p = api.params(L=7)
    plain = api.sal_spectral_energy(V, p)
    model, _ = _model(seed=6)
    pred = model.forward(V)
    E_all, c_all = model.infer(V, p, threshold=0.0)          # every block recomputed by the plain method
    E_none, c_none = model.infer(V, p, threshold=1e30)       # none recomputed
    torch.cuda.synchronize()
    nb = int(c_all[1])
    assert int(c_all[0]) == nb and int(c_none[0]) == 0 and int(c_none[1]) == nb
    assert torch.equal(E_all, plain)
    assert torch.equal(E_none, pred)
    E_mid, c_mid = model.infer(V, p, threshold=2e-2)
    torch.cuda.synchronize()
    k = int(c_mid[0])
    assert 0 <= k <= nb
    # every voxel is either the plain value or the prediction
    same = (E_mid == plain).all(dim=0) | (E_mid == pred).all(dim=0)
    assert bool(same.all())
