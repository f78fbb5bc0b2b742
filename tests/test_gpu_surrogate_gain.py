"""What training the surrogate gains, measured on held-out volumes against the plain method.

The network is trained for a short, fixed budget (seeded crops of F3-kind 64^3 volumes
labelled by the plain FP32 method) and compared with the same network untrained: its error
against the plain E on volumes it never saw must fall well below the untrained one's.  The
per-block fallback keeps the final E within the threshold either way; the test also reports
the fraction of check blocks each network keeps and the time of the network against the
plain energy kernel on the same volume (on GB300 the plain sliding-DFT path is the faster one,
which the printed numbers state)."""
import numpy as np
import pytest
import torch

from paper_1901_11095_gb300 import api, surrogate, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel_l2(P, E):
    return [float(torch.linalg.vector_norm((P[m] - E[m]).double()) / torch.linalg.vector_norm(E[m].double()))
            for m in range(3)]


def _ms(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def test_training_gains_accuracy_on_held_out_volumes():
    p = api.params(L=7)
    train = [torch.from_numpy(synth.make_volume((64, 64, 64), seed=200 + i, kind="f3")).to(DEV) for i in range(12)]
    labels = [api.sal_spectral_energy(V, p) for V in train]
    held = [torch.from_numpy(synth.make_volume((64, 64, 96), seed=950 + i, kind="f3")).to(DEV) for i in range(2)]
    held_E = [api.sal_spectral_energy(V, p) for V in held]

    untrained = surrogate.Surrogate(DEV, seed=0)
    model = surrogate.Surrogate(DEV, seed=0)
    hist = surrogate.train(model, train, labels, steps=1500, crop=40, lr=3e-3, lr_final=3e-4, seed=1, log_every=500)
    assert hist[-1][1] < hist[0][1]

    err_u = np.mean([_rel_l2(untrained.forward(V, training=True), E) for V, E in zip(held, held_E)], axis=0)
    err_t = np.mean([_rel_l2(model.forward(V, training=True), E) for V, E in zip(held, held_E)], axis=0)
    kept = {}
    for thr in (2e-2, 1e-1, 3e-1):
        ct = model.infer(held[0], threshold=thr)[1].cpu().numpy()
        cu = untrained.infer(held[0], threshold=thr)[1].cpu().numpy()
        kept[thr] = (1 - ct[0] / ct[1], 1 - cu[0] / cu[1])
        assert kept[thr][0] >= kept[thr][1]          # training never loses blocks to the fallback
    V = held[1]
    t_plain = _ms(lambda: api.sal_spectral_energy(V, p))
    t_net = _ms(lambda: model.forward(V, training=False, p=api.params(L=7, precision="bf16")))
    api.sal_device_status()
    print(f"held-out E rel-L2 per map: trained {err_t.round(4).tolist()}, untrained {err_u.round(4).tolist()}; "
          f"blocks kept (trained, untrained) per threshold {kept}; network {t_net:.3f} ms vs plain energies "
          f"{t_plain:.3f} ms on {tuple(V.shape)}")
    # the gain of training: the held-out error falls to well under half the untrained network's
    assert float(err_t.mean()) < 0.5 * float(err_u.mean())
    assert np.isfinite(t_net) and np.isfinite(t_plain)
