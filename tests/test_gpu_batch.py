"""Batched uneven volumes (one persistent launch per stage), the library-captured CUDA
graph and the autotuner, through the C ABI, against per-volume calls and the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import _native as N, api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _batch(n=9, lo=5, hi=70, seed=0):
    rng = np.random.default_rng(seed)
    shapes = [tuple(int(v) for v in rng.integers(lo, hi + 1, size=3)) for _ in range(n)]
    shapes[0] = (1, 1, 1)                      # degenerate member
    return [synth.make_volume(s, seed=i) for i, s in enumerate(shapes)]


ORC_STENCIL = {"26": O.STENCIL_26, "line": O.STENCIL_LINE, "diag_tx": O.STENCIL_DIAG_TX}


@pytest.mark.parametrize("stencil,L", [("26", 7), ("line", 5), ("diag_tx", 7)])
def test_batched_equals_per_volume_and_oracle(stencil, L):
    api.sal_autotune_clear()
    vols = _batch()
    Vs = [torch.from_numpy(v).to(DEV) for v in vols]
    p = api.params(L=L, stencil=stencil)
    stats = torch.empty((len(Vs), 9), dtype=torch.float64, device=DEV)
    Ss, _ = api.sal_saliency_batched(Vs, p, stats=stats)
    torch.cuda.synchronize()
    for i, V in enumerate(Vs):
        st1 = torch.empty(9, dtype=torch.float64, device=DEV)
        S1, _ = api.sal_saliency(V, p, stats=st1)
        assert torch.equal(Ss[i], S1), i                       # same kernels, same arithmetic
        assert torch.equal(stats[i].view(3, 3)[:, :2], st1.view(3, 3)[:, :2])
        torch.testing.assert_close(stats[i].view(3, 3)[:, 2], st1.view(3, 3)[:, 2], rtol=1e-12, atol=0)
    for i in (1, len(vols) - 1):
        S_ref = O.saliency(vols[i], L=L, stencil=ORC_STENCIL[stencil])
        err = np.abs(Ss[i].cpu().numpy() - S_ref).max() / max(np.abs(S_ref).max(), 1e-30)
        assert err < 1e-4


def test_graph_replays_the_batch():
    api.sal_autotune_clear()
    vols = _batch(n=12, seed=3)
    Vs = [torch.from_numpy(v).to(DEV) for v in vols]
    p = api.params(L=7)
    stats = torch.empty((len(Vs), 9), dtype=torch.float64, device=DEV)
    g = api.SalGraph(Vs, p, stats=stats)              # runs the autotuner first (empty cache)
    ref, _ = api.sal_saliency_batched(Vs, p)          # the same (tuned) tile shape, outside the graph
    for _ in range(3):
        for S in g.Ss:
            S.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        for a, b in zip(g.Ss, ref):
            assert torch.equal(a, b)
    # the inputs are read at replay time: new data in the same buffers gives new results
    Vs[2].mul_(-1.0)
    g.launch()
    torch.cuda.synchronize()
    S2, _ = api.sal_saliency(Vs[2], p)
    assert torch.equal(g.Ss[2], S2)
    g.close()
    c = api.sal_autotune_query(7, 0, max(v.size for v in vols))
    assert c["ms"] > 0 and c["bt"] > 0


def test_autotune_single_volume_and_identical_results():
    api.sal_autotune_clear()
    V = torch.from_numpy(synth.make_volume((48, 40, 96), seed=5)).to(DEV)
    p = api.params(L=7)
    ref = api.sal_spectral_energy(V, p)
    c = api.sal_autotune(V, p)
    assert c["ms"] > 0 and c["shape"] >= 0
    got = api.sal_spectral_energy(V, p)                 # now with the tuned tile shape
    # every tile shape computes the same values up to the rounding of its sliding steps
    assert float((got - ref).abs().max()) <= 5e-6 * float(ref.abs().max())
    api.sal_autotune_clear()


@pytest.mark.parametrize("L", [3, 5, 7, 9])
def test_every_tile_shape_and_mode_agrees(L, tmp_path):
    """Each candidate (tile shape, staging mode) is forced through a cache file.  The kernels
    differ in how work is split and staged and in where the sliding recurrence along x
    restarts (every BX outputs), so the energies agree to a few FP32 roundings; candidates
    with the same x tile width and the sliding x stage (modes 0, 3 and 4) agree bit for bit."""
    V = torch.from_numpy(synth.make_volume((19, 37, 75), seed=8)).to(DEV)
    p = api.params(L=L)
    api.sal_autotune_clear()
    ref = api.sal_spectral_energy(V, p)
    ref_shape = api.sal_autotune_query(L, 0, V.numel())
    shape = 0
    while True:
        f = tmp_path / f"cache_{L}_{shape}.txt"
        f.write_text(f"# sal autotune cache v1: L precision size_class shape ms\n{L} 0 0 {shape} 1.0\n")
        try:
            api.sal_autotune_load(str(f))
        except N.SalError:
            break                                         # past the last candidate
        c = api.sal_autotune_query(L, 0, V.numel())
        assert c["shape"] == shape
        got = api.sal_spectral_energy(V, p)
        assert float((got - ref).abs().max()) <= 5e-6 * float(ref.abs().max()), f"shape {shape}"
        if c["bx"] == ref_shape["bx"] and c["mode"] in (0, 3, 4):
            assert torch.equal(got, ref), f"shape {shape}"
        shape += 1
    api.sal_autotune_clear()
    assert shape >= 2
