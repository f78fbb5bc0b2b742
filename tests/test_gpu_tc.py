"""Tensor-core form of the DFT stage (tcgen05, BF16 or TF32 operands, FP32 accumulation)
against the FP64 oracle, with the error stated per output map.

Tolerances (normwise, relative to the largest value of the map): the operands are rounded
once, to 8 (BF16) or 11 (TF32) significant bits, so each spectral coefficient carries a
relative error of order 2^-9 (BF16) or 2^-12 (TF32) of its inputs' magnitude; E averages
hundreds of such magnitudes.  Bars: E_m 1e-2 (BF16) and 2e-3 (TF32); S by relative L2
2e-2 (BF16, the stated target) and 5e-3 (TF32).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import api, synth
from paper_1901_11095_gb300 import _native as N

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_E = {"bf16": 1e-2, "tf32": 2e-3}
TOL_S = {"bf16": 2e-2, "tf32": 5e-3}


def nerr(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(np.asarray(got, dtype=np.float64) - ref).max() / max(np.abs(ref).max(), 1e-300))


def l2err(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(got, dtype=np.float64) - ref) / max(np.linalg.norm(ref), 1e-300))


CASES = [((64, 64, 64), 7, "reflect"), ((37, 45, 70), 5, "reflect"), ((20, 17, 33), 9, "periodic"),
         ((13, 29, 31), 3, "reflect"), ((12, 21, 40), 11, "periodic"), ((14, 15, 36), 13, "reflect"),
         ((16, 18, 35), 15, "reflect")]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("shape,L,bnd", CASES)
def test_tc_energy_and_saliency_match_oracle(prec, shape, L, bnd):
    if prec == "tf32" and L > 11:
        pytest.skip("TF32 operands of L > 11 do not fit one CTA's shared memory")
    V = synth.make_volume(shape, seed=L)
    p = api.params(L=L, boundary=bnd, precision=prec)
    Vd = torch.from_numpy(V).to(DEV)
    E = api.sal_spectral_energy(Vd, p).cpu().numpy()
    api.sal_device_status()
    S, E_ref, _, _ = O.saliency(V, L=L, bnd=O.REFLECT if bnd == "reflect" else O.PERIODIC, full=True)
    errs = [nerr(E[m], E_ref[m]) for m in range(3)]
    S_gpu, _ = api.sal_saliency(Vd, p)
    es = l2err(S_gpu.cpu().numpy(), S)
    print(f"{prec} L={L} {shape}: E errors {errs}, S rel-L2 {es:.2e}")
    assert max(errs) < TOL_E[prec]
    assert es < TOL_S[prec]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_constant_volume_is_exactly_zero(prec):
    V = torch.full((19, 23, 41), -2.5, device=DEV)
    p = api.params(L=7, precision=prec)
    assert bool((api.sal_spectral_energy(V, p) == 0).all())
    S, _ = api.sal_saliency(V, p)
    assert bool((S == 0).all())


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (5, 1, 7), (3, 40, 3)])
def test_tc_degenerate_volumes(shape):
    V = synth.make_volume(shape, seed=4)
    p = api.params(L=5, precision="bf16")
    E = api.sal_spectral_energy(torch.from_numpy(V).to(DEV), p).cpu().numpy()
    E_ref = O.energy(V, 5)
    for m in range(3):
        assert np.abs(E[m] - E_ref[m]).max() <= TOL_E["bf16"] * max(np.abs(E_ref).max(), 1e-30)


def test_tc_batched_equals_single():
    rng = np.random.default_rng(2)
    vols = [synth.make_volume(tuple(int(v) for v in rng.integers(8, 60, size=3)), seed=i) for i in range(6)]
    Vs = [torch.from_numpy(v).to(DEV) for v in vols]
    p = api.params(L=7, precision="bf16")
    Ss, _ = api.sal_saliency_batched(Vs, p)
    for V, S in zip(Vs, Ss):
        S1, _ = api.sal_saliency(V, p)
        assert torch.equal(S, S1)
    api.sal_device_status()


def test_tc_wait_timeout_is_reported_and_recovers():
    V = torch.from_numpy(synth.make_volume((9, 16, 40), seed=3)).to(DEV)
    p = api.params(L=7, precision="bf16")
    ref = api.sal_spectral_energy(V, p)
    api.sal_device_status()
    api.sal_test_stall_tensor_cores(True)
    try:
        api.sal_spectral_energy(V, p)
        with pytest.raises(N.SalError) as ei:
            api.sal_device_status()
        assert ei.value.status == N.SAL_ERR_TIMEOUT
    finally:
        api.sal_test_stall_tensor_cores(False)
    api.sal_device_status()                       # cleared; the context stays usable
    again = api.sal_spectral_energy(V, p)
    api.sal_device_status()
    assert torch.equal(again, ref)


def test_bf16_batch_members_match_oracle():
    """The batched configuration (64 uneven volumes, axes U[32, 192], BF16, one persistent launch
    per stage): two members, the smallest and one of median size, against the oracle's S."""
    shapes = synth.batch_shapes()
    vols = [synth.make_volume(s, seed=i) for i, s in enumerate(shapes)]
    Vs = [torch.from_numpy(v).to(DEV) for v in vols]
    p = api.params(L=7, precision="bf16")
    Ss, _ = api.sal_saliency_batched(Vs, p)
    api.sal_device_status()
    sizes = [v.size for v in vols]
    order = np.argsort(sizes)
    for i in (int(order[0]), int(order[len(order) // 2])):
        S_ref = O.saliency(vols[i], L=7)
        err = l2err(Ss[i].cpu().numpy(), S_ref)
        print(f"batch member {i} {shapes[i]}: S rel-L2 {err:.2e}")
        assert err < TOL_S["bf16"]
