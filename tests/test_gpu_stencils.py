"""Parity of the tunable directional comparisons (Eq. 5 with the t-x diagonal of Fig. 3 and
with caller-given offsets and weights) with the FP64 oracle, through the C ABI."""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1901_11095_gb300 import api, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL_MAP = 2e-5
TOL_S = 1e-4
BND = {"reflect": O.REFLECT, "periodic": O.PERIODIC}


def nerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (scale if scale > 0 else 1.0))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("L,bnd,sigma,shape", [(7, "reflect", 1.0, (21, 19, 67)), (5, "periodic", 0.7, (16, 23, 64)),
                                               (15, "reflect", 2.0, (30, 17, 70)), (3, "periodic", 1.3, (9, 9, 9)),
                                               # several chunks of 128 planes, the last one ragged
                                               (7, "reflect", 1.0, (150, 13, 70)), (5, "periodic", 0.9, (260, 9, 33))])
def test_diag_tx_compare_matches_oracle(L, bnd, sigma, shape):
    rng = np.random.default_rng(11)
    E = rng.uniform(0.0, 1.0, size=(3,) + shape).astype(np.float32)
    p = api.params(L=L, boundary=bnd, stencil="diag_tx", sigma=sigma)
    Sm, st = api.sal_directional_compare(to_dev(E), p)
    Sm_ref = O.dcs(E.astype(np.float64), bnd=BND[bnd], stencil=O.STENCIL_DIAG_TX, L=L, sigma=sigma)
    Smh = Sm.cpu().numpy()
    for m in range(3):
        assert nerr(Smh[m], Sm_ref[m]) < TOL_MAP, m
    sth = st.cpu().numpy().reshape(3, 3)
    for m in range(3):
        assert sth[m, 0] == float(Sm[m].min()) and sth[m, 1] == float(Sm[m].max())
    np.testing.assert_allclose(sth[:, 2], O.stats(Sm_ref)[:, 2], rtol=1e-5)


def _random_stencil(rng, q, radius):
    offs, wts = [], []
    for m in range(3):
        cand = [o for o in itertools.product(range(-radius, radius + 1), repeat=3) if o != (0, 0, 0)]
        pick = rng.choice(len(cand), size=q[m], replace=False)
        offs.append([cand[i] for i in pick])
        wts.append(list(rng.uniform(-1.0, 1.5, size=q[m])))
    return offs, wts


@pytest.mark.parametrize("q,radius,bnd,shape", [((1, 5, 12), 2, "reflect", (19, 21, 70)),
                                                ((64, 30, 3), 7, "periodic", (24, 20, 66)),
                                                ((9, 9, 9), 4, "reflect", (8, 9, 64)),
                                                ((10, 7, 20), 3, "reflect", (150, 12, 70)),
                                                ((5, 40, 6), 7, "periodic", (131, 10, 67))])
def test_user_stencil_matches_oracle(q, radius, bnd, shape):
    rng = np.random.default_rng(sum(q))
    offs, wts = _random_stencil(rng, q, radius)
    E = rng.uniform(0.0, 1.0, size=(3,) + shape).astype(np.float32)
    p = api.params(boundary=bnd)
    st_u = api.user_stencil(offs, wts)
    Sm, st = api.sal_directional_compare_user(to_dev(E), p, st_u)
    # the oracle sees the weights the library was given (float32)
    w32 = [list(np.float32(w).astype(np.float64)) for w in wts]
    Sm_ref = O.dcs_user(E.astype(np.float64), offs, w32, bnd=BND[bnd])
    Smh = Sm.cpu().numpy()
    for m in range(3):
        assert nerr(Smh[m], Sm_ref[m]) < TOL_MAP, m
    sth = st.cpu().numpy().reshape(3, 3)
    for m in range(3):
        assert sth[m, 0] == float(Sm[m].min()) and sth[m, 1] == float(Sm[m].max())


def test_user_stencil_of_the_26_neighbourhood_matches_the_built_in():
    rng = np.random.default_rng(3)
    E = to_dev(rng.uniform(0.0, 1.0, size=(3, 40, 18, 100)).astype(np.float32))
    sigma = 1.2
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0)]
    w = [math.exp(-sum(c * c for c in o) / (2 * sigma * sigma)) for o in offs]
    p = api.params(sigma=sigma)
    Sm_u, _ = api.sal_directional_compare_user(E, p, api.user_stencil([offs] * 3, [w] * 3))
    Sm_b, _ = api.sal_directional_compare(E, p)
    scale = float(Sm_b.abs().max())
    assert float((Sm_u - Sm_b).abs().max()) <= 4e-7 * scale


def test_diag_tx_whole_method_matches_oracle():
    V = synth.make_volume((26, 30, 41), seed=12)
    L, sigma = 7, 1.1
    p = api.params(L=L, stencil="diag_tx", sigma=sigma)
    S, _ = api.sal_saliency(to_dev(V), p, stats=torch.empty(9, dtype=torch.float64, device=DEV))
    S_ref = O.saliency(V, L=L, stencil=O.STENCIL_DIAG_TX, sigma=sigma)
    assert nerr(S.cpu().numpy(), S_ref) < TOL_S


def test_user_stencil_rejects_bad_offsets():
    E = torch.zeros((3, 4, 4, 8), device=DEV)
    p = api.params()
    for offs, wts in (([[(0, 0, 0)], [(1, 0, 0)], [(1, 0, 0)]], [[1.0]] * 3),
                      ([[(8, 0, 0)], [(1, 0, 0)], [(1, 0, 0)]], [[1.0]] * 3),
                      ([[(1, 0, 0)], [], [(1, 0, 0)]], [[1.0], [], [1.0]]),
                      ([[(1, 0, 0)], [(1, 0, 0)], [(1, 0, 0)]], [[float("nan")], [1.0], [1.0]])):
        with pytest.raises(api.N.SalError) as ei:
            api.sal_directional_compare_user(E, p, api.user_stencil(offs, wts))
        assert ei.value.status == api.N.SAL_ERR_INVALID_ARG
