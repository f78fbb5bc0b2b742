"""The learned surrogate of the spectral energies: parameters, training and inference,
driving the library's kernels (sal_surrogate_* in include/sal.h).

Network: 5 layers of 3x3x3 convolution, 1 -> 24 -> 24 -> 24 -> 24 -> 3 channels, GELU after
the first four; BF16 weights (rounded from FP32 master parameters by the kernels), FP32
accumulation.  It predicts E_t, E_x, E_y from the amplitudes.  Training: Adam on random
crops of labelled volumes, the loss restricted to voxels whose receptive field lies inside
the crop.  Inference falls back, per check block, to the plain method wherever sampled
exact values show an error above the threshold.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from . import api
from ._native import SalDims, check

WIDTHS = [1] + [N.SAL_SURR_WIDTH] * (N.SAL_SURR_LAYERS - 1) + [3]
MARGIN = N.SAL_SURR_LAYERS            # receptive-field radius: one voxel per layer


def param_count() -> int:
    n = ctypes.c_int64()
    check(N.lib().sal_surrogate_param_count(ctypes.byref(n)))
    return n.value


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (27 cin))), zero biases; the output layer scaled down."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(len(WIDTHS) - 1):
        cin, cout = WIDTHS[l], WIDTHS[l + 1]
        std = np.sqrt(2.0 / (27 * cin)) * (0.1 if l == len(WIDTHS) - 2 else 1.0)
        out.append(rng.standard_normal(cout * cin * 27) * std)
        out.append(np.zeros(cout))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == param_count()
    return p


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Surrogate:
    """Device-resident parameters and Adam state."""

    def __init__(self, device="cuda:0", seed: int = 0, params: np.ndarray | None = None):
        self.device = torch.device(device)
        p = init_params(seed) if params is None else np.asarray(params, dtype=np.float32)
        self.params = torch.from_numpy(p.copy()).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.step = 0
        self.p = api.params()
        self._ws = {}

    def _workspace(self, shape, training: bool) -> torch.Tensor:
        key = (tuple(shape), training)
        if key not in self._ws:
            n = ctypes.c_size_t()
            check(N.lib().sal_surrogate_workspace_size(SalDims(*shape), int(training), ctypes.byref(n)))
            self._ws = {key: torch.empty(n.value, dtype=torch.uint8, device=self.device)}
        return self._ws[key]

    def forward(self, V: torch.Tensor, training: bool = False, E: torch.Tensor | None = None, stream=None,
                p=None):
        """E from V.  Inference (training=False) with p.precision = bf16 runs the hidden layers
        on the tensor cores."""
        p = p if p is not None else self.p
        if E is None:
            E = torch.empty((3,) + tuple(V.shape), device=V.device, dtype=torch.float32)
        ws = self._workspace(V.shape, training)
        check(N.lib().sal_surrogate_forward(_ptr(V), api.dims_of(V), ctypes.byref(p), _ptr(self.params),
                                            _ptr(E), int(training), _ptr(ws), ws.numel(), _stream(stream)))
        return E

    def train_step(self, V: torch.Tensor, E_target: torch.Tensor, lr: float = 1e-3, margin: int = MARGIN,
                   betas=(0.9, 0.999), eps: float = 1e-8, stream=None) -> torch.Tensor:
        """One forward/backward/Adam step on one crop; returns the loss (device tensor)."""
        ws = self._workspace(V.shape, True)
        s = _stream(stream)
        check(N.lib().sal_surrogate_forward(_ptr(V), api.dims_of(V), ctypes.byref(self.p), _ptr(self.params), None,
                                            1, _ptr(ws), ws.numel(), s))
        check(N.lib().sal_surrogate_backward(_ptr(V), api.dims_of(V), ctypes.byref(self.p), _ptr(self.params),
                                             _ptr(E_target), int(margin), _ptr(self.grads), _ptr(self.loss),
                                             _ptr(ws), ws.numel(), s))
        self.step += 1
        check(N.lib().sal_surrogate_adam_step(_ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v),
                                              self.step, float(lr), float(betas[0]), float(betas[1]), float(eps), s))
        return self.loss

    def infer(self, V: torch.Tensor, p=None, threshold: float = 2e-2, E: torch.Tensor | None = None,
              stream=None):
        """E with the per-block fallback; returns (E, blocks recomputed, blocks checked) (counts on the device)."""
        p = p if p is not None else self.p
        if E is None:
            E = torch.empty((3,) + tuple(V.shape), device=V.device, dtype=torch.float32)
        n = ctypes.c_size_t()
        check(N.lib().sal_surrogate_infer_workspace_size(api.dims_of(V), ctypes.byref(p), ctypes.byref(n)))
        ws = torch.empty(n.value, dtype=torch.uint8, device=V.device)
        counts = torch.zeros(2, dtype=torch.int32, device=V.device)
        check(N.lib().sal_surrogate_infer(_ptr(V), api.dims_of(V), ctypes.byref(p), _ptr(self.params), _ptr(E),
                                          float(threshold), _ptr(counts), _ptr(ws), ws.numel(), _stream(stream)))
        return E, counts

    def state(self) -> dict:
        return {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "step": np.int64(self.step)}

    def save(self, path: str) -> None:
        np.savez(path, **self.state())

    def load(self, path: str) -> None:
        z = np.load(path)
        self.params.copy_(torch.from_numpy(z["params"]))
        self.m.copy_(torch.from_numpy(z["m"]))
        self.v.copy_(torch.from_numpy(z["v"]))
        self.step = int(z["step"])


def train(model: Surrogate, volumes, labels, steps: int, crop: int = 40, lr: float = 2e-3, seed: int = 0,
          log_every: int = 0, lr_final: float | None = None):
    """Adam on random crops (one per step) of the labelled volumes; returns the loss history.

    ``volumes`` are device tensors [T][X][Y]; ``labels`` the plain method's E for each, [3][T][X][Y].
    The crop's receptive-field margin keeps the loss on voxels whose prediction depends on the
    crop only, so a crop and the full volume agree there.
    """
    rng = np.random.default_rng(seed)
    hist = []
    lr_final = lr if lr_final is None else lr_final
    for it in range(steps):
        i = int(rng.integers(len(volumes)))
        V, E = volumes[i], labels[i]
        c = [min(crop, s) for s in V.shape]
        o = [int(rng.integers(0, s - k + 1)) for s, k in zip(V.shape, c)]
        sl = tuple(slice(a, a + k) for a, k in zip(o, c))
        Vc = V[sl].contiguous()
        Ec = E[(slice(None),) + sl].contiguous()
        frac = it / max(steps - 1, 1)
        cur = lr * (lr_final / lr) ** frac
        loss = model.train_step(Vc, Ec, lr=cur)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, float(loss.item())))
    return hist
