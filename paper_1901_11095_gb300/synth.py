"""Seeded synthetic seismic volumes.

These stand in for the F3 North-Sea block the paper evaluates on (Sec. 3), which is not
available here.  The module holds no arithmetic of the saliency method: it only builds
input amplitude volumes, and it is the one piece of code that both the CPU oracle tests
and the CUDA path use.

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* time axis sampled at 4 ms; layer interfaces spaced U[4, 12] samples apart;
* interface ``i`` at base depth ``z_i`` dips along crossline and inline by
  ``U[-1, 1] * 0.15 * z_i / T`` samples per trace (flat at the top, dipping at depth);
* reflection coefficient per interface U[-1, 1];
* the reflectivity series is convolved along time with a 25 Hz Ricker wavelet sampled
  at 4 ms over +-64 ms;
* vertical fault planes shift every interface on one side down by ``throw`` samples
  (6 by default);
* the ``"f3"`` kind adds three faults and an ellipsoidal dome whose interior amplitude
  is zero (a salt-like body);
* Gaussian noise with variance = signal power / 10^(SNR/10), SNR = 10 dB.

Volumes are float32, C-order ``[t][x][y]`` (time, crossline, inline).
"""
from __future__ import annotations

import numpy as np

__all__ = ["ricker", "make_volume", "batch_shapes", "plane_wave"]


def ricker(f_hz: float = 25.0, dt: float = 0.004, half_len_s: float = 0.064) -> np.ndarray:
    """Ricker wavelet (1 - 2 a) exp(-a), a = (pi f tau)^2, sampled every ``dt`` over +-half_len."""
    n = int(round(half_len_s / dt))
    tau = np.arange(-n, n + 1, dtype=np.float64) * dt
    a = (np.pi * f_hz * tau) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def _fault_sides(X: int, Y: int, n_faults: int, rng: np.random.Generator) -> list[np.ndarray]:
    """Boolean (X, Y) masks: True on the downthrown side of each vertical fault plane."""
    xs = np.arange(X, dtype=np.float64)[:, None]
    ys = np.arange(Y, dtype=np.float64)[None, :]
    sides = []
    for _ in range(n_faults):
        x0 = rng.uniform(0.3, 0.7) * X
        y0 = rng.uniform(0.3, 0.7) * Y
        ang = rng.uniform(0.0, np.pi)
        nx, ny = np.cos(ang), np.sin(ang)
        sides.append((xs - x0) * nx + (ys - y0) * ny > 0.0)
    return sides


def _convolve_t(refl: np.ndarray, w: np.ndarray, chunk: int = 8) -> np.ndarray:
    """Convolve every trace (axis 0) with the centred wavelet ``w``; zero outside the volume."""
    T = refl.shape[0]
    n = (len(w) - 1) // 2
    out = np.empty_like(refl)
    for x0 in range(0, refl.shape[1], chunk):
        src = np.ascontiguousarray(refl[:, x0:x0 + chunk, :])
        acc = np.zeros_like(src)
        for k, wk in enumerate(w):
            s = k - n  # output t receives w[k] * refl[t - s]
            if s >= T or -s >= T:
                continue
            if s >= 0:
                acc[s:] += wk * src[:T - s]
            else:
                acc[:T + s] += wk * src[-s:]
        out[:, x0:x0 + chunk, :] = acc
    return out


def make_volume(shape, seed: int = 0, kind: str = "basic", snr_db: float = 10.0,
                throw: int = 6, noise: bool = True) -> np.ndarray:
    """Seeded synthetic seismic volume of ``shape`` = (T, X, Y), float32.

    ``kind="basic"``: flat-to-dipping reflectors with one vertical fault.
    ``kind="f3"``: the same with three faults and a zero-amplitude dome.
    """
    T, X, Y = (int(s) for s in shape)
    if min(T, X, Y) < 1:
        raise ValueError("every axis must be >= 1")
    rng = np.random.default_rng(seed)
    n_faults = 3 if kind == "f3" else 1
    sides = _fault_sides(X, Y, n_faults, rng)
    shift = np.zeros((X, Y), dtype=np.int64)
    for s in sides:
        shift += throw * s.astype(np.int64)

    xs = (np.arange(X, dtype=np.float64) - 0.5 * X)[:, None]
    ys = (np.arange(Y, dtype=np.float64) - 0.5 * Y)[None, :]
    xi = np.broadcast_to(np.arange(X)[:, None], (X, Y))
    yi = np.broadcast_to(np.arange(Y)[None, :], (X, Y))

    refl = np.zeros((T, X, Y), dtype=np.float32)
    z = rng.uniform(0.0, 8.0) - throw * n_faults - 0.15 * max(X, Y)
    z_end = T + 0.15 * max(X, Y)
    while z < z_end:
        z += rng.uniform(4.0, 12.0)
        frac = min(max(z, 0.0) / max(T, 1), 1.0)
        dx = rng.uniform(-1.0, 1.0) * 0.15 * frac
        dy = rng.uniform(-1.0, 1.0) * 0.15 * frac
        r = np.float32(rng.uniform(-1.0, 1.0))
        depth = np.rint(z + dx * xs + dy * ys).astype(np.int64) + shift
        m = (depth >= 0) & (depth < T)
        refl[depth[m], xi[m], yi[m]] += r

    vol = _convolve_t(refl, ricker())
    del refl

    if kind == "f3":
        tc = rng.uniform(0.45, 0.6) * T
        xc = rng.uniform(0.3, 0.7) * X
        yc = rng.uniform(0.3, 0.7) * Y
        rx = rng.uniform(0.12, 0.2) * X
        ry = rng.uniform(0.12, 0.2) * Y
        height = rng.uniform(0.25, 0.4) * T
        d2 = ((np.arange(X)[:, None] - xc) / rx) ** 2 + ((np.arange(Y)[None, :] - yc) / ry) ** 2
        top = tc - height * (1.0 - d2)          # dome top; body extends down to the base of the volume
        inside_xy = d2 < 1.0
        tt = np.arange(T, dtype=np.float64)
        for x in range(X):
            ys_in = np.nonzero(inside_xy[x])[0]
            if ys_in.size:
                body = tt[:, None] >= top[x, ys_in][None, :]
                vol[:, x, ys_in] = np.where(body, np.float32(0.0), vol[:, x, ys_in])

    if noise:
        p = float(np.mean(vol.astype(np.float64) ** 2))
        sigma = np.sqrt(p / 10.0 ** (snr_db / 10.0)) if p > 0 else 0.0
        vol += np.float32(sigma) * rng.standard_normal(vol.shape, dtype=np.float32)
    return np.ascontiguousarray(vol, dtype=np.float32)


def batch_shapes(n: int = 64, lo: int = 32, hi: int = 192, base_seed: int = 1000) -> list[tuple[int, int, int]]:
    """Shapes of the uneven batch: every axis drawn uniformly from [lo, hi] by default_rng(base_seed + i)."""
    out = []
    for i in range(n):
        r = np.random.default_rng(base_seed + i)
        out.append(tuple(int(v) for v in r.integers(lo, hi + 1, size=3)))
    return out


def plane_wave(shape, k, period) -> np.ndarray:
    """cos(2 pi (k_t t + k_x x + k_y y) / period) on the grid of ``shape``, float32.

    With a periodic boundary and every axis a multiple of ``period``, each local cube of
    side ``period`` holds whole periods, so its spectrum is known in closed form.
    """
    T, X, Y = shape
    t = np.arange(T)[:, None, None]
    x = np.arange(X)[None, :, None]
    y = np.arange(Y)[None, None, :]
    ph = (k[0] * t + k[1] * x + k[2] * y) % period
    return np.cos(2.0 * np.pi * ph / period).astype(np.float32)
