"""Python face of the C ABI: one function per entry point of include/sal.h, same names.

Marshalling only: torch CUDA tensors provide device memory and the current stream; the
library's kernels do all the computing.  Outputs and workspaces that the caller does not
pass are allocated with torch (the library itself never allocates).
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from ._native import SalDims, SalParams, SalTileChoice, SalUserStencil, SalVolume, check

_PREC = {"fp32": N.SAL_PREC_FP32, "tf32": N.SAL_PREC_TF32, "bf16": N.SAL_PREC_BF16}
_BND = {"reflect": N.SAL_BND_REFLECT, "periodic": N.SAL_BND_PERIODIC}
_STENCIL = {"26": N.SAL_STENCIL_26, "line": N.SAL_STENCIL_LINE, "diag_tx": N.SAL_STENCIL_DIAG_TX}


def sal_params_default() -> SalParams:
    p = SalParams()
    check(N.lib().sal_params_default(ctypes.byref(p)))
    return p


def params(L: int = 7, precision="fp32", boundary="reflect", stencil="26", sigma: float = 1.0,
           a: float = 1 / 3, b: float = 1 / 3, c: float = 1 / 3, eps: float = 1e-6, stride: int = 1) -> SalParams:
    """A sal_params struct from readable values (names or the enum integers)."""
    p = sal_params_default()
    p.stride = int(stride)
    p.L = int(L)
    p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    p.boundary = _BND[boundary] if isinstance(boundary, str) else int(boundary)
    p.stencil = _STENCIL[str(stencil)] if isinstance(stencil, str) else int(stencil)
    p.sigma, p.a, p.b, p.c, p.eps = float(sigma), float(a), float(b), float(c), float(eps)
    return p


def dims_of(V: torch.Tensor) -> SalDims:
    if V.dim() != 3:
        raise ValueError("volume must be 3-D [T, X, Y]")
    return SalDims(*[int(s) for s in V.shape])


def _dev(t: torch.Tensor, dtype=torch.float32, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def sal_workspace_size(dims: SalDims, p: SalParams) -> int:
    n = ctypes.c_size_t()
    check(N.lib().sal_workspace_size(dims, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_dcs_workspace_size(dims: SalDims, p: SalParams) -> int:
    n = ctypes.c_size_t()
    check(N.lib().sal_dcs_workspace_size(dims, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_local_spectra(V: torch.Tensor, p: SalParams, roi_lo, roi_ext, mag: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """|F| of every voxel of a region: [ext_t, ext_x, ext_y, L, L, L], centred slots."""
    L = p.L
    if mag is None:
        mag = torch.empty(tuple(int(e) for e in roi_ext) + (L, L, L), device=V.device, dtype=torch.float32)
    lo = (ctypes.c_int64 * 3)(*[int(v) for v in roi_lo])
    ex = (ctypes.c_int64 * 3)(*[int(v) for v in roi_ext])
    check(N.lib().sal_local_spectra(_dev(V, name="V"), dims_of(V), ctypes.byref(p), lo, ex,
                                    _dev(mag, name="mag"), _stream(stream)))
    return mag


def sal_project(mag: torch.Tensor, L: int, E: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Spectral energies [3, n] from spectra [..., L, L, L]."""
    n = mag.numel() // (L ** 3)
    if E is None:
        E = torch.empty((3, n), device=mag.device, dtype=torch.float32)
    check(N.lib().sal_project(_dev(mag, name="mag"), n, int(L), _dev(E, name="E"), _stream(stream)))
    return E


def sal_spectral_energy(V: torch.Tensor, p: SalParams, E: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """E_t, E_x, E_y of every voxel: [3, T, X, Y]."""
    if E is None:
        E = torch.empty((3,) + tuple(V.shape), device=V.device, dtype=torch.float32)
    check(N.lib().sal_spectral_energy(_dev(V, name="V"), dims_of(V), ctypes.byref(p), _dev(E, name="E"),
                                      _stream(stream)))
    return E


def sal_lattice_dims(dims: SalDims, p: SalParams) -> SalDims:
    """(Tc, Xc, Yc): the cube centres of stride p.stride along each axis."""
    out = SalDims()
    check(N.lib().sal_lattice_dims(dims, ctypes.byref(p), ctypes.byref(out)))
    return out


def sal_lattice_energy(V: torch.Tensor, p: SalParams, Ec: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """E_m of the cubes centred on the lattice points: [3, Tc, Xc, Yc]."""
    lat = sal_lattice_dims(dims_of(V), p)
    if Ec is None:
        Ec = torch.empty((3, lat.T, lat.X, lat.Y), device=V.device, dtype=torch.float32)
    check(N.lib().sal_lattice_energy(_dev(V, name="V"), dims_of(V), ctypes.byref(p), _dev(Ec, name="Ec"),
                                     _stream(stream)))
    return Ec


def sal_interpolate_lattice(Ec: torch.Tensor, shape, p: SalParams, E: torch.Tensor | None = None,
                            stream=None) -> torch.Tensor:
    """Trilinear interpolation of lattice energies back to every voxel of `shape`: [3, T, X, Y]."""
    dims = SalDims(*[int(v) for v in shape])
    if E is None:
        E = torch.empty((3,) + tuple(int(v) for v in shape), device=Ec.device, dtype=torch.float32)
    check(N.lib().sal_interpolate_lattice(_dev(Ec, name="Ec"), dims, ctypes.byref(p), _dev(E, name="E"),
                                          _stream(stream)))
    return E


def sal_directional_compare(E: torch.Tensor, p: SalParams, Sm: torch.Tensor | None = None,
                            stats: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """S_t, S_x, S_y [3, T, X, Y] and their FP64 (min, max, sum) [9]."""
    dims = SalDims(*[int(s) for s in E.shape[1:]])
    if Sm is None:
        Sm = torch.empty_like(E)
    if stats is None:
        stats = torch.empty(N.SAL_STATS_LEN, device=E.device, dtype=torch.float64)
    need = sal_dcs_workspace_size(dims, p)
    if ws is None:
        ws = torch.empty(need, device=E.device, dtype=torch.uint8)
    check(N.lib().sal_directional_compare(_dev(E, name="E"), dims, ctypes.byref(p), _dev(Sm, name="Sm"),
                                          _dev(stats, torch.float64, "stats"), _dev(ws, torch.uint8, "ws"),
                                          ws.numel(), _stream(stream)))
    return Sm, stats


def sal_directional_compare_static(E: torch.Tensor, p: SalParams, Sm: torch.Tensor | None = None,
                                   stats: torch.Tensor | None = None, stream=None):
    """sal_directional_compare without a workspace: the library's fixed scratch serves the
    reduction, for callers that may not allocate device memory (outputs must be passed in
    by such callers; the defaults here allocate them with torch only for convenience)."""
    dims = SalDims(*[int(s) for s in E.shape[1:]])
    if Sm is None:
        Sm = torch.empty_like(E)
    if stats is None:
        stats = torch.empty(N.SAL_STATS_LEN, device=E.device, dtype=torch.float64)
    check(N.lib().sal_directional_compare_static(_dev(E, name="E"), dims, ctypes.byref(p), _dev(Sm, name="Sm"),
                                                 _dev(stats, torch.float64, "stats"), _stream(stream)))
    return Sm, stats


def user_stencil(offsets, weights) -> SalUserStencil:
    """A sal_user_stencil from per-map lists: offsets[m] = [(dt, dx, dy), ...], weights[m] = [w, ...]."""
    st = SalUserStencil()
    for m in range(3):
        if len(offsets[m]) != len(weights[m]):
            raise ValueError(f"map {m}: {len(offsets[m])} offsets but {len(weights[m])} weights")
        if len(offsets[m]) > N.SAL_STENCIL_MAX_OFFSETS:
            raise ValueError(f"map {m}: at most {N.SAL_STENCIL_MAX_OFFSETS} offsets")
        st.count[m] = len(offsets[m])
        for k, (o, w) in enumerate(zip(offsets[m], weights[m])):
            st.offset[m][k][0], st.offset[m][k][1], st.offset[m][k][2] = (int(v) for v in o)
            st.weight[m][k] = float(w)
    return st


def sal_directional_compare_user(E: torch.Tensor, p: SalParams, st: SalUserStencil, Sm: torch.Tensor | None = None,
                                 stats: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """Eq. 5 with the caller's neighbourhood per map (see user_stencil): (S_m, stats)."""
    dims = SalDims(*[int(s) for s in E.shape[1:]])
    if Sm is None:
        Sm = torch.empty_like(E)
    if stats is None:
        stats = torch.empty(N.SAL_STATS_LEN, device=E.device, dtype=torch.float64)
    if ws is None:
        ws = torch.empty(sal_dcs_workspace_size(dims, p), device=E.device, dtype=torch.uint8)
    check(N.lib().sal_directional_compare_user(_dev(E, name="E"), dims, ctypes.byref(p), ctypes.byref(st),
                                               _dev(Sm, name="Sm"), _dev(stats, torch.float64, "stats"),
                                               _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)))
    return Sm, stats


def sal_slab_halo(p: SalParams) -> int:
    """Planes of V a slab needs beyond its own on each side."""
    n = ctypes.c_int64()
    check(N.lib().sal_slab_halo(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_slab_workspace_size(ext_planes: int, X: int, Y: int, p: SalParams) -> int:
    n = ctypes.c_size_t()
    check(N.lib().sal_slab_workspace_size(int(ext_planes), int(X), int(Y), ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_slab_maps(V_ext: torch.Tensor, dims: SalDims, ext_lo: int, ext_hi: int, own_lo: int, own_hi: int,
                  p: SalParams, Sm_own: torch.Tensor | None = None, stats_local: torch.Tensor | None = None,
                  ws: torch.Tensor | None = None, stream=None):
    """Steps 1-4 of one slab: (S_m of its own planes [3, own, X, Y], their local (min, max, sum) [9]).

    V_ext holds the planes [ext_lo, ext_hi) of V as its own 16-byte aligned buffer (a slice of a
    larger tensor along t is generally not aligned: clone it)."""
    X, Y = int(dims.X), int(dims.Y)
    if Sm_own is None:
        Sm_own = torch.empty((3, int(own_hi) - int(own_lo), X, Y), device=V_ext.device, dtype=torch.float32)
    if stats_local is None:
        stats_local = torch.empty(N.SAL_STATS_LEN, device=V_ext.device, dtype=torch.float64)
    if ws is None:
        ws = torch.empty(sal_slab_workspace_size(int(ext_hi) - int(ext_lo), X, Y, p), device=V_ext.device,
                         dtype=torch.uint8)
    check(N.lib().sal_slab_maps(_dev(V_ext, name="V_ext"), dims, int(ext_lo), int(ext_hi), int(own_lo), int(own_hi),
                                ctypes.byref(p), _dev(Sm_own, name="Sm_own"),
                                _dev(stats_local, torch.float64, "stats_local"), _dev(ws, torch.uint8, "ws"),
                                ws.numel(), _stream(stream)))
    return Sm_own, stats_local


def sal_stats_merge(stats: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Merges statistics records [n, 9] (device) into one [9]: min, max and FP64 sum per map."""
    if out is None:
        out = torch.empty(N.SAL_STATS_LEN, device=stats.device, dtype=torch.float64)
    n = stats.numel() // N.SAL_STATS_LEN
    check(N.lib().sal_stats_merge(_dev(stats, torch.float64, "stats"), n, _dev(out, torch.float64, "out"),
                                  _stream(stream)))
    return out


def sal_combine(Sm: torch.Tensor, stats: torch.Tensor, p: SalParams, S: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Eq. 6 on the min-max normalised maps: S [T, X, Y]."""
    dims = SalDims(*[int(s) for s in Sm.shape[1:]])
    if S is None:
        S = torch.empty(Sm.shape[1:], device=Sm.device, dtype=torch.float32)
    check(N.lib().sal_combine(_dev(Sm, name="Sm"), _dev(stats, torch.float64, "stats"), dims, ctypes.byref(p),
                              _dev(S, name="S"), _stream(stream)))
    return S


def sal_saliency(V: torch.Tensor, p: SalParams, S: torch.Tensor | None = None, stats: torch.Tensor | None = None,
                 ws: torch.Tensor | None = None, stream=None):
    """The whole method, V -> S.  Returns (S, stats or None)."""
    dims = dims_of(V)
    if S is None:
        S = torch.empty_like(V)
    need = sal_workspace_size(dims, p)
    if ws is None:
        ws = torch.empty(need, device=V.device, dtype=torch.uint8)
    sp = _dev(stats, torch.float64, "stats") if stats is not None else None
    check(N.lib().sal_saliency(_dev(V, name="V"), dims, ctypes.byref(p), _dev(S, name="S"), sp,
                               _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)))
    return S, stats


def _host(t: torch.Tensor, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be torch.float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def sal_host_workspace_size(dims: SalDims, p: SalParams) -> int:
    n = ctypes.c_size_t()
    check(N.lib().sal_host_workspace_size(dims, ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_saliency_host(V_host: torch.Tensor, p: SalParams, S_host: torch.Tensor | None = None,
                      stats: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None,
                      done_event=None, device=None) -> torch.Tensor:
    """The whole method on a volume in host memory (pin it for overlap): V_host -> S_host.

    The library copies V in, runs the kernels and copies S out; successive calls on the same
    workspace overlap their copies with each other's kernels.  With `done_event` (a
    torch.cuda.Event) S_host is ready when the event completes; otherwise when `stream` does.
    """
    dims = SalDims(*[int(v) for v in V_host.shape])
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if S_host is None:
        S_host = torch.empty(tuple(V_host.shape), dtype=torch.float32, pin_memory=V_host.is_pinned())
    if ws is None:
        ws = torch.empty(sal_host_workspace_size(dims, p), device=dev, dtype=torch.uint8)
    sp = _dev(stats, torch.float64, "stats") if stats is not None else None
    ev = None
    if done_event is not None:
        if not done_event.cuda_event:
            done_event.record(stream if stream is not None else torch.cuda.current_stream(dev))
        ev = done_event.cuda_event
    check(N.lib().sal_saliency_host(_host(V_host, "V_host"), dims, ctypes.byref(p), _host(S_host, "S_host"), sp,
                                    _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream), ev))
    return S_host


def sal_host_release(ws: torch.Tensor) -> None:
    """Releases the streams and events the library keeps for this workspace."""
    check(N.lib().sal_host_release(_dev(ws, torch.uint8, "ws")))


def _volumes(Vs, Ss):
    arr = (SalVolume * len(Vs))()
    for i, (V, S) in enumerate(zip(Vs, Ss)):
        arr[i] = SalVolume(_dev(V, name="V"), _dev(S, name="S"), *[int(v) for v in V.shape])
    return arr


def _shape_volumes(shapes):
    arr = (SalVolume * len(shapes))()
    for i, sh in enumerate(shapes):
        arr[i] = SalVolume(None, None, *[int(v) for v in sh])
    return arr


def sal_batch_workspace_size(shapes, p: SalParams) -> int:
    """Workspace bytes of a batch of volumes with these [T, X, Y] shapes."""
    n = ctypes.c_size_t()
    check(N.lib().sal_batch_workspace_size(_shape_volumes(shapes), len(shapes), ctypes.byref(p), ctypes.byref(n)))
    return n.value


def sal_saliency_batched(Vs, p: SalParams, Ss=None, stats: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None):
    """The whole method on a list of volumes, each stage one persistent launch.  Returns (Ss, stats)."""
    if Ss is None:
        Ss = [torch.empty_like(V) for V in Vs]
    if ws is None:
        ws = torch.empty(sal_batch_workspace_size([V.shape for V in Vs], p), device=Vs[0].device, dtype=torch.uint8)
    sp = _dev(stats, torch.float64, "stats") if stats is not None else None
    check(N.lib().sal_saliency_batched(_volumes(Vs, Ss), len(Vs), ctypes.byref(p), sp, _dev(ws, torch.uint8, "ws"),
                                       ws.numel(), _stream(stream)))
    return Ss, stats


class SalGraph:
    """A batch captured once into a CUDA graph by the library (sal_graph_create_batched);
    launch() replays it.  Holds references to every buffer the graph uses."""

    def __init__(self, Vs, p: SalParams, Ss=None, stats: torch.Tensor | None = None,
                 ws: torch.Tensor | None = None, stream=None):
        self.Vs = list(Vs)
        self.Ss = Ss if Ss is not None else [torch.empty_like(V) for V in self.Vs]
        self.stats = stats
        self.ws = ws if ws is not None else torch.empty(sal_batch_workspace_size([V.shape for V in self.Vs], p),
                                                        device=self.Vs[0].device, dtype=torch.uint8)
        self.p = p
        h = ctypes.c_void_p()
        sp = _dev(stats, torch.float64, "stats") if stats is not None else None
        check(N.lib().sal_graph_create_batched(_volumes(self.Vs, self.Ss), len(self.Vs), ctypes.byref(p), sp,
                                               _dev(self.ws, torch.uint8, "ws"), self.ws.numel(), _stream(stream),
                                               ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        check(N.lib().sal_graph_launch(self._h, _stream(stream)))
        return self.Ss

    def close(self):
        if self._h:
            check(N.lib().sal_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sal_graph_create_batched(Vs, p: SalParams, **kw) -> SalGraph:
    return SalGraph(Vs, p, **kw)


def _choice(c: SalTileChoice) -> dict:
    return {k: getattr(c, k) for k, _ in SalTileChoice._fields_}


def sal_autotune(V: torch.Tensor, p: SalParams, E: torch.Tensor | None = None, stream=None) -> dict:
    """Times the candidate tile shapes on V, caches and returns the fastest."""
    if E is None:
        E = torch.empty((3,) + tuple(V.shape), device=V.device, dtype=torch.float32)
    c = SalTileChoice()
    check(N.lib().sal_autotune(_dev(V, name="V"), dims_of(V), ctypes.byref(p), _dev(E, name="E"), _stream(stream),
                               ctypes.byref(c)))
    return _choice(c)


def sal_autotune_batched(Vs, p: SalParams, ws: torch.Tensor | None = None, stream=None) -> dict:
    Ss = [torch.empty_like(V) for V in Vs]
    if ws is None:
        ws = torch.empty(sal_batch_workspace_size([V.shape for V in Vs], p), device=Vs[0].device, dtype=torch.uint8)
    c = SalTileChoice()
    check(N.lib().sal_autotune_batched(_volumes(Vs, Ss), len(Vs), ctypes.byref(p), _dev(ws, torch.uint8, "ws"),
                                       ws.numel(), _stream(stream), ctypes.byref(c)))
    return _choice(c)


def sal_autotune_query(L: int, precision: int, n_vox: int) -> dict:
    c = SalTileChoice()
    check(N.lib().sal_autotune_query(int(L), int(precision), int(n_vox), ctypes.byref(c)))
    return _choice(c)


def sal_autotune_save(path: str) -> None:
    check(N.lib().sal_autotune_save(str(path).encode()))


def sal_autotune_load(path: str) -> None:
    check(N.lib().sal_autotune_load(str(path).encode()))


def sal_autotune_clear() -> None:
    check(N.lib().sal_autotune_clear())


def sal_device_status(stream=None) -> None:
    """Raises SalError (SAL_ERR_TIMEOUT) if a tensor-core kernel's bounded wait ran out."""
    check(N.lib().sal_device_status(_stream(stream)))


def sal_test_stall_tensor_cores(on: bool) -> None:
    check(N.lib().sal_test_stall_tensor_cores(1 if on else 0))


def sal_probe_fma_rate(out: torch.Tensor, iters: int, packed: bool = False, stream=None) -> float:
    """Launches the FP32 FMA-rate probe (one float per thread into ``out``); returns the FP32
    flops the launch performs (time it with events on ``stream``)."""
    n = out.numel()
    check(N.lib().sal_probe_fma_rate(_dev(out, name="out"), n, int(iters), 1 if packed else 0, _stream(stream)))
    return 2.0 * N.SAL_PROBE_CHAINS * iters * n
