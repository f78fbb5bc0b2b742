"""ctypes binding of the plain C FP64 oracle (``sal_oracle.c``).

TEST INFRASTRUCTURE ONLY: shares no code with the CUDA path and imports nothing from it.
``build()`` compiles ``liboracle.so`` next to this file with gcc (OpenMP for the per-voxel
loops).  All arrays cross as numpy float32 (volumes) or float64 (everything the oracle
computes).

Parity status: every function below is pinned by the ``-m "not gpu"`` tests against
closed forms, library special cases (numpy FFT, numpy.pad) or brute force; none is
"parity unpinned" against the method's own definition.  Against the paper's own printed
output parity is unpinned: the paper prints no values (its result figure is an image of
data not available here).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sal_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

REFLECT, PERIODIC = 0, 1
STENCIL_26, STENCIL_LINE, STENCIL_DIAG_TX = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc if it is missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        f64p = ctypes.POINTER(ctypes.c_double)
        f32p = ctypes.POINTER(ctypes.c_float)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L_, I_, D_ = ctypes.c_long, ctypes.c_int, ctypes.c_double
        lib.orc_ext_index.argtypes = [L_, L_, I_]
        lib.orc_ext_index.restype = L_
        for name in ("oracle_local_spectrum_brute", "oracle_local_spectrum_separable"):
            fn = getattr(lib, name)
            fn.argtypes = [f32p, L_, L_, L_, I_, I_, L_, L_, L_, f64p]
            fn.restype = I_
        lib.oracle_weights.argtypes = [I_, f64p]
        lib.oracle_weights.restype = None
        lib.oracle_project.argtypes = [f64p, L_, I_, f64p]
        lib.oracle_project.restype = None
        lib.oracle_energy.argtypes = [f32p, L_, L_, L_, I_, I_, I_, I_, f64p]
        lib.oracle_energy.restype = I_
        lib.oracle_energy_at.argtypes = [f32p, L_, L_, L_, I_, I_, i64p, L_, I_, f64p]
        lib.oracle_energy_at.restype = I_
        lib.oracle_maps_at.argtypes = [f32p, L_, L_, L_, I_, I_, I_, D_, i64p, L_, I_, f64p, f64p]
        lib.oracle_maps_at.restype = I_
        lib.oracle_dcs.argtypes = [f64p, L_, L_, L_, I_, I_, I_, D_, I_, f64p]
        lib.oracle_dcs.restype = I_
        ip_ = ctypes.POINTER(ctypes.c_int)
        lib.oracle_dcs_user.argtypes = [f64p, L_, L_, L_, I_, ip_, ip_, f64p, I_, I_, f64p]
        lib.oracle_dcs_user.restype = I_
        lib.oracle_stats.argtypes = [f64p, L_, f64p]
        lib.oracle_stats.restype = None
        lib.oracle_combine.argtypes = [f64p, f64p, L_, D_, D_, D_, D_, f64p]
        lib.oracle_combine.restype = None
        lib.oracle_saliency.argtypes = [f32p, L_, L_, L_, I_, I_, I_, D_, D_, D_, D_, D_, I_,
                                        f64p, f64p, f64p, f64p]
        lib.oracle_saliency.restype = I_
        lib.oracle_conv3d.argtypes = [f64p, L_, L_, L_, I_, I_, f64p, f64p, I_, f64p]
        lib.oracle_conv3d.restype = None
        lib.oracle_gelu.argtypes = [D_]
        lib.oracle_gelu.restype = D_
        lib.oracle_gelu_grad.argtypes = [D_]
        lib.oracle_gelu_grad.restype = D_
        lib.oracle_conv3d_grad.argtypes = [f64p, L_, L_, L_, I_, I_, f64p, I_, f64p, f64p, f64p, f64p]
        lib.oracle_conv3d_grad.restype = None
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_surrogate_forward.argtypes = [f64p, L_, L_, L_, I_, ip, f64p, I_, f64p, f64p]
        lib.oracle_surrogate_forward.restype = I_
        lib.oracle_surrogate_loss_grad.argtypes = [f64p, L_, L_, L_, I_, ip, f64p, I_, f64p, f64p, f64p]
        lib.oracle_surrogate_loss_grad.restype = D_
        _lib = lib
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def ext_index(i: int, n: int, bnd: int = REFLECT) -> int:
    """Boundary extension of one coordinate onto 0..n-1."""
    return int(_load().orc_ext_index(int(i), int(n), int(bnd)))


def local_spectrum(V, t, x, y, L, bnd=REFLECT, brute=False) -> np.ndarray:
    """|F| of the local cube at voxel (t, x, y): [L][L][L], centred signed frequency order."""
    V, vp = _f32(V)
    out, op = _f64(np.zeros((L, L, L)))
    fn = _load().oracle_local_spectrum_brute if brute else _load().oracle_local_spectrum_separable
    rc = fn(vp, *V.shape, L, bnd, t, x, y, op)
    if rc:
        raise ValueError(f"oracle local spectrum failed ({rc})")
    return out


def weights(L) -> np.ndarray:
    """Projection weights w[3][L][L][L] (t, x, y), centred order, 0 at DC."""
    out, op = _f64(np.zeros((3, L, L, L)))
    _load().oracle_weights(L, op)
    return out


def project(mag, L) -> np.ndarray:
    """Spectral energies [3][n] from magnitude spectra [n][L][L][L]."""
    mag, mp = _f64(np.asarray(mag).reshape(-1, L * L * L))
    n = mag.shape[0]
    out, op = _f64(np.zeros((3, n)))
    _load().oracle_project(mp, n, L, op)
    return out


def energy(V, L, bnd=REFLECT, brute=False, threads=None) -> np.ndarray:
    """E_t, E_x, E_y of every voxel: [3][T][X][Y] float64."""
    V, vp = _f32(V)
    out, op = _f64(np.zeros((3,) + V.shape))
    rc = _load().oracle_energy(vp, *V.shape, L, bnd, int(brute), threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_energy failed ({rc})")
    return out


def energy_at(V, coords, L, bnd=REFLECT, threads=None) -> np.ndarray:
    """E_m at selected voxels ``coords`` [n][3] (int): [3][n] float64."""
    V, vp = _f32(V)
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, 3))
    n = c.shape[0]
    out, op = _f64(np.zeros((3, n)))
    rc = _load().oracle_energy_at(vp, *V.shape, L, bnd, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  n, threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_energy_at failed ({rc})")
    return out


def maps_at(V, coords, L, bnd=REFLECT, stencil=STENCIL_26, sigma=1.0, threads=None):
    """(E, S_m) at selected voxels ``coords`` [n][3]: two [3][n] float64 arrays."""
    V, vp = _f32(V)
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.int64).reshape(-1, 3))
    n = c.shape[0]
    E, ep = _f64(np.zeros((3, n)))
    S, sp = _f64(np.zeros((3, n)))
    rc = _load().oracle_maps_at(vp, *V.shape, L, bnd, stencil, float(sigma),
                                c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n, threads or default_threads(), ep, sp)
    if rc:
        raise ValueError(f"oracle_maps_at failed ({rc})")
    return E, S


def dcs(E, bnd=REFLECT, stencil=STENCIL_26, L=7, sigma=1.0, threads=None) -> np.ndarray:
    """S_t, S_x, S_y from E [3][T][X][Y] (Eq. 5)."""
    E, ep = _f64(E)
    shape = E.shape[1:]
    out, op = _f64(np.zeros(E.shape))
    rc = _load().oracle_dcs(ep, *shape, bnd, stencil, L, float(sigma), threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_dcs failed ({rc})")
    return out


def dcs_user(E, offsets, weights, bnd=REFLECT, threads=None) -> np.ndarray:
    """Eq. 5 with caller-given neighbourhoods: offsets[m] is a list of (dt, dx, dy), weights[m]
    the matching weights; S_m = mean over k of |E_m - w_k E_m(v + o_k)|."""
    E, ep = _f64(E)
    shape = E.shape[1:]
    qmax = max(len(o) for o in offsets)
    off = np.zeros((3, qmax, 3), dtype=np.intc)
    w = np.zeros((3, qmax))
    Q = np.zeros(3, dtype=np.intc)
    for m in range(3):
        Q[m] = len(offsets[m])
        off[m, :Q[m]] = np.asarray(offsets[m], dtype=np.intc).reshape(-1, 3)
        w[m, :Q[m]] = weights[m]
    w, wp = _f64(w)
    ip = ctypes.POINTER(ctypes.c_int)
    out, op = _f64(np.zeros(E.shape))
    rc = _load().oracle_dcs_user(ep, *shape, bnd, Q.ctypes.data_as(ip), off.ctypes.data_as(ip), wp, qmax,
                                 threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_dcs_user failed ({rc})")
    return out


def stats(Sm) -> np.ndarray:
    """[3][3] = (min, max, sum) of each map."""
    Sm, sp = _f64(Sm)
    out, op = _f64(np.zeros(9))
    _load().oracle_stats(sp, Sm[0].size, op)
    return out.reshape(3, 3)


def combine(Sm, st, a=1 / 3, b=1 / 3, c=1 / 3, eps=1e-6) -> np.ndarray:
    """Eq. 6 on min-max normalised maps."""
    Sm, sp = _f64(Sm)
    st, tp = _f64(np.asarray(st).reshape(9))
    out, op = _f64(np.zeros(Sm.shape[1:]))
    _load().oracle_combine(sp, tp, Sm[0].size, a, b, c, eps, op)
    return out


def saliency(V, L=7, bnd=REFLECT, stencil=STENCIL_26, sigma=1.0, a=1 / 3, b=1 / 3, c=1 / 3,
             eps=1e-6, threads=None, full=False):
    """The whole method.  Returns S, or (S, E, Sm, stats) when ``full``."""
    V, vp = _f32(V)
    S, sp = _f64(np.zeros(V.shape))
    E, ep = _f64(np.zeros((3,) + V.shape))
    Sm, mp = _f64(np.zeros((3,) + V.shape))
    st, tp = _f64(np.zeros(9))
    rc = _load().oracle_saliency(vp, *V.shape, L, bnd, stencil, float(sigma), a, b, c, eps,
                                 threads or default_threads(), sp, ep, mp, tp)
    if rc:
        raise ValueError(f"oracle_saliency failed ({rc})")
    return (S, E, Sm, st.reshape(3, 3)) if full else S


# ---- learned surrogate (plain FP64 reference of its layers) ----------------------------

def conv3d(x, w, b=None, bnd=REFLECT):
    """3x3x3 cross-correlation with bias: x [Cin][T][X][Y], w [Cout][Cin][3][3][3] -> [Cout][T][X][Y]."""
    x, xp = _f64(x)
    w, wp = _f64(w)
    cout, cin = w.shape[0], w.shape[1]
    if b is not None:
        b, bp = _f64(b)
    else:
        bp = None
    out, op = _f64(np.zeros((cout,) + x.shape[1:]))
    _load().oracle_conv3d(xp, *x.shape[1:], cin, cout, wp, bp, bnd, op)
    return out


def gelu(v):
    f = np.vectorize(_load().oracle_gelu)
    return f(np.asarray(v, dtype=np.float64))


def gelu_grad(v):
    f = np.vectorize(_load().oracle_gelu_grad)
    return f(np.asarray(v, dtype=np.float64))


def conv3d_grad(x, w, gout, bnd=REFLECT, need_input_grad=True):
    """(dW, db, dX) of conv3d given dL/dout."""
    x, xp = _f64(x)
    w, wp = _f64(w)
    gout, gp = _f64(gout)
    gw, gwp = _f64(np.zeros_like(w))
    gb, gbp = _f64(np.zeros(w.shape[0]))
    gin, gip = _f64(np.zeros_like(x))
    _load().oracle_conv3d_grad(xp, *x.shape[1:], w.shape[1], w.shape[0], wp, bnd, gp, gwp, gbp,
                               gip if need_input_grad else None)
    return gw, gb, (gin if need_input_grad else None)


def _widths(widths):
    arr = (ctypes.c_int * len(widths))(*[int(v) for v in widths])
    return arr


def surrogate_forward(x, widths, params, bnd=REFLECT):
    """Output [widths[-1]][T][X][Y] of the layer stack for input x [widths[0]][T][X][Y]."""
    x, xp = _f64(x)
    params, pp = _f64(params)
    out, op = _f64(np.zeros((widths[-1],) + x.shape[1:]))
    _load().oracle_surrogate_forward(xp, *x.shape[1:], len(widths) - 1, _widths(widths), pp, bnd, op, None)
    return out


def surrogate_loss_grad(x, widths, params, target, mask=None, bnd=REFLECT):
    """(loss, grads) of 0.5 * sum mask * (out - target)^2; grads in the layout of params."""
    x, xp = _f64(x)
    params, pp = _f64(params)
    target, tp = _f64(target)
    mp = None
    if mask is not None:
        mask, mp = _f64(mask)
    grads, gp = _f64(np.zeros_like(params))
    loss = _load().oracle_surrogate_loss_grad(xp, *x.shape[1:], len(widths) - 1, _widths(widths), pp, bnd, tp,
                                              mp, gp)
    return loss, grads


# ---- coarse-stride cubes (cube centres on a lattice of step s, E interpolated back) ------

def _lattice_protos():
    lib = _load()
    if not getattr(lib, "_lattice_ready", False):
        f64p = ctypes.POINTER(ctypes.c_double)
        f32p = ctypes.POINTER(ctypes.c_float)
        L_, I_, D_ = ctypes.c_long, ctypes.c_int, ctypes.c_double
        lib.oracle_lattice_size.argtypes = [L_, I_]
        lib.oracle_lattice_size.restype = L_
        lib.oracle_energy_lattice.argtypes = [f32p, L_, L_, L_, I_, I_, I_, I_, f64p]
        lib.oracle_energy_lattice.restype = I_
        lib.oracle_interp_lattice.argtypes = [f64p, I_, L_, L_, L_, I_, f64p]
        lib.oracle_interp_lattice.restype = None
        lib.oracle_energy_strided.argtypes = [f32p, L_, L_, L_, I_, I_, I_, I_, f64p]
        lib.oracle_energy_strided.restype = I_
        lib.oracle_saliency_strided.argtypes = [f32p, L_, L_, L_, I_, I_, I_, I_, D_, D_, D_, D_, D_, I_,
                                                f64p, f64p, f64p, f64p]
        lib.oracle_saliency_strided.restype = I_
        lib._lattice_ready = True
    return lib


def lattice_size(n: int, s: int) -> int:
    """Number of cube centres along an axis of n samples at stride s."""
    return int(_lattice_protos().oracle_lattice_size(int(n), int(s)))


def lattice_shape(shape, s):
    return tuple(lattice_size(n, s) for n in shape)


def energy_lattice(V, L, s, bnd=REFLECT, threads=None) -> np.ndarray:
    """E_m of the cubes centred on the lattice points: [3][Tc][Xc][Yc]."""
    V, vp = _f32(V)
    out, op = _f64(np.zeros((3,) + lattice_shape(V.shape, s)))
    rc = _lattice_protos().oracle_energy_lattice(vp, *V.shape, L, bnd, int(s), threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_energy_lattice failed ({rc})")
    return out


def interp_lattice(Ec, shape, s) -> np.ndarray:
    """Trilinear interpolation of lattice values [C][Tc][Xc][Yc] to every voxel of `shape`."""
    Ec, ep = _f64(Ec)
    out, op = _f64(np.zeros((Ec.shape[0],) + tuple(shape)))
    _lattice_protos().oracle_interp_lattice(ep, Ec.shape[0], *shape, int(s), op)
    return out


def energy_strided(V, L, s, bnd=REFLECT, threads=None) -> np.ndarray:
    V, vp = _f32(V)
    out, op = _f64(np.zeros((3,) + V.shape))
    rc = _lattice_protos().oracle_energy_strided(vp, *V.shape, L, bnd, int(s), threads or default_threads(), op)
    if rc:
        raise ValueError(f"oracle_energy_strided failed ({rc})")
    return out


def saliency_strided(V, L=7, s=2, bnd=REFLECT, stencil=STENCIL_26, sigma=1.0, a=1 / 3, b=1 / 3, c=1 / 3,
                     eps=1e-6, threads=None, full=False):
    V, vp = _f32(V)
    S, sp = _f64(np.zeros(V.shape))
    E, ep = _f64(np.zeros((3,) + V.shape))
    Sm, mp = _f64(np.zeros((3,) + V.shape))
    st, tp = _f64(np.zeros(9))
    rc = _lattice_protos().oracle_saliency_strided(vp, *V.shape, L, bnd, stencil, int(s), float(sigma), a, b, c, eps,
                                                   threads or default_threads(), sp, ep, mp, tp)
    if rc:
        raise ValueError(f"oracle_saliency_strided failed ({rc})")
    return (S, E, Sm, st.reshape(3, 3)) if full else S
