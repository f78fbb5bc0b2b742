"""GB300-native seismic saliency by local 3D-DFT spectral projections and directional
centre-surround comparison (Shafiq, Long, Alshawi, AlRegib, ICIP 2017, Sec. 2).

The computing happens in libsal.so (hand-written CUDA for sm_103a, C ABI in
include/sal.h); ``api`` exposes its entry points with the same names.  Importing the
package does not load the library; the first call does, and fails loudly if it is
missing.
"""
__all__ = ["api", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
