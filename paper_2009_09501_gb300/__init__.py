"""GB300-native depth-image-based rendering (DIBR) pseudo-stereo synthesis.

The compute path is the C-ABI library ``libdibr.so`` (CUDA kernels for sm_103a, sources in
``csrc/``, declarations in ``include/dibr.h``).  ``dibr`` is its thin ctypes binding;
``scenes`` draws seeded synthetic inputs.  Submodules are imported on first use so that
the scene generator can be used without loading the native library.
"""
__all__ = ["dibr", "scenes"]
