"""GB300-native (sm_103a) hot path of Deformable Radial Kernel splatting.

``drk``    -- ctypes binding of the C-ABI library ``libdrk`` (CUDA kernels).
``synth``  -- seeded synthetic scenes and cameras.

The CUDA library is loaded lazily on first use; a missing library raises.
"""
__all__ = ["drk", "synth"]
