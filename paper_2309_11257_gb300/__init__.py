"""GB300-native (sm_103a) MS-GWaM-3D gravity-wave ray-volume tracer.

``gwam``  -- ctypes binding of the C-ABI library ``libgwam.so`` (CUDA kernels);
             importing it loads the library and fails loudly if it is missing.
``synth`` -- seeded synthetic inputs (grids, backgrounds, ray populations).

Nothing is loaded at package import, so the input generator stays usable on
machines without the compiled library.
"""
__all__ = ["gwam", "synth"]
