"""GB300-native multi-resolution approximation (M-RA) of Gaussian processes.

The computation lives in the CUDA library ``libmra_gb300.so`` (sources in
``csrc/``, C ABI in ``include/mra.h``); :mod:`.mra` is its Python binding and
:mod:`.synth` generates seeded synthetic inputs.
"""
__all__ = ["mra", "synth", "build"]
