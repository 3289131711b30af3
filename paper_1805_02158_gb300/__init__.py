"""GB300-native RED + vector extrapolation.

The compute path is the CUDA library `libred.so` (sources in csrc/, C-ABI declared in
include/red.h); `red` is its thin ctypes binding and `synth` the seeded input generator.
"""
__all__ = ["red", "synth", "build"]
