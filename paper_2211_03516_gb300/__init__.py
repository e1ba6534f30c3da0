"""vamrt: GB300-native 3D ray-traced projection and dose operators for tomographic VAM.

The compute path is the CUDA library libvamrt.so (csrc/, C ABI in include/vamrt.h);
`vamrt` is its ctypes binding, `inputs` the seeded synthetic workloads.
"""
__all__ = ["vamrt", "inputs", "build"]
