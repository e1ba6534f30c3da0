"""FP64 CPU oracle for the 3D ray-traced VAM projection/dose operators (test infrastructure).

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
