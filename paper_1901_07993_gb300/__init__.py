"""GB300-native inverse factorization of block-sparse SPD overlap matrices.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through ``paper_1901_07993_gb300.ifac`` (a ctypes binding of the C ABI declared
in ``include/ifac.h``).  ``synth`` generates seeded synthetic inputs.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
