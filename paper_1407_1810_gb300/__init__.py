"""GB300-native (sm_103a) particle hot path of the PICsar method (arXiv 1407.1810).

The compute path is the CUDA shared library built from ``csrc/``; ``picsar``
is its thin ctypes binding with the same names as the C-ABI.
"""
