"""GB300-native voxel-driven cone-beam (Feldkamp) backprojection.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``); this package is a thin ctypes binding over it plus the
PyTorch glue (device memory, streams, autograd) and the seeded input
generators in ``synth``.
"""
