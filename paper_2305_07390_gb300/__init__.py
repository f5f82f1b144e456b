"""GB300-native temporally blocked iterative stencils (EBISU-style, ICS '23).

The compute path is the C-ABI shared library built from ``csrc/`` (hand-written
CUDA for sm_103a); :mod:`.ebisu` is a thin ctypes binding with the same names.
:mod:`.synth` draws the seeded synthetic inputs.
"""
