"""FAST-BCC biconnected components on one GB300 (sm_103a).

The compute path is the C-ABI library ``libfbcc`` (hand-written CUDA kernels);
:mod:`.fbcc` is its thin ctypes binding and :mod:`.graphgen` makes seeded inputs.
"""
