"""B300-native platelet fluid-structure step (Wu, Xu, Kim, Alber).

The compute path is the C-ABI CUDA library ``libplatelet_fsi.so`` built from
``csrc/``; :mod:`paper_1312_2234_b300.fsi` is its thin ctypes binding and
:mod:`paper_1312_2234_b300.workload` builds seeded synthetic inputs.  The
library is loaded on first use and a missing build raises immediately.
"""
