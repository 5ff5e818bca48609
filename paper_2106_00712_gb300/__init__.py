"""GB300-native DQMC sweep for network-initialized Monte Carlo (arXiv 2106.00712).

The compute path is the C-ABI library ``libnmc.so`` (``include/nmc.h``) built from
``csrc/``; ``nmc`` is its thin ctypes binding. Import ``paper_2106_00712_gb300.nmc``
explicitly: importing this package loads nothing.
"""
