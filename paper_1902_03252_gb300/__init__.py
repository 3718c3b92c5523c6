"""GB300-native (sm_103a) image-plane chi^2 evaluation for LENSTOOL-style
parametric strong-lens modelling (Rexroth et al. 2019).

The compute path is the C-ABI library built from ``csrc/`` (declared in
``include/lt.h``); ``lt`` is its thin ctypes binding and ``workloads`` holds
the seeded synthetic inputs.
"""
