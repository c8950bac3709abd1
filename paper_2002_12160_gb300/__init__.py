"""GB300-native hot path of sim-in-the-loop in-hand object pose tracking.

The compute path is hand-written sm_103a CUDA behind a C ABI
(``libinhand.so``, declared in ``include/inhand.h``); ``inhand`` is its thin
ctypes binding and ``workloads`` builds the seeded synthetic inputs.
Importing the package does not load the CUDA library; the first use of the
binding does, and fails loudly if it is missing.
"""
