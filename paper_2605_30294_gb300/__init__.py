"""GB300-native work forwarding (RaFI hot path) for sm_103a.

``rafi`` is the ctypes binding of the C-ABI library ``librafi_gb.so``;
``inputs`` makes the seeded synthetic workloads.  Importing the package does
not load the CUDA library; ``rafi.lib()`` does, and fails loudly when the
library is missing.
"""
