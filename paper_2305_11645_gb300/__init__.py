"""GB300-native reduced QMC matrix-vector product (Dick, Ebert, Herrmann,
Kritzer, Longo: "The fast reduced QMC matrix-vector product").

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/qmc.h``).  Importing this package does not load it; the first call
into ``paper_2305_11645_gb300.api`` does, and fails loudly if it is missing.
"""
