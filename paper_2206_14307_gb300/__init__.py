"""GB300-native (sm_103a) projected-RBM variational Monte Carlo with a
Lanczos step, for the J1-J2 Heisenberg model on L x L periodic lattices.

The compute path is the CUDA library built from csrc/ (C ABI in
include/nnqs.h); ``nnqs`` is its Python binding.  ``synth`` holds the seeded
synthetic inputs.
"""
