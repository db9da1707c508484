"""GB300-native online tensor-subspace tracker for undersampled dynamic MRI.

The compute path lives in the CUDA library built from csrc/ (see build.py) and is
reached through the C-ABI binding in tts.py; inputs.py synthesises seeded inputs.
"""
