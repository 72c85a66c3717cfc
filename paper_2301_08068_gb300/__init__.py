"""GB300-native raycast-RMP evaluation (arXiv 2301.08068): Halton rays marched through a
voxel map by an exact fixed-point DDA, per-ray obstacle RMPs, cross-ray reduction and an
FP64 3x3 pseudo-inverse resolve, all in hand-written sm_103a CUDA behind a C ABI.

Importing the package loads nothing native; ``paper_2301_08068_gb300.rmp`` loads the
CUDA library and fails loudly when it is missing.
"""
