"""GB300-native GRNND (GPU-parallel Relative NN-Descent) graph construction.

The compute path is the CUDA library ``libgrnnd.so`` built from ``csrc/``; this
package only marshals arguments to its C ABI (``include/grnnd.h``).
"""
