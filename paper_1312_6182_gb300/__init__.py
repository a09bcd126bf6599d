"""GB300-native generalized power method for sparse PCA (GP-SPCA).

The compute path is the CUDA library ``libgpspca.so`` behind the C-ABI in
``include/gpspca.h``; ``binding`` marshals arguments to it.  Importing this
package does not load the library: ``binding.load()`` does, and raises if the
library has not been built.
"""

__all__ = ["binding", "synth"]
