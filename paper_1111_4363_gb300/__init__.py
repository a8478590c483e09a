"""GB300-native least-action TDSE propagator: subvolume relaxation sweep driven by a multigrid V-cycle.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI declared in
``include/leastaction.h``); ``binding`` marshals arguments to it.  Importing this
package does not load the library; ``binding.lib()`` does, and raises if it is missing.
"""
