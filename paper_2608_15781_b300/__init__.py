"""B300-native colour-gradient lattice Boltzmann step for gas-generating reactive flow.

The compute path is the C-ABI library ``libcglbm.so`` (hand-written CUDA for
sm_103a, built in-tree by ``paper_2608_15781_b300.build``); ``lbm`` is its thin
ctypes binding.  ``synth`` generates seeded synthetic inputs.  Importing the
package does not load the library; the first call into ``lbm`` does, and it
raises if the library is missing -- there is no CPU fallback.
"""
__all__ = ["lbm", "synth", "configs"]
