"""GB300-native Super Smoother periodograms (arXiv 2111.07396).

The compute path is the C-ABI library ``libssp.so`` (hand-written sm_103a CUDA,
sources in ``csrc/``); ``ssp`` is its thin ctypes binding.  Importing the
package does not load the library; ``ssp.lib()`` does, and fails loudly if it
has not been built.
"""
__all__ = ["ssp", "synth"]
