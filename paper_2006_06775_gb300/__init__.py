"""GB300-native agent-mechanics hot path of the BioDynaMo simulation loop (arXiv 2006.06775).

The compute path lives in the CUDA shared library ``libbdm.so`` built from ``csrc/``; ``bdm`` is its
thin ctypes binding.  Importing this package does not load the library; ``bdm.load()`` does.
"""
__all__ = ["bdm", "synth"]
