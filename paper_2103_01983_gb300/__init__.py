"""GB300-native projection-tree reduced-order model (arXiv 2103.01983).

The compute path lives in the C-ABI library ``libptrom.so`` (CUDA for sm_103a,
sources in ``csrc/``); ``ptrom`` is its thin Python binding.  Importing this
package does not load the library: ``paper_2103_01983_gb300.ptrom`` does, and
fails loudly when it is missing.
"""
__all__ = ["workloads"]
