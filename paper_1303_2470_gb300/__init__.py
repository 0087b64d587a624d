"""GB300-native sorption-modified moment propagation (arXiv:1303.2470).

The compute lives in the CUDA library ``libmp.so`` (sources under ``csrc/``, C-ABI in
``include/mp.h``); ``paper_1303_2470_gb300.mp`` is the thin ctypes binding with the same
entry-point names. ``media`` makes seeded synthetic inputs, ``validation`` runs the paper's
validation experiments and ``surrogate`` drives the learned LB warm start. Importing this
package does not load the CUDA library; importing ``paper_1303_2470_gb300.mp`` does, and
fails loudly when the library has not been built.
"""
__all__ = ["media", "mp", "validation", "surrogate"]
