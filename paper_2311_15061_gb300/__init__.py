"""GB300-native Beta-Process Factor Analysis (BPFA) inpainting.

The hot path -- the Gibbs sweep over all overlapping N-D patches of a
subsampled frame -- runs as hand-written CUDA for sm_103a inside
``libsensai.so`` behind a small C ABI (``include/sensai.h``).  ``sensai`` is
the thin ctypes binding; ``synth`` draws seeded synthetic inputs.

Importing the package does not load the CUDA library; importing
``paper_2311_15061_gb300.sensai`` does, and raises if it has not been built.
"""
__all__ = ["sensai", "synth"]
