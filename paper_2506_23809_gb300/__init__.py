"""GB300-native local-energy evaluation for NQS quantum chemistry (arxiv 2506.23809).

The compute path is ``libqc_eloc.so`` (hand-written sm_103a CUDA behind a C ABI, see
``include/qc_eloc.h``); ``binding`` is a thin ctypes layer with the same names.  Importing
this package does not load the CUDA library; ``binding`` loads it on first use and raises
if it is missing.  ``inputs`` holds the seeded synthetic input generators.
"""
__all__ = ["binding", "inputs"]
