"""GB300-native hot path of the Phylogenetic Topographer (arXiv 1811.11007).

The compute lives in ``libpt.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/pt.h``); :mod:`paper_1811_11007_gb300.pt` is the thin
ctypes binding.  :mod:`paper_1811_11007_gb300.synth` draws seeded synthetic
inputs and holds none of the method's arithmetic.  Importing this package does
not load the CUDA library; ``pt`` loads it on first use and raises if it is
missing.
"""
