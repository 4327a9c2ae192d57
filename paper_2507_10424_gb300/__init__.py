"""GB300-native flooding Min-Sum LDPC decoding (arXiv 2507.10424), CUDA path for sm_103a.

The decoder lives in the C-ABI library ``libldpc.so`` built from ``csrc/``; the Python
binding in :mod:`paper_2507_10424_gb300.ldpc` only marshals arguments to it. Importing
this package does not load the library; :mod:`paper_2507_10424_gb300.ldpc` does, and
raises if it is missing.
"""
