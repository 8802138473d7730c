"""GB300 sliced bucket-elimination contraction (arXiv 2004.10892, Sections II-III).

The package keeps imports light: ``inputs`` (seeded circuit generator) imports
nothing else, and the native library is loaded only when ``tnq`` is used.
"""
