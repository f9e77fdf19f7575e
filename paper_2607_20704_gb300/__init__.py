"""GB300-native AMR level step of compressible Euler (cell-by-cell octree).

Importing the package loads nothing native; ``paper_2607_20704_gb300.amr``
loads the CUDA library and fails loudly when it is missing.
"""
